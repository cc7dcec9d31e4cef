"""Write the FP64 oracle's time-averaged Rayleigh-Benard statistics over an
ensemble of independent runs (reference for the GPU statistics test at a
flat 2%).  Calls only oracle/ and the seeded-input module.

Cell and start as in make_rb_statistics.py: a cube of N^3 nodes, hot bottom
wall (T = +1/2), cold top wall (T = -1/2), adiabatic no-slip sidewalls,
free-fall scaling with U = 0.1 (t_f = H/U steps), the linear conduction
profile plus a seeded uniform perturbation of amplitude 1e-3, at rest
(Sec. 4 set-up).  Member k uses the seed seed0 + k; each discards `transient`
free-fall times and then samples the diagnostics every `every` steps for
`average` free-fall times.  The members run as separate single-threaded
processes: in a chaotic cell, M independent windows of length L fix the
time averages as well as one window of length M L, and they run in parallel.

Ensemble statistics pool the members' samples: the mean over the members for
the quantities linear in the sampled sums (Nu_vol, Nu_wall, Nu_kin, Nu_th, E)
and the root mean square for the rms Reynolds numbers (Re_rms, Re_w), which
with equal sample counts is the Sec. 4 average over all samples.

Each member writes snapshots of its running sums to DIR/member_<k>.json every
100 samples; `--combine-only` pools the snapshots already written, at the
largest sample count every member has reached.

  python tests/golden/make_rb_ensemble.py N Ra Pr transient average every seed0 members DIR [--combine-only] > out.json
"""
import json
import os
import sys
import time

os.environ.setdefault("OMP_NUM_THREADS", "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import oracle  # noqa: E402
from paper_1903_08882_gb300 import inputs  # noqa: E402

U = 0.1
SNAP = 100  # samples between snapshots
ROW = 10    # samples between series rows
LINEAR = ("Nu_vol", "Nu_wall", "Nu_kin", "Nu_th", "E")
RMS = ("Re_rms", "Re_w")


def _stats(p, r):
    d = oracle.finalize(p, r)
    return dict(Nu_vol=float(d["Nu_vol"]), Nu_wall=float(0.5 * (d["Nu_face"][4] - d["Nu_face"][5])),
                Nu_kin=float(d["Nu_kin"]), Nu_th=float(d["Nu_th"]), Re_rms=float(d["Re_rms"]),
                Re_w=float(d["Re_w"]), E=float(d["E"]))


def member(job):
    N, Ra, Pr, transient, average, every, seed, path = job
    t0 = time.time()
    p = oracle.cell(N, Ra, Pr, oracle.rayleigh_benard_walls(), U=U)
    tf = N / U
    T = inputs.rb_initial_temperature(N, N, N, seed=seed)
    f, g = oracle.init_equilibrium(p, 1.0, np.zeros(3), T)
    n_tr = int(round(transient * tf / every)) * every
    n_av = int(round(average * tf / every)) * every
    f, g = oracle.run(p, f, g, n_tr)
    acc = np.zeros(oracle.NDIAG)
    snaps, series = [], []
    for k in range(n_av // every):
        r = oracle.raw_diagnostics(p, f, g)
        acc += r
        if k % ROW == 0:
            s = _stats(p, r)
            # rows: step, Nu_vol, Nu_wall, Re_rms, Nu_kin, Nu_th, Re_w
            series.append([k * every, s["Nu_vol"], s["Nu_wall"], s["Re_rms"], s["Nu_kin"], s["Nu_th"], s["Re_w"]])
        if (k + 1) % SNAP == 0:
            snaps.append([k + 1, acc.tolist()])
            tmp = path + ".tmp"
            with open(tmp, "w") as fh:
                json.dump(dict(seed=seed, transient_steps=n_tr, sample_every=every, snapshots=snaps,
                               series=series, seconds=time.time() - t0), fh)
            os.replace(tmp, path)
        f, g = oracle.run(p, f, g, every)
    return path


def combine(N, Ra, Pr, every, paths):
    p = oracle.cell(N, Ra, Pr, oracle.rayleigh_benard_walls(), U=U)
    runs = [json.load(open(q)) for q in paths]
    common = min(r["snapshots"][-1][0] for r in runs)
    per = []
    for r in runs:
        acc = dict((n, a) for n, a in r["snapshots"])[common]
        per.append(_stats(p, np.array(acc) / common))
    ens = {k: float(np.mean([m[k] for m in per])) for k in LINEAR}
    ens.update({k: float(np.sqrt(np.mean([m[k] ** 2 for m in per]))) for k in RMS})
    rows = common // ROW
    out = {
        "what": "FP64 oracle Rayleigh-Benard statistics, ensemble of independent runs (volume and time averages of Sec. 4)",
        "N": N, "Ra": Ra, "Pr": Pr, "U": U, "seeds": [r["seed"] for r in runs],
        "transient_steps": runs[0]["transient_steps"], "average_steps": common * every, "sample_every": every,
        "samples": common, "cpu_seconds": float(max(r["seconds"] for r in runs)),
        "members": per, **ens,
        # per member, rows every 10 samples: step, Nu_vol, Nu_wall, Re_rms, Nu_kin, Nu_th, Re_w
        "series": [r["series"][:rows] for r in runs],
    }
    return out


def main():
    N, Ra, Pr = int(sys.argv[1]), float(sys.argv[2]), float(sys.argv[3])
    transient, average, every = float(sys.argv[4]), float(sys.argv[5]), int(sys.argv[6])
    seed0, members, outdir = int(sys.argv[7]), int(sys.argv[8]), sys.argv[9]
    os.makedirs(outdir, exist_ok=True)
    paths = [os.path.join(outdir, f"member_{k}.json") for k in range(members)]
    if "--combine-only" not in sys.argv:
        import multiprocessing as mp

        jobs = [(N, Ra, Pr, transient, average, every, seed0 + k, paths[k]) for k in range(members)]
        with mp.get_context("spawn").Pool(members) as pool:
            pool.map(member, jobs)
    json.dump(combine(N, Ra, Pr, every, paths), sys.stdout, indent=1)
    sys.stdout.write("\n")


if __name__ == "__main__":
    main()
