"""Write the FP64 oracle's time-averaged Rayleigh-Benard statistics (reference
for the GPU statistics test).  Calls only oracle/ and the seeded-input module.

Cell: cube of N^3 nodes, hot bottom wall (T = +1/2), cold top wall
(T = -1/2), four adiabatic sidewalls, all no-slip; free-fall scaling with
U = 0.1, t_f = H/U steps.  Start: the linear conduction profile plus a seeded
uniform perturbation of amplitude 1e-3, at rest (Sec. 4 set-up).  Protocol:
`transient` free-fall times discarded, then the volume-and-time averages of
Sec. 4 over `average` free-fall times, sampled every `every` steps.

  python tests/golden/make_rb_statistics.py N Ra Pr transient average every seed > out.json
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import oracle  # noqa: E402
from paper_1903_08882_gb300 import inputs  # noqa: E402


def main():
    N, Ra, Pr = int(sys.argv[1]), float(sys.argv[2]), float(sys.argv[3])
    transient, average, every, seed = float(sys.argv[4]), float(sys.argv[5]), int(sys.argv[6]), int(sys.argv[7])
    U = 0.1
    t0 = time.time()
    p = oracle.cell(N, Ra, Pr, oracle.rayleigh_benard_walls(), U=U)
    tf = N / U
    T = inputs.rb_initial_temperature(N, N, N, seed=seed)
    f, g = oracle.init_equilibrium(p, 1.0, np.zeros(3), T)
    n_tr = int(round(transient * tf / every)) * every
    n_av = int(round(average * tf / every)) * every
    f, g = oracle.run(p, f, g, n_tr)
    acc = np.zeros(oracle.NDIAG)
    samples = 0
    series = []
    for k in range(n_av // every):
        r = oracle.raw_diagnostics(p, f, g)
        acc += r
        samples += 1
        if k % 10 == 0:
            d = oracle.finalize(p, r)
            series.append([k * every, d["Nu_vol"], 0.5 * (d["Nu_face"][4] - d["Nu_face"][5]), d["Re_rms"],
                           d["Nu_kin"], d["Nu_th"], d["Re_w"]])
            sys.stderr.write(f"sample {k} Nu_vol {d['Nu_vol']:.4f} Re {d['Re_rms']:.3f}\n")
            sys.stderr.flush()
        f, g = oracle.run(p, f, g, every)
    d = oracle.finalize(p, acc / samples)
    out = {
        "what": "FP64 oracle Rayleigh-Benard statistics (volume and time averages of Sec. 4)",
        "N": N, "Ra": Ra, "Pr": Pr, "U": U, "seed": seed, "transient_steps": n_tr, "average_steps": n_av,
        "sample_every": every, "samples": samples,
        "Re_rms": float(d["Re_rms"]), "Re_w": float(d["Re_w"]), "Nu_vol": float(d["Nu_vol"]),
        "Nu_wall": float(0.5 * (d["Nu_face"][4] - d["Nu_face"][5])), "Nu_kin": float(d["Nu_kin"]),
        "Nu_th": float(d["Nu_th"]), "E": float(d["E"]),
        # rows: step, Nu_vol, Nu_wall, Re_rms, Nu_kin, Nu_th, Re_w
        "series_step_Nuvol_Nuwall_Re": series,
        "cpu_seconds": round(time.time() - t0, 1),
    }
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
