"""Write the FP64 oracle's volume-and-time histograms of the local dissipation
rates in a Rayleigh-Benard cell (the PDFs of Sec. 4).  Calls only oracle/ and
the seeded-input module.

Cell and start as in make_rb_statistics.py (cube of N^3 nodes, hot bottom and
cold top plates, adiabatic no-slip sidewalls, free-fall scaling with U = 0.1,
conduction profile plus a seeded perturbation).  After `transient` free-fall
times, one sample every `every` steps over `average` free-fall times: per node
eps_u = nu/2 sum_ij (d_i u_j + d_j u_i)^2 and eps_T = kappa |grad T|^2.  Each
sample is binned as eps / r0 (r0: the first sample's rms) in `nbins` bins on
[0, xmax); the rms over volume and time r is stored too, so X = eps / r has
bin edges (r0 / r) x the stored ones.  The counts and the sums of the
samples' squared rms are also stored per block of `block` consecutive samples,
from which a test estimates the statistical error of quantities of the PDFs.

  python tests/golden/make_rb_dissipation_pdf.py N Ra Pr transient average every seed nbins xmax block > out.json
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
    nbins, xmax = int(sys.argv[8]), float(sys.argv[9])
    block = int(sys.argv[10]) if len(sys.argv) > 10 else 0
    U = 0.1
    t0 = time.time()
    p = oracle.cell(N, Ra, Pr, oracle.rayleigh_benard_walls(), U=U)
    tf = N / U
    T = inputs.rb_initial_temperature(N, N, N, seed=seed)
    f, g = oracle.init_equilibrium(p, 1.0, np.zeros(3), T)
    n_tr = int(round(transient * tf / every)) * every
    n_av = int(round(average * tf / every)) * every
    f, g = oracle.run(p, f, g, n_tr)
    edges = np.linspace(0.0, xmax, nbins + 1)
    counts = [np.zeros(nbins, dtype=np.int64), np.zeros(nbins, dtype=np.int64)]
    sq = np.zeros(2)
    r0 = None
    samples = 0
    blocks = []
    bc = [np.zeros(nbins, dtype=np.int64), np.zeros(nbins, dtype=np.int64)]
    bsq = np.zeros(2)
    for k in range(n_av // every):
        f, g = oracle.run(p, f, g, every)
        eps = oracle.local_dissipation(p, f, g)
        own = np.array([np.sqrt(np.mean(e * e)) for e in eps])
        if r0 is None:
            r0 = own
        for c, b, e, r in zip(counts, bc, eps, r0):
            h = np.histogram(e.ravel() / r, bins=edges)[0]
            c += h
            b += h
        sq += own**2
        bsq += own**2
        samples += 1
        if block and samples % block == 0:
            blocks.append({"counts_u": bc[0].tolist(), "counts_T": bc[1].tolist(), "sum_rms2": bsq.tolist()})
            bc = [np.zeros(nbins, dtype=np.int64), np.zeros(nbins, dtype=np.int64)]
            bsq = np.zeros(2)
        sys.stderr.write(f"sample {k} rms_u {own[0]:.4e} rms_T {own[1]:.4e}\n")
        sys.stderr.flush()
    r = np.sqrt(sq / samples)
    out = {
        "what": "FP64 oracle volume-and-time histograms of the local dissipation rates (Sec. 4 PDFs)",
        "N": N, "Ra": Ra, "Pr": Pr, "U": U, "seed": seed, "transient_steps": n_tr, "average_steps": n_av,
        "sample_every": every, "samples": samples, "nodes": N**3, "nbins": nbins, "xmax_in_r0": xmax,
        "r0_u": float(r0[0]), "r0_T": float(r0[1]), "rms_u": float(r[0]), "rms_T": float(r[1]),
        "counts_u": counts[0].tolist(), "counts_T": counts[1].tolist(),
        "block_samples": block, "blocks": blocks,
        "cpu_seconds": round(time.time() - t0, 1),
    }
    json.dump(out, sys.stdout)


if __name__ == "__main__":
    main()
