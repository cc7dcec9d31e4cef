"""Write the FP64 oracle's steady state of the side-heated cell (reference for
the GPU steady-state test).  Calls only oracle/ and the seeded-input module.

Cell: cube of N^3 nodes, Ra = 1e6, Pr = 0.71, U = 0.1, hot wall x = 0
(T = +1/2), cold wall x = H (T = -1/2), four adiabatic walls, all no-slip.
Steady criterion: relative change of the hot-wall Nusselt number below 1e-7
over 1000 steps, checked every 1000 steps.  The run starts from the oracle's
own converged 33^3 solution interpolated to N^3 (the steady state does not
depend on the start; this only shortens the run); N = 33 starts from rest.

  python tests/golden/make_steady_side_heated.py [N] > tests/golden/steady_side_heated_65.json
"""
import json
import os
import sys
import time

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))
import oracle  # noqa: E402

RA, PR, U = 1e6, 0.71, 0.1
TOL, EVERY = 1e-7, 1000


def converge(p, f, g, max_steps, log):
    d = oracle.diagnostics(p, f, g)
    prev, steps = d["Nu_face"][0], 0
    while steps < max_steps:
        f, g = oracle.run(p, f, g, EVERY)
        steps += EVERY
        d = oracle.diagnostics(p, f, g)
        nu = d["Nu_face"][0]
        rel = abs(nu - prev) / abs(nu)
        log.write(f"N={p.nx} step {steps} Nu_hot {nu:.10f} rel {rel:.3e}\n")
        log.flush()
        if rel < TOL:
            return f, g, steps, d, True
        prev = nu
    return f, g, steps, d, False


def interpolate(field, n_new):
    """Trilinear interpolation of a node-centred field (n^3) to n_new^3 nodes."""
    n = field.shape[-1]
    c_old = (np.arange(n) + 0.5) / n
    c_new = (np.arange(n_new) + 0.5) / n_new
    out = field
    for axis in (-1, -2, -3):
        out = np.apply_along_axis(lambda v: np.interp(c_new, c_old, v), axis, out)
    return out


def main():
    N = int(sys.argv[1]) if len(sys.argv) > 1 else 65
    log = sys.stderr
    t0 = time.time()
    pc = oracle.cell(33, RA, PR, oracle.side_heated_walls(), U=U)
    f, g = oracle.init_equilibrium(pc, 1.0, np.zeros(3), 0.0)
    f, g, sc, dc, okc = converge(pc, f, g, 200000, log)
    if N == 33:
        p, steps, d, ok, sc = pc, sc, dc, okc, 0
    else:
        rho, u, T = oracle.moments(pc, f, g)
        p = oracle.cell(N, RA, PR, oracle.side_heated_walls(), U=U)
        ui = np.stack([interpolate(u[a], N) for a in range(3)])
        Ti = interpolate(T, N)
        f, g = oracle.init_equilibrium(p, 1.0, ui, Ti)
        f, g, steps, d, ok = converge(p, f, g, 400000, log)
    out = {
        "what": "FP64 oracle steady state, side-heated cube, Ra=1e6, Pr=0.71, U=0.1",
        "N": N, "steps": steps, "converged": bool(ok), "coarse_steps": sc,
        "criterion": "relative change of Nu_hot < 1e-7 over 1000 steps",
        "Nu_hot": float(d["Nu_face"][0]), "Nu_cold": float(-d["Nu_face"][1]),
        "Nu_hot_link": float(d["Nu_face_link"][0]), "Nu_cold_link": float(-d["Nu_face_link"][1]),
        "E": float(d["E"]), "Nu_vol": float(d["Nu_vol"]), "rms_div": float(d["rms_div"]),
        "max_u": float(d["max_u"]), "cpu_seconds": round(time.time() - t0, 1),
    }
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
