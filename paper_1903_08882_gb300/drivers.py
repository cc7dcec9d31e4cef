"""Run drivers over the C ABI: steady-state runs (Sec. 3), statistically
averaged runs (Sec. 4) and the host-side formulas of the paper.

These only sequence lbm_step / lbm_sample / lbm_diagnostics calls and do
scalar arithmetic on the returned diagnostics; every lattice operation runs
in the CUDA library.
"""
from __future__ import annotations

import json
import math
import os
import time

import numpy as np


class RunLog:
    """Append-only JSON-lines log of a run: one object per line with the
    record kind, the wall-clock time and the given fields (numbers, strings,
    lists; numpy values are converted).  Opened in append mode, so a resumed
    run continues the same file.  Use as a context manager or call close()."""

    def __init__(self, path: str):
        self.path = path
        d = os.path.dirname(os.path.abspath(path))
        os.makedirs(d, exist_ok=True)
        self._fh = open(path, "a")

    @staticmethod
    def _plain(v):
        if isinstance(v, dict):
            return {k: RunLog._plain(x) for k, x in v.items()}
        if isinstance(v, (list, tuple)):
            return [RunLog._plain(x) for x in v]
        if isinstance(v, np.ndarray):
            return v.tolist()
        if isinstance(v, np.generic):
            return v.item()
        return v

    def write(self, kind: str, **fields):
        rec = {"kind": kind, "time": time.time()}
        rec.update({k: self._plain(v) for k, v in fields.items()})
        self._fh.write(json.dumps(rec) + "\n")
        self._fh.flush()

    def close(self):
        if self._fh:
            self._fh.close()
            self._fh = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def read_log(path: str):
    """The records of a RunLog file, in order."""
    with open(path) as fh:
        return [json.loads(line) for line in fh if line.strip()]


def free_fall_steps(H: float, U: float) -> float:
    """Lattice steps per free-fall time t_f = sqrt(H/(g beta dT)) = H/U."""
    return H / U


def run_to_steady(lat, every: int = 1000, tol: float = 1e-7, max_steps: int = 2_000_000, face: int = 0,
                  min_steps: int = 0, average: int = 1, log: RunLog | None = None):
    """Advance until the relative change of the Nusselt number of Dirichlet
    face `face` over `every` steps is below `tol` (the steady criterion on the
    hot-wall Nusselt number; Sec. 3 uses a field criterion instead).
    With average = k > 1 the criterion compares the means of the last k
    samples and of the k before them (for storages whose stochastic rounding
    leaves a small sample-to-sample noise on Nu), and Nu is the mean of the
    last k samples.
    Returns dict(steps, converged, Nu, history, diag, diag_mean): diag is the
    last sample's diagnostics, diag_mean the wall Nusselt numbers (Nu_face,
    Nu_link) averaged over the last k samples.  With a RunLog every sample is
    written as a "sample" record (step, Nu, Re_rms, E) and the outcome as a
    "steady" record."""
    k = max(1, int(average))
    lat.sample()
    prev = lat.diagnostics()["Nu_face"][face]
    hist, steps, walls = [prev], 0, []

    def done(converged, d):
        nu_face = np.mean([w[0] for w in walls[-k:]], axis=0)
        nu_link = np.mean([w[1] for w in walls[-k:]], axis=0)
        out = dict(steps=steps, converged=converged, Nu=float(np.mean(hist[-k:])), history=np.array(hist),
                   diag=d, diag_mean=dict(Nu_face=nu_face, Nu_link=nu_link))
        if log is not None:
            log.write("steady", steps=steps, converged=converged, Nu=out["Nu"], tol=tol, average=k,
                      Nu_face=nu_face, Nu_link=nu_link)
        return out

    while steps < max_steps:
        lat.step(every)
        steps += every
        lat.sample()
        d = lat.diagnostics(reset=True)
        hist.append(d["Nu_face"][face])
        walls.append((np.array(d["Nu_face"]), np.array(d.get("Nu_link", d["Nu_face"]))))
        if log is not None:
            log.write("sample", step=steps, Nu=d["Nu_face"][face], Re_rms=d.get("Re_rms"), E=d.get("E"))
        walls = walls[-k:]
        if len(hist) > 2 * k and steps >= min_steps:
            new, old = float(np.mean(hist[-k:])), float(np.mean(hist[-2 * k:-k]))
            if abs(new - old) <= tol * abs(new):
                return done(True, d)
    return done(False, d)


def grid_convergence(meshes, values):
    """Grid-convergence estimate of Sec. 3 (Table 2): the asymptotic value
    f_inf is the h = 0 value of the polynomial in h = 1/N that interpolates
    the results on all meshes (degree = number of meshes - 1), and the order
    n is the least-squares slope of log(|f_N - f_inf| / |f_inf|) against
    -log N.  Returns (f_inf, n)."""
    N = np.asarray(meshes, dtype=np.float64)
    f = np.asarray(values, dtype=np.float64)
    if len(N) < 3 or len(N) != len(f):
        raise ValueError("need the same number (>= 3) of meshes and values")
    f_inf = float(np.polyfit(1.0 / N, f, len(N) - 1)[-1])
    err = np.abs(f - f_inf) / abs(f_inf)
    n = float(-np.polyfit(np.log(N), np.log(err), 1)[0])
    return f_inf, n


def field_residuals(u_new, u_old, T_new, T_old):
    """Steady-state residuals of Sec. 3: sum |u(t+dt) - u(t)|_2 / sum |u(t)|_2
    and sum |T(t+dt) - T(t)| / sum |T(t)| over the nodes."""
    du = np.sqrt(((u_new - u_old) ** 2).sum(axis=0)).sum() / max(np.sqrt((u_old**2).sum(axis=0)).sum(), 1e-300)
    dT = np.abs(T_new - T_old).sum() / max(np.abs(T_old).sum(), 1e-300)
    return du, dT


def blocking_standard_error(x, first_block: int = 8, min_blocks: int = 5) -> float:
    """Standard error of the mean of a correlated series by blocking: the
    series is cut into blocks of length b = first_block, 2 first_block, ...
    while at least min_blocks blocks remain, the standard error is taken from
    the spread of the block means for each b, and the largest is returned.
    Once blocks are longer than the correlation time the block means are
    independent and the estimate levels off at the true error; for shorter
    blocks it is too small, so the maximum is the conservative choice.  Used
    for the time averages of Sec. 4, whose samples stay correlated over many
    free-fall times."""
    x = np.asarray(x, dtype=np.float64)
    se, b = 0.0, int(first_block)
    if b < 1 or len(x) // b < min_blocks:
        raise ValueError("series too short for the first block length")
    while len(x) // b >= min_blocks:
        nb = len(x) // b
        means = x[: nb * b].reshape(nb, b).mean(axis=1)
        se = max(se, float(means.std(ddof=1) / math.sqrt(nb)))
        b *= 2
    return se


def dissipation_pdf(eps, nbins: int = 200, xmax: float = 20.0, rms: float | None = None):
    """Probability density of X = eps / eps_rms over the nodes (Sec. 4, the
    PDFs of the kinetic and thermal dissipation rates), eps_rms = sqrt(<eps^2>)
    unless given (a time series normalises by the rms over all its samples).
    Returns (bin centres, density, eps_rms); the density integrates to the
    fraction of nodes with X < xmax."""
    e = np.asarray(eps, dtype=np.float64).ravel()
    if rms is None:
        rms = float(np.sqrt(np.mean(e * e)))
    if not rms > 0:
        raise ValueError("eps is zero everywhere")
    edges = np.linspace(0.0, xmax, nbins + 1)
    counts, _ = np.histogram(e / rms, bins=edges)
    width = edges[1] - edges[0]
    return 0.5 * (edges[1:] + edges[:-1]), counts / (e.size * width), rms


def averaged_dissipation_pdf(lat, transient_steps: int, average_steps: int, every: int, nbins: int = 400,
                             xmax: float = 40.0):
    """Volume-and-time PDFs of the local dissipation rates (Sec. 4): after the
    transient, one sample every `every` steps over `average_steps`, each
    binned as eps / r0 with r0 the first sample's eps_rms; the rms over
    volume and time, r = sqrt(<eps^2>_{V,t}), is known only at the end, and
    the histogram of eps / r is the same histogram with its abscissa scaled
    by r0 / r.  Returns the bin centres and densities of X = eps / r for
    eps_u and eps_T, the two r, and the sample count."""
    if every < 1 or average_steps < every:
        raise ValueError("need at least one sample")
    lat.step(int(transient_steps))
    cu = np.zeros(nbins)
    ct = np.zeros(nbins)
    sq = np.zeros(2)
    r0 = None
    samples = 0
    for _ in range(int(average_steps) // int(every)):
        lat.step(int(every))
        _, _, own = lat.dissipation_pdf(nbins=1, xmax=1e300)  # this sample's eps_rms
        if r0 is None:
            if not (own[0] > 0 and own[1] > 0):
                raise ValueError("a dissipation rate is zero everywhere in the first sample")
            r0 = own
        u, t, _ = lat.dissipation_pdf(nbins=nbins, xmax=xmax, rms=r0)
        cu += u
        ct += t
        sq += np.square(own)
        samples += 1
    r = np.sqrt(sq / samples)
    nodes = int(np.prod(lat.shape))
    out = dict(rms_u=float(r[0]), rms_T=float(r[1]), samples=samples)
    for key, counts, k in (("u", cu, 0), ("T", ct, 1)):
        width = xmax / nbins * r0[k] / r[k]
        out["x_" + key] = (np.arange(nbins) + 0.5) * width
        out["pdf_" + key] = counts / (nodes * samples * width)
    return out


def fit_stretched_exponential(x, pdf, x_min: float = 0.0, alphas=(0.05, 3.0)):
    """Fit of the PDF tail to the stretched exponential of Sec. 4,
    p(X*) = C / sqrt(X*) exp(-m X*^alpha), X* = X - X_mp, with X_mp the
    abscissa of the most probable value.  The fit is least squares on
    log p over the tail bins, X* > x_min, with a non-zero density: for a given
    alpha, log p + log(X*)/2 = log C - m X*^alpha is linear in (log C, m),
    and alpha minimises the residual.  Each bin is weighted by its density:
    a histogram bin's log has a variance of about 1/count, so the sparse far
    tail would otherwise dominate.  Returns C, m, alpha, X_mp and the
    adjusted R^2 of the fit in log p (three parameters, same weights)."""
    from scipy.optimize import minimize_scalar

    x = np.asarray(x, dtype=np.float64)
    pdf = np.asarray(pdf, dtype=np.float64)
    x_mp = float(x[int(np.argmax(pdf))])
    sel = (x - x_mp > x_min) & (pdf > 0)
    xs = x[sel] - x_mp
    y = np.log(pdf[sel]) + 0.5 * np.log(xs)
    if xs.size < 4:
        raise ValueError("too few tail bins to fit")

    wt = pdf[sel] / pdf[sel].sum()
    sw = np.sqrt(wt)

    def solve(alpha):
        A = np.stack([np.ones_like(xs), -xs**alpha], axis=1)
        coef, *_ = np.linalg.lstsq(A * sw[:, None], y * sw, rcond=None)
        return coef, float((wt * (A @ coef - y) ** 2).sum())

    res = minimize_scalar(lambda a: solve(a)[1], bounds=alphas, method="bounded", options={"xatol": 1e-6})
    (logC, m), sse = solve(res.x)
    lp = np.log(pdf[sel])
    sst = float((wt * (lp - (wt * lp).sum()) ** 2).sum())
    n = xs.size
    r2 = 1.0 - sse / sst if sst > 0 else 1.0
    r2_adj = 1.0 - (1.0 - r2) * (n - 1) / max(n - 4, 1)
    return dict(C=float(np.exp(logC)), m=float(m), alpha=float(res.x), x_mp=x_mp, r2_adj=float(r2_adj))


def averaged_statistics(lat, transient_steps: int, average_steps: int, diag_every: int):
    """Sec. 4 protocol: discard a transient, then average the sampled
    diagnostics over average_steps (samples every diag_every steps are taken
    by the library when it was created with that diag_every).  Returns the
    volume-and-time averages Re^rms, Re_w^rms, Nu_vol, Nu_wall, Nu_kin, Nu_th."""
    lat.step(transient_steps)
    lat.diagnostics(reset=True)
    lat.step(average_steps)
    d = lat.diagnostics(reset=False)
    nu_wall = 0.5 * (d["avg_Nu_face"][4] - d["avg_Nu_face"][5])
    return dict(Re_rms=d["avg_Re_rms"], Re_w=d["avg_Re_w"], Nu_vol=d["avg_Nu_vol"], Nu_wall=nu_wall,
                Nu_kin=d["avg_Nu_kin"], Nu_th=d["avg_Nu_th"], E=d["avg_E"], samples=d["samples"], diag=d)


def resolution(Ra: float, Pr: float, Nu: float, H: float):
    """Resolution estimates of Sec. 4 (Table 5): Kolmogorov length
    eta = H Pr^(1/2) / [Ra (Nu - 1)]^(1/4), Batchelor length eta_B = eta Pr^(-1/2),
    Kolmogorov time tau_eta = sqrt(Pr/(Nu - 1)) in free-fall units, and the nodes
    in the thermal boundary layer N_BL = H/(2 Nu); grid spacing 1, time step
    U/H free-fall units (lattice units with U the free-fall velocity)."""
    eta = H * math.sqrt(Pr) / (Ra * (Nu - 1.0)) ** 0.25
    eta_B = eta / math.sqrt(Pr)
    tau_eta = math.sqrt(Pr / (Nu - 1.0))
    return dict(dg_over_eta=1.0 / eta, dg_over_etaB=1.0 / eta_B, tau_eta=tau_eta, N_BL=H / (2.0 * Nu))


def _centre_pair(n: int):
    """Node indices whose centres bracket the mid-point H/2 of an axis of n
    nodes (node j at j + 1/2): one node for odd n, two for even n."""
    return sorted({(n - 1) // 2, n // 2})


def centerline_probes(u3, U: float):
    """Table 1 probes of the side-heated cell (hot wall at x = 0 here, so the
    paper's y is our x): maximum horizontal velocity u along the vertical
    centreline of the mid-plane y = 1/2, with its height z, and maximum
    vertical velocity w along the horizontal centreline, with its position x.
    Velocities in free-fall units; positions at node centres (j + 1/2)/N.
    On an even mesh the mid-plane falls between two node planes, and the
    centreline values are interpolated linearly (the mean of the two, or of
    the four lines around the centre)."""
    nz, ny, nx = u3.shape[1:]
    ys, xs, zs = _centre_pair(ny), _centre_pair(nx), _centre_pair(nz)
    col = np.mean([u3[0][:, jy, jx] for jy in ys for jx in xs], axis=0) / U
    row = np.mean([u3[2][jz, jy, :] for jz in zs for jy in ys], axis=0) / U
    k = int(np.argmax(np.abs(col)))
    i = int(np.argmax(np.abs(row)))
    return dict(u_max=float(col[k]), z=(k + 0.5) / nz, w_max=float(row[i]), x=(i + 0.5) / nx)


def sweep_cells(lbm, seed: int = 190308882, ncells: int = 64, storage: str = "fp32", stream=None,
                min_bl_nodes: float = 2.0):
    """Cells of a batched sweep: half side-heated, half Rayleigh-Benard, drawn
    from inputs.cell_candidates.  A draw is skipped when the library rejects
    its parameters (for instance a_T >= 1, a negative D3Q7 rest weight) or when
    fewer than `min_bl_nodes` nodes would fall in the thermal boundary layer
    H/(2 Nu), Nu estimated from the fit Nu = 0.153 Ra^0.289 of Sec. 4.
    Returns (lattices, draws) with the lattices at rest."""
    from . import inputs

    lats, draws = [], []
    for edge, Ra, Pr in inputs.cell_candidates(seed, 50 * ncells):
        if len(lats) == ncells:
            break
        if edge / (2.0 * 0.153 * Ra ** 0.289) < min_bl_nodes:
            continue
        kind = "side" if len(lats) < ncells // 2 else "rb"
        walls = lbm.walls_side_heated() if kind == "side" else lbm.walls_rayleigh_benard()
        try:
            lat = lbm.Lattice(edge, edge, edge, walls, Ra=Ra, Pr=Pr, storage=storage, stream=stream)
        except lbm.LbmError as e:
            if e.status == lbm.LBM_ERR_PARAM:
                continue
            raise
        lats.append(lat)
        draws.append(dict(edge=edge, Ra=Ra, Pr=Pr, kind=kind))
    if len(lats) < ncells:
        raise RuntimeError(f"only {len(lats)} usable cells drawn")
    return lats, draws
