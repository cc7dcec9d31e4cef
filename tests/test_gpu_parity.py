"""GPU parity: the CUDA library against the FP64 oracle, element by element.

Tolerances (relative L-infinity, normalised by the largest deviation of the
reference from the rest state):
  FP32 storage: populations and fields within 2e-6 after a few steps from a
  shared state (FP32 rounding of O(1e-2) deviations through ~600 operations),
  fields within 1e-6 after one step, and within 1e-5 along a 2000-step run.
  FP16 storage: 2e-3 after one step; BF16: 1.6e-2 (8-bit significand).
Fields are rho - rho0, the velocity vector field and T.
"""
import os
import tempfile

import numpy as np
import pytest

import oracle
from paper_1903_08882_gb300 import inputs

pytestmark = pytest.mark.gpu

A, D, P = 0, 1, 2
W19 = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)


@pytest.fixture(scope="module")
def lbm():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1903_08882_gb300 import _build
    from paper_1903_08882_gb300 import lbm as L

    _build.build()
    oracle.build()
    return L


def _orc_params(n, walls, nu=0.03, kappa=0.02, gbeta=4e-3, H=None, U=0.1, bf=(0, 0, 0)):
    nx, ny, nz = n
    return oracle.Params(nx, ny, nz, walls, nu, kappa, gbeta, float(H or nz), U, bf)


def _lattice(L, n, walls, storage="fp32", streaming="aa", nu=0.03, kappa=0.02, gbeta=4e-3, H=0.0, U=0.1,
             bf=(0, 0, 0), **kw):
    return L.Lattice(*n, walls, nu=nu, kappa=kappa, gbeta=gbeta, H=H, U=U, body_force=bf, storage=storage,
                     streaming=streaming, **kw)


def _random_state(p, seed, du=0.03, nf=1e-4, ng=1e-3):
    sh = (p.nz, p.ny, p.nx)
    rho, u, T = inputs.random_fields(sh, seed, du=du)
    f, g = oracle.init_equilibrium(p, rho, u, T)
    f = f + inputs.noise(f.shape, seed, 20, nf)
    g = g + inputs.noise(g.shape, seed, 21, ng)
    return f, g


def _rel_pop(fa, ga, fb, gb):
    w = W19.reshape((19,) + (1,) * (fb.ndim - 1))
    ef = np.abs(fa - fb).max() / np.abs(fb - w).max()
    eg = np.abs(ga - gb).max() / max(np.abs(gb).max(), 1e-30)
    return ef, eg


def _rel_fields(a, b):
    """Relative L-inf of the fields rho - rho0, u (as one vector field) and T:
    ||a - b||_inf / ||b||_inf, the velocity norm taken over all components."""
    (ra, ua, Ta), (rb, ub, Tb) = a, b
    out = []
    for x, y in [(ra - 1, rb - 1), (ua, ub), (Ta, Tb)]:
        den = np.abs(y).max()
        out.append(np.abs(x - y).max() / den if den > 0 else np.abs(x).max())
    return np.array(out)


WALLS = {
    "side_heated": [(D, 0.5), (D, -0.5), (A, 0), (A, 0), (A, 0), (A, 0)],
    "rayleigh_benard": [(A, 0), (A, 0), (A, 0), (A, 0), (D, 0.5), (D, -0.5)],
    "periodic_xy": [(P, 0), (P, 0), (P, 0), (P, 0), (D, 0.3), (D, -0.2)],
    "mixed": [(A, 0), (A, 0), (D, 0.4), (D, 0.1), (P, 0), (P, 0)],
    "all_periodic": [(P, 0)] * 6,
}


SCHEMES = {  # streaming, nodes per thread, AA pipeline
    "aa1": ("aa", 1, "register"), "aa2": ("aa", 2, "register"), "staged": ("aa", 2, "staged"),
    "pull2": ("pull2", 2, "default"),
}


@pytest.mark.parametrize("scheme", list(SCHEMES))
@pytest.mark.parametrize("walls", list(WALLS))
@pytest.mark.parametrize("n", [(5, 6, 7), (13, 11, 12), (3, 3, 3), (34, 9, 5), (45, 37, 13), (80, 7, 6),
                               (101, 9, 5), (16, 40, 6), (17, 45, 5)])
def test_random_state_steps(lbm, walls, scheme, n):
    """AA register kernels with one and two nodes per thread, the staged AA
    kernels, and the pull scheme.  45 x 37 x 13 spans several 448-node tiles
    per plane of the staged kernels with a ragged tail; 80 x 7 x 6 and
    101 x 9 x 5 give the two-node-per-thread row kernel, which updates the
    x-face nodes of its rows itself, runs of several warps per row; 16 x 40
    x 6 and 17 x 45 x 5 put dozens of rows (and x-face nodes) into one
    448-node tile of the staged kernels."""
    p = _orc_params(n, WALLS[walls])
    f0, g0 = _random_state(p, 3)
    streaming, npt, pipe = SCHEMES[scheme]
    with _lattice(lbm, n, WALLS[walls], streaming=streaming, nodes_per_thread=npt, pipeline=pipe) as lat:
        lat.set_populations(f0, g0)
        f, g = lat.populations()
        ef, eg = _rel_pop(f, g, f0, g0)
        assert ef < 1e-6 and eg < 1e-6  # FP32 round trip
        fo, go = f0, g0
        for k in (1, 2, 3):
            lat.step(1)
            fo, go = oracle.run(p, fo, go, 1)
            f, g = lat.populations()
            ef, eg = _rel_pop(f, g, fo, go)
            assert ef < 2e-6 and eg < 2e-6, (k, ef, eg)
        m = lat.moments()
        e = _rel_fields(m, oracle.moments(p, fo, go))
        assert (e < 2e-6).all(), e


@pytest.mark.parametrize("storage", ["fp16s", "fp16m"])
@pytest.mark.parametrize("walls", list(WALLS))
@pytest.mark.parametrize("n", [(5, 6, 7), (13, 11, 12), (3, 3, 3), (45, 37, 13), (97, 41, 23), (17, 45, 5),
                               (20, 3, 40)])
def test_staged_reduced_storage_random_states(lbm, walls, storage, n):
    """The staged kernels with the 2-byte storages, whose odd step leaves the
    y/z-face nodes (every face node for rows shorter than 16 nodes) to the
    face kernel, on every wall set.  Shapes from a single tile (most blocks
    get none) to several tiles per plane and rows shorter than 16 nodes; four steps
    (two odd) from a random state against the register kernels with the
    same storage (same roundings and random bits: agreement to the last bit
    of the 11-bit significand but for multiply-add contraction, 2e-3) and
    against the oracle (one storage rounding per step, 4e-3)."""
    p = _orc_params(n, WALLS[walls])
    f0, g0 = _random_state(p, 5)
    out = []
    for pipe in ("register", "staged"):
        with _lattice(lbm, n, WALLS[walls], storage=storage, nodes_per_thread=2, pipeline=pipe) as lat:
            lat.set_populations(f0, g0)
            lat.step(4)
            out.append(lat.populations())
    fo, go = oracle.run(p, f0, g0, 4)
    ef, eg = _rel_pop(*out[1], *out[0])
    assert ef < 2e-3 and eg < 2e-3, (ef, eg)
    ef, eg = _rel_pop(*out[1], fo, go)
    assert ef < 4e-3 and eg < 4e-3, (ef, eg)


def test_shared_state_one_step_cfg1(lbm):
    """Side-heated 33^3, Ra=1e4, Pr=0.71: the oracle state after 500 steps from
    rest, loaded into the library; one and two steps."""
    n = (33, 33, 33)
    p = oracle.cell(33, 1e4, 0.71, oracle.side_heated_walls())
    f0, g0 = oracle.init_equilibrium(p, 1.0, np.zeros(3), 0.0)
    f0, g0 = oracle.run(p, f0, g0, 500)
    with lbm.Lattice(*n, lbm.walls_side_heated(), Ra=1e4, Pr=0.71) as lat:
        lat.set_populations(f0, g0)
        fo, go = f0, g0
        for k in (1, 2):
            lat.step(1)
            fo, go = oracle.run(p, fo, go, 1)
            e = _rel_fields(lat.moments(), oracle.moments(p, fo, go))
            assert (e < 1e-6).all(), (k, e)


def test_cfg1_trajectory_2000_steps(lbm):
    """Side-heated 33^3 from rest, 2000 steps; fields and wall Nusselt numbers
    compared with the oracle every 100 steps."""
    n = (33, 33, 33)
    p = oracle.cell(33, 1e4, 0.71, oracle.side_heated_walls())
    fo, go = oracle.init_equilibrium(p, 1.0, np.zeros(3), 0.0)
    worst, worst_nu = 0.0, 0.0
    with lbm.Lattice(*n, lbm.walls_side_heated(), Ra=1e4, Pr=0.71) as lat:
        for t in range(100, 2001, 100):
            lat.step(100)
            fo, go = oracle.run(p, fo, go, 100)
            e = _rel_fields(lat.moments(), oracle.moments(p, fo, go))
            worst = max(worst, e.max())
            lat.sample()
            d = lat.diagnostics()
            od = oracle.diagnostics(p, fo, go)
            for k in (0, 1):
                worst_nu = max(worst_nu, abs(d["Nu_face"][k] - od["Nu_face"][k]) / abs(od["Nu_face"][k]))
    assert worst < 1e-5, worst
    assert worst_nu < 1e-5, worst_nu
    assert od["Nu_face"][0] > 1.5  # convection has set in


@pytest.mark.parametrize("diag_every", [0, 40])
def test_rayleigh_benard_trajectory(lbm, diag_every):
    """Rayleigh-Benard cell 24^3, Ra=1e6, Pr=7, from the seeded linear profile:
    the early trajectory (before chaos) against the oracle every 500 steps,
    with and without diagnostic sampling inside the steps.  The conduction
    state is linearly unstable at this Ra (Sec. 4), so FP32 rounding
    differences grow with the convective mode: two FP32 kernels that differ
    only in where the compiler fuses multiply-adds land 1.0e-4 and 1.1e-4 from
    the FP64 oracle at t = 3000.  The bound is 3e-4; a wrong term in the
    update gives errors of order one."""
    N = 24
    p = oracle.cell(N, 1e6, 7.0, oracle.rayleigh_benard_walls())
    T0 = inputs.rb_initial_temperature(N, N, N, seed=190308882)
    fo, go = oracle.init_equilibrium(p, 1.0, np.zeros(3), T0)
    worst, hist = 0.0, []
    with lbm.Lattice(N, N, N, lbm.walls_rayleigh_benard(), Ra=1e6, Pr=7.0, diag_every=diag_every) as lat:
        lat.set_fields(1.0, np.zeros(3), T0)
        for t in range(500, 3001, 500):
            lat.step(500)
            fo, go = oracle.run(p, fo, go, 500)
            e = _rel_fields(lat.moments(), oracle.moments(p, fo, go))
            worst = max(worst, e.max())
            hist.append(float(e.max()))
    assert worst < 3e-4, hist


@pytest.mark.parametrize("kernels", ["aa1", "aa2", "staged"])
@pytest.mark.parametrize("storage,tol", [("fp16s", 2e-3), ("bf16s", 1.6e-2), ("fp16m", 2e-3)])
def test_reduced_storage_one_step(lbm, storage, tol, kernels):
    n = (33, 33, 33)
    p = oracle.cell(33, 1e4, 0.71, oracle.side_heated_walls())
    f0, g0 = oracle.init_equilibrium(p, 1.0, np.zeros(3), 0.0)
    f0, g0 = oracle.run(p, f0, g0, 500)
    fo, go = oracle.run(p, f0, g0, 1)
    _, npt, pipe = SCHEMES[kernels]
    with lbm.Lattice(*n, lbm.walls_side_heated(), Ra=1e4, Pr=0.71, storage=storage,
                     nodes_per_thread=npt, pipeline=pipe) as lat:
        lat.set_populations(f0, g0)
        lat.step(1)
        e = _rel_fields(lat.moments(), oracle.moments(p, fo, go))
        lat.step(1)
        e2 = _rel_fields(lat.moments(), oracle.moments(p, *oracle.run(p, fo, go, 1)))
    assert (e < tol).all() and (e2 < 2 * tol).all(), (e, e2)


def test_diagnostics_parity(lbm):
    n = (33, 33, 33)
    for walls, owalls in ((lbm.walls_side_heated(), oracle.side_heated_walls()),
                          (lbm.walls_rayleigh_benard(), oracle.rayleigh_benard_walls())):
        p = oracle.cell(33, 1e5, 0.71, owalls)
        f0, g0 = _random_state(p, 5, du=0.02, nf=0, ng=0)
        f0, g0 = oracle.run(p, f0, g0, 20)
        od = oracle.diagnostics(p, f0, g0)
        with lbm.Lattice(*n, walls, Ra=1e5, Pr=0.71) as lat:
            lat.set_populations(f0, g0)
            lat.sample()
            d = lat.diagnostics()
        for k in ("E", "rms_drho", "rms_div", "Re_rms", "Re_w", "Nu_vol", "Nu_kin", "Nu_th"):
            assert abs(d[k] - od[k]) <= 1e-5 * abs(od[k]) + 1e-12, (k, d[k], od[k])
        assert np.allclose(d["Nu_face"], od["Nu_face"], rtol=1e-5, atol=1e-9)
        assert np.allclose(d["Nu_link"], od["Nu_face_link"], rtol=1e-4, atol=1e-7)
        assert abs(d["mass"] - od["mass"]) < 1e-6 * od["mass"]


def test_aa_matches_pull2_long_run(lbm):
    n = (21, 19, 20)
    p = _orc_params(n, WALLS["rayleigh_benard"])
    f0, g0 = _random_state(p, 8, du=0.01)
    out = []
    for streaming in ("aa", "pull2"):
        with _lattice(lbm, n, WALLS["rayleigh_benard"], streaming=streaming) as lat:
            lat.set_populations(f0, g0)
            lat.step(301)
            out.append(lat.populations())
    ef, eg = _rel_pop(*out[0], *out[1])
    assert ef < 1e-5 and eg < 1e-5, (ef, eg)


def test_poiseuille_gpu(lbm):
    N, nu, F = 16, 0.1, 1e-6
    walls = [(P, 0), (P, 0), (A, 0), (A, 0), (P, 0), (P, 0)]
    with _lattice(lbm, (3, N, 3), walls, nu=nu, kappa=0.05, gbeta=0.0, bf=(F, 0, 0)) as lat:
        lat.step(12000)
        rho, u, T = lat.moments()
    j = np.arange(N) + 0.5
    exact = F / (2 * nu) * j * (N - j)
    assert np.abs(u[0][:, :, 1] - exact[None, :]).max() / exact.max() < 1e-5


def test_conservation_gpu(lbm):
    n = (24, 20, 22)
    walls = [(A, 0)] * 6
    p = _orc_params(n, walls)
    f0, g0 = _random_state(p, 12, du=0.01)
    with _lattice(lbm, n, walls) as lat:
        lat.set_populations(f0, g0)
        lat.sample()
        d0 = lat.diagnostics()
        lat.step(1000)
        lat.sample()
        d1 = lat.diagnostics()
    nn = np.prod(n)
    assert abs(d1["mass"] - d0["mass"]) / nn < 1e-5
    assert abs(d1["mean_T"] - d0["mean_T"]) < 1e-5


def test_checkpoint_resume_bit_identical(lbm):
    n = (17, 15, 16)
    with lbm.Lattice(*n, lbm.walls_rayleigh_benard(), Ra=1e5, Pr=0.7, diag_every=5) as lat:
        T0 = inputs.rb_initial_temperature(*n, seed=4)
        lat.set_fields(1.0, np.zeros(3), T0)
        lat.step(37)
        with tempfile.TemporaryDirectory() as td:
            path = os.path.join(td, "ck.bin")
            lat.save(path)
            lat.step(20)
            fa, ga = lat.populations()
            da = lat.diagnostics()
            lat.load(path)
            lat.step(20)
            fb, gb = lat.populations()
            db = lat.diagnostics()
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)
    assert da["samples"] == db["samples"] and da["avg_Nu_vol"] == db["avg_Nu_vol"]


@pytest.mark.parametrize("storage", ["fp32", "fp16s"])
def test_staged_matches_register_kernels(lbm, storage):
    """The staged and the register AA kernels run the same collision and
    differ only in data movement (97 x 41 x 23 cell: several tiles per plane;
    50 steps with samples every 10).  The compiler may contract multiply-adds
    differently in the two kernels, so agreement is asserted to accumulated
    FP32 rounding (50 steps x ~6e-8 x a small growth factor: 1e-5; FP16:
    one storage rounding), not bit for bit."""
    n = (97, 41, 23)
    p = oracle.cell(n, 1e6, 0.71, oracle.side_heated_walls())
    f0, g0 = _random_state(p, 9, du=0.02)
    out = []
    for pipe in ("register", "staged"):
        with lbm.Lattice(*n, lbm.walls_side_heated(), Ra=1e6, Pr=0.71, storage=storage, pipeline=pipe,
                         diag_every=10) as lat:
            lat.set_populations(f0, g0)
            lat.step(50)
            out.append(lat.populations())
            d = lat.diagnostics()
            out.append(d["avg_Nu_face"][0])
    tol = 1e-5 if storage == "fp32" else 2e-3
    ef, eg = _rel_pop(*out[2], *out[0])
    assert ef < tol and eg < tol, (ef, eg)
    assert abs(out[1] - out[3]) <= tol * abs(out[1])


def test_staged_wait_timeout_is_reported(lbm):
    """A zero cycle budget makes every pipeline wait of the staged kernels run
    out: the kernels raise the error flag and return, synchronize reports
    LBM_ERR_TIMEOUT, and the context works again once the budget is back."""
    n = (40, 30, 20)
    p = _orc_params(n, WALLS["side_heated"])
    f0, g0 = _random_state(p, 4)
    with _lattice(lbm, n, WALLS["side_heated"], pipeline="staged") as lat:
        lat.set_populations(f0, g0)
        lat.set_wait_budget(0)
        lat.step(2)
        with pytest.raises(lbm.LbmError) as ei:
            lat.synchronize()
        assert ei.value.status == lbm.LBM_ERR_TIMEOUT
        lat.set_wait_budget(1 << 31)
        lat.set_populations(f0, g0)
        lat.step(2)
        lat.synchronize()
        f, g = lat.populations()
    fo, go = oracle.run(p, f0, g0, 2)
    ef, eg = _rel_pop(f, g, fo, go)
    assert ef < 2e-6 and eg < 2e-6, (ef, eg)


def test_divergence_is_reported(lbm):
    """A state with |u| above the sound speed is flagged (host-side check of the
    diagnostic maxima; nothing faults)."""
    n = (8, 8, 8)
    with lbm.Lattice(*n, lbm.walls_side_heated(), Ra=1e4, Pr=0.71) as lat:
        u = np.zeros((3, 8, 8, 8))
        u[0, 4, 4, 4] = 0.9
        lat.set_fields(1.0, u, 0.0)
        lat.sample()
        with pytest.raises(lbm.LbmError) as ei:
            lat.diagnostics()
        assert ei.value.status == lbm.LBM_ERR_DIVERGED
        d = lat.diagnostics(raise_on_diverged=False)
        assert d["diverged"] and d["max_u"] > 0.5


@pytest.mark.parametrize("pipe", ["register", "staged"])
def test_injected_nan_is_reported(lbm, pipe):
    """A NaN planted on the host in one node's populations spreads through the
    steps without any fault and is reported: the next sample counts
    non-finite nodes and lbm_diagnostics returns LBM_ERR_DIVERGED."""
    n = (20, 18, 16)
    p = _orc_params(n, WALLS["side_heated"])
    f0, g0 = _random_state(p, 6)
    f0[3, 8, 9, 10] = np.nan
    with _lattice(lbm, n, WALLS["side_heated"], storage="fp16s", pipeline=pipe) as lat:
        lat.set_populations(f0, g0)
        lat.step(5)
        lat.sample()
        with pytest.raises(lbm.LbmError) as ei:
            lat.diagnostics()
        assert ei.value.status == lbm.LBM_ERR_DIVERGED
        d = lat.diagnostics(raise_on_diverged=False)
        assert d["diverged"] and d["nonfinite"] > 0


def _neighbourhood_reference(p, fields, centre, k):
    """Oracle populations at `centre` after k steps from the equilibrium of
    `fields`, computed on the (2k+1)^3 box around it (clipped to the lattice)."""
    rho, u, T = fields
    lo = [max(c - k, 0) for c in centre]
    hi = [min(c + k, n - 1) for c, n in zip(centre, (p.nx, p.ny, p.nz))]
    sl = (slice(lo[2], hi[2] + 1), slice(lo[1], hi[1] + 1), slice(lo[0], hi[0] + 1))
    box = (hi[2] - lo[2] + 1, hi[1] - lo[1] + 1, hi[0] - lo[0] + 1)
    bp = oracle.Params(box[2], box[1], box[0], p.walls, p.nu, p.kappa, p.gbeta, p.H, p.U)
    f, g = oracle.init_equilibrium(bp, rho[sl], u[(slice(None),) + sl], T[sl])
    for _ in range(k):
        f, g = oracle.step_box(p, lo, f, g)
    c = (centre[2] - lo[2], centre[1] - lo[1], centre[0] - lo[0])
    return f[(slice(None),) + c], g[(slice(None),) + c]


@pytest.mark.parametrize("storage,tol", [("fp32", 2e-6), ("fp16s", 4e-3), ("fp16m", 4e-3)])
def test_full_size_257_sampled(lbm, storage, tol):
    """257^3 side-heated cell, Ra=1e7, the benchmark's launch configuration:
    random smooth-free fields, one and two steps; 600 sampled nodes (walls,
    edges, corners and interior) against the oracle on their neighbourhoods."""
    N = 257
    p = oracle.cell(N, 1e7, 0.71, oracle.side_heated_walls())
    sh = (N, N, N)
    fields = inputs.random_fields(sh, 257, du=0.02)
    rng = np.random.default_rng(0)
    pts = [tuple(int(v) for v in rng.integers(0, N, 3)) for _ in range(400)]
    for c in (0, N - 1):
        pts += [(c, int(rng.integers(0, N)), int(rng.integers(0, N))) for _ in range(40)]
        pts += [(int(rng.integers(0, N)), c, c) for _ in range(20)]
    pts += [(0, 0, 0), (N - 1, N - 1, N - 1), (0, N - 1, 0), (N - 1, 0, N - 1)]
    nodes = np.array([x + N * (y + N * z) for x, y, z in pts], dtype=np.int64)
    with lbm.Lattice(N, N, N, lbm.walls_side_heated(), Ra=1e7, Pr=0.71, storage=storage) as lat:
        lat.set_fields(*fields)
        for k in (1, 2):
            lat.step(1)
            fg, gg = lat.populations_at(nodes)
            worst_f = worst_g = 0.0
            scale_f = scale_g = 0.0
            for j, c in enumerate(pts):
                fr, gr = _neighbourhood_reference(p, fields, c, k)
                worst_f = max(worst_f, np.abs(fg[j] - fr).max())
                worst_g = max(worst_g, np.abs(gg[j] - gr).max())
                scale_f = max(scale_f, np.abs(fr - W19).max())
                scale_g = max(scale_g, np.abs(gr).max())
            assert worst_f / scale_f < tol and worst_g / scale_g < tol, (k, worst_f / scale_f, worst_g / scale_g)


@pytest.mark.parametrize("storage", ["fp32", "fp16s"])
def test_upload_apply_fields_match_set_fields(lbm, storage):
    """lbm_upload_fields + lbm_apply_fields build the same state as
    lbm_set_fields, bit for bit, also when the next fields are uploaded on the
    copy stream while the steps from the previous ones run (the pipelined
    pattern of the end-to-end benchmark), on a side-heated and a
    Rayleigh-Benard cell;
    lbm_apply_fields with no pending upload is LBM_ERR_STATE and the pull
    scheme refuses uploads with LBM_ERR_PARAM."""
    n = (45, 37, 13)
    sh = (n[2], n[1], n[0])
    fields = [inputs.random_fields(sh, seed, du=0.02) for seed in (11, 12, 13)]
    import torch

    # pinned copies, so that the uploads run asynchronously
    pin = [tuple(torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy() for a in f) for f in fields]
    for walls in ("side_heated", "rayleigh_benard"):
        out = []
        with _lattice(lbm, n, WALLS[walls], storage=storage) as lat:
            for rho, u, T in fields:
                lat.set_fields(rho, u, T)
                lat.step(7)
            out.append(lat.populations())
        with _lattice(lbm, n, WALLS[walls], storage=storage) as lat:
            lat.upload_fields(*pin[0])
            for k in range(3):
                lat.apply_fields()
                lat.step(7)
                if k < 2:
                    lat.upload_fields(*pin[k + 1])  # beside the steps just queued
            out.append(lat.populations())
            with pytest.raises(lbm.LbmError) as ei:
                lat.apply_fields()
            assert ei.value.status == lbm.LBM_ERR_STATE
        for a, b in zip(out[0], out[1]):
            assert np.array_equal(a, b)
    with _lattice(lbm, n, WALLS["side_heated"], storage=storage, streaming="pull2") as lat:
        with pytest.raises(lbm.LbmError) as ei:
            lat.upload_fields(*fields[0])
        assert ei.value.status == lbm.LBM_ERR_PARAM
