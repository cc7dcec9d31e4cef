"""GPU parity of the Nusselt numbers of Sec. 3 beyond the wall averages and
of the Table 1 probes, against the FP64 oracle.

lbm_nusselt_profile (the plane-averaged Nu along an axis, Fig. 4, and the
mid-line wall Nu_mean, Table 2) is compared with oracle.nusselt_profile on
the same states: random states a few steps into their evolution, on odd and
even meshes (the mid-line interpolates between two node lines on an even
axis), for the side-heated, Rayleigh-Benard and mixed wall sets.  The GPU
sums FP32 node values in FP64; against FP64 node values that leaves about
1e-6 of the profile's scale, bounded here by 1e-5.
The centreline probes of Table 1 (drivers.centerline_probes) are computed
from the GPU's and from the oracle's moments of one state, on an odd and an
even mesh, and agree to the same bound."""
import numpy as np
import pytest

import oracle
from paper_1903_08882_gb300 import drivers, inputs

pytestmark = pytest.mark.gpu

A, D, P = 0, 1, 2
WALLS = {
    "side_heated": [(D, 0.5), (D, -0.5), (A, 0), (A, 0), (A, 0), (A, 0)],
    "rayleigh_benard": [(A, 0), (A, 0), (A, 0), (A, 0), (D, 0.5), (D, -0.5)],
    "mixed": [(A, 0), (A, 0), (D, 0.4), (D, 0.1), (P, 0), (P, 0)],
}


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


def _state(n, walls, seed):
    nx, ny, nz = n
    p = oracle.Params(nx, ny, nz, walls, 0.03, 0.02, 4e-3, float(nz), 0.1)
    rho, u, T = inputs.random_fields((nz, ny, nx), seed, du=0.03)
    f, g = oracle.init_equilibrium(p, rho, u, T)
    f, g = oracle.run(p, f, g, 5)
    return p, f, g


@pytest.mark.parametrize("walls", list(WALLS))
@pytest.mark.parametrize("n", [(9, 9, 9), (10, 12, 14), (33, 8, 11)])
def test_nusselt_profile_against_oracle(lbm, walls, n):
    p, f, g = _state(n, WALLS[walls], seed=sum(n))
    with lbm.Lattice(*n, WALLS[walls], nu=p.nu, kappa=p.kappa, gbeta=p.gbeta, U=p.U) as lat:
        lat.set_populations(f, g)
        for axis in range(3):
            prof, mid = lat.nusselt_profile(axis)
            oprof, omid = oracle.nusselt_profile(p, f, g, axis)
            scale = max(np.abs(oprof).max(), 1.0)
            assert np.abs(prof - oprof).max() <= 1e-5 * scale, (axis, prof - oprof)
            assert np.abs(mid - omid).max() <= 1e-5 * max(np.abs(omid).max(), 1.0), (mid, omid)
            assert ((omid == 0) == (mid == 0)).all()


@pytest.mark.parametrize("N", [33, 32])
def test_centerline_probes_against_oracle(lbm, N):
    """Side-heated cell at Ra = 1e4 (the 33^3 benchmark case and an even
    32^3 mesh), the oracle's state after 300 steps from rest: the Table 1
    probes from the GPU's moments of that state and from the oracle's."""
    p = oracle.cell(N, 1e4, 0.71, oracle.side_heated_walls())
    f, g = oracle.init_equilibrium(p, 1.0, np.zeros(3), 0.0)
    f, g = oracle.run(p, f, g, 300)
    with lbm.Lattice(N, N, N, lbm.walls_side_heated(), Ra=1e4, Pr=0.71) as lat:
        lat.set_populations(f, g)
        _, u3, _ = lat.moments()
    _, ou3, _ = oracle.moments(p, f, g)
    got, want = drivers.centerline_probes(u3, 0.1), drivers.centerline_probes(ou3, 0.1)
    # the flow is centro-symmetric: each extreme is attained twice (z and 1 - z,
    # x and 1 - x, opposite signs) to within rounding, so either may be reported
    assert min(abs(got["z"] - want["z"]), abs(got["z"] - (1 - want["z"]))) < 1e-12
    assert min(abs(got["x"] - want["x"]), abs(got["x"] - (1 - want["x"]))) < 1e-12
    assert abs(abs(got["u_max"]) - abs(want["u_max"])) <= 1e-5 * abs(want["u_max"])
    assert abs(abs(got["w_max"]) - abs(want["w_max"])) <= 1e-5 * abs(want["w_max"])
    # the whole centrelines agree point by point
    for a, (sl) in ((0, (slice(None), N // 2, N // 2)), (2, (N // 2, N // 2, slice(None)))):
        if N % 2:
            assert np.abs(u3[a][sl] - ou3[a][sl]).max() <= 1e-5 * np.abs(ou3[a][sl]).max()
