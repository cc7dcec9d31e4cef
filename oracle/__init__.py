"""FP64 CPU oracle for the thermal lattice Boltzmann step (arXiv:1903.08882).

TEST INFRASTRUCTURE ONLY.  The test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only code allowed to import this
package.  The product path (the CUDA library and its binding) never does.

The arithmetic lives in ``lbm_oracle.c`` (plain C, FP64, two buffers, pull
streaming), written from the paper's equations:
  * D3Q19 MRT with Guo forcing and half-way bounce-back (Sec. 2.2, Eq. MRT),
  * D3Q7 MRT with the fourth-order-isotropic rates, anti-bounce-back Dirichlet
    and bounce-back adiabatic walls (Sec. 2.3, Eq. MRT_T, Eq. magic/4th/qk/qnu),
  * the diagnostics of Sec. 3 (E, rms density and divergence, wall Nusselt
    numbers) and Sec. 4 (Re^rms, Re_w^rms, Nu_vol, Nu_wall, Nu_kin, Nu_th),
  * the per-node dissipation rates eps_u and eps_T whose PDFs Sec. 4 reports.
This module only marshals numpy arrays to it and turns raw sums into the
paper's dimensionless numbers (free-fall units, dT = 1).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB = os.path.join(_HERE, "liborc.so")

ADIABATIC, DIRICHLET, PERIODIC = 0, 1, 2
NDIAG = 24


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP over z-slabs of the lattice)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("wall_kind", ctypes.c_int * 6), ("wall_T", ctypes.c_double * 6),
        ("nu", ctypes.c_double), ("kappa", ctypes.c_double), ("gbeta", ctypes.c_double),
        ("body_force", ctypes.c_double * 3),
        ("rho0", ctypes.c_double), ("T0", ctypes.c_double),
        ("a_T", ctypes.c_double),
        ("s", ctypes.c_double * 19), ("q", ctypes.c_double * 7),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        d, i64, ip = ctypes.POINTER(ctypes.c_double), ctypes.c_int64, ctypes.POINTER(ctypes.c_int)
        P = ctypes.POINTER(_Params)
        _lib.orc_set_rates.argtypes = [P]
        _lib.orc_set_rates.restype = ctypes.c_int
        _lib.orc_free_fall.argtypes = [ctypes.c_double] * 4 + [d, d, d]
        _lib.orc_tables.argtypes = [d, d, d, d, ip, d, d, d, ip]
        _lib.orc_collide.argtypes = [P, d, d, d, d, d]
        _lib.orc_equilibrium.argtypes = [P, ctypes.c_double, d, ctypes.c_double, d, d]
        _lib.orc_meq.argtypes = [ctypes.c_double, d, d]
        _lib.orc_mf.argtypes = [d, d, d]
        _lib.orc_init_equilibrium.argtypes = [P, d, d, d, d, d]
        _lib.orc_moments.argtypes = [P, d, d, d, d, d]
        _lib.orc_step_box.argtypes = [P, ip, ip, d, d, d, d]
        _lib.orc_run.argtypes = [P, d, d, i64]
        _lib.orc_diagnostics.argtypes = [P, d, d, d]
        _lib.orc_local_dissipation.argtypes = [P, d, d, d, d]
        _lib.orc_nusselt_profile.argtypes = [P, d, d, ctypes.c_int, ctypes.c_double, d]
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


@dataclass
class Params:
    """Lattice, walls and transport coefficients of one cell (lattice units).

    walls: six (kind, T_w) pairs for faces -x, +x, -y, +y, -z, +z.
    H, U: length and velocity scales of the free-fall units (Sec. 2.1).
    """
    nx: int
    ny: int
    nz: int
    walls: list
    nu: float
    kappa: float
    gbeta: float
    H: float
    U: float
    body_force: tuple = (0.0, 0.0, 0.0)
    rho0: float = 1.0
    T0: float = 0.0
    s: np.ndarray | None = None  # override of the D3Q19 rates (tests)
    q: np.ndarray | None = None  # override of the D3Q7 rates (tests)
    a_T_override: float | None = None
    _c: _Params = field(default=None, repr=False)

    def __post_init__(self):
        c = _Params()
        c.nx, c.ny, c.nz = self.nx, self.ny, self.nz
        for k, (kind, tw) in enumerate(self.walls):
            c.wall_kind[k] = int(kind)
            c.wall_T[k] = float(tw)
        c.nu, c.kappa, c.gbeta = self.nu, self.kappa, self.gbeta
        for a in range(3):
            c.body_force[a] = self.body_force[a]
        c.rho0, c.T0 = self.rho0, self.T0
        self.valid = lib().orc_set_rates(ctypes.byref(c)) == 0
        if self.s is not None:
            for k in range(19):
                c.s[k] = float(self.s[k])
        if self.q is not None:
            for k in range(7):
                c.q[k] = float(self.q[k])
        if self.a_T_override is not None:
            c.a_T = float(self.a_T_override)
        self._c = c

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def a_T(self) -> float:
        return self._c.a_T

    @property
    def rates(self):
        return np.array(self._c.s[:]), np.array(self._c.q[:])

    @property
    def tau(self) -> float:
        return 3.0 * self.nu + 0.5

    def ref(self):
        return ctypes.byref(self._c)


def free_fall(H: float, Ra: float, Pr: float, U: float = 0.1):
    """nu, kappa, g beta of the free-fall scaling (Sec. 2.1, dT = 1)."""
    nu, ka, gb = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    lib().orc_free_fall(H, Ra, Pr, U, ctypes.byref(nu), ctypes.byref(ka), ctypes.byref(gb))
    return nu.value, ka.value, gb.value


def cell(n, Ra, Pr, walls, U=0.1, H=None, body_force=(0.0, 0.0, 0.0)) -> Params:
    """A cubic-or-box cell in free-fall units; H defaults to nz."""
    nx, ny, nz = (n, n, n) if np.isscalar(n) else n
    H = float(nz if H is None else H)
    nu, kappa, gbeta = free_fall(H, Ra, Pr, U)
    return Params(nx, ny, nz, walls, nu, kappa, gbeta, H, U, body_force)


def side_heated_walls():
    """Hot -x (T=+1/2), cold +x (T=-1/2), the other four faces adiabatic."""
    return [(DIRICHLET, 0.5), (DIRICHLET, -0.5), (ADIABATIC, 0.0), (ADIABATIC, 0.0),
            (ADIABATIC, 0.0), (ADIABATIC, 0.0)]


def rayleigh_benard_walls():
    """Hot bottom -z (T=+1/2), cold top +z (T=-1/2), four adiabatic sidewalls."""
    return [(ADIABATIC, 0.0), (ADIABATIC, 0.0), (ADIABATIC, 0.0), (ADIABATIC, 0.0),
            (DIRICHLET, 0.5), (DIRICHLET, -0.5)]


def tables():
    e19, w19, m, minv = np.zeros(57), np.zeros(19), np.zeros(361), np.zeros(361)
    e7, n7, ninv = np.zeros(21), np.zeros(49), np.zeros(49)
    opp19, p19 = _ip(np.zeros(19))
    opp7, p7 = _ip(np.zeros(7))
    lib().orc_tables(_dp(e19), _dp(w19), _dp(m), _dp(minv), p19, _dp(e7), _dp(n7), _dp(ninv), p7)
    return dict(e19=e19.reshape(19, 3).astype(int), w19=w19, M=m.reshape(19, 19),
                Minv=minv.reshape(19, 19), opp19=opp19.copy(), e7=e7.reshape(7, 3).astype(int),
                N=n7.reshape(7, 7), Ninv=ninv.reshape(7, 7), opp7=opp7.copy())


def collide(p: Params, f, g):
    """Post-collision populations of one node, plus (rho, u, v, w, T)."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    fo, go, mom = np.zeros(19), np.zeros(7), np.zeros(5)
    lib().orc_collide(p.ref(), _dp(f), _dp(g), _dp(fo), _dp(go), _dp(mom))
    return fo, go, mom


def equilibrium(p: Params, rho, u, T):
    u = np.ascontiguousarray(u, dtype=np.float64)
    fe, ge = np.zeros(19), np.zeros(7)
    lib().orc_equilibrium(p.ref(), float(rho), _dp(u), float(T), _dp(fe), _dp(ge))
    return fe, ge


def meq(rho, u):
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros(19)
    lib().orc_meq(float(rho), _dp(u), _dp(out))
    return out


def mf(u, F):
    u = np.ascontiguousarray(u, dtype=np.float64)
    F = np.ascontiguousarray(F, dtype=np.float64)
    out = np.zeros(19)
    lib().orc_mf(_dp(u), _dp(F), _dp(out))
    return out


def init_equilibrium(p: Params, rho, u3, T):
    """Equilibrium populations f (19,nz,ny,nx), g (7,nz,ny,nx) from fields."""
    sh = (p.nz, p.ny, p.nx)
    rho = np.ascontiguousarray(np.broadcast_to(rho, sh), dtype=np.float64)
    u3 = np.asarray(u3, dtype=np.float64)
    if u3.ndim == 1:
        u3 = u3.reshape(3, 1, 1, 1)
    u3 = np.ascontiguousarray(np.broadcast_to(u3, (3,) + sh), dtype=np.float64)
    T = np.ascontiguousarray(np.broadcast_to(T, sh), dtype=np.float64)
    f, g = np.zeros((19,) + sh), np.zeros((7,) + sh)
    lib().orc_init_equilibrium(p.ref(), _dp(rho), _dp(u3), _dp(T), _dp(f), _dp(g))
    return f, g


def moments(p: Params, f, g):
    """rho (nz,ny,nx), u (3,nz,ny,nx), T (nz,ny,nx) of pre-collision populations."""
    sh = (p.nz, p.ny, p.nx)
    f = np.ascontiguousarray(f, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    rho, u3, T = np.zeros(sh), np.zeros((3,) + sh), np.zeros(sh)
    lib().orc_moments(p.ref(), _dp(f), _dp(g), _dp(rho), _dp(u3), _dp(T))
    return rho, u3, T


def step_box(p: Params, org, f, g):
    """One step on a box of the lattice starting at global node org (x, y, z).

    f: (19, bz, by, bx), g: (7, bz, by, bx).  Nodes whose result needs data
    outside the box come back as NaN."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    dim = (f.shape[3], f.shape[2], f.shape[1])
    o, po = _ip(org)
    dd, pd = _ip(dim)
    fo, go = np.empty_like(f), np.empty_like(g)
    lib().orc_step_box(p.ref(), po, pd, _dp(f), _dp(g), _dp(fo), _dp(go))
    return fo, go


def run(p: Params, f, g, nsteps: int):
    """nsteps whole-lattice steps; returns new arrays."""
    f = np.array(f, dtype=np.float64, order="C", copy=True)
    g = np.array(g, dtype=np.float64, order="C", copy=True)
    lib().orc_run(p.ref(), _dp(f), _dp(g), int(nsteps))
    return f, g


def raw_diagnostics(p: Params, f, g):
    f = np.ascontiguousarray(f, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    out = np.zeros(NDIAG)
    lib().orc_diagnostics(p.ref(), _dp(f), _dp(g), _dp(out))
    return out


def local_dissipation(p: Params, f, g):
    """Per-node dissipation rates eps_u = nu/2 sum_ij (d_i u_j + d_j u_i)^2 and
    eps_T = kappa |grad T|^2 (Sec. 4), each (nz, ny, nx), same stencils as the
    global diagnostics."""
    sh = (p.nz, p.ny, p.nx)
    f = np.ascontiguousarray(f, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    eu, et = np.zeros(sh), np.zeros(sh)
    lib().orc_local_dissipation(p.ref(), _dp(f), _dp(g), _dp(eu), _dp(et))
    return eu, et


def nusselt_profile(p: Params, f, g, axis: int = 0):
    """Plane-averaged Nusselt number along `axis` (Sec. 3, Nu(y) of Fig. 4:
    the mean over each node plane of u_a T H / kappa - H dT/dx_a) and the
    mid-line Nusselt numbers of the six faces (Sec. 3, Nu_mean of Table 2;
    0 for faces that are not Dirichlet walls).  Returns (profile, nu_mid)."""
    na = (p.nx, p.ny, p.nz)[axis]
    f = np.ascontiguousarray(f, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    out = np.zeros(na + 6)
    lib().orc_nusselt_profile(p.ref(), _dp(f), _dp(g), int(axis), float(p.H), _dp(out))
    return out[:na], out[na:]


def diagnostics(p: Params, f, g) -> dict:
    """The paper's global quantities of one state (free-fall units, dT = 1).

    E (Sec. 3), rms density fluctuation and rms divergence (Sec. 3, Table 3),
    Re^rms and Re_w^rms, Nu_vol, Nu_kin, Nu_th (Sec. 4), and per Dirichlet face
    the wall Nusselt number -H <dT/dn> (Sec. 3 Nu_overall, Sec. 4 Nu_wall) and
    its link-flux counterpart <q_link> H / kappa."""
    r = raw_diagnostics(p, f, g)
    return finalize(p, r)


def finalize(p: Params, r) -> dict:
    n = r[0]
    H, U, nu, ka = p.H, p.U, p.nu, p.kappa
    area = [p.ny * p.nz, p.ny * p.nz, p.nx * p.nz, p.nx * p.nz, p.nx * p.ny, p.nx * p.ny]
    out = dict(
        rms_drho=np.sqrt(r[1] / n),
        E=0.5 * r[2] / n / U**2,
        Re_rms=np.sqrt(r[2] / n) * H / nu,
        Re_w=np.sqrt(r[3] / n) * H / nu,
        Nu_vol=1.0 + r[4] / n * H / ka,
        Nu_kin=1.0 + nu * r[5] / n * H**2 / (ka * U**2),
        Nu_th=r[6] / n * H**2,
        rms_div=np.sqrt(r[7] / n) * H / U,
        mean_T=r[14] / n,
        mass=r[15],
        max_u=r[16],
        nonfinite=r[17],
    )
    out["Nu_face"] = np.array([H * r[8 + k] / area[k] for k in range(6)])
    out["Nu_face_link"] = np.array([r[18 + k] / area[k] * H / ka for k in range(6)])
    return out
