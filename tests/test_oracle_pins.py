"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Nothing here compares the oracle with itself: each test checks it against a
printed table, an algebraic identity the paper states, a textbook special
case written independently in velocity space, a closed-form solution, an
exact invariant or an exact symmetry.
"""
import os

import numpy as np
import pytest

from paper_1903_08882_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
SQ3 = np.sqrt(3.0)


def _load(name):
    return np.loadtxt(os.path.join(GOLDEN, name), comments="#").astype(int)


def _walls(kinds, temps=(0, 0, 0, 0, 0, 0)):
    return list(zip(kinds, temps))


A, D, P = 0, 1, 2


# ------------------------------------------------------------------ tables --

def test_M_equals_printed_matrix(orc):
    """M built from the moment polynomials equals the matrix printed in Sec. 2.2."""
    t = orc.tables()
    assert np.array_equal(t["M"].astype(int), _load("paper_M.txt"))
    assert np.allclose(t["M"], np.rint(t["M"]), atol=0)


def test_M_orthogonal_with_known_norms(orc):
    t = orc.tables()
    G = t["M"] @ t["M"].T
    norms = [19, 2394, 252, 10, 40, 10, 40, 10, 40, 36, 72, 12, 24, 4, 4, 4, 8, 8, 8]
    assert np.allclose(G, np.diag(norms), atol=1e-12)
    assert np.allclose(t["Minv"] @ t["M"], np.eye(19), atol=1e-13)


def test_N_printed_except_ez_row(orc):
    """N from its definitions equals the printed N of Sec. 2.3 in every row but
    <e_z|, whose printed entries (..., -1, -1) contradict e_5 = +z, e_6 = -z."""
    t = orc.tables()
    printed = _load("paper_N.txt")
    N = t["N"].astype(int)
    for k in range(7):
        if k == 3:
            continue
        assert np.array_equal(N[k], printed[k])
    assert np.array_equal(N[3], [0, 0, 0, 0, 0, 1, -1])
    assert not np.array_equal(printed[3], N[3])
    assert np.allclose(t["N"] @ t["N"].T, np.diag([7, 2, 2, 2, 42, 12, 4]), atol=1e-13)


def test_velocity_sets_and_opposites(orc):
    t = orc.tables()
    e19, e7 = t["e19"], t["e7"]
    assert e19.shape == (19, 3) and len({tuple(v) for v in e19}) == 19
    assert sorted((v @ v) for v in e19) == [0] + [1] * 6 + [2] * 12
    for i in range(19):
        assert np.array_equal(e19[t["opp19"][i]], -e19[i])
    for i in range(7):
        assert np.array_equal(e7[t["opp7"][i]], -e7[i])
    # weights: isotropy up to fourth order with c_s^2 = 1/3
    w = t["w19"]
    assert abs(w.sum() - 1) < 1e-15
    assert np.allclose(np.einsum("i,ia,ib->ab", w, e19, e19), np.eye(3) / 3, atol=1e-15)
    fourth = np.einsum("i,ia,ib,ic,id->abcd", w, e19, e19, e19, e19)
    d = np.eye(3)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
           + np.einsum("ad,bc->abcd", d, d)) / 9
    assert np.allclose(fourth, iso, atol=1e-15)


def test_meq_is_M_times_feq(orc):
    """The printed m^eq (Sec. 2.2) equals M f^eq of the printed f^eq."""
    t = orc.tables()
    p = orc.Params(4, 4, 4, _walls([A] * 6), 0.05, 0.02, 0.0, 4, 0.1)
    rng = np.random.default_rng(1)
    for _ in range(20):
        rho = 1 + 0.1 * rng.standard_normal()
        u = 0.1 * rng.standard_normal(3)
        feq, _ = orc.equilibrium(p, rho, u, 0.3)
        assert np.allclose(t["M"] @ feq, orc.meq(rho, u), atol=1e-14)


def test_MF_is_M_times_guo_force(orc):
    """The printed M F~ (Sec. 2.2) equals M applied to Guo's forcing
    F~_i = w_i [(e_i - u)/cs^2 + (e_i.u) e_i/cs^4] . F."""
    t = orc.tables()
    e, w = t["e19"].astype(float), t["w19"]
    rng = np.random.default_rng(2)
    for _ in range(20):
        u, F = 0.1 * rng.standard_normal(3), 1e-3 * rng.standard_normal(3)
        Ft = w * (3 * (e - u) @ F + 9 * (e @ u) * (e @ F))
        assert np.allclose(t["M"] @ Ft, orc.mf(u, F), atol=1e-17)


def test_neq_is_N_times_geq(orc):
    t = orc.tables()
    for kappa in (0.002, 0.03, 0.09):
        p = orc.Params(4, 4, 4, _walls([A] * 6), 0.05, kappa, 0.0, 4, 0.1)
        aT = p.a_T
        rng = np.random.default_rng(3)
        u, T = 0.1 * rng.standard_normal(3), rng.standard_normal()
        _, geq = orc.equilibrium(p, 1.0, u, T)
        assert np.allclose(t["N"] @ geq, [T, u[0] * T, u[1] * T, u[2] * T, aT * T, 0, 0], atol=1e-15)
        # weights: 2 w_1 equals the anti-bounce-back factor (6 + a_T)/21
        _, g1 = orc.equilibrium(p, 1.0, np.zeros(3), 1.0)
        assert abs(2 * g1[1] - (6 + aT) / 21) < 1e-16
        assert abs(g1.sum() - 1) < 1e-15


# ------------------------------------------------------------------ rates --

def test_flow_rates_and_magic_product(orc):
    for nu in (0.0068, 0.0278, 0.1, 0.5):
        p = orc.Params(4, 4, 4, _walls([A] * 6), nu, 0.01, 0.0, 4, 0.1)
        s, _ = p.rates
        tau = 3 * nu + 0.5
        assert np.allclose(s[[0, 3, 5, 7]], 0)
        assert np.allclose(s[[1, 2, 9, 10, 11, 12, 13, 14, 15]], 1 / tau)
        assert np.allclose(s[[4, 6, 8, 16, 17, 18]], 8 * (2 * tau - 1) / (8 * tau - 1))
        # TRT "magic" combination of the flow rates is 3/16 for every tau_f
        assert abs((1 / s[1] - 0.5) * (1 / s[4] - 0.5) - 3 / 16) < 1e-13


def test_thermal_rates_fourth_order(orc):
    """q_k = 3 - sqrt3, q_e = q_nu = 4 sqrt3 - 6, a_T = 42 sqrt3 kappa - 6
    satisfy Eq. magic and Eq. 4th for every a_T, and kappa is recovered."""
    for kappa in (0.0024, 0.0096, 0.039, 0.08):
        p = orc.Params(4, 4, 4, _walls([A] * 6), 0.02, kappa, 0.0, 4, 0.1)
        _, q = p.rates
        qk, qe, qn, aT = q[1], q[4], q[5], p.a_T
        assert q[0] == 0 and q[1] == q[2] == q[3] and q[5] == q[6]
        assert abs((1 / qk - 0.5) * (1 / qe - 0.5) - 1 / 6) < 1e-14
        lhs = 1 / qn - 0.5
        rhs = (aT + 6) / (1 - aT) * (1 / qk - 0.5) - (4 + 3 * aT) / (12 * (1 - aT)) / (1 / qk - 0.5)
        assert abs(lhs - rhs) < 1e-12
        qnu_qk = 6 * (1 - aT) * (2 - qk) * qk / ((11 + 3 * aT) * (qk - 6) * qk + 12 * (aT + 6))
        assert abs(qnu_qk - qn) < 1e-12
        assert abs((6 + aT) / 21 * (1 / qk - 0.5) - kappa) < 1e-15


def test_rate_validation(orc):
    assert not orc.Params(4, 4, 4, _walls([A] * 6), 0.02, 0.2, 0.0, 4, 0.1).valid  # a_T > 1
    assert not orc.Params(4, 4, 4, _walls([A] * 6), -0.01, 0.02, 0.0, 4, 0.1).valid  # tau <= 1/2
    assert orc.Params(4, 4, 4, _walls([A] * 6), 0.02, 0.02, 0.0, 4, 0.1).valid


# ------------------------------------------------------- collision forms --

def _rand_node(rng, p, orc):
    rho = 1 + 0.01 * rng.standard_normal()
    u = 0.05 * rng.standard_normal(3)
    T = 0.4 * rng.standard_normal()
    feq, geq = orc.equilibrium(p, rho, u, T)
    return feq + 1e-3 * rng.standard_normal(19) / 19, geq + 1e-2 * rng.standard_normal(7) / 7


def _guo(t, u, F):
    e, w = t["e19"].astype(float), t["w19"]
    return w * (3 * (e - u) @ F + 9 * (e @ u) * (e @ F))


@pytest.mark.parametrize("H,Ra,Pr,U", [(33, 1e4, 0.71, 0.1), (257, 1e7, 0.71, 0.1 / SQ3), (64, 1e6, 7.0, 0.05)])
def test_free_fall_scaling_definitions(orc, H, Ra, Pr, U):
    """Sec. 2.1: with dT = 1 the free-fall velocity is U = sqrt(g beta dT H),
    Ra = g beta dT H^3 / (nu kappa) and Pr = nu / kappa; the oracle's nu,
    kappa and g beta must give these back."""
    nu, ka, gb = orc.free_fall(H, Ra, Pr, U)
    assert np.sqrt(gb * H) == pytest.approx(U, rel=1e-14)
    assert gb * H**3 / (nu * ka) == pytest.approx(Ra, rel=1e-13)
    assert nu / ka == pytest.approx(Pr, rel=1e-14)


def test_bgk_limit(orc):
    """With every rate equal to 1/tau the MRT collision is BGK with Guo
    forcing: f+ = f - (f - f^eq)/tau + (1 - 1/(2 tau)) F~ (velocity space)."""
    t = orc.tables()
    rng = np.random.default_rng(4)
    tau, qq = 0.73, 1.21
    p = orc.Params(4, 4, 4, _walls([A] * 6), 0.02, 0.03, 2e-3, 4, 0.1,
                   body_force=(1e-4, -2e-4, 3e-5), s=np.full(19, 1 / tau), q=np.full(7, qq))
    for _ in range(10):
        f, g = _rand_node(rng, p, orc)
        fo, go, mom = orc.collide(p, f, g)
        rho, T = f.sum(), g.sum()
        F = np.array([1e-4, -2e-4, 3e-5 + rho * 2e-3 * T])
        u = (t["e19"].T @ f + F / 2) / rho
        feq, geq = orc.equilibrium(p, rho, u, T)
        assert np.allclose(mom, [rho, *u, T], atol=1e-15)
        assert np.allclose(fo, f - (f - feq) / tau + (1 - 0.5 / tau) * _guo(t, u, F), atol=1e-15)
        assert np.allclose(go, g - qq * (g - geq), atol=1e-15)


def test_trt_form_with_paper_rates(orc):
    """With the paper's rates the D3Q19 MRT collision equals a two-relaxation-
    time collision (w+ = 1/tau_f on symmetric parts, w- = s_q on antisymmetric
    parts, Guo forcing split alike), and the D3Q7 one equals TRT with w+ = q_e,
    w- = q_kappa.  Written here in velocity space."""
    t = orc.tables()
    o19, o7 = t["opp19"], t["opp7"]
    rng = np.random.default_rng(5)
    for nu, kappa in ((0.0278, 0.039), (0.0068, 0.0096), (0.2, 0.06)):
        p = orc.Params(4, 4, 4, _walls([A] * 6), nu, kappa, 3e-4, 4, 0.1, body_force=(2e-5, 0, -1e-5))
        s, q = p.rates
        wp, wm = s[1], s[4]
        for _ in range(5):
            f, g = _rand_node(rng, p, orc)
            fo, go, _ = orc.collide(p, f, g)
            rho, T = f.sum(), g.sum()
            F = np.array([2e-5, 0, -1e-5 + rho * 3e-4 * T])
            u = (t["e19"].T @ f + F / 2) / rho
            feq, geq = orc.equilibrium(p, rho, u, T)
            Ft = _guo(t, u, F)
            sym = lambda a: 0.5 * (a + a[o19])
            asy = lambda a: 0.5 * (a - a[o19])
            ref = (f - wp * sym(f - feq) - wm * asy(f - feq)
                   + (1 - wp / 2) * sym(Ft) + (1 - wm / 2) * asy(Ft))
            assert np.allclose(fo, ref, atol=2e-16 * 50)
            sym7 = lambda a: 0.5 * (a + a[o7])
            asy7 = lambda a: 0.5 * (a - a[o7])
            ref7 = g - q[4] * sym7(g - geq) - q[1] * asy7(g - geq)
            assert np.allclose(go, ref7, atol=1e-15)


# ---------------------------------------------------------- lattice runs --

def _state(orc, p, seed, noise_f=1e-4, noise_g=1e-3, du=0.03):
    sh = (p.nz, p.ny, p.nx)
    rho, u, T = inputs.random_fields(sh, seed, du=du)
    f, g = orc.init_equilibrium(p, rho, u, T)
    f = f + inputs.noise(f.shape, seed, 20, noise_f)
    g = g + inputs.noise(g.shape, seed, 21, noise_g)
    return f, g


def test_rest_state_is_preserved(orc):
    """T = 0 everywhere, walls at T_w = 0: the rest equilibrium is a fixed point."""
    walls = _walls([A, D, A, D, D, A], (0, 0, 0, 0, 0, 0))
    p = orc.Params(6, 5, 7, walls, 0.03, 0.02, 3e-4, 7, 0.1)
    f, g = orc.init_equilibrium(p, 1.0, np.zeros(3), 0.0)
    f1, g1 = orc.run(p, f, g, 50)
    assert np.abs(f1 - f).max() < 1e-15
    assert np.abs(g1).max() == 0.0


def test_mass_and_heat_conservation(orc):
    """Bounce-back returns every population: sum f is exact; with every face
    adiabatic sum g is exact too (s_rho = 0 and q_0 = 0)."""
    p = orc.Params(8, 7, 6, _walls([A] * 6), 0.03, 0.02, 5e-3, 6, 0.1, body_force=(1e-4, 0, 0))
    f, g = _state(orc, p, 7)
    m0, h0 = f.sum(), g.sum()
    f1, g1 = orc.run(p, f, g, 300)
    assert abs(f1.sum() - m0) / m0 < 1e-13
    assert abs(g1.sum() - h0) / abs(h0) < 1e-12
    assert np.isfinite(f1).all() and np.abs(f1 - f).max() > 1e-6  # it did move


def test_conduction_linear_profile_and_unit_nusselt(orc):
    """Hot bottom / cold top, periodic sides, no buoyancy: the steady state is
    the linear profile T = 1/2 - (k + 1/2)/N and every Nusselt number is 1."""
    N = 16
    walls = _walls([P, P, P, P, D, D], (0, 0, 0, 0, 0.5, -0.5))
    p = orc.Params(3, 3, N, walls, 0.05, 0.05, 0.0, N, 0.1)
    f, g = orc.init_equilibrium(p, 1.0, np.zeros(3), 0.0)
    f, g = orc.run(p, f, g, 16000)
    _, u, T = orc.moments(p, f, g)
    exact = 0.5 - (np.arange(N) + 0.5) / N
    assert np.abs(T - exact[:, None, None]).max() < 1e-10
    d = orc.diagnostics(p, f, g)
    assert abs(d["Nu_face"][4] - 1) < 1e-9 and abs(-d["Nu_face"][5] - 1) < 1e-9
    assert abs(d["Nu_face_link"][4] - 1) < 1e-9 and abs(-d["Nu_face_link"][5] - 1) < 1e-9
    assert abs(d["Nu_th"] - 1) < 1e-9
    assert abs(d["Nu_vol"] - 1) < 1e-12


def test_conduction_below_onset_with_buoyancy(orc):
    """Ra = 1000 < 1708: with buoyancy on, the conduction state stays (Nu = 1).

    The scheme keeps a small staggered (odd-even in z) velocity in the
    hydrostatic state, linear in g beta (about 4e-3 g beta here), so Nu is 1
    only to O(1e-5) instead of round-off."""
    N = 16
    walls = _walls([P, P, P, P, D, D], (0, 0, 0, 0, 0.5, -0.5))
    nu = kappa = 0.05
    gbeta = 1000 * nu * kappa / N**3
    p = orc.Params(3, 3, N, walls, nu, kappa, gbeta, N, 0.1)
    f, g = orc.init_equilibrium(p, 1.0, np.zeros(3), 0.0)
    f, g = orc.run(p, f, g, 16000)
    d = orc.diagnostics(p, f, g)
    assert abs(d["Nu_face"][4] - 1) < 1e-4
    assert d["max_u"] < 1e-2 * gbeta
    rho, u, T = orc.moments(p, f, g)
    # hydrostatic density: densest where the upward buoyancy changes sign
    prof = rho[:, 1, 1]
    assert prof.argmax() in (N // 2 - 1, N // 2) and abs(prof.sum() - N) < 1e-12


def _neutral_rayleigh(a):
    """Rayleigh number at which a roll of wavenumber a (in units of 1/H) is
    neutrally stable in a layer between rigid isothermal plates (the classical
    linear stability problem of Rayleigh-Benard convection): (D^2 - a^2)^3 W =
    -Ra a^2 W on |z| < 1/2 with W = DW = (D^2 - a^2)^2 W = 0 at the plates.
    The even solution is a sum of cosh(q_k z) with q_k^2 - a^2 the three cube
    roots of -Ra a^2; the plate conditions give a 3x3 determinant, purely
    imaginary for real Ra, whose zero is found by bisection."""
    from scipy.optimize import brentq

    def det(Ra):
        r = (Ra * a * a) ** (1.0 / 3.0)
        taus = [-r, r * np.exp(1j * np.pi / 3), r * np.exp(-1j * np.pi / 3)]
        q = [np.sqrt(a * a + t + 0j) for t in taus]
        M = np.array([[np.cosh(qk / 2) for qk in q],
                      [qk * np.sinh(qk / 2) for qk in q],
                      [t * t * np.cosh(qk / 2) for t, qk in zip(taus, q)]])
        return np.linalg.det(M).imag

    return brentq(det, 1000.0, 3000.0, xtol=1e-9)


def test_neutral_rayleigh_textbook_minimum():
    """The stability solver above reproduces the textbook critical point of
    rigid-rigid Rayleigh-Benard convection, Ra_c = 1707.76 at a_c = 3.117."""
    from scipy.optimize import minimize_scalar

    res = minimize_scalar(_neutral_rayleigh, bounds=(2.5, 3.8), method="bounded", options={"xatol": 1e-7})
    assert abs(res.fun - 1707.76) < 0.01 and abs(res.x - 3.117) < 2e-3, res


def _onset_rayleigh(orc, H, Pr, nu, ras=(1680.0, 1740.0)):
    """Rayleigh number where the oracle's convection roll in a 2H x 3 x H box
    (x, y periodic, plates at z = 0 and H held at +-1/2) neither grows nor
    decays: the growth rate of the roll's vertical velocity, projected on
    cos(2 pi x / 2H) so that the scheme's x-independent hydrostatic velocity
    drops out, measured at two Rayleigh numbers and interpolated to zero."""
    kappa = nu / Pr
    nx = 2 * H
    walls = _walls([P, P, P, P, D, D], (0, 0, 0, 0, 0.5, -0.5))
    z = (np.arange(H) + 0.5) / H
    cx = np.cos(2 * np.pi * (np.arange(nx) + 0.5) / nx)
    td = H * H / kappa  # diffusive time in steps
    chunk = int(td / 8)
    rates = []
    for Ra in ras:
        p = orc.Params(nx, 3, H, walls, nu, kappa, Ra * nu * kappa / H**3, H, 0.1)
        T = (0.5 - z)[:, None, None] + 1e-4 * np.sin(np.pi * z)[:, None, None] * cx[None, None, :] * np.ones((H, 3, nx))
        f, g = orc.init_equilibrium(p, 1.0, np.zeros((3, H, 3, nx)), T)
        t, amp = [], []
        for k in range(24):  # three diffusive times; the faster modes are gone after the first
            f, g = orc.run(p, f, g, chunk)
            u = orc.moments(p, f, g)[1]
            t.append((k + 1) * chunk / td)
            amp.append(abs((u[2][:, 1, :] * cx[None, :]).sum()))
        t, la = np.array(t), np.log(np.array(amp))
        rates.append(np.polyfit(t[t > 1.0], la[t > 1.0], 1)[0])
    assert rates[0] < 0 < rates[1], rates
    return ras[0] - rates[0] * (ras[1] - ras[0]) / (rates[1] - rates[0])


def test_convection_onset_at_the_critical_rayleigh_number(orc):
    """Buoyancy (Sec. 2.2), the Dirichlet plates and both collisions together:
    the oracle's roll of wavelength 2H sets in at the exact neutral Rayleigh
    number of that wavenumber (a = pi: 1707.92), independently of Pr, with an
    error that falls with the mesh at about second order (measured: 0.49% at
    H = 8 and 0.18% at H = 12 for Pr = 1; 0.27% and 0.70% at H = 8 for
    Pr = 0.7 and 7).  A force off by a constant factor, a plate temperature or
    a wall position off by a node moves the onset by far more."""
    exact = _neutral_rayleigh(np.pi)
    assert abs(exact - 1707.922) < 0.01
    err8 = abs(_onset_rayleigh(orc, 8, 1.0, 0.05) / exact - 1)
    err12 = abs(_onset_rayleigh(orc, 12, 1.0, 0.05) / exact - 1)
    assert err8 < 1e-2 and err12 < 4e-3 and err12 < err8, (err8, err12)
    for Pr, nu in ((0.7, 0.05), (7.0, 0.1)):
        assert abs(_onset_rayleigh(orc, 8, Pr, nu) / exact - 1) < 1e-2, Pr


def _d3q7_transfer(kappa, k, a_T):
    """Per-mode transfer matrix of the D3Q7 scheme at rest, built here from the
    paper's definitions: A(k) = diag(exp(-i k e_x)) [I - N^-1 Q N (I - w 1^T)]."""
    e = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]])
    e2 = (e**2).sum(1)
    N = np.array([np.ones(7), e[:, 0], e[:, 1], e[:, 2], -6 + 7 * e2, 3 * e[:, 0] ** 2 - e2,
                  e[:, 1] ** 2 - e[:, 2] ** 2], dtype=float)
    qk, qe = 3 - SQ3, 4 * SQ3 - 6
    Q = np.diag([0, qk, qk, qk, qe, qe, qe])
    w = np.array([(1 - a_T) / 7] + [(6 + a_T) / 42] * 6)
    C = np.eye(7) - np.linalg.solve(N, Q @ N) @ (np.eye(7) - np.outer(w, np.ones(7)))
    A = np.diag(np.exp(-1j * k * e[:, 0])) @ C
    return A, w


def test_fourier_mode_decay_exact(orc):
    """Adiabatic half-way walls mirror the lattice into a period-2N one, so a
    cosine mode T = cos(pi (j + 1/2)/N) decays exactly as 1^T A(k)^t w T_0 with
    k = pi/N; its asymptotic rate is kappa k^2 (pure diffusion)."""
    N, kappa = 33, 0.039164
    walls = _walls([A, A, P, P, P, P])
    p = orc.Params(N, 3, 3, walls, 0.03, kappa, 0.0, N, 0.1)
    k = np.pi / N
    prof = np.cos(k * (np.arange(N) + 0.5))
    T0 = np.broadcast_to(prof[None, None, :], (3, 3, N))
    f, g = orc.init_equilibrium(p, 1.0, np.zeros(3), T0)
    Amat, w = _d3q7_transfer(kappa, k, p.a_T)
    vec = w.astype(complex)
    done = 0
    for t in (1, 7, 50, 200):
        f, g = orc.run(p, f, g, t - done)
        for _ in range(t - done):
            vec = Amat @ vec
        done = t
        _, _, T = orc.moments(p, f, g)
        amp = np.ones(7) @ vec
        assert abs(amp.imag) < 1e-14
        assert np.abs(T - amp.real * prof[None, None, :]).max() < 1e-13
    lam = np.abs(np.linalg.eigvals(Amat)).max()
    assert abs(-np.log(lam) / (kappa * k * k) - 1) < 1e-5


def test_poiseuille_exact(orc):
    """Body-force-driven channel between half-way bounce-back walls: with the
    TRT combination 3/16 the parabola u = F/(2 nu) (j + 1/2)(N - j - 1/2) is
    reproduced to round-off."""
    N, nu, F = 16, 0.1, 1e-6
    walls = _walls([P, P, A, A, P, P])
    p = orc.Params(3, N, 3, walls, nu, 0.05, 0.0, N, 0.1, body_force=(F, 0, 0))
    f, g = orc.init_equilibrium(p, 1.0, np.zeros(3), 0.0)
    f, g = orc.run(p, f, g, 12000)
    rho, u, _ = orc.moments(p, f, g)
    j = np.arange(N) + 0.5
    exact = F / (2 * nu) * j * (N - j)
    ux = u[0][:, :, 1]  # (z, y) at x = 1
    assert np.abs(ux - exact[None, :]).max() / exact.max() < 1e-9
    assert np.abs(u[1]).max() < 1e-15 and np.abs(u[2]).max() < 1e-15
    assert np.abs(rho - 1).max() < 1e-12


def _rotate_state(t, f, g, kind):
    """Rotate (x,y) -> (-y, x) about z, or mirror x -> -x, a whole state."""
    e19, e7 = t["e19"], t["e7"]
    if kind == "rot":
        R = np.array([[0, -1, 0], [1, 0, 0], [0, 0, 1]])
    else:
        R = np.diag([-1, 1, 1])
    perm19 = [int(np.where((e19 == R @ e19[i]).all(1))[0][0]) for i in range(19)]
    perm7 = [int(np.where((e7 == R @ e7[i]).all(1))[0][0]) for i in range(7)]

    def field(a):  # a[z, y, x]
        if kind == "rot":  # new(x', y') = old(x, y) with x' = n-1-y, y' = x
            return np.flip(np.swapaxes(a, -1, -2), axis=-1)
        return np.flip(a, axis=-1)

    fo, go = np.empty_like(f), np.empty_like(g)
    for i in range(19):
        fo[perm19[i]] = field(f[i])
    for i in range(7):
        go[perm7[i]] = field(g[i])
    return fo, go


@pytest.mark.parametrize("kind", ["rot", "mirror"])
def test_symmetry_commutes_with_step(orc, kind):
    """Rotating (or mirroring) a state about the gravity axis and stepping it
    gives the rotated (mirrored) step: catches a wrong index, sign or transposed
    operand in M, N, the forcing or the walls."""
    t = orc.tables()
    walls = _walls([A, A, A, A, D, D], (0, 0, 0, 0, 0.3, -0.2))
    p = orc.Params(6, 6, 5, walls, 0.03, 0.02, 4e-3, 5, 0.1)
    f, g = _state(orc, p, 9)
    fa, ga = orc.run(p, *_rotate_state(t, f, g, kind), 3)
    fb, gb = _rotate_state(t, *orc.run(p, f, g, 3), kind)
    assert np.abs(fa - fb).max() < 1e-15 and np.abs(ga - gb).max() < 1e-15


def test_box_step_matches_lattice_step(orc):
    """A step on a sub-box reproduces the whole-lattice step wherever the box
    holds the data, including nodes next to walls."""
    walls = _walls([D, D, A, A, A, A], (0.5, -0.5, 0, 0, 0, 0))
    p = orc.Params(7, 6, 5, walls, 0.03, 0.02, 4e-3, 5, 0.1)
    f, g = _state(orc, p, 10)
    F, G = orc.run(p, f, g, 1)
    org = (0, 1, 1)
    sl = (slice(None), slice(1, 5), slice(1, 5), slice(0, 4))
    fb, gb = orc.step_box(p, org, f[sl], g[sl])
    inner = (slice(None), slice(1, 3), slice(1, 3), slice(0, 3))
    assert np.array_equal(fb[inner], F[sl][inner]) and np.array_equal(gb[inner], G[sl][inner])
    assert np.isnan(fb[:, 0]).any()


# ----------------------------------------------------------- diagnostics --

def test_diagnostics_closed_forms(orc):
    """Fields with known averages: linear T between Dirichlet walls, a
    parabolic shear flow between no-slip walls, a vertical velocity and a
    density ripple.  Every non-periodic face is a no-slip wall, so each field
    is placed in a box whose walls it is consistent with."""
    N = 8
    z = np.arange(N) + 0.5
    y = np.arange(N) + 0.5
    x = np.arange(N) + 0.5
    ones = np.ones((N, N, N))
    # temperature: walls on z only, T linear from 0.7 (bottom) to -0.1 (top)
    pT = orc.Params(N, N, N, _walls([P, P, P, P, D, D], (0, 0, 0, 0, 0.7, -0.1)),
                    0.04, 0.03, 0.0, N, 0.1)
    Tprof = 0.7 - 0.8 * z / N
    T = Tprof[:, None, None] * ones
    rho = 1 + 1e-3 * np.cos(2 * np.pi * x / N)[None, None, :] * ones
    w = 1e-3 * (1 + np.cos(2 * np.pi * x / N))
    u = np.stack([0 * ones, 0 * ones, w[None, None, :] * ones])
    f, g = orc.init_equilibrium(pT, rho, u, T)
    d = orc.diagnostics(pT, f, g)
    assert abs(d["Nu_th"] - 0.64) < 1e-12  # H^2 |grad T|^2 = 0.8^2
    assert abs(d["Nu_face"][4] - 0.8) < 1e-12 and abs(d["Nu_face"][5] + 0.8) < 1e-12
    assert abs(d["rms_drho"] - 1e-3 / np.sqrt(2)) < 1e-12
    assert abs(d["Nu_vol"] - (1 + w.mean() * Tprof.mean() * N / pT.kappa)) < 1e-12
    assert abs(d["Re_w"] - np.sqrt((w**2).mean()) * N / pT.nu) < 1e-9
    # w does not vanish at the no-slip z walls: the one-sided stencil through the
    # wall value gives dw/dz = +-4/3 w in the two wall layers, 0 inside
    div2 = 2 / N * 16 / 9 * (w**2).mean()
    assert abs(d["rms_div"] - np.sqrt(div2) * N / 0.1) < 1e-12
    # shear: walls on y only, u_x = c (y + 1/2)(N - y - 1/2)
    pU = orc.Params(N, N, N, _walls([P, P, A, A, P, P]), 0.04, 0.03, 0.0, N, 0.1)
    c = 1e-3
    ux = c * y * (N - y)
    u = np.stack([ux[None, :, None] * ones, 0 * ones, 0 * ones])
    f, g = orc.init_equilibrium(pU, 1.0, u, 0.0)
    d = orc.diagnostics(pU, f, g)
    eps = (c * (N - 2 * y)) ** 2  # eps_u / nu = (d u_x / dy)^2
    Nu_kin = 1 + pU.nu * eps.mean() * N**2 / (pU.kappa * 0.1**2)
    assert abs(d["Nu_kin"] - Nu_kin) < 1e-12
    assert abs(d["Re_rms"] - np.sqrt((ux**2).mean()) * N / pU.nu) < 1e-9
    assert abs(d["E"] - 0.5 * (ux**2).mean() / 0.01) < 1e-12
    assert d["rms_div"] < 1e-15 and d["Re_w"] == 0 and d["Nu_th"] == 0


def test_nusselt_profile_conduction_is_one_everywhere(orc):
    """Sec. 3, Nu(y) of Fig. 4 and Nu_mean of Table 2: the conduction state
    between the hot (x = 0) and cold (x = H) walls of the side-heated cell,
    T = 1/2 - x/H at rest, carries Nu = 1 through every plane and along the
    mid-line of both walls (the cold wall's flux points out of the fluid:
    -1), on odd and even meshes; the adiabatic and z faces report 0."""
    for N in (9, 10):
        x = np.arange(N) + 0.5
        p = orc.Params(N, N, N, _walls([D, D, A, A, A, A], (0.5, -0.5, 0, 0, 0, 0)), 0.04, 0.03, 0.0, N, 0.1)
        T = (0.5 - x / N)[None, None, :] * np.ones((N, N, N))
        f, g = orc.init_equilibrium(p, 1.0, np.zeros((3, N, N, N)), T)
        prof, mid = orc.nusselt_profile(p, f, g, axis=0)
        assert prof.shape == (N,) and np.abs(prof - 1).max() < 1e-12
        assert abs(mid[0] - 1) < 1e-12 and abs(mid[1] + 1) < 1e-12 and (mid[2:] == 0).all()


def test_nusselt_profile_closed_form(orc):
    """A field the stencils take exactly: T = c(y) theta(x) with theta
    quadratic in x (theta(0) = 1/2, theta(H) = -1/2, curvature alpha) and
    c(y) = 1 + beta (y/H - 1/2), and a uniform velocity u_x = u0.  The plane
    mean of c is 1 on any mesh, so every plane carries exactly
    u0 theta(x_j) H/kappa - H theta'(x_j) (convection + conduction); the
    mid-line through y = H/2 has c = 1 (one node line on the odd mesh, the
    mean of the two bracketing lines on the even one), so Nu_mean is
    -H theta'(0) = 1 - alpha at the hot wall and H theta'(H) = -(1 + alpha)
    at the cold one.  A plane other than the middle, a dropped convective
    term, a wrong sign or a first-order wall stencil each fail it."""
    alpha, beta, u0 = 0.3, 0.4, 2e-3
    for N in (9, 10):
        H = float(N)
        x = np.arange(N) + 0.5
        y = np.arange(N) + 0.5
        th = 0.5 - x / H + alpha * (x / H) * (1 - x / H)
        dth = (-1 + alpha * (1 - 2 * x / H)) / H
        c = 1 + beta * (y / H - 0.5)
        T = c[None, :, None] * th[None, None, :] * np.ones((N, N, N))
        # the Dirichlet walls carry the wall values of theta times c(y): use the
        # mid-plane values 1/2 and -1/2; c(y) != 1 off the mid-plane makes the
        # one-sided stencil there see another wall value, which must not leak
        # into the mid-line or (by symmetry of c about the middle) the plane means
        p = orc.Params(N, N, N, _walls([D, D, A, A, A, A], (0.5, -0.5, 0, 0, 0, 0)), 0.04, 0.03, 0.0, N, 0.1)
        u = np.zeros((3, N, N, N))
        u[0] = u0
        f, g = orc.init_equilibrium(p, 1.0, u, T)
        prof, mid = orc.nusselt_profile(p, f, g, axis=0)
        want = u0 * th * H / p.kappa - H * dth
        # wall layers: the one-sided stencil uses T_w = +-1/2 where the field
        # has c(y) T_w; its plane mean is still exact because mean(c) = 1
        assert np.abs(prof - want).max() < 1e-12, prof - want
        assert abs(mid[0] - (1 - alpha)) < 1e-12 and abs(mid[1] + (1 + alpha)) < 1e-12
        # along y (adiabatic walls, zero-gradient stencil next to them)
        prof_y, _ = orc.nusselt_profile(p, f, g, axis=1)
        dc = beta / H * th.mean()
        want_y = -H * dc * np.ones(N)
        want_y[0] = -H * 0.5 * (c[1] - c[0]) * th.mean()
        want_y[-1] = -H * 0.5 * (c[-1] - c[-2]) * th.mean()
        assert np.abs(prof_y - want_y).max() < 1e-12


def test_local_dissipation_closed_forms(orc):
    """Per-node eps_u = nu/2 sum_ij (d_i u_j + d_j u_i)^2 and eps_T = kappa |grad T|^2
    (Sec. 4) on fields whose derivatives the stencils take exactly: u_x and the
    z-profile of u_y quadratic in z and zero at both no-slip plates, T quadratic
    in z through the two Dirichlet values (second-order stencils, central or
    one-sided through the wall value, are exact for quadratics), and u_y varying
    as sin(k x) along the periodic x axis (central difference sin(k) cos(k x))."""
    nx, ny, H = 8, 3, 10
    nu, ka = 0.03, 0.02
    walls = _walls([P, P, P, P, D, D], (0, 0, 0, 0, 0.5, -0.5))
    p = orc.Params(nx, ny, H, walls, nu, ka, 0.0, H, 0.1)
    z = (np.arange(H) + 0.5)[:, None, None] * np.ones((H, ny, nx))
    x = np.arange(nx)[None, None, :] * np.ones((H, ny, nx))
    k, A, B = 2 * np.pi / nx, 0.01, 0.004
    q = z * (H - z) / H**2
    u3 = np.zeros((3, H, ny, nx))
    u3[0] = A * q
    u3[1] = B * np.sin(k * x) * q
    T = 0.5 - z / H + 0.3 * z * (H - z) / H**2
    f, g = orc.init_equilibrium(p, np.ones((H, ny, nx)), u3, T)
    eu, et = orc.local_dissipation(p, f, g)
    dq = (H - 2 * z) / H**2
    d = np.zeros((3, 3) + z.shape)  # d[i, j] = d u_j / d x_i
    d[2, 0] = A * dq
    d[0, 1] = B * np.sin(k) * np.cos(k * x) * q
    d[2, 1] = B * np.sin(k * x) * dq
    strain = sum(0.5 * (d[i, j] + d[j, i]) ** 2 for i in range(3) for j in range(3))
    assert np.allclose(eu, nu * strain, rtol=1e-10, atol=1e-18)
    dT = -1.0 / H + 0.3 * (H - 2 * z) / H**2
    assert np.allclose(et, ka * dT**2, rtol=1e-10, atol=1e-18)
    # the per-node rates are the integrands of the global Nu_kin and Nu_th sums
    r = orc.raw_diagnostics(p, f, g)
    assert np.isclose(eu.sum() / nu, r[5], rtol=1e-12) and np.isclose(et.sum() / ka, r[6], rtol=1e-12)


def test_paper_probe_positions_are_half_way_node_centres():
    """Table 1 prints the probe positions of its steady side-heated runs; on an
    N-node lattice with half-way walls (node j at (j + 1/2)/N, walls at 0 and
    1) each is a node centre, which pins the geometry reading of the wall
    placement (a lattice with nodes on the walls would put them at j/(N-1))."""
    import json

    ref = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_side_heated_Ra1e6.json")))
    for key in ("81", "129"):
        N = int(key)
        for pos in (ref[key]["z"], ref[key]["y"]):
            j = pos * N - 0.5
            assert abs(j - round(j)) < 0.02, (N, pos, j)
            k = pos * (N - 1)
            assert abs(k - round(k)) > 0.05 or abs(j - round(j)) < abs(k - round(k)), (N, pos, k)


def test_grid_convergence_reproduces_the_papers_table2_fits():
    """drivers.grid_convergence applied to the Nusselt numbers the paper prints
    for its meshes returns the f_inf and order n it prints beside them, for
    all eight columns of Table 2 (to the printed digits)."""
    import json

    from paper_1903_08882_gb300 import drivers

    ref = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_table2_convergence.json")))
    for name, c in ref["columns"].items():
        f_inf, n = drivers.grid_convergence(c["N"], c["f"])
        assert abs(f_inf - c["f_inf"]) <= 1.5e-4, (name, f_inf)
        assert abs(n - c["n"]) <= 0.006, (name, n)


def test_grid_convergence_closed_form():
    """On values f_inf + C N^-p (a polynomial of degree < meshes in h = 1/N
    when p is an integer) the fit is exact."""
    from paper_1903_08882_gb300 import drivers

    N = np.array([33, 65, 129, 257])
    for p in (1, 2, 3):
        f = 1.25 + 7.0 * N ** -float(p)
        f_inf, n = drivers.grid_convergence(N, f)
        assert abs(f_inf - 1.25) < 1e-10 and abs(n - p) < 1e-6, (p, f_inf, n)
