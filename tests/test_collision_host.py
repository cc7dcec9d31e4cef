"""The library's fused collision, compiled for the host from the same device
header, against the FP64 oracle's collision on random node states (no GPU).

Tolerance: FP32 arithmetic on deviations of O(1e-2); 2e-6 of the largest
deviation of each node's result, 1e-6 relative on the moments."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "native", "collide_host.cu")
W19 = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)


@pytest.fixture(scope="module")
def harness():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc) and not shutil.which("nvcc"):
        pytest.skip("nvcc not available")
    out = os.path.join(HERE, "native", "_build", "collide_host")
    os.makedirs(os.path.dirname(out), exist_ok=True)
    deps = [SRC, os.path.join(HERE, "..", "paper_1903_08882_gb300", "csrc", "lbm_device.cuh")]
    if not os.path.exists(out) or any(os.path.getmtime(d) > os.path.getmtime(out) for d in deps):
        subprocess.check_call([nvcc, "-O2", "-std=c++17", "--expt-relaxed-constexpr", "-o", out, SRC])
    return out


def _run(exe, phys, nodes, mode="float"):
    txt = " ".join(f"{v:.9e}" for v in phys) + "\n"
    txt += "\n".join(" ".join(f"{v:.17e}" for v in row) for row in nodes) + "\n"
    r = subprocess.run([exe, mode], input=txt, capture_output=True, text=True, check=True)
    return np.array([[float(x) for x in l.split()] for l in r.stdout.strip().splitlines()])


@pytest.mark.parametrize("nu,kappa,gbeta,bf", [
    (0.0068, 0.0096, 3.9e-5, (0, 0, 0)),      # 257^3 side-heated Ra=1e7
    (0.0278, 0.0392, 3.0e-4, (0, 0, 0)),      # 33^3 Ra=1e4
    (0.1, 0.05, 2e-3, (1e-4, -2e-4, 5e-5)),   # body force on every axis
    (0.5, 0.09, 0.0, (0, 0, 0)),
])
def test_host_collision_matches_oracle(harness, nu, kappa, gbeta, bf):
    p = oracle.Params(4, 4, 4, [(0, 0)] * 6, nu, kappa, gbeta, 4.0, 0.1, bf)
    s, q = p.rates
    phys = [s[1], s[4], q[1], q[4], p.a_T, gbeta, *bf]
    rng = np.random.default_rng(7)
    rows, ref = [], []
    for _ in range(200):
        rho = 1 + 2e-3 * rng.standard_normal()
        u = 0.04 * rng.standard_normal(3)
        T = 0.5 * rng.uniform(-1, 1)
        fe, ge = oracle.equilibrium(p, rho, u, T)
        f = fe + 1e-4 * rng.standard_normal(19)
        g = ge + 1e-3 * rng.standard_normal(7)
        # the harness works on what the GPU stores: FP32 deviations f - w
        f32 = (f - W19).astype(np.float32).astype(np.float64)
        g32 = g.astype(np.float32).astype(np.float64)
        rows.append(np.concatenate([f32, g32]))
        fo, go, mom = oracle.collide(p, f32 + W19, g32)
        ref.append(np.concatenate([fo - W19, go, [mom[0] - 1], mom[1:]]))
    out = _run(harness, phys, rows)
    ref = np.array(ref)
    for k in range(len(rows)):
        scale_f = np.abs(ref[k, :19]).max()
        scale_g = np.abs(ref[k, 19:26]).max()
        assert np.abs(out[k, :19] - ref[k, :19]).max() < 2e-6 * scale_f + 1e-9
        assert np.abs(out[k, 19:26] - ref[k, 19:26]).max() < 2e-6 * scale_g + 1e-9
        umax = np.abs(ref[k, 27:30]).max()
        assert np.abs(out[k, 27:30] - ref[k, 27:30]).max() < 1e-6 * umax + 1e-9
        assert abs(out[k, 26] - ref[k, 26]) < 1e-6 * abs(ref[k, 26]) + 1e-9
        assert abs(out[k, 30] - ref[k, 30]) < 1e-6 * abs(ref[k, 30]) + 1e-9


@pytest.mark.parametrize("nu,kappa,gbeta,bf", [
    (0.0068, 0.0096, 3.9e-5, (0, 0, 0)),
    (0.1, 0.05, 2e-3, (1e-4, -2e-4, 5e-5)),
    (0.5, 0.09, 0.0, (0, 0, 0)),
])
def test_host_collision_algebra_fp64(harness, nu, kappa, gbeta, bf):
    """The same collision instantiated in FP64 (only the rates and constants
    stay FP32 numbers: relative error ~6e-8, and (1 - s_e)/2 multiplies the
    whole pair sum, so the bound is 2e-7 of the node's largest population
    deviation) against the oracle's moment-space MRT: the pairwise
    velocity-space evaluation must agree with Eq. MRT / Eq. MRT_T to that
    level, two orders below the smallest term of the collision here (the
    forcing, ~1e-6), so an algebraic slip in it (a coefficient, a sign, a
    weight) fails."""
    p = oracle.Params(4, 4, 4, [(0, 0)] * 6, nu, kappa, gbeta, 4.0, 0.1, bf)
    s, q = p.rates
    phys = [s[1], s[4], q[1], q[4], p.a_T, gbeta, *bf]
    rng = np.random.default_rng(11)
    rows, ref = [], []
    for _ in range(100):
        rho = 1 + 2e-2 * rng.standard_normal()
        u = 0.08 * rng.standard_normal(3)
        T = 0.5 * rng.uniform(-1, 1)
        fe, ge = oracle.equilibrium(p, rho, u, T)
        f = fe + 1e-3 * rng.standard_normal(19)
        g = ge + 1e-2 * rng.standard_normal(7)
        rows.append(np.concatenate([f - W19, g]))
        fo, go, mom = oracle.collide(p, f, g)
        ref.append(np.concatenate([fo - W19, go, [mom[0] - 1], mom[1:]]))
    out = _run(harness, phys, rows, mode="double")
    ref = np.array(ref)
    for k in range(len(rows)):
        sf = np.abs(ref[k, :19]).max()
        sg = np.abs(ref[k, 19:26]).max()
        assert np.abs(out[k, :19] - ref[k, :19]).max() < 2e-7 * sf + 1e-12
        # D3Q7: a_T = 42 sqrt(3) kappa - 6 as an FP32 number carries ~4e-7 absolute
        assert np.abs(out[k, 19:26] - ref[k, 19:26]).max() < 1e-6 * sg + 1e-12
        assert np.abs(out[k, 26:31] - ref[k, 26:31]).max() < 1e-7 * np.abs(ref[k, 26:31]).max() + 1e-12
