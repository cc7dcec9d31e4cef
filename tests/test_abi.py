"""The C ABI library builds, loads and exports every declared entry point, and
rejects invalid parameter sets before touching a GPU (no GPU needed here)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_1903_08882_gb300 import _build, lbm

    _build.build()
    return lbm


def _declared(header=None):
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        if header and os.path.basename(h) != header:
            continue
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", src))
    return names


def test_header_declares_entry_points():
    names = _declared()
    for must in ("lbm_create", "lbm_step", "lbm_moments", "lbm_diagnostics", "lbm_destroy",
                 "lbm_set_populations", "lbm_get_populations", "lbm_set_fields"):
        assert must in names


def test_library_exports_every_declared_symbol(L):
    lib = ctypes.CDLL(L.LIB_PATH)
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(L):
    from paper_1903_08882_gb300 import unet

    for n in _declared("lbm.h"):
        assert hasattr(L, n), n
    assert _declared("lbm_nn.h") == set(unet.NN_SIGNATURES)


def _status(L, p):
    ctx = ctypes.c_void_p()
    return L.lib().lbm_create(ctypes.byref(p), None, None, ctypes.byref(ctx)), ctx


@pytest.mark.parametrize("bad", [
    dict(nx=2),
    dict(kappa=0.2),            # a_T > 1: negative rest weight of D3Q7
    dict(nu=-0.1),              # tau_f < 1/2
    dict(U=0.5),
    dict(walls="half_periodic"),
    dict(storage=7),
    dict(block_size=48),
    dict(diag_every=-1),
    dict(pipeline=3),
    dict(nx=1700, ny=1700, nz=1700),  # 4.9e9 nodes: beyond 32-bit node indices
])
def test_invalid_parameters_rejected_on_host(L, bad):
    kw = dict(nx=8, ny=8, nz=8, walls=L.walls_side_heated(), nu=0.02, kappa=0.02, gbeta=1e-4)
    if "walls" in bad and bad["walls"] == "half_periodic":
        kw["walls"] = [(L.PERIODIC, 0), (L.ADIABATIC, 0)] + [(L.ADIABATIC, 0)] * 4
        bad = {}
    kw.update(bad)
    nx, ny, nz, walls = kw.pop("nx"), kw.pop("ny"), kw.pop("nz"), kw.pop("walls")
    p = L.make_params(nx, ny, nz, walls, **kw)
    st, ctx = _status(L, p)
    assert st == L.LBM_ERR_PARAM and not ctx.value
    assert L.lib().lbm_last_error(None)


def test_null_arguments(L):
    ctx = ctypes.c_void_p()
    assert L.lib().lbm_create(None, None, None, ctypes.byref(ctx)) == L.LBM_ERR_PARAM
    assert L.lib().lbm_step(None, 1) == L.LBM_ERR_PARAM
    assert L.lib().lbm_destroy(None) is None
