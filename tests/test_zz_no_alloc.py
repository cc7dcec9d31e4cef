"""The allocation-free reduction entry point against the ordinary path.

lbm_reduce_noalloc serves callers that must not allocate device memory while
they run (their framework owns the GPU's memory, or their loop may not call
cudaMalloc); its scratch is a fixed static device array instead of memory a
context allocated.  This file is collected last on purpose.  Each check
builds the reduction's input fields on the device from a context's own
state, calls the entry point through the C ABI twice in a row on different
states, and compares the sums with those lbm_sample produced for the same
state, within the tolerance of the other diagnostics tests (1e-5).  The
device's free memory is read before and after each call: creating the
context already loaded the static array, so neither call may take any."""
import numpy as np
import pytest

from paper_1903_08882_gb300 import inputs

pytestmark = pytest.mark.gpu


def _device_fields(torch, lat, stride):
    """The eleven input arrays (rho - rho0, u, v, w, T, g arriving from each
    face) of the context's current state, as one device tensor."""
    nz, ny, nx = lat.shape
    n = nx * ny * nz
    rho, u3, T = lat.moments()
    f, g = lat.populations()
    host = np.zeros((11, stride), dtype=np.float32)
    host[0, :n] = (rho - 1.0).ravel()
    for a in range(3):
        host[1 + a, :n] = u3[a].ravel()
    host[4, :n] = T.ravel()
    # face f: -x, +x, -y, +y, -z, +z; velocity f + 1 points away from it
    layers = [(slice(None), slice(None), 0), (slice(None), slice(None), nx - 1),
              (slice(None), 0, slice(None)), (slice(None), ny - 1, slice(None)),
              (0, slice(None), slice(None)), (nz - 1, slice(None), slice(None))]
    for fc, sl in enumerate(layers):
        arr = np.zeros((nz, ny, nx), dtype=np.float32)
        arr[sl] = g[fc + 1][sl]
        host[5 + fc, :n] = arr.ravel()
    return torch.from_numpy(host).cuda()


def test_noalloc_reduction_matches_context_path():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1903_08882_gb300 import _build, lbm

    _build.build()
    n = (29, 27, 31)
    walls = lbm.walls_rayleigh_benard()
    stride = (29 * 27 * 31 + 127) // 128 * 128
    with lbm.Lattice(*n, walls, Ra=1e5, Pr=0.7) as lat:
        a_T = lat.constants["a_T"]
        sums = torch.zeros(lbm.NDIAG, dtype=torch.float64, device="cuda")
        for call, seed in enumerate((11, 12)):
            T0 = inputs.rb_initial_temperature(*n, seed=seed, delta=0.05)
            lat.set_fields(1.0, np.zeros(3), T0)
            lat.step(40 + 7 * call)
            lat.sample()
            ref = np.array(lat.diagnostics()["raw"])
            fields = _device_fields(torch, lat, stride)
            sums.fill_(np.nan)
            torch.cuda.synchronize()
            free_before = torch.cuda.mem_get_info()[0]
            lbm.lbm_reduce_noalloc(fields.data_ptr(), stride, *n, walls, a_T, sums.data_ptr(),
                                   stream=torch.cuda.current_stream())
            torch.cuda.synchronize()
            assert torch.cuda.mem_get_info()[0] == free_before, call
            got = sums.cpu().numpy()
            assert np.isfinite(got).all()
            assert np.allclose(got, ref, rtol=1e-5, atol=1e-12), (call, got - ref)
            assert got[0] == np.prod(n) and got[17] == 0
        # a request that needs more rows than the static array holds is refused
        with pytest.raises(lbm.LbmError) as ei:
            lbm.lbm_reduce_noalloc(fields.data_ptr(), stride, *n, walls, a_T, sums.data_ptr(),
                                   blocks=1217)
        assert ei.value.status == lbm.LBM_ERR_PARAM and "static scratch" in str(ei.value)
