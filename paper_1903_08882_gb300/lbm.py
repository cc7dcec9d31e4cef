"""Python binding of the C ABI declared in include/lbm.h.

Argument marshalling only: every step of the method runs in the CUDA library
liblbm_gb300.so.  There is no Python or CPU fallback; if the library is
missing, loading it raises.  Device memory is provided by PyTorch's caching
allocator through the lbm_allocator hook; streams are PyTorch streams.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "liblbm_gb300.so")

LBM_OK, LBM_ERR_PARAM, LBM_ERR_CUDA, LBM_ERR_OOM, LBM_ERR_DIVERGED, LBM_ERR_TIMEOUT, LBM_ERR_STATE = range(7)
ADIABATIC, DIRICHLET, PERIODIC = 0, 1, 2
STORAGE = {"fp32": 0, "fp16s": 1, "bf16s": 2, "fp16m": 3}
STREAMING = {"aa": 0, "pull2": 1}
PIPELINE = {"default": 0, "register": 1, "staged": 2}
NDIAG = 24

c_int, c_double, c_int64, c_void_p, c_size_t = (ctypes.c_int, ctypes.c_double, ctypes.c_int64,
                                                 ctypes.c_void_p, ctypes.c_size_t)


class LbmWall(ctypes.Structure):
    _fields_ = [("kind", c_int), ("T_w", c_double)]


class LbmParams(ctypes.Structure):
    _fields_ = [
        ("nx", c_int), ("ny", c_int), ("nz", c_int),
        ("Ra", c_double), ("Pr", c_double), ("U", c_double), ("H", c_double),
        ("derive", c_int),
        ("nu", c_double), ("kappa", c_double), ("gbeta", c_double),
        ("body_force", c_double * 3),
        ("wall", LbmWall * 6),
        ("storage", c_int), ("streaming", c_int), ("diag_every", c_int), ("block_size", c_int),
        ("nodes_per_thread", c_int), ("pipeline", c_int),
    ]


ALLOC_FN = ctypes.CFUNCTYPE(c_void_p, c_size_t, c_void_p, c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, c_void_p, c_size_t, c_void_p, c_void_p)


class LbmAllocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", c_void_p)]


class LbmConstants(ctypes.Structure):
    _fields_ = [(k, c_double) for k in ("nu", "kappa", "gbeta", "tau_f", "s_e", "s_q", "q_kappa", "q_e",
                                         "q_nu", "a_T", "w0_T", "w1_T", "H", "U")] + [
        ("nodes", c_int64), ("device_bytes", c_int64)]


class LbmDiag(ctypes.Structure):
    _fields_ = ([("step", c_int64), ("sample_step", c_int64), ("samples", c_int64)]
                + [(k, c_double) for k in ("E", "rms_drho", "rms_div", "Re_rms", "Re_w", "Nu_vol", "Nu_kin",
                                           "Nu_th", "mean_T", "mass", "max_u")]
                + [("Nu_face", c_double * 6), ("Nu_link", c_double * 6)]
                + [(k, c_double) for k in ("avg_E", "avg_Re_rms", "avg_Re_w", "avg_Nu_vol", "avg_Nu_kin",
                                           "avg_Nu_th")]
                + [("avg_Nu_face", c_double * 6), ("nonfinite", c_int64), ("raw", c_double * NDIAG)])

    def as_dict(self) -> dict:
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = np.array(v[:]) if isinstance(v, ctypes.Array) else v
        return out


class LbmSchedule(ctypes.Structure):
    _fields_ = [("block_size", c_int), ("blocks_per_sm", c_int), ("steps_per_launch", c_int), ("graph_chunk", c_int),
                ("tile_span", c_int), ("mode", c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class LbmError(RuntimeError):
    def __init__(self, status: int, message: str, diag: dict | None = None):
        super().__init__(f"lbm status {status}: {message}")
        self.status = status
        self.diag = diag


_lib = None


def lib():
    """The loaded CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() (nvcc, sm_103a)")
    L = ctypes.CDLL(LIB_PATH)
    P, C = ctypes.POINTER, ctypes.POINTER(ctypes.c_void_p)
    dp, i64p = P(c_double), P(c_int64)
    sig = {
        "lbm_create": ([P(LbmParams), P(LbmAllocator), c_void_p, C], c_int),
        "lbm_destroy": ([c_void_p], None),
        "lbm_last_error": ([c_void_p], ctypes.c_char_p),
        "lbm_get_constants": ([c_void_p, P(LbmConstants)], c_int),
        "lbm_set_fields": ([c_void_p, dp, dp, dp], c_int),
        "lbm_upload_fields": ([c_void_p, dp, dp, dp], c_int),
        "lbm_apply_fields": ([c_void_p], c_int),
        "lbm_set_populations": ([c_void_p, dp, dp], c_int),
        "lbm_get_populations": ([c_void_p, dp, dp], c_int),
        "lbm_get_populations_at": ([c_void_p, i64p, c_int64, dp, dp], c_int),
        "lbm_step": ([c_void_p, c_int64], c_int),
        "lbm_moments": ([c_void_p, dp, dp, dp], c_int),
        "lbm_sample": ([c_void_p], c_int),
        "lbm_dissipation_pdf": ([c_void_p, c_int, c_double, dp, dp, P(ctypes.c_uint64), P(ctypes.c_uint64)], c_int),
        "lbm_nusselt_profile": ([c_void_p, c_int, dp, dp], c_int),
        "lbm_diagnostics": ([c_void_p, P(LbmDiag), c_int], c_int),
        "lbm_synchronize": ([c_void_p], c_int),
        "lbm_set_wait_budget": ([c_void_p, c_int64], c_int),
        "lbm_save": ([c_void_p, ctypes.c_char_p], c_int),
        "lbm_load": ([c_void_p, ctypes.c_char_p], c_int),
        "lbm_device_view": ([c_void_p, C, C, i64p, P(c_int)], c_int),
        "lbm_reduce_noalloc": ([c_void_p, c_int64, c_int, c_int, c_int, P(LbmWall), c_double, c_int, c_void_p,
                                c_void_p], c_int),
        "lbm_batch_create": ([P(c_void_p), c_int, c_void_p, C], c_int),
        "lbm_batch_destroy": ([c_void_p], None),
        "lbm_batch_step": ([c_void_p, c_int64], c_int),
        "lbm_batch_get_schedule": ([c_void_p, P(LbmSchedule)], c_int),
        "lbm_batch_set_schedule": ([c_void_p, P(LbmSchedule)], c_int),
        "lbm_batch_autotune": ([c_void_p, c_int, P(LbmSchedule)], c_int),
        "lbm_batch_set_barrier_budget": ([c_void_p, c_int64], c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(c_double))


def _f64(a, shape):
    a = np.ascontiguousarray(np.broadcast_to(np.asarray(a, dtype=np.float64), shape))
    return a


# ------------------------------------------------------------- allocator --

_torch_alloc = None


def torch_allocator() -> LbmAllocator:
    """An lbm_allocator backed by PyTorch's CUDA caching allocator."""
    global _torch_alloc
    if _torch_alloc is None:
        import torch

        def _alloc(nbytes, stream, user):
            try:
                return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
            except Exception:  # out of memory: the library reports LBM_ERR_OOM
                return None

        def _free(ptr, nbytes, stream, user):
            try:
                torch.cuda.caching_allocator_delete(int(ptr))
            except Exception:
                pass

        a = LbmAllocator()
        a.alloc = ALLOC_FN(_alloc)
        a.free = FREE_FN(_free)
        a.user = None
        _torch_alloc = a
    return _torch_alloc


# ---------------------------------------------------------------- params --

def walls_side_heated(T_hot=0.5, T_cold=-0.5):
    """Hot face -x, cold face +x, four adiabatic faces (all no-slip)."""
    return [(DIRICHLET, T_hot), (DIRICHLET, T_cold)] + [(ADIABATIC, 0.0)] * 4


def walls_rayleigh_benard(T_bottom=0.5, T_top=-0.5):
    """Four adiabatic sidewalls, hot bottom -z, cold top +z (all no-slip)."""
    return [(ADIABATIC, 0.0)] * 4 + [(DIRICHLET, T_bottom), (DIRICHLET, T_top)]


def make_params(nx, ny, nz, walls, Ra=1e6, Pr=0.71, U=0.1, H=0.0, nu=None, kappa=None, gbeta=None,
                body_force=(0.0, 0.0, 0.0), storage="fp32", streaming="aa", diag_every=0,
                block_size=0, nodes_per_thread=0, pipeline=0) -> LbmParams:
    p = LbmParams()
    p.nx, p.ny, p.nz = int(nx), int(ny), int(nz)
    p.Ra, p.Pr, p.U, p.H = float(Ra), float(Pr), float(U), float(H)
    if nu is not None:
        p.derive = 0
        p.nu, p.kappa, p.gbeta = float(nu), float(kappa), float(gbeta)
    else:
        p.derive = 1
    for a in range(3):
        p.body_force[a] = float(body_force[a])
    for k, (kind, tw) in enumerate(walls):
        p.wall[k].kind = int(kind)
        p.wall[k].T_w = float(tw)
    p.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
    p.streaming = STREAMING[streaming] if isinstance(streaming, str) else int(streaming)
    p.diag_every = int(diag_every)
    p.block_size = int(block_size)
    p.nodes_per_thread = int(nodes_per_thread)
    p.pipeline = PIPELINE[pipeline] if isinstance(pipeline, str) else int(pipeline)
    return p


# --------------------------------------------------------------- context --

def _check(ctx, status, diag=None):
    if status != LBM_OK:
        msg = lib().lbm_last_error(ctx).decode() if ctx is not None else lib().lbm_last_error(None).decode()
        raise LbmError(status, msg, diag)


def lbm_create(params: LbmParams, allocator="torch", stream=None):
    """Create a context.  allocator: "torch" (PyTorch caching allocator) or None
    (the library calls cudaMalloc).  stream: a torch.cuda.Stream, a raw
    cudaStream_t as int, or None for the current PyTorch stream."""
    L = lib()
    if allocator == "torch":
        alloc = ctypes.byref(torch_allocator())
    else:
        alloc = None
    if stream is None:
        import torch

        stream = torch.cuda.current_stream().cuda_stream
    elif hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    ctx = ctypes.c_void_p()
    st = L.lbm_create(ctypes.byref(params), alloc, c_void_p(int(stream) or None), ctypes.byref(ctx))
    if st != LBM_OK:
        raise LbmError(st, L.lbm_last_error(None).decode())
    return ctx


def lbm_destroy(ctx):
    lib().lbm_destroy(ctx)


def lbm_last_error(ctx) -> str:
    return lib().lbm_last_error(ctx).decode()


def lbm_get_constants(ctx) -> dict:
    c = LbmConstants()
    _check(ctx, lib().lbm_get_constants(ctx, ctypes.byref(c)))
    return {k: getattr(c, k) for k, _ in c._fields_}


def _dims(ctx):
    c = LbmConstants()
    lib().lbm_get_constants(ctx, ctypes.byref(c))
    return int(c.nodes)


def lbm_set_fields(ctx, rho, u3, T, shape):
    """shape = (nz, ny, nx); rho and T broadcast to it, u3 to (3,) + shape."""
    u3 = np.asarray(u3, dtype=np.float64)
    if u3.ndim == 1:
        u3 = u3.reshape(3, 1, 1, 1)
    r, u, t = _f64(rho, shape), _f64(u3, (3,) + tuple(shape)), _f64(T, shape)
    _check(ctx, lib().lbm_set_fields(ctx, _dp(r), _dp(u), _dp(t)))


def lbm_upload_fields(ctx, rho, u3, T, shape):
    """Queue the copy of the fields (marshalled as for lbm_set_fields) on the
    context's copy stream.  Returns the marshalled arrays: the caller keeps
    them alive until a synchronising call after the lbm_apply_fields that
    uses them (the copy reads them asynchronously)."""
    u3 = np.asarray(u3, dtype=np.float64)
    if u3.ndim == 1:
        u3 = u3.reshape(3, 1, 1, 1)
    r, u, t = _f64(rho, shape), _f64(u3, (3,) + tuple(shape)), _f64(T, shape)
    _check(ctx, lib().lbm_upload_fields(ctx, _dp(r), _dp(u), _dp(t)))
    return r, u, t


def lbm_apply_fields(ctx):
    _check(ctx, lib().lbm_apply_fields(ctx))


def lbm_set_populations(ctx, f19, g7):
    f = np.ascontiguousarray(f19, dtype=np.float64)
    g = np.ascontiguousarray(g7, dtype=np.float64)
    n = _dims(ctx)
    assert f.size == 19 * n and g.size == 7 * n
    _check(ctx, lib().lbm_set_populations(ctx, _dp(f), _dp(g)))


def lbm_get_populations(ctx, shape):
    f = np.empty((19,) + tuple(shape))
    g = np.empty((7,) + tuple(shape))
    _check(ctx, lib().lbm_get_populations(ctx, _dp(f), _dp(g)))
    return f, g


def lbm_get_populations_at(ctx, nodes):
    nodes = np.ascontiguousarray(nodes, dtype=np.int64)
    f = np.empty((len(nodes), 19))
    g = np.empty((len(nodes), 7))
    st = lib().lbm_get_populations_at(ctx, nodes.ctypes.data_as(ctypes.POINTER(c_int64)), len(nodes), _dp(f),
                                      _dp(g))
    _check(ctx, st)
    return f, g


def lbm_step(ctx, n: int):
    _check(ctx, lib().lbm_step(ctx, int(n)))


def lbm_moments(ctx, shape):
    rho = np.empty(tuple(shape))
    u3 = np.empty((3,) + tuple(shape))
    T = np.empty(tuple(shape))
    _check(ctx, lib().lbm_moments(ctx, _dp(rho), _dp(u3), _dp(T)))
    return rho, u3, T


def lbm_dissipation_pdf(ctx, nbins: int = 200, xmax: float = 20.0, rms=None):
    """Counts of X = eps/eps_rms of the local dissipation rates (Sec. 4) in nbins
    bins on [0, xmax): returns (counts_u, counts_T, rms) with rms = (eps_u,
    eps_T) rms used (given, or of this state)."""
    cu = np.zeros(int(nbins), dtype=np.uint64)
    ct = np.zeros(int(nbins), dtype=np.uint64)
    out = np.zeros(2)
    rin = None if rms is None else np.ascontiguousarray(rms, dtype=np.float64)
    u64 = ctypes.POINTER(ctypes.c_uint64)
    _check(ctx, lib().lbm_dissipation_pdf(ctx, int(nbins), float(xmax), None if rin is None else _dp(rin), _dp(out),
                                           cu.ctypes.data_as(u64), ct.ctypes.data_as(u64)))
    return cu, ct, (float(out[0]), float(out[1]))


def lbm_nusselt_profile(ctx, shape, axis: int = 0):
    """Plane-averaged Nusselt number along `axis` and the six mid-line wall
    Nusselt numbers (Sec. 3: Nu(y) of Fig. 4, Nu_mean of Table 2) of the
    current state; shape = (nz, ny, nx).  Returns (profile, nu_mid)."""
    na = (shape[2], shape[1], shape[0])[int(axis)]
    prof = np.zeros(na)
    mid = np.zeros(6)
    _check(ctx, lib().lbm_nusselt_profile(ctx, int(axis), _dp(prof), _dp(mid)))
    return prof, mid


def lbm_sample(ctx):
    _check(ctx, lib().lbm_sample(ctx))


def lbm_diagnostics(ctx, reset: bool = False, raise_on_diverged: bool = True) -> dict:
    d = LbmDiag()
    st = lib().lbm_diagnostics(ctx, ctypes.byref(d), int(bool(reset)))
    out = d.as_dict()
    if st == LBM_ERR_DIVERGED and not raise_on_diverged:
        out["diverged"] = True
        return out
    _check(ctx, st, out)
    out["diverged"] = False
    return out


def lbm_synchronize(ctx):
    _check(ctx, lib().lbm_synchronize(ctx))


def lbm_set_wait_budget(ctx, cycles: int):
    _check(ctx, lib().lbm_set_wait_budget(ctx, int(cycles)))


def lbm_save(ctx, path: str):
    _check(ctx, lib().lbm_save(ctx, os.fsencode(path)))


def lbm_load(ctx, path: str):
    _check(ctx, lib().lbm_load(ctx, os.fsencode(path)))


def lbm_device_view(ctx):
    f, g = ctypes.c_void_p(), ctypes.c_void_p()
    stride, eb = c_int64(), c_int()
    _check(ctx, lib().lbm_device_view(ctx, ctypes.byref(f), ctypes.byref(g), ctypes.byref(stride),
                                      ctypes.byref(eb)))
    return f.value, g.value, stride.value, eb.value


def lbm_reduce_noalloc(fields_ptr: int, stride: int, nx: int, ny: int, nz: int, walls, a_T: float,
                       sums_ptr: int, blocks: int = 0, stream=None):
    """Allocation-free diagnostics reduction over caller-held device fields
    (device pointers as ints; see include/lbm.h).  The paper has no
    counterpart; it serves callers that must not allocate device memory."""
    w = (LbmWall * 6)()
    for k, (kind, tw) in enumerate(walls):
        w[k].kind, w[k].T_w = int(kind), float(tw)
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    st = lib().lbm_reduce_noalloc(c_void_p(fields_ptr), int(stride), int(nx), int(ny), int(nz), w, float(a_T),
                                  int(blocks), c_void_p(sums_ptr), c_void_p(int(stream or 0) or None))
    _check(None, st)


# ----------------------------------------------------------------- batches --

def _bcheck(status):
    if status != LBM_OK:
        raise LbmError(status, lib().lbm_last_error(None).decode())


def lbm_batch_create(ctxs, stream=None):
    """Batch over existing contexts (ctypes handles).  stream: torch.cuda.Stream,
    raw cudaStream_t int, or None for the current PyTorch stream."""
    L = lib()
    if stream is None:
        import torch

        stream = torch.cuda.current_stream().cuda_stream
    elif hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    arr = (c_void_p * len(ctxs))(*[c.value for c in ctxs])
    out = ctypes.c_void_p()
    _bcheck(L.lbm_batch_create(arr, len(ctxs), c_void_p(int(stream) or None), ctypes.byref(out)))
    return out


def lbm_batch_destroy(batch):
    lib().lbm_batch_destroy(batch)


def lbm_batch_step(batch, n: int):
    _bcheck(lib().lbm_batch_step(batch, int(n)))


def lbm_batch_get_schedule(batch) -> dict:
    s = LbmSchedule()
    _bcheck(lib().lbm_batch_get_schedule(batch, ctypes.byref(s)))
    return s.as_dict()


def lbm_batch_set_schedule(batch, block_size=256, blocks_per_sm=2, steps_per_launch=100, graph_chunk=1000,
                           tile_span=1, mode=0):
    s = LbmSchedule(block_size, blocks_per_sm, steps_per_launch, graph_chunk, tile_span, mode)
    _bcheck(lib().lbm_batch_set_schedule(batch, ctypes.byref(s)))


def lbm_batch_autotune(batch, trial_steps=20) -> dict:
    s = LbmSchedule()
    _bcheck(lib().lbm_batch_autotune(batch, int(trial_steps), ctypes.byref(s)))
    return s.as_dict()


def lbm_batch_set_barrier_budget(batch, cycles: int):
    _bcheck(lib().lbm_batch_set_barrier_budget(batch, int(cycles)))


class Batch:
    """Owns a batch over Lattice objects (which must outlive it)."""

    def __init__(self, lattices, stream=None):
        self.lattices = list(lattices)
        self.handle = lbm_batch_create([l.ctx for l in self.lattices], stream=stream)

    def close(self):
        if self.handle is not None and self.handle.value:
            lbm_batch_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def step(self, n):
        lbm_batch_step(self.handle, n)

    schedule = property(lambda self: lbm_batch_get_schedule(self.handle))

    def set_schedule(self, **kw):
        cur = self.schedule
        cur.update(kw)
        lbm_batch_set_schedule(self.handle, **cur)

    def autotune(self, trial_steps=20):
        return lbm_batch_autotune(self.handle, trial_steps)

    def set_barrier_budget(self, cycles):
        lbm_batch_set_barrier_budget(self.handle, cycles)


class Lattice:
    """Owns one context; methods forward to the lbm_* functions above."""

    def __init__(self, nx, ny, nz, walls, allocator="torch", stream=None, **kw):
        self.shape = (nz, ny, nx)
        self.params = make_params(nx, ny, nz, walls, **kw)
        self.ctx = lbm_create(self.params, allocator=allocator, stream=stream)
        # host fields of asynchronous uploads: not yet applied (their copies
        # may run until an apply makes the stream wait for them), and applied
        # (done once the stream has been synchronised)
        self._uploaded, self._applied = [], []

    def close(self):
        if self.ctx is not None and self.ctx.value:
            lbm_destroy(self.ctx)
        self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    constants = property(lambda self: lbm_get_constants(self.ctx))

    def set_fields(self, rho, u3, T):
        lbm_set_fields(self.ctx, rho, u3, T, self.shape)

    def upload_fields(self, rho, u3, T):
        """Asynchronous half of set_fields: the copy of the next fields runs
        on the context's copy stream beside the steps queued meanwhile; the
        arrays are kept here until a synchronising call after the
        apply_fields that uses them."""
        self._uploaded.append(lbm_upload_fields(self.ctx, rho, u3, T, self.shape))

    def apply_fields(self):
        lbm_apply_fields(self.ctx)
        self._applied += self._uploaded
        self._uploaded = []

    def set_populations(self, f, g):
        lbm_set_populations(self.ctx, f, g)

    def populations(self):
        return lbm_get_populations(self.ctx, self.shape)

    def populations_at(self, nodes):
        return lbm_get_populations_at(self.ctx, nodes)

    def step(self, n=1):
        lbm_step(self.ctx, n)

    def moments(self):
        out = lbm_moments(self.ctx, self.shape)
        self._applied = []
        return out

    def sample(self):
        lbm_sample(self.ctx)

    def dissipation_pdf(self, nbins=200, xmax=20.0, rms=None):
        return lbm_dissipation_pdf(self.ctx, nbins, xmax, rms)

    def nusselt_profile(self, axis=0):
        return lbm_nusselt_profile(self.ctx, self.shape, axis)

    def diagnostics(self, reset=False, raise_on_diverged=True):
        out = lbm_diagnostics(self.ctx, reset, raise_on_diverged)
        self._applied = []
        return out

    def synchronize(self):
        lbm_synchronize(self.ctx)
        self._applied = []

    def set_wait_budget(self, cycles):
        lbm_set_wait_budget(self.ctx, cycles)

    def save(self, path):
        lbm_save(self.ctx, path)

    def load(self, path):
        lbm_load(self.ctx, path)
