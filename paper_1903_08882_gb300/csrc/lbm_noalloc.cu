// Allocation-free variant of the diagnostics reduction (lbm_reduce_noalloc).
//
// The paper has no counterpart: this exists for callers that must not
// allocate device memory.  The ordinary path (lbm_sample) keeps its per-block
// partial sums in memory the context allocated at creation.  Here those
// partial sums live in one file-scope device array of fixed size instead, so
// the call itself allocates nothing.
//
// The array: LBM_NOALLOC_MAX_BLOCKS rows of LBM_NDIAG doubles (one row per
// reduction block) plus LBM_NDIAG + 1 accumulator slots, 233,672 bytes.  All
// calls share it and it keeps the contents of the last call; the accumulator
// slots, which must start at zero, are cleared at the start of every call.
// Two calls whose kernels overlap on a GPU (different streams, or different
// host threads) race on the array and give undefined sums.
//
// When the memory is taken: CUDA loads a library's device code per context,
// lazily by default (CUDA_MODULE_LOADING=LAZY), and the array is allocated
// when the code module holding it is loaded.  noalloc_setup() loads it: it
// looks up the array's device address with cudaGetSymbolAddress, with the
// device current, and caches the address per CUDA context (a reset device
// gets a new context, whose module may sit elsewhere, so the address is
// looked up again).  lbm_create runs it for its device, so a caller that
// creates a context holds the array from then on; otherwise the first
// lbm_reduce_noalloc call on a device does it, and that first call should
// come during set-up, before any stream capture.  In host code the array's
// name only stands for the device object: only the looked-up address is
// passed to kernels.
#include <algorithm>
#include <mutex>
#include <string>

#include <cuda.h>

#include "../../include/lbm.h"
#include "lbm_internal.h"

namespace {

constexpr int kRows = LBM_NOALLOC_MAX_BLOCKS;
constexpr int kScratchDoubles = kRows * lbm::kNDiag + lbm::kNDiag + 1;

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
struct Cached {
    unsigned long long ctx_id; // CUDA context the address belongs to (0: none yet)
    double *ptr;
};
Cached g_scratch[kMaxDevices] = {};

// Driver calls that name the current context, reached through the runtime
// (no link-time dependency on the driver library).
using CtxGetCurrentFn = CUresult (*)(CUcontext *);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long *);
CtxGetCurrentFn g_ctx_current = nullptr;
CtxGetIdFn g_ctx_id = nullptr;
bool g_driver_looked_up = false;

// ID of the calling thread's current context, 0 if none or unknown.
unsigned long long current_context_id() {
    if (!g_driver_looked_up) {
        g_driver_looked_up = true;
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_current = reinterpret_cast<CtxGetCurrentFn>(fn);
        fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_id = reinterpret_cast<CtxGetIdFn>(fn);
        cudaGetLastError();
    }
    if (!g_ctx_current || !g_ctx_id) return 0;
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (g_ctx_current(&c) != CUDA_SUCCESS || !c || g_ctx_id(c, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Device address of g_noalloc_scratch in the current device's context, looked
// up (which loads the module holding the array) once per context.
double *scratch_address(std::string &why) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        why = std::string("no usable CUDA device: ") + cudaGetErrorString(e);
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    const unsigned long long id = current_context_id();
    Cached &c = g_scratch[dev];
    if (!c.ptr || id == 0 || id != c.ctx_id) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) {
            why = std::string("cudaGetSymbolAddress failed: ") + cudaGetErrorString(e);
            return nullptr;
        }
        c.ptr = static_cast<double *>(ptr);
        // the lookup makes the primary context current if none was
        c.ctx_id = id ? id : current_context_id();
    }
    return c.ptr;
}

lbm_status reject(lbm_status s, const std::string &why) {
    lbm::set_global_error(why);
    return s;
}

} // namespace

namespace lbm {
cudaError_t noalloc_setup() {
    std::string why;
    return scratch_address(why) ? cudaSuccess : cudaErrorInitializationError;
}
} // namespace lbm

extern "C" lbm_status lbm_reduce_noalloc(const float *fields, int64_t stride, int nx, int ny, int nz,
                                         const lbm_wall *walls, double a_T, int blocks, double *sums,
                                         void *stream) {
    if (!fields || !sums || !walls) return reject(LBM_ERR_PARAM, "lbm_reduce_noalloc: NULL pointer");
    if (nx < 3 || ny < 3 || nz < 3) return reject(LBM_ERR_PARAM, "lbm_reduce_noalloc: every dimension must be >= 3");
    const double nodes = (double)nx * ny * nz;
    if (nodes > 2147482624.0)
        return reject(LBM_ERR_PARAM, "lbm_reduce_noalloc: lattice too large (at most 2^31 - 1024 nodes)");
    if (stride < (int64_t)nodes) return reject(LBM_ERR_PARAM, "lbm_reduce_noalloc: stride smaller than nx ny nz");
    if (!(a_T > -6.0 && a_T < 1.0)) return reject(LBM_ERR_PARAM, "lbm_reduce_noalloc: a_T outside (-6, 1)");
    for (int a = 0; a < 3; ++a) {
        const int k0 = walls[2 * a].kind, k1 = walls[2 * a + 1].kind;
        if (k0 < 0 || k0 > 2 || k1 < 0 || k1 > 2 || ((k0 == LBM_WALL_PERIODIC) != (k1 == LBM_WALL_PERIODIC)))
            return reject(LBM_ERR_PARAM, "lbm_reduce_noalloc: invalid wall kinds");
    }

    lbm::Geom G{};
    G.nx = nx;
    G.ny = ny;
    G.nz = nz;
    G.n = (uint32_t)nodes;
    G.nxy = (uint32_t)nx * (uint32_t)ny;
    G.stride = stride;
    G.mag_nx = UINT64_MAX / (uint32_t)nx + 1;
    G.mag_nxy = UINT64_MAX / G.nxy + 1;
    for (int a = 0; a < 3; ++a)
        if (walls[2 * a].kind == LBM_WALL_PERIODIC) G.periodic |= 1 << a;
    if (blocks == 0) blocks = std::min(lbm::diag_blocks(G), kRows);
    if (blocks < 0 || blocks > kRows)
        return reject(LBM_ERR_PARAM, "lbm_reduce_noalloc: blocks must lie in [0, " + std::to_string(kRows) +
                                         "]: the static scratch holds one row per block");

    lbm::Phys P{};
    float wallT[6];
    for (int f = 0; f < 6; ++f) {
        const bool dir = walls[f].kind == LBM_WALL_DIRICHLET;
        wallT[f] = dir ? (float)walls[f].T_w : 0.f;
        P.abbT[f] = dir ? (float)((6.0 + a_T) / 21.0 * walls[f].T_w) : 0.f;
        if (dir) P.dir_mask |= 1 << f;
    }

    std::string why;
    double *scratch = scratch_address(why);
    if (!scratch) return reject(LBM_ERR_CUDA, "lbm_reduce_noalloc: " + why);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    double *acc = scratch + (size_t)kRows * lbm::kNDiag;
    cudaError_t e = cudaMemsetAsync(acc, 0, (lbm::kNDiag + 1) * sizeof(double), st);
    if (e == cudaSuccess) e = lbm::launch_diag(fields, G, P, wallT, scratch, blocks, sums, acc, st);
    if (e != cudaSuccess) return reject(LBM_ERR_CUDA, std::string("lbm_reduce_noalloc: ") + cudaGetErrorString(e));
    return LBM_OK;
}
