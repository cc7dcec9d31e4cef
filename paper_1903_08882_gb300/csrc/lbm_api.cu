// Host side of the C ABI declared in include/lbm.h: parameter validation and
// derivation (Secs. 2.1-2.3), device memory, layout bookkeeping of the AA and
// pull schemes, launch sequencing, diagnostics finalisation and checkpoints.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/lbm.h"
#include "lbm_internal.h"

namespace {
// Named range on the profiler timeline (NVTX; a no-op unless a tool listens).
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
};
} // namespace

using namespace lbm;

namespace {

thread_local std::string g_create_error;

const int kMagic = 0x4c424d33; // "LBM3"

} // namespace

namespace lbm {
// Message returned by lbm_last_error(NULL) after a failed context-free call.
void set_global_error(const std::string &msg) { g_create_error = msg; }
} // namespace lbm

struct lbm_ctx {
    lbm_params p{};
    lbm_constants c{};
    Geom G{};
    Phys P{};
    float wallT[6]{};
    int dev = 0;
    cudaStream_t stream = nullptr;
    lbm_allocator alloc{};
    bool have_alloc = false;
    void *pop = nullptr, *pop2 = nullptr; // population buffer(s): 26 arrays of `stride` elements
    size_t pop_bytes = 0;
    float *mom = nullptr;                 // kMomArrays x stride floats
    size_t mom_bytes = 0;
    double *dsum = nullptr;               // partial[nblocks][kNDiag], raw[kNDiag], acc[kNDiag + 1]
    size_t dsum_bytes = 0;
    uint32_t *face = nullptr;             // flat indices of the nodes next to a face (AA odd step),
    size_t face_bytes = 0;                // those on a y or z face first
    uint32_t nface = 0, nface_yz = 0;
    bool staged = false;                  // AA steps without a sample use the staged kernels
    StagedGeom T{};
    int *flag = nullptr;                  // device error flag of the staged kernels
    int nblocks = 0;
    int elem = 4;   // bytes per flow population (f)
    int elem_g = 4; // bytes per thermal population (g)
    int parity = 0;        // AA: 0 natural (next step even), 1 reversed
    int64_t step = 0;
    int64_t sample_step = -1;
    int block = 256;
    float *hstage = nullptr; // pinned host staging, grown on demand
    size_t hstage_bytes = 0;
    // lbm_upload_fields / lbm_apply_fields: fields copied on their own stream
    // into a device staging buffer (rho, u, v, w, T: n doubles each)
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_uploaded = nullptr, ev_consumed = nullptr;
    double *fields = nullptr;
    size_t fields_bytes = 0;
    bool upload_pending = false, consumed_recorded = false;
    std::string err;

    float *host_stage(size_t bytes) {
        if (bytes <= hstage_bytes) return hstage;
        if (hstage) cudaFreeHost(hstage);
        hstage = nullptr;
        hstage_bytes = 0;
        void *ptr = nullptr;
        if (cudaMallocHost(&ptr, bytes) != cudaSuccess) return nullptr;
        hstage = static_cast<float *>(ptr);
        hstage_bytes = bytes;
        return hstage;
    }

    void *dalloc(size_t bytes) {
        if (have_alloc) return alloc.alloc(bytes, stream, alloc.user);
        void *ptr = nullptr;
        return cudaMalloc(&ptr, bytes) == cudaSuccess ? ptr : nullptr;
    }
    void dfree(void *ptr, size_t bytes) {
        if (!ptr) return;
        if (have_alloc) alloc.free(ptr, bytes, stream, alloc.user);
        else cudaFree(ptr);
    }
    double *raw() { return dsum + (size_t)nblocks * kNDiag; }
    double *acc() { return dsum + (size_t)nblocks * kNDiag + kNDiag; }
    void *fbase(int which) { return which ? pop2 : pop; }
    void *gbase(int which) {
        return static_cast<char *>(which ? pop2 : pop) + (size_t)19 * G.stride * elem;  // g follows the 19 f arrays
    }
    int layout() const { return p.streaming == LBM_STREAM_PULL2 ? 2 : (parity ? 1 : 0); }
};

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

lbm_status fail(lbm_ctx *ctx, lbm_status s, const std::string &msg) {
    if (ctx) ctx->err = msg;
    else g_create_error = msg;
    return s;
}

#define CK(ctx, call)                                                                          \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return fail(ctx, LBM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// Device staging buffer released on scope exit.
struct Scratch {
    lbm_ctx *ctx;
    void *ptr = nullptr;
    size_t bytes = 0;
    Scratch(lbm_ctx *c, size_t b) : ctx(c), bytes(b) { ptr = c->dalloc(b); }
    ~Scratch() {
        if (ptr) {
            cudaStreamSynchronize(ctx->stream);
            ctx->dfree(ptr, bytes);
        }
    }
};

lbm_status validate_and_derive(const lbm_params &p, lbm_constants &c, std::string &why) {
    if (p.nx < 3 || p.ny < 3 || p.nz < 3) {
        why = "every lattice dimension must be >= 3";
        return LBM_ERR_PARAM;
    }
    // 32-bit node indices; wrap-around offsets of a periodic axis span up to the
    // whole lattice and are 32-bit signed
    const double nodes = (double)p.nx * p.ny * p.nz;
    const bool any_periodic = p.wall[0].kind == LBM_WALL_PERIODIC || p.wall[2].kind == LBM_WALL_PERIODIC ||
                              p.wall[4].kind == LBM_WALL_PERIODIC;
    if (nodes > (any_periodic ? 2147482624.0 : 4294966272.0)) {
        why = "lattice too large for 32-bit node indices (2^32 - 1024 nodes, 2^31 - 1024 with a periodic axis)";
        return LBM_ERR_PARAM;
    }
    for (int a = 0; a < 3; ++a) {
        const int k0 = p.wall[2 * a].kind, k1 = p.wall[2 * a + 1].kind;
        if (k0 < 0 || k0 > 2 || k1 < 0 || k1 > 2) {
            why = "unknown wall kind";
            return LBM_ERR_PARAM;
        }
        if ((k0 == LBM_WALL_PERIODIC) != (k1 == LBM_WALL_PERIODIC)) {
            why = "an axis must be periodic on both faces or on neither";
            return LBM_ERR_PARAM;
        }
    }
    if (p.storage < 0 || p.storage > 3 || p.streaming < 0 || p.streaming > 1) {
        why = "unknown storage or streaming scheme";
        return LBM_ERR_PARAM;
    }
    if (p.block_size != 0 && (p.block_size < 32 || p.block_size > 256 || p.block_size % 32)) {
        why = "block_size must be 0 or a multiple of 32 in [32, 256]";
        return LBM_ERR_PARAM;
    }
    if (p.nodes_per_thread < 0 || p.nodes_per_thread > 2) {
        why = "nodes_per_thread must be 0, 1 or 2";
        return LBM_ERR_PARAM;
    }
    if (p.pipeline < 0 || p.pipeline > 2) {
        why = "pipeline must be 0, 1 or 2";
        return LBM_ERR_PARAM;
    }
    if (p.diag_every < 0) {
        why = "diag_every must be >= 0";
        return LBM_ERR_PARAM;
    }
    if (!(p.U > 0.0 && p.U <= 0.2)) {
        why = "U must lie in (0, 0.2]";
        return LBM_ERR_PARAM;
    }
    const double H = p.H > 0 ? p.H : (double)p.nz;
    double nu, kappa, gbeta;
    if (p.derive) {
        if (!(p.Ra > 0 && p.Pr > 0)) {
            why = "Ra and Pr must be positive";
            return LBM_ERR_PARAM;
        }
        // free-fall scaling, Sec. 2.1 (dT = 1)
        nu = p.U * H * std::sqrt(p.Pr / p.Ra);
        kappa = nu / p.Pr;
        gbeta = p.U * p.U / H;
    } else {
        nu = p.nu;
        kappa = p.kappa;
        gbeta = p.gbeta;
    }
    // Sec. 2.2: nu = c_s^2 (tau_f - 1/2), s_e = 1/tau_f, s_q = 8 (2 tau_f - 1)/(8 tau_f - 1)
    const double tau = 3.0 * nu + 0.5;
    if (!(tau > 0.5) || !std::isfinite(tau)) {
        why = "tau_f = 3 nu + 1/2 must exceed 1/2";
        return LBM_ERR_PARAM;
    }
    // Sec. 2.3: q_kappa = 3 - sqrt3, q_e = q_nu = 4 sqrt3 - 6, a_T = 42 sqrt3 kappa - 6
    const double s3 = std::sqrt(3.0);
    const double aT = 42.0 * s3 * kappa - 6.0;
    if (!(aT > -6.0 && aT < 1.0)) {
        why = "a_T = 42 sqrt(3) kappa - 6 must lie in (-6, 1), i.e. 0 < kappa < 1/(6 sqrt 3)";
        return LBM_ERR_PARAM;
    }
    c.nu = nu;
    c.kappa = kappa;
    c.gbeta = gbeta;
    c.tau_f = tau;
    c.s_e = 1.0 / tau;
    c.s_q = 8.0 * (2.0 * tau - 1.0) / (8.0 * tau - 1.0);
    c.q_kappa = 3.0 - s3;
    c.q_e = c.q_nu = 4.0 * s3 - 6.0;
    c.a_T = aT;
    c.w0_T = (1.0 - aT) / 7.0;
    c.w1_T = (6.0 + aT) / 42.0;
    c.H = H;
    c.U = p.U;
    c.nodes = (int64_t)p.nx * p.ny * p.nz;
    return LBM_OK;
}

// ceil(2^64 / d) for fast_div; d = 1 is encoded as 0.
uint64_t magic_of(uint32_t d) { return d <= 1 ? 0 : UINT64_MAX / d + 1; }

void finalize(const lbm_ctx *ctx, const double *r, double &E, double &rms_drho, double &rms_div,
              double &Re, double &Rew, double &Nuv, double &Nuk, double &Nut, double *Nuf,
              double *Nul) {
    const double n = r[0] > 0 ? r[0] : 1.0;
    const double H = ctx->c.H, U = ctx->c.U, nu = ctx->c.nu, ka = ctx->c.kappa;
    const double area[6] = {(double)ctx->p.ny * ctx->p.nz, (double)ctx->p.ny * ctx->p.nz,
                            (double)ctx->p.nx * ctx->p.nz, (double)ctx->p.nx * ctx->p.nz,
                            (double)ctx->p.nx * ctx->p.ny, (double)ctx->p.nx * ctx->p.ny};
    rms_drho = std::sqrt(r[1] / n);
    E = 0.5 * r[2] / n / (U * U);
    Re = std::sqrt(r[2] / n) * H / nu;
    Rew = std::sqrt(r[3] / n) * H / nu;
    Nuv = 1.0 + r[4] / n * H / ka;
    Nuk = 1.0 + nu * r[5] / n * H * H / (ka * U * U);
    Nut = r[6] / n * H * H;
    rms_div = std::sqrt(r[7] / n) * H / U;
    for (int f = 0; f < 6; ++f) {
        if (Nuf) Nuf[f] = H * r[8 + f] / area[f];
        if (Nul) Nul[f] = r[18 + f] / area[f] * H / ka;
    }
}

lbm_status release(lbm_ctx *ctx) {
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    ctx->dfree(ctx->pop, ctx->pop_bytes);
    ctx->dfree(ctx->pop2, ctx->pop_bytes);
    ctx->dfree(ctx->mom, ctx->mom_bytes);
    ctx->dfree(ctx->dsum, ctx->dsum_bytes);
    ctx->dfree(ctx->face, ctx->face_bytes);
    ctx->dfree(ctx->flag, 256);
    ctx->face = nullptr;
    ctx->flag = nullptr;
    ctx->pop = ctx->pop2 = nullptr;
    ctx->mom = nullptr;
    ctx->dsum = nullptr;
    if (ctx->hstage) cudaFreeHost(ctx->hstage);
    ctx->hstage = nullptr;
    ctx->hstage_bytes = 0;
    if (ctx->copy_stream) {
        cudaStreamSynchronize(ctx->copy_stream);
        cudaStreamDestroy(ctx->copy_stream);
    }
    if (ctx->ev_uploaded) cudaEventDestroy(ctx->ev_uploaded);
    if (ctx->ev_consumed) cudaEventDestroy(ctx->ev_consumed);
    ctx->dfree(ctx->fields, ctx->fields_bytes);
    ctx->copy_stream = nullptr;
    ctx->ev_uploaded = ctx->ev_consumed = nullptr;
    ctx->fields = nullptr;
    ctx->fields_bytes = 0;
    return LBM_OK;
}

// Natural-order float populations [26][n] at host -> device layout.
lbm_status upload_natural(lbm_ctx *ctx, const float *host) {
    const size_t bytes = (size_t)26 * (size_t)ctx->c.nodes * sizeof(float);
    Scratch st(ctx, bytes);
    if (!st.ptr) return fail(ctx, LBM_ERR_OOM, "staging allocation failed");
    CK(ctx, cudaMemcpyAsync(st.ptr, host, bytes, cudaMemcpyHostToDevice, ctx->stream));
    int which = 0;
    if (ctx->p.streaming == LBM_STREAM_AA) ctx->parity = 0;
    const int layout = ctx->p.streaming == LBM_STREAM_PULL2 ? 2 : 0;
    CK(ctx, launch_convert(ctx->p.storage, 0, (float *)st.ptr, ctx->fbase(which), ctx->gbase(which),
                           ctx->G, ctx->P, layout, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    return LBM_OK;
}

lbm_status sample_into(lbm_ctx *ctx) {
    CK(ctx, launch_diag(ctx->mom, ctx->G, ctx->P, ctx->wallT, ctx->dsum, ctx->nblocks, ctx->raw(),
                        ctx->acc(), ctx->stream));
    ctx->sample_step = ctx->step;
    return LBM_OK;
}

} // namespace

extern "C" {

// Read (and clear) the staged kernels' error flag.  Synchronises the stream.
static lbm_status check_flag(lbm_ctx *ctx) {
    if (!ctx->staged) return LBM_OK;
    int h = 0;
    CK(ctx, cudaMemcpyAsync(&h, ctx->flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    if (!h) return LBM_OK;
    CK(ctx, cudaMemsetAsync(ctx->flag, 0, sizeof(int), ctx->stream));
    return fail(ctx, LBM_ERR_TIMEOUT, "a staged step kernel's pipeline wait ran out of its cycle budget; the state is undefined");
}

lbm_status lbm_create(const lbm_params *params, const lbm_allocator *alloc, void *stream, lbm_ctx **out) {
    Range range("lbm_create");
    if (!out) return fail(nullptr, LBM_ERR_PARAM, "out is NULL");
    *out = nullptr;
    if (!params) return fail(nullptr, LBM_ERR_PARAM, "params is NULL");
    lbm_constants c{};
    std::string why;
    if (validate_and_derive(*params, c, why) != LBM_OK) return fail(nullptr, LBM_ERR_PARAM, why);
    if (alloc && (!alloc->alloc || !alloc->free))
        return fail(nullptr, LBM_ERR_PARAM, "allocator needs both alloc and free");

    lbm_ctx *ctx = new lbm_ctx();
    ctx->p = *params;
    ctx->c = c;
    if (alloc) {
        ctx->alloc = *alloc;
        ctx->have_alloc = true;
    }
    ctx->stream = static_cast<cudaStream_t>(stream);
    if (cudaGetDevice(&ctx->dev) != cudaSuccess) {
        delete ctx;
        return fail(nullptr, LBM_ERR_CUDA, "no CUDA device");
    }
    // take the static scratch of lbm_reduce_noalloc on this device now, at set-up
    if (noalloc_setup() != cudaSuccess) {
        delete ctx;
        return fail(nullptr, LBM_ERR_CUDA, "cannot load the library's device code on this device");
    }
    ctx->block = params->block_size ? params->block_size : 128;
    ctx->elem = params->storage == LBM_FP32 ? 4 : 2;
    ctx->elem_g = (params->storage == LBM_FP32 || params->storage == LBM_FP16M) ? 4 : 2;

    Geom &G = ctx->G;
    G.nx = params->nx;
    G.ny = params->ny;
    G.nz = params->nz;
    G.n = (uint32_t)c.nodes;
    G.nxy = (uint32_t)params->nx * (uint32_t)params->ny;
    G.stride = (c.nodes + 127) / 128 * 128;
    G.mag_nx = magic_of((uint32_t)params->nx);
    G.mag_nxy = magic_of(G.nxy);
    G.periodic = 0;
    for (int a = 0; a < 3; ++a)
        if (params->wall[2 * a].kind == LBM_WALL_PERIODIC) G.periodic |= 1 << a;
    G.nix = (uint32_t)(params->nx - 2);
    G.nixy = G.nix * (uint32_t)(params->ny - 2);
    G.ni = G.nixy * (uint32_t)(params->nz - 2);
    G.mag_nix = magic_of(G.nix);
    G.mag_nixy = magic_of(G.nixy);
    G.cpp = ((uint32_t)params->nx * (uint32_t)(params->ny - 2) + 63u) / 64u;
    G.mag_cpp = magic_of(G.cpp);
    {
        const int ex[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
        const int ey[19] = {0, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 1, -1, 1, -1};
        const int ez[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1};
        for (int i = 0; i < 19; ++i) G.off[i] = ex[i] + params->nx * ey[i] + (int)G.nxy * ez[i];
    }

    Phys &P = ctx->P;
    P.s_e = (float)c.s_e;
    P.s_q = (float)c.s_q;
    P.q_k = (float)c.q_kappa;
    P.q_e = (float)c.q_e;
    P.a_T = (float)c.a_T;
    P.gbeta = (float)c.gbeta;
    for (int a = 0; a < 3; ++a) P.bf[a] = (float)params->body_force[a];
    P.dir_mask = 0;
    for (int f = 0; f < 6; ++f) {
        const bool dir = params->wall[f].kind == LBM_WALL_DIRICHLET;
        ctx->wallT[f] = dir ? (float)params->wall[f].T_w : 0.f;
        P.abbT[f] = dir ? (float)((6.0 + c.a_T) / 21.0 * params->wall[f].T_w) : 0.f;
        if (dir) P.dir_mask |= 1 << f;
    }

    ctx->pop_bytes = (size_t)G.stride * (19 * (size_t)ctx->elem + 7 * (size_t)ctx->elem_g);
    ctx->mom_bytes = (size_t)kMomArrays * G.stride * sizeof(float);
    ctx->nblocks = diag_blocks(G);
    ctx->dsum_bytes = ((size_t)ctx->nblocks * kNDiag + 2 * kNDiag + 1) * sizeof(double);
    // nodes next to a face: the general-path share of the AA odd step; those
    // on a y or z face first (the staged odd kernel handles the x faces itself)
    std::vector<uint32_t> face;
    face.reserve((size_t)(c.nodes - G.ni));
    for (int pass = 0; pass < 2; ++pass) {
        for (int z = 0; z < G.nz; ++z)
            for (int y = 0; y < G.ny; ++y)
                for (int x = 0; x < G.nx; ++x) {
                    const bool yz = y == 0 || z == 0 || y == G.ny - 1 || z == G.nz - 1;
                    const bool xf = x == 0 || x == G.nx - 1;
                    if (pass == 0 ? yz : (xf && !yz))
                        face.push_back((uint32_t)x + (uint32_t)G.nx * ((uint32_t)y + (uint32_t)G.ny * (uint32_t)z));
                }
        if (pass == 0) ctx->nface_yz = (uint32_t)face.size();
    }
    ctx->nface = (uint32_t)face.size();
    ctx->face_bytes = face.size() * sizeof(uint32_t);
    ctx->face = (uint32_t *)ctx->dalloc(ctx->face_bytes);
    ctx->pop = ctx->dalloc(ctx->pop_bytes);
    if (params->streaming == LBM_STREAM_PULL2) ctx->pop2 = ctx->dalloc(ctx->pop_bytes);
    ctx->mom = (float *)ctx->dalloc(ctx->mom_bytes);
    ctx->dsum = (double *)ctx->dalloc(ctx->dsum_bytes);
    ctx->flag = (int *)ctx->dalloc(256);
    if (!ctx->pop || !ctx->mom || !ctx->dsum || !ctx->face || !ctx->flag ||
        (params->streaming == LBM_STREAM_PULL2 && !ctx->pop2)) {
        release(ctx);
        delete ctx;
        return fail(nullptr, LBM_ERR_OOM, "device allocation failed");
    }
    ctx->c.device_bytes = (int64_t)(ctx->pop_bytes * (ctx->pop2 ? 2 : 1) + ctx->mom_bytes + ctx->dsum_bytes +
                                    ctx->face_bytes + 256);
    // staged kernels: AA streaming, 16-byte aligned arrays (bulk copies), and
    // at least one block of them resident per SM
    // (library default: staged for the 2-byte flow storages, where they
    // measure faster than the register kernels; register kernels for FP32,
    // whose register kernels already run at the copy bandwidth)
    const bool want = params->pipeline == 2 || (params->pipeline == 0 && params->storage != LBM_FP32);
    if (params->streaming == LBM_STREAM_AA && want && ((uintptr_t)ctx->pop & 15) == 0) {
        int per_sm = 0, nsm = 0;
        if (staged_prepare(params->storage, &per_sm) == cudaSuccess && per_sm > 0 &&
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->dev) == cudaSuccess && nsm > 0) {
            const uint32_t tile_even = (uint32_t)staged_tile_nodes(0), tile_odd = (uint32_t)staged_tile_nodes(1);
            StagedGeom &T = ctx->T;
            T.even_tiles = (uint32_t)((c.nodes + tile_even - 1) / tile_even);
            T.tpp = (G.nxy - 2u * (uint32_t)G.nx + 1u + tile_odd - 1u) / tile_odd;
            T.mag_tpp = magic_of(T.tpp);
            T.odd_tiles = T.tpp * (uint32_t)(G.nz - 2);
            T.grid = nsm * per_sm; // persistent: every block resident
            T.xf = G.nx >= staged_xf_min_nx() ? 1 : 0;
            T.budget = 1ll << 31;
            staged_store_offsets(params->storage, G, T);
            ctx->staged = true;
        }
        cudaGetLastError(); // a failed opt-in leaves the register kernels in use
    }
    if (params->pipeline == 2 && !ctx->staged) {
        release(ctx);
        delete ctx;
        return fail(nullptr, LBM_ERR_PARAM,
                    "staged kernels unavailable (they need AA streaming, 16-byte aligned memory and room on an SM)");
    }
    // rest state: all deviations zero (f = w rho0, g = 0); pad entries zero too
    cudaError_t e = cudaMemsetAsync(ctx->pop, 0, ctx->pop_bytes, ctx->stream);
    if (e == cudaSuccess && ctx->pop2) e = cudaMemsetAsync(ctx->pop2, 0, ctx->pop_bytes, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->mom, 0, ctx->mom_bytes, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->dsum, 0, ctx->dsum_bytes, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->flag, 0, 256, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ctx->face, face.data(), ctx->face_bytes, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        release(ctx);
        delete ctx;
        return fail(nullptr, LBM_ERR_CUDA, std::string("initialisation: ") + cudaGetErrorString(e));
    }
    if (params->streaming == LBM_STREAM_PULL2) {
        // the pull layout stores wall links as reflected values: load the rest
        // state through the layout conversion so that T = 0 next to walls too
        std::vector<float> zero((size_t)26 * (size_t)c.nodes, 0.f);
        if (upload_natural(ctx, zero.data()) != LBM_OK) {
            g_create_error = ctx->err;
            release(ctx);
            delete ctx;
            return LBM_ERR_CUDA;
        }
    }
    *out = ctx;
    return LBM_OK;
}

void lbm_destroy(lbm_ctx *ctx) {
    if (!ctx) return;
    DeviceGuard dg(ctx->dev);
    release(ctx);
    delete ctx;
}

const char *lbm_last_error(const lbm_ctx *ctx) {
    return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

lbm_status lbm_get_constants(const lbm_ctx *ctx, lbm_constants *out) {
    if (!ctx || !out) return LBM_ERR_PARAM;
    *out = ctx->c;
    return LBM_OK;
}

lbm_status lbm_upload_fields(lbm_ctx *ctx, const double *rho, const double *u3, const double *T) {
    if (!ctx || !rho || !u3 || !T) return ctx ? fail(ctx, LBM_ERR_PARAM, "NULL array") : LBM_ERR_PARAM;
    if (ctx->p.streaming != LBM_STREAM_AA) return fail(ctx, LBM_ERR_PARAM, "lbm_upload_fields needs AA streaming");
    DeviceGuard dg(ctx->dev);
    const size_t n = (size_t)ctx->c.nodes;
    if (!ctx->copy_stream) {
        CK(ctx, cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
        CK(ctx, cudaEventCreateWithFlags(&ctx->ev_uploaded, cudaEventDisableTiming));
        CK(ctx, cudaEventCreateWithFlags(&ctx->ev_consumed, cudaEventDisableTiming));
    }
    if (!ctx->fields) {
        ctx->fields = static_cast<double *>(ctx->dalloc(5 * n * sizeof(double)));
        if (!ctx->fields) return fail(ctx, LBM_ERR_OOM, "field staging allocation failed");
        ctx->fields_bytes = 5 * n * sizeof(double);
    }
    // the staging buffer may still feed the kernel of the last lbm_apply_fields
    if (ctx->consumed_recorded) CK(ctx, cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_consumed, 0));
    double *d = ctx->fields;
    CK(ctx, cudaMemcpyAsync(d, rho, n * sizeof(double), cudaMemcpyHostToDevice, ctx->copy_stream));
    CK(ctx, cudaMemcpyAsync(d + n, u3, 3 * n * sizeof(double), cudaMemcpyHostToDevice, ctx->copy_stream));
    CK(ctx, cudaMemcpyAsync(d + 4 * n, T, n * sizeof(double), cudaMemcpyHostToDevice, ctx->copy_stream));
    CK(ctx, cudaEventRecord(ctx->ev_uploaded, ctx->copy_stream));
    ctx->upload_pending = true;
    return LBM_OK;
}

lbm_status lbm_apply_fields(lbm_ctx *ctx) {
    if (!ctx) return LBM_ERR_PARAM;
    if (!ctx->upload_pending) return fail(ctx, LBM_ERR_STATE, "lbm_apply_fields: no fields uploaded since the last call");
    DeviceGuard dg(ctx->dev);
    const size_t n = (size_t)ctx->c.nodes;
    double *d = ctx->fields;
    CK(ctx, cudaStreamWaitEvent(ctx->stream, ctx->ev_uploaded, 0));
    CK(ctx, launch_fields_natural(ctx->p.storage, d, d + n, d + 4 * n, ctx->fbase(0), ctx->gbase(0), ctx->G,
                                  ctx->P, ctx->stream));
    CK(ctx, cudaEventRecord(ctx->ev_consumed, ctx->stream));
    ctx->consumed_recorded = true;
    ctx->upload_pending = false;
    ctx->parity = 0;
    return LBM_OK;
}

lbm_status lbm_set_populations(lbm_ctx *ctx, const double *f19, const double *g7) {
    if (!ctx || !f19 || !g7) return ctx ? fail(ctx, LBM_ERR_PARAM, "NULL array") : LBM_ERR_PARAM;
    DeviceGuard dg(ctx->dev);
    const size_t n = (size_t)ctx->c.nodes;
    float *host = ctx->host_stage((size_t)26 * n * sizeof(float));
    if (!host) return fail(ctx, LBM_ERR_OOM, "pinned host staging allocation failed");
    CK(ctx, cudaStreamSynchronize(ctx->stream)); // the staging may still feed an earlier copy
    for (int i = 0; i < 19; ++i) {
        const double w = i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0);
        for (size_t k = 0; k < n; ++k) host[i * n + k] = (float)(f19[i * n + k] - w);
    }
    for (int i = 0; i < 7; ++i)
        for (size_t k = 0; k < n; ++k) host[(19 + i) * n + k] = (float)g7[i * n + k];
    return upload_natural(ctx, host);
}

lbm_status lbm_set_fields(lbm_ctx *ctx, const double *rho, const double *u3, const double *T) {
    if (!ctx || !rho || !u3 || !T) return ctx ? fail(ctx, LBM_ERR_PARAM, "NULL array") : LBM_ERR_PARAM;
    DeviceGuard dg(ctx->dev);
    const size_t n = (size_t)ctx->c.nodes;
    if (ctx->p.streaming == LBM_STREAM_AA) {
        // the fields go to the device as they are (FP64) into the sample
        // arrays, which the next sample rewrites anyway (5 doubles fit in
        // their 11 floats per node), and one kernel writes the equilibrium
        // state into the natural layout: no allocation, no host conversion
        static_assert(kMomArrays * sizeof(float) >= 5 * sizeof(double), "sample arrays too small for the fields");
        double *d = reinterpret_cast<double *>(ctx->mom);
        CK(ctx, cudaMemcpyAsync(d, rho, n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
        CK(ctx, cudaMemcpyAsync(d + n, u3, 3 * n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
        CK(ctx, cudaMemcpyAsync(d + 4 * n, T, n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
        CK(ctx, launch_fields_natural(ctx->p.storage, d, d + n, d + 4 * n, ctx->fbase(0), ctx->gbase(0), ctx->G,
                                      ctx->P, ctx->stream));
        ctx->parity = 0;
        CK(ctx, cudaStreamSynchronize(ctx->stream));
        return LBM_OK;
    }
    float *fields = ctx->host_stage(5 * n * sizeof(float));
    if (!fields) return fail(ctx, LBM_ERR_OOM, "pinned host staging allocation failed");
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    for (size_t k = 0; k < n; ++k) {
        fields[k] = (float)(rho[k] - 1.0);
        fields[n + k] = (float)u3[k];
        fields[2 * n + k] = (float)u3[n + k];
        fields[3 * n + k] = (float)u3[2 * n + k];
        fields[4 * n + k] = (float)T[k];
    }
    Scratch fd(ctx, 5 * n * sizeof(float));
    Scratch st(ctx, (size_t)26 * n * sizeof(float));
    if (!fd.ptr || !st.ptr) return fail(ctx, LBM_ERR_OOM, "staging allocation failed");
    CK(ctx, cudaMemcpyAsync(fd.ptr, fields, 5 * n * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    CK(ctx, launch_equilibrium((float *)st.ptr, (const float *)fd.ptr, (uint32_t)n, ctx->P, ctx->stream));
    // the pull layout stores wall links as reflected values (layout conversion)
    CK(ctx, launch_convert(ctx->p.storage, 0, (float *)st.ptr, ctx->fbase(0), ctx->gbase(0), ctx->G, ctx->P, 2,
                           ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    return LBM_OK;
}

lbm_status lbm_get_populations(lbm_ctx *ctx, double *f19, double *g7) {
    if (!ctx || !f19 || !g7) return ctx ? fail(ctx, LBM_ERR_PARAM, "NULL array") : LBM_ERR_PARAM;
    DeviceGuard dg(ctx->dev);
    const size_t n = (size_t)ctx->c.nodes;
    Scratch st(ctx, (size_t)26 * n * sizeof(float));
    if (!st.ptr) return fail(ctx, LBM_ERR_OOM, "staging allocation failed");
    CK(ctx, launch_convert(ctx->p.storage, 1, (float *)st.ptr, ctx->fbase(0), ctx->gbase(0), ctx->G,
                           ctx->P, ctx->layout(), ctx->stream));
    float *host = ctx->host_stage((size_t)26 * n * sizeof(float));
    if (!host) return fail(ctx, LBM_ERR_OOM, "pinned host staging allocation failed");
    CK(ctx, cudaMemcpyAsync(host, st.ptr, (size_t)26 * n * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    if (lbm_status fs = check_flag(ctx); fs != LBM_OK) return fs;
    for (int i = 0; i < 19; ++i) {
        const double w = i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0);
        for (size_t k = 0; k < n; ++k) f19[i * n + k] = (double)host[i * n + k] + w;
    }
    for (int i = 0; i < 7; ++i)
        for (size_t k = 0; k < n; ++k) g7[i * n + k] = (double)host[(19 + i) * n + k];
    return LBM_OK;
}

lbm_status lbm_get_populations_at(lbm_ctx *ctx, const int64_t *nodes, int64_t count, double *f19,
                                  double *g7) {
    if (!ctx) return LBM_ERR_PARAM;
    if (count < 0 || (count > 0 && (!nodes || !f19 || !g7))) return fail(ctx, LBM_ERR_PARAM, "bad arguments");
    if (count == 0) return LBM_OK;
    for (int64_t k = 0; k < count; ++k)
        if (nodes[k] < 0 || nodes[k] >= ctx->c.nodes) return fail(ctx, LBM_ERR_PARAM, "node index out of range");
    DeviceGuard dg(ctx->dev);
    Scratch dn(ctx, (size_t)count * sizeof(int64_t));
    Scratch dout(ctx, (size_t)count * 26 * sizeof(float));
    if (!dn.ptr || !dout.ptr) return fail(ctx, LBM_ERR_OOM, "staging allocation failed");
    CK(ctx, cudaMemcpyAsync(dn.ptr, nodes, count * sizeof(int64_t), cudaMemcpyHostToDevice, ctx->stream));
    CK(ctx, launch_gather(ctx->p.storage, (float *)dout.ptr, (const int64_t *)dn.ptr, count, ctx->fbase(0),
                          ctx->gbase(0), ctx->G, ctx->P, ctx->layout(), ctx->stream));
    std::vector<float> host((size_t)count * 26);
    CK(ctx, cudaMemcpyAsync(host.data(), dout.ptr, host.size() * sizeof(float), cudaMemcpyDeviceToHost,
                            ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    if (lbm_status fs = check_flag(ctx); fs != LBM_OK) return fs;
    for (int64_t k = 0; k < count; ++k) {
        for (int i = 0; i < 19; ++i) {
            const double w = i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0);
            f19[k * 19 + i] = (double)host[k * 26 + i] + w;
        }
        for (int i = 0; i < 7; ++i) g7[k * 7 + i] = (double)host[k * 26 + 19 + i];
    }
    return LBM_OK;
}

lbm_status lbm_step(lbm_ctx *ctx, int64_t nsteps) {
    Range range("lbm_step");
    if (!ctx) return LBM_ERR_PARAM;
    if (nsteps < 0) return fail(ctx, LBM_ERR_PARAM, "negative step count");
    DeviceGuard dg(ctx->dev);
    StepArgs a{};
    a.storage = ctx->p.storage;
    a.scheme = ctx->p.streaming == LBM_STREAM_PULL2 ? 1 : 0;
    a.block = ctx->block;
    a.wide = ctx->p.nodes_per_thread != 1;
    a.G = ctx->G;
    a.P = ctx->P;
    a.face = ctx->face;
    a.nface = ctx->nface;
    a.nface_yz = ctx->nface_yz;
    a.T = ctx->T;
    a.err = ctx->flag;
    a.stream = ctx->stream;
    for (int64_t t = 0; t < nsteps; ++t) {
        const bool sample = ctx->p.diag_every > 0 && ctx->step % ctx->p.diag_every == 0;
        a.mom = sample ? ctx->mom : nullptr;
        a.parity = ctx->parity;
        a.P.t = (uint32_t)ctx->step;
        a.f = ctx->fbase(0);
        a.g = ctx->gbase(0);
        a.f2 = ctx->fbase(1);
        a.g2 = ctx->gbase(1);
        if (ctx->staged && !sample) CK(ctx, launch_staged(a));
        else CK(ctx, launch_step(a));
        if (sample) {
            lbm_status s = sample_into(ctx);
            if (s != LBM_OK) return s;
        }
        if (a.scheme == 0) ctx->parity ^= 1;
        else std::swap(ctx->pop, ctx->pop2);
        ctx->step += 1;
    }
    return LBM_OK;
}

lbm_status lbm_moments(lbm_ctx *ctx, double *rho, double *u3, double *T) {
    if (!ctx || !rho || !u3 || !T) return ctx ? fail(ctx, LBM_ERR_PARAM, "NULL array") : LBM_ERR_PARAM;
    DeviceGuard dg(ctx->dev);
    CK(ctx, launch_convert(ctx->p.storage, 2, ctx->mom, ctx->fbase(0), ctx->gbase(0), ctx->G, ctx->P,
                           ctx->layout(), ctx->stream));
    const size_t n = (size_t)ctx->c.nodes, s = (size_t)ctx->G.stride;
    float *host = ctx->host_stage(5 * s * sizeof(float));
    if (!host) return fail(ctx, LBM_ERR_OOM, "pinned host staging allocation failed");
    CK(ctx, cudaMemcpyAsync(host, ctx->mom, 5 * s * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    if (lbm_status fs = check_flag(ctx); fs != LBM_OK) return fs;
    for (size_t k = 0; k < n; ++k) {
        rho[k] = 1.0 + (double)host[k];
        u3[k] = host[s + k];
        u3[n + k] = host[2 * s + k];
        u3[2 * n + k] = host[3 * s + k];
        T[k] = host[4 * s + k];
    }
    return LBM_OK;
}

lbm_status lbm_dissipation_pdf(lbm_ctx *ctx, int nbins, double xmax, const double *rms_in, double *rms_out,
                               uint64_t *counts_u, uint64_t *counts_T) {
    if (!ctx) return LBM_ERR_PARAM;
    if (nbins < 1 || nbins > kPdfMaxBins) return fail(ctx, LBM_ERR_PARAM, "nbins must lie in [1, 4096]");
    if (!(xmax > 0.0) || !std::isfinite(xmax)) return fail(ctx, LBM_ERR_PARAM, "xmax must be positive");
    if (!counts_u || !counts_T) return fail(ctx, LBM_ERR_PARAM, "NULL count array");
    if (rms_in && (!(rms_in[0] >= 0.0) || !(rms_in[1] >= 0.0)))
        return fail(ctx, LBM_ERR_PARAM, "rms_in must be >= 0");
    DeviceGuard dg(ctx->dev);
    // moments of the current state into the sample arrays, as lbm_moments does
    CK(ctx, launch_convert(ctx->p.storage, 2, ctx->mom, ctx->fbase(0), ctx->gbase(0), ctx->G, ctx->P,
                           ctx->layout(), ctx->stream));
    const size_t bytes = (2 + 2 * (size_t)nbins) * sizeof(double);
    Scratch sc(ctx, bytes);
    if (!sc.ptr) return fail(ctx, LBM_ERR_OOM, "staging allocation failed");
    double *sums = static_cast<double *>(sc.ptr);
    unsigned long long *counts = reinterpret_cast<unsigned long long *>(sums + 2);
    CK(ctx, cudaMemsetAsync(sc.ptr, 0, bytes, ctx->stream));
    const float nu = (float)ctx->c.nu, ka = (float)ctx->c.kappa;
    double rms[2];
    if (rms_in) {
        rms[0] = rms_in[0];
        rms[1] = rms_in[1];
    } else {
        CK(ctx, launch_eps_sq(ctx->mom, ctx->G, ctx->P, ctx->wallT, nu, ka, sums, ctx->stream));
        double h[2];
        CK(ctx, cudaMemcpyAsync(h, sums, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
        CK(ctx, cudaStreamSynchronize(ctx->stream));
        rms[0] = std::sqrt(h[0] / (double)ctx->c.nodes);
        rms[1] = std::sqrt(h[1] / (double)ctx->c.nodes);
    }
    const double scale_u = rms[0] > 0.0 ? nbins / (xmax * rms[0]) : 0.0;
    const double scale_t = rms[1] > 0.0 ? nbins / (xmax * rms[1]) : 0.0;
    CK(ctx, launch_eps_hist(ctx->mom, ctx->G, ctx->P, ctx->wallT, nu, ka, scale_u, scale_t, nbins, counts,
                            ctx->stream));
    std::vector<unsigned long long> host(2 * (size_t)nbins);
    CK(ctx, cudaMemcpyAsync(host.data(), counts, host.size() * sizeof(unsigned long long),
                            cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    if (lbm_status fs = check_flag(ctx); fs != LBM_OK) return fs;
    for (int i = 0; i < nbins; ++i) {
        counts_u[i] = host[i];
        counts_T[i] = host[(size_t)nbins + i];
    }
    if (rms_out) {
        rms_out[0] = rms[0];
        rms_out[1] = rms[1];
    }
    return LBM_OK;
}

lbm_status lbm_nusselt_profile(lbm_ctx *ctx, int axis, double *profile, double *nu_mid) {
    if (!ctx) return LBM_ERR_PARAM;
    if (axis < 0 || axis > 2) return fail(ctx, LBM_ERR_PARAM, "axis must be 0, 1 or 2");
    if (!profile) return fail(ctx, LBM_ERR_PARAM, "NULL profile array");
    DeviceGuard dg(ctx->dev);
    const int na = axis == 0 ? ctx->G.nx : axis == 1 ? ctx->G.ny : ctx->G.nz;
    // moments of the current state into the sample arrays, as lbm_moments does
    CK(ctx, launch_convert(ctx->p.storage, 2, ctx->mom, ctx->fbase(0), ctx->gbase(0), ctx->G, ctx->P,
                           ctx->layout(), ctx->stream));
    const size_t bytes = ((size_t)na + 6) * sizeof(double);
    Scratch sc(ctx, bytes);
    if (!sc.ptr) return fail(ctx, LBM_ERR_OOM, "staging allocation failed");
    double *dev = static_cast<double *>(sc.ptr);
    CK(ctx, cudaMemsetAsync(sc.ptr, 0, bytes, ctx->stream));
    CK(ctx, launch_nu_profile(ctx->mom, ctx->G, ctx->P, ctx->wallT, axis, (float)ctx->c.H, (float)ctx->c.kappa,
                              dev, dev + na, ctx->stream));
    std::vector<double> host((size_t)na + 6);
    CK(ctx, cudaMemcpyAsync(host.data(), dev, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    if (lbm_status fs = check_flag(ctx); fs != LBM_OK) return fs;
    const double area = (double)ctx->c.nodes / na;
    for (int j = 0; j < na; ++j) profile[j] = host[j] / area;
    if (nu_mid)
        for (int f = 0; f < 6; ++f) nu_mid[f] = host[(size_t)na + f];
    return LBM_OK;
}

lbm_status lbm_sample(lbm_ctx *ctx) {
    Range range("lbm_sample");
    if (!ctx) return LBM_ERR_PARAM;
    DeviceGuard dg(ctx->dev);
    CK(ctx, launch_convert(ctx->p.storage, 2, ctx->mom, ctx->fbase(0), ctx->gbase(0), ctx->G, ctx->P,
                           ctx->layout(), ctx->stream));
    return sample_into(ctx);
}

lbm_status lbm_diagnostics(lbm_ctx *ctx, lbm_diag *out, int reset) {
    Range range("lbm_diagnostics");
    if (!ctx || !out) return ctx ? fail(ctx, LBM_ERR_PARAM, "out is NULL") : LBM_ERR_PARAM;
    DeviceGuard dg(ctx->dev);
    double host[2 * kNDiag + 1];
    CK(ctx, cudaMemcpyAsync(host, ctx->raw(), sizeof(host), cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    if (lbm_status fs = check_flag(ctx); fs != LBM_OK) return fs;
    std::memset(out, 0, sizeof(*out));
    const double *raw = host, *acc = host + kNDiag;
    const double ns = acc[kNDiag];
    out->step = ctx->step;
    out->sample_step = ctx->sample_step;
    out->samples = (int64_t)ns;
    finalize(ctx, raw, out->E, out->rms_drho, out->rms_div, out->Re_rms, out->Re_w, out->Nu_vol, out->Nu_kin,
             out->Nu_th, out->Nu_face, out->Nu_link);
    out->mean_T = raw[0] > 0 ? raw[14] / raw[0] : 0.0;
    out->mass = raw[15];
    out->max_u = raw[16];
    out->nonfinite = (int64_t)raw[17];
    for (int k = 0; k < kNDiag; ++k) out->raw[k] = raw[k];
    if (ns > 0) {
        double avg[kNDiag];
        for (int k = 0; k < kNDiag; ++k) avg[k] = k == 16 ? acc[k] : acc[k] / ns;
        double d1, d2;
        finalize(ctx, avg, out->avg_E, d1, d2, out->avg_Re_rms, out->avg_Re_w, out->avg_Nu_vol, out->avg_Nu_kin,
                 out->avg_Nu_th, out->avg_Nu_face, nullptr);
    }
    if (reset) {
        CK(ctx, cudaMemsetAsync(ctx->acc(), 0, (kNDiag + 1) * sizeof(double), ctx->stream));
        CK(ctx, cudaStreamSynchronize(ctx->stream));
    }
    if (ctx->sample_step >= 0 && (out->nonfinite > 0 || !(out->max_u <= 1.0 / std::sqrt(3.0))))
        return fail(ctx, LBM_ERR_DIVERGED, "state diverged: non-finite moment or |u| above the sound speed");
    return LBM_OK;
}

lbm_status lbm_set_wait_budget(lbm_ctx *ctx, int64_t cycles) {
    if (!ctx) return LBM_ERR_PARAM;
    if (cycles < 0) return fail(ctx, LBM_ERR_PARAM, "negative cycle budget");
    ctx->T.budget = cycles;
    return LBM_OK;
}

lbm_status lbm_synchronize(lbm_ctx *ctx) {
    if (!ctx) return LBM_ERR_PARAM;
    DeviceGuard dg(ctx->dev);
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    return check_flag(ctx);
}

struct CkptHeader {
    int magic, version, nx, ny, nz, storage, streaming, parity;
    int64_t step, sample_step, stride;
};

lbm_status lbm_save(lbm_ctx *ctx, const char *path) {
    if (!ctx || !path) return ctx ? fail(ctx, LBM_ERR_PARAM, "path is NULL") : LBM_ERR_PARAM;
    DeviceGuard dg(ctx->dev);
    std::vector<char> pop(ctx->pop_bytes);
    double sums[2 * kNDiag + 1];
    CK(ctx, cudaMemcpyAsync(pop.data(), ctx->pop, ctx->pop_bytes, cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaMemcpyAsync(sums, ctx->raw(), sizeof(sums), cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    FILE *fp = std::fopen(path, "wb");
    if (!fp) return fail(ctx, LBM_ERR_PARAM, std::string("cannot open ") + path);
    CkptHeader h{kMagic, 1, ctx->p.nx, ctx->p.ny, ctx->p.nz, ctx->p.storage, ctx->p.streaming, ctx->parity,
                 ctx->step, ctx->sample_step, ctx->G.stride};
    bool ok = std::fwrite(&h, sizeof(h), 1, fp) == 1 && std::fwrite(pop.data(), 1, pop.size(), fp) == pop.size() &&
              std::fwrite(sums, sizeof(sums), 1, fp) == 1;
    ok = (std::fclose(fp) == 0) && ok;
    return ok ? LBM_OK : fail(ctx, LBM_ERR_PARAM, std::string("write failed: ") + path);
}

lbm_status lbm_load(lbm_ctx *ctx, const char *path) {
    if (!ctx || !path) return ctx ? fail(ctx, LBM_ERR_PARAM, "path is NULL") : LBM_ERR_PARAM;
    DeviceGuard dg(ctx->dev);
    FILE *fp = std::fopen(path, "rb");
    if (!fp) return fail(ctx, LBM_ERR_PARAM, std::string("cannot open ") + path);
    CkptHeader h{};
    std::vector<char> pop(ctx->pop_bytes);
    double sums[2 * kNDiag + 1];
    bool ok = std::fread(&h, sizeof(h), 1, fp) == 1;
    ok = ok && h.magic == kMagic && h.version == 1 && h.nx == ctx->p.nx && h.ny == ctx->p.ny &&
         h.nz == ctx->p.nz && h.storage == ctx->p.storage && h.streaming == ctx->p.streaming &&
         h.stride == ctx->G.stride;
    ok = ok && std::fread(pop.data(), 1, pop.size(), fp) == pop.size() && std::fread(sums, sizeof(sums), 1, fp) == 1;
    std::fclose(fp);
    if (!ok) return fail(ctx, LBM_ERR_PARAM, std::string("checkpoint does not match this context: ") + path);
    CK(ctx, cudaMemcpyAsync(ctx->pop, pop.data(), ctx->pop_bytes, cudaMemcpyHostToDevice, ctx->stream));
    CK(ctx, cudaMemcpyAsync(ctx->raw(), sums, sizeof(sums), cudaMemcpyHostToDevice, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->parity = h.parity;
    ctx->step = h.step;
    ctx->sample_step = h.sample_step;
    return LBM_OK;
}

lbm_status lbm_device_view(lbm_ctx *ctx, void **f, void **g, int64_t *stride, int *elem_bytes) {
    if (!ctx) return LBM_ERR_PARAM;
    if (f) *f = ctx->fbase(0);
    if (g) *g = ctx->gbase(0);
    if (stride) *stride = ctx->G.stride;
    if (elem_bytes) *elem_bytes = ctx->elem;
    return LBM_OK;
}

} // extern "C"

// ------------------------------------------------------------------ batches --

struct lbm_batch {
    std::vector<lbm_ctx *> cells;
    int storage = 0;
    int dev = 0;
    int nsm = 0;
    cudaStream_t stream = nullptr;
    lbm_schedule sched{256, 2, 100, 1000, 1, 0};
    long long budget = 1LL << 31;
    CellDev *d_cells = nullptr;
    Tile *d_tiles = nullptr; // even tiles, then odd tiles
    size_t tiles_bytes = 0;
    GridBarrier *d_bar = nullptr;
    int n_even = 0, n_odd = 0, n_rows = 0, n_faces = 0, tiles_block = 0, tiles_span = 0;
    int grid_k[3] = {0, 0, 0}; // per-step mode: grid of each tile kind's kernel
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    lbm_schedule graph_sched{};
    int graph_parity = -1;
    long long graph_budget = 0;
    std::string err;
};

namespace {

lbm_status bfail(lbm_batch *b, lbm_status s, const std::string &msg) {
    if (b) b->err = msg;
    g_create_error = msg;
    return s;
}

#define BCK(b, call)                                                                            \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess)                                                                  \
            return bfail(b, LBM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));  \
    } while (0)

void drop_graph(lbm_batch *b) {
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->gexec = nullptr;
    b->graph = nullptr;
    b->graph_parity = -1;
}

// Tile lists for a block size and tile span: per cell, runs of `span`
// consecutive blocks of its single-cell kernels; stored as even tiles, row
// tiles, face tiles (the odd step's list is the last two together).
lbm_status build_tiles(lbm_batch *b, int block, int span) {
    std::vector<Tile> even, rows, faces;
    for (int c = 0; c < (int)b->cells.size(); ++c) {
        const lbm_ctx *x = b->cells[c];
        const Geom &G = x->G;
        const uint32_t ne = (uint32_t)(((uint64_t)G.n + 1) / 2 + block - 1) / block;
        const uint32_t sp = (uint32_t)span;
        for (uint32_t k = 0; k < ne; k += sp) even.push_back({c, TILE_EVEN, k, ne - k < sp ? ne - k : sp});
        const uint64_t warps = (uint64_t)G.cpp * (uint64_t)(G.nz - 2);
        const uint32_t nr = (uint32_t)((warps + block / 32 - 1) / (block / 32));
        for (uint32_t k = 0; k < nr; k += sp) rows.push_back({c, TILE_ROWS, k, nr - k < sp ? nr - k : sp});
        // the row tiles cover the x faces of their rows; the y/z-face nodes remain
        const uint32_t fb = (uint32_t)(face_nodes_per_thread(b->storage) * block); // face nodes per block
        const uint32_t nf = (x->nface_yz + fb - 1) / fb;
        for (uint32_t k = 0; k < nf; k += sp) faces.push_back({c, TILE_FACE, k, nf - k < sp ? nf - k : sp});
    }
    const size_t bytes = (even.size() + rows.size() + faces.size()) * sizeof(Tile);
    lbm_ctx *a = b->cells[0];
    if (bytes > b->tiles_bytes) {
        cudaStreamSynchronize(b->stream);
        a->dfree(b->d_tiles, b->tiles_bytes);
        b->d_tiles = (Tile *)a->dalloc(bytes);
        b->tiles_bytes = b->d_tiles ? bytes : 0;
        if (!b->d_tiles) return bfail(b, LBM_ERR_OOM, "tile table allocation failed");
    }
    Tile *d = b->d_tiles;
    BCK(b, cudaMemcpyAsync(d, even.data(), even.size() * sizeof(Tile), cudaMemcpyHostToDevice, b->stream));
    d += even.size();
    BCK(b, cudaMemcpyAsync(d, rows.data(), rows.size() * sizeof(Tile), cudaMemcpyHostToDevice, b->stream));
    d += rows.size();
    BCK(b, cudaMemcpyAsync(d, faces.data(), faces.size() * sizeof(Tile), cudaMemcpyHostToDevice, b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
    b->n_even = (int)even.size();
    b->n_rows = (int)rows.size();
    b->n_faces = (int)faces.size();
    b->n_odd = b->n_rows + b->n_faces;
    b->tiles_block = block;
    b->tiles_span = span;
    return LBM_OK;
}

// Resident blocks per SM of a kernel at a block size, capped by the schedule.
lbm_status blocks_for_kernel(lbm_batch *b, const void *fn, const lbm_schedule &s, int *grid) {
    int occ = 0;
    BCK(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, s.block_size, 0));
    if (occ < 1) return bfail(b, LBM_ERR_PARAM, "batched kernel does not fit on an SM with this block size");
    *grid = b->nsm * (s.blocks_per_sm < occ ? s.blocks_per_sm : occ);
    return LBM_OK;
}

lbm_status grid_for(lbm_batch *b, const lbm_schedule &s, int *grid) {
    return blocks_for_kernel(b, batch_kernel_ptr(b->storage, s.block_size), s, grid);
}

BatchArgs batch_args(lbm_batch *b, int grid, int nsteps, int parity0) {
    BatchArgs a{};
    a.cells = b->d_cells;
    a.even = b->d_tiles;
    a.odd = b->d_tiles + b->n_even;
    a.rows = a.odd;
    a.faces = a.odd + b->n_rows;
    a.n_even = b->n_even;
    a.n_odd = b->n_odd;
    a.n_rows = b->n_rows;
    a.n_faces = b->n_faces;
    a.nsteps = nsteps;
    a.parity0 = parity0;
    a.bar = b->d_bar;
    a.budget = b->budget;
    a.mode = b->sched.mode;
    a.grid = grid;
    a.block = b->sched.block_size;
    for (int k = 0; k < 3; ++k) a.grid_k[k] = b->grid_k[k];
    a.stream = b->stream;
    return a;
}

lbm_status check_schedule(lbm_batch *b, const lbm_schedule &s) {
    if (s.block_size != 128 && s.block_size != 256) return bfail(b, LBM_ERR_PARAM, "block_size must be 128 or 256");
    if (s.blocks_per_sm < 1 || s.blocks_per_sm > 8) return bfail(b, LBM_ERR_PARAM, "blocks_per_sm must be in [1, 8]");
    if (s.steps_per_launch < 1) return bfail(b, LBM_ERR_PARAM, "steps_per_launch must be >= 1");
    if (s.tile_span < 1 || s.tile_span > 64) return bfail(b, LBM_ERR_PARAM, "tile_span must be in [1, 64]");
    if (s.mode != 0 && s.mode != 1) return bfail(b, LBM_ERR_PARAM, "mode must be 0 or 1");
    if (s.graph_chunk < 0 || (s.graph_chunk > 0 && (s.graph_chunk % s.steps_per_launch || s.graph_chunk % 2)))
        return bfail(b, LBM_ERR_PARAM, "graph_chunk must be 0 or an even multiple of steps_per_launch");
    return LBM_OK;
}

} // namespace

extern "C" {

lbm_status lbm_batch_create(lbm_ctx *const *cells, int ncells, void *stream, lbm_batch **out) {
    if (!out) return bfail(nullptr, LBM_ERR_PARAM, "out is NULL");
    *out = nullptr;
    if (!cells || ncells < 1) return bfail(nullptr, LBM_ERR_PARAM, "need at least one cell");
    for (int c = 0; c < ncells; ++c) {
        if (!cells[c]) return bfail(nullptr, LBM_ERR_PARAM, "NULL cell");
        if (cells[c]->p.streaming != LBM_STREAM_AA)
            return bfail(nullptr, LBM_ERR_PARAM, "batched cells must use the AA streaming scheme");
        if (cells[c]->p.storage != cells[0]->p.storage)
            return bfail(nullptr, LBM_ERR_PARAM, "batched cells must share one storage format");
        if (cells[c]->dev != cells[0]->dev) return bfail(nullptr, LBM_ERR_PARAM, "batched cells must share one device");
    }
    lbm_batch *b = new lbm_batch();
    b->cells.assign(cells, cells + ncells);
    b->storage = cells[0]->p.storage;
    b->dev = cells[0]->dev;
    b->stream = static_cast<cudaStream_t>(stream);
    DeviceGuard dg(b->dev);
    if (cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, b->dev) != cudaSuccess || b->nsm < 1) {
        delete b;
        return bfail(nullptr, LBM_ERR_CUDA, "cannot query the SM count");
    }
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, b->dev);
    if (!coop) {
        delete b;
        return bfail(nullptr, LBM_ERR_CUDA, "device does not support cooperative launches");
    }
    if (!stream) b->sched.graph_chunk = 0; // the legacy default stream cannot be captured
    std::vector<CellDev> cd(ncells);
    for (int c = 0; c < ncells; ++c) {
        lbm_ctx *x = cells[c];
        cd[c].G = x->G;
        cd[c].P = x->P;
        cd[c].P.t = (uint32_t)x->step;
        cd[c].f = x->fbase(0);
        cd[c].g = x->gbase(0);
        cd[c].face = x->face;
        cd[c].nface = x->nface_yz;
    }
    lbm_ctx *a = cells[0];
    b->d_cells = (CellDev *)a->dalloc(cd.size() * sizeof(CellDev));
    b->d_bar = (GridBarrier *)a->dalloc(sizeof(GridBarrier));
    if (!b->d_cells || !b->d_bar) {
        a->dfree(b->d_cells, cd.size() * sizeof(CellDev));
        a->dfree(b->d_bar, sizeof(GridBarrier));
        delete b;
        return bfail(nullptr, LBM_ERR_OOM, "batch table allocation failed");
    }
    cudaError_t e = cudaMemcpyAsync(b->d_cells, cd.data(), cd.size() * sizeof(CellDev), cudaMemcpyHostToDevice,
                                    b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_bar, 0, sizeof(GridBarrier), b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    lbm_status st = e == cudaSuccess ? build_tiles(b, b->sched.block_size, b->sched.tile_span)
                                     : bfail(b, LBM_ERR_CUDA, std::string("batch set-up: ") + cudaGetErrorString(e));
    if (st != LBM_OK) {
        lbm_batch_destroy(b);
        g_create_error = "batch set-up failed";
        return st;
    }
    *out = b;
    return LBM_OK;
}

void lbm_batch_destroy(lbm_batch *b) {
    if (!b) return;
    DeviceGuard dg(b->dev);
    if (b->stream) cudaStreamSynchronize(b->stream);
    drop_graph(b);
    lbm_ctx *a = b->cells.empty() ? nullptr : b->cells[0];
    if (a) {
        a->dfree(b->d_cells, b->cells.size() * sizeof(CellDev));
        a->dfree(b->d_tiles, b->tiles_bytes);
        a->dfree(b->d_bar, sizeof(GridBarrier));
    }
    delete b;
}

lbm_status lbm_batch_get_schedule(const lbm_batch *b, lbm_schedule *out) {
    if (!b || !out) return LBM_ERR_PARAM;
    *out = b->sched;
    return LBM_OK;
}

lbm_status lbm_batch_set_schedule(lbm_batch *b, const lbm_schedule *s) {
    if (!b || !s) return LBM_ERR_PARAM;
    lbm_status st = check_schedule(b, *s);
    if (st != LBM_OK) return st;
    DeviceGuard dg(b->dev);
    b->sched = *s;
    if (!b->stream) b->sched.graph_chunk = 0;
    drop_graph(b);
    if (b->tiles_block != s->block_size || b->tiles_span != s->tile_span)
        return build_tiles(b, s->block_size, s->tile_span);
    return LBM_OK;
}

lbm_status lbm_batch_set_barrier_budget(lbm_batch *b, int64_t cycles) {
    if (!b || cycles < 0) return LBM_ERR_PARAM;
    b->budget = cycles;
    drop_graph(b);
    return LBM_OK;
}

lbm_status lbm_batch_step(lbm_batch *b, int64_t n) {
    Range range("lbm_batch_step");
    if (!b) return LBM_ERR_PARAM;
    if (n < 0) return bfail(b, LBM_ERR_PARAM, "negative step count");
    const int p0 = b->cells[0]->parity;
    for (lbm_ctx *c : b->cells)
        if (c->parity != p0) return bfail(b, LBM_ERR_STATE, "batched cells are at different step parities");
    DeviceGuard dg(b->dev);
    int grid = 0;
    lbm_status st = grid_for(b, b->sched, &grid);
    if (st != LBM_OK) return st;
    if (b->sched.mode == 1)
        for (int k = 0; k < 3; ++k)
            if ((st = blocks_for_kernel(b, bstep_kernel_ptr(b->storage, k, b->sched.block_size), b->sched,
                                        &b->grid_k[k])) != LBM_OK)
                return st;
    int parity = p0;
    int64_t left = n;
    const int chunk = b->sched.graph_chunk, spl = b->sched.steps_per_launch;
    if (chunk > 0 && left >= chunk) {
        if (!b->gexec || b->graph_parity != parity || b->graph_budget != b->budget ||
            std::memcmp(&b->graph_sched, &b->sched, sizeof(lbm_schedule)) != 0) {
            drop_graph(b);
            BCK(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
            cudaError_t e = cudaSuccess;
            for (int k = 0; k < chunk / spl && e == cudaSuccess; ++k)
                e = launch_batch(b->storage, batch_args(b, grid, spl, parity + k * spl));
            cudaGraph_t g = nullptr;
            cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
            if (e != cudaSuccess || e2 != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                return bfail(b, LBM_ERR_CUDA, std::string("graph capture: ") +
                                                  cudaGetErrorString(e != cudaSuccess ? e : e2));
            }
            b->graph = g;
            BCK(b, cudaGraphInstantiate(&b->gexec, b->graph, 0));
            b->graph_sched = b->sched;
            b->graph_parity = parity;
            b->graph_budget = b->budget;
        }
        while (left >= chunk) {
            BCK(b, cudaGraphLaunch(b->gexec, b->stream));
            left -= chunk;
        }
    }
    while (left > 0) {
        const int k = (int)(left < spl ? left : spl);
        BCK(b, launch_batch(b->storage, batch_args(b, grid, k, parity)));
        parity ^= k & 1;
        left -= k;
    }
    GridBarrier hb{};
    BCK(b, cudaMemcpyAsync(&hb, b->d_bar, sizeof(hb), cudaMemcpyDeviceToHost, b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
    for (lbm_ctx *c : b->cells) {
        c->step += n;
        c->parity ^= (int)(n & 1);
    }
    if (hb.err) {
        BCK(b, cudaMemsetAsync(b->d_bar, 0, sizeof(GridBarrier), b->stream));
        BCK(b, cudaStreamSynchronize(b->stream));
        return bfail(b, LBM_ERR_TIMEOUT, "a grid-barrier wait ran out of its cycle budget; cell states are undefined");
    }
    return LBM_OK;
}

lbm_status lbm_batch_autotune(lbm_batch *b, int trial_steps, lbm_schedule *best) {
    if (!b || trial_steps < 2) return b ? bfail(b, LBM_ERR_PARAM, "trial_steps must be >= 2") : LBM_ERR_PARAM;
    DeviceGuard dg(b->dev);
    const lbm_schedule keep = b->sched;
    lbm_schedule win = keep;
    float best_ms = 1e30f;
    cudaEvent_t e0, e1;
    BCK(b, cudaEventCreate(&e0));
    BCK(b, cudaEventCreate(&e1));
    const int blocks[2] = {128, 256};
    const int spans[5] = {1, 2, 4, 8, 16};
    lbm_status st = LBM_OK;
    for (int mode = 0; mode < 2 && st == LBM_OK; ++mode)
    for (int bi = 0; bi < 2 && st == LBM_OK; ++bi) {
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &occ, mode ? bstep_kernel_ptr(b->storage, TILE_EVEN, blocks[bi]) : batch_kernel_ptr(b->storage, blocks[bi]),
            blocks[bi], 0);
        for (int bps = 1; bps <= 4 && bps <= occ && st == LBM_OK; ++bps) {
            for (int si = 0; si < 5 && st == LBM_OK; ++si) {
                lbm_schedule s{blocks[bi], bps, keep.steps_per_launch, 0, spans[si], mode};
                if ((st = lbm_batch_set_schedule(b, &s)) != LBM_OK) break;
                if ((st = lbm_batch_step(b, 2)) != LBM_OK) break; // warm-up
                cudaEventRecord(e0, b->stream);
                if ((st = lbm_batch_step(b, trial_steps)) != LBM_OK) break;
                cudaEventRecord(e1, b->stream);
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms < best_ms) {
                    best_ms = ms;
                    win = s;
                }
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != LBM_OK) return st;
    win.steps_per_launch = keep.steps_per_launch;
    win.graph_chunk = keep.graph_chunk;
    st = lbm_batch_set_schedule(b, &win);
    if (best) *best = b->sched;
    return st;
}

} // extern "C"
