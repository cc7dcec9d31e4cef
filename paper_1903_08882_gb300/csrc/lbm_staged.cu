// Staged AA step kernels: persistent blocks that move the populations from
// HBM into shared memory with bulk asynchronous copies (the TMA engine,
// cp.async.bulk) through a multi-stage mbarrier pipeline, then run the same
// fused D3Q19 + D3Q7 MRT collision (Eq. MRT, Eq. MRT_T) as the register
// kernels and store the post-collision populations straight to HBM.
//
// Why: with 2-byte populations, a thread that loads its 26 values into
// registers keeps too few bytes in flight to cover the HBM latency at the
// occupancy the collision's register count allows.  Here one warp per block
// issues the copies of the next tiles while all threads compute the current
// one, so the loads stay in flight independently of registers.
//
// Tiles hold 512 nodes.  For each of the 26 population arrays a tile needs
// one contiguous window: the tile's own slots on an even step, and on an odd
// step the slots of the upstream nodes, x - e_i, a window shifted by the flat
// offset of e_i.  Windows are rounded out to 16-byte boundaries (a bulk copy
// starts and ends on one) and clamped to the array; the extra elements are
// never used.
//
// Even step: every node, natural -> reversed layout (own slots only); a
// thread takes two adjacent nodes and moves each population pair with one
// vector access.
// Odd step: the nodes 1 <= x <= nx-2 of the rows 1 <= y <= ny-2 of the
// planes 1 <= z <= nz-2; a warp takes 64 consecutive nodes, lane l the nodes
// l and l + 32, so that its stores to the shifted destinations stay
// contiguous.  Every node next to a face goes to the general face kernel.
// (Four ways of updating the x-face nodes here measured slower at 257^3
// than leaving them to the face kernel, 494 us per FP16 odd step: their wall
// links loaded per lane before the wait (740 us), fetched as 16-byte bulk
// copies into the stage (617 us: the copy engine takes tiny copies one by
// one), fetched by per-thread 4-byte asynchronous copies completing on the
// stage's barrier (510 us: the extra flags and addresses push the kernel past
// its 128 registers into local memory), or listed and updated by one warp
// every few tiles (549 us: that warp waits on L2 while the block waits for it
// at the next barrier).  Scheduling the face kernel's x-face work as items of
// this kernel, right after the tiles whose windows hold their neighbourhood,
// gave 490 us: the cost is the general path on strided nodes, not DRAM
// re-reads.)
// Every location a node reads is written by that node only, so the in-place
// update is race-free whatever order the tiles run in.
#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace lbm {

template <int S> using SF = typename Store<FS(S)>::T;
template <int S> using SG = typename Store<GS(S)>::T;

namespace {

constexpr int kThreads = 256;           // threads per block
constexpr int kTile = 2 * kThreads;     // nodes per tile
constexpr int kSlack = 32;              // window bytes beyond the tile: 16-byte rounding at both ends
constexpr int kHead = 1024;             // shared-memory header: mbarriers and window shifts
constexpr long long kDrain = 1ll << 31; // cycles to wait for copies in flight before leaving after a timeout

template <int S> struct Stage {
    static constexpr int fwin = kTile * (int)sizeof(SF<S>) + kSlack;
    static constexpr int gwin = kTile * (int)sizeof(SG<S>) + kSlack;
    static constexpr int bytes = 19 * fwin + 7 * gwin;
    static constexpr int count = (sizeof(SF<S>) == 4) ? 2 : 3; // stages in flight per block
    static constexpr int smem = kHead + count * bytes;
    static __device__ __forceinline__ int offset(int q) { return q < 19 ? q * fwin : 19 * fwin + (q - 19) * gwin; }
};
static_assert(Stage<ST_F32>::bytes % 16 == 0 && Stage<ST_F16>::bytes % 16 == 0 && Stage<ST_F16M>::bytes % 16 == 0,
              "stage buffers must keep 16-byte alignment");
static_assert(Stage<ST_F32>::smem <= 227 * 1024 && Stage<ST_F16M>::smem <= 227 * 1024, "stage buffers too large");

// ------------------------------------------------------ PTX wrappers ----

__device__ __forceinline__ uint32_t sptr(const void *p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sptr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sptr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(sptr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Wait for the phase with the given parity to complete; give up after
// `budget` clock cycles (returns false).  A budget <= 0 fails at once: it
// exercises the timeout path.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, long long budget) {
    if (budget <= 0) return false;
    if (mbar_test(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_test(bar, parity))
        if (clock64() - t0 > budget) return false;
    return true;
}
// Bulk copy global -> shared (this CTA), completion counted on `bar`.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     sptr(dst)),
                 "l"(src), "r"(bytes), "r"(sptr(bar))
                 : "memory");
}

// ------------------------------------------------- element helpers ----

__device__ __forceinline__ float tof(float v) { return v; }
__device__ __forceinline__ float tof(__half v) { return __half2float(v); }
__device__ __forceinline__ float tof(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename E> struct Pair;
// st / st1: round to nearest; sts / st1s: stochastic rounding with the
// random bits r (the thermal populations of the 2-byte storages, see
// lbm_device.cuh).
template <> struct Pair<float> {
    static __device__ __forceinline__ float2 ld(const float *p) { return *reinterpret_cast<const float2 *>(p); }
    static __device__ __forceinline__ void st(float *p, float2 v) { *reinterpret_cast<float2 *>(p) = v; }
    static __device__ __forceinline__ void st1(float *p, float v) { *p = v; }
    static __device__ __forceinline__ void sts(float *p, float2 v, uint32_t, uint32_t) { st(p, v); }
    static __device__ __forceinline__ void st1s(float *p, float v, uint32_t) { *p = v; }
};
template <> struct Pair<__half> {
    static __device__ __forceinline__ float2 ld(const __half *p) {
        return __half22float2(*reinterpret_cast<const __half2 *>(p));
    }
    static __device__ __forceinline__ void st(__half *p, float2 v) {
        *reinterpret_cast<__half2 *>(p) = __float22half2_rn(v);
    }
    static __device__ __forceinline__ void st1(__half *p, float v) { *p = __float2half_rn(v); }
    static __device__ __forceinline__ void sts(__half *p, float2 v, uint32_t r0, uint32_t r1) {
        *reinterpret_cast<__half2 *>(p) = h2_sr(v, r0, r1);
    }
    static __device__ __forceinline__ void st1s(__half *p, float v, uint32_t r) { *p = __float2half_rz(sr_pre16(v, r)); }
};
template <> struct Pair<__nv_bfloat16> {
    static __device__ __forceinline__ float2 ld(const __nv_bfloat16 *p) {
        return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(p));
    }
    static __device__ __forceinline__ void st(__nv_bfloat16 *p, float2 v) {
        *reinterpret_cast<__nv_bfloat162 *>(p) = __float22bfloat162_rn(v);
    }
    static __device__ __forceinline__ void st1(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
    static __device__ __forceinline__ void sts(__nv_bfloat16 *p, float2 v, uint32_t r0, uint32_t r1) {
        *reinterpret_cast<__nv_bfloat162 *>(p) = bf2_sr(v, r0, r1);
    }
    static __device__ __forceinline__ void st1s(__nv_bfloat16 *p, float v, uint32_t r) {
        *p = __float2bfloat16_rz(sr_pre_bf(v, r));
    }
};

// Flat offset of e_i for population q (0..18 flow, 19..25 thermal: the D3Q7
// velocities e_0..e_6 equal the D3Q19 ones).
__device__ __forceinline__ int pop_off(const Geom &G, int q) { return G.off[q < 19 ? q : q - 19]; }
// Opposite velocity index, arithmetically (paper order: (1,2) (3,4) (5,6),
// then the groups 7-10, 11-14, 15-18 pair their first and last, second and
// third members).
__host__ __device__ __forceinline__ int opp_idx(int i) {
    return i == 0 ? 0 : i < 7 ? (i & 1 ? i + 1 : i - 1) : 7 + 4 * ((i - 7) >> 2) + 3 - ((i - 7) & 3);
}
// Array an odd step reads population q from: the opposite slot.
__host__ __device__ __forceinline__ int src_array(int q) { return q < 19 ? opp_idx(q) : 19 + opp_idx(q - 19); }

// Tile t of a step: its first node and the node range it updates.
struct TileSpan {
    uint32_t n0, lo, hi;
};
template <bool ODD> __device__ __forceinline__ TileSpan tile_span(const Geom &G, const StagedGeom &T, uint32_t t) {
    TileSpan s;
    if (!ODD) {
        s.n0 = t * (uint32_t)kTile;
        s.lo = 0;
        s.hi = G.n;
    } else {
        const uint32_t zi = fast_div(t, T.mag_tpp);
        const uint32_t z = zi + 1u;
        s.lo = z * G.nxy + (uint32_t)G.nx;
        s.hi = z * G.nxy + G.nxy - (uint32_t)G.nx;
        s.n0 = (s.lo & ~1u) + (t - zi * T.tpp) * (uint32_t)kTile;
    }
    return s;
}

// Copy the 26 windows of a tile into one stage.  Called by all 32 lanes of
// one warp: lane q < 26 computes and issues window q.  shift[q] receives
// n0 - off_q - (first element copied), so that node n0 + j of the tile sits
// at element j + shift[q] of window q.
template <int S, bool ODD>
__device__ __forceinline__ void issue_tile(const SF<S> *f, const SG<S> *g, const Geom &G, uint32_t n0,
                                           unsigned char *stage, int *shift, uint64_t *bar, int lane) {
    unsigned sz = 0;
    const char *src = nullptr;
    if (lane < 26) {
        const int q = lane;
        const int64_t es = q < 19 ? (int64_t)sizeof(SF<S>) : (int64_t)sizeof(SG<S>);
        const int64_t first = (int64_t)n0 - (ODD ? pop_off(G, q) : 0);
        int64_t a = (first * es) & ~(int64_t)15;
        int64_t b = ((first + kTile) * es + 15) & ~(int64_t)15;
        const int64_t lim = G.stride * es;
        a = a < 0 ? 0 : a;
        b = b > lim ? lim : b;
        sz = b > a ? (unsigned)(b - a) : 0u;
        shift[q] = (int)(first - a / es);
        const int arr = ODD ? src_array(q) : q;
        src = (arr < 19 ? reinterpret_cast<const char *>(f + (int64_t)arr * G.stride)
                        : reinterpret_cast<const char *>(g + (int64_t)(arr - 19) * G.stride)) + a;
    }
    unsigned total = sz;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) total += __shfl_xor_sync(0xffffffffu, total, o);
    if (lane == 0) mbar_expect_tx(bar, total);
    __syncwarp();
    if (sz) bulk_load(stage + Stage<S>::offset(lane), src, sz, bar);
}

template <int S, bool ODD>
__global__ void __launch_bounds__(kThreads, 2)
    k_aa_staged(SF<S> *__restrict__ f, SG<S> *__restrict__ g, Geom G, Phys P, StagedGeom T, int *err) {
    constexpr int NST = Stage<S>::count;
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    int *shift = reinterpret_cast<int *>(smem + 64); // [NST][26]
    unsigned char *stages = smem + kHead;
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const uint32_t ntiles = ODD ? T.odd_tiles : T.even_tiles;
    const int64_t s = G.stride;

    if (tid == 0) {
        for (int k = 0; k < NST; ++k) mbar_init(&bar[k], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (warp == 0) {
        for (int k = 0; k < NST; ++k) {
            const uint32_t t = blockIdx.x + (uint32_t)k * gridDim.x;
            if (t < ntiles)
                issue_tile<S, ODD>(f, g, G, tile_span<ODD>(G, T, t).n0, stages + k * Stage<S>::bytes,
                                   shift + 26 * k, &bar[k], lane);
        }
    }

    int j = 0;
    for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++j) {
        const int st = j % NST;
        const unsigned parity = (unsigned)(j / NST) & 1u;
        const TileSpan sp = tile_span<ODD>(G, T, t);
        // even step: nodes m, m + 1; odd step: m, m + 32
        const uint32_t o = ODD ? 64u * (uint32_t)warp + (uint32_t)lane : 2u * (uint32_t)tid;
        const uint32_t m = sp.n0 + o;
        const uint32_t mb = m + (ODD ? 32u : 1u);
        bool v0 = m >= sp.lo && m < sp.hi;
        bool v1 = mb >= sp.lo && mb < sp.hi;
        if (ODD) { // nodes next to an x face belong to the face kernel
            const uint32_t nx = (uint32_t)G.nx;
            const uint32_t xa = m - nx * fast_div(m, G.mag_nx), xb = mb - nx * fast_div(mb, G.mag_nx);
            v0 = v0 && xa != 0u && xa != nx - 1u;
            v1 = v1 && xb != 0u && xb != nx - 1u;
        }

        const bool ok = mbar_wait(&bar[st], parity, T.budget);
        if (ok && (v0 || v1)) {
            const unsigned char *sb = stages + st * Stage<S>::bytes;
            const int *sh = shift + 26 * st;
            float2 fl[19], gl[7];
            if (!ODD) {
#pragma unroll
                for (int q = 0; q < 19; ++q)
                    fl[q] = Pair<SF<S>>::ld(reinterpret_cast<const SF<S> *>(sb + Stage<S>::offset(q)) + o + sh[q]);
#pragma unroll
                for (int q = 0; q < 7; ++q)
                    gl[q] = Pair<SG<S>>::ld(reinterpret_cast<const SG<S> *>(sb + Stage<S>::offset(19 + q)) + o +
                                            sh[19 + q]);
            } else {
#pragma unroll
                for (int q = 0; q < 19; ++q) {
                    const SF<S> *w = reinterpret_cast<const SF<S> *>(sb + Stage<S>::offset(q)) + o + sh[q];
                    fl[q] = make_float2(tof(w[0]), tof(w[32]));
                }
#pragma unroll
                for (int q = 0; q < 7; ++q) {
                    const SG<S> *w = reinterpret_cast<const SG<S> *>(sb + Stage<S>::offset(19 + q)) + o + sh[19 + q];
                    gl[q] = make_float2(tof(w[0]), tof(w[32]));
                }
            }
            collide(P, fl, gl);
            SF<S> *fo = f;
            SG<S> *go = g;
            asm volatile("" : "+l"(fo), "+l"(go)); // recompute addresses after the collision
            if (!ODD) {
                // own node, opposite slot; a pair that ends past the last node
                // writes the first padding element, which no node reads
                if (v0) {
#pragma unroll
                    for (int q = 0; q < 19; ++q) Pair<SF<S>>::st(fo + opp19(q) * s + m, fl[q]);
                    const uint32_t rb0 = SRG(S) ? rnd_node(m, P.t) : 0u, rb1 = SRG(S) ? rnd_node(mb, P.t) : 0u;
#pragma unroll
                    for (int q = 0; q < 7; ++q)
                        Pair<SG<S>>::sts(go + opp7(q) * s + m, gl[q], rnd_pop(rb0, q), rnd_pop(rb1, q));
                }
            } else {
#pragma unroll
                for (int q = 0; q < 19; ++q) {
                    SF<S> *p = fo + q * s + (int64_t)m + G.off[q];
                    if (v0) Pair<SF<S>>::st1(p, fl[q].x);
                    if (v1) Pair<SF<S>>::st1(p + 32, fl[q].y);
                }
                const uint32_t rb0 = SRG(S) ? rnd_node(m, P.t) : 0u, rb1 = SRG(S) ? rnd_node(mb, P.t) : 0u;
#pragma unroll
                for (int q = 0; q < 7; ++q) {
                    SG<S> *p = go + q * s + (int64_t)m + G.off[q];
                    if (v0) Pair<SG<S>>::st1s(p, gl[q].x, rnd_pop(rb0, q));
                    if (v1) Pair<SG<S>>::st1s(p + 32, gl[q].y, rnd_pop(rb1, q));
                }
            }
        }
        // every thread is done with this stage: refill it with the tile NST ahead
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicExch(err, 1);
                // let the copies still in flight (this tile's and the ones
                // issued ahead) land before the block exits
                for (int k = 0; k < NST; ++k) {
                    const uint32_t tk = t + (uint32_t)k * gridDim.x;
                    if (tk < ntiles) mbar_wait(&bar[(j + k) % NST], (unsigned)((j + k) / NST) & 1u, kDrain);
                }
            }
            return;
        }
        if (warp == 0) {
            const uint32_t tn = t + (uint32_t)NST * gridDim.x;
            if (tn < ntiles)
                issue_tile<S, ODD>(f, g, G, tile_span<ODD>(G, T, tn).n0, stages + st * Stage<S>::bytes,
                                   shift + 26 * st, &bar[st], lane);
        }
    }
}

template <int S> const void *staged_fn() { return reinterpret_cast<const void *>(&k_aa_staged<S, true>); }

template <int S> cudaError_t staged_attr() {
    const int b = Stage<S>::smem;
    cudaError_t e = cudaFuncSetAttribute(k_aa_staged<S, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_aa_staged<S, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    return e;
}

template <int S> cudaError_t staged_launch(const StepArgs &a) {
    auto f = static_cast<SF<S> *>(a.f);
    auto g = static_cast<SG<S> *>(a.g);
    const StagedGeom &T = a.T;
    if (a.parity == 0) {
        k_aa_staged<S, false><<<T.grid, kThreads, Stage<S>::smem, a.stream>>>(f, g, a.G, a.P, T, a.err);
        return cudaGetLastError();
    }
    if (T.odd_tiles) k_aa_staged<S, true><<<T.grid, kThreads, Stage<S>::smem, a.stream>>>(f, g, a.G, a.P, T, a.err);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_face(a, a.nface); // every node next to a face
}

} // namespace

int staged_smem_bytes(int storage) {
    switch (storage) {
    case ST_F32: return Stage<ST_F32>::smem;
    case ST_F16: return Stage<ST_F16>::smem;
    case ST_F16M: return Stage<ST_F16M>::smem;
    default: return Stage<ST_BF16>::smem;
    }
}

int staged_tile_nodes() { return kTile; }

cudaError_t staged_prepare(int storage, int *blocks_per_sm) {
    cudaError_t e;
    const void *fn;
    switch (storage) {
    case ST_F32: e = staged_attr<ST_F32>(); fn = staged_fn<ST_F32>(); break;
    case ST_F16: e = staged_attr<ST_F16>(); fn = staged_fn<ST_F16>(); break;
    case ST_F16M: e = staged_attr<ST_F16M>(); fn = staged_fn<ST_F16M>(); break;
    default: e = staged_attr<ST_BF16>(); fn = staged_fn<ST_BF16>(); break;
    }
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, kThreads, staged_smem_bytes(storage));
}

cudaError_t launch_staged(const StepArgs &a) {
    switch (a.storage) {
    case ST_F32: return staged_launch<ST_F32>(a);
    case ST_F16: return staged_launch<ST_F16>(a);
    case ST_F16M: return staged_launch<ST_F16M>(a);
    default: return staged_launch<ST_BF16>(a);
    }
}

} // namespace lbm
