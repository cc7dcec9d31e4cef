// Staged AA step kernels: persistent blocks that move the populations from
// HBM into shared memory with bulk asynchronous copies (the TMA engine,
// cp.async.bulk) through a multi-stage mbarrier pipeline, then run the same
// fused D3Q19 + D3Q7 MRT collision (Eq. MRT, Eq. MRT_T) as the register
// kernels and store the post-collision populations straight to HBM.
//
// Why: with 2-byte populations, a thread that loads its 26 values into
// registers keeps too few bytes in flight to cover the HBM latency at the
// occupancy the collision's register count allows.  Here one producer warp
// per block issues the copies of the next tiles while the other warps compute
// the current one, so the loads stay in flight independently of registers.
//
// Tiles hold 64 nodes per compute warp.  For each of the 26 population arrays
// a tile needs one contiguous window: the tile's own slots on an even step,
// and on an odd step the slots of the upstream nodes, x - e_i, a window
// shifted by the flat offset of e_i.  Windows are rounded out to 16-byte
// boundaries (a bulk copy starts and ends on one) and clamped to the array;
// the extra elements are never used.
//
// Even step: every node, natural -> reversed layout (own slots only); a
// thread takes two adjacent nodes and moves each population pair with one
// vector access.
// Odd step: the rows 1 <= y <= ny-2 of the planes 1 <= z <= nz-2; a warp
// takes 64 consecutive nodes, lane l the nodes l and l + 32, so that its
// stores to the shifted destinations stay contiguous.  For rows of at least
// kXfMinNx nodes the nodes at x = 0 and x = nx-1 of those rows are updated
// here too: the six values that arrive through the x face (bounce-back from
// the node's own slot, or the far end of the row when x is periodic) are not
// in the shifted windows, so the producer warp also fetches each as one
// 4-byte asynchronous copy (cp.async) into the stage, completing on the
// stage's barrier, and the links that leave through the face are stored to
// the node's own slots.  The nodes next to a y or z face (and, for shorter
// rows, the x-face nodes) go to the general face kernel.  (Leaving the x-face
// nodes to the face kernel costs it strided 32-byte sectors, 594 B read per
// node against 52 B algorithmic; in-tile they cost 5% of the odd step less at
// 257^3.)
// Every location a node reads is written by that node only, so the in-place
// update is race-free whatever order the tiles run in.
#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace lbm {

template <int S> using SF = typename Store<FS(S)>::T;
template <int S> using SG = typename Store<GS(S)>::T;

namespace {

constexpr int kThreads = 256;           // threads per block
constexpr int kWarps = kThreads / 32;
// Warps that update nodes: all of them on an even step (warp 0 also issues
// the copies), all but the producer warp 0 on an odd step.  A tile holds 64
// nodes per compute warp.
template <bool ODD> constexpr int kCompute = ODD ? kWarps - 1 : kWarps;
template <bool ODD> constexpr int kTile = 64 * kCompute<ODD>;
constexpr int kSlack = 32;              // window bytes beyond the tile: 16-byte rounding at both ends
constexpr int kHead = 1024;             // shared-memory header: mbarriers and window offsets
constexpr int kWofs = 28;               // window offsets per stage (26, padded for 16-byte loads)
constexpr long long kDrain = 1ll << 31; // cycles to wait for copies in flight before leaving after a timeout
// In-tile x faces (odd step): a tile of kTile consecutive nodes touches at
// most kXfRows rows of at least kXfMinNx nodes; each row has two x-face nodes
// and each of them 5 + 1 links through its face.
constexpr int kXfMinNx = 16;
constexpr int kXfRows = (kTile<true> - 1) / kXfMinNx + 2;
constexpr int kSide = kXfRows * 2 * 6 * 4; // one 4-byte word per x-face link

template <int S, bool ODD> struct Stage {
    static constexpr int fwin = kTile<ODD> * (int)sizeof(SF<S>) + kSlack;
    static constexpr int gwin = kTile<ODD> * (int)sizeof(SG<S>) + kSlack;
    static constexpr int win = 19 * fwin + 7 * gwin; // the 26 windows, then the x-face words (odd step)
    static constexpr int bytes = win + (ODD ? kSide : 0);
    // stages per block: as many as leave room for two blocks per SM (at most
    // 113 KB each beside the 1 KB the system keeps per block), up to four
    static constexpr int room = (113 * 1024 - kHead) / bytes;
    static constexpr int count = room < 4 ? room : 4;
    static constexpr int smem = kHead + count * bytes;
    static __device__ __forceinline__ int offset(int q) { return q < 19 ? q * fwin : 19 * fwin + (q - 19) * gwin; }
};
template <bool ODD> constexpr bool stages_ok() {
    return Stage<ST_F32, ODD>::bytes % 16 == 0 && Stage<ST_F16, ODD>::bytes % 16 == 0 &&
           Stage<ST_F16M, ODD>::bytes % 16 == 0 && Stage<ST_F32, ODD>::count >= 2 &&
           Stage<ST_F16M, ODD>::count >= 2 && Stage<ST_F16, ODD>::count >= 2;
}
static_assert(stages_ok<false>() && stages_ok<true>(), "stage buffers: 16-byte aligned, two per block at least");
// header: full and empty barriers at 0, window offsets at 64, fill counts at 512
static_assert(2 * 4 * 8 <= 64 && 64 + 4 * kWofs * 4 <= 512 && 512 + 4 * 4 <= kHead, "shared-memory header layout");

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

// 4-byte asynchronous copy global -> shared (both addresses 4-byte aligned).
__device__ __forceinline__ void word_load(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sptr(dst)), "l"(src) : "memory");
}
// One arrival on `bar` once this thread's earlier cp.async copies have landed
// (counted in the barrier's expected arrivals).
__device__ __forceinline__ void word_arrive(uint64_t *bar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(sptr(bar)) : "memory");
}

// ------------------------------------------------- element helpers ----
//
// Per storage format FMT (lbm_device.cuh): one: an element to FP32;
// word: the element with index parity `odd` of the aligned 4-byte word
// holding it; ld: two consecutive elements (first index even); st / st1:
// round to nearest; sts / st1s: the thermal populations' stochastic rounding
// with random bits r.
template <int FMT> struct PairF {
    using E = typename Store<FMT>::T;
    static __device__ __forceinline__ float one(E v) { return Store<FMT>::ld(&v); }
    static __device__ __forceinline__ float word(uint32_t w, uint32_t odd) {
        if (sizeof(E) == 4) return Store<FMT>::ld(reinterpret_cast<const E *>(&w));
        const unsigned short h = (unsigned short)(odd ? w >> 16 : w & 0xffffu);
        return Store<FMT>::ld(reinterpret_cast<const E *>(&h));
    }
    static __device__ __forceinline__ float2 ld(const E *p) { return Store2<FMT>::ld(p); }
    static __device__ __forceinline__ void st(E *p, float2 v) { Store2<FMT>::st(p, v); }
    static __device__ __forceinline__ void st1(E *p, float v) { Store<FMT>::st(p, v); }
    static __device__ __forceinline__ void sts(E *p, float2 v, uint32_t r0, uint32_t r1) {
        Store2<FMT>::sts(p, v, r0, r1);
    }
    static __device__ __forceinline__ void st1s(E *p, float v, uint32_t r) { Store<FMT>::sts(p, v, r); }
};
template <int S> using PF = PairF<FS(S)>; // flow arrays
// thermal arrays: the FP16 thermal format's stored (2^12-scaled) values are
// used as they are, and the collision runs on them (collide<V, true>)
template <int S> constexpr bool kGRaw = GS(S) == ST_F16T;
template <int S> using PG = PairF<kGRaw<S> ? ST_F16 : GS(S)>;
template <int S> constexpr float kGs = kGRaw<S> ? kGScale : 1.f; // scale of g as held in registers

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

// D3Q19 links with e_x = +1 (side 0) or -1 (side 1), j = 0..4: 1 7 9 11 13 / 2 8 10 12 14.
__host__ __device__ constexpr int xlink(int side, int j) { return (j == 0 ? 1 : 5 + 2 * j) + side; }

// Tile t of a step: its first node and the node range it updates.
struct TileSpan {
    uint32_t n0, lo, hi;
};
template <bool ODD> __device__ __forceinline__ TileSpan tile_span(const Geom &G, const StagedGeom &T, uint32_t t) {
    TileSpan s;
    if (!ODD) {
        s.n0 = t * (uint32_t)kTile<false>;
        s.lo = 0;
        s.hi = G.n;
    } else {
        const uint32_t zi = fast_div(t, T.mag_tpp);
        const uint32_t z = zi + 1u;
        s.lo = z * G.nxy + (uint32_t)G.nx;
        s.hi = z * G.nxy + G.nxy - (uint32_t)G.nx;
        s.n0 = (s.lo & ~1u) + (t - zi * T.tpp) * (uint32_t)kTile<true>;
    }
    return s;
}

// Copy one tile into a stage.  Called by all 32 lanes of one warp.
// Lane q < 26 computes and issues window q: wofs[q] receives the byte offset
// in the stage of the element that node n0 of the tile reads, so that node
// n0 + j reads element j from there (the window starts n0 - off_q - (first
// element copied) elements before it).
// XF (odd step, rows of at least kXfMinNx nodes): the values that arrive at
// the tile's x-face nodes through their face are not in the windows (they
// come from the node's own slot at a wall, or from the far end of the row
// when x is periodic); the lanes fetch each one as the aligned 4-byte word
// holding it into the stage's x-face area, word (2 R + side) 6 + j for the
// face node of the tile's R-th row on side 0 (x = 0) or 1 (x = nx-1) and
// its link j (five flow links, then the thermal one), completion counted on
// the same barrier (issue_side).
template <int S, bool ODD>
__device__ __forceinline__ void issue_tile(const SF<S> *f, const SG<S> *g, const Geom &G, const TileSpan &sp,
                                           unsigned char *stage, int *wofs, uint64_t *bar, int lane) {
    unsigned sz = 0;
    const char *src = nullptr;
    if (lane < 26) {
        const int q = lane;
        const int64_t es = q < 19 ? (int64_t)sizeof(SF<S>) : (int64_t)sizeof(SG<S>);
        const int64_t first = (int64_t)sp.n0 - (ODD ? pop_off(G, q) : 0);
        int64_t a = (first * es) & ~(int64_t)15;
        int64_t b = ((first + kTile<ODD>) * es + 15) & ~(int64_t)15;
        const int64_t lim = G.stride * es;
        a = a < 0 ? 0 : a;
        b = b > lim ? lim : b;
        sz = b > a ? (unsigned)(b - a) : 0u;
        wofs[q] = Stage<S, ODD>::offset(q) + (int)((first - a / es) * es);
        const int arr = ODD ? src_array(q) : q;
        src = (arr < 19 ? reinterpret_cast<const char *>(f + (int64_t)arr * G.stride)
                        : reinterpret_cast<const char *>(g + (int64_t)(arr - 19) * G.stride)) + a;
    }
    unsigned total = sz;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) total += __shfl_xor_sync(0xffffffffu, total, o);
    if (lane == 0) mbar_expect_tx(bar, total);
    __syncwarp();
    if (sz) bulk_load(stage + Stage<S, ODD>::offset(lane), src, sz, bar);
}

// The x-face words of a tile (see issue_tile), fetched by all 32 lanes of the
// producer warp: each lane's copies complete on the stage's barrier through
// one counted arrival.
template <int S>
__device__ __forceinline__ void issue_side(const SF<S> *f, const SG<S> *g, const Geom &G, const TileSpan &sp,
                                           unsigned char *stage, uint64_t *bar, int lane) {
    uint32_t *side = reinterpret_cast<uint32_t *>(stage + Stage<S, true>::win);
    const uint32_t nx = (uint32_t)G.nx;
    const uint32_t row0 = fast_div(sp.n0, G.mag_nx);
    const uint32_t rows = fast_div(sp.n0 + (uint32_t)kTile<true> - 1u, G.mag_nx) - row0 + 1u;
    const uint32_t beg = sp.n0 > sp.lo ? sp.n0 : sp.lo;
    const uint32_t end = sp.n0 + (uint32_t)kTile<true> < sp.hi ? sp.n0 + (uint32_t)kTile<true> : sp.hi;
    const bool per = G.periodic & 1;
    const int64_t s = G.stride;
    for (uint32_t k = (uint32_t)lane; k < rows * 12u; k += 32u) {
        const uint32_t R = k / 12u, rem = k - 12u * R, sd = rem / 6u, j = rem - 6u * sd;
        const uint32_t n = (row0 + R) * nx + (sd ? nx - 1u : 0u);
        if (n < beg || n >= end) continue;
        const int q = j < 5u ? xlink((int)sd, (int)j) : 1 + (int)sd; // flow / thermal link index
        // wall: the node's own slot q; periodic: slot qbar of n - e_q wrapped along the row
        const int64_t at = per ? (int64_t)n - G.off[q] + (sd ? -(int64_t)nx : (int64_t)nx) : (int64_t)n;
        const int arr = per ? opp_idx(q) : q;
        const char *p = j < 5u ? reinterpret_cast<const char *>(f + (int64_t)arr * s + at)
                               : reinterpret_cast<const char *>(g + (int64_t)arr * s + at);
        word_load(side + k, reinterpret_cast<const void *>(reinterpret_cast<uintptr_t>(p) & ~(uintptr_t)3));
    }
    word_arrive(bar);
}

// x-face node (hi = false: x = 0, true: x = nx-1) of component K of a pair:
// the links that arrive through its face take the fetched words (w: the
// node's six words), with anti-bounce-back for g at a Dirichlet face.  The
// side is a per-lane value, so that the lanes holding the two ends of a row
// run this once together.
template <int K> __device__ __forceinline__ void set_k(float2 &d, float v) {
    if (K == 0) d.x = v;
    else d.y = v;
}
template <int S, int K>
__device__ __forceinline__ void xface_in(float2 (&fl)[19], float2 (&gl)[7], const uint32_t *w, uint32_t n, bool hi,
                                         const Geom &G, const Phys &P) {
    const bool per = G.periodic & 1;
    const int64_t wrap = hi ? -(int64_t)G.nx : (int64_t)G.nx;
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        const int q0 = xlink(0, j), q1 = xlink(1, j);
        const int oq = hi ? G.off[q1] : G.off[q0];
        const uint32_t at = per ? (uint32_t)((int64_t)n - oq + wrap) : n;
        const float v = PF<S>::word(w[j], at & 1u);
        if (hi) set_k<K>(fl[q1], v);
        else set_k<K>(fl[q0], v);
    }
    const int oq = hi ? G.off[2] : G.off[1];
    const uint32_t at = per ? (uint32_t)((int64_t)n - oq + wrap) : n;
    float v = PG<S>::word(w[5], at & 1u);
    if (!per && ((P.dir_mask >> (hi ? 1 : 0)) & 1)) v = kGs<S> * (hi ? P.abbT[1] : P.abbT[0]) - v; // through the face
    if (hi) set_k<K>(gl[2], v);
    else set_k<K>(gl[1], v);
}

// The links that leave an x-face node through its face: bounce-back into the
// node's own opposite slot (anti-bounce-back for g at a Dirichlet face), or
// the far end of the row when x is periodic.
template <int S, int K>
__device__ __forceinline__ void xface_out(SF<S> *f, SG<S> *g, const float2 (&fl)[19], const float2 (&gl)[7],
                                          uint32_t n, uint32_t rb, bool hi, const Geom &G, const Phys &P) {
    const bool per = G.periodic & 1;
    const int64_t s = G.stride;
    const int64_t wrap = hi ? (int64_t)G.nx : -(int64_t)G.nx; // x = 0 leaves along -x
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        const int qa = xlink(1, j), qb = xlink(0, j); // e_x = -1 at x = 0, +1 at x = nx-1
        const float2 u = hi ? fl[qb] : fl[qa];
        const float v = K == 0 ? u.x : u.y;
        SF<S> *p = per ? f + (hi ? qb : qa) * s + ((int64_t)n + (hi ? G.off[qb] : G.off[qa]) - wrap)
                       : f + (hi ? opp19(qb) : opp19(qa)) * s + n;
        PF<S>::st1(p, v);
    }
    const int q = hi ? 1 : 2;
    const float2 u = hi ? gl[1] : gl[2];
    float v = K == 0 ? u.x : u.y;
    SG<S> *p;
    if (per) {
        p = g + q * s + ((int64_t)n + (hi ? G.off[1] : G.off[2]) - wrap);
    } else {
        p = g + (hi ? 2 : 1) * s + n; // the opposite slot
        if ((P.dir_mask >> (hi ? 1 : 0)) & 1) v = kGs<S> * (hi ? P.abbT[1] : P.abbT[0]) - v; // leaves through the face
    }
    PG<S>::st1s(p, v, rnd_pop(rb, q));
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sptr(bar)) : "memory");
}

// Collide the pair of nodes m, mb (v0, v1: which of them this step updates)
// and store their populations: own slots, opposite direction on an even
// step; on an odd step array q at the node + e_q, the x-face nodes' links
// through their face to their own slots (or the far end of the row).
template <int S, bool ODD, bool XF>
__device__ __forceinline__ void update_pair(SF<S> *f, SG<S> *g, const Geom &G, const Phys &P, const StagedGeom &T,
                                            float2 (&fl)[19], float2 (&gl)[7], uint32_t m, uint32_t mb, bool v0,
                                            bool v1, bool lo0, bool hi0, bool lo1, bool hi1) {
    const int64_t s = G.stride;
    collide<float2, kGRaw<S>>(P, fl, gl);
    SF<S> *fo = f;
    SG<S> *go = g;
    asm volatile("" : "+l"(fo), "+l"(go)); // recompute addresses after the collision
    if (!ODD) {
        // own node, opposite slot; a pair that ends past the last node
        // writes the first padding element, which no node reads
        if (v0) {
#pragma unroll
            for (int q = 0; q < 19; ++q) PF<S>::st(fo + opp19(q) * s + m, fl[q]);
            const uint32_t rb0 = SRG(S) ? rnd_node(m, P.t) : 0u, rb1 = SRG(S) ? rnd_node(mb, P.t) : 0u;
#pragma unroll
            for (int q = 0; q < 7; ++q)
                PG<S>::sts(go + opp7(q) * s + m, gl[q], rnd_pop(rb0, q), rnd_pop(rb1, q));
        }
    } else {
        // a link that leaves an x-face node through its face is stored below instead
        const bool p0 = v0 && !hi0, m0 = v0 && !lo0, p1 = v1 && !hi1, m1 = v1 && !lo1;
        // destination: array q at the node + e_q, a byte offset per q from
        // the node's own element
        const char *fm = reinterpret_cast<const char *>(fo + m), *gm = reinterpret_cast<const char *>(go + m);
#pragma unroll
        for (int q = 0; q < 19; ++q) {
            SF<S> *p = reinterpret_cast<SF<S> *>(const_cast<char *>(fm) + T.soff[q]);
            const bool c0 = ex19(q) > 0 ? p0 : ex19(q) < 0 ? m0 : v0;
            const bool c1 = ex19(q) > 0 ? p1 : ex19(q) < 0 ? m1 : v1;
            if (c0) PF<S>::st1(p, fl[q].x);
            if (c1) PF<S>::st1(p + 32, fl[q].y);
        }
        const uint32_t rb0 = SRG(S) ? rnd_node(m, P.t) : 0u, rb1 = SRG(S) ? rnd_node(mb, P.t) : 0u;
#pragma unroll
        for (int q = 0; q < 7; ++q) {
            SG<S> *p = reinterpret_cast<SG<S> *>(const_cast<char *>(gm) + T.soff[19 + q]);
            const bool c0 = ex7(q) > 0 ? p0 : ex7(q) < 0 ? m0 : v0;
            const bool c1 = ex7(q) > 0 ? p1 : ex7(q) < 0 ? m1 : v1;
            if (c0) PG<S>::st1s(p, gl[q].x, rnd_pop(rb0, q));
            if (c1) PG<S>::st1s(p + 32, gl[q].y, rnd_pop(rb1, q));
        }
        if (XF && (lo0 || hi0 || lo1 || hi1)) {
            if (lo0 || hi0) xface_out<S, 0>(fo, go, fl, gl, m, rb0, hi0, G, P);
            if (lo1 || hi1) xface_out<S, 1>(fo, go, fl, gl, mb, rb1, hi1, G, P);
        }
    }
}

// Hand-over of the stages: a compute warp waits for a stage's "full" barrier
// (the bulk copies' bytes, plus the x-face words), reads its nodes' values
// into registers and arrives on the stage's "empty" barrier (one arrival per
// compute warp) before it updates the nodes; warp 0 refills a stage once
// its empty barrier has completed.  On an odd step warp 0 only issues copies;
// on an even step it also computes, and refills the stage of each tile once
// every warp has read it, before updating its own nodes of it.  No
// block-wide barrier is taken per tile: a
// bulk copy's operands come from uniform registers, so a warp issues its
// lanes' copies one after another, and with a block barrier every warp
// waited for that serial issue each tile (a third of the time of a tile).
// A dedicated producer pays on the odd step (the one with more work per node,
// 15% faster at 257^3); on the even step, which runs near the copy bandwidth,
// the eighth compute warp pays more.
template <int S, bool ODD, bool XF>
__global__ void __launch_bounds__(kThreads, 2)
    k_aa_staged(SF<S> *__restrict__ f, SG<S> *__restrict__ g, Geom G, Phys P, StagedGeom T, int *err) {
    using St = Stage<S, ODD>;
    constexpr int NST = St::count;
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    uint64_t *empty = full + NST;
    int *wofs = reinterpret_cast<int *>(smem + 64); // [NST][kWofs]: window offsets of each stage
    int *fills = reinterpret_cast<int *>(smem + 512); // [NST]: fills issued into each stage
    unsigned char *stages = smem + kHead;
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const uint32_t ntiles = ODD ? T.odd_tiles : T.even_tiles;

    if (tid == 0) {
        for (int k = 0; k < NST; ++k) {
            mbar_init(&full[k], XF ? 33u : 1u); // + one per lane's word copies
            mbar_init(&empty[k], (unsigned)kCompute<ODD>);
            fills[k] = 0;
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    // programmatic dependent launch: the next kernel's blocks may be
    // scheduled as this one's retire, and this one reads nothing before the
    // kernel before it has completed
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");

    if (ODD && warp == 0) {
        int j = 0;
        for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++j) {
            const int st = j % NST;
            if (j >= NST) { // the stage's previous tile has been read by every compute warp
                const bool ok = mbar_wait(&empty[st], (unsigned)(j / NST - 1) & 1u, T.budget);
                if (__any_sync(0xffffffffu, !ok)) {
                    if (lane == 0) atomicExch(err, 1);
                    break;
                }
            }
            const TileSpan sp = tile_span<ODD>(G, T, t);
            unsigned char *sb = stages + st * St::bytes;
            issue_tile<S, ODD>(f, g, G, sp, sb, wofs + kWofs * st, &full[st], lane);
            if (XF) issue_side<S>(f, g, G, sp, sb, &full[st], lane);
            if (lane == 0) fills[st] = j / NST + 1;
        }
    } else {
        if (!ODD && warp == 0) // the first tiles of every stage
            for (int k = 0; k < NST; ++k) {
                const uint32_t t = blockIdx.x + (uint32_t)k * gridDim.x;
                if (t >= ntiles) break;
                issue_tile<S, ODD>(f, g, G, tile_span<ODD>(G, T, t), stages + k * St::bytes, wofs + kWofs * k,
                                   &full[k], lane);
                if (lane == 0) fills[k] = 1;
            }
        const int cw = ODD ? warp - 1 : warp; // compute warp
        int j = 0;
        for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++j) {
            const int st = j % NST;
            const unsigned parity = (unsigned)(j / NST) & 1u;
            const TileSpan sp = tile_span<ODD>(G, T, t);
            // even step: nodes m, m + 1; odd step: m, m + 32
            const uint32_t o = ODD ? 64u * (uint32_t)cw + (uint32_t)lane : 64u * (uint32_t)cw + 2u * (uint32_t)lane;
            const uint32_t m = sp.n0 + o;
            const uint32_t mb = m + (ODD ? 32u : 1u);
            bool v0 = m >= sp.lo && m < sp.hi;
            bool v1 = mb >= sp.lo && mb < sp.hi;
            bool lo0 = false, hi0 = false, lo1 = false, hi1 = false; // x-face nodes (XF)
            uint32_t r0 = 0, r1 = 0;                                  // their rows
            if (ODD) {
                const uint32_t nx = (uint32_t)G.nx;
                r0 = fast_div(m, G.mag_nx);
                const uint32_t xa = m - nx * r0;
                // mb = m + 32 lies at most 32 / nx rows further (two for nx >= 16)
                uint32_t xb = xa + 32u;
                r1 = r0;
                if (xb >= nx) { xb -= nx; ++r1; }
                if (xb >= nx) { xb -= nx; ++r1; }
                if (nx < 16u) { r1 = fast_div(mb, G.mag_nx); xb = mb - nx * r1; }
                if (XF) {
                    lo0 = v0 && xa == 0u;
                    hi0 = v0 && xa == nx - 1u;
                    lo1 = v1 && xb == 0u;
                    hi1 = v1 && xb == nx - 1u;
                } else { // nodes next to an x face belong to the face kernel
                    v0 = v0 && xa != 0u && xa != nx - 1u;
                    v1 = v1 && xb != 0u && xb != nx - 1u;
                }
            }

            const bool ok = mbar_wait(&full[st], parity, T.budget);
            if (__any_sync(0xffffffffu, !ok)) {
                if (lane == 0) atomicExch(err, 1);
                break;
            }
            const unsigned char *sb = stages + st * St::bytes;
            float2 fl[19], gl[7];
            if (!ODD) {
                // even tiles start on a 16-byte boundary of every array, so the
                // windows are not shifted
#pragma unroll
                for (int q = 0; q < 19; ++q)
                    fl[q] = PF<S>::ld(reinterpret_cast<const SF<S> *>(sb + St::offset(q)) + o);
#pragma unroll
                for (int q = 0; q < 7; ++q)
                    gl[q] = PG<S>::ld(reinterpret_cast<const SG<S> *>(sb + St::offset(19 + q)) + o);
            } else {
                // the stage's window offsets, four per 16-byte load
                int wo[kWofs];
                const int4 *w4 = reinterpret_cast<const int4 *>(wofs + kWofs * st);
#pragma unroll
                for (int k = 0; k < kWofs / 4; ++k) {
                    const int4 v = w4[k];
                    wo[4 * k] = v.x;
                    wo[4 * k + 1] = v.y;
                    wo[4 * k + 2] = v.z;
                    wo[4 * k + 3] = v.w;
                }
                const unsigned char *bf = sb + sizeof(SF<S>) * o, *bg = sb + sizeof(SG<S>) * o;
#pragma unroll
                for (int q = 0; q < 19; ++q) {
                    const SF<S> *w = reinterpret_cast<const SF<S> *>(bf + wo[q]);
                    fl[q] = make_float2(PF<S>::one(w[0]), PF<S>::one(w[32]));
                }
#pragma unroll
                for (int q = 0; q < 7; ++q) {
                    const SG<S> *w = reinterpret_cast<const SG<S> *>(bg + wo[19 + q]);
                    gl[q] = make_float2(PG<S>::one(w[0]), PG<S>::one(w[32]));
                }
                if (XF && (lo0 || hi0 || lo1 || hi1)) {
                    const uint32_t *side = reinterpret_cast<const uint32_t *>(sb + St::win);
                    const uint32_t row0 = fast_div(sp.n0, G.mag_nx);
                    if (lo0 || hi0) xface_in<S, 0>(fl, gl, side + 12u * (r0 - row0) + (hi0 ? 6u : 0u), m, hi0, G, P);
                    if (lo1 || hi1) xface_in<S, 1>(fl, gl, side + 12u * (r1 - row0) + (hi1 ? 6u : 0u), mb, hi1, G, P);
                }
            }
            // this warp is done with the stage
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[st]);
            if (!ODD && warp == 0) { // refill the stage once every warp has read it
                const uint32_t tn = t + (uint32_t)NST * gridDim.x;
                if (tn < ntiles) {
                    const bool ready = mbar_wait(&empty[st], parity, T.budget);
                    if (__any_sync(0xffffffffu, !ready)) {
                        if (lane == 0) atomicExch(err, 1);
                        break;
                    }
                    issue_tile<S, ODD>(f, g, G, tile_span<ODD>(G, T, tn), stages + st * St::bytes,
                                       wofs + kWofs * st, &full[st], lane);
                    if (lane == 0) fills[st] = j / NST + 2;
                }
            }
            if (v0 || v1) update_pair<S, ODD, XF>(f, g, G, P, T, fl, gl, m, mb, v0, v1, lo0, hi0, lo1, hi1);
        }
    }
    // after a timeout, let the copies still in flight land before the block exits
    __syncthreads();
    if (tid == 0)
        for (int k = 0; k < NST; ++k)
            if (fills[k] > 0) mbar_wait(&full[k], (unsigned)(fills[k] - 1) & 1u, kDrain);
}

template <int S> cudaError_t staged_attr(int *blocks_per_sm) {
    const void *fn[3] = {reinterpret_cast<const void *>(&k_aa_staged<S, false, false>),
                         reinterpret_cast<const void *>(&k_aa_staged<S, true, false>),
                         reinterpret_cast<const void *>(&k_aa_staged<S, true, true>)};
    const int bytes[3] = {Stage<S, false>::smem, Stage<S, true>::smem, Stage<S, true>::smem};
    int least = 1 << 30;
    for (int i = 0; i < 3; ++i) {
        cudaError_t e = cudaFuncSetAttribute(fn[i], cudaFuncAttributeMaxDynamicSharedMemorySize, bytes[i]);
        int per = 0;
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn[i], kThreads, bytes[i]);
        if (e != cudaSuccess) return e;
        least = per < least ? per : least;
    }
    *blocks_per_sm = least;
    return cudaSuccess;
}

template <int S> cudaError_t staged_launch(const StepArgs &a) {
    SF<S> *f = static_cast<SF<S> *>(a.f);
    SG<S> *g = static_cast<SG<S> *>(a.g);
    Geom G = a.G;
    Phys P = a.P;
    StagedGeom T = a.T;
    int *err = a.err;
    void *args[] = {&f, &g, &G, &P, &T, &err};
    if (a.parity == 0)
        return pdl_launch(reinterpret_cast<const void *>(&k_aa_staged<S, false, false>), T.grid, kThreads,
                          Stage<S, false>::smem, a.stream, args);
    if (T.odd_tiles) {
        const void *fn = T.xf ? reinterpret_cast<const void *>(&k_aa_staged<S, true, true>)
                              : reinterpret_cast<const void *>(&k_aa_staged<S, true, false>);
        const cudaError_t e = pdl_launch(fn, T.grid, kThreads, Stage<S, true>::smem, a.stream, args);
        if (e != cudaSuccess) return e;
    }
    // the nodes next to a y or z face (and, for rows shorter than kXfMinNx,
    // those next to an x face) go through the general face kernel
    return launch_face(a, T.xf ? a.nface_yz : a.nface);
}

} // namespace

cudaError_t pdl_launch(const void *fn, int grid, int block, int smem, cudaStream_t stream, void **args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, fn, args);
}

int staged_tile_nodes(int odd) { return odd ? kTile<true> : kTile<false>; }

int staged_xf_min_nx() { return kXfMinNx; }

void staged_store_offsets(int storage, const Geom &G, StagedGeom &T) {
    const int64_t ef = storage == ST_F32 ? 4 : 2, eg = (storage == ST_F32 || storage == ST_F16M) ? 4 : 2;
    for (int q = 0; q < 19; ++q) T.soff[q] = (q * G.stride + G.off[q]) * ef;
    for (int q = 0; q < 7; ++q) T.soff[19 + q] = (q * G.stride + G.off[q]) * eg;
}

cudaError_t staged_prepare(int storage, int *blocks_per_sm) {
    switch (storage) {
    case ST_F32: return staged_attr<ST_F32>(blocks_per_sm);
    case ST_F16: return staged_attr<ST_F16>(blocks_per_sm);
    case ST_F16M: return staged_attr<ST_F16M>(blocks_per_sm);
    default: return staged_attr<ST_BF16>(blocks_per_sm);
    }
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
