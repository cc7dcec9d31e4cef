// Time-step kernels of the thermal lattice Boltzmann library and the kernels
// that move a state between the device layouts and a plain natural layout.
//
// One thread updates one node: it loads the 19 + 7 populations arriving at
// the node, runs the fused D3Q19 + D3Q7 MRT collision (Eq. MRT, Eq. MRT_T)
// in registers, applies the wall rules of Secs. 2.2-2.3 for links that cross
// a wall, and stores the 26 post-collision populations.  Population arrays
// are structure-of-arrays with x fastest, so a warp reads and writes 32
// consecutive nodes of each array.
//
// Device layouts of a state:
//   LAYOUT_NATURAL   A[i][x] = f_i(x, t), the pre-collision populations.
//   LAYOUT_REVERSED  A[ibar][x] = f_i+(x, t-1): the AA pattern after an even
//                    step (post-collision values kept in the opposite slot of
//                    their own node, not yet streamed).
//   LAYOUT_PULL      B[i][x] = f_i+(x, t-1): the two-buffer pull scheme.
// In both post-collision layouts, a link that arrives at x from a wall takes
// the value that left x towards that wall, f_ibar+(x, t-1) (bounce-back); g
// takes the same value, or minus it plus (6 + a_T)/21 T_w at a Dirichlet wall
// (anti-bounce-back).
#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace lbm {

enum Layout { LAYOUT_NATURAL = 0, LAYOUT_REVERSED = 1, LAYOUT_PULL = 2 };


// Read the pre-collision populations of node (x, y, z) from a device layout.
template <int S>
__device__ __forceinline__ void read_natural(const SEF<S> *__restrict__ f, const SEG<S> *__restrict__ g,
                                             const Geom &G, const Phys &P, int layout, uint32_t n,
                                             int x, int y, int z, float (&fl)[19], float (&gl)[7]) {
    const int64_t s = G.stride;
    if (layout == LAYOUT_NATURAL) {
#pragma unroll
        for (int i = 0; i < 19; ++i) fl[i] = Store<FS(S)>::ld(f + i * s + n);
#pragma unroll
        for (int i = 0; i < 7; ++i) gl[i] = Store<GS(S)>::ld(g + i * s + n);
        return;
    }
    const Nbr b = neighbours(G, x, y, z);
    const bool rev = layout == LAYOUT_REVERSED;
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const int slot_in = rev ? opp19(i) : i, slot_wall = rev ? i : opp19(i);
        if (!src_wall(b, ex19(i), ey19(i), ez19(i)))
            fl[i] = Store<FS(S)>::ld(f + slot_in * s + (int64_t)n + src_off(b, ex19(i), ey19(i), ez19(i)));
        else
            fl[i] = Store<FS(S)>::ld(f + slot_wall * s + n);
    }
#pragma unroll
    for (int i = 0; i < 7; ++i) {
        const int slot_in = rev ? opp7(i) : i, slot_wall = rev ? i : opp7(i);
        if (!src_wall(b, ex7(i), ey7(i), ez7(i))) {
            gl[i] = Store<GS(S)>::ld(g + slot_in * s + (int64_t)n + src_off(b, ex7(i), ey7(i), ez7(i)));
        } else {
            const int fc = face_of(-ex7(i), -ey7(i), -ez7(i));
            const float v = Store<GS(S)>::ld(g + slot_wall * s + n);
            gl[i] = ((P.dir_mask >> fc) & 1) ? P.abbT[fc] - v : v;
        }
    }
}

// ------------------------------------------------------------ AA pattern ----

// Even step: natural -> reversed.  Reads and writes only the node's own slots.
template <int S, bool MOM>
__global__ void __launch_bounds__(256, 3) k_aa_even(SEF<S> *__restrict__ f, SEG<S> *__restrict__ g, Geom G,
                                                 Phys P, float *__restrict__ mom) {
    const uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= G.n) return;
    const int64_t s = G.stride;
    float fl[19], gl[7];
#pragma unroll
    for (int i = 0; i < 19; ++i) fl[i] = Store<FS(S)>::ld(f + i * s + n);
#pragma unroll
    for (int i = 0; i < 7; ++i) gl[i] = Store<GS(S)>::ld(g + i * s + n);
    float g0[7];
#pragma unroll
    for (int i = 0; i < 7; ++i) g0[i] = gl[i];
    const Macro m = collide(P, fl, gl);
    f = opaque(f);
    g = opaque(g);
#pragma unroll
    for (int i = 0; i < 19; ++i) Store<FS(S)>::st(f + opp19(i) * s + n, fl[i]);
    const uint32_t rb = SRG(S) ? rnd_node(n, P.t) : 0u;
#pragma unroll
#pragma unroll
    for (int i = 0; i < 7; ++i) Store<GS(S)>::sts(g + opp7(i) * s + n, gl[i], rnd_pop(rb, i));
    if (MOM) {
        int x, y, z;
        node_xyz(G, n, x, y, z);
        write_sample(mom, s, n, m, neighbours(G, x, y, z), g0);
    }
}

// Odd step: reversed -> natural.  Gathers f_i+(x - e_i) from the opposite
// slot of the upstream node and scatters f_i+(x) to slot i of x + e_i; every
// location a thread reads is written by that same thread only, so the update
// is in place without a second buffer, and any partition of the nodes into
// separately launched sets is valid.  Interior nodes (no face next to them)
// take the uniform offsets e_i of the flat index; nodes next to a face go
// through the general path with wrap-around and wall rules.
template <int S, bool MOM>
__global__ void __launch_bounds__(256, 3) k_aa_odd_interior(SEF<S> *__restrict__ f, SEG<S> *__restrict__ g,
                                                            Geom G, Phys P, float *__restrict__ mom) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= G.ni) return;
    const uint32_t zi = fast_div(t, G.mag_nixy);
    const uint32_t r = t - zi * G.nixy;
    const uint32_t yi = fast_div(r, G.mag_nix);
    const uint32_t xi = r - yi * G.nix;
    const uint32_t n = (xi + 1) + static_cast<uint32_t>(G.nx) * ((yi + 1) + static_cast<uint32_t>(G.ny) * (zi + 1));
    const int64_t s = G.stride;
    float fl[19], gl[7];
    fl[0] = Store<FS(S)>::ld(f + n);
#pragma unroll
    for (int i = 1; i < 19; ++i) fl[i] = Store<FS(S)>::ld(f + opp19(i) * s + (int64_t)(n - G.off[i]));
    gl[0] = Store<GS(S)>::ld(g + n);
#pragma unroll
    for (int i = 1; i < 7; ++i) gl[i] = Store<GS(S)>::ld(g + opp7(i) * s + (int64_t)(n - G.off[i]));
    const Macro m = collide(P, fl, gl);
    f = opaque(f);
    g = opaque(g);
    Store<FS(S)>::st(f + n, fl[0]);
#pragma unroll
    for (int i = 1; i < 19; ++i) Store<FS(S)>::st(f + i * s + (int64_t)(n + G.off[i]), fl[i]);
    const uint32_t rb = SRG(S) ? rnd_node(n, P.t) : 0u;
    Store<GS(S)>::sts(g + n, gl[0], rnd_pop(rb, 0));
#pragma unroll
    for (int i = 1; i < 7; ++i) Store<GS(S)>::sts(g + i * s + (int64_t)(n + G.off[i]), gl[i], rnd_pop(rb, i));
    if (MOM) {
        mom[n] = m.drho;
        mom[s + n] = m.u;
        mom[2 * s + n] = m.v;
        mom[3 * s + n] = m.w;
        mom[4 * s + n] = m.T;
    }
}

// Nodes next to a face, listed in `list`.  With the 2-byte storages two per
// thread (a warp takes 64 consecutive entries, lane l the entries l and
// l + 32), so that the collision runs on the packed FP32 instructions: the
// FP16 odd step at 257^3 is 4% shorter.  With FP32 one per thread: the two-node
// form needs more than 128 registers there and gains nothing (small cells
// lose 1%).  A block covers kFacePer<S> * bdim entries.
template <int S, bool MOM>
__device__ __forceinline__ void k_aa_odd_face_tile(SEF<S> *__restrict__ f, SEG<S> *__restrict__ g, const Geom &G,
                                                        const Phys &P, float *__restrict__ mom,
                                                        const uint32_t *__restrict__ list, uint32_t count, uint32_t blk, uint32_t tid, uint32_t bdim) {
    if (kFacePer<S> == 1) {
        const uint32_t t = blk * bdim + tid;
        if (t >= count) return;
        odd_step_node<S, MOM>(f, g, G, P, mom, list[t]);
    } else {
        const uint32_t a = 2u * (blk * bdim + (tid & ~31u)) + (tid & 31u);
        if (a >= count) return;
        const bool vb = a + 32u < count;
        odd_step_node2<S, MOM>(f, g, G, P, mom, list[a], vb ? list[a + 32u] : 0u, vb);
    }
}

template <int S, bool MOM>
__global__ void __launch_bounds__(256, kFacePer<S> == 1 ? 3 : 2) k_aa_odd_face(SEF<S> *__restrict__ f, SEG<S> *__restrict__ g, Geom G,
                                                        Phys P, float *__restrict__ mom,
                                                        const uint32_t *__restrict__ list, uint32_t count) {
    k_aa_odd_face_tile<S, MOM>(f, g, G, P, mom, list, count, blockIdx.x, threadIdx.x, blockDim.x);
}

// ------------------------------------------- two nodes per thread (f32x2) ----
//
// The same updates with one thread per two nodes: the collision runs on
// float2 values with the packed FP32 instructions, halving its instruction
// count per node.  Even step: nodes 2t and 2t+1 share aligned vector loads
// and stores (for an odd node count the last pair includes the first padding
// element, which no real node ever reads).

template <int S, bool MOM>
__device__ __forceinline__ void k_aa_even2_tile(SEF<S> *__restrict__ f, SEG<S> *__restrict__ g, const Geom &G,
                                                     const Phys &P, float *__restrict__ mom, uint32_t blk, uint32_t tid, uint32_t bdim) {
    const uint32_t n = 2u * (blk * bdim + tid);
    if (n >= G.n) return;
    const int64_t s = G.stride;
    float2 fl[19], gl[7];
#pragma unroll
    for (int i = 0; i < 19; ++i) fl[i] = Store2<FS(S)>::ld(f + i * s + n);
#pragma unroll
    for (int i = 0; i < 7; ++i) gl[i] = Store2<GS(S)>::ld(g + i * s + n);
    float2 g0[7];
#pragma unroll
    for (int i = 0; i < 7; ++i) g0[i] = gl[i];
    const MacroT<float2> m = collide(P, fl, gl);
    f = opaque(f);
    g = opaque(g);
#pragma unroll
    for (int i = 0; i < 19; ++i) Store2<FS(S)>::st(f + opp19(i) * s + n, fl[i]);
    const uint32_t rb0 = SRG(S) ? rnd_node(n, P.t) : 0u, rb1 = SRG(S) ? rnd_node(n + 1u, P.t) : 0u;
#pragma unroll
#pragma unroll
    for (int i = 0; i < 7; ++i) Store2<GS(S)>::sts(g + opp7(i) * s + n, gl[i], rnd_pop(rb0, i), rnd_pop(rb1, i));
    if (MOM) {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const uint32_t nk = n + k;
            if (nk >= G.n) break;
            Macro mk;
            mk.drho = k ? m.drho.y : m.drho.x;
            mk.u = k ? m.u.y : m.u.x;
            mk.v = k ? m.v.y : m.v.x;
            mk.w = k ? m.w.y : m.w.x;
            mk.T = k ? m.T.y : m.T.x;
            float gk[7];
#pragma unroll
            for (int i = 0; i < 7; ++i) gk[i] = k ? g0[i].y : g0[i].x;
            int x, y, z;
            node_xyz(G, nk, x, y, z);
            write_sample(mom, s, nk, mk, neighbours(G, x, y, z), gk);
        }
    }
}

template <int S, bool MOM>
__global__ void __launch_bounds__(256, 2) k_aa_even2(SEF<S> *__restrict__ f, SEG<S> *__restrict__ g, Geom G,
                                                     Phys P, float *__restrict__ mom) {
    k_aa_even2_tile<S, MOM>(f, g, G, P, mom, blockIdx.x, threadIdx.x, blockDim.x);
}

__device__ __forceinline__ uint32_t interior_node(const Geom &G, uint32_t t) {
    const uint32_t zi = fast_div(t, G.mag_nixy);
    const uint32_t r = t - zi * G.nixy;
    const uint32_t yi = fast_div(r, G.mag_nix);
    const uint32_t xi = r - yi * G.nix;
    return (xi + 1) + static_cast<uint32_t>(G.nx) * ((yi + 1) + static_cast<uint32_t>(G.ny) * (zi + 1));
}

// Odd step over the rows with 1 <= y <= ny-2 and 1 <= z <= nz-2, which lie
// contiguously in each z-plane.  A warp takes 64 consecutive nodes of such a
// run, lane l the nodes l and l + 32, so every access of the warp is
// contiguous and the second node's addresses are the first's plus 32.  Lanes
// past the end of the run load in bounds and store nothing.
//
// Nodes at x = 0 or x = nx-1 are updated here too: a link that arrives
// through the x face takes the node's own opposite slot (bounce-back, with
// anti-bounce-back for g at a Dirichlet face) or, when x is periodic, the
// far end of the row; a link that leaves through it is stored there.  Only
// the addresses change, chosen per lane, so these nodes cost no extra loads.
template <int S, bool MOM>
__device__ __forceinline__ void k_aa_odd_rows_tile(SEF<S> *__restrict__ f, SEG<S> *__restrict__ g, const Geom &G,
                                                        const Phys &P, float *__restrict__ mom, uint32_t blk, uint32_t tid, uint32_t bdim) {
    const uint32_t warp = blk * (bdim >> 5) + (tid >> 5);
    const uint32_t lane = tid & 31u;
    const uint32_t zi = fast_div(warp, G.mag_cpp);
    if (zi >= static_cast<uint32_t>(G.nz - 2)) return;
    const uint32_t c = warp - zi * G.cpp;
    const uint32_t nx = static_cast<uint32_t>(G.nx);
    const uint32_t len = nx * static_cast<uint32_t>(G.ny - 2);
    const uint32_t o0 = c * 64u + lane;
    const uint32_t n0 = nx * (1u + static_cast<uint32_t>(G.ny) * (zi + 1u)) + o0;
    const uint32_t x0 = n0 - nx * fast_div(n0, G.mag_nx);
    const uint32_t x1 = (n0 + 32u) - nx * fast_div(n0 + 32u, G.mag_nx);
    const bool a0 = o0 < len;
    const bool a1 = o0 + 32u < len;
    if (!a0 && !a1) return;
    const bool lo0 = a0 && x0 == 0u, hi0 = a0 && x0 == nx - 1u;
    const bool lo1 = a1 && x1 == 0u, hi1 = a1 && x1 == nx - 1u;
    const bool per = G.periodic & 1;
    const int64_t s = G.stride;
    float2 fl[19], gl[7];
    fl[0] = make_float2(Store<FS(S)>::ld(f + n0), Store<FS(S)>::ld(f + n0 + 32));
#pragma unroll
    for (int i = 1; i < 19; ++i) {
        const SEF<S> *q = f + opp19(i) * s + (int64_t)(n0 - G.off[i]);
        if (ex19(i) == 0) {
            fl[i] = make_float2(Store<FS(S)>::ld(q), Store<FS(S)>::ld(q + 32));
        } else {
            // the link arrives through the x face at lo (e_x = +1) or hi (e_x = -1) nodes
            const bool w0 = ex19(i) > 0 ? lo0 : hi0, w1 = ex19(i) > 0 ? lo1 : hi1;
            const SEF<S> *own = per ? q + (ex19(i) > 0 ? (int64_t)nx : -(int64_t)nx) : f + i * s + n0;
            fl[i] = make_float2(Store<FS(S)>::ld(w0 ? own : q), Store<FS(S)>::ld(w1 ? own + 32 : q + 32));
        }
    }
    gl[0] = make_float2(Store<GS(S)>::ld(g + n0), Store<GS(S)>::ld(g + n0 + 32));
#pragma unroll
    for (int i = 1; i < 7; ++i) {
        const SEG<S> *q = g + opp7(i) * s + (int64_t)(n0 - G.off[i]);
        if (ex7(i) == 0) {
            gl[i] = make_float2(Store<GS(S)>::ld(q), Store<GS(S)>::ld(q + 32));
        } else {
            const bool w0 = ex7(i) > 0 ? lo0 : hi0, w1 = ex7(i) > 0 ? lo1 : hi1;
            const SEG<S> *own = per ? q + (ex7(i) > 0 ? (int64_t)nx : -(int64_t)nx) : g + i * s + n0;
            float2 v = make_float2(Store<GS(S)>::ld(w0 ? own : q), Store<GS(S)>::ld(w1 ? own + 32 : q + 32));
            const int fc = ex7(i) > 0 ? 0 : 1; // face the link comes through
            if (!per && ((P.dir_mask >> fc) & 1)) {
                if (w0) v.x = P.abbT[fc] - v.x;
                if (w1) v.y = P.abbT[fc] - v.y;
            }
            gl[i] = v;
        }
    }
    // pre-collision g arriving from the x faces (diagnostic sample)
    const float gin_lo0 = gl[1].x, gin_lo1 = gl[1].y, gin_hi0 = gl[2].x, gin_hi1 = gl[2].y;
    const MacroT<float2> m = collide(P, fl, gl);
    f = opaque(f);
    g = opaque(g);
    if (a0) Store<FS(S)>::st(f + n0, fl[0].x);
    if (a1) Store<FS(S)>::st(f + n0 + 32, fl[0].y);
#pragma unroll
    for (int i = 1; i < 19; ++i) {
        SEF<S> *q = f + i * s + (int64_t)(n0 + G.off[i]);
        if (ex19(i) == 0) {
            if (a0) Store<FS(S)>::st(q, fl[i].x);
            if (a1) Store<FS(S)>::st(q + 32, fl[i].y);
        } else {
            // the link leaves through the x face at hi (e_x = +1) or lo (e_x = -1) nodes
            const bool w0 = ex19(i) > 0 ? hi0 : lo0, w1 = ex19(i) > 0 ? hi1 : lo1;
            SEF<S> *own = per ? q - (ex19(i) > 0 ? (int64_t)nx : -(int64_t)nx) : f + opp19(i) * s + n0;
            if (a0) Store<FS(S)>::st(w0 ? own : q, fl[i].x);
            if (a1) Store<FS(S)>::st(w1 ? own + 32 : q + 32, fl[i].y);
        }
    }
    const uint32_t rb0 = SRG(S) ? rnd_node(n0, P.t) : 0u, rb1 = SRG(S) ? rnd_node(n0 + 32u, P.t) : 0u;
    if (a0) Store<GS(S)>::sts(g + n0, gl[0].x, rnd_pop(rb0, 0));
    if (a1) Store<GS(S)>::sts(g + n0 + 32, gl[0].y, rnd_pop(rb1, 0));
#pragma unroll
    for (int i = 1; i < 7; ++i) {
        SEG<S> *q = g + i * s + (int64_t)(n0 + G.off[i]);
        if (ex7(i) == 0) {
            if (a0) Store<GS(S)>::sts(q, gl[i].x, rnd_pop(rb0, i));
            if (a1) Store<GS(S)>::sts(q + 32, gl[i].y, rnd_pop(rb1, i));
        } else {
            const bool w0 = ex7(i) > 0 ? hi0 : lo0, w1 = ex7(i) > 0 ? hi1 : lo1;
            SEG<S> *own = per ? q - (ex7(i) > 0 ? (int64_t)nx : -(int64_t)nx) : g + opp7(i) * s + n0;
            float2 v = gl[i];
            const int fc = ex7(i) > 0 ? 1 : 0; // face the link leaves through
            if (!per && ((P.dir_mask >> fc) & 1)) {
                if (w0) v.x = P.abbT[fc] - v.x;
                if (w1) v.y = P.abbT[fc] - v.y;
            }
            if (a0) Store<GS(S)>::sts(w0 ? own : q, v.x, rnd_pop(rb0, i));
            if (a1) Store<GS(S)>::sts(w1 ? own + 32 : q + 32, v.y, rnd_pop(rb1, i));
        }
    }
    if (MOM) {
        if (a0) {
            mom[n0] = m.drho.x;
            mom[s + n0] = m.u.x;
            mom[2 * s + n0] = m.v.x;
            mom[3 * s + n0] = m.w.x;
            mom[4 * s + n0] = m.T.x;
            if (lo0 && !per) mom[5 * s + n0] = gin_lo0;
            if (hi0 && !per) mom[6 * s + n0] = gin_hi0;
        }
        if (a1) {
            const uint32_t n1 = n0 + 32u;
            mom[n1] = m.drho.y;
            mom[s + n1] = m.u.y;
            mom[2 * s + n1] = m.v.y;
            mom[3 * s + n1] = m.w.y;
            mom[4 * s + n1] = m.T.y;
            if (lo1 && !per) mom[5 * s + n1] = gin_lo1;
            if (hi1 && !per) mom[6 * s + n1] = gin_hi1;
        }
    }
}

template <int S, bool MOM>
__global__ void __launch_bounds__(256, 2) k_aa_odd_rows(SEF<S> *__restrict__ f, SEG<S> *__restrict__ g, Geom G,
                                                        Phys P, float *__restrict__ mom) {
    k_aa_odd_rows_tile<S, MOM>(f, g, G, P, mom, blockIdx.x, threadIdx.x, blockDim.x);
}

// ------------------------------------------------- batched persistent launch ----
//
// Many independent cells advance in one launch.  The cells' tiles (a tile is
// a run of consecutive blocks of one cell's single-cell kernels: 512-node
// pair ranges of the even step, 512-node row chunks of the odd step, or
// ranges of face nodes; the run length is the schedule's tile span) are
// listed per step parity; the blocks of a persistent grid stride over the
// list and meet at a grid-wide barrier after every time step.  The launch is
// cooperative, so all blocks are resident; the barrier still gives up after
// a cycle budget and reports it instead of waiting forever.

template <int S, int BS>
__global__ void __launch_bounds__(BS, BS == 128 ? 3 : 2)
    k_batch(const CellDev *__restrict__ cells, const Tile *__restrict__ even, int n_even, const Tile *__restrict__ odd,
            int n_odd, int nsteps, int parity0, GridBarrier *bar, long long budget) {
    // the current tile's cell description, staged in shared memory so that its
    // fields are re-read cheaply instead of held in registers
    __shared__ CellDev sc;
    __shared__ Tile st;
    // steps the batch took before this launch: every block reads it before the
    // first grid barrier, block 0 advances it after the last one
    const uint32_t t0 = *reinterpret_cast<volatile unsigned *>(&bar->steps);
    for (int step = 0; step < nsteps; ++step) {
        const bool odd_step = ((parity0 + step) & 1) != 0;
        const Tile *tl = odd_step ? odd : even;
        const int nt = odd_step ? n_odd : n_even;
        for (int t = blockIdx.x; t < nt; t += gridDim.x) {
            __syncthreads();
            if (threadIdx.x == 0) {
                st = tl[t];
                sc = cells[st.cell];
                sc.P.t += t0 + (uint32_t)step; // the cell's time step (stochastic rounding counter)
            }
            __syncthreads();
            SEF<S> *f = static_cast<SEF<S> *>(sc.f);
            SEG<S> *g = static_cast<SEG<S> *>(sc.g);
            for (uint32_t k = 0; k < st.nblk; ++k) {
                const uint32_t blk = st.blk + k;
                if (st.kind == TILE_EVEN)
                    k_aa_even2_tile<S, false>(f, g, sc.G, sc.P, nullptr, blk, threadIdx.x, BS);
                else if (st.kind == TILE_ROWS)
                    k_aa_odd_rows_tile<S, false>(f, g, sc.G, sc.P, nullptr, blk, threadIdx.x, BS);
                else
                    k_aa_odd_face_tile<S, false>(f, g, sc.G, sc.P, nullptr, sc.face, sc.nface, blk, threadIdx.x, BS);
            }
        }
        if (!grid_barrier(bar, gridDim.x, budget)) return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) bar->steps = t0 + (uint32_t)nsteps;
}

// Per-step mode: one launch per time step and tile kind (even tiles; or row
// tiles, then face tiles), each a persistent grid striding over that kind's
// tiles.  The launch boundaries order the steps, so there is no grid barrier,
// and each kind gets its own register allocation (the three tile bodies in
// one kernel need 168 registers per thread, each alone at most 128).  k_bump
// advances the batch's step counter after each step.
template <int S, int KIND, int BS>
__global__ void __launch_bounds__(BS, BS == 128 ? 4 : 2)
    k_bstep(const CellDev *__restrict__ cells, const Tile *__restrict__ tl, int nt, const GridBarrier *bar) {
    __shared__ CellDev sc;
    __shared__ Tile st;
    const uint32_t t0 = *reinterpret_cast<const volatile unsigned *>(&bar->steps);
    for (int t = blockIdx.x; t < nt; t += gridDim.x) {
        __syncthreads();
        if (threadIdx.x == 0) {
            st = tl[t];
            sc = cells[st.cell];
            sc.P.t += t0;
        }
        __syncthreads();
        SEF<S> *f = static_cast<SEF<S> *>(sc.f);
        SEG<S> *g = static_cast<SEG<S> *>(sc.g);
        for (uint32_t k = 0; k < st.nblk; ++k) {
            const uint32_t blk = st.blk + k;
            if (KIND == TILE_EVEN)
                k_aa_even2_tile<S, false>(f, g, sc.G, sc.P, nullptr, blk, threadIdx.x, BS);
            else if (KIND == TILE_ROWS)
                k_aa_odd_rows_tile<S, false>(f, g, sc.G, sc.P, nullptr, blk, threadIdx.x, BS);
            else
                k_aa_odd_face_tile<S, false>(f, g, sc.G, sc.P, nullptr, sc.face, sc.nface, blk, threadIdx.x, BS);
        }
    }
}

__global__ void k_bump(GridBarrier *bar) { bar->steps += 1u; }

template <int S> static const void *bstep_kernel(int kind, int block) {
    if (block == 128)
        return kind == TILE_EVEN ? reinterpret_cast<const void *>(&k_bstep<S, TILE_EVEN, 128>)
             : kind == TILE_ROWS ? reinterpret_cast<const void *>(&k_bstep<S, TILE_ROWS, 128>)
                                 : reinterpret_cast<const void *>(&k_bstep<S, TILE_FACE, 128>);
    return kind == TILE_EVEN ? reinterpret_cast<const void *>(&k_bstep<S, TILE_EVEN, 256>)
         : kind == TILE_ROWS ? reinterpret_cast<const void *>(&k_bstep<S, TILE_ROWS, 256>)
                             : reinterpret_cast<const void *>(&k_bstep<S, TILE_FACE, 256>);
}

const void *bstep_kernel_ptr(int storage, int kind, int block) {
    switch (storage) {
    case ST_F32: return bstep_kernel<ST_F32>(kind, block);
    case ST_F16: return bstep_kernel<ST_F16>(kind, block);
    case ST_F16M: return bstep_kernel<ST_F16M>(kind, block);
    default: return bstep_kernel<ST_BF16>(kind, block);
    }
}

template <int S> static const void *batch_kernel(int block) {
    return block == 128 ? reinterpret_cast<const void *>(&k_batch<S, 128>)
                        : reinterpret_cast<const void *>(&k_batch<S, 256>);
}

const void *batch_kernel_ptr(int storage, int block) {
    switch (storage) {
    case ST_F32: return batch_kernel<ST_F32>(block);
    case ST_F16: return batch_kernel<ST_F16>(block);
    case ST_F16M: return batch_kernel<ST_F16M>(block);
    default: return batch_kernel<ST_BF16>(block);
    }
}

cudaError_t launch_batch(int storage, const BatchArgs &a) {
    if (a.mode == 1) {
        for (int k = 0; k < a.nsteps; ++k) {
            const bool odd_step = ((a.parity0 + k) & 1) != 0;
            const int kinds[2] = {odd_step ? TILE_ROWS : TILE_EVEN, odd_step ? TILE_FACE : -1};
            for (int kind : kinds) {
                if (kind < 0) continue;
                const Tile *tl = kind == TILE_EVEN ? a.even : kind == TILE_ROWS ? a.rows : a.faces;
                int nt = kind == TILE_EVEN ? a.n_even : kind == TILE_ROWS ? a.n_rows : a.n_faces;
                if (nt == 0) continue;
                const GridBarrier *bar = a.bar;
                void *args[] = {(void *)&a.cells, (void *)&tl, (void *)&nt, (void *)&bar};
                const cudaError_t e = cudaLaunchKernel(bstep_kernel_ptr(storage, kind, a.block), dim3(a.grid_k[kind]),
                                                       dim3(a.block), args, 0, a.stream);
                if (e != cudaSuccess) return e;
            }
            k_bump<<<1, 1, 0, a.stream>>>(a.bar);
            const cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    void *args[] = {(void *)&a.cells, (void *)&a.even, (void *)&a.n_even, (void *)&a.odd, (void *)&a.n_odd,
                    (void *)&a.nsteps, (void *)&a.parity0, (void *)&a.bar, (void *)&a.budget};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(a.grid);
    cfg.blockDim = dim3(a.block);
    cfg.stream = a.stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, batch_kernel_ptr(storage, a.block), args);
}

// ------------------------------------------------------ two-buffer pull ----

template <int S, bool MOM>
__global__ void __launch_bounds__(256, 3) k_pull(const SEF<S> *__restrict__ fs, const SEG<S> *__restrict__ gs,
                                              SEF<S> *__restrict__ fd, SEG<S> *__restrict__ gd, Geom G,
                                              Phys P, float *__restrict__ mom) {
    const uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= G.n) return;
    int x, y, z;
    node_xyz(G, n, x, y, z);
    float fl[19], gl[7];
    read_natural<S>(fs, gs, G, P, LAYOUT_PULL, n, x, y, z, fl, gl);
    float g0[7];
#pragma unroll
    for (int i = 0; i < 7; ++i) g0[i] = gl[i];
    const Macro m = collide(P, fl, gl);
    const int64_t s = G.stride;
#pragma unroll
    for (int i = 0; i < 19; ++i) Store<FS(S)>::st(fd + i * s + n, fl[i]);
    const uint32_t rb = SRG(S) ? rnd_node(n, P.t) : 0u;
#pragma unroll
#pragma unroll
    for (int i = 0; i < 7; ++i) Store<GS(S)>::sts(gd + i * s + n, gl[i], rnd_pop(rb, i));
    if (MOM) write_sample(mom, s, n, m, neighbours(G, x, y, z), g0);
}

// ------------------------------------------------- layout conversions ----

// Natural host-order staging (float, [26][n], no padding) -> device layout.
// For LAYOUT_PULL, B[j][m] must make the pull reproduce the natural state:
// B[j][m] = f_j(m + e_j), or, where m + e_j is behind a wall, the value that
// bounces back into f_jbar(m).
template <int S>
__global__ void k_load(const float *__restrict__ st, SEF<S> *__restrict__ f, SEG<S> *__restrict__ g,
                       Geom G, Phys P, int layout) {
    const uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= G.n) return;
    const int64_t s = G.stride, N = G.n;
    if (layout == LAYOUT_NATURAL) {
        for (int i = 0; i < 19; ++i) Store<FS(S)>::st(f + i * s + n, st[i * N + n]);
        for (int i = 0; i < 7; ++i) Store<GS(S)>::st(g + i * s + n, st[(19 + i) * N + n]);
        return;
    }
    int x, y, z;
    node_xyz(G, n, x, y, z);
    const Nbr b = neighbours(G, x, y, z);
#pragma unroll
    for (int j = 0; j < 19; ++j) {
        float v;
        if (!dst_wall(b, ex19(j), ey19(j), ez19(j)))
            v = st[j * N + (int64_t)n + dst_off(b, ex19(j), ey19(j), ez19(j))];
        else
            v = st[opp19(j) * N + n];
        Store<FS(S)>::st(f + j * s + n, v);
    }
#pragma unroll
    for (int j = 0; j < 7; ++j) {
        float v;
        if (!dst_wall(b, ex7(j), ey7(j), ez7(j))) {
            v = st[(19 + j) * N + (int64_t)n + dst_off(b, ex7(j), ey7(j), ez7(j))];
        } else {
            const int fc = face_of(ex7(j), ey7(j), ez7(j));
            const float gin = st[(19 + opp7(j)) * N + n];
            v = ((P.dir_mask >> fc) & 1) ? P.abbT[fc] - gin : gin;
        }
        Store<GS(S)>::st(g + j * s + n, v);
    }
}

// Device layout -> natural staging (float [26][n]).
template <int S>
__global__ void k_store(float *__restrict__ st, const SEF<S> *__restrict__ f, const SEG<S> *__restrict__ g,
                        Geom G, Phys P, int layout) {
    const uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= G.n) return;
    int x, y, z;
    node_xyz(G, n, x, y, z);
    float fl[19], gl[7];
    read_natural<S>(f, g, G, P, layout, n, x, y, z, fl, gl);
    const int64_t N = G.n;
#pragma unroll
    for (int i = 0; i < 19; ++i) st[i * N + n] = fl[i];
#pragma unroll
    for (int i = 0; i < 7; ++i) st[(19 + i) * N + n] = gl[i];
}

// Pre-collision populations of listed nodes -> out[k][26].
template <int S>
__global__ void k_gather(float *__restrict__ out, const int64_t *__restrict__ nodes, int64_t count,
                         const SEF<S> *__restrict__ f, const SEG<S> *__restrict__ g, Geom G, Phys P,
                         int layout) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= count) return;
    const uint32_t n = static_cast<uint32_t>(nodes[k]);
    int x, y, z;
    node_xyz(G, n, x, y, z);
    float fl[19], gl[7];
    read_natural<S>(f, g, G, P, layout, n, x, y, z, fl, gl);
#pragma unroll
    for (int i = 0; i < 19; ++i) out[k * 26 + i] = fl[i];
#pragma unroll
    for (int i = 0; i < 7; ++i) out[k * 26 + 19 + i] = gl[i];
}

// Diagnostic sample of the state -> mom[11][stride] (see write_sample).
template <int S>
__global__ void k_moments(float *__restrict__ mom, const SEF<S> *__restrict__ f,
                          const SEG<S> *__restrict__ g, Geom G, Phys P, int layout) {
    const uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= G.n) return;
    int x, y, z;
    node_xyz(G, n, x, y, z);
    float fl[19], gl[7];
    read_natural<S>(f, g, G, P, layout, n, x, y, z, fl, gl);
    write_sample(mom, G.stride, n, macro(P, fl, gl), neighbours(G, x, y, z), gl);
}

// Equilibrium deviations from fields (float [5][n]: rho - rho0, u, v, w, T)
// into natural staging [26][n]:
//   f_i^eq - w_i rho0 = w_i [drho + rho (3 e.u + 9/2 (e.u)^2 - 3/2 |u|^2)]
//   g_i^eq = w_i^T T [1 + 7/(6 + a_T) 3 e.u]            (Sec. 2.2, 2.3)
__global__ void k_equilibrium(float *__restrict__ st, const float *__restrict__ fields, uint32_t N,
                              Phys P) {
    const uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const float dr = fields[n], u = fields[N + n], v = fields[2 * (int64_t)N + n];
    const float w = fields[3 * (int64_t)N + n], T = fields[4 * (int64_t)N + n];
    const float rho = 1.f + dr, uu = u * u + v * v + w * w;
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const float eu = ex19(i) * u + ey19(i) * v + ez19(i) * w;
        st[i * (int64_t)N + n] = w19(i) * (dr + rho * (3.f * eu + 4.5f * eu * eu - 1.5f * uu));
    }
    const float w0 = (1.f - P.a_T) / 7.f, w1 = (6.f + P.a_T) / 42.f, c = 21.f / (6.f + P.a_T);
#pragma unroll
    for (int i = 0; i < 7; ++i) {
        const float eu = ex7(i) * u + ey7(i) * v + ez7(i) * w;
        st[(19 + i) * (int64_t)N + n] = (i == 0 ? w0 : w1) * T * (1.f + c * eu);
    }
}

// Equilibrium state of host-order FP64 fields (rho, u3[3][n], T, as given to
// lbm_set_fields and copied to the device), stored straight into the natural
// device layout (the AA pattern before an even step): the deviations of
// k_equilibrium, rounded to the storage format once.
template <int S>
__global__ void k_fields_natural(const double *__restrict__ rho, const double *__restrict__ u3,
                                 const double *__restrict__ Tf, SEF<S> *__restrict__ f, SEG<S> *__restrict__ g,
                                 uint32_t N, int64_t s, Phys P) {
    const uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const float dr = (float)(rho[n] - 1.0), u = (float)u3[n], v = (float)u3[(int64_t)N + n];
    const float w = (float)u3[2 * (int64_t)N + n], T = (float)Tf[n];
    const float r = 1.f + dr, uu = u * u + v * v + w * w;
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const float eu = ex19(i) * u + ey19(i) * v + ez19(i) * w;
        Store<FS(S)>::st(f + i * s + n, w19(i) * (dr + r * (3.f * eu + 4.5f * eu * eu - 1.5f * uu)));
    }
    const float w0 = (1.f - P.a_T) / 7.f, w1 = (6.f + P.a_T) / 42.f, c = 21.f / (6.f + P.a_T);
#pragma unroll
    for (int i = 0; i < 7; ++i) {
        const float eu = ex7(i) * u + ey7(i) * v + ez7(i) * w;
        Store<GS(S)>::st(g + i * s + n, (i == 0 ? w0 : w1) * T * (1.f + c * eu));
    }
}

// ---------------------------------------------------------- launchers ----

static inline unsigned blocks_for(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

template <int S>
static cudaError_t step_t(const StepArgs &a) {
    const unsigned nb = blocks_for(a.G.n, a.block);
    auto f = static_cast<SEF<S> *>(a.f);
    auto g = static_cast<SEG<S> *>(a.g);
    if (a.scheme == 0 && a.wide) {
        if (a.parity == 0) {
            const unsigned nb2 = blocks_for((a.G.n + 1) / 2, a.block);
            if (a.mom) k_aa_even2<S, true><<<nb2, a.block, 0, a.stream>>>(f, g, a.G, a.P, a.mom);
            else k_aa_even2<S, false><<<nb2, a.block, 0, a.stream>>>(f, g, a.G, a.P, nullptr);
        } else {
            // the row kernel covers the x faces of its rows; the listed y/z-face nodes remain
            const unsigned nwarps = a.G.cpp * (unsigned)(a.G.nz - 2);
            const unsigned ni = blocks_for(nwarps, a.block / 32), nf = blocks_for(a.nface_yz, kFacePer<S> * a.block);
            if (a.mom) {
                if (ni) k_aa_odd_rows<S, true><<<ni, a.block, 0, a.stream>>>(f, g, a.G, a.P, a.mom);
                if (nf) k_aa_odd_face<S, true><<<nf, a.block, 0, a.stream>>>(f, g, a.G, a.P, a.mom, a.face, a.nface_yz);
            } else {
                if (ni) k_aa_odd_rows<S, false><<<ni, a.block, 0, a.stream>>>(f, g, a.G, a.P, nullptr);
                if (nf)
                    k_aa_odd_face<S, false><<<nf, a.block, 0, a.stream>>>(f, g, a.G, a.P, nullptr, a.face, a.nface_yz);
            }
        }
    } else if (a.scheme == 0) {
        if (a.parity == 0) {
            if (a.mom) k_aa_even<S, true><<<nb, a.block, 0, a.stream>>>(f, g, a.G, a.P, a.mom);
            else k_aa_even<S, false><<<nb, a.block, 0, a.stream>>>(f, g, a.G, a.P, nullptr);
        } else {
            const unsigned ni = blocks_for(a.G.ni, a.block), nf = blocks_for(a.nface, kFacePer<S> * a.block);
            if (a.mom) {
                if (ni) k_aa_odd_interior<S, true><<<ni, a.block, 0, a.stream>>>(f, g, a.G, a.P, a.mom);
                if (nf) k_aa_odd_face<S, true><<<nf, a.block, 0, a.stream>>>(f, g, a.G, a.P, a.mom, a.face, a.nface);
            } else {
                if (ni) k_aa_odd_interior<S, false><<<ni, a.block, 0, a.stream>>>(f, g, a.G, a.P, nullptr);
                if (nf)
                    k_aa_odd_face<S, false><<<nf, a.block, 0, a.stream>>>(f, g, a.G, a.P, nullptr, a.face, a.nface);
            }
        }
    } else {
        auto f2 = static_cast<SEF<S> *>(a.f2);
        auto g2 = static_cast<SEG<S> *>(a.g2);
        if (a.mom) k_pull<S, true><<<nb, a.block, 0, a.stream>>>(f, g, f2, g2, a.G, a.P, a.mom);
        else k_pull<S, false><<<nb, a.block, 0, a.stream>>>(f, g, f2, g2, a.G, a.P, nullptr);
    }
    return cudaGetLastError();
}

// The face kernel after the staged odd kernel: a programmatic dependent
// launch (see pdl_launch), waiting for that kernel before it reads.
template <int S>
__global__ void __launch_bounds__(256, kFacePer<S> == 1 ? 3 : 2) k_aa_odd_face_pdl(SEF<S> *__restrict__ f,
                                                                                  SEG<S> *__restrict__ g, Geom G,
                                                                                  Phys P,
                                                                                  const uint32_t *__restrict__ list,
                                                                                  uint32_t count) {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
    k_aa_odd_face_tile<S, false>(f, g, G, P, nullptr, list, count, blockIdx.x, threadIdx.x, blockDim.x);
}

template <int S> static cudaError_t face_t(const StepArgs &a, uint32_t count) {
    if (!count) return cudaGetLastError();
    SEF<S> *f = static_cast<SEF<S> *>(a.f);
    SEG<S> *g = static_cast<SEG<S> *>(a.g);
    Geom G = a.G;
    Phys P = a.P;
    const uint32_t *list = a.face;
    void *args[] = {&f, &g, &G, &P, &list, &count};
    return pdl_launch(reinterpret_cast<const void *>(&k_aa_odd_face_pdl<S>), blocks_for(count, kFacePer<S> * 256),
                      256, 0, a.stream, args);
}

int face_nodes_per_thread(int storage) { return storage == ST_F32 ? kFacePer<ST_F32> : kFacePer<ST_F16>; }

cudaError_t launch_face(const StepArgs &a, uint32_t count) {
    switch (a.storage) {
    case ST_F32: return face_t<ST_F32>(a, count);
    case ST_F16: return face_t<ST_F16>(a, count);
    case ST_F16M: return face_t<ST_F16M>(a, count);
    default: return face_t<ST_BF16>(a, count);
    }
}

cudaError_t launch_step(const StepArgs &a) {
    switch (a.storage) {
    case ST_F32: return step_t<ST_F32>(a);
    case ST_F16: return step_t<ST_F16>(a);
    case ST_F16M: return step_t<ST_F16M>(a);
    default: return step_t<ST_BF16>(a);
    }
}

template <int S>
static cudaError_t convert_t(int op, float *st, void *f, void *g, const Geom &G, const Phys &P,
                             int layout, cudaStream_t stream) {
    const unsigned nb = blocks_for(G.n, 256);
    if (op == 0) k_load<S><<<nb, 256, 0, stream>>>(st, (SEF<S> *)f, (SEG<S> *)g, G, P, layout);
    else if (op == 1) k_store<S><<<nb, 256, 0, stream>>>(st, (const SEF<S> *)f, (const SEG<S> *)g, G, P, layout);
    else k_moments<S><<<nb, 256, 0, stream>>>(st, (const SEF<S> *)f, (const SEG<S> *)g, G, P, layout);
    return cudaGetLastError();
}

cudaError_t launch_convert(int storage, int op, float *st, void *f, void *g, const Geom &G,
                           const Phys &P, int layout, cudaStream_t stream) {
    switch (storage) {
    case ST_F32: return convert_t<ST_F32>(op, st, f, g, G, P, layout, stream);
    case ST_F16: return convert_t<ST_F16>(op, st, f, g, G, P, layout, stream);
    case ST_F16M: return convert_t<ST_F16M>(op, st, f, g, G, P, layout, stream);
    default: return convert_t<ST_BF16>(op, st, f, g, G, P, layout, stream);
    }
}

template <int S>
static cudaError_t gather_t(float *out, const int64_t *nodes, int64_t count, const void *f, const void *g,
                            const Geom &G, const Phys &P, int layout, cudaStream_t stream) {
    k_gather<S><<<blocks_for(count, 128), 128, 0, stream>>>(out, nodes, count, (const SEF<S> *)f,
                                                             (const SEG<S> *)g, G, P, layout);
    return cudaGetLastError();
}

cudaError_t launch_gather(int storage, float *out, const int64_t *nodes, int64_t count, const void *f,
                          const void *g, const Geom &G, const Phys &P, int layout, cudaStream_t stream) {
    switch (storage) {
    case ST_F32: return gather_t<ST_F32>(out, nodes, count, f, g, G, P, layout, stream);
    case ST_F16: return gather_t<ST_F16>(out, nodes, count, f, g, G, P, layout, stream);
    case ST_F16M: return gather_t<ST_F16M>(out, nodes, count, f, g, G, P, layout, stream);
    default: return gather_t<ST_BF16>(out, nodes, count, f, g, G, P, layout, stream);
    }
}

template <int S>
static cudaError_t fields_t(const double *rho, const double *u3, const double *T, void *f, void *g, const Geom &G,
                            const Phys &P, cudaStream_t stream) {
    k_fields_natural<S><<<blocks_for(G.n, 256), 256, 0, stream>>>(rho, u3, T, (SEF<S> *)f, (SEG<S> *)g, G.n,
                                                                   G.stride, P);
    return cudaGetLastError();
}

cudaError_t launch_fields_natural(int storage, const double *rho, const double *u3, const double *T, void *f,
                                  void *g, const Geom &G, const Phys &P, cudaStream_t stream) {
    switch (storage) {
    case ST_F32: return fields_t<ST_F32>(rho, u3, T, f, g, G, P, stream);
    case ST_F16: return fields_t<ST_F16>(rho, u3, T, f, g, G, P, stream);
    case ST_F16M: return fields_t<ST_F16M>(rho, u3, T, f, g, G, P, stream);
    default: return fields_t<ST_BF16>(rho, u3, T, f, g, G, P, stream);
    }
}

cudaError_t launch_equilibrium(float *st, const float *fields, uint32_t n, const Phys &P,
                               cudaStream_t stream) {
    k_equilibrium<<<blocks_for(n, 256), 256, 0, stream>>>(st, fields, n, P);
    return cudaGetLastError();
}

} // namespace lbm
