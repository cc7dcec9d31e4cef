// Diagnostic reductions: the global quantities of Secs. 3 and 4 from one
// sample of node moments.
//
// Per node (FP32 from the FP32 moment arrays), summed per thread in FP32
// (runs of at most 32 nodes, then the runs' sums), across a warp in
// double-float (two FP32 words), then across warps and blocks in FP64:
//   [0] 1                       [1] (rho - rho0)^2        [2] |u|^2
//   [3] w^2                     [4] w T                   [5] 1/2 sum_ij (d_i u_j + d_j u_i)^2
//   [6] |grad T|^2              [7] (div u)^2             [8+f] -dT/dn at Dirichlet face f
//   [14] T                      [15] rho                  [16] max |u|
//   [17] nodes with a non-finite moment                   [18+f] 2 g_in - (6 + a_T)/21 T_w
// Derivatives: central differences inside (periodic axes wrap); next to a
// wall with a known value (velocity 0 at every no-slip wall, T_w at a
// Dirichlet wall) the one-sided second-order stencil through the wall point,
// d/ds = -4/3 phi_w + phi_0 + phi_1/3; next to an adiabatic wall the
// zero-gradient stencil (phi_1 - phi_0)/2.  Wall flux at a Dirichlet face:
// dT/dn = (-8 T_w + 9 T_0 - T_1)/3 with n pointing into the fluid.
//
// Reduction: warp shuffles, then shared memory, one FP64 partial per block
// and quantity; a one-block kernel sums the partials in a fixed order.  The
// wall terms go through shared FP64 atomics, so their last bits depend on
// the order the warps add them.
#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace lbm {

constexpr int kDiagThreads = 256;

__device__ __forceinline__ float deriv(const float *__restrict__ phi, uint32_t n, const Nbr &b, int a,
                                       bool lo_val, float lo_w, bool hi_val, float hi_w) {
    const float p0 = phi[n];
    if (!b.wm[a] && !b.wp[a]) return 0.5f * (phi[(int64_t)n + b.op[a]] - phi[(int64_t)n + b.om[a]]);
    if (b.wm[a] && b.wp[a]) return 0.f;
    if (b.wm[a]) {
        const float p1 = phi[(int64_t)n + b.op[a]];
        return lo_val ? (-4.f / 3.f) * lo_w + p0 + p1 * (1.f / 3.f) : 0.5f * (p1 - p0);
    }
    const float p1 = phi[(int64_t)n + b.om[a]];
    return hi_val ? (4.f / 3.f) * hi_w - p0 - p1 * (1.f / 3.f) : 0.5f * (p0 - p1);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// Double-float value hi + lo (two FP32 words, about 48 significant bits).
// FP64 arithmetic is slow on this GPU, so the warp stage of the reductions
// adds these pairs with FP32 instructions (Knuth's error-free TwoSum, then a
// renormalisation) and only the few per-warp results become FP64.
struct DF {
    float hi, lo;
};
__device__ __forceinline__ DF df_add(DF a, DF b) {
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    const float err = (a.hi - (s - bb)) + (b.hi - bb);
    const float lo = a.lo + b.lo + err;
    const float hi = s + lo;
    return {hi, lo - (hi - s)};
}
__device__ __forceinline__ DF df_warp_sum(DF a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const DF b = {__shfl_down_sync(0xffffffffu, a.hi, o), __shfl_down_sync(0xffffffffu, a.lo, o)};
        a = df_add(a, b);
    }
    return a;
}
__device__ __forceinline__ double df_value(DF a) { return (double)a.hi + (double)a.lo; }

struct WallT {
    float Tw[6];
};

// Compensated (Kahan) FP32 running sum: FP64 arithmetic is slow on this
// GPU, and a thread sums only a few dozen nodes, so FP32 with compensation is
// as accurate as the FP64 block and grid reductions that follow.
struct KSum {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x) {
        const float y = x - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
    __device__ __forceinline__ DF df() const { return {s, -c}; }
};

// Derivative along an axis from the values at the node and its two
// neighbours, with the stencils of the file header (wm / wp: a wall behind
// the -1 / +1 neighbour; vlo / vhi: a known wall value wlo / whi there), as
// coefficients d = m phi_-1 + o phi_0 + p phi_+1 + k chosen per node with
// selects rather than branches (the lanes of a warp next to a wall take
// different stencils).
struct Coef {
    float m, o, p, k;
};
__device__ __forceinline__ Coef coef(bool wm, bool wp, bool vlo, float wlo, bool vhi, float whi) {
    Coef c = {-0.5f, 0.f, 0.5f, 0.f};
    if (wm && wp) c = {0.f, 0.f, 0.f, 0.f};
    else if (wm) c = vlo ? Coef{0.f, 1.f, 1.f / 3.f, (-4.f / 3.f) * wlo} : Coef{0.f, -0.5f, 0.5f, 0.f};
    else if (wp) c = vhi ? Coef{-1.f / 3.f, -1.f, 0.f, (4.f / 3.f) * whi} : Coef{-0.5f, 0.5f, 0.f, 0.f};
    return c;
}
__device__ __forceinline__ float apply(const Coef &c, float pm, float p0, float pp) {
    return fmaf(c.m, pm, fmaf(c.o, p0, fmaf(c.p, pp, c.k)));
}

// Diagnostic sums of one sample.  The lattice is cut into columns of
// kDiagTX x kDiagTY nodes in x, y and segments of kDiagSeg planes in z; a
// block takes one such brick at a time (bricks strided over the grid, so any
// grid size works) and each thread marches up its column.  A thread keeps
// its column's u, v, w, T of the planes z - 1, z and z + 1 in registers
// (the z derivatives) and loads plane z + 2 one plane ahead; the x and y
// neighbours come straight from memory, where the block's other lanes and
// warps have just read them (L1 hits), so every field value leaves HBM about
// once without shared-memory staging or a block barrier per plane.  A warp
// whose nodes have no wall or wrap next to them takes plain central
// differences.  Each thread sums its column of a brick (at most kDiagSeg
// nodes) in FP32 and adds the column sums into FP32 totals (a few dozen at
// most); the wall terms of a column (x and y faces) or of a plane (z faces)
// go into shared FP64 sums.
constexpr int kDiagTX = 32, kDiagTY = kDiagThreads / kDiagTX, kDiagSeg = 32;

__global__ void __launch_bounds__(kDiagThreads, 3) k_diag(const float *__restrict__ mom, Geom G, Phys P,
                                                       WallT W, double *__restrict__ partial) {
    __shared__ double sh[kDiagThreads / 32][kNDiag];
    __shared__ double wall[12]; // slots 8..13 and 18..23
    __shared__ float tot[9][kDiagThreads]; // slots 1..7, 14, 15: sums of each thread's column sums
    const int tx = threadIdx.x % kDiagTX, ty = threadIdx.x / kDiagTX;
    if (threadIdx.x < 12) wall[threadIdx.x] = 0.0;
#pragma unroll
    for (int k = 0; k < 9; ++k) tot[k][threadIdx.x] = 0.f;
    float umax2 = 0.f;
    uint32_t count = 0, bad = 0;
    const int64_t s = G.stride;
    const float *F[4] = {mom + s, mom + 2 * s, mom + 3 * s, mom + 4 * s};
    const float *dr = mom;
    const int nx = G.nx, ny = G.ny, nz = G.nz;
    const bool perx = G.periodic & 1, pery = (G.periodic >> 1) & 1, perz = (G.periodic >> 2) & 1;
    const int bx = (nx + kDiagTX - 1) / kDiagTX, by = (ny + kDiagTY - 1) / kDiagTY, bz = (nz + kDiagSeg - 1) / kDiagSeg;
    const int nbricks = bx * by * bz;
    const bool dir[6] = {(P.dir_mask & 1) != 0, (P.dir_mask & 2) != 0, (P.dir_mask & 4) != 0,
                         (P.dir_mask & 8) != 0, (P.dir_mask & 16) != 0, (P.dir_mask & 32) != 0};
    const bool anydir = P.dir_mask != 0;
    __syncthreads();
    for (int br = blockIdx.x; br < nbricks; br += gridDim.x) {
        const int ib = br % bx, jb = (br / bx) % by, kb = br / (bx * by);
        const int x = ib * kDiagTX + tx, y = jb * kDiagTY + ty;
        const bool col = x < nx && y < ny;
        const int z0 = kb * kDiagSeg, z1 = min(nz, z0 + kDiagSeg);
        const int64_t c = col ? (int64_t)x + (int64_t)nx * y : 0; // column offset
        const bool xlo = x == 0 && !perx, xhi = x == nx - 1 && !perx;
        const bool ylo = y == 0 && !pery, yhi = y == ny - 1 && !pery;
        // in-plane offsets of the x and y neighbours (wrapped on periodic
        // axes; 0, the node itself, behind a wall, where no value is used)
        const int oxm = x > 0 ? -1 : perx ? nx - 1 : 0, oxp = x < nx - 1 ? 1 : perx ? -(nx - 1) : 0;
        const int oym = y > 0 ? -nx : pery ? nx * (ny - 1) : 0, oyp = y < ny - 1 ? nx : pery ? -nx * (ny - 1) : 0;
        const bool wrapxy = (perx && (x == 0 || x == nx - 1)) || (pery && (y == 0 || y == ny - 1));
        // the Dirichlet x and y faces this column lies on (-1: none; nx, ny >= 3,
        // so at most one of each) and its wall terms summed over the brick
        const int fxc = !col || perx ? -1 : (x == 0 && dir[0]) ? 0 : (x == nx - 1 && dir[1]) ? 1 : -1;
        const int fyc = !col || pery ? -1 : (y == 0 && dir[2]) ? 2 : (y == ny - 1 && dir[3]) ? 3 : -1;
        float wxa = 0.f, wxb = 0.f, wya = 0.f, wyb = 0.f;
        // u, v, w, T (and rho - rho0) of the column in plane zz, wrapped on a
        // periodic z; planes outside the lattice are never read
        auto plane_of = [&](int zz) -> int64_t {
            const int za = zz < 0 ? (perz ? zz + nz : -1) : zz >= nz ? (perz ? zz - nz : -1) : zz;
            return za < 0 ? -1 : (int64_t)G.nxy * za;
        };
        float pm[4] = {}, p0[4] = {}, pp[4] = {}, nn[4] = {};
        float d0 = 0.f, dn = 0.f;
        if (col) {
            const int64_t am = plane_of(z0 - 1), a0 = plane_of(z0), ap = plane_of(z0 + 1);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (am >= 0) pm[q] = F[q][am + c];
                p0[q] = F[q][a0 + c];
                if (ap >= 0) pp[q] = F[q][ap + c];
            }
            d0 = dr[a0 + c];
        }
        float bs[9]; // plain FP32 sums over the brick's column (at most kDiagSeg nodes)
#pragma unroll
        for (int k = 0; k < 9; ++k) bs[k] = 0.f;
        for (int z = z0; z < z1; ++z) {
            const int64_t pz = (int64_t)G.nxy * z;
            // plane z + 2 for the next plane's z + 1
            if (col && z + 1 < z1) {
                const int64_t an = plane_of(z + 2);
                if (an >= 0) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) nn[q] = F[q][an + c];
                }
                dn = dr[pz + G.nxy + c]; // z + 1 < z1 <= nz
            }
            const bool zlo = z == 0 && !perz, zhi = z == nz - 1 && !perz;
            // a warp with no wall and no wrap among its nodes takes central
            // differences throughout
            const bool plain = !col || !(xlo || xhi || ylo || yhi || zlo || zhi || wrapxy);
            const bool fast = __all_sync(0xffffffffu, plain);
            if (col) {
                const int64_t n = pz + c;
                float du[3][3], gT[3];
                float tx1 = 0.f, ty1 = 0.f; // T of the next node inward from an x / y face
                // x then y: the neighbours of one axis at a time, so that only
                // eight of them are live
#pragma unroll
                for (int a = 0; a < 2; ++a) {
                    const int om = a == 0 ? oxm : oym, op = a == 0 ? oxp : oyp;
                    const bool wlo = a == 0 ? xlo : ylo, whi = a == 0 ? xhi : yhi;
                    float vm[4], vp[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float *fq = F[q] + n; // 32-bit neighbour offsets from the node's own address
                        vm[q] = fq[om];
                        vp[q] = fq[op];
                    }
                    if (fast) {
#pragma unroll
                        for (int q = 0; q < 3; ++q) du[a][q] = 0.5f * (vp[q] - vm[q]);
                        gT[a] = 0.5f * (vp[3] - vm[3]);
                    } else {
                        const Coef cv = coef(wlo, whi, true, 0.f, true, 0.f);
                        const Coef ct = coef(wlo, whi, dir[2 * a], W.Tw[2 * a], dir[2 * a + 1], W.Tw[2 * a + 1]);
#pragma unroll
                        for (int q = 0; q < 3; ++q) du[a][q] = apply(cv, vm[q], p0[q], vp[q]);
                        gT[a] = apply(ct, vm[3], p0[3], vp[3]);
                    }
                    const float t1 = (a == 0 ? fxc == 0 : fyc == 2) ? vp[3] : vm[3];
                    if (a == 0) tx1 = t1;
                    else ty1 = t1;
                }
                if (fast) {
#pragma unroll
                    for (int q = 0; q < 3; ++q) du[2][q] = 0.5f * (pp[q] - pm[q]);
                    gT[2] = 0.5f * (pp[3] - pm[3]);
                } else {
                    const Coef cv = coef(zlo, zhi, true, 0.f, true, 0.f);
                    const Coef ct = coef(zlo, zhi, dir[4], W.Tw[4], dir[5], W.Tw[5]);
#pragma unroll
                    for (int q = 0; q < 3; ++q) du[2][q] = apply(cv, pm[q], p0[q], pp[q]);
                    gT[2] = apply(ct, pm[3], p0[3], pp[3]);
                }
                const float d = d0, u = p0[0], vv = p0[1], w = p0[2], t = p0[3];
                const float uu = u * u + vv * vv + w * w;
                float eps = 0.f;
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        const float sij = du[i][j] + du[j][i];
                        eps += 0.5f * sij * sij;
                    }
                const float dv = du[0][0] + du[1][1] + du[2][2];
                count += 1;
                bs[0] += d * d;
                bs[1] += uu;
                bs[2] += w * w;
                bs[3] += w * t;
                bs[4] += eps;
                bs[5] += gT[0] * gT[0] + gT[1] * gT[1] + gT[2] * gT[2];
                bs[6] += dv * dv;
                bs[7] += t;
                bs[8] += d; // sum rho = nodes + sum (rho - rho0)
                umax2 = fmaxf(umax2, uu);
                if (!(fabsf(uu) + fabsf(t) + fabsf(d) < INFINITY)) bad += 1; // a NaN or infinite moment
                // Dirichlet faces: wall gradient -dT/dn (from the node and the
                // next one inward) and anti-bounce-back link flux
                // 2 g_in - (6 + a_T)/21 T_w; x and y faces summed per column
                // (constant-index selects keep the wall tables out of local memory)
                if (anydir && !fast) {
                    if (fxc >= 0) {
                        const bool lo = fxc == 0;
                        wxa += (8.f * (lo ? W.Tw[0] : W.Tw[1]) - 9.f * p0[3] + tx1) * (1.f / 3.f);
                        wxb += 2.f * mom[(5 + fxc) * s + n] - (lo ? P.abbT[0] : P.abbT[1]);
                    }
                    if (fyc >= 0) {
                        const bool lo = fyc == 2;
                        wya += (8.f * (lo ? W.Tw[2] : W.Tw[3]) - 9.f * p0[3] + ty1) * (1.f / 3.f);
                        wyb += 2.f * mom[(5 + fyc) * s + n] - (lo ? P.abbT[2] : P.abbT[3]);
                    }
                }
            }
            // z faces (a whole plane): per warp, then shared FP64 sums
            const int fzc = perz || !anydir ? -1 : (zlo && dir[4]) ? 4 : (zhi && dir[5]) ? 5 : -1; // uniform
            if (fzc >= 0) {
                const bool lo = fzc == 4;
                float ta = 0.f, tb = 0.f;
                if (col) {
                    ta = (8.f * (lo ? W.Tw[4] : W.Tw[5]) - 9.f * p0[3] + (lo ? pp[3] : pm[3])) * (1.f / 3.f);
                    tb = 2.f * mom[(5 + fzc) * s + pz + c] - (lo ? P.abbT[4] : P.abbT[5]);
                }
                const DF da = df_warp_sum({ta, 0.f}), db = df_warp_sum({tb, 0.f});
                if ((threadIdx.x & 31) == 0) {
                    atomicAdd(&wall[fzc], df_value(da));
                    atomicAdd(&wall[6 + fzc], df_value(db));
                }
            }
            // march: planes z, z + 1, z + 2 become z - 1, z, z + 1
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                pm[q] = p0[q];
                p0[q] = pp[q];
                pp[q] = nn[q];
            }
            d0 = dn;
        }
        // the column's sums into the thread's totals; its x and y wall terms
        // into the shared FP64 sums
#pragma unroll
        for (int k = 0; k < 9; ++k) tot[k][threadIdx.x] += bs[k];
        if (fxc >= 0) {
            atomicAdd(&wall[fxc], (double)wxa);
            atomicAdd(&wall[6 + fxc], (double)wxb);
        }
        if (fyc >= 0) {
            atomicAdd(&wall[fyc], (double)wya);
            atomicAdd(&wall[6 + fyc], (double)wyb);
        }
    }
    const float vmax = sqrtf(umax2);
    // block reduction: double-float warp sums, FP64 across the warps
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    constexpr int slot[10] = {0, 1, 2, 3, 4, 5, 6, 7, 14, 15};
#pragma unroll
    for (int k = 1; k < 10; ++k) {
        const DF r = df_warp_sum({tot[k - 1][threadIdx.x], 0.f});
        if (lane == 0) sh[wid][slot[k]] = df_value(r);
    }
    count = __reduce_add_sync(0xffffffffu, count);
    bad = __reduce_add_sync(0xffffffffu, bad);
    float vm = vmax;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) vm = fmaxf(vm, __shfl_down_sync(0xffffffffu, vm, o));
    if (lane == 0) {
        sh[wid][0] = (double)count;
        sh[wid][15] += (double)count; // sum rho = nodes + sum (rho - rho0)
        sh[wid][16] = (double)vm;
        sh[wid][17] = (double)bad;
    }
    __syncthreads();
    if (wid == 0) {
        double v[kNDiag];
        constexpr int nw = kDiagThreads / 32;
#pragma unroll
        for (int k = 0; k < kNDiag; ++k) {
            if ((k >= 8 && k <= 13) || k >= 18) continue; // wall slots: below
            double r = lane < nw ? sh[lane][k] : 0.0;
#pragma unroll
            for (int o = nw / 2; o > 0; o >>= 1) {
                const double t = __shfl_down_sync(0xffffffffu, r, o);
                r = k == 16 ? fmax(r, t) : r + t;
            }
            v[k] = r;
        }
        if (lane == 0) {
#pragma unroll
            for (int fc = 0; fc < 6; ++fc) {
                v[8 + fc] = wall[fc];
                v[18 + fc] = wall[6 + fc];
            }
#pragma unroll
            for (int k = 0; k < kNDiag; ++k) partial[(int64_t)blockIdx.x * kNDiag + k] = v[k];
        }
    }
}

// Sum of the blocks' partials: warp w takes the quantities w, w + 8, ...,
// its lanes the blocks in turn (a fixed order, so the sums are reproducible),
// then a shuffle tree.  FP64 arithmetic is slow on this GPU, so the
// quantities run side by side in different warps rather than one after
// another in one.
__global__ void __launch_bounds__(kDiagThreads) k_diag_finish(const double *__restrict__ partial,
                                                              int nblocks, double *__restrict__ raw,
                                                              double *__restrict__ acc) {
    constexpr int nw = kDiagThreads / 32, per = (kNDiag + nw - 1) / nw;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double v[per];
#pragma unroll
    for (int i = 0; i < per; ++i) v[i] = 0.0;
    for (int b = lane; b < nblocks; b += 32) {
#pragma unroll
        for (int i = 0; i < per; ++i) {
            const int k = wid + nw * i;
            if (k >= kNDiag) continue;
            const double p = partial[(int64_t)b * kNDiag + k];
            v[i] = k == 16 ? fmax(v[i], p) : v[i] + p;
        }
    }
#pragma unroll
    for (int i = 0; i < per; ++i) {
        const int k = wid + nw * i;
        const double r = k == 16 ? warp_max(v[i]) : warp_sum(v[i]);
        if (lane == 0 && k < kNDiag) {
            raw[k] = r;
            acc[k] = k == 16 ? fmax(acc[k], r) : acc[k] + r;
        }
    }
    if (threadIdx.x == 0) acc[kNDiag] += 1.0;
}

// Local dissipation rates (Sec. 4): eps_u = nu/2 sum_ij (d_i u_j + d_j u_i)^2
// and eps_T = kappa |grad T|^2 of node n, with the stencils of k_diag.
__device__ __forceinline__ void local_eps(const float *__restrict__ mom, int64_t s, const Geom &G,
                                          const Phys &P, const WallT &W, uint32_t n, float nu,
                                          float ka, float &eu, float &et) {
    int x, y, z;
    node_xyz(G, n, x, y, z);
    const Nbr b = neighbours(G, x, y, z);
    const float *phi[3] = {mom + s, mom + 2 * s, mom + 3 * s};
    const float *T = mom + 4 * s;
    float du[3][3]; // du[i][j] = d u_j / d x_i
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) du[i][j] = deriv(phi[j], n, b, i, true, 0.f, true, 0.f);
    float e = 0.f, gg = 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const float sij = du[i][j] + du[j][i];
            e += 0.5f * sij * sij;
        }
        const float gi = deriv(T, n, b, i, (P.dir_mask >> (2 * i)) & 1, W.Tw[2 * i],
                               (P.dir_mask >> (2 * i + 1)) & 1, W.Tw[2 * i + 1]);
        gg += gi * gi;
    }
    eu = nu * e;
    et = ka * gg;
}

// Pass 1 of the dissipation PDFs: sums of eps_u^2 and eps_T^2 over the nodes
// (compensated FP32 per thread, double-float across the warp, FP64 across
// warps), one atomic add per block and quantity into sums[0..1].
__global__ void __launch_bounds__(kDiagThreads) k_eps_sq(const float *__restrict__ mom, Geom G, Phys P,
                                                         WallT W, float nu, float ka,
                                                         double *__restrict__ sums) {
    __shared__ double sh[kDiagThreads / 32][2];
    KSum a0, a1;
    for (uint32_t n = blockIdx.x * blockDim.x + threadIdx.x; n < G.n; n += gridDim.x * blockDim.x) {
        float eu, et;
        local_eps(mom, G.stride, G, P, W, n, nu, ka, eu, et);
        a0.add(eu * eu);
        a1.add(et * et);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const DF r0 = df_warp_sum(a0.df()), r1 = df_warp_sum(a1.df());
    if (lane == 0) {
        sh[wid][0] = df_value(r0);
        sh[wid][1] = df_value(r1);
    }
    __syncthreads();
    if (wid == 0) {
        const double b0 = warp_sum(lane < nw ? sh[lane][0] : 0.0);
        const double b1 = warp_sum(lane < nw ? sh[lane][1] : 0.0);
        if (lane == 0) {
            atomicAdd(&sums[0], b0);
            atomicAdd(&sums[1], b1);
        }
    }
}

// Pass 2: counts of X = eps / eps_rms in nbins equal bins on [0, xmax),
// eps_u into counts[0..nbins), eps_T into counts[nbins..2 nbins).  Bins are
// counted per block in shared memory (2 nbins unsigned ints) and added to the
// global counters once per block.  A value outside [0, xmax), NaN included,
// is not counted.
__global__ void __launch_bounds__(kDiagThreads) k_eps_hist(const float *__restrict__ mom, Geom G, Phys P,
                                                           WallT W, float nu, float ka, double scale_u,
                                                           double scale_t, int nbins,
                                                           unsigned long long *__restrict__ counts) {
    extern __shared__ unsigned int hs[];
    for (int i = threadIdx.x; i < 2 * nbins; i += blockDim.x) hs[i] = 0u;
    __syncthreads();
    const double top = (double)nbins;
    for (uint32_t n = blockIdx.x * blockDim.x + threadIdx.x; n < G.n; n += gridDim.x * blockDim.x) {
        float eu, et;
        local_eps(mom, G.stride, G, P, W, n, nu, ka, eu, et);
        const double xu = (double)eu * scale_u, xt = (double)et * scale_t;
        if (xu >= 0.0 && xu < top) atomicAdd(&hs[(int)xu], 1u);
        if (xt >= 0.0 && xt < top) atomicAdd(&hs[nbins + (int)xt], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 2 * nbins; i += blockDim.x)
        if (hs[i]) atomicAdd(&counts[i], (unsigned long long)hs[i]);
}

// Blocks for a grid-stride kernel over the nodes: as many as the device
// holds at once at the kernel's own occupancy (its registers and shared
// memory), at most max_per_sm per SM (each block flushes its partial sums
// with global atomics once), no more than the nodes need.  (k_diag's brick
// grid, which these kernels used before, is sized for k_diag's registers: at
// 257^3 it left the PDF passes 16% slower.)
static int resident_blocks(const void *fn, size_t smem, uint32_t n, int max_per_sm = 4) {
    int dev = 0, nsm = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess || nsm < 1)
        nsm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, kDiagThreads, smem) != cudaSuccess || per < 1)
        per = 1;
    cudaGetLastError();
    per = per < max_per_sm ? per : max_per_sm;
    const int64_t need = ((int64_t)n + kDiagThreads - 1) / kDiagThreads;
    const int64_t cap = (int64_t)per * nsm;
    return (int)(need < cap ? need : cap);
}

cudaError_t launch_eps_sq(const float *mom, const Geom &G, const Phys &P, const float *wallT, float nu,
                          float ka, double *sums, cudaStream_t stream) {
    WallT W;
    for (int k = 0; k < 6; ++k) W.Tw[k] = wallT[k];
    k_eps_sq<<<resident_blocks(reinterpret_cast<const void *>(&k_eps_sq), 0, G.n), kDiagThreads, 0, stream>>>(
        mom, G, P, W, nu, ka, sums);
    return cudaGetLastError();
}

cudaError_t launch_eps_hist(const float *mom, const Geom &G, const Phys &P, const float *wallT, float nu,
                            float ka, double scale_u, double scale_t, int nbins, unsigned long long *counts,
                            cudaStream_t stream) {
    WallT W;
    for (int k = 0; k < 6; ++k) W.Tw[k] = wallT[k];
    const size_t shmem = (size_t)2 * nbins * sizeof(unsigned int);
    k_eps_hist<<<resident_blocks(reinterpret_cast<const void *>(&k_eps_hist), shmem, G.n), kDiagThreads, shmem,
                 stream>>>(mom, G, P, W, nu, ka, scale_u, scale_t, nbins, counts);
    return cudaGetLastError();
}

// Plane-averaged Nusselt number along axis a (Sec. 3, Nu(y) of Fig. 4):
// adds, for every node, u_a T H/kappa - H dT/dx_a (stencils of k_diag) into
// prof[j] of its plane j.  Sums per block in shared memory (FP64; SHARED =
// false adds straight into global memory for axes too long for it), a warp
// whose nodes share one plane adds its shuffled sum once.
template <bool SHARED>
__global__ void __launch_bounds__(kDiagThreads) k_nu_profile(const float *__restrict__ mom, Geom G, Phys P, WallT W,
                                                             int axis, float hk, float H,
                                                             double *__restrict__ prof) {
    extern __shared__ double acc[];
    const int na = axis == 0 ? G.nx : axis == 1 ? G.ny : G.nz;
    double *out = SHARED ? acc : prof;
    if (SHARED) {
        for (int i = threadIdx.x; i < na; i += blockDim.x) acc[i] = 0.0;
        __syncthreads();
    }
    const int64_t s = G.stride;
    const float *ua = mom + (1 + axis) * s, *T = mom + 4 * s;
    const int lane = threadIdx.x & 31;
    const uint32_t step = gridDim.x * blockDim.x;
    for (uint32_t base = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < G.n; base += step) {
        const uint32_t n = base + (uint32_t)lane;
        const bool valid = n < G.n;
        double v = 0.0;
        int j = -1;
        if (valid) {
            int x, y, z;
            node_xyz(G, n, x, y, z);
            const Nbr b = neighbours(G, x, y, z);
            const float dT = deriv(T, n, b, axis, (P.dir_mask >> (2 * axis)) & 1, W.Tw[2 * axis],
                                   (P.dir_mask >> (2 * axis + 1)) & 1, W.Tw[2 * axis + 1]);
            v = (double)(ua[n] * T[n] * hk - H * dT);
            j = axis == 0 ? x : axis == 1 ? y : z;
        }
        const int j0 = __shfl_sync(0xffffffffu, j, 0);
        if (__all_sync(0xffffffffu, j == j0 || !valid)) {
            v = warp_sum(v);
            if (lane == 0) atomicAdd(&out[j0], v);
        } else if (valid) {
            atomicAdd(&out[j], v);
        }
    }
    if (SHARED) {
        __syncthreads();
        for (int i = threadIdx.x; i < na; i += blockDim.x)
            if (acc[i] != 0.0) atomicAdd(&prof[i], acc[i]);
    }
}

// Mid-line wall Nusselt numbers (Sec. 3, Nu_mean of Table 2): block f takes
// face f and writes mid[f] = the mean of -H dT/dn at the wall (one-sided
// stencil of k_diag) over the nodes next to the face on the line along z
// (along x for the z faces) through the middle of the third axis: one node
// line for an odd node count, the two bracketing lines for an even one.
// 0 for faces that are not Dirichlet walls.
__global__ void __launch_bounds__(kDiagThreads) k_nu_midline(const float *__restrict__ mom, Geom G, Phys P,
                                                             WallT W, float H, double *__restrict__ mid) {
    __shared__ double sh[kDiagThreads / 32];
    const int fc = blockIdx.x;
    if (!((P.dir_mask >> fc) & 1)) {
        if (threadIdx.x == 0) mid[fc] = 0.0;
        return;
    }
    const int nn[3] = {G.nx, G.ny, G.nz};
    const int b = fc / 2, hi = fc % 2, l = b == 2 ? 0 : 2, m = 3 - b - l;
    const int m0 = (nn[m] - 1) / 2, lines = nn[m] % 2 ? 1 : 2;
    const int count = lines * nn[l];
    const float *T = mom + 4 * G.stride;
    double acc = 0.0;
    for (int k = threadIdx.x; k < count; k += blockDim.x) {
        int c0[3], c1[3];
        c0[b] = hi ? nn[b] - 1 : 0;
        c1[b] = hi ? nn[b] - 2 : 1;
        c0[l] = c1[l] = k % nn[l];
        c0[m] = c1[m] = m0 + k / nn[l];
        const float t0 = T[(uint32_t)c0[0] + (uint32_t)G.nx * ((uint32_t)c0[1] + (uint32_t)G.ny * (uint32_t)c0[2])];
        const float t1 = T[(uint32_t)c1[0] + (uint32_t)G.nx * ((uint32_t)c1[1] + (uint32_t)G.ny * (uint32_t)c1[2])];
        acc += (double)(-H * (-8.f * W.Tw[fc] + 9.f * t0 - t1) * (1.f / 3.f));
    }
    acc = warp_sum(acc);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) sh[wid] = acc;
    __syncthreads();
    if (wid == 0) {
        acc = warp_sum(lane < nw ? sh[lane] : 0.0);
        if (lane == 0) mid[fc] = acc / count;
    }
}

constexpr int kProfileSharedMax = 6144; // axis length held in shared memory (48 KB)

cudaError_t launch_nu_profile(const float *mom, const Geom &G, const Phys &P, const float *wallT, int axis,
                              float H, float kappa, double *prof, double *mid, cudaStream_t stream) {
    WallT W;
    for (int k = 0; k < 6; ++k) W.Tw[k] = wallT[k];
    const int na = axis == 0 ? G.nx : axis == 1 ? G.ny : G.nz;
    if (na <= kProfileSharedMax)
        k_nu_profile<true><<<resident_blocks(reinterpret_cast<const void *>(&k_nu_profile<true>),
                                             (size_t)na * sizeof(double), G.n),
                             kDiagThreads, (size_t)na * sizeof(double), stream>>>(mom, G, P, W, axis, H / kappa, H,
                                                                                  prof);
    else
        k_nu_profile<false><<<resident_blocks(reinterpret_cast<const void *>(&k_nu_profile<false>), 0, G.n),
                              kDiagThreads, 0, stream>>>(mom, G, P, W, axis, H / kappa, H, prof);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_nu_midline<<<6, kDiagThreads, 0, stream>>>(mom, G, P, W, H, mid);
    return cudaGetLastError();
}

int diag_blocks(const Geom &G) {
    // one brick per block at most, and no more blocks than the device holds
    // at once (k_diag's occupancy times the SM count), so that the bricks are
    // shared out in a single wave and each block reduces its sums once
    const int64_t need = (int64_t)((G.nx + kDiagTX - 1) / kDiagTX) * ((G.ny + kDiagTY - 1) / kDiagTY) *
                         ((G.nz + kDiagSeg - 1) / kDiagSeg);
    int dev = 0, nsm = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess || nsm < 1)
        nsm = 152;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_diag, kDiagThreads, 0) != cudaSuccess || per < 1)
        per = 3;
    cudaGetLastError();
    const int64_t cap = (int64_t)per * nsm;
    return (int)(need < cap ? need : cap);
}

cudaError_t launch_diag(const float *mom, const Geom &G, const Phys &P, const float *wallT,
                        double *partial, int nblocks, double *raw, double *acc, cudaStream_t stream) {
    WallT W;
    for (int k = 0; k < 6; ++k) W.Tw[k] = wallT[k];
    k_diag<<<nblocks, kDiagThreads, 0, stream>>>(mom, G, P, W, partial);
    k_diag_finish<<<1, kDiagThreads, 0, stream>>>(partial, nblocks, raw, acc);
    return cudaGetLastError();
}

} // namespace lbm
