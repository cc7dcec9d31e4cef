// Diagnostic reductions: the global quantities of Secs. 3 and 4 from one
// sample of node moments.
//
// Per node (FP32 from the FP32 moment arrays), summed per thread in FP32 with
// Kahan compensation, then across threads and blocks in FP64:
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
// and quantity; a one-block kernel sums the partials in a fixed order, so a
// sample is bit-reproducible for a given launch shape.
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

// Sum (max for slot 16) of v[k] over the block; result valid in thread 0.
__device__ __forceinline__ void block_reduce(double (&v)[kNDiag], double (*sh)[kNDiag]) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < kNDiag; ++k) {
        const double r = k == 16 ? warp_max(v[k]) : warp_sum(v[k]);
        if (lane == 0) sh[wid][k] = r;
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < kNDiag; ++k) {
            double r = lane < nw ? sh[lane][k] : 0.0;
            v[k] = k == 16 ? warp_max(r) : warp_sum(r);
        }
    }
}

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
};

__global__ void __launch_bounds__(kDiagThreads) k_diag(const float *__restrict__ mom, Geom G, Phys P,
                                                       WallT W, double *__restrict__ partial) {
    __shared__ double sh[kDiagThreads / 32][kNDiag];
    KSum acc[kNDiag];
    float vmax = 0.f;
    uint32_t count = 0, bad = 0;
    const int64_t s = G.stride;
    const float *dr = mom, *U = mom + s, *V = mom + 2 * s, *Wv = mom + 3 * s, *T = mom + 4 * s;
    const float *phi[3] = {U, V, Wv};
    for (uint32_t n = blockIdx.x * blockDim.x + threadIdx.x; n < G.n; n += gridDim.x * blockDim.x) {
        int x, y, z;
        node_xyz(G, n, x, y, z);
        const Nbr b = neighbours(G, x, y, z);
        const float d = dr[n], u = U[n], vv = V[n], w = Wv[n], t = T[n];
        const float uu = u * u + vv * vv + w * w;
        float du[3][3]; // du[i][j] = d u_j / d x_i
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) du[i][j] = deriv(phi[j], n, b, i, true, 0.f, true, 0.f);
        float gT[3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
            gT[i] = deriv(T, n, b, i, (P.dir_mask >> (2 * i)) & 1, W.Tw[2 * i],
                          (P.dir_mask >> (2 * i + 1)) & 1, W.Tw[2 * i + 1]);
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
        acc[1].add(d * d);
        acc[2].add(uu);
        acc[3].add(w * w);
        acc[4].add(w * t);
        acc[5].add(eps);
        acc[6].add(gT[0] * gT[0] + gT[1] * gT[1] + gT[2] * gT[2]);
        acc[7].add(dv * dv);
        acc[14].add(t);
        acc[15].add(d); // sum rho = nodes + sum (rho - rho0)
        vmax = fmaxf(vmax, sqrtf(uu));
        if (!isfinite(uu) || !isfinite(t) || !isfinite(d)) bad += 1;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
#pragma unroll
            for (int side = 0; side < 2; ++side) {
                const int fc = 2 * a + side;
                const bool at = side == 0 ? b.wm[a] : b.wp[a];
                if (!at || !((P.dir_mask >> fc) & 1)) continue;
                const float t1 = T[(int64_t)n + (side == 0 ? b.op[a] : b.om[a])];
                const float dTdn = (-8.f * W.Tw[fc] + 9.f * t - t1) * (1.f / 3.f);
                acc[8 + fc].add(-dTdn);
                const float gin = mom[(5 + fc) * s + n];
                acc[18 + fc].add(2.f * gin - P.abbT[fc]);
            }
        }
    }
    double v[kNDiag];
#pragma unroll
    for (int k = 0; k < kNDiag; ++k) v[k] = acc[k].value();
    v[0] = (double)count;
    v[15] += (double)count;
    v[16] = (double)vmax;
    v[17] = (double)bad;
    block_reduce(v, sh);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < kNDiag; ++k) partial[(int64_t)blockIdx.x * kNDiag + k] = v[k];
    }
}

__global__ void __launch_bounds__(kDiagThreads) k_diag_finish(const double *__restrict__ partial,
                                                              int nblocks, double *__restrict__ raw,
                                                              double *__restrict__ acc) {
    __shared__ double sh[kDiagThreads / 32][kNDiag];
    double v[kNDiag];
#pragma unroll
    for (int k = 0; k < kNDiag; ++k) v[k] = 0.0;
    for (int bidx = threadIdx.x; bidx < nblocks; bidx += blockDim.x) {
#pragma unroll
        for (int k = 0; k < kNDiag; ++k) {
            const double p = partial[(int64_t)bidx * kNDiag + k];
            v[k] = k == 16 ? fmax(v[k], p) : v[k] + p;
        }
    }
    block_reduce(v, sh);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < kNDiag; ++k) {
            raw[k] = v[k];
            acc[k] = k == 16 ? fmax(acc[k], v[k]) : acc[k] + v[k];
        }
        acc[kNDiag] += 1.0;
    }
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
// (FP64), one atomic add per block and quantity into sums[0..1].
__global__ void __launch_bounds__(kDiagThreads) k_eps_sq(const float *__restrict__ mom, Geom G, Phys P,
                                                         WallT W, float nu, float ka,
                                                         double *__restrict__ sums) {
    __shared__ double sh[kDiagThreads / 32][2];
    double a0 = 0.0, a1 = 0.0;
    for (uint32_t n = blockIdx.x * blockDim.x + threadIdx.x; n < G.n; n += gridDim.x * blockDim.x) {
        float eu, et;
        local_eps(mom, G.stride, G, P, W, n, nu, ka, eu, et);
        a0 += (double)eu * (double)eu;
        a1 += (double)et * (double)et;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    a0 = warp_sum(a0);
    a1 = warp_sum(a1);
    if (lane == 0) {
        sh[wid][0] = a0;
        sh[wid][1] = a1;
    }
    __syncthreads();
    if (wid == 0) {
        a0 = warp_sum(lane < nw ? sh[lane][0] : 0.0);
        a1 = warp_sum(lane < nw ? sh[lane][1] : 0.0);
        if (lane == 0) {
            atomicAdd(&sums[0], a0);
            atomicAdd(&sums[1], a1);
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

cudaError_t launch_eps_sq(const float *mom, const Geom &G, const Phys &P, const float *wallT, float nu,
                          float ka, double *sums, cudaStream_t stream) {
    WallT W;
    for (int k = 0; k < 6; ++k) W.Tw[k] = wallT[k];
    k_eps_sq<<<diag_blocks(G), kDiagThreads, 0, stream>>>(mom, G, P, W, nu, ka, sums);
    return cudaGetLastError();
}

cudaError_t launch_eps_hist(const float *mom, const Geom &G, const Phys &P, const float *wallT, float nu,
                            float ka, double scale_u, double scale_t, int nbins, unsigned long long *counts,
                            cudaStream_t stream) {
    WallT W;
    for (int k = 0; k < 6; ++k) W.Tw[k] = wallT[k];
    const size_t shmem = (size_t)2 * nbins * sizeof(unsigned int);
    k_eps_hist<<<diag_blocks(G), kDiagThreads, shmem, stream>>>(mom, G, P, W, nu, ka, scale_u, scale_t, nbins,
                                                               counts);
    return cudaGetLastError();
}

int diag_blocks(const Geom &G) {
    const int64_t need = ((int64_t)G.n + kDiagThreads - 1) / kDiagThreads;
    return (int)(need < 152 * 8 ? need : 152 * 8);
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
