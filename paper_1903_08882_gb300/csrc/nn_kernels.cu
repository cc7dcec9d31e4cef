// Kernels of the warm-start network (declared in include/lbm_nn.h): 3x3x3
// convolutions on the tensor cores with FP32 accumulation (forward, data
// gradient, weight gradient), ReLU backward, ceil average pooling, nearest
// upsampling, trilinear interpolation, MSE loss, Adam.
//
// The convolutions are implicit GEMMs on mma.sync (m16n8k16, BF16 x BF16 ->
// FP32): forward and data gradient (a forward convolution of the output
// gradient with the flipped, transposed weights) take voxels as GEMM rows and
// output channels as columns; the weight gradient takes output channels by
// input channels per tap, reducing over voxels.  The weights are BF16; an
// FP32 activation or gradient operand enters as the sum of two BF16 terms
// (see split_bf16), so the products carry FP32-level accuracy.
#include <cuda_bf16.h>

#include <string>

#include "../../include/lbm_nn.h"
#include "lbm_internal.h"

namespace {

constexpr int kT = 256; // threads per block


struct Vox {
    int z, y, x;
};
__device__ __forceinline__ Vox vox(int64_t v, int H, int W) {
    Vox r;
    r.x = (int)(v % W);
    const int64_t q = v / W;
    r.y = (int)(q % H);
    r.z = (int)(q / H);
    return r;
}

// Bit t set when tap t = (dz+1)*9 + (dy+1)*3 + (dx+1) of voxel p lies inside.
__device__ __forceinline__ uint32_t tap_mask(const Vox &p, int D, int H, int W) {
    uint32_t m = 0;
#pragma unroll
    for (int t = 0; t < 27; ++t) {
        const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
        const bool in = p.z + dz >= 0 && p.z + dz < D && p.y + dy >= 0 && p.y + dy < H && p.x + dx >= 0 &&
                        p.x + dx < W;
        m |= (in ? 1u : 0u) << t;
    }
    return m;
}

// ------------------------------------------------ tensor-core convolutions ----
//
// Implicit GEMM on the tensor cores: mma.sync.m16n8k16 with BF16 operands and
// FP32 accumulation.  An FP32 operand x is split into hi = bf16(x) and
// lo = bf16(x - hi) (both nearest even; x - hi is exact in FP32) and enters
// as two products, after the BF16 splitting of Henry, Tang and Heinecke
// (ARITH 2019): |x - hi - lo| <= 2^-18 |x|.  Weights are BF16 already, so the
// forward and data-gradient products take two MMAs; the weight gradient,
// with both operands FP32, takes hi*hi + hi*lo + lo*hi (the dropped lo*lo is
// below 2^-16 of the product).  Sums stay FP32.
//
// Fragment layout of m16n8k16 (g = lane / 4, q = lane % 4; each 32-bit
// register holds two BF16, the lower index in the low half):
//   A (16 x 16, row-major): {a0,a1} = (g, 2q..2q+1), {a2,a3} = (g+8, 2q..2q+1),
//                           {a4,a5} = (g, 2q+8..2q+9), {a6,a7} = (g+8, 2q+8..2q+9)
//   B (16 x 8, k by n):     {b0,b1} = (2q..2q+1, g), {b2,b3} = (2q+8..2q+9, g)
//   C (16 x 8, FP32):       c0, c1 = (g, 2q..2q+1), c2, c3 = (g+8, 2q..2q+1)

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}
// Two FP32 values as BF16 pairs hi (nearest) and lo (nearest of the rest).
struct Split2 {
    uint32_t hi, lo;
};
__device__ __forceinline__ Split2 split_bf16(float a, float b) {
    Split2 r;
    r.hi = pack_bf16(a, b);
    const float ah = __uint_as_float(r.hi << 16), bh = __uint_as_float(r.hi & 0xFFFF0000u);
    r.lo = pack_bf16(a - ah, b - bh);
    return r;
}
__device__ __forceinline__ uint32_t pack_u16(uint16_t lo, uint16_t hi) {
    return (uint32_t)lo | ((uint32_t)hi << 16);
}
__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
                 "{%8, %9}, {%0, %1, %2, %3};"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

constexpr int kTcWarps = 8;            // warps per block
constexpr int kTcM = 16 * kTcWarps;    // output voxels per block (16 per warp)
constexpr int kTcN = 32;               // output channels per block (4 n-tiles of 8)
constexpr int kTcChunk = 16;           // input channels staged at a time (one k-step)
constexpr int kTcPitch = kTcN + 8;     // words per staged weight row: the fragment reads hit 32 banks

// y[co][v] = bias + sum_{ci, tap} w[co][ci][tap] x[ci][v + tap]: rows of the
// GEMM are voxels, columns output channels, the reduction runs over taps and
// 16-channel chunks.  The block stages the weights of its kTcN output
// channels for all 27 taps of one chunk in shared memory, as channel pairs
// ([tap][ci / 2][co] words, the lower channel in the low half), so a B
// fragment register is one 32-bit read; each warp builds its A fragments
// straight from global memory (the taps of neighbouring voxels overlap in
// L1) and reuses them for its four n-tiles.
__global__ void __launch_bounds__(32 * kTcWarps) k_conv_fwd_tc(const float *__restrict__ x, int Cin, int D, int H,
                                                               int W, const uint16_t *__restrict__ w,
                                                               const float *__restrict__ bias, int Cout,
                                                               float *__restrict__ y, int relu, int accumulate) {
    __shared__ uint32_t wt[27][kTcChunk / 2][kTcPitch];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, q = lane & 3;
    const int64_t V = (int64_t)D * H * W, HW = (int64_t)H * W;
    const int co0 = blockIdx.y * kTcN;
    const int64_t v0 = (int64_t)blockIdx.x * kTcM + warp * 16;
    // the warp's two voxel rows g and g + 8: positions and in-range taps
    const int64_t va = v0 + g, vb = v0 + g + 8;
    const bool la = va < V, lb = vb < V;
    const uint32_t ma = la ? tap_mask(vox(va, H, W), D, H, W) : 0u;
    const uint32_t mb = lb ? tap_mask(vox(vb, H, W), D, H, W) : 0u;
    float acc[4][4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[j][i] = 0.f;
    for (int ci_base = 0; ci_base < Cin; ci_base += kTcChunk) {
        const int cspan = Cin - ci_base < kTcChunk ? Cin - ci_base : kTcChunk;
        __syncthreads(); // the previous chunk's weights are no longer read
        for (int k = threadIdx.x; k < 27 * (kTcChunk / 2) * kTcN; k += blockDim.x) {
            const int c = k % kTcN, r = k / kTcN, pr = r % (kTcChunk / 2), t = r / (kTcChunk / 2);
            const int ci = 2 * pr, co = co0 + c;
            uint16_t lo = 0, hi = 0;
            if (co < Cout) {
                const uint16_t *wc = w + ((int64_t)co * Cin + ci_base + ci) * 27 + t;
                if (ci < cspan) lo = wc[0];
                if (ci + 1 < cspan) hi = wc[27];
            }
            wt[t][pr][c] = pack_u16(lo, hi);
        }
        __syncthreads();
        // the channels this lane's A fragment holds: 2q, 2q+1, 2q+8, 2q+9
        const float *xc[4];
        bool cok[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int c = 2 * q + (u & 1) + (u >> 1) * 8;
            cok[u] = c < cspan;
            xc[u] = x + (int64_t)(ci_base + (cok[u] ? c : 0)) * V;
        }
#pragma unroll 3
        for (int t = 0; t < 27; ++t) {
            const int dz = t / 9 - 1, dyy = (t / 3) % 3 - 1, dx = t % 3 - 1;
            const int64_t off = dz * HW + dyy * W + dx;
            const bool ta = (ma >> t) & 1u, tb = (mb >> t) & 1u;
            float xa[4], xb[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                xa[u] = (cok[u] && ta) ? xc[u][va + off] : 0.f;
                xb[u] = (cok[u] && tb) ? xc[u][vb + off] : 0.f;
            }
            const Split2 s0 = split_bf16(xa[0], xa[1]), s1 = split_bf16(xb[0], xb[1]),
                         s2 = split_bf16(xa[2], xa[3]), s3 = split_bf16(xb[2], xb[3]);
            const uint32_t ah[4] = {s0.hi, s1.hi, s2.hi, s3.hi}, al[4] = {s0.lo, s1.lo, s2.lo, s3.lo};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint32_t b0 = wt[t][q][j * 8 + g], b1 = wt[t][q + 4][j * 8 + g];
                mma_bf16(acc[j], al, b0, b1);
                mma_bf16(acc[j], ah, b0, b1);
            }
        }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int co = co0 + j * 8 + 2 * q + (i & 1);
            const int64_t v = (i < 2) ? va : vb;
            if (co >= Cout || v >= V) continue;
            float r = acc[j][i] + (bias ? bias[co] : 0.f);
            float *out = y + (int64_t)co * V + v;
            if (accumulate) r += *out;
            if (relu) r = fmaxf(r, 0.f);
            *out = r;
        }
}

// dw[co][ci][tap] += sum_v dy[co][v] x[ci][v + tap]: for each tap a GEMM of
// output channels (rows, one 16-channel m-tile per block) by input channels
// (columns, all of them: up to kTcNtMax n-tiles of 8) over voxels.  Block
// (row batch, tap, m-tile): its warps take the rows (z, y) of the batch in
// turn and walk each along x in steps of 16 voxels, so the tap's range
// check is per row plus the x edges; the A fragment (dy) of a step serves
// every n-tile.  The warps' sums meet in shared memory, then go to dw with
// one atomic add per element.  NT >= ceil(Cin / 8) sizes the accumulators.
constexpr int kTcNtMax = 16; // n-tiles per warp: 16 x 8 = 128 input channels
template <int NT>
__global__ void __launch_bounds__(32 * kTcWarps) k_conv_bww_tc(const float *__restrict__ x, int Cin, int D, int H,
                                                               int W, const float *__restrict__ dy, int Cout,
                                                               float *__restrict__ dw, int rows_per_block) {
    __shared__ float red[16][8 * NT];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, q = lane & 3;
    const int t = blockIdx.y, co0 = blockIdx.z * 16;
    const int dz = t / 9 - 1, dyy = (t / 3) % 3 - 1, dx = t % 3 - 1;
    const int64_t V = (int64_t)D * H * W, HW = (int64_t)H * W;
    const int nrows = D * H, nt = (Cin + 7) / 8;
    for (int k = threadIdx.x; k < 16 * 8 * NT; k += blockDim.x) (&red[0][0])[k] = 0.f;
    float acc[NT][4];
#pragma unroll
    for (int j = 0; j < NT; ++j)
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[j][i] = 0.f;
    const int r0 = blockIdx.x * rows_per_block, r1 = min(nrows, r0 + rows_per_block);
    const bool coa = co0 + g < Cout, cob = co0 + g + 8 < Cout;
    const float *dya = dy + (int64_t)(coa ? co0 + g : 0) * V, *dyb = dy + (int64_t)(cob ? co0 + g + 8 : 0) * V;
    for (int r = r0 + warp; r < r1; r += kTcWarps) {
        const int z = r / H, yy = r - z * H;
        const bool row_ok = z + dz >= 0 && z + dz < D && yy + dyy >= 0 && yy + dyy < H;
        const int64_t rb = (int64_t)z * HW + (int64_t)yy * W; // row start
        const int64_t sb = rb + dz * HW + dyy * W + dx;       // shifted row start
        for (int x0 = 0; x0 < W; x0 += 16) {
            // A fragment: dy[co][row, x0 + k] for k = 2q, 2q+1, 2q+8, 2q+9
            float fa[4], fb[4];
            bool kin[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int xk = x0 + 2 * q + (u & 1) + (u >> 1) * 8;
                const bool in = xk < W;
                fa[u] = (in && coa) ? dya[rb + xk] : 0.f;
                fb[u] = (in && cob) ? dyb[rb + xk] : 0.f;
                kin[u] = row_ok && in && xk + dx >= 0 && xk + dx < W;
            }
            const Split2 s0 = split_bf16(fa[0], fa[1]), s1 = split_bf16(fb[0], fb[1]),
                         s2 = split_bf16(fa[2], fa[3]), s3 = split_bf16(fb[2], fb[3]);
            const uint32_t ah[4] = {s0.hi, s1.hi, s2.hi, s3.hi}, al[4] = {s0.lo, s1.lo, s2.lo, s3.lo};
            // B fragment of n-tile j: x[ci][row + tap, x0 + k] for ci = 8 j + g
            const float *xs = x + sb + x0 + 2 * q;
#pragma unroll
            for (int j = 0; j < NT; ++j) {
                if (j >= nt) break; // warp-uniform
                const int ci = j * 8 + g;
                const float *xc = xs + (int64_t)(ci < Cin ? ci : 0) * V;
                float xv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) xv[u] = (ci < Cin && kin[u]) ? xc[(u & 1) + (u >> 1) * 8] : 0.f;
                const Split2 b = split_bf16(xv[0], xv[1]), c = split_bf16(xv[2], xv[3]);
                mma_bf16(acc[j], al, b.hi, c.hi);
                mma_bf16(acc[j], ah, b.lo, c.lo);
                mma_bf16(acc[j], ah, b.hi, c.hi);
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < NT; ++j) {
        if (j >= nt) break;
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (acc[j][i] != 0.f) atomicAdd(&red[g + (i < 2 ? 0 : 8)][j * 8 + 2 * q + (i & 1)], acc[j][i]);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < 16 * Cin; k += blockDim.x) {
        const int m = k / Cin, ci = k - m * Cin, co = co0 + m;
        const float v = red[m][ci];
        if (co < Cout && v != 0.f) atomicAdd(&dw[((int64_t)co * Cin + ci) * 27 + t], v);
    }
}

// db[co] += sum_v dy[co][v] (FP32 gradients, not rounded).
__global__ void __launch_bounds__(kT) k_bias_grad(const float *__restrict__ dy, int64_t V, float *__restrict__ db,
                                                 int64_t chunk) {
    __shared__ float red[kT / 32];
    const int co = blockIdx.y;
    const int64_t v0 = (int64_t)blockIdx.x * chunk, v1 = v0 + chunk < V ? v0 + chunk : V;
    float s = 0.f;
    for (int64_t v = v0 + threadIdx.x; v < v1; v += kT) s += dy[(int64_t)co * V + v];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float b = 0.f;
        for (int k = 0; k < kT / 32; ++k) b += red[k];
        atomicAdd(&db[co], b);
    }
}

// w_t[ci][co][26 - t] = w[co][ci][t]: the data gradient is a forward
// convolution of dy with these weights.
__global__ void k_flip_transpose(const uint16_t *__restrict__ w, uint16_t *__restrict__ wt, int Cout, int Cin) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (int64_t)Cout * Cin * 27) return;
    const int t = (int)(k % 27);
    const int64_t r = k / 27;
    const int ci = (int)(r % Cin), co = (int)(r / Cin);
    wt[((int64_t)ci * Cout + co) * 27 + (26 - t)] = w[k];
}


__global__ void k_relu_bwd(float *__restrict__ dy, const float *__restrict__ y, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (!(y[i] > 0.f)) dy[i] = 0.f;
}

__global__ void k_pool_fwd(const float *__restrict__ x, int C, int D, int H, int W, float *__restrict__ y) {
    const int d = (D + 1) / 2, h = (H + 1) / 2, w = (W + 1) / 2;
    const int64_t n = (int64_t)C * d * h * w;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int X = (int)(i % w), Y = (int)((i / w) % h), Z = (int)((i / ((int64_t)w * h)) % d);
        const int c = (int)(i / ((int64_t)w * h * d));
        float s = 0.f;
        int cnt = 0;
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b)
                for (int e = 0; e < 2; ++e) {
                    const int z = 2 * Z + a, yy = 2 * Y + b, xx = 2 * X + e;
                    if (z < D && yy < H && xx < W) {
                        s += x[(((int64_t)c * D + z) * H + yy) * W + xx];
                        ++cnt;
                    }
                }
        y[i] = s / (float)cnt;
    }
}

__global__ void k_pool_bwd(const float *__restrict__ dy, int C, int D, int H, int W, float *__restrict__ dx,
                           int accumulate) {
    const int d = (D + 1) / 2, h = (H + 1) / 2, w = (W + 1) / 2;
    const int64_t n = (int64_t)C * D * H * W;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int xx = (int)(i % W), yy = (int)((i / W) % H), z = (int)((i / ((int64_t)W * H)) % D);
        const int c = (int)(i / ((int64_t)W * H * D));
        const int Z = z / 2, Y = yy / 2, X = xx / 2;
        const int cz = (2 * Z + 1 < D) ? 2 : 1, cy = (2 * Y + 1 < H) ? 2 : 1, cx = (2 * X + 1 < W) ? 2 : 1;
        const float g = dy[(((int64_t)c * d + Z) * h + Y) * w + X] / (float)(cz * cy * cx);
        dx[i] = accumulate ? dx[i] + g : g;
    }
}

__global__ void k_up_fwd(const float *__restrict__ x, int C, int D, int H, int W, float *__restrict__ y) {
    const int d = (D + 1) / 2, h = (H + 1) / 2, w = (W + 1) / 2;
    const int64_t n = (int64_t)C * D * H * W;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int xx = (int)(i % W), yy = (int)((i / W) % H), z = (int)((i / ((int64_t)W * H)) % D);
        const int c = (int)(i / ((int64_t)W * H * D));
        y[i] = x[(((int64_t)c * d + z / 2) * h + yy / 2) * w + xx / 2];
    }
}

__global__ void k_up_bwd(const float *__restrict__ dy, int C, int D, int H, int W, float *__restrict__ dx) {
    const int d = (D + 1) / 2, h = (H + 1) / 2, w = (W + 1) / 2;
    const int64_t n = (int64_t)C * d * h * w;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int X = (int)(i % w), Y = (int)((i / w) % h), Z = (int)((i / ((int64_t)w * h)) % d);
        const int c = (int)(i / ((int64_t)w * h * d));
        float s = 0.f;
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b)
                for (int e = 0; e < 2; ++e) {
                    const int z = 2 * Z + a, yy = 2 * Y + b, xx = 2 * X + e;
                    if (z < D && yy < H && xx < W) s += dy[(((int64_t)c * D + z) * H + yy) * W + xx];
                }
        dx[i] = s;
    }
}

// Source index pair and weight of output node j (coordinate in FP64: in FP32
// the rounding of (j + 1/2) n_in / n_out near n_in = 64 reaches 4e-6).
__device__ __forceinline__ void lin_idx(int j, int n_out, int n_in, int &i0, int &i1, float &f) {
    const double s = ((double)j + 0.5) * (double)n_in / (double)n_out - 0.5;
    if (s <= 0.0) {
        i0 = i1 = 0;
        f = 0.f;
        return;
    }
    i0 = (int)s;
    if (i0 >= n_in - 1) {
        i0 = i1 = n_in - 1;
        f = 0.f;
        return;
    }
    i1 = i0 + 1;
    f = (float)(s - (double)i0);
}

__global__ void k_trilinear(const float *__restrict__ x, int C, int d, int h, int w, float *__restrict__ y, int D,
                            int H, int W) {
    const int64_t n = (int64_t)C * D * H * W;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int xx = (int)(i % W), yy = (int)((i / W) % H), z = (int)((i / ((int64_t)W * H)) % D);
        const int c = (int)(i / ((int64_t)W * H * D));
        int z0, z1, y0, y1, x0, x1;
        float fz, fy, fx;
        lin_idx(z, D, d, z0, z1, fz);
        lin_idx(yy, H, h, y0, y1, fy);
        lin_idx(xx, W, w, x0, x1, fx);
        const float *xc = x + (int64_t)c * d * h * w;
        auto at = [&](int a, int b, int e) { return xc[((int64_t)a * h + b) * w + e]; };
        const float c00 = at(z0, y0, x0) * (1 - fx) + at(z0, y0, x1) * fx;
        const float c01 = at(z0, y1, x0) * (1 - fx) + at(z0, y1, x1) * fx;
        const float c10 = at(z1, y0, x0) * (1 - fx) + at(z1, y0, x1) * fx;
        const float c11 = at(z1, y1, x0) * (1 - fx) + at(z1, y1, x1) * fx;
        const float c0 = c00 * (1 - fy) + c01 * fy, c1 = c10 * (1 - fy) + c11 * fy;
        y[i] = c0 * (1 - fz) + c1 * fz;
    }
}

__global__ void k_axpy(float a, const float *__restrict__ x, float *__restrict__ y, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] += a * x[i];
}

__global__ void __launch_bounds__(kT) k_mse(const float *__restrict__ p, const float *__restrict__ t, int64_t n,
                                            double *__restrict__ loss, float *__restrict__ grad) {
    __shared__ double red[kT / 32];
    double s = 0.0;
    const float sc = 2.f / (float)n;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float e = p[i] - t[i];
        s += (double)e * e;
        if (grad) grad[i] = sc * e;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int k = 0; k < kT / 32; ++k) b += red[k];
        atomicAdd(loss, b / (double)n);
    }
}

__global__ void k_adam(float *__restrict__ w, uint16_t *__restrict__ wb, float *__restrict__ g,
                       float *__restrict__ m, float *__restrict__ v, int64_t n, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        w[i] = wi;
        if (wb) {
            const __nv_bfloat16 h = __float2bfloat16_rn(wi);
            wb[i] = *reinterpret_cast<const uint16_t *>(&h);
        }
        g[i] = 0.f;
    }
}

__global__ void k_to_bf16(const float *__restrict__ x, uint16_t *__restrict__ y, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const __nv_bfloat16 h = __float2bfloat16_rn(x[i]);
        y[i] = *reinterpret_cast<const uint16_t *>(&h);
    }
}

unsigned grid_1d(int64_t n) {
    const int64_t b = (n + kT - 1) / kT;
    return (unsigned)(b < 152 * 32 ? (b > 0 ? b : 1) : 152 * 32);
}

lbm_status done(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return LBM_OK;
    lbm::set_global_error(std::string(what) + ": " + cudaGetErrorString(e));
    return LBM_ERR_CUDA;
}

lbm_status bad(const char *what) {
    lbm::set_global_error(std::string(what) + ": invalid argument");
    return LBM_ERR_PARAM;
}

cudaStream_t S(void *s) { return static_cast<cudaStream_t>(s); }

} // namespace

extern "C" {

lbm_status lbm_nn_conv3d_forward(const float *x, int Cin, int D, int H, int W, const uint16_t *w, const float *bias,
                                 int Cout, float *y, int relu, void *stream) {
    if (!x || !w || !y || Cin < 1 || Cout < 1 || D < 1 || H < 1 || W < 1) return bad("lbm_nn_conv3d_forward");
    const int64_t V = (int64_t)D * H * W;
    dim3 grid((unsigned)((V + kTcM - 1) / kTcM), (unsigned)((Cout + kTcN - 1) / kTcN));
    k_conv_fwd_tc<<<grid, 32 * kTcWarps, 0, S(stream)>>>(x, Cin, D, H, W, w, bias, Cout, y, relu, 0);
    return done(cudaGetLastError(), "lbm_nn_conv3d_forward");
}

lbm_status lbm_nn_conv3d_backward_data(const float *dy, int Cout, int D, int H, int W, const uint16_t *w,
                                       uint16_t *wt, int Cin, float *dx, int accumulate, void *stream) {
    if (!dy || !w || !wt || !dx || Cin < 1 || Cout < 1 || D < 1 || H < 1 || W < 1)
        return bad("lbm_nn_conv3d_backward_data");
    const int64_t nw = (int64_t)Cout * Cin * 27;
    k_flip_transpose<<<(unsigned)((nw + kT - 1) / kT), kT, 0, S(stream)>>>(w, wt, Cout, Cin);
    const int64_t V = (int64_t)D * H * W;
    dim3 grid((unsigned)((V + kTcM - 1) / kTcM), (unsigned)((Cin + kTcN - 1) / kTcN));
    k_conv_fwd_tc<<<grid, 32 * kTcWarps, 0, S(stream)>>>(dy, Cout, D, H, W, wt, nullptr, Cin, dx, 0, accumulate);
    return done(cudaGetLastError(), "lbm_nn_conv3d_backward_data");
}

lbm_status lbm_nn_conv3d_backward_weight(const float *x, int Cin, int D, int H, int W, const float *dy, int Cout,
                                         float *dw, float *db, void *stream) {
    if (!x || !dy || !dw || Cin < 1 || Cout < 1 || D < 1 || H < 1 || W < 1 || Cin > 8 * kTcNtMax)
        return bad("lbm_nn_conv3d_backward_weight");
    const int64_t V = (int64_t)D * H * W;
    const int nrows = D * H;
    const int rpb = nrows / 64 > 32 ? nrows / 64 : 32; // about 64 row batches per tap and channel tile
    dim3 grid((unsigned)((nrows + rpb - 1) / rpb), 27u, (unsigned)((Cout + 15) / 16));
    const int nt = (Cin + 7) / 8;
    auto kern = nt <= 1 ? k_conv_bww_tc<1> : nt <= 2 ? k_conv_bww_tc<2> : nt <= 4 ? k_conv_bww_tc<4>
              : nt <= 8 ? k_conv_bww_tc<8> : k_conv_bww_tc<16>;
    kern<<<grid, 32 * kTcWarps, 0, S(stream)>>>(x, Cin, D, H, W, dy, Cout, dw, rpb);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && db) {
        const int64_t chunk = (int64_t)kT * 64;
        dim3 gb((unsigned)((V + chunk - 1) / chunk), (unsigned)Cout);
        k_bias_grad<<<gb, kT, 0, S(stream)>>>(dy, V, db, chunk);
        e = cudaGetLastError();
    }
    return done(e, "lbm_nn_conv3d_backward_weight");
}

lbm_status lbm_nn_relu_backward(float *dy, const float *y, int64_t n, void *stream) {
    if (!dy || !y || n < 1) return bad("lbm_nn_relu_backward");
    k_relu_bwd<<<grid_1d(n), kT, 0, S(stream)>>>(dy, y, n);
    return done(cudaGetLastError(), "lbm_nn_relu_backward");
}

lbm_status lbm_nn_avgpool2_forward(const float *x, int C, int D, int H, int W, float *y, void *stream) {
    if (!x || !y || C < 1 || D < 1 || H < 1 || W < 1) return bad("lbm_nn_avgpool2_forward");
    k_pool_fwd<<<grid_1d((int64_t)C * ((D + 1) / 2) * ((H + 1) / 2) * ((W + 1) / 2)), kT, 0, S(stream)>>>(x, C, D, H,
                                                                                                        W, y);
    return done(cudaGetLastError(), "lbm_nn_avgpool2_forward");
}

lbm_status lbm_nn_avgpool2_backward(const float *dy, int C, int D, int H, int W, float *dx, int accumulate,
                                    void *stream) {
    if (!dy || !dx || C < 1 || D < 1 || H < 1 || W < 1) return bad("lbm_nn_avgpool2_backward");
    k_pool_bwd<<<grid_1d((int64_t)C * D * H * W), kT, 0, S(stream)>>>(dy, C, D, H, W, dx, accumulate);
    return done(cudaGetLastError(), "lbm_nn_avgpool2_backward");
}

lbm_status lbm_nn_upsample2_forward(const float *x, int C, int D, int H, int W, float *y, void *stream) {
    if (!x || !y || C < 1 || D < 1 || H < 1 || W < 1) return bad("lbm_nn_upsample2_forward");
    k_up_fwd<<<grid_1d((int64_t)C * D * H * W), kT, 0, S(stream)>>>(x, C, D, H, W, y);
    return done(cudaGetLastError(), "lbm_nn_upsample2_forward");
}

lbm_status lbm_nn_upsample2_backward(const float *dy, int C, int D, int H, int W, float *dx, void *stream) {
    if (!dy || !dx || C < 1 || D < 1 || H < 1 || W < 1) return bad("lbm_nn_upsample2_backward");
    k_up_bwd<<<grid_1d((int64_t)C * ((D + 1) / 2) * ((H + 1) / 2) * ((W + 1) / 2)), kT, 0, S(stream)>>>(dy, C, D, H,
                                                                                                      W, dx);
    return done(cudaGetLastError(), "lbm_nn_upsample2_backward");
}

lbm_status lbm_nn_trilinear(const float *x, int C, int d, int h, int w, float *y, int D, int H, int W, void *stream) {
    if (!x || !y || C < 1 || d < 1 || h < 1 || w < 1 || D < 1 || H < 1 || W < 1) return bad("lbm_nn_trilinear");
    k_trilinear<<<grid_1d((int64_t)C * D * H * W), kT, 0, S(stream)>>>(x, C, d, h, w, y, D, H, W);
    return done(cudaGetLastError(), "lbm_nn_trilinear");
}

lbm_status lbm_nn_axpy(float a, const float *x, float *y, int64_t n, void *stream) {
    if (!x || !y || n < 1) return bad("lbm_nn_axpy");
    k_axpy<<<grid_1d(n), kT, 0, S(stream)>>>(a, x, y, n);
    return done(cudaGetLastError(), "lbm_nn_axpy");
}

lbm_status lbm_nn_mse(const float *p, const float *t, int64_t n, double *loss, float *grad, void *stream) {
    if (!p || !t || !loss || n < 1) return bad("lbm_nn_mse");
    k_mse<<<grid_1d(n), kT, 0, S(stream)>>>(p, t, n, loss, grad);
    return done(cudaGetLastError(), "lbm_nn_mse");
}

lbm_status lbm_nn_adam(float *w, uint16_t *wb, float *g, float *m, float *v, int64_t n, float lr, float beta1,
                       float beta2, float eps, int t, void *stream) {
    if (!w || !g || !m || !v || n < 1 || t < 1) return bad("lbm_nn_adam");
    const float c1 = 1.f - powf(beta1, (float)t), c2 = 1.f - powf(beta2, (float)t);
    k_adam<<<grid_1d(n), kT, 0, S(stream)>>>(w, wb, g, m, v, n, lr, beta1, beta2, eps, c1, c2);
    return done(cudaGetLastError(), "lbm_nn_adam");
}

lbm_status lbm_nn_to_bf16(const float *x, uint16_t *y, int64_t n, void *stream) {
    if (!x || !y || n < 1) return bad("lbm_nn_to_bf16");
    k_to_bf16<<<grid_1d(n), kT, 0, S(stream)>>>(x, y, n);
    return done(cudaGetLastError(), "lbm_nn_to_bf16");
}

} // extern "C"
