// Kernels of the warm-start network (declared in include/lbm_nn.h): 3x3x3
// convolutions with BF16 weights and FP32 accumulation (forward, data
// gradient, weight gradient), ReLU backward, ceil average pooling, nearest
// upsampling, trilinear interpolation, MSE loss, Adam.
//
// Convolution forward: one thread per output voxel and eight output channels;
// the block stages the weights of its eight output channels for sixteen input
// channels at a time in shared memory as [ci][tap][co] (so a thread reads the
// eight weights of one (ci, tap) as two 16-byte words); input voxels come
// through L1, where the 27-point neighbourhoods of a block's 256 consecutive
// voxels overlap.
#include <cuda_bf16.h>

#include <string>

#include "../../include/lbm_nn.h"
#include "lbm_internal.h"

namespace {

constexpr int kT = 256; // threads per block
constexpr int kCO = 8;  // output channels per thread
constexpr int kCI = 16; // input channels staged per round

__device__ __forceinline__ float bf(const uint16_t u) {
    return __uint_as_float(static_cast<uint32_t>(u) << 16);
}

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

__global__ void __launch_bounds__(kT) k_conv_fwd(const float *__restrict__ x, int Cin, int D, int H, int W,
                                                 const uint16_t *__restrict__ w, const float *__restrict__ bias,
                                                 int Cout, float *__restrict__ y, int relu, int accumulate) {
    __shared__ __align__(16) float ws[kCI][27][kCO];
    const int64_t V = (int64_t)D * H * W;
    const int64_t v = (int64_t)blockIdx.x * kT + threadIdx.x;
    const int co0 = blockIdx.y * kCO;
    const bool live = v < V;
    Vox p{0, 0, 0};
    uint32_t mask = 0;
    if (live) {
        p = vox(v, H, W);
        mask = tap_mask(p, D, H, W);
    }
    const int64_t HW = (int64_t)H * W;
    float acc[kCO];
#pragma unroll
    for (int c = 0; c < kCO; ++c) acc[c] = (bias && co0 + c < Cout) ? bias[co0 + c] : 0.f;
    for (int ci0 = 0; ci0 < Cin; ci0 += kCI) {
        __syncthreads();
        for (int k = threadIdx.x; k < kCI * 27 * kCO; k += kT) {
            const int c = k % kCO, t = (k / kCO) % 27, ci = k / (kCO * 27);
            const bool ok = co0 + c < Cout && ci0 + ci < Cin;
            ws[ci][t][c] = ok ? bf(w[((int64_t)(co0 + c) * Cin + ci0 + ci) * 27 + t]) : 0.f;
        }
        __syncthreads();
        if (!live) continue;
        const int cmax = Cin - ci0 < kCI ? Cin - ci0 : kCI;
        for (int ci = 0; ci < cmax; ++ci) {
            const float *xc = x + (int64_t)(ci0 + ci) * V + v;
#pragma unroll
            for (int t = 0; t < 27; ++t) {
                const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
                const float xv = ((mask >> t) & 1u) ? xc[dz * HW + dy * W + dx] : 0.f;
                const float4 wa = *reinterpret_cast<const float4 *>(&ws[ci][t][0]);
                const float4 wb = *reinterpret_cast<const float4 *>(&ws[ci][t][4]);
                acc[0] = fmaf(wa.x, xv, acc[0]);
                acc[1] = fmaf(wa.y, xv, acc[1]);
                acc[2] = fmaf(wa.z, xv, acc[2]);
                acc[3] = fmaf(wa.w, xv, acc[3]);
                acc[4] = fmaf(wb.x, xv, acc[4]);
                acc[5] = fmaf(wb.y, xv, acc[5]);
                acc[6] = fmaf(wb.z, xv, acc[6]);
                acc[7] = fmaf(wb.w, xv, acc[7]);
            }
        }
    }
    if (!live) return;
#pragma unroll
    for (int c = 0; c < kCO; ++c) {
        if (co0 + c >= Cout) break;
        float r = acc[c];
        float *out = y + (int64_t)(co0 + c) * V + v;
        if (accumulate) r += *out;
        if (relu) r = fmaxf(r, 0.f);
        *out = r;
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

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// One block per (voxel chunk, co, ci): 27 tap sums over the chunk, reduced in
// the block and added to dw; the ci == 0 blocks also add the bias gradient.
__global__ void __launch_bounds__(kT) k_conv_bww(const float *__restrict__ x, int Cin, int D, int H, int W,
                                                 const float *__restrict__ dy, int Cout, float *__restrict__ dw,
                                                 float *__restrict__ db, int64_t chunk) {
    __shared__ float red[kT / 32][28];
    const int co = blockIdx.y, ci = blockIdx.z;
    const int64_t V = (int64_t)D * H * W, HW = (int64_t)H * W;
    const int64_t v0 = (int64_t)blockIdx.x * chunk;
    const int64_t v1 = v0 + chunk < V ? v0 + chunk : V;
    float acc[28];
#pragma unroll
    for (int t = 0; t < 28; ++t) acc[t] = 0.f;
    const float *xc = x + (int64_t)ci * V;
    const float *gc = dy + (int64_t)co * V;
    for (int64_t v = v0 + threadIdx.x; v < v1; v += kT) {
        const float gv = gc[v];
        const Vox p = vox(v, H, W);
        const uint32_t mask = tap_mask(p, D, H, W);
#pragma unroll
        for (int t = 0; t < 27; ++t) {
            const int dz = t / 9 - 1, dyy = (t / 3) % 3 - 1, dx = t % 3 - 1;
            const float xv = ((mask >> t) & 1u) ? xc[v + dz * HW + dyy * W + dx] : 0.f;
            acc[t] = fmaf(gv, xv, acc[t]);
        }
        acc[27] += gv;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int t = 0; t < 28; ++t) {
        const float s = warp_sum_f(acc[t]);
        if (lane == 0) red[wid][t] = s;
    }
    __syncthreads();
    if (threadIdx.x < 28) {
        float s = 0.f;
        for (int k = 0; k < kT / 32; ++k) s += red[k][threadIdx.x];
        if (threadIdx.x < 27) atomicAdd(&dw[((int64_t)co * Cin + ci) * 27 + threadIdx.x], s);
        else if (ci == 0 && db) atomicAdd(&db[co], s);
    }
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
    dim3 grid((unsigned)((V + kT - 1) / kT), (unsigned)((Cout + kCO - 1) / kCO));
    k_conv_fwd<<<grid, kT, 0, S(stream)>>>(x, Cin, D, H, W, w, bias, Cout, y, relu, 0);
    return done(cudaGetLastError(), "lbm_nn_conv3d_forward");
}

lbm_status lbm_nn_conv3d_backward_data(const float *dy, int Cout, int D, int H, int W, const uint16_t *w,
                                       uint16_t *wt, int Cin, float *dx, int accumulate, void *stream) {
    if (!dy || !w || !wt || !dx || Cin < 1 || Cout < 1 || D < 1 || H < 1 || W < 1)
        return bad("lbm_nn_conv3d_backward_data");
    const int64_t nw = (int64_t)Cout * Cin * 27;
    k_flip_transpose<<<(unsigned)((nw + kT - 1) / kT), kT, 0, S(stream)>>>(w, wt, Cout, Cin);
    const int64_t V = (int64_t)D * H * W;
    dim3 grid((unsigned)((V + kT - 1) / kT), (unsigned)((Cin + kCO - 1) / kCO));
    k_conv_fwd<<<grid, kT, 0, S(stream)>>>(dy, Cout, D, H, W, wt, nullptr, Cin, dx, 0, accumulate);
    return done(cudaGetLastError(), "lbm_nn_conv3d_backward_data");
}

lbm_status lbm_nn_conv3d_backward_weight(const float *x, int Cin, int D, int H, int W, const float *dy, int Cout,
                                         float *dw, float *db, void *stream) {
    if (!x || !dy || !dw || Cin < 1 || Cout < 1 || D < 1 || H < 1 || W < 1 || Cin > 65535)
        return bad("lbm_nn_conv3d_backward_weight");
    const int64_t V = (int64_t)D * H * W;
    const int64_t chunk = (int64_t)kT * 32;
    dim3 grid((unsigned)((V + chunk - 1) / chunk), (unsigned)Cout, (unsigned)Cin);
    k_conv_bww<<<grid, kT, 0, S(stream)>>>(x, Cin, D, H, W, dy, Cout, dw, db, chunk);
    return done(cudaGetLastError(), "lbm_nn_conv3d_backward_weight");
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
