// Device-side building blocks of the thermal lattice Boltzmann step:
// lattice tables, storage formats, node geometry and the fused MRT collision.
//
// Lattices (paper order): D3Q19 e_0..e_18 of Sec. 2.2, D3Q7 e_0..e_6 of
// Sec. 2.3.  Populations are stored as deviations from the rest state,
// f'_i = f_i - w_i rho0 and g'_i = g_i - w_i T0 with rho0 = 1 and T0 = 0, so
// g' = g.  All arithmetic is FP32.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {

// ------------------------------------------------------------ lattices ----

__host__ __device__ constexpr int ex19(int i) {
    constexpr int t[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
    return t[i];
}
__host__ __device__ constexpr int ey19(int i) {
    constexpr int t[19] = {0, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 1, -1, 1, -1};
    return t[i];
}
__host__ __device__ constexpr int ez19(int i) {
    constexpr int t[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1};
    return t[i];
}
__host__ __device__ constexpr int opp19(int i) {
    constexpr int t[19] = {0, 2, 1, 4, 3, 6, 5, 10, 9, 8, 7, 14, 13, 12, 11, 18, 17, 16, 15};
    return t[i];
}
__host__ __device__ constexpr int ex7(int i) {
    constexpr int t[7] = {0, 1, -1, 0, 0, 0, 0};
    return t[i];
}
__host__ __device__ constexpr int ey7(int i) {
    constexpr int t[7] = {0, 0, 0, 1, -1, 0, 0};
    return t[i];
}
__host__ __device__ constexpr int ez7(int i) {
    constexpr int t[7] = {0, 0, 0, 0, 0, 1, -1};
    return t[i];
}
__host__ __device__ constexpr int opp7(int i) {
    constexpr int t[7] = {0, 2, 1, 4, 3, 6, 5};
    return t[i];
}

// D3Q19 weights w_i (Sec. 2.2).
__host__ __device__ constexpr float w19(int i) {
    return i == 0 ? 1.0f / 3.0f : (i < 7 ? 1.0f / 18.0f : 1.0f / 36.0f);
}

// -------------------------------------------------------- storage types ----

enum StorageKind { ST_F32 = 0, ST_F16 = 1, ST_BF16 = 2, ST_F16M = 3 };
// Element format of the FP16 thermal arrays: g times kGScale in FP16.  The
// D3Q7 weights make the moving populations small (w_1 T ~ 1e-4 - 1e-2, and
// far less where T ~ 0), and FP16 below 6.1e-5 is subnormal, with a fixed
// spacing of 6e-8 and a biased stochastic rounding (see below); scaled by
// 2^12 every |g| above 1.5e-8 is a normal number, and |g| up to 16 still fits.
constexpr int ST_F16T = 4;
constexpr float kGScale = 4096.f, kGUnscale = 1.f / 4096.f;

// Element format of the flow (f) and thermal (g) arrays of a storage kind:
// ST_F16M keeps f in FP16 and g in FP32; ST_F16 keeps g in scaled FP16.
__host__ __device__ constexpr int FS(int S) { return S == ST_F16M ? ST_F16 : S; }
__host__ __device__ constexpr int GS(int S) { return S == ST_F16M ? ST_F32 : S == ST_F16 ? ST_F16T : S; }

// ------------------------------------------------- stochastic rounding ----
//
// The 2-byte storages round the thermal populations stochastically: a value
// is stored as one of the two neighbouring 2-byte numbers, the one above with
// probability equal to the fraction of the gap it covers, so the stored value
// is unbiased.  Rounding to nearest loses every update smaller than half the
// spacing, which freezes the slow approach to a steady state far from it: the
// rest population g_0 = (1 - a_T)/7 T holds 60-97% of T ~ 1/2 to ~2e-4 while
// a step changes T by ~1e-6, and the rounding of the moving ones biases the
// wall heat flux they carry by ~0.5% on a 33^3 cell.  Unbiased rounding keeps
// those updates on average.  The random bits are a counter-based hash of
// (node, time step) spread over the populations, so runs are reproducible
// and every kernel variant draws the same bits for a value.
__host__ __device__ constexpr bool SRG(int S) { return S == ST_F16 || S == ST_BF16; }

// 32 random bits of node n at time step t (multiply-xorshift hash).
__host__ __device__ __forceinline__ uint32_t rnd_node(uint32_t n, uint32_t t) {
    uint32_t x = (n ^ (t * 0x9E3779B9u)) * 0x85EBCA6Bu;
    x ^= x >> 13;
    return x * 0xC2B2AE35u;
}
// Bits for population q of that node: the node's bits times an odd constant
// per population (the high bits are used).
__host__ __device__ __forceinline__ uint32_t rnd_pop(uint32_t r, int q) {
    return r * (0x9E3779B1u + 0x3C6EF372u * static_cast<uint32_t>(q));
}
// Stochastic rounding of an FP32 value to FP16 / BF16: add random bits below
// the kept significand to the magnitude, then truncate towards zero (exact
// for normal numbers; below the FP16 normal range, 6.1e-5, the result can be
// biased towards zero by up to one FP16 subnormal spacing, 6e-8, which is
// why the thermal populations are stored scaled, ST_F16T).
__device__ __forceinline__ float sr_pre16(float v, uint32_t r) {
    return __uint_as_float(__float_as_uint(v) + (r >> 19));
}
__device__ __forceinline__ float sr_pre_bf(float v, uint32_t r) {
    return __uint_as_float(__float_as_uint(v) + (r >> 16));
}
__device__ __forceinline__ __half2 h2_sr(float2 v, uint32_t r0, uint32_t r1) {
    uint32_t o;
    asm("cvt.rz.f16x2.f32 %0, %1, %2;" : "=r"(o) : "f"(sr_pre16(v.y, r1)), "f"(sr_pre16(v.x, r0)));
    return *reinterpret_cast<__half2 *>(&o);
}
__device__ __forceinline__ __nv_bfloat162 bf2_sr(float2 v, uint32_t r0, uint32_t r1) {
    uint32_t o;
    asm("cvt.rz.bf16x2.f32 %0, %1, %2;" : "=r"(o) : "f"(sr_pre_bf(v.y, r1)), "f"(sr_pre_bf(v.x, r0)));
    return *reinterpret_cast<__nv_bfloat162 *>(&o);
}

template <int S> struct Store;
// st: round to nearest; sts: the thermal populations' rounding, given 32
// random bits r (stochastic for the 2-byte formats, see SRG above).
template <> struct Store<ST_F32> {
    using T = float;
    static __device__ __forceinline__ float ld(const float *p) { return *p; }
    static __device__ __forceinline__ void st(float *p, float v) { *p = v; }
    static __device__ __forceinline__ void sts(float *p, float v, uint32_t) { *p = v; }
};
template <> struct Store<ST_F16> {
    using T = __half;
    static __device__ __forceinline__ float ld(const __half *p) { return __half2float(*p); }
    static __device__ __forceinline__ void st(__half *p, float v) { *p = __float2half_rn(v); }
    static __device__ __forceinline__ void sts(__half *p, float v, uint32_t r) {
        *p = __float2half_rz(sr_pre16(v, r));
    }
};
template <> struct Store<ST_F16T> {
    using T = __half;
    static __device__ __forceinline__ float ld(const __half *p) { return __half2float(*p) * kGUnscale; }
    static __device__ __forceinline__ void st(__half *p, float v) { *p = __float2half_rn(v * kGScale); }
    static __device__ __forceinline__ void sts(__half *p, float v, uint32_t r) {
        *p = __float2half_rz(sr_pre16(v * kGScale, r));
    }
};
template <> struct Store<ST_BF16> {
    using T = __nv_bfloat16;
    static __device__ __forceinline__ float ld(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
    static __device__ __forceinline__ void st(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
    static __device__ __forceinline__ void sts(__nv_bfloat16 *p, float v, uint32_t r) {
        *p = __float2bfloat16_rz(sr_pre_bf(v, r));
    }
};

// Two consecutive elements (first index even, so 4- or 8-byte aligned).
template <int S> struct Store2;
template <> struct Store2<ST_F32> {
    static __device__ __forceinline__ float2 ld(const float *p) { return *reinterpret_cast<const float2 *>(p); }
    static __device__ __forceinline__ void st(float *p, float2 v) { *reinterpret_cast<float2 *>(p) = v; }
    static __device__ __forceinline__ void sts(float *p, float2 v, uint32_t, uint32_t) { st(p, v); }
};
template <> struct Store2<ST_F16> {
    static __device__ __forceinline__ float2 ld(const __half *p) {
        return __half22float2(*reinterpret_cast<const __half2 *>(p));
    }
    static __device__ __forceinline__ void st(__half *p, float2 v) {
        *reinterpret_cast<__half2 *>(p) = __float22half2_rn(v);
    }
    static __device__ __forceinline__ void sts(__half *p, float2 v, uint32_t r0, uint32_t r1) {
        *reinterpret_cast<__half2 *>(p) = h2_sr(v, r0, r1);
    }
};
template <> struct Store2<ST_F16T> {
    static __device__ __forceinline__ float2 ld(const __half *p) {
        const float2 v = __half22float2(*reinterpret_cast<const __half2 *>(p));
        return make_float2(v.x * kGUnscale, v.y * kGUnscale);
    }
    static __device__ __forceinline__ void st(__half *p, float2 v) {
        *reinterpret_cast<__half2 *>(p) = __float22half2_rn(make_float2(v.x * kGScale, v.y * kGScale));
    }
    static __device__ __forceinline__ void sts(__half *p, float2 v, uint32_t r0, uint32_t r1) {
        *reinterpret_cast<__half2 *>(p) = h2_sr(make_float2(v.x * kGScale, v.y * kGScale), r0, r1);
    }
};
template <> struct Store2<ST_BF16> {
    static __device__ __forceinline__ float2 ld(const __nv_bfloat16 *p) {
        return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(p));
    }
    static __device__ __forceinline__ void st(__nv_bfloat16 *p, float2 v) {
        *reinterpret_cast<__nv_bfloat162 *>(p) = __float22bfloat162_rn(v);
    }
    static __device__ __forceinline__ void sts(__nv_bfloat16 *p, float2 v, uint32_t r0, uint32_t r1) {
        *reinterpret_cast<__nv_bfloat162 *>(p) = bf2_sr(v, r0, r1);
    }
};

// ------------------------------------------------------ kernel arguments ----

// Lattice geometry.  Node index n = x + nx (y + ny z) < 2^32; population q of
// node n lives at base + q * stride + n.
struct Geom {
    int nx, ny, nz;
    uint32_t n, nxy;
    int64_t stride;
    uint64_t mag_nx, mag_nxy; // ceil(2^64 / d): exact quotients for 32-bit numerators
    int periodic;             // bit a: axis a wraps
    // interior nodes (1 <= x <= nx-2, ...; no neighbour behind a face): count,
    // row length nx-2 and plane size (nx-2)(ny-2) with their division magics
    uint32_t ni, nix, nixy;
    uint64_t mag_nix, mag_nixy;
    int off[19]; // flat offset of e_i: ex + nx ey + nx ny ez
    // 64-node chunks per z-plane over the rows 1 <= y <= ny-2, and its magic
    uint32_t cpp;
    uint64_t mag_cpp;
};

// Physical constants of one cell (FP32).
struct Phys {
    float s_e, s_q;  // flow rates: s_e = s_eps = s_nu = s_pi = 1/tau_f, s_q = s_m
    float q_k, q_e;  // D3Q7 rates: q_kappa and q_e = q_nu
    float a_T;
    float gbeta;
    float bf[3];     // constant body-force density
    float abbT[6];   // (6 + a_T)/21 T_w of each Dirichlet face
    int dir_mask;    // bit f: face f is a Dirichlet wall
    uint32_t t;      // time step being taken (low 32 bits): the stochastic rounding's counter
};

// a / d for 32-bit a and d, given mag = ceil(2^64 / d) (exact: the rounding
// error a (mag - 2^64/d) / 2^64 stays below 2^-32 <= 1/d); d = 1 has no
// 64-bit magic and is passed as mag = 0.
__device__ __forceinline__ uint32_t fast_div(uint32_t a, uint64_t mag) {
    return mag ? static_cast<uint32_t>(__umul64hi(static_cast<uint64_t>(a), mag)) : a;
}

// Offsets to the neighbours along each axis and which sides are walls.
struct Nbr {
    int om[3], op[3]; // offset of the -1 / +1 neighbour (wrapped when periodic)
    bool wm[3], wp[3]; // the -1 / +1 neighbour lies behind a wall
};

__device__ __forceinline__ void node_xyz(const Geom &G, uint32_t n, int &x, int &y, int &z) {
    uint32_t zz = fast_div(n, G.mag_nxy);
    uint32_t r = n - zz * G.nxy;
    uint32_t yy = fast_div(r, G.mag_nx);
    x = static_cast<int>(r - yy * static_cast<uint32_t>(G.nx));
    y = static_cast<int>(yy);
    z = static_cast<int>(zz);
}

__device__ __forceinline__ Nbr neighbours(const Geom &G, int x, int y, int z) {
    Nbr b;
    const int c[3] = {x, y, z};
    const int len[3] = {G.nx, G.ny, G.nz};
    const int step[3] = {1, G.nx, static_cast<int>(G.nxy)};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const bool per = (G.periodic >> a) & 1;
        const bool lo = c[a] == 0, hi = c[a] == len[a] - 1;
        b.om[a] = lo ? (len[a] - 1) * step[a] : -step[a];
        b.op[a] = hi ? -(len[a] - 1) * step[a] : step[a];
        b.wm[a] = lo && !per;
        b.wp[a] = hi && !per;
    }
    return b;
}

// Source x - e and destination x + e of a compile-time velocity e.
__device__ __forceinline__ int src_off(const Nbr &b, int ex, int ey, int ez) {
    return (ex > 0 ? b.om[0] : ex < 0 ? b.op[0] : 0) + (ey > 0 ? b.om[1] : ey < 0 ? b.op[1] : 0) +
           (ez > 0 ? b.om[2] : ez < 0 ? b.op[2] : 0);
}
__device__ __forceinline__ bool src_wall(const Nbr &b, int ex, int ey, int ez) {
    return (ex > 0 ? b.wm[0] : ex < 0 ? b.wp[0] : false) ||
           (ey > 0 ? b.wm[1] : ey < 0 ? b.wp[1] : false) ||
           (ez > 0 ? b.wm[2] : ez < 0 ? b.wp[2] : false);
}
__device__ __forceinline__ int dst_off(const Nbr &b, int ex, int ey, int ez) {
    return src_off(b, -ex, -ey, -ez);
}
__device__ __forceinline__ bool dst_wall(const Nbr &b, int ex, int ey, int ez) {
    return src_wall(b, -ex, -ey, -ez);
}
// Face crossed by an axis-aligned link leaving the node along e.
__host__ __device__ constexpr int face_of(int ex, int ey, int ez) {
    return ex != 0 ? (ex > 0 ? 1 : 0) : ey != 0 ? (ey > 0 ? 3 : 2) : (ez > 0 ? 5 : 4);
}

// ------------------------------------------------------------- collision ----
//
// Opposite velocity pairs (i, ibar) in paper order: (1,2) (3,4) (5,6) (7,10)
// (8,9) (11,14) (12,13) (15,18) (16,17) for D3Q19 and (1,2) (3,4) (5,6) for
// D3Q7.  Every row of M and N is a polynomial that is even or odd in e, so an
// even moment sees a pair only through s = f_i + f_ibar and an odd moment only
// through d = f_i - f_ibar; likewise M^T splits into an even part E and an odd
// part O with f_i+ = f_i - E - O and f_ibar+ = f_ibar - E + O.  The sums below
// are the rows of M and N of Secs. 2.2-2.3 written over s and d.

// ----------------------------------------------------- grid-wide barrier ----
//
// All blocks of a cooperative launch arrive on a counter; the last one resets
// it and advances the generation that the others wait on.  Each wait gives up
// after `budget` clock cycles, raises the shared error flag and lets every
// block leave; the caller reads the flag after the launch.  Returns false once
// the flag is up.
template <typename B> __device__ __forceinline__ bool grid_barrier(B *bar, unsigned nblocks, long long budget) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *gen = &bar->gen;
        volatile int *err = &bar->err;
        const unsigned g0 = *gen;
        __threadfence();
        if (atomicAdd(&bar->count, 1u) == nblocks - 1u) {
            atomicExch(&bar->count, 0u);
            __threadfence();
            atomicAdd(&bar->gen, 1u);
        } else {
            const long long t0 = clock64();
            while (*gen == g0) {
                if (*err) break;
                if (clock64() - t0 > budget) {
                    atomicExch(&bar->err, 1);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return *reinterpret_cast<volatile int *>(&bar->err) == 0;
}

// ------------------------------------------------------ vector arithmetic ----
//
// The collision is written once for a value type V: float (one node per
// thread) or float2 (two nodes per thread, evaluated with the packed FP32
// instructions of sm_100 and later: one instruction updates both nodes).

__host__ __device__ __forceinline__ float2 operator+(float2 a, float2 b) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
    return __fadd2_rn(a, b);
#else
    return make_float2(a.x + b.x, a.y + b.y);
#endif
}
__host__ __device__ __forceinline__ float2 operator-(float2 a) { return make_float2(-a.x, -a.y); }
__host__ __device__ __forceinline__ float2 operator-(float2 a, float2 b) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
    return __fadd2_rn(a, -b);
#else
    return make_float2(a.x - b.x, a.y - b.y);
#endif
}
__host__ __device__ __forceinline__ float2 operator*(float2 a, float2 b) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
    return __fmul2_rn(a, b);
#else
    return make_float2(a.x * b.x, a.y * b.y);
#endif
}
__host__ __device__ __forceinline__ float2 operator*(float a, float2 b) { return make_float2(a, a) * b; }
__host__ __device__ __forceinline__ float2 operator*(float2 a, float b) { return a * make_float2(b, b); }
__host__ __device__ __forceinline__ float2 &operator+=(float2 &a, float2 b) { return a = a + b; }
__host__ __device__ __forceinline__ float2 &operator-=(float2 &a, float2 b) { return a = a - b; }

__host__ __device__ __forceinline__ float vfma(float a, float b, float c) { return fmaf(a, b, c); }
__host__ __device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
    return __ffma2_rn(a, b, c);
#else
    return make_float2(fmaf(a.x, b.x, c.x), fmaf(a.y, b.y, c.y));
#endif
}
__host__ __device__ __forceinline__ float vsplat(float a, float) { return a; }
__host__ __device__ __forceinline__ float2 vsplat(float a, float2) { return make_float2(a, a); }
// correctly rounded reciprocal
__host__ __device__ __forceinline__ float vrcp(float a) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
    return __frcp_rn(a);
#else
    return 1.0f / a;
#endif
}
__host__ __device__ __forceinline__ float2 vrcp(float2 a) { return make_float2(vrcp(a.x), vrcp(a.y)); }

// ------------------------------------------------------------- collision ----
//
// Opposite velocity pairs (i, ibar) in paper order: (1,2) (3,4) (5,6) (7,10)
// (8,9) (11,14) (12,13) (15,18) (16,17) for D3Q19 and (1,2) (3,4) (5,6) for
// D3Q7.  Every row of M and N is a polynomial that is even or odd in e, so an
// even moment sees a pair only through s = f_i + f_ibar and an odd moment only
// through d = f_i - f_ibar; likewise M^T splits into an even part E and an odd
// part O with f_i+ = f_i - E - O and f_ibar+ = f_ibar - E + O.  The sums below
// are the rows of M and N of Secs. 2.2-2.3 written over s and d.

// Moments of one node: rho - rho0, rho, u = (sum e f + F/2)/rho, T, and the
// force F = body force + rho g beta T z-hat (Sec. 2.2).
template <typename V> struct MacroT {
    V drho, rho, u, v, w, T, Fx, Fy, Fz;
};
using Macro = MacroT<float>;

template <typename V>
__host__ __device__ __forceinline__ MacroT<V> macro_from(const Phys &P, V drho, V jx, V jy, V jz, V T) {
    MacroT<V> m;
    const V one = vsplat(1.0f, drho);
    const V rho = one + drho;
    m.drho = drho;
    m.rho = rho;
    m.T = T;
    m.Fx = vsplat(P.bf[0], drho);
    m.Fy = vsplat(P.bf[1], drho);
    m.Fz = vfma(P.gbeta * rho, T, vsplat(P.bf[2], drho));
    const V inv = vrcp(rho);
    m.u = vfma(vsplat(0.5f, drho), m.Fx, jx) * inv;
    m.v = vfma(vsplat(0.5f, drho), m.Fy, jy) * inv;
    m.w = vfma(vsplat(0.5f, drho), m.Fz, jz) * inv;
    return m;
}

template <typename V>
__host__ __device__ __forceinline__ MacroT<V> macro(const Phys &P, const V (&f)[19], const V (&g)[7]) {
    const V dr = f[0] + ((f[1] + f[2]) + (f[3] + f[4]) + (f[5] + f[6])) +
                 (((f[7] + f[10]) + (f[8] + f[9])) + ((f[11] + f[14]) + (f[12] + f[13])) +
                  ((f[15] + f[18]) + (f[16] + f[17])));
    const V jx = (f[1] - f[2]) + ((f[7] - f[10]) - (f[8] - f[9])) + ((f[11] - f[14]) - (f[12] - f[13]));
    const V jy = (f[3] - f[4]) + ((f[7] - f[10]) + (f[8] - f[9])) + ((f[15] - f[18]) - (f[16] - f[17]));
    const V jz = (f[5] - f[6]) + ((f[11] - f[14]) + (f[12] - f[13])) + ((f[15] - f[18]) + (f[16] - f[17]));
    const V T = g[0] + (g[1] + g[2]) + (g[3] + g[4]) + (g[5] + g[6]);
    return macro_from(P, dr, jx, jy, jz, T);
}

// One fused collision of both distributions at one node (or two nodes for
// V = float2), in place:
//   f+ = f - M^-1 [S (m - m^eq) - (I - S/2) M F~]      (Eq. MRT)
//   g+ = g - N^-1 Q (n - n^eq)                          (Eq. MRT_T)
// f holds deviations f - w rho0; the rest-state moments M w rho0 =
// (rho0, -11 rho0, 3 rho0, 0, ...) are folded into m - m^eq below.
// M^-1 = M^T diag(1/|M_k|^2), N^-1 = N^T diag(1/|N_k|^2).
template <typename V>
__host__ __device__ __forceinline__ MacroT<V> collide(const Phys &P, V (&f)[19], V (&g)[7]) {
    constexpr int I[9] = {1, 3, 5, 7, 8, 11, 12, 15, 16};
    constexpr int J[9] = {2, 4, 6, 10, 9, 14, 13, 18, 17};
    V s[9], d[9];
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        s[p] = f[I[p]] + f[J[p]];
        d[p] = f[I[p]] - f[J[p]];
    }
    const V f0 = f[0];
    const V s34 = s[3] + s[4], s56 = s[5] + s[6], s78 = s[7] + s[8];
    const V Sax = (s[0] + s[1]) + s[2];
    const V Sdg = (s34 + s56) + s78;
    const V dx = (d[3] - d[4]) + (d[5] - d[6]); // diagonal parts of j
    const V dy = (d[3] + d[4]) + (d[7] - d[8]);
    const V dz = (d[5] + d[6]) + (d[7] + d[8]);
    const V gs0 = g[1] + g[2], gs1 = g[3] + g[4], gs2 = g[5] + g[6];
    const V T = g[0] + (gs0 + gs1) + gs2;
    const MacroT<V> mc = macro_from(P, f0 + Sax + Sdg, d[0] + dx, d[1] + dy, d[2] + dz, T);
    const V rho = mc.rho, u = mc.u, v = mc.v, w = mc.w;
    const V Fx = mc.Fx, Fy = mc.Fy, Fz = mc.Fz;

    // m - m^eq (Sec. 2.2 m^eq) of the non-conserved moments
    const V uu = u * u + v * v + w * w;
    const V ru = rho * u, rv = rho * v, rw = rho * w;
    const V pxx = rho * (2.f * (u * u) - v * v - w * w);
    const V pww = rho * (v * v - w * w);
    const V s3456 = s34 + s56;
    const V ruu = rho * uu;
    const V d1 = (-30.f * f0 - 11.f * Sax + 8.f * Sdg) + 11.f * mc.drho - 19.f * ruu;
    const V d2 = (12.f * f0 - 4.f * Sax + Sdg) - 3.f * mc.drho + 5.5f * ruu;
    const V d4 = (-4.f * d[0] + dx) + (2.f / 3.f) * ru;
    const V d6 = (-4.f * d[1] + dy) + (2.f / 3.f) * rv;
    const V d8 = (-4.f * d[2] + dz) + (2.f / 3.f) * rw;
    const V d9 = (2.f * s[0] - s[1] - s[2] + s3456 - 2.f * s78) - pxx;
    const V d10 = (-4.f * s[0] + 2.f * s[1] + 2.f * s[2] + s3456 - 2.f * s78) + 0.5f * pxx;
    const V d11 = (s[1] - s[2] + s34 - s56) - pww;
    const V d12 = (-2.f * s[1] + 2.f * s[2] + s34 - s56) + 0.5f * pww;
    const V d13 = (s[3] - s[4]) - ru * v;
    const V d14 = (s[7] - s[8]) - rv * w;
    const V d15 = (s[5] - s[6]) - ru * w;
    const V d16 = (d[3] - d[4]) - (d[5] - d[6]);
    const V d17 = (d[7] - d[8]) - (d[3] + d[4]);
    const V d18 = (d[5] + d[6]) - (d[7] + d[8]);

    // a_k, b_k = [S (m - m^eq) - (I - S/2) M F~]_k / |M_k|^2 (even k: a, odd k: b)
    const V uFx = u * Fx, vFy = v * Fy, wFz = w * Fz;
    const V uF = uFx + vFy + wFz;
    const float se = P.s_e, sq = P.s_q;
    const float ce = 1.f - 0.5f * se, cq = 1.f - 0.5f * sq;
    const V a1 = (se * d1 - (ce * 38.f) * uF) * (1.f / 2394.f);
    const V a2 = (se * d2 + (ce * 11.f) * uF) * (1.f / 252.f);
    const V a9 = (se * d9 - ce * (4.f * uFx - 2.f * vFy - 2.f * wFz)) * (1.f / 36.f);
    const V a10 = (se * d10 - ce * (-2.f * uFx + vFy + wFz)) * (1.f / 72.f);
    const V a11 = (se * d11 - ce * (2.f * vFy - 2.f * wFz)) * (1.f / 12.f);
    const V a12 = (se * d12 - ce * (wFz - vFy)) * (1.f / 24.f);
    const V a13 = (se * d13 - ce * (u * Fy + v * Fx)) * 0.25f;
    const V a14 = (se * d14 - ce * (v * Fz + w * Fy)) * 0.25f;
    const V a15 = (se * d15 - ce * (u * Fz + w * Fx)) * 0.25f;
    const V b3 = -0.1f * Fx, b5 = -0.1f * Fy, b7 = -0.1f * Fz;
    const V b4 = (sq * d4 + (cq * (2.f / 3.f)) * Fx) * (1.f / 40.f);
    const V b6 = (sq * d6 + (cq * (2.f / 3.f)) * Fy) * (1.f / 40.f);
    const V b8 = (sq * d8 + (cq * (2.f / 3.f)) * Fz) * (1.f / 40.f);
    const V b16 = (sq * 0.125f) * d16, b17 = (sq * 0.125f) * d17, b18 = (sq * 0.125f) * d18;

    // M^T applied to (a, b): even parts E_p and odd parts O_p of each pair
    const V Cax = -11.f * a1 - 4.f * a2, Cdg = 8.f * a1 + a2;
    const V X = a9 + a10, Y = a11 + a12, Z = a11 - 2.f * a12;
    const V Jx = b3 + b4, Jy = b5 + b6, Jz = b7 + b8;
    const V CaxX = Cax - a9 + 2.f * a10, CdgXY = Cdg + X + Y, CdgXmY = Cdg + X - Y, Cdg2X = Cdg - 2.f * X;
    V E[9], O[9];
    E[0] = Cax + 2.f * a9 - 4.f * a10;
    E[1] = CaxX + Z;
    E[2] = CaxX - Z;
    E[3] = CdgXY + a13;
    E[4] = CdgXY - a13;
    E[5] = CdgXmY + a15;
    E[6] = CdgXmY - a15;
    E[7] = Cdg2X + a14;
    E[8] = Cdg2X - a14;
    O[0] = b3 - 4.f * b4;
    O[1] = b5 - 4.f * b6;
    O[2] = b7 - 4.f * b8;
    O[3] = Jx + Jy + (b16 - b17);
    O[4] = Jy - Jx - (b16 + b17);
    O[5] = Jx + Jz + (b18 - b16);
    O[6] = Jz - Jx + (b16 + b18);
    O[7] = Jy + Jz + (b17 - b18);
    O[8] = Jz - Jy - (b17 + b18);
    // f_i = (s + d)/2 and f_ibar = (s - d)/2: the pair sums replace f here, so
    // the 19 inputs need not stay live through the collision
    f[0] = f0 - (-30.f * a1 + 12.f * a2);
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        f[I[p]] = vfma(vsplat(0.5f, f0), s[p] + d[p], -(E[p] + O[p]));
        f[J[p]] = vfma(vsplat(0.5f, f0), s[p] - d[p], O[p] - E[p]);
    }

    // D3Q7: n - n^eq with n^eq = (T, uT, vT, wT, a_T T, 0, 0); |N_k|^2 = 7, 2, 2, 2, 42, 12, 4
    const float hk = 0.5f * P.q_k;
    const V e1 = hk * ((g[1] - g[2]) - u * T);
    const V e2 = hk * ((g[3] - g[4]) - v * T);
    const V e3 = hk * ((g[5] - g[6]) - w * T);
    const V e4 = (P.q_e * (1.f / 42.f)) * ((-6.f * g[0] + (gs0 + gs1) + gs2) - P.a_T * T);
    const V e5 = (P.q_e * (1.f / 12.f)) * (2.f * gs0 - gs1 - gs2);
    const V e6 = (P.q_e * 0.25f) * (gs1 - gs2);
    g[0] += 6.f * e4;
    const V E1 = e4 + 2.f * e5, E2 = e4 - e5 + e6, E3 = e4 - e5 - e6;
    g[1] -= E1 + e1;
    g[2] -= E1 - e1;
    g[3] -= E2 + e2;
    g[4] -= E2 - e2;
    g[5] -= E3 + e3;
    g[6] -= E3 - e3;
    return mc;
}


// ------------------------------------------------ shared kernel helpers ----

template <int S> using SEF = typename Store<FS(S)>::T; // flow element type
template <int S> using SEG = typename Store<GS(S)>::T; // thermal element type

// Hide a pointer's value from the compiler so that addresses computed from it
// before the collision are not kept live across it (recomputing 26 addresses
// costs a few instructions; keeping them costs 52 registers).
template <typename T> __device__ __forceinline__ T *opaque(T *p) {
    asm volatile("" : "+l"(p));
    return p;
}

// Diagnostic sample of one node: moments (rho - rho0, u, v, w, T) of the
// pre-collision state, and for a node next to a wall on face f the
// pre-collision g arriving from that wall (velocity index f + 1 points away
// from face f).  gin holds g before the collision.
__device__ __forceinline__ void write_sample(float *__restrict__ mom, int64_t s, uint32_t n,
                                             const Macro &m, const Nbr &b, const float (&gin)[7]) {
    mom[n] = m.drho;
    mom[s + n] = m.u;
    mom[2 * s + n] = m.v;
    mom[3 * s + n] = m.w;
    mom[4 * s + n] = m.T;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (b.wm[a]) mom[(5 + 2 * a) * s + n] = gin[2 * a + 1];
        if (b.wp[a]) mom[(6 + 2 * a) * s + n] = gin[2 * a + 2];
    }
}

// AA odd step of one node through the general path: every link checked for
// a wall (bounce-back, anti-bounce-back for g at a Dirichlet face) or a
// periodic wrap.  Used for the nodes next to a face.
template <int S, bool MOM>
__device__ __forceinline__ void odd_step_node(SEF<S> *__restrict__ f, SEG<S> *__restrict__ g, const Geom &G,
                                              const Phys &P, float *__restrict__ mom, uint32_t n) {
    const int64_t s = G.stride;
    int x, y, z;
    node_xyz(G, n, x, y, z);
    const Nbr b = neighbours(G, x, y, z);
    float fl[19], gl[7];
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        if (!src_wall(b, ex19(i), ey19(i), ez19(i)))
            fl[i] = Store<FS(S)>::ld(f + opp19(i) * s + (int64_t)n + src_off(b, ex19(i), ey19(i), ez19(i)));
        else
            fl[i] = Store<FS(S)>::ld(f + i * s + n);
    }
#pragma unroll
    for (int i = 0; i < 7; ++i) {
        if (!src_wall(b, ex7(i), ey7(i), ez7(i))) {
            gl[i] = Store<GS(S)>::ld(g + opp7(i) * s + (int64_t)n + src_off(b, ex7(i), ey7(i), ez7(i)));
        } else {
            const int fc = face_of(-ex7(i), -ey7(i), -ez7(i));
            const float v = Store<GS(S)>::ld(g + i * s + n);
            gl[i] = ((P.dir_mask >> fc) & 1) ? P.abbT[fc] - v : v;
        }
    }
    float g0[7];
#pragma unroll
    for (int i = 0; i < 7; ++i) g0[i] = gl[i];
    const Macro m = collide(P, fl, gl);
    f = opaque(f);
    g = opaque(g);
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        if (!dst_wall(b, ex19(i), ey19(i), ez19(i)))
            Store<FS(S)>::st(f + i * s + (int64_t)n + dst_off(b, ex19(i), ey19(i), ez19(i)), fl[i]);
        else
            Store<FS(S)>::st(f + opp19(i) * s + n, fl[i]);
    }
    const uint32_t rb = SRG(S) ? rnd_node(n, P.t) : 0u;
    Store<GS(S)>::sts(g + n, gl[0], rnd_pop(rb, 0));
#pragma unroll
    for (int i = 1; i < 7; ++i) {
        if (!dst_wall(b, ex7(i), ey7(i), ez7(i))) {
            Store<GS(S)>::sts(g + i * s + (int64_t)n + dst_off(b, ex7(i), ey7(i), ez7(i)), gl[i], rnd_pop(rb, i));
        } else {
            const int fc = face_of(ex7(i), ey7(i), ez7(i));
            const float v = gl[i];
            Store<GS(S)>::sts(g + opp7(i) * s + n, ((P.dir_mask >> fc) & 1) ? P.abbT[fc] - v : v, rnd_pop(rb, i));
        }
    }
    if (MOM) write_sample(mom, s, n, m, b, g0);
}

} // namespace lbm
