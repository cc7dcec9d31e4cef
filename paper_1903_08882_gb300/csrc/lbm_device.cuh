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
__host__ __device__ __forceinline__ double vfma(double a, double b, double c) { return fma(a, b, c); }
__host__ __device__ __forceinline__ float vsplat(float a, float) { return a; }
__host__ __device__ __forceinline__ double vsplat(float a, double) { return a; }
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
__host__ __device__ __forceinline__ double vrcp(double a) { return 1.0 / a; }

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
// With the rates of Sec. 2.2 (s_e = s_eps = s_nu = s_pi, s_q = s_m) S takes
// one value s_e on the even non-conserved moments and one value s_q on the odd
// ones; m^eq is M times the quadratic equilibrium
//   f_i^eq = w_i rho (1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u.u)
// and M F~ is M times the forcing term
//   F_i = w_i (3 (c - u).F + 9 (c.u)(c.F)),
// and the rows of M are orthogonal and each even or odd in c.  So M^-1 S M
// relaxes the part of f - f^eq that is even under c -> -c at s_e and the odd
// part at s_q, apart from rho and j, where S is 0; there the two forms differ
// by (s_e P_rho + s_q P_j)(f - f^eq + F/2), which is zero because
// j = rho u - F/2.  The collision is therefore evaluated pair by pair in
// velocity space: for a pair (i, ibar), S = f_i + f_ibar and D = f_i - f_ibar,
//   S+ = S - s_e (S - S^eq) + (1 - s_e/2) (F_i + F_ibar)
//   D+ = D - s_q (D - D^eq) + (1 - s_q/2) (F_i - F_ibar)
//   f_i+ = (S+ + D+)/2,  f_ibar+ = (S+ - D+)/2,
// which takes fewer instructions than the moment transform.  f holds
// deviations f - w rho0, so the equilibria below are deviations too.
// c . (x, y, z) for the first velocity e_i of pair p (its components are 0
// or +-1, so a sum or difference, no products).
template <typename V> __host__ __device__ __forceinline__ V cdot_pair(int p, V x, V y, V z) {
    switch (p) {
    case 0: return x;     // e_1 = (1, 0, 0)
    case 1: return y;     // e_3 = (0, 1, 0)
    case 2: return z;     // e_5 = (0, 0, 1)
    case 3: return x + y; // e_7 = (1, 1, 0)
    case 4: return y - x; // e_8 = (-1, 1, 0)
    case 5: return x + z; // e_11 = (1, 0, 1)
    case 6: return z - x; // e_12 = (-1, 0, 1)
    case 7: return y + z; // e_15 = (0, 1, 1)
    default: return z - y; // e_16 = (0, -1, 1)
    }
}

// GSC: g holds the thermal populations times kGScale (the FP16 storage's
// stored values, not scaled back).  The D3Q7 update is linear and
// homogeneous in (g, T), and a power-of-two scale commutes with FP32
// rounding, so it runs on the scaled values unchanged and bit for bit the
// same; only T for the force and the returned moments is scaled back.
template <typename V, bool GSC = false>
__host__ __device__ __forceinline__ MacroT<V> collide(const Phys &P, V (&f)[19], V (&g)[7]) {
    constexpr int I[9] = {1, 3, 5, 7, 8, 11, 12, 15, 16};
    constexpr int J[9] = {2, 4, 6, 10, 9, 14, 13, 18, 17};
    V S[9], D[9];
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        S[p] = f[I[p]] + f[J[p]];
        D[p] = f[I[p]] - f[J[p]];
    }
    const V f0 = f[0];
    const V drho = f0 + (((S[0] + S[1]) + S[2]) + (((S[3] + S[4]) + (S[5] + S[6])) + (S[7] + S[8])));
    const V jx = D[0] + ((D[3] - D[4]) + (D[5] - D[6]));
    const V jy = D[1] + ((D[3] + D[4]) + (D[7] - D[8]));
    const V jz = D[2] + ((D[5] + D[6]) + (D[7] + D[8]));
    const V gs0 = g[1] + g[2], gs1 = g[3] + g[4], gs2 = g[5] + g[6];
    const V T = g[0] + (gs0 + gs1) + gs2;
    const MacroT<V> mc = macro_from(P, drho, jx, jy, jz, GSC ? kGUnscale * T : T);
    const V rho = mc.rho, u = mc.u, v = mc.v, w = mc.w;
    const V Fx = mc.Fx, Fy = mc.Fy, Fz = mc.Fz;

    // Each update is written as a small correction to the pair's halves S/2
    // and D/2, so that an equilibrium pair stays exactly as it is (writing
    // (1 - s) S + s S^eq instead rounds the two complementary coefficients
    // separately, and the steady state then drifts by ~1e-5 over the viscous
    // time of a 16-node channel).  Per node and weight class w:
    //   S^eq = 2 w (drho - 3/2 rho u.u) + 9 w rho (c.u)^2,   D^eq = 6 w rho c.u
    //   F_i + F_ibar = 18 w (c.u)(c.F) - 6 w u.F,           F_i - F_ibar = 6 w c.F
    //   S+/2 = S/2 - s_e/2 (S - S^eq) + (1 - s_e/2)/2 (F_i + F_ibar)   (h)
    //   D+/2 = D/2 - s_q/2 (D - D^eq) + (1 - s_q/2)/2 (F_i - F_ibar)   (k)
    const float se = P.s_e, sq = P.s_q;
    const float ce = 1.f - 0.5f * se, cq = 1.f - 0.5f * sq;
    const V uu = vfma(u, u, vfma(v, v, w * w));
    const V uF = vfma(u, Fx, vfma(v, Fy, w * Fz));
    const V A0 = vfma(-1.5f * rho, uu, drho); // drho - 3/2 rho u.u
    const V K0a = (2.f / 18.f) * A0, K0d = (2.f / 36.f) * A0;
    const V Kca = (9.f / 18.f) * rho, Kcd = (9.f / 36.f) * rho;
    const V L0a = (-6.f / 18.f) * uF, L0d = (-6.f / 36.f) * uF;
    const V M1a = (-6.f / 18.f) * rho, M1d = (-6.f / 36.f) * rho;
    const float hse = -0.5f * se, hsq = -0.5f * sq, hce = 0.5f * ce;
    const float Lca = 18.f / 18.f, Lcd = 18.f / 36.f;
    const float Nca = 0.5f * cq * (6.f / 18.f), Ncd = 0.5f * cq * (6.f / 36.f);
    // rest population: f_0^eq = w_0 (drho - 3/2 rho u.u), F_0 = -3 w_0 u.F
    {
        const V n0 = f0 - (1.f / 3.f) * A0;
        f[0] = vfma(vsplat(-se, f0), n0, vfma(vsplat(-ce, f0), uF, f0));
    }
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        const bool axis = p < 3;
        const V cu = cdot_pair(p, u, v, w), cF = cdot_pair(p, Fx, Fy, Fz);
        const V nS = S[p] - vfma(axis ? Kca : Kcd, cu * cu, axis ? K0a : K0d);
        const V FS = vfma((axis ? Lca : Lcd) * cu, cF, axis ? L0a : L0d);
        const V h = vfma(vsplat(hse, u), nS, vfma(vsplat(0.5f, u), S[p], hce * FS));
        const V nD = vfma(axis ? M1a : M1d, cu, D[p]);
        const V k = vfma(vsplat(hsq, u), nD, vfma(vsplat(0.5f, u), D[p], (axis ? Nca : Ncd) * cF));
        f[I[p]] = h + k;
        f[J[p]] = h - k;
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

// Face nodes per thread of the face kernel: one with FP32 storage, two with
// the 2-byte storages (odd_step_node2).
template <int S> constexpr int kFacePer = S == ST_F32 ? 1 : 2;

// The same update for two nodes at once, na in the .x and nb in the .y
// component, so that the collision runs on float2 values with the packed
// FP32 instructions; vb = false leaves nb out (its lane recomputes na and
// stores nothing).  The loads and stores take one node at a time, so that
// only one node's neighbour descriptor is live.
template <int S, bool MOM, int K>
__device__ __forceinline__ void odd_load_one(const SEF<S> *__restrict__ f, const SEG<S> *__restrict__ g,
                                             const Geom &G, const Phys &P, uint32_t n, float2 (&fl)[19],
                                             float2 (&gl)[7]) {
    const int64_t s = G.stride;
    int x, y, z;
    node_xyz(G, n, x, y, z);
    const Nbr b = neighbours(G, x, y, z);
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const int ex = ex19(i), ey = ey19(i), ez = ez19(i);
        const float v = Store<FS(S)>::ld(src_wall(b, ex, ey, ez) ? f + i * s + n
                                                                 : f + opp19(i) * s + (int64_t)n + src_off(b, ex, ey, ez));
        if (K == 0) fl[i].x = v;
        else fl[i].y = v;
    }
#pragma unroll
    for (int i = 0; i < 7; ++i) {
        const int ex = ex7(i), ey = ey7(i), ez = ez7(i);
        const bool w = src_wall(b, ex, ey, ez);
        float v = Store<GS(S)>::ld(w ? g + i * s + n : g + opp7(i) * s + (int64_t)n + src_off(b, ex, ey, ez));
        if (i > 0 && w) { // a link through a Dirichlet face: anti-bounce-back
            const int fc = face_of(-ex, -ey, -ez);
            if ((P.dir_mask >> fc) & 1) v = P.abbT[fc] - v;
        }
        if (K == 0) gl[i].x = v;
        else gl[i].y = v;
    }
}
template <int S, int K>
__device__ __forceinline__ void odd_store_one(SEF<S> *__restrict__ f, SEG<S> *__restrict__ g, const Geom &G,
                                              const Phys &P, uint32_t n, const float2 (&fl)[19],
                                              const float2 (&gl)[7]) {
    const int64_t s = G.stride;
    int x, y, z;
    node_xyz(G, n, x, y, z);
    const Nbr b = neighbours(G, x, y, z);
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const int ex = ex19(i), ey = ey19(i), ez = ez19(i);
        Store<FS(S)>::st(dst_wall(b, ex, ey, ez) ? f + opp19(i) * s + n
                                                 : f + i * s + (int64_t)n + dst_off(b, ex, ey, ez),
                         K == 0 ? fl[i].x : fl[i].y);
    }
    const uint32_t r = SRG(S) ? rnd_node(n, P.t) : 0u;
    Store<GS(S)>::sts(g + n, K == 0 ? gl[0].x : gl[0].y, rnd_pop(r, 0));
#pragma unroll
    for (int i = 1; i < 7; ++i) {
        const int ex = ex7(i), ey = ey7(i), ez = ez7(i);
        const int fc = face_of(ex, ey, ez);
        const bool w = dst_wall(b, ex, ey, ez);
        const float u = K == 0 ? gl[i].x : gl[i].y;
        const float v = w && ((P.dir_mask >> fc) & 1) ? P.abbT[fc] - u : u;
        Store<GS(S)>::sts(w ? g + opp7(i) * s + n : g + i * s + (int64_t)n + dst_off(b, ex, ey, ez), v, rnd_pop(r, i));
    }
}

template <int S, bool MOM>
__device__ __forceinline__ void odd_step_node2(SEF<S> *__restrict__ f, SEG<S> *__restrict__ g, const Geom &G,
                                               const Phys &P, float *__restrict__ mom, uint32_t na, uint32_t nb,
                                               bool vb) {
    if (!vb) nb = na;
    float2 fl[19], gl[7];
    odd_load_one<S, MOM, 0>(f, g, G, P, na, fl, gl);
    odd_load_one<S, MOM, 1>(f, g, G, P, nb, fl, gl);
    float2 g0[7];
#pragma unroll
    for (int i = 0; i < 7; ++i) g0[i] = gl[i];
    const MacroT<float2> m = collide(P, fl, gl);
    f = opaque(f);
    g = opaque(g);
    asm volatile("" : "+r"(na), "+r"(nb));
    odd_store_one<S, 0>(f, g, G, P, na, fl, gl);
    if (vb) odd_store_one<S, 1>(f, g, G, P, nb, fl, gl);
    if (MOM) {
        const int64_t s = G.stride;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            if (k == 1 && !vb) break;
            const uint32_t n = k ? nb : na;
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
            node_xyz(G, n, x, y, z);
            write_sample(mom, s, n, mk, neighbours(G, x, y, z), gk);
        }
    }
}

} // namespace lbm
