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

// D3Q19 transformation matrix M of Sec. 2.2 (rows: moments rho, e, eps, jx,
// qx, jy, qy, jz, qz, 3pxx, 3pixx, pww, piww, pxy, pyz, pxz, mx, my, mz).
__host__ __device__ constexpr int Mk(int k, int i) {
    constexpr int t[19][19] = {
        {1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1},
        {-30, -11, -11, -11, -11, -11, -11, 8, 8, 8, 8, 8, 8, 8, 8, 8, 8, 8, 8},
        {12, -4, -4, -4, -4, -4, -4, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1},
        {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0},
        {0, -4, 4, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0},
        {0, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 1, -1, 1, -1},
        {0, 0, 0, -4, 4, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 1, -1, 1, -1},
        {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1},
        {0, 0, 0, 0, 0, -4, 4, 0, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1},
        {0, 2, 2, -1, -1, -1, -1, 1, 1, 1, 1, 1, 1, 1, 1, -2, -2, -2, -2},
        {0, -4, -4, 2, 2, 2, 2, 1, 1, 1, 1, 1, 1, 1, 1, -2, -2, -2, -2},
        {0, 0, 0, 1, 1, -1, -1, 1, 1, 1, 1, -1, -1, -1, -1, 0, 0, 0, 0},
        {0, 0, 0, -2, -2, 2, 2, 1, 1, 1, 1, -1, -1, -1, -1, 0, 0, 0, 0},
        {0, 0, 0, 0, 0, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 0, 0, 0, 0},
        {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, -1, -1, 1},
        {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0},
        {0, 0, 0, 0, 0, 0, 0, 1, -1, 1, -1, -1, 1, -1, 1, 0, 0, 0, 0},
        {0, 0, 0, 0, 0, 0, 0, -1, -1, 1, 1, 0, 0, 0, 0, 1, -1, 1, -1},
        {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 1, -1, -1, -1, -1, 1, 1}};
    return t[k][i];
}
// Squared row norms of M: M^-1 = M^T diag(1/|M_k|^2).
__host__ __device__ constexpr int Mnorm(int k) {
    constexpr int t[19] = {19, 2394, 252, 10, 40, 10, 40, 10, 40, 36, 72, 12, 24, 4, 4, 4, 8, 8, 8};
    return t[k];
}
// D3Q7 transformation matrix N of Sec. 2.3 with the <e_z| row taken from its
// definition (0, 0, 0, 0, 0, 1, -1).
__host__ __device__ constexpr int Nk(int k, int i) {
    constexpr int t[7][7] = {{1, 1, 1, 1, 1, 1, 1},   {0, 1, -1, 0, 0, 0, 0},
                             {0, 0, 0, 1, -1, 0, 0},  {0, 0, 0, 0, 0, 1, -1},
                             {-6, 1, 1, 1, 1, 1, 1},  {0, 2, 2, -1, -1, -1, -1},
                             {0, 0, 0, 1, 1, -1, -1}};
    return t[k][i];
}
__host__ __device__ constexpr int Nnorm(int k) {
    constexpr int t[7] = {7, 2, 2, 2, 42, 12, 4};
    return t[k];
}
// D3Q19 weights w_i (Sec. 2.2).
__host__ __device__ constexpr float w19(int i) {
    return i == 0 ? 1.0f / 3.0f : (i < 7 ? 1.0f / 18.0f : 1.0f / 36.0f);
}

// Accumulate c * x for a compile-time integer coefficient c.
__device__ __forceinline__ void acc_int(float &s, int c, float x) {
    if (c == 1) s += x;
    else if (c == -1) s -= x;
    else if (c != 0) s = fmaf(static_cast<float>(c), x, s);
}

// -------------------------------------------------------- storage types ----

enum StorageKind { ST_F32 = 0, ST_F16 = 1, ST_BF16 = 2 };

template <int S> struct Store;
template <> struct Store<ST_F32> {
    using T = float;
    static __device__ __forceinline__ float ld(const float *p) { return *p; }
    static __device__ __forceinline__ void st(float *p, float v) { *p = v; }
};
template <> struct Store<ST_F16> {
    using T = __half;
    static __device__ __forceinline__ float ld(const __half *p) { return __half2float(*p); }
    static __device__ __forceinline__ void st(__half *p, float v) { *p = __float2half_rn(v); }
};
template <> struct Store<ST_BF16> {
    using T = __nv_bfloat16;
    static __device__ __forceinline__ float ld(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
    static __device__ __forceinline__ void st(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
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
};

__device__ __forceinline__ uint32_t fast_div(uint32_t a, uint64_t mag) {
    return static_cast<uint32_t>(__umul64hi(static_cast<uint64_t>(a), mag));
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

// Moments of one node: mom = (rho - rho0, u, v, w, T) with
// u = (sum e f + F/2)/rho and F = body force + rho g beta T z-hat (Sec. 2.2).
struct Macro {
    float drho, rho, u, v, w, T, Fx, Fy, Fz;
};

__device__ __forceinline__ Macro macro(const Phys &P, const float (&f)[19], const float (&g)[7]) {
    Macro m;
    float dr = 0.f, jx = 0.f, jy = 0.f, jz = 0.f, T = 0.f;
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        dr += f[i];
        acc_int(jx, ex19(i), f[i]);
        acc_int(jy, ey19(i), f[i]);
        acc_int(jz, ez19(i), f[i]);
    }
#pragma unroll
    for (int i = 0; i < 7; ++i) T += g[i];
    const float rho = 1.0f + dr;
    m.drho = dr;
    m.rho = rho;
    m.T = T;
    m.Fx = P.bf[0];
    m.Fy = P.bf[1];
    m.Fz = fmaf(rho * P.gbeta, T, P.bf[2]);
    const float inv = 1.0f / rho;
    m.u = fmaf(0.5f, m.Fx, jx) * inv;
    m.v = fmaf(0.5f, m.Fy, jy) * inv;
    m.w = fmaf(0.5f, m.Fz, jz) * inv;
    return m;
}

// One fused collision of both distributions at one node, in place:
//   f+ = f - M^-1 [S (m - m^eq) - (I - S/2) M F~]      (Eq. MRT)
//   g+ = g - N^-1 Q (n - n^eq)                          (Eq. MRT_T)
// f holds deviations f - w rho0; the rest-state moments M w rho0 =
// (rho0, -11 rho0, 3 rho0, 0, ...) are folded into m - m^eq below.
__device__ __forceinline__ Macro collide(const Phys &P, float (&f)[19], float (&g)[7]) {
    const Macro mc = macro(P, f, g);
    const float rho = mc.rho, u = mc.u, v = mc.v, w = mc.w, T = mc.T;
    const float Fx = mc.Fx, Fy = mc.Fy, Fz = mc.Fz;

    // non-conserved moments of the deviations
    float m[19];
#pragma unroll
    for (int k = 0; k < 19; ++k) {
        m[k] = 0.f;
        if (k == 0 || k == 3 || k == 5 || k == 7) continue;
#pragma unroll
        for (int i = 0; i < 19; ++i) acc_int(m[k], Mk(k, i), f[i]);
    }
    const float uu = u * u + v * v + w * w;
    const float ru = rho * u, rv = rho * v, rw = rho * w;
    const float pxx = rho * (2.f * u * u - v * v - w * w);
    const float pww = rho * (v * v - w * w);
    // m - m^eq in deviation form (Sec. 2.2 m^eq)
    float d[19];
    d[1] = m[1] + 11.f * mc.drho - 19.f * rho * uu;
    d[2] = m[2] - 3.f * mc.drho + 5.5f * rho * uu;
    d[4] = m[4] + (2.f / 3.f) * ru;
    d[6] = m[6] + (2.f / 3.f) * rv;
    d[8] = m[8] + (2.f / 3.f) * rw;
    d[9] = m[9] - pxx;
    d[10] = m[10] + 0.5f * pxx;
    d[11] = m[11] - pww;
    d[12] = m[12] + 0.5f * pww;
    d[13] = m[13] - ru * v;
    d[14] = m[14] - rv * w;
    d[15] = m[15] - ru * w;
    d[16] = m[16];
    d[17] = m[17];
    d[18] = m[18];
    // forcing moments M F~ (Sec. 2.2)
    const float uF = u * Fx + v * Fy + w * Fz;
    const float ce = 1.f - 0.5f * P.s_e, cq = 1.f - 0.5f * P.s_q;
    float D[19]; // S (m - m^eq) - (I - S/2) M F~, divided by |M_k|^2
    D[0] = 0.f;
    D[1] = (P.s_e * d[1] - ce * 38.f * uF) * (1.f / Mnorm(1));
    D[2] = (P.s_e * d[2] + ce * 11.f * uF) * (1.f / Mnorm(2));
    D[3] = -Fx * (1.f / Mnorm(3));
    D[4] = (P.s_q * d[4] + cq * (2.f / 3.f) * Fx) * (1.f / Mnorm(4));
    D[5] = -Fy * (1.f / Mnorm(5));
    D[6] = (P.s_q * d[6] + cq * (2.f / 3.f) * Fy) * (1.f / Mnorm(6));
    D[7] = -Fz * (1.f / Mnorm(7));
    D[8] = (P.s_q * d[8] + cq * (2.f / 3.f) * Fz) * (1.f / Mnorm(8));
    D[9] = (P.s_e * d[9] - ce * (4.f * u * Fx - 2.f * v * Fy - 2.f * w * Fz)) * (1.f / Mnorm(9));
    D[10] = (P.s_e * d[10] - ce * (-2.f * u * Fx + v * Fy + w * Fz)) * (1.f / Mnorm(10));
    D[11] = (P.s_e * d[11] - ce * (2.f * v * Fy - 2.f * w * Fz)) * (1.f / Mnorm(11));
    D[12] = (P.s_e * d[12] - ce * (-v * Fy + w * Fz)) * (1.f / Mnorm(12));
    D[13] = (P.s_e * d[13] - ce * (u * Fy + v * Fx)) * (1.f / Mnorm(13));
    D[14] = (P.s_e * d[14] - ce * (v * Fz + w * Fy)) * (1.f / Mnorm(14));
    D[15] = (P.s_e * d[15] - ce * (u * Fz + w * Fx)) * (1.f / Mnorm(15));
    D[16] = P.s_q * d[16] * (1.f / Mnorm(16));
    D[17] = P.s_q * d[17] * (1.f / Mnorm(17));
    D[18] = P.s_q * d[18] * (1.f / Mnorm(18));
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        float c = 0.f;
#pragma unroll
        for (int k = 1; k < 19; ++k) acc_int(c, Mk(k, i), D[k]);
        f[i] -= c;
    }

    // D3Q7: n - n^eq with n^eq = (T, uT, vT, wT, a_T T, 0, 0)
    float n[7];
#pragma unroll
    for (int k = 1; k < 7; ++k) {
        n[k] = 0.f;
#pragma unroll
        for (int i = 0; i < 7; ++i) acc_int(n[k], Nk(k, i), g[i]);
    }
    float E[7];
    E[0] = 0.f;
    E[1] = P.q_k * (n[1] - u * T) * (1.f / Nnorm(1));
    E[2] = P.q_k * (n[2] - v * T) * (1.f / Nnorm(2));
    E[3] = P.q_k * (n[3] - w * T) * (1.f / Nnorm(3));
    E[4] = P.q_e * (n[4] - P.a_T * T) * (1.f / Nnorm(4));
    E[5] = P.q_e * n[5] * (1.f / Nnorm(5));
    E[6] = P.q_e * n[6] * (1.f / Nnorm(6));
#pragma unroll
    for (int i = 0; i < 7; ++i) {
        float c = 0.f;
#pragma unroll
        for (int k = 1; k < 7; ++k) acc_int(c, Nk(k, i), E[k]);
        g[i] -= c;
    }
    return mc;
}

} // namespace lbm
