/*
 * FP64 CPU oracle for the thermal lattice Boltzmann step of Xu, Shi & Xi,
 * "Lattice Boltzmann simulations of three-dimensional thermal convective flows
 * at high Rayleigh number" (arXiv:1903.08882).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant with the CUDA library: every table below is built
 * here from the paper's definitions.
 *
 * It is written to be read against the paper, not to be fast:
 *   - lattice D3Q19 velocities e_0..e_18 in the paper's order (Sec. 2.2);
 *   - M built from its moment polynomials <1|, <19e^2-30|, ... (Sec. 2.2),
 *     M^-1 = M^T diag(1/|M_k|^2) because the rows are orthogonal;
 *   - equilibrium moments m^eq and forcing moments M F~ exactly as printed
 *     (Sec. 2.2), S = diag(s_rho, s_e, ...) with the paper's rate choice;
 *   - D3Q7 with N built from its moment polynomials (Sec. 2.3).  The printed
 *     row <e_z| carries a sign typo; the definition e_5 = +z, e_6 = -z is used;
 *   - thermal rates q_kappa = 3 - sqrt(3), q_e = q_nu = 4 sqrt(3) - 6,
 *     a_T = 42 sqrt(3) kappa - 6 (Sec. 2.3, Eq. qk / Eq. qnu);
 *   - half-way bounce-back for the flow (Sec. 2.2), half-way anti-bounce-back
 *     for Dirichlet temperature walls and half-way bounce-back for adiabatic
 *     walls (Sec. 2.3);
 *   - two buffers and pull streaming.
 *
 * Parity status: every function here is pinned by the CPU test suite
 * (rest state, conservation, conduction, Fourier-mode decay, Poiseuille flow,
 * BGK/TRT special cases, printed tables, symmetry, the onset of convection at
 * the exact critical Rayleigh number, and closed-form diagnostics including
 * the per-node dissipation rates).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define Q19 19
#define Q7 7
#define ORC_NDIAG 24

enum { ORC_ADIABATIC = 0, ORC_DIRICHLET = 1, ORC_PERIODIC = 2 };

/* Faces are ordered -x, +x, -y, +y, -z, +z.  Gravity points along -z, so the
 * buoyancy force F = rho g beta (T - T0) z-hat points along +z (Eq. NS). */
typedef struct {
    int nx, ny, nz;
    int wall_kind[6];
    double wall_T[6];
    double nu, kappa, gbeta;
    double body_force[3]; /* constant force density added to the buoyancy force */
    double rho0, T0;
    double a_T;
    double s[Q19]; /* D3Q19 relaxation rates, moment order of M */
    double q[Q7];  /* D3Q7 relaxation rates, moment order of N */
} orc_params;

/* D3Q19 velocities, paper order (Sec. 2.2, the e_i matrix). */
static const int E19[Q19][3] = {
    {0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},   {0, -1, 0},
    {0, 0, 1},  {0, 0, -1}, {1, 1, 0},  {-1, 1, 0},  {1, -1, 0},
    {-1, -1, 0}, {1, 0, 1}, {-1, 0, 1}, {1, 0, -1},  {-1, 0, -1},
    {0, 1, 1},  {0, -1, 1}, {0, 1, -1}, {0, -1, -1}};
/* D3Q7 velocities, paper order (Sec. 2.3). */
static const int E7[Q7][3] = {{0, 0, 0}, {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},
                              {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};

static double M[Q19][Q19], Minv[Q19][Q19], W19[Q19];
static double N7[Q7][Q7], Ninv[Q7][Q7];
static int OPP19[Q19], OPP7[Q7];

/* Row k of M evaluated at velocity e: the moment polynomials of Sec. 2.2. */
static double m_poly(int k, const int *e) {
    double ex = e[0], ey = e[1], ez = e[2];
    double e2 = ex * ex + ey * ey + ez * ez;
    switch (k) {
    case 0: return 1.0;
    case 1: return 19.0 * e2 - 30.0;
    case 2: return 21.0 / 2.0 * e2 * e2 - 53.0 / 2.0 * e2 + 12.0;
    case 3: return ex;
    case 4: return (5.0 * e2 - 9.0) * ex;
    case 5: return ey;
    case 6: return (5.0 * e2 - 9.0) * ey;
    case 7: return ez;
    case 8: return (5.0 * e2 - 9.0) * ez;
    case 9: return 3.0 * ex * ex - e2;
    case 10: return (3.0 * e2 - 5.0) * (3.0 * ex * ex - e2);
    case 11: return ey * ey - ez * ez;
    case 12: return (3.0 * e2 - 5.0) * (ey * ey - ez * ez);
    case 13: return ex * ey;
    case 14: return ey * ez;
    case 15: return ex * ez;
    case 16: return (ey * ey - ez * ez) * ex;
    case 17: return (ez * ez - ex * ex) * ey;
    case 18: return (ex * ex - ey * ey) * ez;
    }
    return 0.0;
}

/* Row k of N evaluated at velocity e: the moment polynomials of Sec. 2.3. */
static double n_poly(int k, const int *e) {
    double ex = e[0], ey = e[1], ez = e[2];
    double e2 = ex * ex + ey * ey + ez * ez;
    switch (k) {
    case 0: return 1.0;
    case 1: return ex;
    case 2: return ey;
    case 3: return ez;
    case 4: return -6.0 + 7.0 * e2;
    case 5: return 3.0 * ex * ex - e2;
    case 6: return ey * ey - ez * ez;
    }
    return 0.0;
}

static void build_tables(void) {
    for (int k = 0; k < Q19; ++k)
        for (int i = 0; i < Q19; ++i) M[k][i] = m_poly(k, E19[i]);
    for (int k = 0; k < Q19; ++k) {
        double n2 = 0.0;
        for (int i = 0; i < Q19; ++i) n2 += M[k][i] * M[k][i];
        for (int i = 0; i < Q19; ++i) Minv[i][k] = M[k][i] / n2;
    }
    for (int i = 0; i < Q19; ++i) {
        int e2 = E19[i][0] * E19[i][0] + E19[i][1] * E19[i][1] + E19[i][2] * E19[i][2];
        W19[i] = e2 == 0 ? 1.0 / 3.0 : (e2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
        for (int j = 0; j < Q19; ++j)
            if (E19[j][0] == -E19[i][0] && E19[j][1] == -E19[i][1] && E19[j][2] == -E19[i][2])
                OPP19[i] = j;
    }
    for (int k = 0; k < Q7; ++k)
        for (int i = 0; i < Q7; ++i) N7[k][i] = n_poly(k, E7[i]);
    for (int k = 0; k < Q7; ++k) {
        double n2 = 0.0;
        for (int i = 0; i < Q7; ++i) n2 += N7[k][i] * N7[k][i];
        for (int i = 0; i < Q7; ++i) Ninv[i][k] = N7[k][i] / n2;
    }
    for (int i = 0; i < Q7; ++i)
        for (int j = 0; j < Q7; ++j)
            if (E7[j][0] == -E7[i][0] && E7[j][1] == -E7[i][1] && E7[j][2] == -E7[i][2])
                OPP7[i] = j;
}

__attribute__((constructor)) static void orc_init_tables(void) { build_tables(); }

/* ---------------------------------------------------------------- tables -- */

void orc_tables(double *e19, double *w19, double *m, double *minv, int *opp19,
                double *e7, double *n7, double *ninv, int *opp7) {
    for (int i = 0; i < Q19; ++i) {
        for (int a = 0; a < 3; ++a) e19[3 * i + a] = E19[i][a];
        w19[i] = W19[i];
        opp19[i] = OPP19[i];
    }
    for (int k = 0; k < Q19; ++k)
        for (int i = 0; i < Q19; ++i) {
            m[k * Q19 + i] = M[k][i];
            minv[i * Q19 + k] = Minv[i][k];
        }
    for (int i = 0; i < Q7; ++i) {
        for (int a = 0; a < 3; ++a) e7[3 * i + a] = E7[i][a];
        opp7[i] = OPP7[i];
    }
    for (int k = 0; k < Q7; ++k)
        for (int i = 0; i < Q7; ++i) {
            n7[k * Q7 + i] = N7[k][i];
            ninv[i * Q7 + k] = Ninv[i][k];
        }
}

/* D3Q7 weights: w_0 = (1 - a_T)/7, w_1..6 = (6 + a_T)/42 (Sec. 2.3). */
static double w7(const orc_params *p, int i) {
    return i == 0 ? (1.0 - p->a_T) / 7.0 : (6.0 + p->a_T) / 42.0;
}

/* --------------------------------------------------------- parameters -- */

/* Free-fall scaling (Sec. 2.1): with cell height H, free-fall velocity U,
 * Ra = g beta dT H^3/(nu kappa) and Pr = nu/kappa, dT = 1:
 *   nu = U H sqrt(Pr/Ra), kappa = nu/Pr, g beta = U^2/H. */
void orc_free_fall(double H, double Ra, double Pr, double U, double *nu, double *kappa,
                   double *gbeta) {
    *nu = U * H * sqrt(Pr / Ra);
    *kappa = *nu / Pr;
    *gbeta = U * U / H;
}

/* Relaxation rates from nu and kappa.
 * Flow (Sec. 2.2): nu = c_s^2 (tau_f - 1/2), c_s^2 = 1/3;
 *   s_rho = s_j = 0, s_e = s_eps = s_nu = s_pi = 1/tau_f,
 *   s_q = s_m = 8 (2 tau_f - 1)/(8 tau_f - 1).
 * Heat (Sec. 2.3): q_kappa = 3 - sqrt(3), q_e = q_nu = 4 sqrt(3) - 6,
 *   a_T = 42 sqrt(3) kappa - 6, Q = diag(0, q_k, q_k, q_k, q_e, q_nu, q_nu).
 * Returns 0, or 1 if tau_f <= 1/2 or a_T is outside (-6, 1). */
int orc_set_rates(orc_params *p) {
    double tau = p->nu / (1.0 / 3.0) + 0.5;
    double se = 1.0 / tau, sq = 8.0 * (2.0 * tau - 1.0) / (8.0 * tau - 1.0);
    /* order: rho, e, eps, jx, qx, jy, qy, jz, qz, 3pxx, 3pixx, pww, piww,
     *        pxy, pyz, pxz, mx, my, mz */
    const double s[Q19] = {0.0, se, se, 0.0, sq, 0.0, sq, 0.0, sq, se,
                           se,  se, se, se,  se, se,  sq, sq,  sq};
    memcpy(p->s, s, sizeof(s));
    double qk = 3.0 - sqrt(3.0), qe = 4.0 * sqrt(3.0) - 6.0;
    const double q[Q7] = {0.0, qk, qk, qk, qe, qe, qe};
    memcpy(p->q, q, sizeof(q));
    p->a_T = 42.0 * sqrt(3.0) * p->kappa - 6.0;
    if (!(tau > 0.5)) return 1;
    if (!(p->a_T > -6.0 && p->a_T < 1.0)) return 1;
    return 0;
}

/* ------------------------------------------------------------ node ops -- */

/* Force at a node: F = rho g beta (T - T0) z-hat (Sec. 2.2) plus the constant
 * body force density. */
static void node_force(const orc_params *p, double rho, double T, double F[3]) {
    F[0] = p->body_force[0];
    F[1] = p->body_force[1];
    F[2] = p->body_force[2] + rho * p->gbeta * (T - p->T0);
}

/* rho = sum f, T = sum g, u = (sum e f + F/2)/rho (Sec. 2.2, 2.3). */
static void node_moments(const orc_params *p, const double *f, const double *g, double *rho,
                         double u[3], double *T, double F[3]) {
    double r = 0.0, t = 0.0, j[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < Q19; ++i) {
        r += f[i];
        for (int a = 0; a < 3; ++a) j[a] += E19[i][a] * f[i];
    }
    for (int i = 0; i < Q7; ++i) t += g[i];
    node_force(p, r, t, F);
    for (int a = 0; a < 3; ++a) u[a] = (j[a] + 0.5 * F[a]) / r;
    *rho = r;
    *T = t;
}

/* Equilibrium moments m^eq (Sec. 2.2), as printed. */
static void meq_moments(double rho, const double u3[3], double meq[Q19]) {
    double u = u3[0], v = u3[1], w = u3[2], uu = u * u + v * v + w * w;
    meq[0] = rho;
    meq[1] = rho * (-11.0 + 19.0 * uu);
    meq[2] = rho * (3.0 - 11.0 / 2.0 * uu);
    meq[3] = rho * u;
    meq[4] = rho * (-2.0 / 3.0 * u);
    meq[5] = rho * v;
    meq[6] = rho * (-2.0 / 3.0 * v);
    meq[7] = rho * w;
    meq[8] = rho * (-2.0 / 3.0 * w);
    meq[9] = rho * (2.0 * u * u - v * v - w * w);
    meq[10] = rho * (-0.5 * (2.0 * u * u - v * v - w * w));
    meq[11] = rho * (v * v - w * w);
    meq[12] = rho * (-0.5 * (v * v - w * w));
    meq[13] = rho * u * v;
    meq[14] = rho * v * w;
    meq[15] = rho * u * w;
    meq[16] = 0.0;
    meq[17] = 0.0;
    meq[18] = 0.0;
}

/* Forcing moments M F~ (Sec. 2.2), as printed. */
static void mf_moments(const double u3[3], const double F[3], double mf[Q19]) {
    double u = u3[0], v = u3[1], w = u3[2];
    double Fx = F[0], Fy = F[1], Fz = F[2];
    double uF = u * Fx + v * Fy + w * Fz;
    mf[0] = 0.0;
    mf[1] = 38.0 * uF;
    mf[2] = -11.0 * uF;
    mf[3] = Fx;
    mf[4] = -2.0 / 3.0 * Fx;
    mf[5] = Fy;
    mf[6] = -2.0 / 3.0 * Fy;
    mf[7] = Fz;
    mf[8] = -2.0 / 3.0 * Fz;
    mf[9] = 4.0 * u * Fx - 2.0 * v * Fy - 2.0 * w * Fz;
    mf[10] = -2.0 * u * Fx + v * Fy + w * Fz;
    mf[11] = 2.0 * v * Fy - 2.0 * w * Fz;
    mf[12] = -v * Fy + w * Fz;
    mf[13] = u * Fy + v * Fx;
    mf[14] = v * Fz + w * Fy;
    mf[15] = u * Fz + w * Fx;
    mf[16] = 0.0;
    mf[17] = 0.0;
    mf[18] = 0.0;
}

/* One collision at one node: the right-hand sides of Eq. MRT and Eq. MRT_T.
 *   f+ = f - M^-1 S (m - m^eq) + M^-1 (I - S/2) M F~
 *   g+ = g - N^-1 Q (n - n^eq),  n^eq = [T, uT, vT, wT, a_T T, 0, 0]
 * mom (optional) receives rho, u, v, w, T of this node. */
void orc_collide(const orc_params *p, const double *f, const double *g, double *fout,
                 double *gout, double *mom) {
    double rho, u[3], T, F[3];
    node_moments(p, f, g, &rho, u, &T, F);
    double m[Q19], meq[Q19], mf[Q19], d[Q19];
    for (int k = 0; k < Q19; ++k) {
        m[k] = 0.0;
        for (int i = 0; i < Q19; ++i) m[k] += M[k][i] * f[i];
    }
    meq_moments(rho, u, meq);
    mf_moments(u, F, mf);
    for (int k = 0; k < Q19; ++k)
        d[k] = p->s[k] * (m[k] - meq[k]) - (1.0 - 0.5 * p->s[k]) * mf[k];
    for (int i = 0; i < Q19; ++i) {
        double acc = 0.0;
        for (int k = 0; k < Q19; ++k) acc += Minv[i][k] * d[k];
        fout[i] = f[i] - acc;
    }
    double n[Q7], neq[Q7], dn[Q7];
    for (int k = 0; k < Q7; ++k) {
        n[k] = 0.0;
        for (int i = 0; i < Q7; ++i) n[k] += N7[k][i] * g[i];
    }
    neq[0] = T;
    neq[1] = u[0] * T;
    neq[2] = u[1] * T;
    neq[3] = u[2] * T;
    neq[4] = p->a_T * T;
    neq[5] = 0.0;
    neq[6] = 0.0;
    for (int k = 0; k < Q7; ++k) dn[k] = p->q[k] * (n[k] - neq[k]);
    for (int i = 0; i < Q7; ++i) {
        double acc = 0.0;
        for (int k = 0; k < Q7; ++k) acc += Ninv[i][k] * dn[k];
        gout[i] = g[i] - acc;
    }
    if (mom) {
        mom[0] = rho;
        mom[1] = u[0];
        mom[2] = u[1];
        mom[3] = u[2];
        mom[4] = T;
    }
}

/* f^eq_i = w_i rho [1 + e.u/cs^2 + (e.u)^2/(2 cs^4) - |u|^2/(2 cs^2)] (Sec. 2.2)
 * g^eq_i = w_i T [1 + 7/(6 + a_T) e.u/cs^2]                      (Sec. 2.3) */
void orc_equilibrium(const orc_params *p, double rho, const double *u, double T, double *feq,
                     double *geq) {
    const double cs2 = 1.0 / 3.0;
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < Q19; ++i) {
        double eu = E19[i][0] * u[0] + E19[i][1] * u[1] + E19[i][2] * u[2];
        feq[i] = W19[i] * rho * (1.0 + eu / cs2 + eu * eu / (2.0 * cs2 * cs2) - uu / (2.0 * cs2));
    }
    for (int i = 0; i < Q7; ++i) {
        double eu = E7[i][0] * u[0] + E7[i][1] * u[1] + E7[i][2] * u[2];
        geq[i] = w7(p, i) * T * (1.0 + 7.0 / (6.0 + p->a_T) * eu / cs2);
    }
}

/* Equilibrium M F~ and m^eq exported for the table tests. */
void orc_meq(double rho, const double *u, double *meq) { meq_moments(rho, u, meq); }
void orc_mf(const double *u, const double *F, double *mf) { mf_moments(u, F, mf); }

/* ------------------------------------------------------- whole lattice -- */

/* Arrays are component-major, x fastest: a[c][z][y][x]. */
static inline int64_t nidx(int nx, int ny, int x, int y, int z) {
    return (int64_t)x + (int64_t)nx * ((int64_t)y + (int64_t)ny * z);
}

/* Equilibrium populations from host fields rho, u (3 x n), T. */
void orc_init_equilibrium(const orc_params *p, const double *rho, const double *u3,
                          const double *T, double *f, double *g) {
    int64_t n = (int64_t)p->nx * p->ny * p->nz;
    for (int64_t c = 0; c < n; ++c) {
        double u[3] = {u3[c], u3[n + c], u3[2 * n + c]}, fe[Q19], ge[Q7];
        orc_equilibrium(p, rho[c], u, T[c], fe, ge);
        for (int i = 0; i < Q19; ++i) f[i * n + c] = fe[i];
        for (int i = 0; i < Q7; ++i) g[i * n + c] = ge[i];
    }
}

/* Moments of the (pre-collision) populations: rho, u (3 x n), T. */
void orc_moments(const orc_params *p, const double *f, const double *g, double *rho,
                 double *u3, double *T) {
    int64_t n = (int64_t)p->nx * p->ny * p->nz;
    for (int64_t c = 0; c < n; ++c) {
        double fl[Q19], gl[Q7], r, u[3], t, F[3];
        for (int i = 0; i < Q19; ++i) fl[i] = f[i * n + c];
        for (int i = 0; i < Q7; ++i) gl[i] = g[i * n + c];
        node_moments(p, fl, gl, &r, u, &t, F);
        rho[c] = r;
        for (int a = 0; a < 3; ++a) u3[a * n + c] = u[a];
        T[c] = t;
    }
}

/* Where does the population arriving at global node (x,y,z) along velocity e
 * come from?  Returns 1 with the (wrapped) source node when the source lies in
 * the lattice, or 0 with the face the link crosses when it comes off a wall. */
static int pull_source(const orc_params *p, const int g[3], const int *e, int src[3],
                       int *face) {
    const int n[3] = {p->nx, p->ny, p->nz};
    int inside = 1;
    *face = -1;
    for (int a = 0; a < 3; ++a) {
        int s = g[a] - e[a];
        if (s < 0 || s >= n[a]) {
            int fc = 2 * a + (s < 0 ? 0 : 1);
            if (p->wall_kind[fc] == ORC_PERIODIC) {
                s = (s + n[a]) % n[a];
            } else {
                inside = 0;
                *face = fc;
            }
        }
        src[a] = s;
    }
    return inside;
}

/* One time step on a box of the lattice.
 *
 * The box starts at global node `org` and has `dim` nodes per axis; f, g hold
 * its pre-collision populations, f_out, g_out receive those of the next step.
 * With org = 0 and dim = (nx, ny, nz) this is the ordinary whole-lattice step.
 * For a smaller box, a node whose pull source lies in the lattice but outside
 * the box gets NaN (its result needs data the box does not hold).
 *
 * Order: collide every node (Eq. MRT, Eq. MRT_T right-hand sides), then pull:
 *   f_i(x, t+1) = f_i+(x - e_i), or f_ibar+(x) when the link comes off a wall
 *     (half-way bounce-back, Sec. 2.2);
 *   g_i(x, t+1) = g_i+(x - e_i), or g_ibar+(x) at an adiabatic wall, or
 *     -g_ibar+(x) + (6 + a_T)/21 T_w at a Dirichlet wall (Sec. 2.3). */
void orc_step_box(const orc_params *p, const int *org, const int *dim, const double *f,
                  const double *g, double *f_out, double *g_out) {
    int64_t nb = (int64_t)dim[0] * dim[1] * dim[2];
    double *fp = (double *)malloc(sizeof(double) * Q19 * nb);
    double *gp = (double *)malloc(sizeof(double) * Q7 * nb);
#pragma omp parallel for schedule(static)
    for (int z = 0; z < dim[2]; ++z)
        for (int y = 0; y < dim[1]; ++y)
            for (int x = 0; x < dim[0]; ++x) {
                int64_t c = nidx(dim[0], dim[1], x, y, z);
                double fl[Q19], gl[Q7], fo[Q19], go[Q7];
                for (int i = 0; i < Q19; ++i) fl[i] = f[i * nb + c];
                for (int i = 0; i < Q7; ++i) gl[i] = g[i * nb + c];
                orc_collide(p, fl, gl, fo, go, NULL);
                for (int i = 0; i < Q19; ++i) fp[i * nb + c] = fo[i];
                for (int i = 0; i < Q7; ++i) gp[i * nb + c] = go[i];
            }
    const double w_abb = (6.0 + p->a_T) / 21.0;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < dim[2]; ++z)
        for (int y = 0; y < dim[1]; ++y)
            for (int x = 0; x < dim[0]; ++x) {
                int64_t c = nidx(dim[0], dim[1], x, y, z);
                int gx[3] = {org[0] + x, org[1] + y, org[2] + z}, src[3], face;
                for (int i = 0; i < Q19; ++i) {
                    double v;
                    if (pull_source(p, gx, E19[i], src, &face)) {
                        int l[3] = {src[0] - org[0], src[1] - org[1], src[2] - org[2]};
                        if (l[0] < 0 || l[1] < 0 || l[2] < 0 || l[0] >= dim[0] ||
                            l[1] >= dim[1] || l[2] >= dim[2])
                            v = NAN;
                        else
                            v = fp[i * nb + nidx(dim[0], dim[1], l[0], l[1], l[2])];
                    } else {
                        v = fp[OPP19[i] * nb + c];
                    }
                    f_out[i * nb + c] = v;
                }
                for (int i = 0; i < Q7; ++i) {
                    double v;
                    if (pull_source(p, gx, E7[i], src, &face)) {
                        int l[3] = {src[0] - org[0], src[1] - org[1], src[2] - org[2]};
                        if (l[0] < 0 || l[1] < 0 || l[2] < 0 || l[0] >= dim[0] ||
                            l[1] >= dim[1] || l[2] >= dim[2])
                            v = NAN;
                        else
                            v = gp[i * nb + nidx(dim[0], dim[1], l[0], l[1], l[2])];
                    } else if (p->wall_kind[face] == ORC_DIRICHLET) {
                        v = -gp[OPP7[i] * nb + c] + w_abb * p->wall_T[face];
                    } else {
                        v = gp[OPP7[i] * nb + c];
                    }
                    g_out[i * nb + c] = v;
                }
            }
    free(fp);
    free(gp);
}

/* nsteps whole-lattice steps, in place. */
void orc_run(const orc_params *p, double *f, double *g, int64_t nsteps) {
    int64_t n = (int64_t)p->nx * p->ny * p->nz;
    const int org[3] = {0, 0, 0}, dim[3] = {p->nx, p->ny, p->nz};
    double *f2 = (double *)malloc(sizeof(double) * Q19 * n);
    double *g2 = (double *)malloc(sizeof(double) * Q7 * n);
    for (int64_t t = 0; t < nsteps; ++t) {
        orc_step_box(p, org, dim, f, g, f2, g2);
        memcpy(f, f2, sizeof(double) * Q19 * n);
        memcpy(g, g2, sizeof(double) * Q7 * n);
    }
    free(f2);
    free(g2);
}

/* ---------------------------------------------------------- diagnostics -- */

/* Derivative along axis a of a node field phi at node (x,y,z) (lattice units).
 * Interior or periodic: second-order central difference.
 * Next to a wall whose side is flagged in has_value (no-slip velocity,
 * Dirichlet T), with the wall value phi_w:
 *   second-order one-sided difference through the wall point (distance 1/2)
 *   and the two nearest nodes, d/ds at the node = -4/3 phi_w + phi_0 + 1/3 phi_1.
 * Next to a wall with zero normal gradient (adiabatic T): (phi_1 - phi_0)/2,
 *   the same difference a mirrored ghost node gives. */
static double ddx(const orc_params *p, const double *phi, int a, int x, int y, int z,
                  const int *has_value, const double *wall_value) {
    const int n[3] = {p->nx, p->ny, p->nz};
    int c[3] = {x, y, z};
    int lo = c[a] - 1, hi = c[a] + 1;
    int lo_wall = 0, hi_wall = 0;
    if (lo < 0) {
        if (p->wall_kind[2 * a] == ORC_PERIODIC) lo += n[a];
        else lo_wall = 1;
    }
    if (hi >= n[a]) {
        if (p->wall_kind[2 * a + 1] == ORC_PERIODIC) hi -= n[a];
        else hi_wall = 1;
    }
    int cl[3] = {x, y, z}, ch[3] = {x, y, z};
    cl[a] = lo;
    ch[a] = hi;
    double p0 = phi[nidx(p->nx, p->ny, x, y, z)];
    if (!lo_wall && !hi_wall) {
        return 0.5 * (phi[nidx(p->nx, p->ny, ch[0], ch[1], ch[2])] -
                      phi[nidx(p->nx, p->ny, cl[0], cl[1], cl[2])]);
    }
    if (lo_wall && hi_wall) return 0.0; /* a single node across: undefined, report 0 */
    if (lo_wall) {
        double p1 = phi[nidx(p->nx, p->ny, ch[0], ch[1], ch[2])];
        if (has_value[2 * a]) return -4.0 / 3.0 * wall_value[2 * a] + p0 + p1 / 3.0;
        return 0.5 * (p1 - p0);
    }
    double p1 = phi[nidx(p->nx, p->ny, cl[0], cl[1], cl[2])];
    if (has_value[2 * a + 1]) return 4.0 / 3.0 * wall_value[2 * a + 1] - p0 - p1 / 3.0;
    return 0.5 * (p0 - p1);
}

/* Local energy dissipation rates of a pre-collision state, per node (Sec. 4,
 * the fields whose probability densities the paper reports):
 *   eps_u = nu/2 sum_ij (d_i u_j + d_j u_i)^2,   eps_T = kappa |grad T|^2,
 * with the derivative stencils of orc_diagnostics (central inside; one-sided
 * through the wall value next to a no-slip or Dirichlet wall; zero-gradient
 * next to an adiabatic wall).  Arrays of nx ny nz doubles, x fastest. */
void orc_local_dissipation(const orc_params *p, const double *f, const double *g, double *eps_u,
                           double *eps_T) {
    const int nx = p->nx, ny = p->ny, nz = p->nz;
    int64_t n = (int64_t)nx * ny * nz;
    double *rho = (double *)malloc(sizeof(double) * n);
    double *u3 = (double *)malloc(sizeof(double) * 3 * n);
    double *T = (double *)malloc(sizeof(double) * n);
    orc_moments(p, f, g, rho, u3, T);
    const double zero_wall[6] = {0, 0, 0, 0, 0, 0};
    const int all_walls[6] = {1, 1, 1, 1, 1, 1};
    double Tw[6];
    int t_has_value[6];
    for (int fc = 0; fc < 6; ++fc) {
        Tw[fc] = p->wall_T[fc];
        t_has_value[fc] = p->wall_kind[fc] == ORC_DIRICHLET;
    }
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                int64_t c = nidx(nx, ny, x, y, z);
                double du[3][3]; /* du[i][j] = d u_j / d x_i */
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j)
                        du[i][j] = ddx(p, u3 + j * n, i, x, y, z, all_walls, zero_wall);
                double e = 0.0, gg = 0.0;
                for (int i = 0; i < 3; ++i) {
                    for (int j = 0; j < 3; ++j) {
                        double sij = du[i][j] + du[j][i];
                        e += 0.5 * sij * sij;
                    }
                    double gi = ddx(p, T, i, x, y, z, t_has_value, Tw);
                    gg += gi * gi;
                }
                eps_u[c] = p->nu * e;
                eps_T[c] = p->kappa * gg;
            }
    free(rho);
    free(u3);
    free(T);
}

/* Raw diagnostic sums of a pre-collision state (all over the nx ny nz nodes):
 *  out[0]  node count
 *  out[1]  sum (rho - rho0)^2                     (rms density, Sec. 3)
 *  out[2]  sum |u|^2                              (E, Re^rms, Sec. 3 and 4)
 *  out[3]  sum w^2                                (Re_w^rms, Sec. 4)
 *  out[4]  sum w T                                (Nu_vol, Sec. 4)
 *  out[5]  sum 1/2 sum_ij (d_i u_j + d_j u_i)^2    (eps_u / nu, Sec. 4)
 *  out[6]  sum |grad T|^2                         (eps_T / kappa, Sec. 4)
 *  out[7]  sum (div u)^2                          (rms divergence, Sec. 3)
 *  out[8+f]  for each Dirichlet face f: sum over its nodes of -dT/dn at the
 *            wall, n pointing into the fluid, one-sided second order
 *            (-8 T_w + 9 T_0 - T_1)/3                (Nu_wall, Nu_overall)
 *  out[14] sum T, out[15] sum rho, out[16] max |u|
 *  out[17] non-finite node count
 *  out[18+f] for each Dirichlet face f: sum over its nodes of the heat the
 *            anti-bounce-back link carries into the fluid per step,
 *            2 g_in - (6 + a_T)/21 T_w (g_in: population arriving from the wall). */
void orc_diagnostics(const orc_params *p, const double *f, const double *g, double *out) {
    const int nx = p->nx, ny = p->ny, nz = p->nz;
    int64_t n = (int64_t)nx * ny * nz;
    double *rho = (double *)malloc(sizeof(double) * n);
    double *u3 = (double *)malloc(sizeof(double) * 3 * n);
    double *T = (double *)malloc(sizeof(double) * n);
    orc_moments(p, f, g, rho, u3, T);
    for (int k = 0; k < ORC_NDIAG; ++k) out[k] = 0.0;
    /* velocity: every non-periodic face is a no-slip wall with u = 0;
     * temperature: a Dirichlet face has the value T_w, an adiabatic one a zero
     * normal gradient */
    const double zero_wall[6] = {0, 0, 0, 0, 0, 0};
    const int all_walls[6] = {1, 1, 1, 1, 1, 1};
    double Tw[6];
    int t_has_value[6];
    for (int fc = 0; fc < 6; ++fc) {
        Tw[fc] = p->wall_T[fc];
        t_has_value[fc] = p->wall_kind[fc] == ORC_DIRICHLET;
    }
    out[0] = (double)n;
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                int64_t c = nidx(nx, ny, x, y, z);
                double u[3] = {u3[c], u3[n + c], u3[2 * n + c]};
                double du[3][3]; /* du[i][j] = d u_j / d x_i */
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j)
                        du[i][j] = ddx(p, u3 + j * n, i, x, y, z, all_walls, zero_wall);
                double gT[3];
                for (int i = 0; i < 3; ++i) gT[i] = ddx(p, T, i, x, y, z, t_has_value, Tw);
                double dr = rho[c] - p->rho0, uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
                double eps = 0.0;
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) {
                        double sij = du[i][j] + du[j][i];
                        eps += 0.5 * sij * sij;
                    }
                double divu = du[0][0] + du[1][1] + du[2][2];
                out[1] += dr * dr;
                out[2] += uu;
                out[3] += u[2] * u[2];
                out[4] += u[2] * T[c];
                out[5] += eps;
                out[6] += gT[0] * gT[0] + gT[1] * gT[1] + gT[2] * gT[2];
                out[7] += divu * divu;
                out[14] += T[c];
                out[15] += rho[c];
                double um = sqrt(uu);
                if (um > out[16]) out[16] = um;
                if (!isfinite(uu) || !isfinite(T[c]) || !isfinite(rho[c])) out[17] += 1.0;
            }
    /* Dirichlet wall fluxes. */
    const double w_abb = (6.0 + p->a_T) / 21.0;
    const int nn[3] = {nx, ny, nz};
    for (int fc = 0; fc < 6; ++fc) {
        if (p->wall_kind[fc] != ORC_DIRICHLET) continue;
        int a = fc / 2, hi = fc % 2;
        int b = (a + 1) % 3, cax = (a + 2) % 3;
        /* population index arriving from this wall: e along +a for the low face */
        int iin = -1;
        for (int i = 0; i < Q7; ++i)
            if (E7[i][a] == (hi ? -1 : 1)) iin = i;
        for (int jb = 0; jb < nn[b]; ++jb)
            for (int jc = 0; jc < nn[cax]; ++jc) {
                int c0[3], c1[3];
                c0[a] = hi ? nn[a] - 1 : 0;
                c1[a] = hi ? nn[a] - 2 : 1;
                c0[b] = c1[b] = jb;
                c0[cax] = c1[cax] = jc;
                int64_t i0 = nidx(nx, ny, c0[0], c0[1], c0[2]);
                int64_t i1 = nidx(nx, ny, c1[0], c1[1], c1[2]);
                double dTdn = (-8.0 * p->wall_T[fc] + 9.0 * T[i0] - T[i1]) / 3.0;
                out[8 + fc] += -dTdn;
                out[18 + fc] += 2.0 * g[iin * n + i0] - w_abb * p->wall_T[fc];
            }
    }
    free(rho);
    free(u3);
    free(T);
}

/* Nusselt numbers of Sec. 3 beyond the wall averages, of a pre-collision
 * state, in lattice units (free-fall velocity U, wall temperature difference
 * 1, length H).
 *
 * Plane-averaged profile along axis a (the x-z plane average Nu(y) of Fig. 4,
 * taken here along any axis): for every node plane j of axis a,
 *   out[j] = mean over the plane's nodes of (u_a T H / kappa - H dT/dx_a).
 * The paper's integrand v T sqrt(Ra Pr) - dT/dy becomes u_a T H / kappa
 * - H dT/dx_a with v = u_a / U, sqrt(Ra Pr) = U H / kappa and y = x_a / H;
 * dT/dx_a uses the stencils of orc_diagnostics (central inside, one-sided
 * through T_w next to a Dirichlet wall, zero-gradient next to an adiabatic
 * wall).
 *
 * Mid-line wall Nusselt numbers (Nu_mean of Sec. 3 and Table 2), out[n_a + f]
 * for faces f = 0..5: the mean of -H dT/dn at the wall (n into the fluid,
 * the one-sided stencil (-8 T_w + 9 T_0 - T_1)/3 of orc_diagnostics) over
 * the nodes next to face f on the line that runs along z (along x for the
 * two z faces) through the middle of the third axis.  When that axis has an
 * even number of nodes its middle lies between two node lines, and the mean
 * is taken over both (linear interpolation to the middle).  0 for a face
 * that is not a Dirichlet wall. */
void orc_nusselt_profile(const orc_params *p, const double *f, const double *g, int a, double H,
                         double *out) {
    const int nx = p->nx, ny = p->ny, nz = p->nz;
    const int nn[3] = {nx, ny, nz};
    int64_t n = (int64_t)nx * ny * nz;
    double *rho = (double *)malloc(sizeof(double) * n);
    double *u3 = (double *)malloc(sizeof(double) * 3 * n);
    double *T = (double *)malloc(sizeof(double) * n);
    orc_moments(p, f, g, rho, u3, T);
    double Tw[6];
    int t_has_value[6];
    for (int fc = 0; fc < 6; ++fc) {
        Tw[fc] = p->wall_T[fc];
        t_has_value[fc] = p->wall_kind[fc] == ORC_DIRICHLET;
    }
    for (int j = 0; j < nn[a]; ++j) out[j] = 0.0;
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const int c[3] = {x, y, z};
                int64_t i = nidx(nx, ny, x, y, z);
                double dT = ddx(p, T, a, x, y, z, t_has_value, Tw);
                out[c[a]] += u3[a * n + i] * T[i] * H / p->kappa - H * dT;
            }
    const double area = (double)n / nn[a];
    for (int j = 0; j < nn[a]; ++j) out[j] /= area;
    for (int fc = 0; fc < 6; ++fc) {
        double *o = out + nn[a] + fc;
        *o = 0.0;
        if (p->wall_kind[fc] != ORC_DIRICHLET) continue;
        const int b = fc / 2, hi = fc % 2;      /* normal axis */
        const int l = b == 2 ? 0 : 2;           /* the line's axis */
        const int m = 3 - b - l;                /* the axis whose middle the line passes through */
        const int m0 = (nn[m] - 1) / 2, m1 = nn[m] / 2;
        double sum = 0.0;
        int count = 0;
        for (int mm = m0; mm <= m1; ++mm)
            for (int k = 0; k < nn[l]; ++k) {
                int c0[3], c1[3];
                c0[b] = hi ? nn[b] - 1 : 0;
                c1[b] = hi ? nn[b] - 2 : 1;
                c0[l] = c1[l] = k;
                c0[m] = c1[m] = mm;
                const double T0 = T[nidx(nx, ny, c0[0], c0[1], c0[2])];
                const double T1 = T[nidx(nx, ny, c1[0], c1[1], c1[2])];
                sum += -H * (-8.0 * Tw[fc] + 9.0 * T0 - T1) / 3.0;
                count += 1;
            }
        *o = sum / count;
    }
    free(rho);
    free(u3);
    free(T);
}
