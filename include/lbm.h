/*
 * lbm.h - C ABI of the GB300 thermal lattice Boltzmann library.
 *
 * The library advances the double-distribution thermal lattice Boltzmann model
 * of Xu, Shi & Xi (arXiv:1903.08882) on one GPU:
 *   - a D3Q19 multiple-relaxation-time flow distribution f with Guo forcing
 *     and Boussinesq buoyancy F = rho g beta (T - T0) z-hat (Sec. 2.2, Eq. MRT);
 *   - a D3Q7 multiple-relaxation-time temperature distribution g whose rates
 *     make the fourth-order error isotropic (Sec. 2.3, Eq. MRT_T, Eq. magic,
 *     Eq. 4th, Eq. qk, Eq. qnu);
 *   - half-way bounce-back no-slip walls for f (Sec. 2.2), half-way
 *     anti-bounce-back Dirichlet walls and half-way bounce-back adiabatic walls
 *     for g (Sec. 2.3).
 *
 * Conventions shared by every entry point:
 *   - Lattice units, delta_x = delta_t = 1.  Node (x, y, z), 0 <= x < nx, sits
 *     at x + 1/2; the walls of a non-periodic axis lie at 0 and nx (half-way).
 *   - Faces are indexed 0..5 = -x, +x, -y, +y, -z, +z.  Gravity points along
 *     -z, so buoyancy pushes warm fluid along +z.
 *   - Host arrays are component-major with x fastest: a[c][z][y][x].  Velocity
 *     fields have 3 components (u, v, w); f has 19 and g has 7, in the
 *     paper's velocity order (e_0..e_18 of Sec. 2.2, e_0..e_6 of Sec. 2.3).
 *   - Populations exchanged with the host are absolute values in double
 *     precision.  Inside the library they are stored as deviations from the
 *     rest state, f_i - w_i rho0 and g_i - w_i T0 (rho0 = 1, T0 = 0), in FP32,
 *     FP16 or BF16; all arithmetic is FP32 and global sums are FP64.
 *   - Every function returns an lbm_status; nothing throws.  On failure
 *     lbm_last_error() holds a message.  Calls on one context must not overlap
 *     from several host threads.
 *   - lbm_step and lbm_set_* are asynchronous on the context's stream; the
 *     functions that return host data synchronise that stream.
 */
#ifndef LBM_GB300_H
#define LBM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LBM_OK = 0,
    LBM_ERR_PARAM = 1,    /* invalid argument or parameter set            */
    LBM_ERR_CUDA = 2,     /* a CUDA runtime call failed                    */
    LBM_ERR_OOM = 3,      /* device allocation failed                      */
    LBM_ERR_DIVERGED = 4, /* non-finite value or |u| > c_s in the state    */
    LBM_ERR_TIMEOUT = 5,  /* a bounded device wait ran out                 */
    LBM_ERR_STATE = 6     /* call not valid in the context's current state */
} lbm_status;

typedef enum {
    LBM_WALL_ADIABATIC = 0, /* no-slip, zero heat flux (half-way bounce-back) */
    LBM_WALL_DIRICHLET = 1, /* no-slip, T = T_w (half-way anti-bounce-back)   */
    LBM_WALL_PERIODIC = 2   /* no wall: the axis wraps (both faces of an axis) */
} lbm_wall_kind;

typedef enum {
    LBM_FP32 = 0,  /* 4 bytes per population, 104 B per node                      */
    LBM_FP16S = 1, /* IEEE half deviations, 52 B per node                          */
    LBM_BF16S = 2, /* bfloat16 deviations, 52 B per node                           */
    LBM_FP16M = 3  /* f as IEEE half deviations, g in FP32: 66 B per node          */
} lbm_storage;

typedef enum {
    LBM_STREAM_AA = 0,   /* in-place AA pattern, one population buffer      */
    LBM_STREAM_PULL2 = 1 /* two buffers, pull streaming (fallback kernel)   */
} lbm_streaming;

typedef struct {
    int kind;   /* lbm_wall_kind */
    double T_w; /* wall temperature, used when kind == LBM_WALL_DIRICHLET */
} lbm_wall;

/* Parameters of one cell.
 * With derive = 1 the transport coefficients follow the free-fall scaling of
 * Sec. 2.1 with dT = 1: nu = U H sqrt(Pr/Ra), kappa = nu/Pr, g beta = U^2/H
 * (H <= 0 means H = nz).  With derive = 0, nu, kappa and gbeta are used as
 * given and Ra, Pr only label the run; U and H still scale the diagnostics.
 * Validity (else LBM_ERR_PARAM): every n >= 3; tau_f = 3 nu + 1/2 > 1/2;
 * a_T = 42 sqrt(3) kappa - 6 in (-6, 1) so that both D3Q7 weights are
 * positive; 0 < U <= 0.2; both faces of an axis periodic or neither. */
typedef struct {
    int nx, ny, nz;
    double Ra, Pr, U, H;
    int derive;
    double nu, kappa, gbeta;
    double body_force[3]; /* constant force density added to the buoyancy force */
    lbm_wall wall[6];
    int storage;    /* lbm_storage */
    int streaming;  /* lbm_streaming */
    int diag_every; /* lbm_step samples the diagnostics every diag_every steps (0: never) */
    int block_size; /* threads per block of the register step kernels, 0 = library default (128) */
    int nodes_per_thread; /* AA step kernels: 1, or 2 (packed FP32 arithmetic); 0 = library default (2) */
    int pipeline; /* AA steps without a diagnostic sample: 1 = register kernels (each thread loads its
                     populations into registers), 2 = staged kernels (persistent blocks copy the
                     population windows of the next tiles into shared memory with bulk asynchronous
                     copies while the current tile is updated; LBM_ERR_PARAM where they cannot run),
                     0 = library default (register for LBM_FP32, staged for the others) */
} lbm_params;

/* Device memory provider.  alloc returns device memory of at least `bytes`
 * bytes usable on `stream` (NULL on failure); free releases it.  A NULL
 * allocator makes the library call cudaMalloc / cudaFree itself.  The Python
 * binding passes PyTorch's caching allocator here. */
typedef struct {
    void *(*alloc)(size_t bytes, void *stream, void *user);
    void (*free)(void *ptr, size_t bytes, void *stream, void *user);
    void *user;
} lbm_allocator;

/* Constants derived from the parameters (all in lattice units). */
typedef struct {
    double nu, kappa, gbeta, tau_f;
    double s_e, s_q;            /* s_e = s_eps = s_nu = s_pi = 1/tau_f; s_q = s_m */
    double q_kappa, q_e, q_nu;  /* D3Q7 rates, Sec. 2.3 */
    double a_T, w0_T, w1_T;     /* D3Q7 constant and weights */
    double H, U;
    int64_t nodes;              /* nx ny nz */
    int64_t device_bytes;       /* device memory held by the context */
} lbm_constants;

#define LBM_NDIAG 24

/* Global diagnostics (free-fall units, dT = 1), definitions of Secs. 3 and 4:
 *   E        = 1/2 <|u|^2> / U^2                 (mean kinetic energy, Sec. 3)
 *   rms_drho = sqrt(<(rho - rho0)^2>)            (Table 3)
 *   rms_div  = sqrt(<(div u)^2>) H / U           (Table 3)
 *   Re_rms   = sqrt(<|u|^2>) H / nu, Re_w = sqrt(<w^2>) H / nu      (Sec. 4)
 *   Nu_vol   = 1 + <w T> H / kappa                                  (Sec. 4)
 *   Nu_kin   = 1 + <eps_u> H^2 / (kappa U^2), eps_u = nu/2 sum (d_i u_j + d_j u_i)^2
 *   Nu_th    = <eps_T> H^2 / kappa, eps_T = kappa |grad T|^2        (Sec. 4)
 *   Nu_face[f] = -H <dT/dn> over the nodes of Dirichlet face f, n into the
 *              fluid (Nu_overall of Sec. 3, Nu_wall of Sec. 4); 0 elsewhere.
 *              Side-heated cell: Nu_hot = Nu_face[0], Nu_cold = -Nu_face[1];
 *              Rayleigh-Benard: Nu_wall = (Nu_face[4] - Nu_face[5]) / 2.
 *   Nu_link[f] = H/kappa times the mean heat per step that the anti-bounce-
 *              back links of face f carry into the fluid.
 * Averages <.> run over the nx ny nz nodes.  Derivatives: central differences
 * inside, a one-sided second-order stencil through the wall value next to a
 * no-slip or Dirichlet wall, a zero-gradient stencil next to an adiabatic wall.
 * The avg_* members use the same formulas on the raw sums averaged over every
 * sample since the last reset, i.e. volume-and-time averages <.>_{V,t}. */
typedef struct {
    int64_t step;      /* time step of the state */
    int64_t sample_step; /* time step of the last sample (-1: none) */
    int64_t samples;   /* samples in the time averages */
    double E, rms_drho, rms_div, Re_rms, Re_w, Nu_vol, Nu_kin, Nu_th;
    double mean_T, mass, max_u;
    double Nu_face[6], Nu_link[6];
    double avg_E, avg_Re_rms, avg_Re_w, avg_Nu_vol, avg_Nu_kin, avg_Nu_th;
    double avg_Nu_face[6];
    int64_t nonfinite; /* nodes with a non-finite moment in the last sample */
    double raw[LBM_NDIAG];
} lbm_diag;

typedef struct lbm_ctx lbm_ctx;

/* Create a cell on the current CUDA device.  stream: a cudaStream_t (NULL: the
 * legacy default stream).  alloc: may be NULL.  The state starts at rest,
 * rho = 1, u = 0, T = 0.  *out receives the
 * context, owned by the caller until lbm_destroy.  On failure *out is NULL and
 * lbm_last_error(NULL) describes the error. */
lbm_status lbm_create(const lbm_params *params, const lbm_allocator *alloc, void *stream,
                      lbm_ctx **out);

/* Release the context and its device memory.  NULL is ignored. */
void lbm_destroy(lbm_ctx *ctx);

/* Message of the last failed call on ctx (or of the last failed lbm_create on
 * this thread when ctx is NULL).  Valid until the next call. */
const char *lbm_last_error(const lbm_ctx *ctx);

/* Derived constants of the context. */
lbm_status lbm_get_constants(const lbm_ctx *ctx, lbm_constants *out);

/* Replace the state by the equilibrium populations f^eq(rho, u), g^eq(T, u)
 * (Sec. 2.2, 2.3) of host fields rho[n], u3[3][n], T[n] (n = nx ny nz).  The
 * step counter is kept; time averages are not touched. */
lbm_status lbm_set_fields(lbm_ctx *ctx, const double *rho, const double *u3, const double *T);

/* The state replacement of lbm_set_fields in two asynchronous halves, so that
 * the host-to-device copy of the next fields overlaps the steps that run
 * before they are needed (AA streaming only; LBM_ERR_PARAM otherwise).
 *
 * lbm_upload_fields queues the copy of host fields rho[n], u3[3][n], T[n]
 * (n = nx ny nz, x fastest) into a device staging buffer of 5 n doubles that
 * the context owns (allocated at the first call, through the context's
 * allocator) on a copy stream of its own, and returns at once.  The copy
 * waits for the kernel of the previous lbm_apply_fields, so the buffer is
 * never overwritten while it is read.  The host arrays must stay valid and
 * unchanged until the copy has completed: until the next synchronising call
 * (lbm_diagnostics, lbm_moments, lbm_synchronize, ...) after the
 * lbm_apply_fields that uses them.  With pinned host memory the copy runs
 * beside the context's kernels; with pageable memory cudaMemcpyAsync copies
 * before it returns.
 *
 * lbm_apply_fields makes the context's stream wait for the last upload and
 * then writes the equilibrium populations f^eq(rho, u), g^eq(T, u)
 * (Sec. 2.2, 2.3) of the uploaded fields, as lbm_set_fields does, without
 * synchronising.  The step counter is kept; time averages are not touched.
 * LBM_ERR_STATE when no upload is pending (each upload is applied once); a
 * second upload before lbm_apply_fields replaces the first. */
lbm_status lbm_upload_fields(lbm_ctx *ctx, const double *rho, const double *u3, const double *T);
lbm_status lbm_apply_fields(lbm_ctx *ctx);

/* Replace the state by host populations f19[19][n], g7[7][n]: the
 * pre-collision populations f_i(x, t) of Eq. MRT and g_i(x, t) of Eq. MRT_T. */
lbm_status lbm_set_populations(lbm_ctx *ctx, const double *f19, const double *g7);

/* Read the pre-collision populations of the current state (same layout). */
lbm_status lbm_get_populations(lbm_ctx *ctx, double *f19, double *g7);

/* Read the pre-collision populations of `count` nodes with flat indices
 * nodes[k] = x + nx (y + ny z) into f19[k][19] and g7[k][7] (node-major). */
lbm_status lbm_get_populations_at(lbm_ctx *ctx, const int64_t *nodes, int64_t count, double *f19,
                                  double *g7);

/* Advance n time steps (Eq. MRT and Eq. MRT_T for every node, streaming and
 * walls included).  Asynchronous.  When diag_every > 0, the diagnostics are
 * sampled every diag_every steps (on steps that are multiples of it, from the
 * pre-collision state of that step) and accumulated on the device. */
lbm_status lbm_step(lbm_ctx *ctx, int64_t n);

/* Moments of the current state into host arrays rho[n], u3[3][n], T[n]:
 * rho = sum f, u = (sum e f + F/2)/rho, T = sum g (Sec. 2.2, 2.3). */
lbm_status lbm_moments(lbm_ctx *ctx, double *rho, double *u3, double *T);

/* Probability densities of the local dissipation rates of the current state
 * (Sec. 4): eps_u = nu/2 sum_ij (d_i u_j + d_j u_i)^2 and eps_T = kappa |grad T|^2
 * per node, with the derivative stencils of the diagnostics, normalised as
 * X = eps / eps_rms.  counts_u[nbins] and counts_T[nbins] (host arrays,
 * overwritten) receive the number of nodes with X in each of nbins equal bins
 * on [0, xmax); nodes with X >= xmax are not counted.  rms_in[2] (host,
 * optional) gives eps_rms for eps_u and eps_T, so that the samples of a time
 * series share one normalisation; NULL computes sqrt(<eps^2>) of this state.
 * rms_out[2] (host, optional) receives the values used.  A zero eps_rms
 * counts every node in bin 0.  Synchronises the stream.  Errors:
 * LBM_ERR_PARAM (nbins outside [1, 4096], xmax not positive, a NULL count
 * array, a negative rms_in), LBM_ERR_OOM (device scratch), LBM_ERR_CUDA,
 * LBM_ERR_TIMEOUT (as lbm_synchronize). */
lbm_status lbm_dissipation_pdf(lbm_ctx *ctx, int nbins, double xmax, const double *rms_in, double *rms_out,
                               uint64_t *counts_u, uint64_t *counts_T);

/* Nusselt numbers of Sec. 3 beyond the wall averages, of the current state,
 * with the temperature difference of the walls taken as 1 and lengths in
 * units of H (lbm_constants.H):
 *   profile[n_axis] (host, overwritten): the plane-averaged Nusselt number
 *     along `axis` (0 = x, 1 = y, 2 = z), the x-z plane average Nu(y) of the
 *     paper's Fig. 4 taken along any axis: for every node plane j,
 *     the mean over the plane's nodes of u_a T H / kappa - H dT/dx_a
 *     (the paper's v T sqrt(Ra Pr) - dT/dy in lattice units), dT/dx_a with
 *     the derivative stencils of the diagnostics;
 *   nu_mid[6] (host, optional): for each face -x, +x, -y, +y, -z, +z, the
 *     mid-line Nusselt number Nu_mean of Table 2: the mean of -H dT/dn at the
 *     wall (n into the fluid, the stencil of lbm_diag.Nu_face) over the nodes
 *     next to the face on the line along z (along x for the z faces) through
 *     the middle of the third axis; for an even node count along that axis
 *     the mean over the two node lines that bracket its middle; 0 for a face
 *     that is not a Dirichlet wall.
 * Synchronises the stream.  Errors: LBM_ERR_PARAM (axis outside 0..2, NULL
 * profile), LBM_ERR_OOM (device scratch), LBM_ERR_CUDA, LBM_ERR_TIMEOUT. */
lbm_status lbm_nusselt_profile(lbm_ctx *ctx, int axis, double *profile, double *nu_mid);

/* Sample the diagnostics of the current state now (adds to the averages). */
lbm_status lbm_sample(lbm_ctx *ctx);

/* Fill *out from the last sample and the accumulated averages; reset the
 * averages afterwards when reset != 0.  Returns LBM_ERR_DIVERGED (with *out
 * filled) when the last sample saw a non-finite moment or max |u| > 1/sqrt(3). */
lbm_status lbm_diagnostics(lbm_ctx *ctx, lbm_diag *out, int reset);

/* Wait for the context's stream.  Returns LBM_ERR_TIMEOUT (once) if a
 * pipeline wait of a staged step kernel ran out of its cycle budget since the
 * last check; the state is then undefined.  lbm_diagnostics, lbm_moments and
 * the population readers make the same check after their data arrives. */
lbm_status lbm_synchronize(lbm_ctx *ctx);

/* Cycle budget of one pipeline wait of the staged step kernels (default 2^31
 * cycles, about a second).  After a wait runs out, the kernel raises the
 * context's error flag, lets the copies it has in flight land and returns;
 * lbm_synchronize or lbm_diagnostics then report LBM_ERR_TIMEOUT.  A budget of
 * 0 makes every wait fail at once: used to test that path. */
lbm_status lbm_set_wait_budget(lbm_ctx *ctx, int64_t cycles);

/* Checkpoint: write / read the state (populations, step counter, time
 * accumulators) to / from a file.  lbm_load requires a context created with
 * the same lattice, walls and storage; continuing after a load reproduces the
 * run bit for bit. */
lbm_status lbm_save(lbm_ctx *ctx, const char *path);
lbm_status lbm_load(lbm_ctx *ctx, const char *path);

/* Device view of the population storage, for callers that keep data on the
 * GPU: base pointers of f (19 arrays) and g (7 arrays), elements between
 * consecutive population arrays, and the element size in bytes of f (g uses
 * 4 bytes with LBM_FP16M, else the size of f).  Stored values are deviations
 * from the rest state, f - w rho0 and g - w T0; with LBM_FP16S the g arrays
 * hold 4096 (g - w T0) (scaled to keep small values out of FP16's subnormal
 * range).  The layout of the values depends on the streaming scheme and on
 * the step parity; use lbm_get_populations to read them in a defined layout. */
lbm_status lbm_device_view(lbm_ctx *ctx, void **f, void **g, int64_t *stride, int *elem_bytes);

/* ------------------------------------------------------------------ batches --
 * Many independent cells advanced together (no counterpart in the paper, whose
 * runs are single cells).  A batch borrows existing contexts; each must use
 * the AA streaming scheme and all must share one storage format.  One batch
 * step advances every cell by one time step inside one persistent,
 * cooperative kernel launch: the cells' tiles (a block's share of one cell's
 * step) are listed per step parity, the blocks stride over the list, and a
 * grid-wide barrier separates time steps.  Runs of graph_chunk steps are
 * captured once into a CUDA graph and replayed. */
typedef struct lbm_batch lbm_batch;

/* Schedule of the persistent launch (a new batch starts at 256 threads, 2 blocks
 * per SM, 100 steps per launch, 1000-step graphs, tiles of one block, mode 0). */
typedef struct {
    int block_size;    /* 128 or 256 threads */
    int blocks_per_sm; /* resident blocks per SM (capped by occupancy); grid = SMs x this */
    int steps_per_launch; /* time steps inside one launch (a launch boundary also synchronises) */
    int graph_chunk;   /* steps per captured graph (a multiple of steps_per_launch, even); 0 = no graph */
    int tile_span;     /* tile shape: consecutive blocks of one cell's kernel per tile, 1..64 (a block
                          fetches a tile's description once and updates its span in a row) */
    int mode;          /* 0: one cooperative launch per steps_per_launch steps, a grid-wide barrier
                          between steps; 1: one persistent launch per time step and tile kind (even
                          tiles; row tiles, then face tiles), ordered by the launches themselves */
} lbm_schedule;

/* Create a batch over `ncells` contexts (borrowed: they must outlive the
 * batch and not be stepped on their own while it is in use).  stream: the
 * cudaStream_t of the batch launches (NULL: legacy default stream).  Errors:
 * LBM_ERR_PARAM (a context uses pull streaming, storage formats differ, or
 * ncells < 1); lbm_last_error(NULL) describes it. */
lbm_status lbm_batch_create(lbm_ctx *const *cells, int ncells, void *stream, lbm_batch **out);
void lbm_batch_destroy(lbm_batch *batch);

/* Advance every cell by n time steps.  All cells must be at the same step
 * parity (LBM_ERR_STATE otherwise; lbm_set_fields / lbm_set_populations put a
 * cell at parity 0).  Diagnostics are not sampled inside a batch step; call
 * lbm_sample on a cell afterwards.  Synchronises the stream and returns
 * LBM_ERR_TIMEOUT if a grid-barrier wait ran out of its cycle budget (the
 * cells' states are then undefined). */
lbm_status lbm_batch_step(lbm_batch *batch, int64_t n);

lbm_status lbm_batch_get_schedule(const lbm_batch *batch, lbm_schedule *out);
lbm_status lbm_batch_set_schedule(lbm_batch *batch, const lbm_schedule *s);

/* Time each candidate schedule (both modes, block size 128/256, 1-4 blocks per
 * SM as they fit, tile spans 1, 2, 4, 8 and 16) over `trial_steps` steps and
 * keep the fastest; the trials advance the cells.  *best receives it when
 * non-NULL. */
lbm_status lbm_batch_autotune(lbm_batch *batch, int trial_steps, lbm_schedule *best);

/* Cycle budget of one grid-barrier wait (default 2^31 cycles, about a second).
 * A budget of 0 makes any wait fail at once: used to test the timeout path. */
lbm_status lbm_batch_set_barrier_budget(lbm_batch *batch, int64_t cycles);

/* Allocation-free diagnostics reduction.  The paper has no counterpart.
 *
 * Some callers cannot allocate device memory at the moment they need the
 * global sums: an application that reserves the whole GPU for its own pool at
 * start-up, a solver loop that must not call cudaMalloc while running (the
 * call may synchronise the device and its latency is unbounded), or a plugin
 * whose host framework owns every device allocation.  This entry point
 * performs the reduction of lbm_sample / lbm_diagnostics on fields the caller
 * already holds on the device, and allocates nothing: its per-block partial
 * sums live in a fixed static device array of LBM_NOALLOC_MAX_BLOCKS rows of
 * LBM_NDIAG doubles plus LBM_NDIAG + 1 accumulator slots (233,672 bytes),
 * which every GPU on which the library's code is loaded holds until the
 * process exits.
 *
 *   fields  device, 11 arrays of `stride` floats, x fastest: rho - rho0, u, v,
 *           w, T of every node, then for each face f = 0..5 the pre-collision
 *           g arriving from that face (velocity index f + 1) at the nodes next
 *           to it (read only where face f is a Dirichlet wall).
 *   stride  elements between consecutive arrays, >= nx ny nz.
 *   walls   six faces -x, +x, -y, +y, -z, +z, as in lbm_params.
 *   a_T     the D3Q7 constant of the cell (lbm_constants.a_T), in (-6, 1).
 *   blocks  reduction blocks, 0 for the default the contexts use; more than
 *           LBM_NOALLOC_MAX_BLOCKS does not fit the static array and returns
 *           LBM_ERR_PARAM.
 *   sums    device, LBM_NDIAG doubles receiving the raw sums (lbm_diag.raw).
 *   stream  cudaStream_t the kernels run on (NULL: legacy default stream).
 * Asynchronous.  When the array's memory is taken: CUDA loads device code
 * per context, lazily by default, and the array is allocated when the code
 * holding it is loaded, which happens at the array's address look-up
 * (cudaGetSymbolAddress).  lbm_create does that look-up for its device, so
 * after creating a context on a device the array is held and no later call
 * allocates.  Without a context, the first call on a device does it: make
 * that first call during set-up, before any stream capture.  The address is
 * cached per CUDA context and looked up again if the device was reset.  All
 * calls share the array and it keeps the last call's contents: the
 * accumulator slots are cleared at the start of every call, and calls that
 * overlap on a GPU race.  Errors: LBM_ERR_PARAM for an invalid argument,
 * LBM_ERR_CUDA for a failed launch; lbm_last_error(NULL) describes it. */
#define LBM_NOALLOC_MAX_BLOCKS 1216
lbm_status lbm_reduce_noalloc(const float *fields, int64_t stride, int nx, int ny, int nz,
                              const lbm_wall *walls, double a_T, int blocks, double *sums, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* LBM_GB300_H */
