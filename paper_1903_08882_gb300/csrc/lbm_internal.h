// Internal interface between the C ABI (lbm_api.cu) and the kernel files.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "lbm_device.cuh"

namespace lbm {

constexpr int kNDiag = 24;     // raw diagnostic sums per sample
constexpr int kMomArrays = 11; // rho - rho0, u, v, w, T, and g arriving from each of the 6 faces

// Tiling of the staged (shared-memory pipelined) AA kernels.
struct StagedGeom {
    uint32_t even_tiles; // tiles of the even step: ceil(n / tile)
    uint32_t odd_tiles;  // tiles of the odd step: tpp per plane 1 <= z <= nz-2
    uint32_t tpp;        // odd-step tiles per z-plane
    uint64_t mag_tpp;    // division magic of tpp
    int grid;            // persistent blocks
    int xf;              // 1: the odd kernel updates the x-face nodes of its rows (nx >= staged_xf_min_nx())
    long long budget;    // clock cycles one pipeline wait may take
    // odd step: byte offset, from the f (q < 19) or g array base, of the slot
    // a node's population q streams to: array q at the node + e_q
    long long soff[26];
};

struct StepArgs {
    int storage;  // StorageKind
    int scheme;   // 0: AA pattern, 1: two-buffer pull
    int parity;   // AA: 0 even step (natural -> reversed), 1 odd step
    int block;    // threads per block
    int wide;     // AA: 1 = two nodes per thread (packed FP32), 0 = one node per thread
    void *f, *g;  // AA buffer, or pull source
    void *f2, *g2; // pull destination
    Geom G;
    Phys P;
    float *mom;   // non-null: also write the node moments of the pre-step state
    const uint32_t *face; // AA odd step: flat indices of the nodes next to a face
    uint32_t nface;
    uint32_t nface_yz;    // the first nface_yz of them lie on a y or z face
    StagedGeom T;         // staged kernels only
    int *err;             // staged kernels: set to 1 when a pipeline wait runs out
    cudaStream_t stream;
};

cudaError_t launch_step(const StepArgs &a);
// Launch `fn` as a programmatic dependent launch: its blocks may be
// scheduled while the kernel before it in the stream finishes, once every
// block of that one has signalled (griddepcontrol.launch_dependents); the
// kernel itself waits for the one before it (griddepcontrol.wait) before it
// touches memory, so the order of the data is that of ordinary launches and
// only the launch and block set-up overlap.
cudaError_t pdl_launch(const void *fn, int grid, int block, int smem, cudaStream_t stream, void **args);
// AA odd step of the listed face nodes face[0 .. count) (general path),
// after the staged odd kernel.
cudaError_t launch_face(const StepArgs &a, uint32_t count);
// Face nodes each thread of the face kernel updates for a storage format.
int face_nodes_per_thread(int storage);
// Staged AA step (no diagnostic sample): even step, or odd step with the
// face nodes through launch_face.
cudaError_t launch_staged(const StepArgs &a);
// Opt in to the staged kernels' shared memory and report how many blocks of
// them fit on an SM.
cudaError_t staged_prepare(int storage, int *blocks_per_sm);
// nodes per tile of the even (odd = 0) and odd (odd = 1) staged step
int staged_tile_nodes(int odd);
int staged_xf_min_nx();
// Fills T.soff for the storage format and lattice.
void staged_store_offsets(int storage, const Geom &G, StagedGeom &T);
// op 0: staging -> device layout, 1: device layout -> staging, 2: moments -> st
cudaError_t launch_convert(int storage, int op, float *st, void *f, void *g, const Geom &G,
                           const Phys &P, int layout, cudaStream_t stream);
cudaError_t launch_gather(int storage, float *out, const int64_t *nodes, int64_t count, const void *f,
                          const void *g, const Geom &G, const Phys &P, int layout, cudaStream_t stream);
cudaError_t launch_equilibrium(float *st, const float *fields, uint32_t n, const Phys &P,
                               cudaStream_t stream);
// Equilibrium of device FP64 fields rho[n], u3[3][n], T[n] straight into the
// natural device layout (AA before an even step).
cudaError_t launch_fields_natural(int storage, const double *rho, const double *u3, const double *T, void *f,
                                  void *g, const Geom &G, const Phys &P, cudaStream_t stream);

// Diagnostics: reduce the moment arrays into per-block partial sums, then sum
// them into raw[kNDiag] (this sample) and add raw to acc[kNDiag] (time sums;
// acc[kNDiag] counts the samples).
int diag_blocks(const Geom &G);
// Dissipation-rate PDFs (Sec. 4) from the moment arrays: sums of eps_u^2 and
// eps_T^2 into sums[2] (added), and counts of eps * scale in [0, nbins) into
// counts[2 nbins] (added; eps_u first).  nbins <= kPdfMaxBins.
constexpr int kPdfMaxBins = 4096;
cudaError_t launch_eps_sq(const float *mom, const Geom &G, const Phys &P, const float *wallT, float nu,
                          float ka, double *sums, cudaStream_t stream);
cudaError_t launch_eps_hist(const float *mom, const Geom &G, const Phys &P, const float *wallT, float nu,
                            float ka, double scale_u, double scale_t, int nbins, unsigned long long *counts,
                            cudaStream_t stream);
// Nusselt profile along axis (Sec. 3, Fig. 4) into prof[n_axis] (sums over
// each plane, added; the caller zeroes and divides by the plane's node count)
// and the six mid-line wall Nusselt numbers (Sec. 3, Table 2) into mid[6].
cudaError_t launch_nu_profile(const float *mom, const Geom &G, const Phys &P, const float *wallT, int axis,
                              float H, float kappa, double *prof, double *mid, cudaStream_t stream);
cudaError_t launch_diag(const float *mom, const Geom &G, const Phys &P, const float *wallT,
                        double *partial, int nblocks, double *raw, double *acc, cudaStream_t stream);

// ---- batched persistent launch ----
struct CellDev {
    Geom G;
    Phys P;               // P.t: the cell's time step when the batch was created
    void *f, *g;          // AA population buffer of the cell (f arrays, then g arrays)
    const uint32_t *face; // nodes next to a face
    uint32_t nface;
};
enum TileKind { TILE_EVEN = 0, TILE_ROWS = 1, TILE_FACE = 2 };
struct Tile {
    int cell, kind;
    uint32_t blk;  // first block index of the single-cell kernel this tile stands for
    uint32_t nblk; // consecutive blocks it covers
};
struct GridBarrier {
    unsigned count, gen;
    int err;        // 1: a wait ran out of its cycle budget
    unsigned steps; // time steps the batch has taken (device-side, so graph replays advance it)
};
struct BatchArgs {
    const CellDev *cells;
    const Tile *even, *odd;         // odd = row tiles followed by face tiles
    const Tile *rows, *faces;
    int n_even, n_odd, n_rows, n_faces, nsteps, parity0;
    GridBarrier *bar;
    long long budget;
    int mode;                       // 0: cooperative multi-step launch, 1: one launch per step and tile kind
    int grid, block;
    int grid_k[3];                  // mode 1: grid of each tile kind's kernel
    cudaStream_t stream;
};
// block is 128 or 256 threads (two compiled variants)
const void *batch_kernel_ptr(int storage, int block);
const void *bstep_kernel_ptr(int storage, int kind, int block);
cudaError_t launch_batch(int storage, const BatchArgs &a);

// Loads, on the current device, the static scratch of lbm_reduce_noalloc
// (see lbm_noalloc.cu); lbm_create calls it so that the array is taken at
// set-up rather than at a later no-allocation call.
cudaError_t noalloc_setup();

// Sets the message lbm_last_error(NULL) returns.
void set_global_error(const std::string &msg);

} // namespace lbm
