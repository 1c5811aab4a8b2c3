// Internal declarations shared by the translation units of liber.so.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>

#include "er.h"

namespace er {

// The FP32 form's multigrid coarsens until a level has at most this many nodes and solves that
// level exactly by its dense inverse; a grid this small is solved without the multigrid.
constexpr int kMgCoarseNodes = 1024;

// Thread-local error message behind er_last_error().
void set_error(const std::string &msg);
er_status fail(er_status s, const std::string &msg);
er_status cuda_fail(cudaError_t e, const char *what);

#define ER_CUDA(call)                                                   \
    do {                                                                \
        cudaError_t _e = (call);                                        \
        if (_e != cudaSuccess) return ::er::cuda_fail(_e, #call);       \
    } while (0)

// Tile geometry shared by every node-by-RHS kernel.  A CTA of kThreads threads
// covers kTPN threads per node (16 bytes each, i.e. kTPN*16/sizeof(T) RHS
// columns) times kNX nodes along x, of which kNX-2 are owned and 2 are halo, and
// sweeps `rows` consecutive y rows of one tier.  Partial dot products are kept per
// (spatial tile, column), so every kernel on one grid uses the same tiling.
constexpr int kThreads = 256;
constexpr int kTPN = 8;
constexpr int kNX = kThreads / kTPN;  // 32 node slots per row
constexpr int kTXI = kNX - 2;         // 30 owned nodes per row

struct Tiling {
    int tiles_x = 0, tiles_y = 0, rows = 0;
    int n_spatial = 0;   // T * tiles_y * tiles_x
    int kb = 0;          // RHS columns per column block
    int n_colblk = 0;    // ceil(k / kb)
    int cb_fast = 1;     // launch order: column blocks of a tile adjacent (1) or outermost (0)
    int64_t n_ctas() const { return (int64_t)n_spatial * n_colblk; }
};

// Device-resident network.  Couplings are those of the Jacobi-scaled matrix
// G~ = D^-1/2 G D^-1/2 (unit diagonal), stored positive: G~_ij = -c_ij.
struct GridDev {
    int T = 0, W = 0, H = 0;
    int64_t n = 0;
    int64_t n_floating = 0, n_tsv = 0, n_pads = 0;
    int64_t ex_slots = 0, ey_slots = 0, n_edges = 0;
    int64_t h2d_bytes = 0;
    int device = 0;
    // scaled couplings: cE[i] to node i+1 (0 at x = W-1), cS[i] to node i+W (0 at y = H-1)
    double *cE64 = nullptr, *cS64 = nullptr;
    float *cE32 = nullptr, *cS32 = nullptr;
    double *dinvs = nullptr;  // D^-1/2, 0 at floating nodes
    // FP32 form: per node {1/d, gE, gS, pad} of the FP32-rounded conductances (edge form)
    float *coef32 = nullptr;
    float *tsv_g32 = nullptr;  // per TSV CSR entry
    // TSV adjacency (both directions), CSR over nodes
    int32_t *tsv_ptr = nullptr;  // n + 1
    int32_t *tsv_nbr = nullptr;
    double *tsv_c64 = nullptr;
    float *tsv_c32 = nullptr;
    // sketch inputs: raw conductances and canonical edge ids
    double *gxr = nullptr, *gyr = nullptr;  // per node: x-segment to the right, y-segment below
    int64_t *tsv_eid = nullptr;             // per CSR entry
    int8_t *tsv_sgn = nullptr;              // +1 if this node is the lower end
    double *tsv_g = nullptr;
    int32_t *pad_ptr = nullptr;             // n + 1
    int64_t *pad_eid = nullptr;
    double *pad_g = nullptr;
    // FP32 sketch: square roots of the same conductances as {hi, lo} FP32 pairs (hi + lo
    // carries about 48 bits), so the FP32 sketch needs no FP64 arithmetic
    float2 *sq_x = nullptr, *sq_y = nullptr;  // per node, as gxr, gyr
    float2 *sq_tsv = nullptr, *sq_pad = nullptr;  // per TSV / pad CSR entry
    uint8_t *floating = nullptr;
    struct Workspace *ws = nullptr;         // cached solve workspace (er_pcg.cu)
    void *aux = nullptr;                    // pairwise R / IR drop scratch (er_pairs.cu)
    struct MgHier *mg = nullptr;            // multigrid hierarchy of the FP32 form (er_mg.cu)
    size_t aux_bytes = 0;
};

// rows: y rows per CTA (0 = default 64, clipped to H); order: 0 default, 1 column blocks
// adjacent in launch order, 2 column blocks outermost.
Tiling make_tiling(const GridDev &g, int k, int elem_bytes, int rows = 0, int order = 0);

// er_pcg.cu
void free_workspace(GridDev *g);

// er_mg.cu
void free_mg(GridDev *g);

// er_noalloc.cu: look up the device address of the no-allocation solve's static workspace on
// `device` (the current device) once; later calls return at once
er_status noalloc_prepare(int device);

// er_grid.cu: grid assembly behind er_grid_create
er_status grid_create(const er_tier *tiers, int32_t n_tiers, const er_tsv *tsv, int64_t n_tsv,
                      const er_pad *pads, int64_t n_pads, const er_options *opt, cudaStream_t stream,
                      er_grid **out);

// er_grid.cu: k a positive multiple of 4, p non-NULL and 16-byte aligned
er_status check_nk(const er_grid *g, int32_t k, const void *p, const char *name);

}  // namespace er

struct er_grid {
    er::GridDev d;
    std::mutex mu;
};
