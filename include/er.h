/*
 * er.h - C ABI of the GB300 effective-resistance library (liber.so).
 *
 * Computes every node's effective resistance to the supply, R_i = e_i^T G^-1 e_i,
 * for a multi-tier 3D-IC power delivery network: per-tier resistive meshes, TSV
 * segments between adjacent tiers and pads to an ideal, grounded supply.
 * Effective resistance is defined in the paper's Sec. II-B, Eq. 2
 * (R(a,b) = (e_a - e_b)^T L^+ (e_a - e_b)); with the supply as node b and its
 * row/column of L deleted, that is R_i = (G^-1)_ii with G = B^T W B + D, the MNA
 * conductance matrix of Sec. II-A, Eq. 1.  The network model (tiers joined by
 * TSV segments Rt_k^{i,i+1}, bumps/pads to the supply) is the paper's Sec. III-A/B.
 *
 * The all-node map is computed as
 *   Y^T = M^T Q^T            (er_sketch; M = [W^{1/2} B; D^{1/2}], Q Rademacher)
 *   Z   = G^-1 Y^T           (er_solve; k right-hand sides, preconditioned CG: Jacobi, or
 *                             one aggregation-multigrid V-cycle per iteration)
 *   R_i = ||Z_i||^2          (er_reff_map)
 * The sketch and the CG solve are not in the paper (it uses a reduced TSV system
 * for bump-load pairs, Sec. III-C/D); they reach the Eq. 2 quantity for all
 * nodes at once.
 *
 * Conventions (every entry point):
 *  - Node id i = (t*H + y)*W + x: tier-major, x fastest.  Node-by-RHS arrays are
 *    row-major [n][k] (the k right-hand sides of a node are contiguous).
 *  - Device arrays are plain device pointers owned by the caller, 16-byte aligned;
 *    k must be a positive multiple of 4.  FP64 arrays for ER_FP64, FP32 for
 *    ER_FP32_REFINE (R is always FP64).
 *  - Host arrays are owned by the caller and copied before the call returns.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  er_sketch and
 *    er_reff_map are asynchronous on it; er_grid_create and er_solve synchronise
 *    it (the solve polls convergence from the host).
 *  - Errors are returned as er_status; nothing is thrown across the ABI.  Invalid
 *    arguments are rejected on the host before any launch.  er_last_error()
 *    returns a thread-local message for the last failing call of this thread.
 *  - Threads: calls on different grids may run concurrently from different host threads
 *    (each grid's solve workspace, hierarchy and scratch are its own).  Calls that use a
 *    grid's cached workspace (er_solve, er_pair_reff, er_ir_drop) are serialised per grid
 *    by a lock; er_sketch and er_reff_map only read the grid.  er_grid_destroy must not
 *    overlap other calls on the same grid.  er_solve_noalloc is the exception (one
 *    process-wide scratch array; see there).
 */
#ifndef ER_H
#define ER_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ER_OK = 0,
    ER_ERR_INVALID_ARG = 1,   /* bad pointer, size, index or conductance */
    ER_ERR_CUDA = 2,          /* a CUDA runtime call failed (message in er_last_error) */
    ER_ERR_OOM = 3,           /* device allocation failed */
    ER_ERR_NO_SUPPLY = 4,     /* the network has no pad: G is singular everywhere */
    ER_ERR_NOT_CONVERGED = 5, /* er_solve hit maxit; Z holds the last iterate */
    ER_ERR_TIMEOUT = 6,       /* a bounded device wait ran out */
    ER_WARN_FLOATING = 7      /* success, but some nodes have no path to a pad: R = +inf */
} er_status;

typedef enum {
    ER_FP64 = 0,        /* FP64 storage and arithmetic throughout */
    ER_FP32_REFINE = 1  /* FP32 storage/stencil/updates; dot sums, iterate and the periodic
                           true-residual replacement in double-float (FP64-class accuracy) */
} er_precision;

/* One tier: a W x H mesh.  gx[y*(W-1) + x] is the conductance (siemens) of segment
 * (x,y)-(x+1,y); gy[y*W + x] that of (x,y)-(x,y+1).  0 means open (no segment);
 * negative or non-finite values are rejected.  All tiers must share W and H. */
typedef struct {
    int32_t W, H;
    const double *gx; /* H*(W-1) entries (may be NULL when W == 1) */
    const double *gy; /* (H-1)*W entries (may be NULL when H == 1) */
} er_tier;

/* A TSV segment joining (tier, x, y) and (tier+1, x, y) with conductance g > 0.
 * A through-stack TSV column is T-1 such segments.  Duplicates act in parallel. */
typedef struct {
    int32_t tier, x, y;
    double g;
} er_tsv;

/* A pad joining (tier, x, y) to the grounded supply with conductance g > 0. */
typedef struct {
    int32_t tier, x, y;
    double g;
} er_pad;

typedef struct er_grid er_grid; /* opaque; owned by the library */

typedef struct {
    int32_t device;       /* CUDA device ordinal; -1 = the current device */
    int32_t reserved[7];  /* zero */
} er_options;

typedef struct {
    double tol;            /* per-column stop: ||D^-1/2 r_j|| <= tol * ||D^-1/2 b_j||
                              (Jacobi-weighted residual; see er_solve) */
    int32_t maxit;         /* iteration cap (both forms, all sweeps together) */
    int32_t check_every;   /* host convergence poll period in iterations (>= 1) */
    int32_t replace_every; /* ER_FP32_REFINE: every m iterations the FP32 correction is
                              folded into the accurate (double-float) iterate and the
                              accurate residual replaces the recursive one (m >= 1) */
    int32_t use_graph;     /* 1: replay each poll period from a captured CUDA graph */
    int32_t profile;       /* 1: time every pass with CUDA events on the solver's stream
                              (disables graphs); fills er_solve_stats.kernel_ms */
    int32_t tile_rows;     /* Jacobi: y rows swept by one CTA of the stencil passes (0 = default
                              64; clipped to H); ignored by the multigrid form */
    int32_t block_order;   /* launch order of the tiled kernels: 0 default, 1 RHS column blocks
                              of a tile adjacent, 2 column blocks outermost.  The multigrid
                              kernels give bitwise the same result in either order */
    int32_t precond;       /* 0 Jacobi (D^-1); 1 aggregation multigrid: one V-cycle per
                              iteration (ER_FP32_REFINE only; see er_solve) */
} er_solve_opts;

/* Pass kinds counted in er_solve_stats.launches / kernel_ms. */
enum { ER_PASS_A = 0,      /* stencil pass: p' = z + beta p, q = G p', dot p'.q */
       ER_PASS_B = 1,      /* update pass: x, r (and p' in the FP32 form), dot r.z; in the
                              FP32 form the odd iterations, which also update x */
       ER_PASS_R = 2,      /* accurate residual pass (FP64 form: FP64; FP32 form: double-float) */
       ER_PASS_OTHER = 3,  /* initialisation, accumulation of x into the accurate iterate, final Z */
       ER_PASS_B0 = 4,     /* FP32 form, even iterations: update pass without x */
       ER_PASS_MG = 5,     /* multigrid V-cycle kernels on the coarse levels (precond = 1) */
       ER_PASS_MG_DOWN = 6,/* multigrid: pre-sweep and restriction on the finest level */
       ER_PASS_MG_UP = 7,  /* multigrid: prolongation and post-sweep on the finest level */
       ER_N_PASS = 8 };

typedef struct {
    int32_t iterations;       /* PCG iterations run */
    int32_t sweeps;           /* accurate residual replacements (ER_FP32_REFINE) */
    int32_t converged_cols;   /* columns meeting tol at the end */
    int32_t k;
    double max_rel_residual;  /* final accurate true residual, max over columns, same norm as tol */
    double seconds;           /* host wall time of the call */
    int32_t launches[ER_N_PASS];  /* kernels launched, by pass kind */
    double kernel_ms[ER_N_PASS];  /* summed CUDA-event durations by pass kind (profile = 1) */
} er_solve_stats;

/* Default solve options: tol 1e-12 (FP64) / 1e-7 (FP32 form; the accurate residual of the
 * accurate iterate), maxit 20000, check_every 10, replace_every 50, use_graph 1,
 * profile 0, tile_rows 0, block_order 0, precond 0. */
er_solve_opts er_default_solve_opts(er_precision prec);

/* Build the device-resident grid: per-node couplings of the Jacobi-scaled matrix
 * D^-1/2 G D^-1/2 (tier-major layout, FP64 and FP32 copies), TSV adjacency as CSR,
 * raw conductances and canonical edge ids for the sketch, and the floating-node
 * mask (nodes without a conducting path to a pad; union-find on the host).
 * Returns ER_OK, ER_WARN_FLOATING (grid usable, those nodes get R = +inf),
 * ER_ERR_NO_SUPPLY, ER_ERR_INVALID_ARG, ER_ERR_OOM or ER_ERR_CUDA.  *out is set
 * only on success/warning.  Synchronises `stream`. */
er_status er_grid_create(const er_tier *tiers, int32_t n_tiers,
                         const er_tsv *tsv, int64_t n_tsv,
                         const er_pad *pads, int64_t n_pads,
                         const er_options *opt, void *stream, er_grid **out);

/* Free the grid and its cached solve workspace.  NULL is accepted. */
er_status er_grid_destroy(er_grid *g);

/* Sizes: n = T*W*H nodes, floating-node count, number of canonical edge slots
 * (mesh segment slots + TSV segments + pads), and the bytes er_grid_create copied
 * host-to-device.  Any output pointer may be NULL. */
er_status er_grid_info(const er_grid *g, int64_t *n_nodes, int64_t *n_floating,
                       int64_t *n_edges, int64_t *h2d_bytes);

/* JL sketch Y^T = M^T Q^T into device array Yt [n][k] (FP64 or FP32 by `prec`).
 * Q[j][e] = +-1/sqrt(k), sign = top bit of SplitMix64(SplitMix64(seed) XOR (e*2^32 + j))
 * (0 -> +); e is the canonical edge id: x-segment slots (t*H+y)*(W-1)+x, then
 * y-segment slots (t*(H-1)+y)*W+x, then TSV segments and pads in input order.
 * Row e of M is +sqrt(w_e) at the lower node id and -sqrt(w_e) at the higher one
 * (pads: +sqrt(g)).  Rows of floating nodes are written as 0.  Async on `stream`. */
er_status er_sketch(er_grid *g, int32_t k, uint64_t seed, er_precision prec, void *Yt,
                    void *stream);

/* Columns j0 .. j0 + k_local - 1 of the k_total-column sketch of er_sketch (the same Q[j][e],
 * scale 1/sqrt(k_total)) into device array Yt [n][k_local]: one column shard of the sketch.
 * Since R_i = sum_j Z_ij^2 runs over independent columns, shards solved separately (one per
 * GPU, say) give partial maps whose sum is the map of the whole sketch.  k_local is a positive
 * multiple of 4, 0 <= j0 and j0 + k_local <= k_total.  Async on `stream`. */
er_status er_sketch_cols(er_grid *g, int32_t k_total, int32_t j0, int32_t k_local, uint64_t seed, er_precision prec,
                         void *Yt, void *stream);

/* Solve G Z = Yt for k right-hand sides (device arrays [n][k], Z written).
 * Preconditioned CG from X0 = 0 (Jacobi, or with precond = 1 one multigrid V-cycle per
 * iteration; see below); a column stops when its Jacobi-weighted residual
 * ||r||_{D^-1} / ||b||_{D^-1} meets opts->tol and is then frozen.
 * ER_FP64: FP64 throughout (run as CG on D^-1/2 G D^-1/2, identical iterates).
 * ER_FP32_REFINE: FP32 vectors, stencil and updates on the network with every
 * conductance rounded to FP32 once (which moves any R by at most a relative 2^-24);
 * dot products accumulated in double-float and FP64; every replace_every iterations the
 * FP32 correction is added to an accurate iterate and the residual is recomputed
 * accurately and substituted (reliable update, no restart); a column stops only when that
 * accurate residual meets tol.  "Accurate" is double-float arithmetic (pairs of FP32
 * numbers, about 48 bits, error-free transformations): FP64 runs at 1/64 of the FP32 rate
 * on GB300, and the residual's error (about 2^-44 of its terms) is far below any
 * tolerance the FP32 form is meant for (>= 1e-10).  Z is written in FP32.
 * precond = 1 (FP32 form): the preconditioner is one V-cycle of an aggregation multigrid
 * instead of D^-1.  Level l+1 aggregates 2 x 2 nodes of every tier of level l; since the
 * Galerkin product P^T G P of a network's matrix is again a network (segments between
 * aggregates kept, those inside dropped, parallel TSVs and pads of an aggregate merged into
 * one), every level is a grid built like er_grid_create's.  Coarsening stops at the first
 * level of at most 1,024 nodes, which is solved exactly by its dense inverse (FP64 Cholesky on
 * the host cores, stored in FP32); one damped-Jacobi sweep (weight 0.9) runs before and after each
 * coarse correction, so the cycle is a fixed symmetric positive definite operator, as CG
 * needs.  The hierarchy is built on the first such call and cached on the grid.  A grid that
 * does not coarsen to at most 2,048 nodes (too many tiers) returns ER_ERR_INVALID_ARG.  The library allocates (and caches on the grid) its workspace.  opts/stats may be NULL.  Returns ER_ERR_NOT_CONVERGED at
 * maxit (Z valid, stats filled), ER_ERR_TIMEOUT if a kernel's bounded wait expired.
 * Synchronises. */
er_status er_solve(er_grid *g, const void *Yt, void *Z, int32_t k, er_precision prec,
                   const er_solve_opts *opts, er_solve_stats *stats, void *stream);

/* The FP64 form of er_solve without any device allocation, for callers that cannot
 * allocate device memory at solve time: code that runs under an allocator that forbids
 * device allocation after start-up, memory-capped serving processes that must not grow,
 * or loops that cannot accept the implicit synchronisation of cudaMalloc/cudaFree.
 * (The paper has no counterpart: this is a deployment variant of the solve.)
 * The solver workspace lives in one file-scope device array of about 9.1 MB; sizes are
 * limited to n*k <= 262144 and k <= 4096, and larger requests return ER_ERR_INVALID_ARG.
 * er_grid_create looks up the array's device address on its device (cudaGetSymbolAddress,
 * which loads the library module that holds the array and commits its 9.1 MB): every GPU on
 * which a grid was created holds the array until the process exits, and a call of
 * er_solve_noalloc neither loads a module nor commits memory.  All calls share the array:
 * each call clears the counters and flags it needs, runs on `stream` without graphs or
 * event timing, and returns when done (after an error, once the stream has drained); calls
 * are serialised by a process-wide lock, and calls that overlap on the GPU would race.  Yt
 * and Z are FP64 [n][k] device arrays as for er_solve; the grid must have been created
 * beforehand.  Same statuses as er_solve. */
er_status er_solve_noalloc(er_grid *g, const void *Yt, void *Z, int32_t k, const er_solve_opts *opts,
                           er_solve_stats *stats, void *stream);

typedef struct {
    int32_t n_grids;
    int32_t iterations;       /* iterations of the batch (the slowest network) */
    int32_t replacements;     /* accurate residual replacements (multigrid mode: the most of any network) */
    int32_t converged;        /* networks whose every column met tol */
    int64_t nodes;            /* non-floating nodes over all networks */
    double max_rel_residual;  /* final accurate residual, max over all networks and columns */
    double seconds;           /* host wall time of the call */
    int32_t launches;         /* kernels launched */
    int32_t graph_captures;   /* CUDA graphs captured (Jacobi: one per change of the work list;
                                 multigrid: one per group of up to 1,024 networks) */
} er_batch_stats;

/* Batching form: the all-node R maps of n networks (e.g. TSV-placement candidates of
 * uneven sizes).  Network c is sketched with seed + c, solved in the FP32 form (the
 * arithmetic of er_solve with ER_FP32_REFINE) and its map written to the device array
 * R_out[c] [n_c] (FP64).  prec must be ER_FP32_REFINE.  Synchronises.
 *   opts->precond == 0 (Jacobi, the default): shared launches.  Every pass of every
 *     iteration is ONE launch over a work list of (network, tile) pairs, captured in a CUDA
 *     graph per poll period; networks leave the work list as they converge.  tile_rows[c]
 *     (nullable) overrides the y rows swept per CTA for network c (the autotuner's choice).
 *     Workspace is allocated for the call and freed before it returns.
 *   opts->precond == 1 (multigrid): er_solve's multigrid iteration on all networks at once.
 *     Every pass (each level's restriction and prolongation, the coarsest solves, direction,
 *     update, the per-column folds, the accurate residual replacement) is ONE persistent
 *     launch over the blocks of the networks still running, found through a device-side work
 *     list; one poll period (opts->check_every iterations) is the body of a device-side WHILE
 *     node of a CUDA graph launched once per group of up to 1,024 networks, whose last kernel
 *     takes each network's decisions exactly where er_solve's host loop would (replace, stop)
 *     and rebuilds the work list, so converged networks leave while the others continue and
 *     no host thread polls.  Every block runs the single-network kernel's body, so each map
 *     equals the single-network map (er_sketch + er_solve + er_reff_map) bitwise.  Networks
 *     of at most 1,024 nodes (their own coarsest level) are solved first
 *     with er_solve's Jacobi path, as alone.  A grid may appear only once
 *     (ER_ERR_INVALID_ARG otherwise).  tile_rows[c] (nullable) is network c's launch order
 *     as er_solve_opts.block_order (the autotuner's choice per size class; 0 = opts'); it
 *     changes the speed, not the result.  Each grid keeps its solve workspace and hierarchy
 *     cached (as after er_solve); the sketch and Z arrays of all networks are allocated for
 *     the call and freed before it returns. */
er_status er_batch_solve(er_grid *const *grids, int32_t n, int32_t k, uint64_t seed, er_precision prec,
                         const int32_t *tile_rows, double *const *R_out, const er_solve_opts *opts,
                         er_batch_stats *stats, void *stream);

/* ---- learned surrogate: a BF16 U-Net from per-node maps to log R -------------------- */

typedef struct {
    int32_t in_ch;   /* input channels per node (a multiple of 32; pad with zeros) */
    int32_t out_ch;  /* outputs per node (log R per tier) */
    int32_t levels;  /* U-Net levels, 2..8 */
    int32_t base;    /* channels of level 0 (a multiple of 32); level l has base * 2^l */
    int32_t H, W;    /* map size, divisible by 2^(levels-1) */
} er_unet_shape;

typedef struct er_surrogate er_surrogate;  /* opaque; owned by the library */

/* Create a U-Net: encoder levels of two 3x3 conv + ReLU with 2x2 max pooling between
 * them, decoder levels of nearest 2x upsampling, concatenation with the encoder's
 * output of the same level and two 3x3 conv + ReLU, and a 1x1 head.  Weights are
 * He-normal from `seed` (FP32 masters, BF16 copies).  The network is not in the paper:
 * it is a screening surrogate of the paper's quantity, with er_solve as the judge. */
er_status er_surrogate_create(const er_unet_shape *shape, uint64_t seed, er_surrogate **out);
er_status er_surrogate_destroy(er_surrogate *s);
/* Parameter count, and FP32 parameters in a fixed order (encoder convolutions level by
 * level, decoder convolutions from the deepest level up, then the head; each layer's
 * weights [cout][3][3][cin] (head [out_ch][base]) before its biases). */
er_status er_surrogate_num_params(const er_surrogate *s, int64_t *n);
er_status er_surrogate_get_params(const er_surrogate *s, float *host, int64_t n);
er_status er_surrogate_set_params(er_surrogate *s, const float *host, int64_t n);
/* Forward pass: maps [B][H][W][in_ch] BF16 (device) -> logR [B][H][W][out_ch] FP32
 * (device).  The 3x3 convolutions run on the tcgen05 tensor cores with the accumulator
 * in tensor memory; their waits are bounded.  Synchronises `stream` at the end and returns
 * ER_ERR_TIMEOUT if a bounded wait expired. */
er_status er_surrogate_infer(er_surrogate *s, const void *maps, int32_t B, float *logR, void *stream);
/* Forward, masked mean-squared error against target [B][H][W][out_ch] (FP32, device;
 * mask uint8 of the same shape, nullable: entries with mask 0 are ignored) and
 * backward; FP32 parameter gradients (same order as the parameters) are copied to
 * grads_host if it is not NULL, the loss to *loss.  Synchronises; ER_ERR_TIMEOUT as for
 * er_surrogate_infer. */
er_status er_surrogate_grad(er_surrogate *s, const void *maps, const float *target, const uint8_t *mask, int32_t B,
                            float *grads_host, double *loss, void *stream);
/* er_surrogate_grad followed by one Adam step (beta 0.9/0.999, eps 1e-8) at rate lr. */
er_status er_surrogate_train_step(er_surrogate *s, const void *maps, const float *target, const uint8_t *mask,
                                  int32_t B, float lr, double *loss, void *stream);

/* Requested output-channel tile width (N of the tcgen05 MMA) of the surrogate's 3x3
 * convolutions: 0 (the default) lets the library choose per layer (the widest of 256, 192,
 * 128, 96, 64, 32 that divides the layer's channels and still gives every SM a tile); 32, 64,
 * 96, 128, 192 or 256 is used on every layer whose output channels it divides.  The
 * arithmetic does not depend on the width.  ER_ERR_INVALID_ARG for other values. */
er_status er_surrogate_set_tile_n(er_surrogate *s, int32_t tile_n);

/* ---- the surrogate's 3x3 convolution layers, one at a time ---------------------------- */

/* What one convolution launch ran. */
typedef struct {
    int32_t kernel;   /* 1: persistent TMA kernel (128-pixel boxes); 2: cp.async-staged kernel */
    int32_t tile_n;   /* output channels per tile (N of the tcgen05 MMA) */
    int32_t k_step;   /* input channels per K step (32 or 64) */
    int32_t reserved;
} er_conv_info;

/* y = act(bias + conv3x3(x, w)) with zero padding: y[b][h][w][o] = bias[o] +
 * sum_{ky,kx,c} x[b][h+ky-1][w+kx-1][c] w[o][ky][kx][c], then ReLU if relu != 0; the layer of
 * er_surrogate_* on its own.  x [B][H][W][cin] and y [B][H][W][cout] are BF16 device arrays,
 * w [cout][3][3][cin] and bias [cout] (nullable) FP32 device arrays; w is rounded to BF16,
 * products are accumulated in FP32 in tensor memory on the tcgen05 tensor cores and y is
 * rounded to BF16.  cin and cout are positive multiples of 32; tile_n as for
 * er_surrogate_set_tile_n.  info (host, nullable) receives what ran.  The BF16 weight copies
 * are allocated and freed in stream order; synchronises `stream`; ER_ERR_TIMEOUT if a
 * bounded wait expired. */
er_status er_conv3x3_forward(const void *x, const float *w, const float *bias, int32_t B, int32_t H, int32_t W,
                             int32_t cin, int32_t cout, int32_t relu, int32_t tile_n, void *y, er_conv_info *info,
                             void *stream);
/* Data gradient of that layer through the ReLU of its input: dx[b][h][w][c] = [x > 0] *
 * sum_{ky,kx,o} dy[b][h-ky+1][w-kx+1][o] w[o][ky][kx][c] (zero outside the image).  dy
 * [B][H][W][cout], x [B][H][W][cin] (the forward input) and dx [B][H][W][cin] are BF16 device
 * arrays; w as for er_conv3x3_forward.  Runs the forward kernels on the flipped, transposed
 * weights.  Same rules as er_conv3x3_forward. */
er_status er_conv3x3_dgrad(const void *dy, const float *w, const void *x, int32_t B, int32_t H, int32_t W,
                           int32_t cin, int32_t cout, int32_t tile_n, void *dx, er_conv_info *info, void *stream);
/* Weight gradient of that layer: dw[o][ky][kx][c] = sum_{b,h,w} dy[b][h][w][o]
 * x[b][h+ky-1][w+kx-1][c] (zero padding), FP32 [cout][3][3][cin] device array, overwritten.
 * x and dy are BF16 device arrays as above; products accumulate in FP32 (on the tcgen05
 * tensor cores when cout is a multiple of 128, cin of 64 and B*H*W tiles into 64-pixel
 * boxes, else on warp-level MMA), split over pixel ranges whose sums are added atomically.
 * Synchronises. */
er_status er_conv3x3_wgrad(const void *x, const void *dy, int32_t B, int32_t H, int32_t W, int32_t cin, int32_t cout,
                           float *dw, void *stream);
/* Launches of the convolution kernels in this process since the last reset (host counters):
 * [0..5] persistent TMA kernel with 32-channel K steps and N tiles of 32, 64, 96, 128, 192,
 * 256; [6..11] the same with 64-channel K steps; [12] cp.async-staged kernel; [13] weight
 * gradient on warp-level mma.sync; [14] weight gradient on tcgen05; [15] zero.  The first min(n, 16) are written to counts; reset != 0 zeroes them. */
er_status er_conv_launch_counts(int64_t *counts, int32_t n, int32_t reset);

/* R_i = sum_j Z_ij^2 into device array R [n] (FP64); +inf for floating nodes.
 * Z is FP64 or FP32 per `prec`.  Async on `stream`. */
er_status er_reff_map(er_grid *g, const void *Z, int32_t k, er_precision prec, double *R,
                      void *stream);

/* ---- pairwise effective resistance and IR drop from the solved sketch ------------------ */

/* Bump-to-load style pair matrix: Rp[a*nv + b] = ||Z_{u[a]} - Z_{v[b]}||^2, the same-seed JL
 * estimate of R(u, v) = (e_u - e_v)^T G^-1 (e_u - e_v), the effective resistance between two
 * network nodes (paper Sec. II-B, Eq. 2; with the supply grounded, Eq. 4 gives
 * (G^-1)_uv = (R_u + R_v - R(u, v)) / 2).  Paths through the supply count: pads are joined
 * through it.  Z is the er_solve output [n][k] (FP64 or FP32 by `prec`, device); u [m] and
 * v [nv] are HOST arrays of node ids (validated, then copied); Rp is a device array
 * [m][nv] (FP64).  Pairs touching a floating node get +inf; u == v gives 0.  FP32 Z:
 * differences and squares in FP32 over runs of 64 columns, run sums in FP64.  Uses a
 * scratch buffer cached on the grid (grown with cudaMalloc when needed).  Synchronises
 * `stream`.  m or nv = 0 is a no-op. */
er_status er_pair_reff(er_grid *g, const void *Z, int32_t k, er_precision prec, const int64_t *u, int32_t m,
                       const int64_t *v, int32_t nv, double *Rp, void *stream);

/* IR drop under S load scenarios (paper Sec. II-A, Eq. 1: G V = I with the supply as
 * reference): drop[i*S + s] = Z_i . w_s with w_s = sum_l I[l*S + s] Z_{loads[l]}, the same-seed
 * JL estimate of (G^-1 I_s)_i, the voltage drop at node i when current I[l*S + s] (amperes,
 * positive = drawn from the network) leaves at node loads[l].  loads [n_loads] and
 * I [n_loads][S] are HOST arrays (validated, copied); drop is a device array [n][S] (FP64).
 * 1 <= S <= 8 and S*k <= 8192.  Currents at floating nodes have zero Z rows and add nothing;
 * the drop at a floating node is +inf.  The fold over loads is deterministic (fixed order)
 * and runs in FP64; the final dot products run in the precision of Z (FP32 Z: rounding of
 * a few units of 1e-7 of ||Z_i|| ||w_s||, the level of Z's own FP32 rounding).
 * Uses the grid's cached scratch buffer; synchronises `stream`. */
er_status er_ir_drop(er_grid *g, const void *Z, int32_t k, er_precision prec, const int64_t *loads, const double *I,
                     int64_t n_loads, int32_t S, double *drop, void *stream);

/* Through-bump currents (the statistic of the paper's TSV-planning study, Sec. IV-B):
 * I_pad[idx*S + s] = g_idx * V[i*S + s] for pad idx (input order of er_grid_create) at node
 * i, the current it carries from the ideal supply into the network when node voltages drop
 * by V (amperes for V in volts).  V is a device array [n][S] in the precision `prec` (FP64
 * or FP32), e.g. the er_solve result for load currents as right-hand sides (G V = I, Eq. 1;
 * the pad currents then add up to the total load current); I_pad is a device array
 * [n_pads][S] (FP64).  g is the pad's conductance as given.  Async on `stream`. */
er_status er_pad_currents(er_grid *g, const void *V, int32_t S, er_precision prec, double *I_pad, void *stream);

/* ---- the paper's own bump-to-load pipeline on a uniform die stack --------------------- */

/* A stack of d uniform dies (paper Sec. III-A/B, notation table): die i is an M x N mesh
 * whose x-directed segments have resistance r[i] and y-directed segments s[i] (ohms); p TSV
 * columns at (tsv_xy[2k], tsv_xy[2k+1]) join every pair of adjacent dies, segment k between
 * die i and die i+1 having resistance Rt[i*p + k].  There is no supply: the quantity is the
 * two-terminal resistance between a bump on die 0 and a load on die d-1. */
typedef struct {
    int32_t M, N;          /* mesh nodes along x and y (every die) */
    int32_t d;             /* dies, 2..64 */
    int32_t p;             /* TSV columns, >= 1 */
    const double *r;       /* [d] */
    const double *s;       /* [d] */
    const int32_t *tsv_xy; /* [p][2] */
    const double *Rt;      /* [d-1][p] */
} er_stack;

typedef struct {
    int32_t n_system;   /* order of the reduced system, (p + 1)(d - 1) */
    int64_t wu_pairs;   /* Eq. 3 evaluations */
    double ms_wu;       /* CUDA-event phase times: cosine tables + Wu double sums */
    double ms_build;    /* reduced system and right-hand sides */
    double ms_lu;       /* LU factorisation */
    double ms_solve;    /* m + n substitutions */
    double ms_dot;      /* m x n pair dot products */
    double seconds;     /* host wall time of the call */
} er_stack_stats;

/* R[i*n + j] = effective resistance between bump i (bump_xy[2i], bump_xy[2i+1] on die 0)
 * and load j (load_xy[2j], load_xy[2j+1] on die d-1), by the paper's divide-and-conquer
 * method (Sec. III-C/D/E): intra-die resistances from Wu's closed form (Eq. 3) with the
 * cosines from the multiple-angle recursion, the pair-independent reduced TSV system
 * (Eq. 13), one LU factorisation, m + n substitutions (Eq. 14) and the pair dot products
 * (Eq. 15).  FP64 throughout.  Host inputs (copied); R is a device array [m][n] (FP64).
 * Limits: M + N <= 3200, (p + 1)(d - 1) <= 46000.  Device workspace is allocated for the
 * call and freed before it returns; synchronises `stream`.  Returns ER_ERR_INVALID_ARG for
 * bad sizes, positions outside the mesh, non-positive resistances or a singular reduced
 * system.  m or n = 0 is a no-op. */
er_status er_stack_pairs(const er_stack *st, const int32_t *bump_xy, int32_t m, const int32_t *load_xy, int32_t n,
                         double *R, er_stack_stats *stats, void *stream);

/* One call from host data to the host R map: create the grid, sketch, solve, map,
 * copy R [n] (FP64) back to R_host, destroy.  Device memory comes from a cached
 * per-device pool (er_release_pool frees it).  stats may be NULL. */
er_status er_reff_map_host(const er_tier *tiers, int32_t n_tiers, const er_tsv *tsv,
                           int64_t n_tsv, const er_pad *pads, int64_t n_pads, int32_t k,
                           uint64_t seed, er_precision prec, const er_solve_opts *opts,
                           double *R_host, er_solve_stats *stats, void *stream);

/* Free the cached device pool of er_reff_map_host on the current device. */
er_status er_release_pool(void);

const char *er_status_str(er_status s);
const char *er_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* ER_H */
