// Device helpers, kernel arguments and the solve workspace shared by the PCG translation
// units (er_pcg.cu: FP64 form and the host loop; er_fp32.cu: FP32 form with TMA staging).
#pragma once

#include <cuda.h>

#include <chrono>
#include <utility>
#include <vector>

#include "er_internal.h"

namespace er {

enum Mode {
    MODE_A_DOT = 0,    // p' = z + beta p, q = G p', dot p'.q (no stores)
    MODE_A_STORE = 1,  // as A, storing p' and q
    MODE_B = 2,        // recompute p', q; x += alpha p'; r -= alpha q; store x, r, p'; dot r.z
    MODE_R = 3,        // residual r = b - G x (FP64 form; double-float in the FP32 form); dot r.z
    MODE_S = 4,        // streaming x += alpha p', r -= alpha q; dot r.r
    MODE_INIT = 5,     // r = b (scaled in the FP64 form), x = 0, p = 0; dot r.z
    MODE_UNSCALE = 6,  // final Z from the iterate
    MODE_ACCUM = 7,    // FP32 form: xhl += x, x = 0
    MODE_B0 = 8        // FP32 form, even iterations: as B without touching x (x is updated
                       // with two iterations' steps in the following odd one)
};

// Arguments of every node-by-RHS kernel.  T: storage type of the [n][k] vectors,
// C: arithmetic type of the stencil.
template <typename T, typename C>
struct KArgs {
    int T_, W, H, k;
    int tiles_x, tiles_y, rows, n_spatial, n_colblk, cb_fast;
    const T *r_in, *p_in, *b_in, *q_in;
    T *x, *r_out, *p_out, *q_out;
    float2 *xhl;                        // FP32 form: iterate as double-float pairs {hi, lo}
    const C *cE, *cS, *tsv_c;           // FP64 form: couplings of D^-1/2 G D^-1/2
    const float4 *coef;                 // FP32 form: per node {1/d, gE, gS, pad}
    const float *tsv_g32;               // FP32 form: TSV conductance per CSR entry
    const int32_t *tsv_ptr, *tsv_nbr;
    const double *dinvs;                // FP64 form: D^-1/2
    double *alpha, *beta, *rho, *rho0, *resid, *alpha_prev;
    int *active, *col_active, *err;
    unsigned *counter;
    double *part;
    double tol;  // per column: ||r||_{D^-1} <= tol ||b||_{D^-1}
    int freeze;  // MODE_B/S: 1 freeze columns at tol; 0 only count columns still above tol
    int rmode;   // MODE_R: 1 residual replacement (and freeze at tol), 0 record only
};

// ---------------------------------------------------------------------------------------
// accumulators

// hi + lo += a*b with TwoProduct (FMA) and TwoSum (Knuth); Ogita, Rump and Oishi,
// "Accurate sum and dot product", SIAM J. Sci. Comput. 26 (2005).  The _rn intrinsics are
// never contracted into FMAs, which would corrupt the error terms.
__device__ inline void two_prod_sum(float &hi, float &lo, float a, float b) {
    float p = __fmul_rn(a, b);
    float pe = fmaf(a, b, -p);
    float t = __fadd_rn(hi, p);
    float bp = __fsub_rn(t, hi);
    float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bp)), __fsub_rn(p, bp));
    hi = t;
    lo = __fadd_rn(lo, __fadd_rn(e, pe));
}

template <typename C>
struct Acc;
template <>
struct Acc<double> {
    double s = 0.0;
    __device__ void add(double a, double b) { s = fma(a, b, s); }
    __device__ double val() const { return s; }
};
template <>
struct Acc<float> {
    float hi = 0.f, lo = 0.f;
    __device__ void add(float a, float b) { two_prod_sum(hi, lo, a, b); }
    __device__ double val() const { return (double)hi + (double)lo; }
};

// 16-byte vector load/store of storage type T into compute type C registers.
template <typename T, typename C, int V>
__device__ inline void ldv(const T *p, C (&v)[V]) {
    if constexpr (sizeof(T) == 4) {
        float4 a = *reinterpret_cast<const float4 *>(p);
        v[0] = (C)a.x; v[1] = (C)a.y; v[2] = (C)a.z; v[3] = (C)a.w;
    } else {
        double2 a = *reinterpret_cast<const double2 *>(p);
        v[0] = (C)a.x; v[1] = (C)a.y;
    }
}
template <typename T, typename C, int V>
__device__ inline void stv(T *p, const C (&v)[V]) {
    if constexpr (sizeof(T) == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4((float)v[0], (float)v[1], (float)v[2], (float)v[3]);
    } else {
        *reinterpret_cast<double2 *>(p) = make_double2((double)v[0], (double)v[1]);
    }
}

// ---------------------------------------------------------------------------------------
// block reduction + last-CTA finalisation of the per-column scalars

template <typename T, typename C, int MODE>
__device__ inline void finalize_column(const KArgs<T, C> &a, int j, double total, int &nact) {
    if constexpr (MODE == MODE_A_DOT || MODE == MODE_A_STORE) {
        a.alpha_prev[j] = a.alpha[j];
        if (a.active[j] && total > 0.0 && isfinite(total)) {
            a.alpha[j] = a.rho[j] / total;
        } else {
            a.alpha[j] = 0.0;
            a.active[j] = 0;
        }
    } else if constexpr (MODE == MODE_B || MODE == MODE_B0 || MODE == MODE_S) {
        if (a.active[j]) {
            const double rho = a.rho[j];
            a.beta[j] = rho > 0.0 ? total / rho : 0.0;
            a.rho[j] = total;
            const double rel = a.rho0[j] > 0.0 ? sqrt(total / a.rho0[j]) : 0.0;
            if (a.freeze) {
                if (!(rel > a.tol)) {
                    a.active[j] = 0;
                    a.beta[j] = 0.0;
                }
                nact += a.active[j];
            } else {
                nact += rel > a.tol;
            }
        } else {
            a.beta[j] = 0.0;
        }
        return;
    } else if constexpr (MODE == MODE_R) {
        const double rel = a.rho0[j] > 0.0 ? sqrt(total / a.rho0[j]) : 0.0;
        a.resid[j] = rel;
        if (a.rmode == 1 && a.active[j]) {
            // reliable update: the recursion continues from the recomputed residual.  If the
            // recursion already claims tol while the accurate residual does not, or it has fallen
            // more than 100x below the true residual, it ran on past its attainable accuracy
            // and the search direction is stale: restart it (beta = 0, a refinement sweep on
            // the correction) instead of rescaling it.
            const double rho = a.rho[j];
            const double rec = a.rho0[j] > 0.0 ? sqrt(rho / a.rho0[j]) : 0.0;
            const bool stale = !(rho > 0.0) || rho < 1e-4 * total || (!(rec > a.tol) && rel > a.tol);
            a.beta[j] = stale ? 0.0 : a.beta[j] * (total / rho);
            a.rho[j] = total;
            if (!(rel > a.tol)) {
                a.active[j] = 0;
                a.beta[j] = 0.0;
            }
        }
    } else if constexpr (MODE == MODE_INIT) {
        a.rho0[j] = total;
        a.rho[j] = total;
        a.alpha[j] = 0.0;
        a.alpha_prev[j] = 0.0;
        a.beta[j] = 0.0;
        a.active[j] = total > 0.0 ? 1 : 0;
        a.resid[j] = total > 0.0 ? 1.0 : 0.0;
    }
    nact += a.active[j];
}

// Threads < KB hold this CTA's partial s of column cb * KB + threadIdx.x.  Writes the CTA's
// column partials, and the last CTA of the column block folds all spatial partials in tile
// order into the per-column scalars; sred is scratch of at least (kThreads / KB) * KB
// doubles, free on entry (reads of it by threads < KB must precede the call).
template <typename T, typename C, int MODE, int KB>
__device__ inline void write_and_finalize(const KArgs<T, C> &a, double *sred, double s, int spatial, int cb) {
    __shared__ bool s_last;
    __shared__ int s_nact;
    if (threadIdx.x < KB) {
        const int j = cb * KB + threadIdx.x;
        if (j < a.k) a.part[(int64_t)spatial * a.k + j] = s;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned prev = atomicAdd(&a.counter[cb], 1u);
        s_last = (prev == (unsigned)(a.n_spatial - 1));
        s_nact = 0;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    constexpr int G = kThreads / KB;
    const int cj = threadIdx.x % KB, gl = threadIdx.x / KB;
    const int j = cb * KB + cj;
    double acc = 0.0;
    if (j < a.k)
        for (int t = gl; t < a.n_spatial; t += G) acc += __ldcg(&a.part[(int64_t)t * a.k + j]);
    sred[gl * KB + cj] = acc;
    __syncthreads();
    if (threadIdx.x < KB && j < a.k) {
        double tot = 0.0;
        for (int g = 0; g < G; ++g) tot += sred[g * KB + cj];
        int nact = 0;
        finalize_column<T, C, MODE>(a, j, tot, nact);
        atomicAdd(&s_nact, nact);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (MODE != MODE_A_DOT && MODE != MODE_A_STORE) a.col_active[cb] = s_nact;
        a.counter[cb] = 0u;
    }
}

// sred holds kNX * KB per-thread partials on entry (and at least (kThreads / KB) * KB
// doubles of room): sums them per column and calls write_and_finalize.
template <typename T, typename C, int MODE, int KB>
__device__ inline void reduce_and_finalize(const KArgs<T, C> &a, double *sred, int spatial, int cb) {
    double s = 0.0;
    if (threadIdx.x < KB)
        for (int xx = 0; xx < kNX; ++xx) s += sred[xx * KB + threadIdx.x];
    __syncthreads();
    write_and_finalize<T, C, MODE, KB>(a, sred, s, spatial, cb);
}

// Block index -> (tile x, tile y, tier, column block).  With cb_fast the column blocks
// of one spatial tile are adjacent in launch order, so the CTAs that read the same node
// rows run together and share DRAM pages and the per-node coefficients in L2.
template <typename T, typename C>
__device__ inline void decode_block(const KArgs<T, C> &a, int block_id, int &tx, int &tyi, int &t, int &cb) {
    int b = block_id;
    if (a.cb_fast) {
        cb = b % a.n_colblk;
        b /= a.n_colblk;
    }
    tx = b % a.tiles_x;
    b /= a.tiles_x;
    tyi = b % a.tiles_y;
    b /= a.tiles_y;
    t = b % a.T_;
    if (!a.cb_fast) cb = b / a.T_;
}

// ---------------------------------------------------------------------------------------
// host side: workspace and launch bookkeeping

struct Workspace {
    int k = 0;
    er_precision prec = ER_FP64;
    Tiling til;
    void *r[2] = {nullptr, nullptr}, *p[2] = {nullptr, nullptr}, *q = nullptr;
    float2 *xhl = nullptr;                    // FP32 form: iterate as double-float pairs {hi, lo}
    double *part = nullptr, *scal = nullptr;  // scal: alpha, beta, rho, rho0, resid, alpha_prev (k each)
    int *ints = nullptr;                      // active[k], col_active[n_colblk], err
    unsigned *counter = nullptr;
    int *h_poll = nullptr;                    // host: col_active + err (pinned in the cached workspace)
    double *h_resid = nullptr;                // host: k final residuals
    cudaStream_t s = nullptr;
    cudaEvent_t ev = nullptr;
    cudaGraphExec_t gexec = nullptr;
    std::vector<cudaEvent_t> evpool;  // timing events for profile = 1
    const void *g_Yt = nullptr;
    void *g_Z = nullptr;
    double g_tol = -1.0;
    int g_iters = 0, g_parity = -1;
    // FP32 form: TMA descriptors of the workspace vectors and of the caller's arrays
    CUtensorMap tm_r[2], tm_p[2], tm_xhl, tm_coef, tm_c, tm_b;
    const void *tm_c_ptr = nullptr, *tm_b_ptr = nullptr;
};

template <typename T, typename C>
KArgs<T, C> base_args(const GridDev &g, const Workspace &w, double tol) {
    KArgs<T, C> a{};
    a.T_ = g.T; a.W = g.W; a.H = g.H; a.k = w.k;
    a.tiles_x = w.til.tiles_x; a.tiles_y = w.til.tiles_y; a.rows = w.til.rows; a.n_spatial = w.til.n_spatial;
    a.n_colblk = w.til.n_colblk; a.cb_fast = w.til.cb_fast;
    a.tsv_ptr = g.tsv_ptr; a.tsv_nbr = g.tsv_nbr; a.dinvs = g.dinvs;
    a.coef = reinterpret_cast<const float4 *>(g.coef32); a.tsv_g32 = g.tsv_g32;
    a.alpha = w.scal; a.beta = w.scal + w.k; a.rho = w.scal + 2 * w.k; a.rho0 = w.scal + 3 * w.k;
    a.resid = w.scal + 4 * w.k; a.alpha_prev = w.scal + 5 * w.k;
    a.active = w.ints; a.col_active = w.ints + w.k; a.err = w.ints + w.k + w.til.n_colblk;
    a.counter = w.counter; a.part = w.part; a.tol = tol;
    return a;
}

// Counts every launch by pass kind and, when profiling, brackets it with CUDA events on
// the solver stream (read back at the next host poll).
struct Prof {
    bool on = false;
    int launches[ER_N_PASS] = {};
    double ms[ER_N_PASS] = {};
    size_t used = 0;
    std::vector<int> kinds;
    std::vector<std::pair<int, int>> evs;  // per timed launch: its start and end events in the pool
    // chained timing (the multigrid solve): a launch that directly follows a timed launch on the
    // stream starts at that launch's end event, so each launch records one event; any other
    // stream operation in between breaks the chain (chain = -1)
    bool chained = false;
    int chain = -1, pending = -1;
};

void prof_begin(Workspace &w, Prof *pf, int kind);
void prof_end(Workspace &w, Prof *pf, int kind);
void flush_prof(Workspace &w, Prof &pf);  // after a synchronisation of w.s

// One network of a batch: its tensor maps (r0, r1, p0, p1, x, xhl, b, coef), its kernel
// arguments (geometry, coefficients, scalars, partials) and its vectors.
struct BatchItem {
    CUtensorMap tm[8];
    KArgs<float, float> a;
    float *r[2], *p[2], *c;
    float2 *xhl;
    const float *b;
};

// er_fp32.cu: batched passes (mode = MODE_*) over a work list of (network, block); with `sel`,
// only the networks c with sel[c] != 0 (device array) run
er_status fp32_batch_pass(int mode, const BatchItem *items, const int2 *work, int n_work, int cur, int rmode,
                          cudaStream_t s, const int *sel = nullptr);
// one network's batch item over its own solve workspace: the arguments and tensor maps of
// fp32_init / fp32_accum / fp32_residual / fp32_final on (g, w) for the batched passes
er_status fp32_workspace_item(const GridDev &g, Workspace &w, const void *Yt, void *Z, double tol, BatchItem *it);
er_status fp32_make_map(CUtensorMap *m, bool f64, const void *base, int64_t d0, int box0, const GridDev &g);

// er_pcg.cu: argument checks and the solve loop on a prepared workspace
er_status check_solve_args(const void *Yt, void *Z, int32_t k, er_precision prec, const er_solve_opts &opt);
er_status solve_core(const GridDev &g, Workspace &w, const void *Yt, void *Z, er_precision prec,
                     const er_solve_opts &opt, er_solve_stats *stats, std::chrono::steady_clock::time_point t0);

// er_mg.cu: the FP32 form with the aggregation-multigrid V-cycle as preconditioner
er_status mg_solve_core(GridDev &g, Workspace &w, const void *Yt, void *Z, const er_solve_opts &opt,
                        er_solve_stats *stats, std::chrono::steady_clock::time_point t0);

// er_fp32.cu: the FP32 form's passes (all asynchronous on w.s)
er_status fp32_prepare(const GridDev &g, Workspace &w, const void *Yt, void *Z);
// er_sketch / er_reff_map on a stream (er_grid.cu)
er_status sketch(er_grid *g, int32_t k, uint64_t seed, er_precision prec, void *Yt, cudaStream_t s);
er_status reff_map(er_grid *g, const void *Z, int32_t k, er_precision prec, double *R, cudaStream_t s);
// er_solve with the grid's lock already held (er_pcg.cu)
er_status solve_locked(er_grid *g, const void *Yt, void *Z, int32_t k, er_precision prec, const er_solve_opts *opts,
                       er_solve_stats *stats, cudaStream_t us);
// the grid's cached solve workspace for (k, precision, tiling), allocated on first use
er_status get_workspace(GridDev *g, int k, er_precision prec, int rows, int order, Workspace **out);
// the multigrid batching form: every pass of er_solve's multigrid iteration one persistent
// launch over all running networks, each poll period the body of a device-side WHILE node (er_mg.cu)
er_status mg_batch_solve(er_grid *const *grids, int32_t n, int32_t k, uint64_t seed, const int32_t *tile_rows,
                         double *const *R_out, const er_solve_opts &opt, er_batch_stats *stats, cudaStream_t us,
                         std::chrono::steady_clock::time_point t0);
void fp32_init(const GridDev &g, Workspace &w, const void *Yt, void *Z, double tol, Prof *pf);
int fp32_iterate(const GridDev &g, Workspace &w, void *Z, double tol, int cur, Prof *pf);
void fp32_accum(const GridDev &g, Workspace &w, void *Z, Prof *pf);
void fp32_residual(const GridDev &g, Workspace &w, const void *Yt, double tol, int cur_buf, int rmode, Prof *pf);
void fp32_final(const GridDev &g, Workspace &w, void *Z, Prof *pf);

}  // namespace er
