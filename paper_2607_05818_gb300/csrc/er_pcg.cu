// Multi-RHS Jacobi-preconditioned CG for G Z = Y^T on the GB300 (sm_103a).
//
// Jacobi-PCG on G is run as plain CG on the scaled matrix G~ = D^-1/2 G D^-1/2 (unit
// diagonal): b~ = D^-1/2 b, x~ = D^1/2 x, r~ = D^-1/2 r.  The iterates are those of
// Jacobi-PCG, and the preconditioned residual norm r^T D^-1 r equals r~^T r~, so no
// separate z vector and no per-element diagonal multiply are needed in the loop.
//
// One CG iteration is two passes over the node-by-RHS arrays ([n][k], k innermost):
//   FP64 form   pass A  p' = r + beta p; q = G~ p'; store p', q; dot p'.q -> alpha
//               pass S  x += alpha p'; r -= alpha q (streaming);  dot r.r -> beta
//   FP32 form   pass A  p' = r + beta p; q = G~ p'; dot p'.q -> alpha (no stores)
//               pass B  recompute p', q; x += alpha p'; r' = r - alpha q; store x, r', p'
//                       dot r'.r' -> beta
// The FP32 form moves 8 vector accesses per iteration instead of 10 by recomputing the
// stencil (cheap on the FP32 pipe); the FP64 form keeps q because FP64 arithmetic runs at
// a small fraction of the FP32 rate on this part and would bound the recompute.
//
// Stencil passes sweep y: a CTA owns 30 nodes along x (plus one halo node on each side)
// and `rows` rows of one tier, for one block of RHS columns.  Each thread holds one
// node's 16-byte column slice; the y-neighbours of p' stay in registers as the sweep
// advances, the x-neighbours are exchanged through a two-row shared-memory ring, and the
// next row's loads are issued before the current row is processed.  TSV couplings are
// sparse (CSR per node) and read straight from global memory.
//
// Dot products: per-thread partials (double-float on the FP32 path, FP64 otherwise),
// then a fixed-order CTA reduction, one partial per (spatial tile, column), and the last
// CTA of each column block (atomic ticket) sums the partials in tile order and updates
// alpha/beta/rho and the convergence flags.  Results are deterministic run to run.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "er_internal.h"

namespace er {

enum Mode { MODE_A_DOT = 0, MODE_A_STORE = 1, MODE_B = 2, MODE_R = 3, MODE_S = 4, MODE_INIT = 5, MODE_UNSCALE = 6 };

template <typename T, typename C>
struct KArgs {
    int T_, W, H, k;
    int tiles_x, tiles_y, rows, n_spatial;
    const T *r_in, *p_in, *b_in, *q_in;
    T *x, *r_out, *p_out, *q_out;
    const C *cE, *cS, *tsv_c;
    const int32_t *tsv_ptr, *tsv_nbr;
    const double *dinvs;
    double *alpha, *beta, *rho, *rho0, *resid;
    int *active, *col_active, *n_restart;
    unsigned *counter;
    double *part;
    double tol;
    int restart;  // MODE_R: 1 = residual replacement with restarts, 0 = record only
};

// ---------------------------------------------------------------------------------------
// accumulators

__device__ inline void two_prod_sum(float &hi, float &lo, float a, float b) {
    // hi + lo += a*b with TwoProduct (FMA) and TwoSum (Knuth); see Ogita, Rump and Oishi,
    // "Accurate sum and dot product", SIAM J. Sci. Comput. 26 (2005).  The _rn intrinsics
    // are never contracted into FMAs, which would corrupt the error terms.
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
        const double rho = a.rho[j];
        if (a.active[j] && total > 0.0 && isfinite(total)) {
            a.alpha[j] = rho / total;
        } else {
            a.alpha[j] = 0.0;
            a.active[j] = 0;
        }
    } else if constexpr (MODE == MODE_B || MODE == MODE_S) {
        if (a.active[j]) {
            const double rho = a.rho[j];
            a.beta[j] = rho > 0.0 ? total / rho : 0.0;
            a.rho[j] = total;
            const double rel = a.rho0[j] > 0.0 ? sqrt(total / a.rho0[j]) : 0.0;
            if (!(rel > a.tol)) {
                a.active[j] = 0;
                a.beta[j] = 0.0;
            }
        } else {
            a.beta[j] = 0.0;
        }
    } else if constexpr (MODE == MODE_R) {
        const double rel = a.rho0[j] > 0.0 ? sqrt(total / a.rho0[j]) : 0.0;
        a.resid[j] = rel;
        if (a.restart) {
            if (a.active[j]) {
                const double rho = a.rho[j];
                a.beta[j] = rho > 0.0 ? a.beta[j] * (total / rho) : 0.0;
                a.rho[j] = total;
                if (!(rel > a.tol)) {
                    a.active[j] = 0;
                    a.beta[j] = 0.0;
                }
            } else if (rel > a.tol) {
                a.active[j] = 1;
                a.beta[j] = 0.0;
                a.rho[j] = total;
                atomicAdd(a.n_restart, 1);
            }
        }
    } else if constexpr (MODE == MODE_INIT) {
        a.rho0[j] = total;
        a.rho[j] = total;
        a.alpha[j] = 0.0;
        a.beta[j] = 0.0;
        a.active[j] = total > 0.0 ? 1 : 0;
        a.resid[j] = total > 0.0 ? 1.0 : 0.0;
    }
    nact += a.active[j];
}

// sred must hold at least max(kNX, kThreads / KB) * KB doubles.
template <typename T, typename C, int MODE, int KB>
__device__ inline void reduce_and_finalize(const KArgs<T, C> &a, double *sred, int spatial, int cb) {
    __shared__ bool s_last;
    __shared__ int s_nact;
    if (threadIdx.x < KB) {
        double s = 0.0;
        for (int xx = 0; xx < kNX; ++xx) s += sred[xx * KB + threadIdx.x];
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
    double s = 0.0;
    if (j < a.k)
        for (int t = gl; t < a.n_spatial; t += G) s += __ldcg(&a.part[(int64_t)t * a.k + j]);
    sred[gl * KB + cj] = s;
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

// ---------------------------------------------------------------------------------------
// stencil passes (A, B, R)

template <typename T, typename C, int MODE>
__global__ void __launch_bounds__(kThreads) k_stencil(const KArgs<T, C> a) {
    constexpr int V = 16 / sizeof(T);
    constexpr int KB = kTPN * V;
    constexpr int SRED = (kNX > kThreads / KB ? kNX : kThreads / KB) * KB;
    __shared__ __align__(16) C sp[2][kNX][KB];
    __shared__ double sred[SRED];

    const int lc = threadIdx.x % kTPN, xl = threadIdx.x / kTPN;
    int b = blockIdx.x;
    const int tx = b % a.tiles_x;
    b /= a.tiles_x;
    const int tyi = b % a.tiles_y;
    b /= a.tiles_y;
    const int t = b % a.T_;
    const int cb = b / a.T_;
    const int spatial = (t * a.tiles_y + tyi) * a.tiles_x + tx;
    const int x = tx * kTXI - 1 + xl;
    const int y0 = tyi * a.rows, y1 = min(y0 + a.rows, a.H);
    const int col = cb * KB + lc * V;
    const bool colok = col < a.k;
    const bool xok = x >= 0 && x < a.W;
    const bool own = xl >= 1 && xl <= kNX - 2 && x < a.W && colok;
    const int64_t tbase = (int64_t)t * a.W * a.H;

    C be[V], al[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
        be[v] = (colok && MODE != MODE_R) ? (C)a.beta[col + v] : (C)0;
        al[v] = (colok && MODE == MODE_B) ? (C)a.alpha[col + v] : (C)0;
    }
    C pu[V], pm[V], pc[V], rm[V], rc[V], nr[V], np_[V];
    Acc<C> acc[V];
#pragma unroll
    for (int v = 0; v < V; ++v) pu[v] = pm[v] = rm[v] = nr[v] = np_[v] = (C)0;

    auto load_row = [&](int y) {
        if (y >= 0 && y < a.H && xok && colok) {
            const int64_t idx = (tbase + (int64_t)y * a.W + x) * a.k + col;
            if constexpr (MODE == MODE_R) {
                ldv<T, C, V>(a.x + idx, nr);
            } else {
                ldv<T, C, V>(a.r_in + idx, nr);
                ldv<T, C, V>(a.p_in + idx, np_);
            }
        } else {
#pragma unroll
            for (int v = 0; v < V; ++v) nr[v] = np_[v] = (C)0;
        }
    };

    load_row(y0 - 1);
    for (int y = y0 - 1; y <= y1; ++y) {
#pragma unroll
        for (int v = 0; v < V; ++v) {
            rc[v] = nr[v];
            if constexpr (MODE == MODE_R) pc[v] = nr[v];
            else pc[v] = fma(be[v], np_[v], nr[v]);
        }
        if (y + 1 <= y1) load_row(y + 1);
        const int ym = y - 1;
        if (ym >= y0 && own) {
            const int64_t im = tbase + (int64_t)ym * a.W + x;
            const C cn = ym > 0 ? a.cS[im - a.W] : (C)0;
            const C cs = a.cS[im];
            const C cw = x > 0 ? a.cE[im - 1] : (C)0;
            const C ce = a.cE[im];
            C lf[V], rt[V], q[V];
            if constexpr (V == 4 && sizeof(C) == 4) {
                float4 l4 = *reinterpret_cast<const float4 *>(&sp[ym & 1][xl - 1][lc * V]);
                float4 r4 = *reinterpret_cast<const float4 *>(&sp[ym & 1][xl + 1][lc * V]);
                lf[0] = l4.x; lf[1] = l4.y; lf[2] = l4.z; lf[3] = l4.w;
                rt[0] = r4.x; rt[1] = r4.y; rt[2] = r4.z; rt[3] = r4.w;
            } else {
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    lf[v] = sp[ym & 1][xl - 1][lc * V + v];
                    rt[v] = sp[ym & 1][xl + 1][lc * V + v];
                }
            }
#pragma unroll
            for (int v = 0; v < V; ++v) {
                C acc_q = pm[v];
                acc_q = fma(-cn, pu[v], acc_q);
                acc_q = fma(-cs, pc[v], acc_q);
                acc_q = fma(-cw, lf[v], acc_q);
                acc_q = fma(-ce, rt[v], acc_q);
                q[v] = acc_q;
            }
            const int e1 = a.tsv_ptr[im + 1];
            for (int e = a.tsv_ptr[im]; e < e1; ++e) {
                const int64_t jdx = (int64_t)a.tsv_nbr[e] * a.k + col;
                const C c = a.tsv_c[e];
                C pj[V];
                if constexpr (MODE == MODE_R) {
                    ldv<T, C, V>(a.x + jdx, pj);
                } else {
                    C rj[V], qj[V];
                    ldv<T, C, V>(a.r_in + jdx, rj);
                    ldv<T, C, V>(a.p_in + jdx, qj);
#pragma unroll
                    for (int v = 0; v < V; ++v) pj[v] = fma(be[v], qj[v], rj[v]);
                }
#pragma unroll
                for (int v = 0; v < V; ++v) q[v] = fma(-c, pj[v], q[v]);
            }
            const int64_t idx = im * a.k + col;
            if constexpr (MODE == MODE_A_DOT) {
#pragma unroll
                for (int v = 0; v < V; ++v) acc[v].add(pm[v], q[v]);
            } else if constexpr (MODE == MODE_A_STORE) {
                stv<T, C, V>(a.p_out + idx, pm);
                stv<T, C, V>(a.q_out + idx, q);
#pragma unroll
                for (int v = 0; v < V; ++v) acc[v].add(pm[v], q[v]);
            } else if constexpr (MODE == MODE_B) {
                C xv[V], rn[V];
                ldv<T, C, V>(a.x + idx, xv);
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    xv[v] = fma(al[v], pm[v], xv[v]);
                    rn[v] = fma(-al[v], q[v], rm[v]);
                    acc[v].add(rn[v], rn[v]);
                }
                stv<T, C, V>(a.x + idx, xv);
                stv<T, C, V>(a.r_out + idx, rn);
                stv<T, C, V>(a.p_out + idx, pm);
            } else {  // MODE_R: r = D^-1/2 b - G~ x~, computed in C (FP64)
                C bv[V], rn[V];
                ldv<T, C, V>(a.b_in + idx, bv);
                const C ds = (C)a.dinvs[im];
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    rn[v] = fma(ds, bv[v], -q[v]);
                }
                T rs[V];
#pragma unroll
                for (int v = 0; v < V; ++v) rs[v] = (T)rn[v];
                stv<T, T, V>(a.r_out + idx, rs);
#pragma unroll
                for (int v = 0; v < V; ++v) acc[v].add((C)rs[v], (C)rs[v]);
            }
        }
        if constexpr (V == 4 && sizeof(C) == 4) {
            *reinterpret_cast<float4 *>(&sp[y & 1][xl][lc * V]) = make_float4(pc[0], pc[1], pc[2], pc[3]);
        } else {
#pragma unroll
            for (int v = 0; v < V; ++v) sp[y & 1][xl][lc * V + v] = pc[v];
        }
        __syncthreads();
#pragma unroll
        for (int v = 0; v < V; ++v) {
            pu[v] = pm[v];
            pm[v] = pc[v];
            rm[v] = rc[v];
        }
    }
#pragma unroll
    for (int v = 0; v < V; ++v) sred[xl * KB + lc * V + v] = own ? acc[v].val() : 0.0;
    __syncthreads();
    reduce_and_finalize<T, C, MODE, KB>(a, sred, spatial, cb);
}

// ---------------------------------------------------------------------------------------
// streaming passes (S, INIT, UNSCALE): same tiling, no halo

template <typename T, int MODE>
__global__ void __launch_bounds__(kThreads) k_stream(const KArgs<T, T> a) {
    constexpr int V = 16 / sizeof(T);
    constexpr int KB = kTPN * V;
    constexpr int SRED = (kNX > kThreads / KB ? kNX : kThreads / KB) * KB;
    __shared__ double sred[SRED];
    const int lc = threadIdx.x % kTPN, xl = threadIdx.x / kTPN;
    int b = blockIdx.x;
    const int tx = b % a.tiles_x;
    b /= a.tiles_x;
    const int tyi = b % a.tiles_y;
    b /= a.tiles_y;
    const int t = b % a.T_;
    const int cb = b / a.T_;
    const int spatial = (t * a.tiles_y + tyi) * a.tiles_x + tx;
    const int x = tx * kTXI - 1 + xl;
    const int y0 = tyi * a.rows, y1 = min(y0 + a.rows, a.H);
    const int col = cb * KB + lc * V;
    const bool own = xl >= 1 && xl <= kNX - 2 && x < a.W && col < a.k;
    const int64_t tbase = (int64_t)t * a.W * a.H;
    T al[V];
#pragma unroll
    for (int v = 0; v < V; ++v) al[v] = (own && MODE == MODE_S) ? (T)a.alpha[col + v] : (T)0;
    Acc<T> acc[V];
    if (own) {
        for (int y = y0; y < y1; ++y) {
            const int64_t i = tbase + (int64_t)y * a.W + x;
            const int64_t idx = i * a.k + col;
            if constexpr (MODE == MODE_S) {
                T xv[V], pv[V], qv[V], rv[V];
                ldv<T, T, V>(a.x + idx, xv);
                ldv<T, T, V>(a.p_in + idx, pv);
                ldv<T, T, V>(a.q_in + idx, qv);
                ldv<T, T, V>(a.r_in + idx, rv);
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    xv[v] = fma(al[v], pv[v], xv[v]);
                    rv[v] = fma(-al[v], qv[v], rv[v]);
                    acc[v].add(rv[v], rv[v]);
                }
                stv<T, T, V>(a.x + idx, xv);
                stv<T, T, V>(a.r_out + idx, rv);
            } else if constexpr (MODE == MODE_INIT) {
                double bv[V];
                ldv<T, double, V>(a.b_in + idx, bv);
                const double ds = a.dinvs[i];
                T rv[V], z[V];
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    rv[v] = (T)(ds * bv[v]);
                    z[v] = (T)0;
                    acc[v].add(rv[v], rv[v]);
                }
                stv<T, T, V>(a.r_out + idx, rv);
                stv<T, T, V>(a.x + idx, z);
                stv<T, T, V>(a.p_out + idx, z);
            } else {  // MODE_UNSCALE: Z = D^-1/2 x~
                double xv[V];
                ldv<T, double, V>(a.x + idx, xv);
                const double ds = a.dinvs[i];
                T o[V];
#pragma unroll
                for (int v = 0; v < V; ++v) o[v] = (T)(ds * xv[v]);
                stv<T, T, V>(a.x + idx, o);
            }
        }
    }
    if constexpr (MODE != MODE_UNSCALE) {
#pragma unroll
        for (int v = 0; v < V; ++v) sred[xl * KB + lc * V + v] = own ? acc[v].val() : 0.0;
        __syncthreads();
        reduce_and_finalize<T, T, MODE, KB>(a, sred, spatial, cb);
    }
}

// ---------------------------------------------------------------------------------------
// workspace

struct Workspace {
    int k = 0;
    er_precision prec = ER_FP64;
    Tiling til;
    void *r[2] = {nullptr, nullptr}, *p[2] = {nullptr, nullptr}, *q = nullptr;
    double *part = nullptr, *scal = nullptr;  // scal: alpha, beta, rho, rho0, resid (k each)
    int *ints = nullptr;                      // active[k], col_active[n_colblk], n_restart
    unsigned *counter = nullptr;
    int *h_poll = nullptr;                    // pinned: col_active + n_restart
    cudaStream_t s = nullptr;
    cudaEvent_t ev = nullptr;
    cudaGraphExec_t gexec = nullptr;
    std::vector<cudaEvent_t> evpool;  // timing events for profile = 1
    const void *g_Yt = nullptr;
    void *g_Z = nullptr;
    double g_tol = -1.0;
    int g_iters = 0, g_parity = -1;
};

void free_workspace(GridDev *g) {
    Workspace *w = g->ws;
    if (!w) return;
    void *ptrs[] = {w->r[0], w->r[1], w->p[0], w->p[1], w->q, w->part, w->scal, w->ints, w->counter};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (w->h_poll) cudaFreeHost(w->h_poll);
    if (w->gexec) cudaGraphExecDestroy(w->gexec);
    for (cudaEvent_t e : w->evpool) cudaEventDestroy(e);
    if (w->ev) cudaEventDestroy(w->ev);
    if (w->s) cudaStreamDestroy(w->s);
    delete w;
    g->ws = nullptr;
}

static er_status get_workspace(GridDev *g, int k, er_precision prec, Workspace **out) {
    if (g->ws && g->ws->k == k && g->ws->prec == prec) {
        *out = g->ws;
        return ER_OK;
    }
    free_workspace(g);
    Workspace *w = new Workspace();
    g->ws = w;
    w->k = k;
    w->prec = prec;
    const int es = prec == ER_FP64 ? 8 : 4;
    w->til = make_tiling(*g, k, es);
    const size_t vec = (size_t)g->n * (size_t)k * es;
    ER_CUDA(cudaStreamCreateWithFlags(&w->s, cudaStreamNonBlocking));
    ER_CUDA(cudaEventCreateWithFlags(&w->ev, cudaEventDisableTiming));
    ER_CUDA(cudaMalloc(&w->r[0], vec));
    ER_CUDA(cudaMalloc(&w->p[0], vec));
    ER_CUDA(cudaMalloc(&w->p[1], vec));
    if (prec == ER_FP64) {
        ER_CUDA(cudaMalloc(&w->q, vec));
    } else {
        ER_CUDA(cudaMalloc(&w->r[1], vec));
    }
    ER_CUDA(cudaMalloc(&w->part, (size_t)w->til.n_spatial * k * sizeof(double)));
    ER_CUDA(cudaMalloc(&w->scal, (size_t)5 * k * sizeof(double)));
    ER_CUDA(cudaMalloc(&w->ints, ((size_t)k + w->til.n_colblk + 1) * sizeof(int)));
    ER_CUDA(cudaMalloc(&w->counter, (size_t)w->til.n_colblk * sizeof(unsigned)));
    ER_CUDA(cudaMemset(w->counter, 0, (size_t)w->til.n_colblk * sizeof(unsigned)));
    ER_CUDA(cudaMemset(w->ints, 0, ((size_t)k + w->til.n_colblk + 1) * sizeof(int)));
    ER_CUDA(cudaMallocHost(&w->h_poll, ((size_t)w->til.n_colblk + 1) * sizeof(int)));
    *out = w;
    return ER_OK;
}

template <typename T, typename C>
static KArgs<T, C> base_args(const GridDev &g, Workspace &w, const C *cE, const C *cS, const C *tc, double tol) {
    KArgs<T, C> a{};
    a.T_ = g.T; a.W = g.W; a.H = g.H; a.k = w.k;
    a.tiles_x = w.til.tiles_x; a.tiles_y = w.til.tiles_y; a.rows = w.til.rows; a.n_spatial = w.til.n_spatial;
    a.cE = cE; a.cS = cS; a.tsv_c = tc;
    a.tsv_ptr = g.tsv_ptr; a.tsv_nbr = g.tsv_nbr; a.dinvs = g.dinvs;
    a.alpha = w.scal; a.beta = w.scal + w.k; a.rho = w.scal + 2 * w.k; a.rho0 = w.scal + 3 * w.k;
    a.resid = w.scal + 4 * w.k;
    a.active = w.ints; a.col_active = w.ints + w.k; a.n_restart = w.ints + w.k + w.til.n_colblk;
    a.counter = w.counter; a.part = w.part; a.tol = tol;
    return a;
}

// Launch bookkeeping: counts every launch by pass kind and, when profiling, brackets it
// with CUDA events on the solver stream (read back at the next host poll).
struct Prof {
    bool on = false;
    int launches[ER_N_PASS] = {0, 0, 0, 0};
    double ms[ER_N_PASS] = {0.0, 0.0, 0.0, 0.0};
    size_t used = 0;
    std::vector<int> kinds;
};

static cudaEvent_t next_event(Workspace &w, Prof &pf) {
    if (pf.used == w.evpool.size()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        w.evpool.push_back(e);
    }
    return w.evpool[pf.used++];
}

template <typename K, typename A>
static void launch(K kern, const A &a, Workspace &w, Prof *pf, int kind) {
    if (pf) {
        pf->launches[kind]++;
        if (pf->on) cudaEventRecord(next_event(w, *pf), w.s);
    }
    kern<<<(unsigned)w.til.n_ctas(), kThreads, 0, w.s>>>(a);
    if (pf && pf->on) {
        cudaEventRecord(next_event(w, *pf), w.s);
        pf->kinds.push_back(kind);
    }
}

// after a stream synchronisation: fold the recorded event pairs into pf.ms
static void flush_prof(Workspace &w, Prof &pf) {
    for (size_t i = 0; i < pf.kinds.size(); ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, w.evpool[2 * i], w.evpool[2 * i + 1]) == cudaSuccess) pf.ms[pf.kinds[i]] += ms;
    }
    pf.kinds.clear();
    pf.used = 0;
}

// One CG iteration.  `cur` selects the ping-pong buffers; returns the parity after.
static int iterate(const GridDev &g, Workspace &w, void *Z, double tol, int cur, Prof *pf) {
    if (w.prec == ER_FP64) {
        auto a = base_args<double, double>(g, w, g.cE64, g.cS64, g.tsv_c64, tol);
        a.r_in = (const double *)w.r[0];
        a.p_in = (const double *)w.p[cur];
        a.p_out = (double *)w.p[1 - cur];
        a.q_out = (double *)w.q;
        launch(k_stencil<double, double, MODE_A_STORE>, a, w, pf, ER_PASS_A);
        auto s = a;
        s.x = (double *)Z;
        s.p_in = (const double *)w.p[1 - cur];
        s.q_in = (const double *)w.q;
        s.r_in = (const double *)w.r[0];
        s.r_out = (double *)w.r[0];
        launch(k_stream<double, MODE_S>, s, w, pf, ER_PASS_B);
    } else {
        auto a = base_args<float, float>(g, w, g.cE32, g.cS32, g.tsv_c32, tol);
        a.r_in = (const float *)w.r[cur];
        a.p_in = (const float *)w.p[cur];
        launch(k_stencil<float, float, MODE_A_DOT>, a, w, pf, ER_PASS_A);
        auto bb = a;
        bb.x = (float *)Z;
        bb.r_out = (float *)w.r[1 - cur];
        bb.p_out = (float *)w.p[1 - cur];
        launch(k_stencil<float, float, MODE_B>, bb, w, pf, ER_PASS_B);
    }
    return 1 - cur;
}

// FP64 true residual r = D^-1/2 b - G~ x~ into the r buffer `rbuf`.
static void true_residual(const GridDev &g, Workspace &w, const void *Yt, void *Z, double tol, void *rbuf,
                          int restart, Prof *pf) {
    if (w.prec == ER_FP64) {
        auto a = base_args<double, double>(g, w, g.cE64, g.cS64, g.tsv_c64, tol);
        a.x = (double *)Z;
        a.b_in = (const double *)Yt;
        a.r_out = (double *)rbuf;
        a.restart = restart;
        launch(k_stencil<double, double, MODE_R>, a, w, pf, ER_PASS_R);
    } else {
        auto a = base_args<float, double>(g, w, g.cE64, g.cS64, g.tsv_c64, tol);
        a.x = (float *)Z;
        a.b_in = (const float *)Yt;
        a.r_out = (float *)rbuf;
        a.restart = restart;
        launch(k_stencil<float, double, MODE_R>, a, w, pf, ER_PASS_R);
    }
}

static er_status poll(Workspace &w, Prof &pf, int *n_active, int *n_restart) {
    const int nc = w.til.n_colblk;
    ER_CUDA(cudaMemcpyAsync(w.h_poll, w.ints + w.k, (size_t)(nc + 1) * sizeof(int), cudaMemcpyDeviceToHost, w.s));
    ER_CUDA(cudaStreamSynchronize(w.s));
    flush_prof(w, pf);
    int s = 0;
    for (int i = 0; i < nc; ++i) s += w.h_poll[i];
    *n_active = s;
    *n_restart = w.h_poll[nc];
    return ER_OK;
}

er_status solve(er_grid *gg, const void *Yt, void *Z, int32_t k, er_precision prec, const er_solve_opts *o,
                er_solve_stats *stats, cudaStream_t us) {
    auto t0 = std::chrono::steady_clock::now();
    if (!gg) return fail(ER_ERR_INVALID_ARG, "grid is NULL");
    if (k < 4 || (k & 3)) return fail(ER_ERR_INVALID_ARG, "k must be a positive multiple of 4");
    if (!Yt || !Z) return fail(ER_ERR_INVALID_ARG, "Yt or Z is NULL");
    if (((uintptr_t)Yt & 15u) || ((uintptr_t)Z & 15u)) return fail(ER_ERR_INVALID_ARG, "Yt and Z must be 16-byte aligned");
    if (Yt == Z) return fail(ER_ERR_INVALID_ARG, "Yt and Z must not alias");
    if (prec != ER_FP64 && prec != ER_FP32_REFINE) return fail(ER_ERR_INVALID_ARG, "bad precision");
    er_solve_opts opt = o ? *o : er_default_solve_opts(prec);
    if (!(opt.tol > 0.0) || opt.maxit < 1 || opt.check_every < 1 || opt.replace_every < 1 || opt.max_sweeps < 0)
        return fail(ER_ERR_INVALID_ARG, "bad solve options");
    std::lock_guard<std::mutex> lock(gg->mu);
    GridDev &g = gg->d;
    ER_CUDA(cudaSetDevice(g.device));
    Workspace *wp = nullptr;
    er_status st = get_workspace(&g, k, prec, &wp);
    if (st != ER_OK) {
        free_workspace(&g);
        return st;
    }
    Workspace &w = *wp;
    ER_CUDA(cudaEventRecord(w.ev, us));
    ER_CUDA(cudaStreamWaitEvent(w.s, w.ev, 0));
    ER_CUDA(cudaMemsetAsync(w.ints + w.k + w.til.n_colblk, 0, sizeof(int), w.s));
    Prof pf;
    pf.on = opt.profile != 0;
    const bool use_graph = opt.use_graph && !pf.on;

    // x~ = 0, r~ = D^-1/2 b, p = 0, rho0 = r~.r~
    if (prec == ER_FP64) {
        auto a = base_args<double, double>(g, w, g.cE64, g.cS64, g.tsv_c64, opt.tol);
        a.b_in = (const double *)Yt; a.r_out = (double *)w.r[0]; a.x = (double *)Z; a.p_out = (double *)w.p[0];
        launch(k_stream<double, MODE_INIT>, a, w, &pf, ER_PASS_OTHER);
    } else {
        auto a = base_args<float, float>(g, w, g.cE32, g.cS32, g.tsv_c32, opt.tol);
        a.b_in = (const float *)Yt; a.r_out = (float *)w.r[0]; a.x = (float *)Z; a.p_out = (float *)w.p[0];
        launch(k_stream<float, MODE_INIT>, a, w, &pf, ER_PASS_OTHER);
    }
    ER_CUDA(cudaGetLastError());

    int cur = 0, it = 0, n_active = 0, n_restart = 0, last_replace = 0, sweeps = 0;
    bool exhausted = false;
    const int block = std::max(2, opt.check_every + (opt.check_every & 1));  // even: parity returns
    st = poll(w, pf, &n_active, &n_restart);
    if (st != ER_OK) return st;
    bool converged = n_active == 0;
    while (!converged && it < opt.maxit) {
        const int todo = std::min(block, opt.maxit - it);
        const bool graphable = use_graph && todo == block;
        if (graphable) {
            if (!w.gexec || w.g_Yt != Yt || w.g_Z != Z || w.g_tol != opt.tol || w.g_iters != block ||
                w.g_parity != cur) {
                if (w.gexec) cudaGraphExecDestroy(w.gexec);
                w.gexec = nullptr;
                cudaGraph_t graph;
                ER_CUDA(cudaStreamBeginCapture(w.s, cudaStreamCaptureModeThreadLocal));
                int c = cur;
                for (int i = 0; i < block; ++i) c = iterate(g, w, Z, opt.tol, c, nullptr);
                ER_CUDA(cudaStreamEndCapture(w.s, &graph));
                cudaError_t e = cudaGraphInstantiate(&w.gexec, graph, 0);
                cudaGraphDestroy(graph);
                if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
                w.g_Yt = Yt; w.g_Z = Z; w.g_tol = opt.tol; w.g_iters = block; w.g_parity = cur;
            }
            ER_CUDA(cudaGraphLaunch(w.gexec, w.s));
            pf.launches[ER_PASS_A] += block;
            pf.launches[ER_PASS_B] += block;
        } else {
            for (int i = 0; i < todo; ++i) cur = iterate(g, w, Z, opt.tol, cur, &pf);
        }
        it += todo;
        ER_CUDA(cudaGetLastError());
        const bool fp32 = prec == ER_FP32_REFINE;
        const int before = n_restart;
        if (fp32 && it - last_replace >= opt.replace_every) {
            true_residual(g, w, Yt, Z, opt.tol, w.r[cur], sweeps < opt.max_sweeps ? 1 : 0, &pf);
            last_replace = it;
        }
        st = poll(w, pf, &n_active, &n_restart);
        if (st != ER_OK) return st;
        if (n_active == 0 && fp32 && last_replace != it) {
            // the FP32 recursion says done: confirm with the FP64 residual
            true_residual(g, w, Yt, Z, opt.tol, w.r[cur], sweeps < opt.max_sweeps ? 1 : 0, &pf);
            last_replace = it;
            st = poll(w, pf, &n_active, &n_restart);
            if (st != ER_OK) return st;
        }
        if (n_restart > before) ++sweeps;
        if (fp32 && n_active == 0 && sweeps >= opt.max_sweeps) exhausted = true;
        converged = n_active == 0;
    }
    // final FP64 residual check (record only) into a scratch buffer
    void *scratch = prec == ER_FP64 ? w.q : w.r[1 - cur];
    true_residual(g, w, Yt, Z, opt.tol, scratch, 0, &pf);
    // Z = D^-1/2 x~
    if (prec == ER_FP64) {
        auto a = base_args<double, double>(g, w, g.cE64, g.cS64, g.tsv_c64, opt.tol);
        a.x = (double *)Z;
        launch(k_stream<double, MODE_UNSCALE>, a, w, &pf, ER_PASS_OTHER);
    } else {
        auto a = base_args<float, float>(g, w, g.cE32, g.cS32, g.tsv_c32, opt.tol);
        a.x = (float *)Z;
        launch(k_stream<float, MODE_UNSCALE>, a, w, &pf, ER_PASS_OTHER);
    }
    ER_CUDA(cudaGetLastError());
    std::vector<double> resid((size_t)k);
    ER_CUDA(cudaMemcpyAsync(resid.data(), w.scal + 4 * k, (size_t)k * sizeof(double), cudaMemcpyDeviceToHost, w.s));
    ER_CUDA(cudaStreamSynchronize(w.s));
    flush_prof(w, pf);
    int ok_cols = 0;
    double mx = 0.0;
    for (double r : resid) {
        mx = std::max(mx, r);
        ok_cols += (r <= opt.tol);
    }
    if (stats) {
        stats->iterations = it;
        stats->sweeps = sweeps;
        stats->converged_cols = ok_cols;
        stats->k = k;
        stats->max_rel_residual = mx;
        stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        for (int i = 0; i < ER_N_PASS; ++i) {
            stats->launches[i] = pf.launches[i];
            stats->kernel_ms[i] = pf.ms[i];
        }
    }
    if (!converged) return fail(ER_ERR_NOT_CONVERGED, "maxit reached with " + std::to_string(n_active) + " active columns");
    if (exhausted && ok_cols < k)
        return fail(ER_ERR_NOT_CONVERGED, "restart budget spent with " + std::to_string(k - ok_cols) +
                                              " columns above tol in the FP64 residual");
    return ER_OK;
}

}  // namespace er

extern "C" {

er_solve_opts er_default_solve_opts(er_precision prec) {
    er_solve_opts o{};
    o.tol = prec == ER_FP64 ? 1e-12 : 1e-6;
    o.maxit = 100000;
    o.check_every = 10;
    o.replace_every = 50;
    o.max_sweeps = 8;
    o.use_graph = 1;
    o.profile = 0;
    return o;
}

er_status er_solve(er_grid *g, const void *Yt, void *Z, int32_t k, er_precision prec, const er_solve_opts *opts,
                   er_solve_stats *stats, void *stream) {
    return er::solve(g, Yt, Z, k, prec, opts, stats, (cudaStream_t)stream);
}

}  // extern "C"
