// Multi-RHS Jacobi-preconditioned CG for G Z = Y^T on the GB300 (sm_103a): the FP64
// form's kernels and the host loop of both forms (the FP32 form's kernels are in
// er_fp32.cu).
//
// FP64 form.  Jacobi-PCG on G is run as plain CG on the scaled matrix
// G~ = D^-1/2 G D^-1/2 (unit diagonal): b~ = D^-1/2 b, x~ = D^1/2 x, r~ = D^-1/2 r.  The
// iterates are those of Jacobi-PCG and r~.r~ = r^T D^-1 r, so no z vector and no
// per-element diagonal multiply are needed.  One iteration is two passes over the
// node-by-RHS arrays ([n][k], k innermost):
//   pass A  p' = r~ + beta p; q = G~ p'; store p', q; dot p'.q -> alpha      (stencil)
//   pass S  x~ += alpha p'; r~ -= alpha q; dot r~.r~ -> beta, convergence    (streaming)
// FP64 arithmetic runs at a small fraction of the FP32 rate on this part, so the stencil
// pass keeps q (10 vector accesses per iteration) rather than recomputing it.
//
// The stencil pass sweeps y: a CTA owns 30 nodes along x (plus one halo node on each
// side) and `rows` rows of one tier, for one block of RHS columns.  Each thread holds one
// node's 16-byte column slice; the y-neighbours of p' stay in registers as the sweep
// advances, the x-neighbours are exchanged through a two-row shared-memory ring, and the
// next row's loads are issued before the current row is processed.  TSV couplings are
// sparse (CSR per node) and read straight from global memory.
//
// Dot products: per-thread FP64 partials, a fixed-order CTA reduction, one partial per
// (spatial tile, column), and the last CTA of each column block (atomic ticket) sums
// the partials in tile order and updates alpha/beta/rho and the convergence flags, so
// results are bit-identical run to run.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "er_common.cuh"

namespace er {

// x~ at element idx for the residual pass.
template <typename T, typename C, int V>
__device__ inline void load_iterate(const KArgs<T, C> &a, int64_t idx, C (&v)[V]) {
    ldv<T, C, V>(a.x + idx, v);
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
    int tx, tyi, t, cb;
    decode_block(a, (int)blockIdx.x, tx, tyi, t, cb);
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
                load_iterate(a, idx, nr);
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
                    load_iterate(a, jdx, pj);
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
    int tx, tyi, t, cb;
    decode_block(a, (int)blockIdx.x, tx, tyi, t, cb);
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
// workspace and launch bookkeeping

void free_workspace(GridDev *g) {
    Workspace *w = g->ws;
    if (!w) return;
    void *ptrs[] = {w->r[0], w->r[1], w->p[0], w->p[1], w->q, w->xhl, w->part, w->scal, w->ints, w->counter};
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

er_status get_workspace(GridDev *g, int k, er_precision prec, int rows, int order, Workspace **out) {
    const int es = prec == ER_FP64 ? 8 : 4;
    const Tiling want = make_tiling(*g, k, es, rows, order);
    if (g->ws && g->ws->k == k && g->ws->prec == prec && g->ws->til.rows == want.rows &&
        g->ws->til.cb_fast == want.cb_fast) {
        *out = g->ws;
        return ER_OK;
    }
    free_workspace(g);
    Workspace *w = new Workspace();
    g->ws = w;
    w->k = k;
    w->prec = prec;
    w->til = want;
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
        ER_CUDA(cudaMalloc((void **)&w->xhl, (size_t)g->n * (size_t)k * sizeof(float2)));
    }
    ER_CUDA(cudaMalloc(&w->part, (size_t)w->til.n_spatial * k * sizeof(double)));
    ER_CUDA(cudaMalloc(&w->scal, (size_t)6 * k * sizeof(double)));
    const size_t nint = (size_t)k + w->til.n_colblk + 1;
    ER_CUDA(cudaMalloc(&w->ints, nint * sizeof(int)));
    ER_CUDA(cudaMalloc(&w->counter, (size_t)w->til.n_colblk * sizeof(unsigned)));
    ER_CUDA(cudaMemset(w->counter, 0, (size_t)w->til.n_colblk * sizeof(unsigned)));
    ER_CUDA(cudaMemset(w->ints, 0, nint * sizeof(int)));
    ER_CUDA(cudaMallocHost(&w->h_poll, ((size_t)w->til.n_colblk + 1) * sizeof(int)));
    *out = w;
    return ER_OK;
}

static cudaEvent_t next_event(Workspace &w, Prof &pf) {
    if (pf.used == w.evpool.size()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        w.evpool.push_back(e);
    }
    return w.evpool[pf.used++];
}

void prof_begin(Workspace &w, Prof *pf, int kind) {
    if (!pf) return;
    pf->launches[kind]++;
    if (!pf->on) return;
    if (pf->chained && pf->chain >= 0) {
        pf->pending = pf->chain;
    } else {
        pf->pending = (int)pf->used;
        cudaEventRecord(next_event(w, *pf), w.s);
    }
}

void prof_end(Workspace &w, Prof *pf, int kind) {
    if (pf && pf->on) {
        const int e = (int)pf->used;
        cudaEventRecord(next_event(w, *pf), w.s);
        pf->kinds.push_back(kind);
        pf->evs.emplace_back(pf->pending, e);
        if (pf->chained) pf->chain = e;
    }
}

// after a stream synchronisation: fold the recorded event pairs into pf.ms
void flush_prof(Workspace &w, Prof &pf) {
    for (size_t i = 0; i < pf.kinds.size(); ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, w.evpool[(size_t)pf.evs[i].first], w.evpool[(size_t)pf.evs[i].second]) ==
            cudaSuccess)
            pf.ms[pf.kinds[i]] += ms;
    }
    pf.kinds.clear();
    pf.evs.clear();
    pf.used = 0;
    pf.chain = -1;
}

template <typename K, typename A>
static void launch(K kern, const A &a, Workspace &w, Prof *pf, int kind) {
    prof_begin(w, pf, kind);
    kern<<<(unsigned)w.til.n_ctas(), kThreads, 0, w.s>>>(a);
    prof_end(w, pf, kind);
}

// ---------------------------------------------------------------------------------------
// FP64 form passes

static int fp64_iterate(const GridDev &g, Workspace &w, void *Z, double tol, int cur, Prof *pf) {
    auto a = base_args<double, double>(g, w, tol);
    a.cE = g.cE64; a.cS = g.cS64; a.tsv_c = g.tsv_c64;
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
    s.freeze = 1;
    launch(k_stream<double, MODE_S>, s, w, pf, ER_PASS_B);
    return 1 - cur;
}

static void fp64_residual(const GridDev &g, Workspace &w, const void *Yt, void *Z, double tol, void *rbuf,
                          Prof *pf) {
    auto a = base_args<double, double>(g, w, tol);
    a.cE = g.cE64; a.cS = g.cS64; a.tsv_c = g.tsv_c64;
    a.x = (double *)Z;
    a.b_in = (const double *)Yt;
    a.r_out = (double *)rbuf;
    a.rmode = 0;
    launch(k_stencil<double, double, MODE_R>, a, w, pf, ER_PASS_R);
}

static er_status poll(Workspace &w, Prof &pf, int *n_active, int *err) {
    const int nc = w.til.n_colblk;
    ER_CUDA(cudaMemcpyAsync(w.h_poll, w.ints + w.k, (size_t)(nc + 1) * sizeof(int), cudaMemcpyDeviceToHost, w.s));
    ER_CUDA(cudaStreamSynchronize(w.s));
    flush_prof(w, pf);
    int s = 0;
    for (int i = 0; i < nc; ++i) s += w.h_poll[i];
    *n_active = s;
    *err = w.h_poll[nc];
    return ER_OK;
}

// Solve G Z = Y^T for k columns.
//  FP64 form: Jacobi-PCG, each column frozen when its recursive residual meets tol.
//  FP32 form: FP32 Jacobi-PCG on the FP32-rounded network with reliable updates: every
//  replace_every iterations (and whenever every column's recursive residual meets tol)
//  the FP32 correction is folded into the double-float iterate and the accurate residual
//  replaces the recursive one; a column stops only when that accurate residual meets tol.
er_status check_solve_args(const void *Yt, void *Z, int32_t k, er_precision prec, const er_solve_opts &opt) {
    if (k < 4 || (k & 3)) return fail(ER_ERR_INVALID_ARG, "k must be a positive multiple of 4");
    if (!Yt || !Z) return fail(ER_ERR_INVALID_ARG, "Yt or Z is NULL");
    if (((uintptr_t)Yt & 15u) || ((uintptr_t)Z & 15u)) return fail(ER_ERR_INVALID_ARG, "Yt and Z must be 16-byte aligned");
    if (Yt == Z) return fail(ER_ERR_INVALID_ARG, "Yt and Z must not alias");
    if (prec != ER_FP64 && prec != ER_FP32_REFINE) return fail(ER_ERR_INVALID_ARG, "bad precision");
    if (!(opt.tol > 0.0) || opt.maxit < 1 || opt.check_every < 1 || opt.replace_every < 1)
        return fail(ER_ERR_INVALID_ARG, "bad solve options");
    if (opt.tile_rows < 0 || opt.block_order < 0 || opt.block_order > 2)
        return fail(ER_ERR_INVALID_ARG, "bad tile options");
    if (opt.precond < 0 || opt.precond > 1) return fail(ER_ERR_INVALID_ARG, "precond must be 0 (Jacobi) or 1 (multigrid)");
    if (opt.precond == 1 && prec != ER_FP32_REFINE)
        return fail(ER_ERR_INVALID_ARG, "the multigrid preconditioner is available in the FP32 form");
    return ER_OK;
}

er_status solve(er_grid *gg, const void *Yt, void *Z, int32_t k, er_precision prec, const er_solve_opts *o,
                er_solve_stats *stats, cudaStream_t us) {
    if (!gg) return fail(ER_ERR_INVALID_ARG, "grid is NULL");
    std::lock_guard<std::mutex> lock(gg->mu);
    return solve_locked(gg, Yt, Z, k, prec, o, stats, us);
}

// er_solve with the grid's lock already held by the caller
er_status solve_locked(er_grid *gg, const void *Yt, void *Z, int32_t k, er_precision prec, const er_solve_opts *o,
                       er_solve_stats *stats, cudaStream_t us) {
    auto t0 = std::chrono::steady_clock::now();
    if (!gg) return fail(ER_ERR_INVALID_ARG, "grid is NULL");
    er_solve_opts opt = o ? *o : er_default_solve_opts(prec);
    er_status st = check_solve_args(Yt, Z, k, prec, opt);
    if (st != ER_OK) return st;
    GridDev &g = gg->d;
    ER_CUDA(cudaSetDevice(g.device));
    // a grid of at most kMgCoarseNodes nodes is the multigrid's coarsest level itself, and 1 x 1 tiers do
    // not coarsen: both use Jacobi
    const bool mg = opt.precond == 1 && g.n > kMgCoarseNodes && std::max(g.W, g.H) > 1;
    Workspace *wp = nullptr;
    // multigrid: tile_rows sets the finest level's V-cycle rows, not the accurate residual's tiling
    st = get_workspace(&g, k, prec, mg ? 0 : opt.tile_rows, opt.block_order, &wp);
    if (st != ER_OK) {
        free_workspace(&g);
        return st;
    }
    Workspace &w = *wp;
    if (prec == ER_FP32_REFINE) {
        st = fp32_prepare(g, w, Yt, Z);
        if (st != ER_OK) return st;
    }
    ER_CUDA(cudaEventRecord(w.ev, us));
    ER_CUDA(cudaStreamWaitEvent(w.s, w.ev, 0));
    std::vector<double> resid((size_t)k);
    w.h_resid = resid.data();
    st = mg ? mg_solve_core(g, w, Yt, Z, opt, stats, t0) : solve_core(g, w, Yt, Z, prec, opt, stats, t0);
    w.h_resid = nullptr;
    return st;
}

// The solve loop on a prepared workspace (stream w.s, poll buffer w.h_poll).  Launches
// kernels and copies only; graphs and event timing only when opt asks for them.
er_status solve_core(const GridDev &g, Workspace &w, const void *Yt, void *Z, er_precision prec,
                     const er_solve_opts &opt, er_solve_stats *stats, std::chrono::steady_clock::time_point t0) {
    const int k = w.k;
    er_status st = ER_OK;
    const bool fp32 = prec == ER_FP32_REFINE;
    const double tol = opt.tol;
    ER_CUDA(cudaMemsetAsync(w.ints + w.k + w.til.n_colblk, 0, sizeof(int), w.s));
    Prof pf;
    pf.on = opt.profile != 0;
    const bool use_graph = opt.use_graph && !pf.on;

    if (fp32) {
        fp32_init(g, w, Yt, Z, tol, &pf);
    } else {
        auto a = base_args<double, double>(g, w, tol);
        a.b_in = (const double *)Yt; a.r_out = (double *)w.r[0]; a.x = (double *)Z; a.p_out = (double *)w.p[0];
        launch(k_stream<double, MODE_INIT>, a, w, &pf, ER_PASS_OTHER);
    }
    ER_CUDA(cudaGetLastError());

    auto iterate = [&](int cur, Prof *p) {
        return fp32 ? fp32_iterate(g, w, Z, tol, cur, p) : fp64_iterate(g, w, Z, tol, cur, p);
    };
    // FP32 form: fold the correction into the double-float iterate and substitute the accurate residual
    auto replace = [&](int cur) {
        fp32_accum(g, w, Z, &pf);
        fp32_residual(g, w, Yt, tol, cur, 1, &pf);
    };

    int cur = 0, it = 0, n_active = 0, err = 0, replacements = 0, last_replace = 0;
    const int block = std::max(2, opt.check_every + (opt.check_every & 1));  // even: parity returns
    st = poll(w, pf, &n_active, &err);
    if (st != ER_OK) return st;
    bool done = n_active == 0;
    while (!done && !err && it < opt.maxit) {
        int todo = std::min(block, opt.maxit - it);
        if (fp32 && (todo & 1)) ++todo;  // the FP32 form updates x in iteration pairs
        const bool graphable = use_graph && todo == block;
        if (graphable) {
            if (!w.gexec || w.g_Yt != Yt || w.g_Z != Z || w.g_tol != tol || w.g_iters != block || w.g_parity != cur) {
                if (w.gexec) cudaGraphExecDestroy(w.gexec);
                w.gexec = nullptr;
                cudaGraph_t graph;
                ER_CUDA(cudaStreamBeginCapture(w.s, cudaStreamCaptureModeThreadLocal));
                int c = cur;
                for (int i = 0; i < block; ++i) c = iterate(c, nullptr);
                ER_CUDA(cudaStreamEndCapture(w.s, &graph));
                cudaError_t e = cudaGraphInstantiate(&w.gexec, graph, 0);
                cudaGraphDestroy(graph);
                if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
                w.g_Yt = Yt; w.g_Z = Z; w.g_tol = tol; w.g_iters = block; w.g_parity = cur;
            }
            ER_CUDA(cudaGraphLaunch(w.gexec, w.s));
            pf.launches[ER_PASS_A] += block;
            if (fp32) {
                pf.launches[ER_PASS_B] += block / 2;
                pf.launches[ER_PASS_B0] += block / 2;
            } else {
                pf.launches[ER_PASS_B] += block;
            }
        } else {
            for (int i = 0; i < todo; ++i) cur = iterate(cur, &pf);
        }
        it += todo;
        ER_CUDA(cudaGetLastError());
        if (fp32 && it - last_replace >= opt.replace_every) {
            replace(cur);
            ++replacements;
            last_replace = it;
        }
        st = poll(w, pf, &n_active, &err);
        if (st != ER_OK) return st;
        if (fp32 && n_active == 0 && last_replace != it) {
            // every column's recursive residual meets tol: the accurate residual decides
            replace(cur);
            ++replacements;
            last_replace = it;
            st = poll(w, pf, &n_active, &err);
            if (st != ER_OK) return st;
        }
        done = n_active == 0;
    }
    if (fp32 && last_replace != it) {  // fold the last correction in
        replace(cur);
        ++replacements;
    }
    // final accurate residual (record only)
    if (fp32) {
        fp32_residual(g, w, Yt, tol, 1 - cur, 0, &pf);
        fp32_final(g, w, Z, &pf);
    } else {
        fp64_residual(g, w, Yt, Z, tol, w.q, &pf);
        auto a = base_args<double, double>(g, w, tol);
        a.x = (double *)Z;
        launch(k_stream<double, MODE_UNSCALE>, a, w, &pf, ER_PASS_OTHER);
    }
    ER_CUDA(cudaGetLastError());
    double *resid = w.h_resid;
    ER_CUDA(cudaMemcpyAsync(resid, w.scal + 4 * k, (size_t)k * sizeof(double), cudaMemcpyDeviceToHost, w.s));
    ER_CUDA(cudaMemcpyAsync(w.h_poll, w.ints + w.k + w.til.n_colblk, sizeof(int), cudaMemcpyDeviceToHost, w.s));
    ER_CUDA(cudaStreamSynchronize(w.s));
    flush_prof(w, pf);
    err |= w.h_poll[0];
    int ok_cols = 0;
    double mx = 0.0;
    for (int j = 0; j < k; ++j) {
        mx = std::max(mx, resid[j]);
        ok_cols += (resid[j] <= tol);
    }
    if (stats) {
        stats->iterations = it;
        stats->sweeps = replacements;
        stats->converged_cols = ok_cols;
        stats->k = k;
        stats->max_rel_residual = mx;
        stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        for (int i = 0; i < ER_N_PASS; ++i) {
            stats->launches[i] = pf.launches[i];
            stats->kernel_ms[i] = pf.ms[i];
        }
    }
    if (err) return fail(ER_ERR_TIMEOUT, "a bounded wait on a bulk copy expired inside a solver kernel");
    if (!done) {
        return fail(ER_ERR_NOT_CONVERGED,
                    std::to_string(n_active) + " columns above tol after " + std::to_string(it) + " iterations");
    }
    return ER_OK;
}

}  // namespace er

extern "C" {

er_solve_opts er_default_solve_opts(er_precision prec) {
    er_solve_opts o{};
    o.tol = prec == ER_FP64 ? 1e-12 : 1e-7;
    o.maxit = 20000;
    o.check_every = 10;
    o.replace_every = 50;
    o.use_graph = 1;
    o.profile = 0;
    o.tile_rows = 0;
    o.block_order = 0;
    o.precond = 0;
    return o;
}

er_status er_solve(er_grid *g, const void *Yt, void *Z, int32_t k, er_precision prec, const er_solve_opts *opts,
                   er_solve_stats *stats, void *stream) {
    return er::solve(g, Yt, Z, k, prec, opts, stats, (cudaStream_t)stream);
}

}  // extern "C"
