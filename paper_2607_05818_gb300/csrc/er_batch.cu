// Batching form: the all-node R map of many uneven networks, in shared launches
// (Jacobi, precond 0; below) or as persistent level-synchronous multigrid launches under a
// device-side graph loop (precond 1; mg_batch_solve in er_mg.cu).
//
// Every network keeps its own grid (coefficients, TSV CSR), its own vectors and its own
// per-column CG scalars, but each pass (A, B/B0, accurate residual, initialisation,
// accumulation, final Z) is ONE launch over a work list of (network, block) pairs, so
// small networks that could not fill the GPU alone run side by side.  A poll period of
// iterations is captured once into a CUDA graph and replayed; when networks finish, the
// work list shrinks and the graph is captured again.  The arithmetic is the FP32 form
// of er_solve (FP32 Jacobi-PCG on the FP32-rounded network, double-float iterate with
// the accurate residual substituted every replace_every iterations, accurate stopping test).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <mutex>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "er_common.cuh"

namespace er {


namespace {

struct DevBuf {
    void *p = nullptr;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
};

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

static er_status batch_solve(er_grid *const *grids, int32_t n, int32_t k, uint64_t seed, er_precision prec,
                             const int32_t *tile_rows, double *const *R_out, const er_solve_opts *o,
                             er_batch_stats *stats, cudaStream_t us) {
    auto t0 = std::chrono::steady_clock::now();
    if (!grids || n < 1 || !R_out) return fail(ER_ERR_INVALID_ARG, "grids, n and R_out are required");
    if (k < 4 || (k & 3)) return fail(ER_ERR_INVALID_ARG, "k must be a positive multiple of 4");
    if (prec != ER_FP32_REFINE) return fail(ER_ERR_INVALID_ARG, "the batching form runs the FP32 form");
    er_solve_opts opt = o ? *o : er_default_solve_opts(prec);
    if (!(opt.tol > 0.0) || opt.maxit < 1 || opt.check_every < 1 || opt.replace_every < 1)
        return fail(ER_ERR_INVALID_ARG, "bad solve options");
    if (opt.precond != 0 && opt.precond != 1) return fail(ER_ERR_INVALID_ARG, "precond must be 0 (Jacobi) or 1 (multigrid)");
    const int dev = grids[0] ? grids[0]->d.device : 0;
    for (int c = 0; c < n; ++c) {
        if (!grids[c] || !R_out[c]) return fail(ER_ERR_INVALID_ARG, "NULL grid or R_out entry");
        if (grids[c]->d.device != dev) return fail(ER_ERR_INVALID_ARG, "all grids must be on one device");
        if (tile_rows && tile_rows[c] < 0) return fail(ER_ERR_INVALID_ARG, "negative tile_rows entry");
        for (int d = 0; d < c && opt.precond == 1; ++d)
            if (grids[d] == grids[c]) return fail(ER_ERR_INVALID_ARG, "a grid appears twice (precond 1 solves networks concurrently)");
    }
    ER_CUDA(cudaSetDevice(dev));
    if (opt.precond == 1) return mg_batch_solve(grids, n, k, seed, tile_rows, R_out, opt, stats, us, t0);
    cudaStream_t s = nullptr;
    ER_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    struct StreamGuard {
        cudaStream_t s;
        ~StreamGuard() { cudaStreamDestroy(s); }
    } sg{s};
    cudaEvent_t ev;
    ER_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    ER_CUDA(cudaEventRecord(ev, us));
    ER_CUDA(cudaStreamWaitEvent(s, ev, 0));
    cudaEventDestroy(ev);

    // ---- layout of the batch workspace
    std::vector<Tiling> til(n);
    std::vector<size_t> off_vec(n), off_part(n), off_int(n), off_cnt(n);
    size_t nvec = 0, npart = 0, nint = 0, ncnt = 0;
    int64_t nodes = 0, total_ctas = 0;
    for (int c = 0; c < n; ++c) {
        const GridDev &g = grids[c]->d;
        til[c] = make_tiling(g, k, 4, tile_rows ? tile_rows[c] : opt.tile_rows, opt.block_order);
        off_vec[c] = nvec;
        nvec += align256((size_t)g.n * k * 4) / 4;  // in floats
        off_part[c] = npart;
        npart += (size_t)til[c].n_spatial * k;
        off_int[c] = nint;
        nint += (size_t)k + til[c].n_colblk + 1;
        off_cnt[c] = ncnt;
        ncnt += (size_t)til[c].n_colblk;
        nodes += g.n - g.n_floating;
        total_ctas += til[c].n_ctas();
    }
    if (total_ctas >= INT32_MAX) return fail(ER_ERR_INVALID_ARG, "batch too large");
    DevBuf b_b, b_c, b_r0, b_r1, b_p0, b_p1, b_xhl, b_part, b_scal, b_int, b_cnt, b_items, b_work;
    const size_t vbytes = nvec * 4;
    ER_CUDA(cudaMalloc(&b_b.p, vbytes));
    ER_CUDA(cudaMalloc(&b_c.p, vbytes));
    ER_CUDA(cudaMalloc(&b_r0.p, vbytes));
    ER_CUDA(cudaMalloc(&b_r1.p, vbytes));
    ER_CUDA(cudaMalloc(&b_p0.p, vbytes));
    ER_CUDA(cudaMalloc(&b_p1.p, vbytes));
    ER_CUDA(cudaMalloc(&b_xhl.p, vbytes * 2));
    ER_CUDA(cudaMalloc(&b_part.p, std::max<size_t>(npart, 1) * 8));
    ER_CUDA(cudaMalloc(&b_scal.p, (size_t)n * 6 * k * 8));
    ER_CUDA(cudaMalloc(&b_int.p, nint * 4));
    ER_CUDA(cudaMalloc(&b_cnt.p, ncnt * 4));
    ER_CUDA(cudaMemsetAsync(b_int.p, 0, nint * 4, s));
    ER_CUDA(cudaMemsetAsync(b_cnt.p, 0, ncnt * 4, s));
    ER_CUDA(cudaMalloc(&b_items.p, (size_t)n * sizeof(BatchItem)));
    ER_CUDA(cudaMalloc(&b_work.p, (size_t)total_ctas * sizeof(int2)));

    // ---- per-network items (tensor maps, arguments, vectors)
    std::vector<BatchItem> items(n);
    auto fvec = [&](DevBuf &b, int c) { return reinterpret_cast<float *>(b.p) + off_vec[c]; };
    for (int c = 0; c < n; ++c) {
        const GridDev &g = grids[c]->d;
        BatchItem &it = items[c];
        std::memset(&it, 0, sizeof(it));
        it.r[0] = fvec(b_r0, c); it.r[1] = fvec(b_r1, c);
        it.p[0] = fvec(b_p0, c); it.p[1] = fvec(b_p1, c);
        it.c = fvec(b_c, c);
        it.b = fvec(b_b, c);
        it.xhl = reinterpret_cast<float2 *>(b_xhl.p) + off_vec[c];
        er_status st = ER_OK;
        const void *bases[8] = {it.r[0], it.r[1], it.p[0], it.p[1], it.c, it.xhl, it.b, g.coef32};
        for (int m = 0; m < 8 && st == ER_OK; ++m)
            st = m == 7 ? fp32_make_map(&it.tm[m], false, bases[m], 4, 4, g)
                        : fp32_make_map(&it.tm[m], m == 5, bases[m], k, 32, g);  // xhl: 8-byte pairs
        if (st != ER_OK) return st;
        KArgs<float, float> &a = it.a;
        a.T_ = g.T; a.W = g.W; a.H = g.H; a.k = k;
        a.tiles_x = til[c].tiles_x; a.tiles_y = til[c].tiles_y; a.rows = til[c].rows;
        a.n_spatial = til[c].n_spatial; a.n_colblk = til[c].n_colblk; a.cb_fast = til[c].cb_fast;
        a.coef = reinterpret_cast<const float4 *>(g.coef32); a.tsv_g32 = g.tsv_g32;
        a.tsv_ptr = g.tsv_ptr; a.tsv_nbr = g.tsv_nbr; a.dinvs = g.dinvs;
        double *sc = reinterpret_cast<double *>(b_scal.p) + (size_t)c * 6 * k;
        a.alpha = sc; a.beta = sc + k; a.rho = sc + 2 * k; a.rho0 = sc + 3 * k; a.resid = sc + 4 * k;
        a.alpha_prev = sc + 5 * k;
        int *in = reinterpret_cast<int *>(b_int.p) + off_int[c];
        a.active = in; a.col_active = in + k; a.err = in + k + til[c].n_colblk;
        a.counter = reinterpret_cast<unsigned *>(b_cnt.p) + off_cnt[c];
        a.part = reinterpret_cast<double *>(b_part.p) + off_part[c];
        a.tol = opt.tol;
    }
    ER_CUDA(cudaMemcpyAsync(b_items.p, items.data(), (size_t)n * sizeof(BatchItem), cudaMemcpyHostToDevice, s));

    // ---- sketches (network c uses seed + c)
    for (int c = 0; c < n; ++c) {
        er_status st = sketch(grids[c], k, seed + (uint64_t)c, ER_FP32_REFINE, (void *)items[c].b, s);
        if (st != ER_OK) return st;
    }

    // ---- work list of the active networks
    std::vector<int2> work;
    std::vector<char> live(n, 1);
    auto build_work = [&]() -> er_status {
        work.clear();
        for (int c = 0; c < n; ++c)
            if (live[c])
                for (int64_t b = 0; b < til[c].n_ctas(); ++b) work.push_back(make_int2(c, (int)b));
        if (!work.empty())
            ER_CUDA(cudaMemcpyAsync(b_work.p, work.data(), work.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
        ER_CUDA(cudaStreamSynchronize(s));  // the host vector is reused
        return ER_OK;
    };
    const BatchItem *d_items = reinterpret_cast<const BatchItem *>(b_items.p);
    const int2 *d_work = reinterpret_cast<const int2 *>(b_work.p);
    int launches = 0, captures = 0;
    auto pass = [&](int mode, int cur, int rmode) -> er_status {
        ++launches;
        return fp32_batch_pass(mode, d_items, d_work, (int)work.size(), cur, rmode, s);
    };
    std::vector<int> h_int(nint);
    std::vector<int> act(n), unconv(n);
    auto poll = [&](std::vector<int> &out, int *err) -> er_status {
        ER_CUDA(cudaMemcpyAsync(h_int.data(), b_int.p, nint * 4, cudaMemcpyDeviceToHost, s));
        ER_CUDA(cudaStreamSynchronize(s));
        *err = 0;
        for (int c = 0; c < n; ++c) {
            int sum = 0;
            for (int b = 0; b < til[c].n_colblk; ++b) sum += h_int[off_int[c] + k + b];
            out[c] = sum;
            *err |= h_int[off_int[c] + k + til[c].n_colblk];
        }
        return ER_OK;
    };

    er_status st = build_work();
    if (st != ER_OK) return st;
    st = pass(MODE_INIT, 0, 0);
    if (st != ER_OK) return st;
    int err = 0;
    st = poll(act, &err);
    if (st != ER_OK) return st;
    for (int c = 0; c < n; ++c) live[c] = act[c] > 0;
    st = build_work();
    if (st != ER_OK) return st;

    const int block = std::max(2, opt.check_every + (opt.check_every & 1));
    int it = 0, cur = 0, replacements = 0, last_replace = 0;
    cudaGraphExec_t gexec = nullptr;
    struct GraphGuard {
        cudaGraphExec_t *g;
        ~GraphGuard() {
            if (*g) cudaGraphExecDestroy(*g);
        }
    } gg{&gexec};
    size_t graph_work = (size_t)-1;
    auto replace = [&]() -> er_status {
        er_status r = pass(MODE_ACCUM, 0, 0);
        if (r == ER_OK) r = pass(MODE_R, cur, 1);
        ++replacements;
        last_replace = it;
        return r;
    };
    auto any_live = [&]() { return std::any_of(live.begin(), live.end(), [](char v) { return v != 0; }); };
    while (any_live() && !err && it < opt.maxit) {
        if (opt.use_graph) {
            if (!gexec || graph_work != work.size()) {
                if (gexec) cudaGraphExecDestroy(gexec);
                gexec = nullptr;
                cudaGraph_t graph;
                ER_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
                int cc = cur;
                for (int i = 0; i < block; ++i) {
                    fp32_batch_pass(MODE_A_DOT, d_items, d_work, (int)work.size(), cc, 0, s);
                    fp32_batch_pass(cc == 1 ? MODE_B : MODE_B0, d_items, d_work, (int)work.size(), cc, 0, s);
                    cc = 1 - cc;
                }
                ER_CUDA(cudaStreamEndCapture(s, &graph));
                cudaError_t e = cudaGraphInstantiate(&gexec, graph, 0);
                cudaGraphDestroy(graph);
                if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate(batch)");
                graph_work = work.size();
                ++captures;
            }
            ER_CUDA(cudaGraphLaunch(gexec, s));
            launches += 2 * block;
        } else {
            for (int i = 0; i < block; ++i) {
                st = pass(MODE_A_DOT, cur, 0);
                if (st == ER_OK) st = pass(cur == 1 ? MODE_B : MODE_B0, cur, 0);
                if (st != ER_OK) return st;
                cur = 1 - cur;
            }
        }
        it += block;
        if (it - last_replace >= opt.replace_every) {
            st = replace();
            if (st != ER_OK) return st;
            st = poll(act, &err);
        } else {
            st = poll(unconv, &err);
            if (st != ER_OK) return st;
            bool need = false;
            for (int c = 0; c < n; ++c) need |= live[c] && unconv[c] == 0;
            if (!need) continue;
            st = replace();  // some network's recursion meets tol everywhere: the accurate residual decides
            if (st != ER_OK) return st;
            st = poll(act, &err);
        }
        if (st != ER_OK) return st;
        bool changed = false;
        for (int c = 0; c < n; ++c)
            if (live[c] && act[c] == 0) {
                live[c] = 0;
                changed = true;
            }
        if (changed) {
            st = build_work();
            if (st != ER_OK) return st;
        }
    }
    const bool done = !any_live();
    // final: every network's correction folded in, accurate residual recorded, Z, R
    std::fill(live.begin(), live.end(), 1);
    st = build_work();
    if (st == ER_OK) st = pass(MODE_ACCUM, 0, 0);
    if (st == ER_OK) st = pass(MODE_R, 1 - cur, 0);
    if (st == ER_OK) st = pass(MODE_UNSCALE, 0, 0);
    for (int c = 0; c < n && st == ER_OK; ++c) st = reff_map(grids[c], items[c].c, k, ER_FP32_REFINE, R_out[c], s);
    if (st != ER_OK) return st;
    std::vector<double> resid((size_t)n * 6 * k);
    ER_CUDA(cudaMemcpyAsync(resid.data(), b_scal.p, resid.size() * 8, cudaMemcpyDeviceToHost, s));
    ER_CUDA(cudaStreamSynchronize(s));
    double mx = 0.0;
    int ok_nets = 0;
    for (int c = 0; c < n; ++c) {
        bool ok = true;
        for (int j = 0; j < k; ++j) {
            const double r = resid[(size_t)c * 6 * k + 4 * k + j];
            mx = std::max(mx, r);
            ok &= r <= opt.tol;
        }
        ok_nets += ok;
    }
    if (stats) {
        stats->n_grids = n;
        stats->iterations = it;
        stats->replacements = replacements;
        stats->converged = ok_nets;
        stats->nodes = nodes;
        stats->max_rel_residual = mx;
        stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        stats->launches = launches + 2 * n + 3;  // + sketch and map per network, final passes
        stats->graph_captures = captures;
    }
    if (err) return fail(ER_ERR_TIMEOUT, "a bounded wait on a bulk copy expired inside a batched kernel");
    if (!done) return fail(ER_ERR_NOT_CONVERGED, "maxit reached with networks still above tol");
    return ER_OK;
}

}  // namespace er

extern "C" er_status er_batch_solve(er_grid *const *grids, int32_t n, int32_t k, uint64_t seed, er_precision prec,
                                    const int32_t *tile_rows, double *const *R_out, const er_solve_opts *opts,
                                    er_batch_stats *stats, void *stream) {
    return er::batch_solve(grids, n, k, seed, prec, tile_rows, R_out, opts, stats, (cudaStream_t)stream);
}
