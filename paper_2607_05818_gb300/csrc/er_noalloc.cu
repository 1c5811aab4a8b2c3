// er_solve_noalloc: the FP64 solve on a workspace that lives in a static device array,
// for callers that must not allocate device memory when they solve.
//
// The workspace (residual, two search directions, the stencil product, per-tile partial
// dot products, per-column scalars, flags and tickets) is carved out of one file-scope
// __device__ array of fixed size.  The CUDA runtime loads the module that holds it lazily,
// on the first lookup of its address; er_grid_create does that lookup for its device
// (noalloc_prepare), so the array is committed when the first grid on a device is created
// and held until the process exits, and no er_solve_noalloc call loads a module or commits
// memory.  All calls share the array, so the counters and flags it carries are cleared at
// the start of each call; the call is blocking and serialised by a process-wide lock, and a
// call must not overlap on the GPU with another use of the array.
#include <chrono>
#include <mutex>

#include "er_common.cuh"

namespace er {

constexpr int64_t kNaMaxElems = 262144;    // n * k of the FP64 vectors
constexpr int64_t kNaMaxPartials = 65536;  // spatial tiles * k
constexpr int kNaMaxK = 4096;
constexpr int kNaMaxColblk = 512;

constexpr size_t na_round(size_t b) { return (b + 255) & ~(size_t)255; }
constexpr size_t kNaVec = na_round(kNaMaxElems * sizeof(double));
constexpr size_t kNaPart = na_round(kNaMaxPartials * sizeof(double));
constexpr size_t kNaScal = na_round(6 * (size_t)kNaMaxK * sizeof(double));
constexpr size_t kNaInts = na_round(((size_t)kNaMaxK + kNaMaxColblk + 1) * sizeof(int));
constexpr size_t kNaCnt = na_round((size_t)kNaMaxColblk * sizeof(unsigned));
constexpr size_t kNaBytes = 4 * kNaVec + kNaPart + kNaScal + kNaInts + kNaCnt;  // about 9.1 MB

static __device__ __align__(256) unsigned char g_na_scratch[kNaBytes];

static std::mutex g_na_mu;      // serialises the solves that use the array
static std::mutex g_na_setup_mu;
static void *g_na_ptr[64];      // device address of g_na_scratch, per device ordinal

// Once per device, with that device current: the host-side name of the array is not a
// device address, so ask the runtime for it.
static er_status na_setup(int dev, unsigned char **out) {
    if (dev < 0 || dev >= 64) return fail(ER_ERR_INVALID_ARG, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_na_setup_mu);
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-alloc scratch)");
        g_na_ptr[dev] = p;
    }
    if (out) *out = static_cast<unsigned char *>(g_na_ptr[dev]);
    return ER_OK;
}

er_status noalloc_prepare(int device) { return na_setup(device, nullptr); }

static er_status solve_noalloc(er_grid *gg, const void *Yt, void *Z, int32_t k, const er_solve_opts *o,
                               er_solve_stats *stats, cudaStream_t s) {
    auto t0 = std::chrono::steady_clock::now();
    if (!gg) return fail(ER_ERR_INVALID_ARG, "grid is NULL");
    er_solve_opts opt = o ? *o : er_default_solve_opts(ER_FP64);
    er_status st = check_solve_args(Yt, Z, k, ER_FP64, opt);
    if (st != ER_OK) return st;
    opt.use_graph = 0;
    opt.profile = 0;
    const GridDev &g = gg->d;
    const Tiling til = make_tiling(g, k, 8, opt.tile_rows, opt.block_order);
    if (k > kNaMaxK || g.n * (int64_t)k > kNaMaxElems || (int64_t)til.n_spatial * k > kNaMaxPartials ||
        til.n_colblk > kNaMaxColblk)
        return fail(ER_ERR_INVALID_ARG,
                    "er_solve_noalloc: n*k must be <= 262144 and k <= 4096 (the static workspace is about 9.1 MB)");
    std::lock_guard<std::mutex> glock(g_na_mu);
    std::lock_guard<std::mutex> lock(gg->mu);
    ER_CUDA(cudaSetDevice(g.device));
    unsigned char *base = nullptr;
    st = na_setup(g.device, &base);
    if (st != ER_OK) return st;

    Workspace w;
    w.k = k;
    w.prec = ER_FP64;
    w.til = til;
    unsigned char *p = base;
    w.r[0] = p; p += kNaVec;
    w.p[0] = p; p += kNaVec;
    w.p[1] = p; p += kNaVec;
    w.q = p; p += kNaVec;
    w.part = reinterpret_cast<double *>(p); p += kNaPart;
    w.scal = reinterpret_cast<double *>(p); p += kNaScal;
    w.ints = reinterpret_cast<int *>(p); p += kNaInts;
    w.counter = reinterpret_cast<unsigned *>(p);
    w.s = s;
    int h_poll[kNaMaxColblk + 1];
    double h_resid[kNaMaxK];
    w.h_poll = h_poll;
    w.h_resid = h_resid;
    // the array keeps the previous call's contents: tickets, flags and counts start at zero
    ER_CUDA(cudaMemsetAsync(w.ints, 0, kNaInts, s));
    ER_CUDA(cudaMemsetAsync(w.counter, 0, kNaCnt, s));
    st = solve_core(g, w, Yt, Z, ER_FP64, opt, stats, t0);
    // an error can return before the stream drains: the next call's clearing of the array
    // must not overlap kernels of this one still in flight, so wait while the lock is held
    if (st != ER_OK) cudaStreamSynchronize(s);
    w.r[0] = w.p[0] = w.p[1] = w.q = nullptr;  // nothing here belongs to the workspace cache
    w.part = w.scal = nullptr;
    w.ints = nullptr;
    w.counter = nullptr;
    w.h_poll = nullptr;
    w.h_resid = nullptr;
    w.s = nullptr;
    return st;
}

}  // namespace er

extern "C" er_status er_solve_noalloc(er_grid *g, const void *Yt, void *Z, int32_t k, const er_solve_opts *opts,
                                      er_solve_stats *stats, void *stream) {
    return er::solve_noalloc(g, Yt, Z, k, opts, stats, (cudaStream_t)stream);
}
