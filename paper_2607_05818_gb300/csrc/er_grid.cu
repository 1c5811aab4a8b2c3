// Grid assembly, JL sketch and R-map kernels, and the host-side entry points of liber.so.
//
// The network is the paper's multi-tier PDN (Sec. III-A/B): per-tier resistive meshes,
// TSV segments between adjacent tiers, pads to an ideal supply.  Its MNA matrix with the
// supply grounded is G = B^T W B + D (Sec. II-A, Eq. 1); the quantity computed is the
// Eq. 2 effective resistance of every node to the supply, R_i = (G^-1)_ii.

#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "er_internal.h"

namespace er {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

er_status fail(er_status s, const std::string &msg) {
    set_error(msg);
    return s;
}

er_status cuda_fail(cudaError_t e, const char *what) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? ER_ERR_OOM : ER_ERR_CUDA;
}

Tiling make_tiling(const GridDev &g, int k, int elem_bytes, int rows, int order) {
    Tiling t;
    t.tiles_x = (g.W + kTXI - 1) / kTXI;
    // rows per CTA: long sweeps amortise the two halo rows; short grids use fewer rows
    if (rows <= 0) rows = 64;
    if (g.H < rows) rows = g.H;
    t.cb_fast = order == 2 ? 0 : 1;
    t.rows = rows;
    t.tiles_y = (g.H + rows - 1) / rows;
    t.n_spatial = g.T * t.tiles_y * t.tiles_x;
    t.kb = kTPN * (16 / elem_bytes);
    t.n_colblk = (k + t.kb - 1) / t.kb;
    return t;
}

// ---------------------------------------------------------------------------------
// SplitMix64 output function (Steele, Lea and Flood, OOPSLA 2014): the counter-based
// generator of the sketch.  Each Rademacher sign is the top bit of one output.
__host__ __device__ inline uint64_t splitmix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

struct SketchView {
    int T, W, H;
    int64_t n, ex_slots, ey_slots;
    const double *gxr, *gyr;
    const int32_t *tsv_ptr;
    const int64_t *tsv_eid;
    const int8_t *tsv_sgn;
    const double *tsv_g;
    const int32_t *pad_ptr;
    const int64_t *pad_eid;
    const double *pad_g;
    const float2 *sq_x, *sq_y, *sq_tsv, *sq_pad;
    const uint8_t *floating;
};

// acc[v] += s * sign(e, j0 + v) for the 4 columns j0..j0+3
__device__ inline void sketch_term(double (&acc)[4], uint64_t key, int64_t e, int j0, double s) {
    const uint64_t hi = (uint64_t)e << 32;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        uint64_t h = splitmix64(key ^ (hi | (uint32_t)(j0 + v)));
        acc[v] += (h >> 63) ? -s : s;
    }
}

// Y^T[i][j] = sum over edges e at node i of sigma_e(i) sqrt(w_e) Q[j][e]; one thread per
// (node, 4 columns).  Edges are visited in canonical-id order.
template <typename T>
__global__ void __launch_bounds__(256) k_sketch(SketchView g, int k, int j_off, uint64_t key, double rk, T *Yt) {
    const int64_t nq = k / 4;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= g.n * nq) return;
    const int64_t i = tid / nq;
    const int jl = (int)(tid - i * nq) * 4;  // stored column; the sketch row hashed is j_off + jl
    const int j0 = j_off + jl;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    if (!g.floating[i]) {
        const int x = (int)(i % g.W);
        const int64_t ty = i / g.W;
        const int y = (int)(ty % g.H);
        const int t = (int)(ty / g.H);
        if (x > 0) {  // x-segment (x-1, y)-(x, y): this node is the higher end
            double w = g.gxr[i - 1];
            if (w > 0.0) sketch_term(acc, key, ((int64_t)t * g.H + y) * (g.W - 1) + x - 1, j0, -sqrt(w) * rk);
        }
        if (x < g.W - 1) {
            double w = g.gxr[i];
            if (w > 0.0) sketch_term(acc, key, ((int64_t)t * g.H + y) * (g.W - 1) + x, j0, sqrt(w) * rk);
        }
        if (y > 0) {
            double w = g.gyr[i - g.W];
            if (w > 0.0)
                sketch_term(acc, key, g.ex_slots + ((int64_t)t * (g.H - 1) + y - 1) * g.W + x, j0, -sqrt(w) * rk);
        }
        if (y < g.H - 1) {
            double w = g.gyr[i];
            if (w > 0.0)
                sketch_term(acc, key, g.ex_slots + ((int64_t)t * (g.H - 1) + y) * g.W + x, j0, sqrt(w) * rk);
        }
        for (int e = g.tsv_ptr[i]; e < g.tsv_ptr[i + 1]; ++e) {
            double s = sqrt(g.tsv_g[e]) * rk;
            sketch_term(acc, key, g.tsv_eid[e], j0, g.tsv_sgn[e] > 0 ? s : -s);
        }
        for (int e = g.pad_ptr[i]; e < g.pad_ptr[i + 1]; ++e)
            sketch_term(acc, key, g.pad_eid[e], j0, sqrt(g.pad_g[e]) * rk);
    }
    T *out = Yt + i * k + jl;
    if constexpr (sizeof(T) == 8) {
        reinterpret_cast<double2 *>(out)[0] = make_double2(acc[0], acc[1]);
        reinterpret_cast<double2 *>(out)[1] = make_double2(acc[2], acc[3]);
    } else {
        reinterpret_cast<float4 *>(out)[0] =
            make_float4((float)acc[0], (float)acc[1], (float)acc[2], (float)acc[3]);
    }
}

// FP32 sketch, the same sums without FP64 arithmetic (FP64 runs at 1/64 of the FP32 rate
// on this GPU, and the FP64 kernel above is bound by it).  Each term sqrt(w_e)/sqrt(k) is
// the double-float product of the stored {hi, lo} square root and {hi, lo} of 1/sqrt(k);
// the terms are summed per column as S + C with TwoSum (Knuth) and rounded once, so the
// output is the FP32 rounding of the sum to within rare one-ulp ties.  The sign is the top
// bit of SplitMix64; its last xor-shift leaves bit 63 unchanged and is skipped.
__device__ __forceinline__ uint32_t sketch_sign(uint64_t key, uint64_t hi, uint32_t j) {
    uint64_t z = (key ^ (hi | j)) + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return (uint32_t)(z >> 63);
}

struct SketchAcc32 {
    float S[4] = {0.f, 0.f, 0.f, 0.f}, C[4] = {0.f, 0.f, 0.f, 0.f};
    // += sigma sqrt(w) rk sign(e, j0 + v); sq = sqrt(w) as {hi, lo}, rk = 1/sqrt(k) as {hi, lo}
    __device__ __forceinline__ void term(uint64_t key, int64_t e, int j0, float2 sq, float2 rk, bool neg) {
        const float p0 = __fmul_rn(sq.x, rk.x);
        const float e0 = fmaf(sq.y, rk.x, fmaf(sq.x, rk.y, fmaf(sq.x, rk.x, -p0)));
        const float p = neg ? -p0 : p0, pe = neg ? -e0 : e0;
        const uint64_t hi = (uint64_t)e << 32;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const bool m = sketch_sign(key, hi, (uint32_t)(j0 + v)) != 0;
            const float a = m ? -p : p, ae = m ? -pe : pe;
            const float t = __fadd_rn(S[v], a);
            const float bb = __fsub_rn(t, S[v]);
            const float err = __fadd_rn(__fsub_rn(S[v], __fsub_rn(t, bb)), __fsub_rn(a, bb));
            S[v] = t;
            C[v] = __fadd_rn(C[v], __fadd_rn(err, ae));
        }
    }
};

__global__ void __launch_bounds__(256) k_sketch32(SketchView g, int k, int j_off, uint64_t key, float2 rk, float *Yt) {
    const int64_t nq = k / 4;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= g.n * nq) return;
    const int64_t i = tid / nq;
    const int jl = (int)(tid - i * nq) * 4;  // stored column; the sketch row hashed is j_off + jl
    const int j0 = j_off + jl;
    SketchAcc32 acc;
    if (!g.floating[i]) {
        const int x = (int)(i % g.W);
        const int64_t ty = i / g.W;
        const int y = (int)(ty % g.H);
        const int t = (int)(ty / g.H);
        // an absent segment has w = 0, so sqrt(w).hi = 0 (tested in FP32: no FP64 compare)
        if (x > 0) {  // x-segment (x-1, y)-(x, y): this node is the higher end
            const float2 q = g.sq_x[i - 1];
            if (q.x > 0.f) acc.term(key, ((int64_t)t * g.H + y) * (g.W - 1) + x - 1, j0, q, rk, true);
        }
        if (x < g.W - 1) {
            const float2 q = g.sq_x[i];
            if (q.x > 0.f) acc.term(key, ((int64_t)t * g.H + y) * (g.W - 1) + x, j0, q, rk, false);
        }
        if (y > 0) {
            const float2 q = g.sq_y[i - g.W];
            if (q.x > 0.f) acc.term(key, g.ex_slots + ((int64_t)t * (g.H - 1) + y - 1) * g.W + x, j0, q, rk, true);
        }
        if (y < g.H - 1) {
            const float2 q = g.sq_y[i];
            if (q.x > 0.f) acc.term(key, g.ex_slots + ((int64_t)t * (g.H - 1) + y) * g.W + x, j0, q, rk, false);
        }
        for (int e = g.tsv_ptr[i]; e < g.tsv_ptr[i + 1]; ++e)
            acc.term(key, g.tsv_eid[e], j0, g.sq_tsv[e], rk, g.tsv_sgn[e] <= 0);
        for (int e = g.pad_ptr[i]; e < g.pad_ptr[i + 1]; ++e) acc.term(key, g.pad_eid[e], j0, g.sq_pad[e], rk, false);
    }
    reinterpret_cast<float4 *>(Yt + i * k + jl)[0] =
        make_float4(__fadd_rn(acc.S[0], acc.C[0]), __fadd_rn(acc.S[1], acc.C[1]), __fadd_rn(acc.S[2], acc.C[2]),
                    __fadd_rn(acc.S[3], acc.C[3]));
}

// Error-free transformations for FP32 dot products with FP64-class accuracy:
// TwoProduct through FMA and Knuth's TwoSum (Ogita, Rump and Oishi, "Accurate sum and dot
// product", SIAM J. Sci. Comput. 2005).  The _rn intrinsics keep the compiler from fusing
// the operations into FMAs, which would break the error terms.
__device__ inline void df_add_prod(float &hi, float &lo, float a, float b) {
    float p = __fmul_rn(a, b);
    float pe = fmaf(a, b, -p);
    float t = __fadd_rn(hi, p);
    float bp = __fsub_rn(t, hi);
    float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bp)), __fsub_rn(p, bp));
    hi = t;
    lo = __fadd_rn(lo, __fadd_rn(e, pe));
}

// R_i = sum_j Z_ij^2: one warp per node, 16-byte loads strided over the row.
template <typename T>
__global__ void __launch_bounds__(256) k_reff_map(const T *Z, int64_t n, int k, const uint8_t *floating, double *R) {
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    double s;
    const T *row = Z + i * k;
    if constexpr (sizeof(T) == 8) {
        double acc = 0.0;
        for (int c = lane * 2; c < k; c += 64) {
            double2 v = *reinterpret_cast<const double2 *>(row + c);
            acc = fma(v.x, v.x, acc);
            acc = fma(v.y, v.y, acc);
        }
        s = acc;
    } else {
        float hi = 0.f, lo = 0.f;
        for (int c = lane * 4; c < k; c += 128) {
            float4 v = *reinterpret_cast<const float4 *>(row + c);
            df_add_prod(hi, lo, v.x, v.x);
            df_add_prod(hi, lo, v.y, v.y);
            df_add_prod(hi, lo, v.z, v.z);
            df_add_prod(hi, lo, v.w, v.w);
        }
        s = (double)hi + (double)lo;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) R[i] = floating[i] ? __longlong_as_double(0x7ff0000000000000LL) : s;
}

// ---------------------------------------------------------------------------------
// host-side assembly

namespace {

struct UnionFind {
    std::vector<int32_t> p;
    explicit UnionFind(int64_t n) : p((size_t)n) { std::iota(p.begin(), p.end(), 0); }
    int32_t find(int32_t a) {
        int32_t r = a;
        while (p[r] != r) r = p[r];
        while (p[a] != r) {
            int32_t nx = p[a];
            p[a] = r;
            a = nx;
        }
        return r;
    }
    void unite(int32_t a, int32_t b) {
        a = find(a);
        b = find(b);
        if (a != b) p[a] = b;
    }
};

template <typename T>
er_status upload(T **dst, const std::vector<T> &src, cudaStream_t s, int64_t *counted) {
    size_t bytes = std::max<size_t>(src.size(), 1) * sizeof(T);
    ER_CUDA(cudaMalloc((void **)dst, bytes));
    if (!src.empty()) ER_CUDA(cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    *counted += (int64_t)(src.size() * sizeof(T));
    return ER_OK;
}

bool finite_nonneg(double v) { return std::isfinite(v) && v >= 0.0; }

void free_grid_arrays(er::GridDev &d) {
    void *ptrs[] = {d.cE64, d.cS64, d.cE32, d.cS32, d.dinvs, d.tsv_ptr, d.tsv_nbr, d.tsv_c64, d.tsv_c32,
                    d.gxr, d.gyr, d.tsv_eid, d.tsv_sgn, d.tsv_g, d.pad_ptr, d.pad_eid, d.pad_g, d.floating,
                    d.coef32, d.tsv_g32, d.aux, d.sq_x, d.sq_y, d.sq_tsv, d.sq_pad};
    for (void *p : ptrs)
        if (p) cudaFree(p);
}

}  // namespace

er_status grid_create(const er_tier *tiers, int32_t n_tiers, const er_tsv *tsv, int64_t n_tsv,
                      const er_pad *pads, int64_t n_pads, const er_options *opt, cudaStream_t stream,
                      er_grid **out) {
    if (!out) return fail(ER_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!tiers || n_tiers < 1) return fail(ER_ERR_INVALID_ARG, "need at least one tier");
    if (n_tsv < 0 || n_pads < 0) return fail(ER_ERR_INVALID_ARG, "negative TSV or pad count");
    if ((n_tsv > 0 && !tsv) || (n_pads > 0 && !pads)) return fail(ER_ERR_INVALID_ARG, "NULL TSV/pad array");
    const int T = n_tiers, W = tiers[0].W, H = tiers[0].H;
    if (W < 1 || H < 1) return fail(ER_ERR_INVALID_ARG, "tier sizes must be positive");
    for (int t = 0; t < T; ++t) {
        if (tiers[t].W != W || tiers[t].H != H) return fail(ER_ERR_INVALID_ARG, "all tiers must share W and H");
        if ((W > 1 && !tiers[t].gx) || (H > 1 && !tiers[t].gy)) return fail(ER_ERR_INVALID_ARG, "NULL tier conductances");
    }
    const int64_t n = (int64_t)T * W * H;
    if (n >= (int64_t)INT32_MAX) return fail(ER_ERR_INVALID_ARG, "more than 2^31-1 nodes");
    if (n_pads == 0) return fail(ER_ERR_NO_SUPPLY, "the network has no pad: G is singular");
    // per-node raw conductances and the diagonal of G
    std::vector<double> gxr((size_t)n, 0.0), gyr((size_t)n, 0.0), diag((size_t)n, 0.0);
    UnionFind uf(n + 1);  // node n is the supply
    for (int t = 0; t < T; ++t)
        for (int y = 0; y < H; ++y) {
            for (int x = 0; x + 1 < W; ++x) {
                double w = tiers[t].gx[(size_t)y * (W - 1) + x];
                if (!finite_nonneg(w)) return fail(ER_ERR_INVALID_ARG, "bad x-segment conductance");
                int64_t i = ((int64_t)t * H + y) * W + x;
                gxr[i] = w;
                diag[i] += w;
                diag[i + 1] += w;
                if (w > 0) uf.unite((int32_t)i, (int32_t)(i + 1));
            }
            if (y + 1 < H)
                for (int x = 0; x < W; ++x) {
                    double w = tiers[t].gy[(size_t)y * W + x];
                    if (!finite_nonneg(w)) return fail(ER_ERR_INVALID_ARG, "bad y-segment conductance");
                    int64_t i = ((int64_t)t * H + y) * W + x;
                    gyr[i] = w;
                    diag[i] += w;
                    diag[i + W] += w;
                    if (w > 0) uf.unite((int32_t)i, (int32_t)(i + W));
                }
        }
    std::vector<int32_t> tcount((size_t)n + 1, 0), pcount((size_t)n + 1, 0);
    for (int64_t e = 0; e < n_tsv; ++e) {
        const er_tsv &s = tsv[e];
        if (s.tier < 0 || s.tier >= T - 1 || s.x < 0 || s.x >= W || s.y < 0 || s.y >= H)
            return fail(ER_ERR_INVALID_ARG, "TSV index out of range (tier must be < T-1)");
        if (!(std::isfinite(s.g) && s.g > 0)) return fail(ER_ERR_INVALID_ARG, "TSV conductance must be positive");
        int64_t a = ((int64_t)s.tier * H + s.y) * W + s.x, b = a + (int64_t)W * H;
        diag[a] += s.g;
        diag[b] += s.g;
        uf.unite((int32_t)a, (int32_t)b);
        tcount[a + 1]++;
        tcount[b + 1]++;
    }
    for (int64_t e = 0; e < n_pads; ++e) {
        const er_pad &p = pads[e];
        if (p.tier < 0 || p.tier >= T || p.x < 0 || p.x >= W || p.y < 0 || p.y >= H)
            return fail(ER_ERR_INVALID_ARG, "pad index out of range");
        if (!(std::isfinite(p.g) && p.g > 0)) return fail(ER_ERR_INVALID_ARG, "pad conductance must be positive");
        int64_t a = ((int64_t)p.tier * H + p.y) * W + p.x;
        diag[a] += p.g;
        uf.unite((int32_t)a, (int32_t)n);
        pcount[a + 1]++;
    }
    const int32_t sroot = uf.find((int32_t)n);
    std::vector<uint8_t> floating((size_t)n);
    std::vector<double> dinvs((size_t)n);
    int64_t n_float = 0;
    for (int64_t i = 0; i < n; ++i) {
        floating[i] = uf.find((int32_t)i) != sroot;
        n_float += floating[i];
        dinvs[i] = floating[i] ? 0.0 : 1.0 / std::sqrt(diag[i]);
    }
    // scaled couplings
    std::vector<double> cE((size_t)n, 0.0), cS((size_t)n, 0.0);
    for (int64_t i = 0; i < n; ++i) {
        int x = (int)(i % W), y = (int)((i / W) % H);
        if (x + 1 < W) cE[i] = gxr[i] * dinvs[i] * dinvs[i + 1];
        if (y + 1 < H) cS[i] = gyr[i] * dinvs[i] * dinvs[i + W];
    }
    // TSV CSR (both directions) and pad CSR
    for (int64_t i = 0; i < n; ++i) {
        tcount[i + 1] += tcount[i];
        pcount[i + 1] += pcount[i];
    }
    const int64_t nnz = tcount[n];
    std::vector<int32_t> tnbr((size_t)nnz);
    std::vector<double> tc((size_t)nnz), tg((size_t)nnz);
    std::vector<int64_t> teid((size_t)nnz);
    std::vector<int8_t> tsgn((size_t)nnz);
    std::vector<int32_t> tfill(tcount.begin(), tcount.end() - 1);
    const int64_t ex = (int64_t)T * H * (W - 1), ey = (int64_t)T * (H - 1) * W;
    for (int64_t e = 0; e < n_tsv; ++e) {
        const er_tsv &s = tsv[e];
        int64_t a = ((int64_t)s.tier * H + s.y) * W + s.x, b = a + (int64_t)W * H;
        double c = s.g * dinvs[a] * dinvs[b];
        int32_t ka = tfill[a]++, kb = tfill[b]++;
        tnbr[ka] = (int32_t)b; tc[ka] = c; tg[ka] = s.g; teid[ka] = ex + ey + e; tsgn[ka] = 1;
        tnbr[kb] = (int32_t)a; tc[kb] = c; tg[kb] = s.g; teid[kb] = ex + ey + e; tsgn[kb] = -1;
    }
    std::vector<int64_t> peid((size_t)n_pads);
    std::vector<double> pg((size_t)n_pads);
    std::vector<int32_t> pfill(pcount.begin(), pcount.end() - 1);
    for (int64_t e = 0; e < n_pads; ++e) {
        const er_pad &p = pads[e];
        int64_t a = ((int64_t)p.tier * H + p.y) * W + p.x;
        int32_t ka = pfill[a]++;
        peid[ka] = ex + ey + n_tsv + e;
        pg[ka] = p.g;
    }
    std::vector<float> cE32(cE.begin(), cE.end()), cS32(cS.begin(), cS.end()), tc32(tc.begin(), tc.end());
    // FP32 form: conductances rounded to FP32 once; the diagonal is summed from the rounded
    // values in FP64 so the Laplacian rows stay exact; floating nodes get all-zero entries
    std::vector<float> coef((size_t)n * 4, 0.0f), tg32((size_t)nnz, 0.0f);
    {
        std::vector<double> pad_tot((size_t)n, 0.0), d32((size_t)n, 0.0);
        for (int64_t e = 0; e < n_pads; ++e) {
            const er_pad &p = pads[e];
            pad_tot[((int64_t)p.tier * H + p.y) * W + p.x] += p.g;
        }
        for (int64_t i = 0; i < n; ++i) {
            if (floating[i]) continue;
            const int x = (int)(i % W), y = (int)((i / W) % H);
            const float ge = x + 1 < W ? (float)gxr[i] : 0.0f, gs = y + 1 < H ? (float)gyr[i] : 0.0f;
            const float gp = (float)pad_tot[i];
            coef[4 * i + 1] = ge;
            coef[4 * i + 2] = gs;
            coef[4 * i + 3] = gp;
            d32[i] += (double)ge + (double)gs + (double)gp;
            if (x + 1 < W) d32[i + 1] += (double)ge;
            if (y + 1 < H) d32[i + W] += (double)gs;
        }
        for (int64_t i = 0; i < n; ++i)
            for (int32_t e = tcount[i]; e < tcount[i + 1]; ++e) {
                if (floating[i]) continue;
                tg32[e] = (float)tg[e];
                d32[i] += (double)tg32[e];
            }
        // 1/d, negated at nodes with TSV segments (a flag the stencil tests instead of the CSR)
        for (int64_t i = 0; i < n; ++i) {
            const float dv = floating[i] ? 0.0f : (float)(1.0 / d32[i]);
            coef[4 * i] = (!floating[i] && tcount[i + 1] > tcount[i]) ? -dv : dv;
        }
    }

    // all host-side validation is done: now touch the device
    int device = (opt && opt->device >= 0) ? opt->device : -1;
    if (device >= 0) ER_CUDA(cudaSetDevice(device));
    ER_CUDA(cudaGetDevice(&device));
    // the no-allocation solve's static workspace on this device: resolved (its module loaded,
    // its memory committed) here, at set-up, so that no er_solve_noalloc call does it
    {
        const er_status ps = noalloc_prepare(device);
        if (ps != ER_OK) return ps;
    }
    er_grid *g = new er_grid();
    GridDev &d = g->d;
    d.T = T; d.W = W; d.H = H; d.n = n;
    d.n_floating = n_float; d.n_tsv = n_tsv; d.n_pads = n_pads;
    d.ex_slots = ex; d.ey_slots = ey; d.n_edges = ex + ey + n_tsv + n_pads;
    d.device = device;
    er_status st = ER_OK;
#define UP(dst, src) if (st == ER_OK) st = upload(&d.dst, src, stream, &d.h2d_bytes)
    UP(cE64, cE); UP(cS64, cS); UP(cE32, cE32); UP(cS32, cS32); UP(dinvs, dinvs);
    UP(tsv_ptr, tcount); UP(tsv_nbr, tnbr); UP(tsv_c64, tc); UP(tsv_c32, tc32);
    UP(gxr, gxr); UP(gyr, gyr); UP(tsv_eid, teid); UP(tsv_sgn, tsgn); UP(tsv_g, tg);
    UP(pad_ptr, pcount); UP(pad_eid, peid); UP(pad_g, pg); UP(floating, floating);
    UP(coef32, coef); UP(tsv_g32, tg32);
    {
        // sqrt(w) as {hi, lo}: hi = sqrt(w) rounded to FP32, lo = the remainder rounded to FP32
        auto pairs = [](const std::vector<double> &w) {
            std::vector<float2> o(w.size());
            for (size_t i = 0; i < w.size(); ++i) {
                const double r = w[i] > 0.0 ? std::sqrt(w[i]) : 0.0;
                const float h = (float)r;
                o[i] = make_float2(h, (float)(r - (double)h));
            }
            return o;
        };
        UP(sq_x, pairs(gxr)); UP(sq_y, pairs(gyr)); UP(sq_tsv, pairs(tg)); UP(sq_pad, pairs(pg));
    }
#undef UP
    if (st == ER_OK) {
        cudaError_t e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) st = cuda_fail(e, "cudaStreamSynchronize(grid upload)");
    }
    if (st != ER_OK) {
        free_grid_arrays(d);
        delete g;
        return st;
    }
    *out = g;
    if (n_float > 0) {
        set_error(std::to_string(n_float) + " floating nodes (R = +inf)");
        return ER_WARN_FLOATING;
    }
    return ER_OK;
}

SketchView sketch_view(const GridDev &d) {
    SketchView v;
    v.T = d.T; v.W = d.W; v.H = d.H; v.n = d.n; v.ex_slots = d.ex_slots; v.ey_slots = d.ey_slots;
    v.gxr = d.gxr; v.gyr = d.gyr; v.tsv_ptr = d.tsv_ptr; v.tsv_eid = d.tsv_eid; v.tsv_sgn = d.tsv_sgn;
    v.tsv_g = d.tsv_g; v.pad_ptr = d.pad_ptr; v.pad_eid = d.pad_eid; v.pad_g = d.pad_g;
    v.sq_x = d.sq_x; v.sq_y = d.sq_y; v.sq_tsv = d.sq_tsv; v.sq_pad = d.sq_pad;
    v.floating = d.floating;
    return v;
}

static bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

er_status check_nk(const er_grid *g, int32_t k, const void *p, const char *name) {
    if (!g) return fail(ER_ERR_INVALID_ARG, "grid is NULL");
    if (k < 4 || (k & 3)) return fail(ER_ERR_INVALID_ARG, "k must be a positive multiple of 4");
    if (k > (1 << 20)) return fail(ER_ERR_INVALID_ARG, "k too large");
    if (!p) return fail(ER_ERR_INVALID_ARG, std::string(name) + " is NULL");
    if (!aligned16(p)) return fail(ER_ERR_INVALID_ARG, std::string(name) + " must be 16-byte aligned");
    return ER_OK;
}

// columns j0 .. j0 + k_local - 1 of the k_total-column sketch (scale 1/sqrt(k_total)), stored
// as a [n][k_local] array
er_status sketch_cols(er_grid *g, int32_t k_total, int32_t j0, int32_t k_local, uint64_t seed, er_precision prec,
                      void *Yt, cudaStream_t s) {
    er_status st = check_nk(g, k_local, Yt, "Yt");
    if (st != ER_OK) return st;
    if (prec != ER_FP64 && prec != ER_FP32_REFINE) return fail(ER_ERR_INVALID_ARG, "bad precision");
    if (j0 < 0 || k_total < 1 || (int64_t)j0 + k_local > (int64_t)k_total)
        return fail(ER_ERR_INVALID_ARG, "need 0 <= j0 and j0 + k_local <= k_total");
    const GridDev &d = g->d;
    ER_CUDA(cudaSetDevice(d.device));
    const int64_t threads = d.n * (k_local / 4);
    const unsigned blocks = (unsigned)((threads + 255) / 256);
    const uint64_t key = splitmix64(seed);
    const double rk = 1.0 / std::sqrt((double)k_total);
    if (prec == ER_FP64)
        k_sketch<double><<<blocks, 256, 0, s>>>(sketch_view(d), k_local, j0, key, rk, (double *)Yt);
    else {
        const float rk_hi = (float)rk;
        const float2 rk2 = make_float2(rk_hi, (float)(rk - (double)rk_hi));
        k_sketch32<<<blocks, 256, 0, s>>>(sketch_view(d), k_local, j0, key, rk2, (float *)Yt);
    }
    ER_CUDA(cudaGetLastError());
    return ER_OK;
}

er_status sketch(er_grid *g, int32_t k, uint64_t seed, er_precision prec, void *Yt, cudaStream_t s) {
    return sketch_cols(g, k, 0, k, seed, prec, Yt, s);
}

er_status reff_map(er_grid *g, const void *Z, int32_t k, er_precision prec, double *R, cudaStream_t s) {
    er_status st = check_nk(g, k, Z, "Z");
    if (st != ER_OK) return st;
    if (!R) return fail(ER_ERR_INVALID_ARG, "R is NULL");
    const GridDev &d = g->d;
    ER_CUDA(cudaSetDevice(d.device));
    const unsigned blocks = (unsigned)((d.n * 32 + 255) / 256);
    if (prec == ER_FP64)
        k_reff_map<double><<<blocks, 256, 0, s>>>((const double *)Z, d.n, k, d.floating, R);
    else if (prec == ER_FP32_REFINE)
        k_reff_map<float><<<blocks, 256, 0, s>>>((const float *)Z, d.n, k, d.floating, R);
    else
        return fail(ER_ERR_INVALID_ARG, "bad precision");
    ER_CUDA(cudaGetLastError());
    return ER_OK;
}

// Cached device buffers for er_reff_map_host, one set per device.
struct Pool {
    std::mutex mu;
    struct Buf { void *p = nullptr; size_t bytes = 0; };
    Buf bufs[64][3];
};
static Pool g_pool;

static er_status pool_get(int dev, int slot, size_t bytes, void **out) {
    if (dev < 0 || dev >= 64) return fail(ER_ERR_INVALID_ARG, "device ordinal out of range");
    Pool::Buf &b = g_pool.bufs[dev][slot];
    if (b.bytes < bytes) {
        if (b.p) ER_CUDA(cudaFree(b.p));
        b.p = nullptr;
        b.bytes = 0;
        ER_CUDA(cudaMalloc(&b.p, bytes));
        b.bytes = bytes;
    }
    *out = b.p;
    return ER_OK;
}

er_status solve(er_grid *g, const void *Yt, void *Z, int32_t k, er_precision prec, const er_solve_opts *opts,
                er_solve_stats *stats, cudaStream_t s);

}  // namespace er

// ----------------------------------------------------------------------------------
// C ABI

extern "C" {

er_status er_grid_create(const er_tier *tiers, int32_t n_tiers, const er_tsv *tsv, int64_t n_tsv,
                         const er_pad *pads, int64_t n_pads, const er_options *opt, void *stream,
                         er_grid **out) {
    return er::grid_create(tiers, n_tiers, tsv, n_tsv, pads, n_pads, opt, (cudaStream_t)stream, out);
}

er_status er_grid_destroy(er_grid *g) {
    if (!g) return ER_OK;
    cudaSetDevice(g->d.device);
    er::free_mg(&g->d);
    er::free_workspace(&g->d);
    er::free_grid_arrays(g->d);
    delete g;
    return ER_OK;
}

er_status er_grid_info(const er_grid *g, int64_t *n_nodes, int64_t *n_floating, int64_t *n_edges,
                       int64_t *h2d_bytes) {
    if (!g) return er::fail(ER_ERR_INVALID_ARG, "grid is NULL");
    if (n_nodes) *n_nodes = g->d.n;
    if (n_floating) *n_floating = g->d.n_floating;
    if (n_edges) *n_edges = g->d.n_edges;
    if (h2d_bytes) *h2d_bytes = g->d.h2d_bytes;
    return ER_OK;
}

er_status er_sketch(er_grid *g, int32_t k, uint64_t seed, er_precision prec, void *Yt, void *stream) {
    return er::sketch(g, k, seed, prec, Yt, (cudaStream_t)stream);
}

er_status er_sketch_cols(er_grid *g, int32_t k_total, int32_t j0, int32_t k_local, uint64_t seed, er_precision prec,
                         void *Yt, void *stream) {
    return er::sketch_cols(g, k_total, j0, k_local, seed, prec, Yt, (cudaStream_t)stream);
}

er_status er_reff_map(er_grid *g, const void *Z, int32_t k, er_precision prec, double *R, void *stream) {
    return er::reff_map(g, Z, k, prec, R, (cudaStream_t)stream);
}

er_status er_reff_map_host(const er_tier *tiers, int32_t n_tiers, const er_tsv *tsv, int64_t n_tsv,
                           const er_pad *pads, int64_t n_pads, int32_t k, uint64_t seed, er_precision prec,
                           const er_solve_opts *opts, double *R_host, er_solve_stats *stats, void *stream) {
    if (!R_host) return er::fail(ER_ERR_INVALID_ARG, "R_host is NULL");
    if (k < 4 || (k & 3)) return er::fail(ER_ERR_INVALID_ARG, "k must be a positive multiple of 4");
    cudaStream_t s = (cudaStream_t)stream;
    er_grid *g = nullptr;
    er_status st = er::grid_create(tiers, n_tiers, tsv, n_tsv, pads, n_pads, nullptr, s, &g);
    if (st != ER_OK && st != ER_WARN_FLOATING) return st;
    const er_status warn = st;
    std::lock_guard<std::mutex> lock(er::g_pool.mu);
    const size_t es = prec == ER_FP64 ? 8 : 4;
    const size_t nk = (size_t)g->d.n * (size_t)k * es;
    void *Yt = nullptr, *Z = nullptr, *R = nullptr;
    st = er::pool_get(g->d.device, 0, nk, &Yt);
    if (st == ER_OK) st = er::pool_get(g->d.device, 1, nk, &Z);
    if (st == ER_OK) st = er::pool_get(g->d.device, 2, (size_t)g->d.n * 8, &R);
    if (st == ER_OK) st = er::sketch(g, k, seed, prec, Yt, s);
    er_status sst = ER_OK;
    if (st == ER_OK) {
        sst = er::solve(g, Yt, Z, k, prec, opts, stats, s);
        if (sst != ER_OK && sst != ER_ERR_NOT_CONVERGED) st = sst;
    }
    if (st == ER_OK) st = er::reff_map(g, Z, k, prec, (double *)R, s);
    if (st == ER_OK) {
        cudaError_t e = cudaMemcpyAsync(R_host, R, (size_t)g->d.n * 8, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = er::cuda_fail(e, "copy R to host");
    }
    er_grid_destroy(g);
    if (st != ER_OK) return st;
    if (sst == ER_ERR_NOT_CONVERGED) return sst;
    return warn;
}

er_status er_release_pool(void) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(er::g_pool.mu);
    for (auto &b : er::g_pool.bufs[dev]) {
        if (b.p) cudaFree(b.p);
        b.p = nullptr;
        b.bytes = 0;
    }
    return ER_OK;
}

const char *er_status_str(er_status s) {
    switch (s) {
        case ER_OK: return "ER_OK";
        case ER_ERR_INVALID_ARG: return "ER_ERR_INVALID_ARG";
        case ER_ERR_CUDA: return "ER_ERR_CUDA";
        case ER_ERR_OOM: return "ER_ERR_OOM";
        case ER_ERR_NO_SUPPLY: return "ER_ERR_NO_SUPPLY";
        case ER_ERR_NOT_CONVERGED: return "ER_ERR_NOT_CONVERGED";
        case ER_ERR_TIMEOUT: return "ER_ERR_TIMEOUT";
        case ER_WARN_FLOATING: return "ER_WARN_FLOATING";
    }
    return "unknown er_status";
}

const char *er_last_error(void) { return er::g_last_error.c_str(); }

}  // extern "C"
