// FP32 form of the multi-RHS Jacobi-PCG solve, with TMA row staging (sm_103a).
//
// The FP32 iterations apply the network operator in edge-difference form,
//   (G v)_i = pad_i v_i + sum_{j ~ i} g_ij (v_i - v_j),
// with every conductance rounded to FP32 once at grid creation.  The accurate residual
// b - G x uses exactly the same FP32 conductances, so the FP32 recursion and the accurate
// residual see one operator, and the Laplacian structure (zero row sums apart from the
// pads) is exact.  Rounding each conductance by at most a relative u = 2^-24 keeps every
// effective resistance within [R/(1+u), R/(1-u)] (Rayleigh monotonicity: the perturbed
// network lies between the original scaled by 1-u and by 1+u).
//
// The accurate iterate and residual are double-float: a value is the unevaluated sum
// hi + lo of two FP32 numbers (about 48 significant bits), and the residual is formed with
// error-free transformations (TwoSum, FMA TwoProduct) on the FP32 pipes.  FP64 arithmetic
// runs at 1/64 of the FP32 rate on this GPU, so an FP64 residual pass was bound by the
// FP64 units, not by memory; the double-float pass moves the same bytes (8 per iterate
// entry) and is bandwidth-bound.
//
// Jacobi preconditioning: z = D^-1 r with D = diag(G) from the same conductances.
// Passes per iteration (vectors [n][k] FP32, k innermost):
//   A  p' = z + beta p; q = G p'; dot p'.q                          reads r, p
//   B  recompute p', q; x += alpha p'; r' = r - alpha q; dot r'.z'  reads r, p, x;
//                                                                  writes x, r', p'
// Every `replace_every` iterations the correction x is folded into the double-float iterate
// (xhl += x, x = 0) and the accurate residual r = b - G xhl replaces the recursive one
// (a reliable update: CG continues with the same search direction).
//
// Staging: a CTA owns 30 nodes along x (one halo node each side) and a run of y rows of
// one tier, for 32 RHS columns.  One thread issues cp.async.bulk.tensor loads of whole
// rows (32 nodes x 128 B per vector, plus 32 x 16 B of per-node coefficients) into a ring
// of shared-memory stages, each completed through an mbarrier; the 256 threads (8 per
// node, 16 B each) compute from shared memory.  Each step reads one row's stage into
// registers and publishes that row's operand p' in a two-row shared ring; q of the row
// above is finished from registers (north, centre, south) and the ring (west, east), so
// only one stage is resident and the others are in flight, many bulk copies per SM
// without costing registers.  The coefficient word carries 1/d with its sign flagging
// nodes that have TSV segments.  Every mbarrier wait is bounded: on expiry the kernel
// raises the error word, stops waiting, drains its own copies and returns; the host
// reports ER_ERR_TIMEOUT.
#include <cudaTypedefs.h>

#include <atomic>
#include <cmath>
#include <cstring>
#include <type_traits>

#include "er_common.cuh"

namespace er {

// ---------------------------------------------------------------------------------------
// PTX wrappers (mbarrier + bulk tensor copies)

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(b)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(b)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void tma_load4(void *dst, const CUtensorMap *m, uint64_t *bar, int c0, int c1, int c2,
                                          int c3) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(m)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_addr(bar))
        : "memory");
}

constexpr uint32_t kSpinLimit = 1u << 22;

// Kernel parameters: tensor maps must live in parameter space (__grid_constant__).
struct TArgs {
    CUtensorMap tm[4];  // stage inputs; meaning per mode (see Layout)
    KArgs<float, float> a;
};

template <int MODE>
struct Layout;
template <>
struct Layout<MODE_A_DOT> {  // stage: r, p, coef
    static constexpr int NS = 5, OFF_R = 0, OFF_P = 4096, OFF_X = -1, OFF_COEF = 8192, BYTES = 8704;
};
template <>
struct Layout<MODE_B> {  // odd iterations; stage: r, p, x, coef
    static constexpr int NS = 4, OFF_R = 0, OFF_P = 4096, OFF_X = 8192, OFF_COEF = 12288, BYTES = 12800;
};
template <>
struct Layout<MODE_B0> {  // even iterations; stage: r, p, coef
    static constexpr int NS = 4, OFF_R = 0, OFF_P = 4096, OFF_X = -1, OFF_COEF = 8192, BYTES = 8704;
};
template <>
struct Layout<MODE_R> {  // stage: xhl (8-byte {hi, lo} pairs), b, coef
    static constexpr int NS = 4, OFF_R = 8192, OFF_P = -1, OFF_X = 0, OFF_COEF = 12288, BYTES = 12800;
};
// dynamic shared memory: NS stages, then a two-row ring of the per-node operand
// (p' in FP32, xhl as {hi, lo} pairs), plus slack for 128-byte alignment
template <int MODE>
constexpr int ring_bytes() { return MODE == MODE_R ? 2 * kNX * 256 : 2 * kNX * 128; }
template <int MODE>
constexpr int dyn_smem() { return Layout<MODE>::NS * Layout<MODE>::BYTES + ring_bytes<MODE>() + 128; }

__device__ __forceinline__ float4 lds4(const unsigned char *p) { return *reinterpret_cast<const float4 *>(p); }

// component v of a float4 (v is a compile-time constant after unrolling)
__device__ __forceinline__ float f4(const float4 &f, int v) { return v == 0 ? f.x : v == 1 ? f.y : v == 2 ? f.z : f.w; }

// Double-float arithmetic of the iterate and the residual.  Error-free transformations:
// TwoSum (Knuth; s + e = a + b exactly) and the FMA TwoProduct (p + e = a * b exactly),
// as in Ogita, Rump and Oishi, "Accurate sum and dot product", SIAM J. Sci. Comput. 26
// (2005).  The _rn intrinsics are never contracted into FMAs, which would corrupt the
// error terms.
__device__ __forceinline__ float2 two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return make_float2(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}

// {hi, lo} + c, renormalised (hi = the sum rounded to FP32, lo = the rest)
__device__ __forceinline__ float2 df_add(float2 X, float c) {
    const float2 t = two_sum(X.x, c);
    return two_sum(t.x, __fadd_rn(t.y, X.y));
}

// q = pad X_i + sum_j g_ij (X_i - X_j) for FP32 conductances and double-float X, held as
// the unevaluated sum S + C (C collects every rounding error of the terms and of S)
struct DfSum {
    float S, C;
    __device__ __forceinline__ void init_prod(float g, float2 X) {  // S + C = g X
        S = __fmul_rn(g, X.x);
        C = fmaf(g, X.y, fmaf(g, X.x, -S));
    }
    __device__ __forceinline__ void add_edge(float g, float2 Xi, float2 Xj) {  // S + C += g (Xi - Xj)
        const float2 d = two_sum(Xi.x, -Xj.x);
        const float dl = __fadd_rn(d.y, __fsub_rn(Xi.y, Xj.y));
        const float p = __fmul_rn(g, d.x);
        const float pe = fmaf(g, dl, fmaf(g, d.x, -p));
        const float2 t = two_sum(S, p);
        S = t.x;
        C = __fadd_rn(C, __fadd_rn(t.y, pe));
    }
    __device__ __forceinline__ float residual(float b) const {  // b - (S + C), rounded once
        const float2 t = two_sum(b, -S);
        return __fadd_rn(t.x, __fsub_rn(t.y, C));
    }
};

// One pass over a CTA's tile.  Step ri (row y = y0 - 1 + ri) waits for its stage, reads the
// thread's own node from it into registers (r, p or xhl, x, coefficients), forms the
// operand v = p' (or xhl) and, for row y - 1, finishes q = G v from registers (north,
// centre, south) and the ring (x-neighbours of the centre row); then it publishes v in the
// ring, synchronises once, and the stage is refilled NS rows ahead.
template <int MODE>
__device__ __forceinline__ void tma_pass(const KArgs<float, float> &a, const CUtensorMap *tm0, const CUtensorMap *tm1,
                                         const CUtensorMap *tm2, const CUtensorMap *tm3, int block_id,
                                         unsigned char *smem_raw) {
    using L = Layout<MODE>;
    constexpr int V = 4, KB = kTPN * V;  // 32 columns per CTA
    constexpr bool R64 = MODE == MODE_R;
    using Cv = typename std::conditional<R64, float2, float>::type;  // operand type ({hi, lo} in MODE_R)
    unsigned char *smem = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
    Cv *ring = reinterpret_cast<Cv *>(smem + L::NS * L::BYTES);  // [2][kNX][KB]
    __shared__ __align__(8) uint64_t bars[L::NS];
    __shared__ int s_abort;
    __shared__ __align__(16) float s_beta[KB], s_alpha[KB], s_alpha_prev[KB];  // per-column CG scalars

    const int lc = threadIdx.x % kTPN, xl = threadIdx.x / kTPN;
    int tx, tyi, t, cb;
    decode_block(a, block_id, tx, tyi, t, cb);
    const int spatial = (t * a.tiles_y + tyi) * a.tiles_x + tx;
    const int c0 = cb * KB;
    const int xb = tx * kTXI - 1;
    const int x = xb + xl;
    const int y0 = tyi * a.rows, y1 = min(y0 + a.rows, a.H);
    const int nrow = y1 - y0 + 2;  // rows y0-1 .. y1
    const int col = c0 + lc * V;
    const bool colok = col < a.k;
    const bool own = xl >= 1 && xl <= kNX - 2 && x < a.W && colok;
    const int64_t tbase = (int64_t)t * a.W * a.H;

    if (threadIdx.x == 0) {
        for (int s = 0; s < L::NS; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
        s_abort = 0;
    }
    if (threadIdx.x < KB) {
        const int j = c0 + threadIdx.x;
        s_beta[threadIdx.x] = (j < a.k && !R64) ? (float)a.beta[j] : 0.f;
        s_alpha[threadIdx.x] = (j < a.k && (MODE == MODE_B || MODE == MODE_B0)) ? (float)a.alpha[j] : 0.f;
        s_alpha_prev[threadIdx.x] = (j < a.k && MODE == MODE_B) ? (float)a.alpha_prev[j] : 0.f;
    }
    __syncthreads();

    auto issue = [&](int ri) {
        const int s = ri % L::NS;
        unsigned char *st = smem + s * L::BYTES;
        const int y = y0 - 1 + ri;
        mbar_arrive_expect_tx(&bars[s], L::BYTES);
        if constexpr (R64) {
            tma_load4(st + L::OFF_X, tm0, &bars[s], c0, xb, y, t);  // xhl
            tma_load4(st + L::OFF_R, tm1, &bars[s], c0, xb, y, t);  // b
        } else {
            tma_load4(st + L::OFF_R, tm0, &bars[s], c0, xb, y, t);
            tma_load4(st + L::OFF_P, tm1, &bars[s], c0, xb, y, t);
            if constexpr (MODE == MODE_B) tma_load4(st + L::OFF_X, tm2, &bars[s], c0, xb, y, t);
        }
        tma_load4(st + L::OFF_COEF, tm3, &bars[s], 0, xb, y, t);
    };
    bool aborted = false;
    auto wait_row = [&](int ri) {
        if (aborted) return;
        const int s = ri % L::NS;
        const uint32_t par = (uint32_t)(ri / L::NS) & 1u;
        uint32_t spins = 0;
        while (!mbar_try_wait(&bars[s], par)) {
            if (++spins > kSpinLimit) {
                aborted = true;
                s_abort = 1;
                atomicExch(a.err, 1);
                return;
            }
        }
    };

    auto load_be = [&](float (&o)[V]) {
        const float4 b4 = *reinterpret_cast<const float4 *>(s_beta + lc * V);
        o[0] = b4.x; o[1] = b4.y; o[2] = b4.z; o[3] = b4.w;
    };

    if (threadIdx.x == 0)
        for (int ri = 0; ri < L::NS && ri < nrow; ++ri) issue(ri);

    // registers: operand at rows y-2 (vn), y-1 (vc); r/x/b and coefficients of row y-1
    Cv vn[V], vc[V];
    float rc[V];
    float4 cfc = make_float4(0.f, 0.f, 0.f, 0.f);  // {+-1/d, gE, gS, pad} of row y-1, own node
    float gwc = 0.f, gsn = 0.f;                    // gE of the west node (row y-1); gS of row y-2
    float run[V] = {0.f, 0.f, 0.f, 0.f};
    float2 acc[V];  // double-float per-column sums of the FP32 runs (no FP64 arithmetic per node)
#pragma unroll
    for (int v = 0; v < V; ++v) acc[v] = make_float2(0.f, 0.f);
    int nrun = 0;
#pragma unroll
    for (int v = 0; v < V; ++v) vn[v] = vc[v] = Cv{}, rc[v] = 0.f;

#pragma unroll 2
    for (int ri = 0; ri < nrow; ++ri) {
        wait_row(ri);
        const unsigned char *st = smem + (ri % L::NS) * L::BYTES;
        // own node of row ri from the stage
        Cv vs[V];
        float rs[V], xs[V], ps[V];
        const float4 cfs = lds4(st + L::OFF_COEF + xl * 16);
        const float gws = xl > 0 ? lds4(st + L::OFF_COEF + (xl - 1) * 16).y : 0.f;
        if constexpr (R64) {
            const float4 c01 = lds4(st + L::OFF_X + xl * 256 + lc * 32);
            const float4 c23 = lds4(st + L::OFF_X + xl * 256 + lc * 32 + 16);
            vs[0] = make_float2(c01.x, c01.y); vs[1] = make_float2(c01.z, c01.w);
            vs[2] = make_float2(c23.x, c23.y); vs[3] = make_float2(c23.z, c23.w);
            const float4 b = lds4(st + L::OFF_R + xl * 128 + lc * 16);
            rs[0] = b.x; rs[1] = b.y; rs[2] = b.z; rs[3] = b.w;
        } else {
            const float dinv = fabsf(cfs.x);
            float be[V];
            load_be(be);
            const float4 r = lds4(st + L::OFF_R + xl * 128 + lc * 16);
            const float4 p = lds4(st + L::OFF_P + xl * 128 + lc * 16);
            rs[0] = r.x; rs[1] = r.y; rs[2] = r.z; rs[3] = r.w;
            ps[0] = p.x; ps[1] = p.y; ps[2] = p.z; ps[3] = p.w;
            vs[0] = fmaf(be[0], p.x, dinv * r.x);
            vs[1] = fmaf(be[1], p.y, dinv * r.y);
            vs[2] = fmaf(be[2], p.z, dinv * r.z);
            vs[3] = fmaf(be[3], p.w, dinv * r.w);
            if constexpr (MODE == MODE_B) {
                const float4 xx = lds4(st + L::OFF_X + xl * 128 + lc * 16);
                xs[0] = xx.x; xs[1] = xx.y; xs[2] = xx.z; xs[3] = xx.w;
            }
        }
        // pass B: p' and (odd iterations) x of row ri need no neighbour: write them now
        if constexpr (MODE == MODE_B || MODE == MODE_B0) {
            if (own && ri >= 1 && ri + 1 < nrow) {
                const int64_t idx = (tbase + (int64_t)(y0 - 1 + ri) * a.W + x) * a.k + col;
                stv<float, float, V>(a.p_out + idx, vs);
                if constexpr (MODE == MODE_B) {  // x += alpha_prev p_prev + alpha p'
                    const float4 a4 = *reinterpret_cast<const float4 *>(s_alpha + lc * V);
                    const float4 b4 = *reinterpret_cast<const float4 *>(s_alpha_prev + lc * V);
                    float xn[V];
#pragma unroll
                    for (int v = 0; v < V; ++v) xn[v] = fmaf(f4(a4, v), vs[v], fmaf(f4(b4, v), ps[v], xs[v]));
                    stv<float, float, V>(a.x + idx, xn);
                }
            }
        }
        // row y-1: q = pad v + gE (v - v_e) + gW (v - v_w) + gS (v - v_s) + gN (v - v_n) + TSVs
        if (ri >= 2 && own) {
            const int y = y0 - 2 + ri;
            const int64_t i = tbase + (int64_t)y * a.W + x;
            const int64_t idx = i * a.k + col;
            const Cv *rw = ring + ((ri - 1) & 1) * kNX * KB;
            Cv vw[V], ve[V];
            float q[V];
            if constexpr (R64) {
                const float4 *pw = reinterpret_cast<const float4 *>(rw + (xl - 1) * KB + lc * V);
                const float4 *pe = reinterpret_cast<const float4 *>(rw + (xl + 1) * KB + lc * V);
                vw[0] = make_float2(pw[0].x, pw[0].y); vw[1] = make_float2(pw[0].z, pw[0].w);
                vw[2] = make_float2(pw[1].x, pw[1].y); vw[3] = make_float2(pw[1].z, pw[1].w);
                ve[0] = make_float2(pe[0].x, pe[0].y); ve[1] = make_float2(pe[0].z, pe[0].w);
                ve[2] = make_float2(pe[1].x, pe[1].y); ve[3] = make_float2(pe[1].z, pe[1].w);
            } else {
                const float4 w4 = *reinterpret_cast<const float4 *>(rw + (xl - 1) * KB + lc * V);
                const float4 e4 = *reinterpret_cast<const float4 *>(rw + (xl + 1) * KB + lc * V);
                vw[0] = w4.x; vw[1] = w4.y; vw[2] = w4.z; vw[3] = w4.w;
                ve[0] = e4.x; ve[1] = e4.y; ve[2] = e4.z; ve[3] = e4.w;
            }
            const float gp = cfc.w, ge = cfc.y, gs = cfc.z, gw = gwc, gn = gsn;
            if constexpr (MODE == MODE_A_DOT) {
                // p'.Gp' as a sum over edges: pad p^2 + gE (p - pE)^2 + gS (p - pS)^2 at each node,
                // plus half of every TSV segment at each of its two ends
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const float de = vc[v] - ve[v], ds = vc[v] - vs[v];
                    float e = gp * vc[v] * vc[v];
                    e = fmaf(ge * de, de, e);
                    e = fmaf(gs * ds, ds, e);
                    q[v] = e;
                }
            } else if constexpr (R64) {
                // edge-difference form in double-float: q = pad X_i + sum_j g_ij (X_i - X_j),
                // held as the unevaluated sum S + C
                DfSum acc4[V];
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    acc4[v].init_prod(gp, vc[v]);
                    acc4[v].add_edge(ge, vc[v], ve[v]);
                    acc4[v].add_edge(gw, vc[v], vw[v]);
                    acc4[v].add_edge(gs, vc[v], vs[v]);
                    acc4[v].add_edge(gn, vc[v], vn[v]);
                }
                if (cfc.x < 0.f) {
                    const int e1 = a.tsv_ptr[i + 1];
                    for (int e = a.tsv_ptr[i]; e < e1; ++e) {
                        const int64_t jdx = (int64_t)a.tsv_nbr[e] * a.k + col;
                        const float g = a.tsv_g32[e];
                        const float4 c01 = *reinterpret_cast<const float4 *>(a.xhl + jdx);
                        const float4 c23 = *reinterpret_cast<const float4 *>(a.xhl + jdx + 2);
                        acc4[0].add_edge(g, vc[0], make_float2(c01.x, c01.y));
                        acc4[1].add_edge(g, vc[1], make_float2(c01.z, c01.w));
                        acc4[2].add_edge(g, vc[2], make_float2(c23.x, c23.y));
                        acc4[3].add_edge(g, vc[3], make_float2(c23.z, c23.w));
                    }
                }
#pragma unroll
                for (int v = 0; v < V; ++v) q[v] = acc4[v].residual(rc[v]);  // b - q, rounded once
            } else {
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    Cv qq = gp * vc[v];
                    qq = fma(ge, vc[v] - ve[v], qq);
                    qq = fma(gw, vc[v] - vw[v], qq);
                    qq = fma(gs, vc[v] - vs[v], qq);
                    qq = fma(gn, vc[v] - vn[v], qq);
                    q[v] = qq;
                }
            }
            if constexpr (!R64) if (cfc.x < 0.f) {  // node with TSV segments (FP32 passes)
                const int e1 = a.tsv_ptr[i + 1];
                for (int e = a.tsv_ptr[i]; e < e1; ++e) {
                    const int j = a.tsv_nbr[e];
                    const int64_t jdx = (int64_t)j * a.k + col;
                    const float g = a.tsv_g32[e];
                    const float4 b4 = *reinterpret_cast<const float4 *>(s_beta + lc * V);
                    const float dj = fabsf(a.coef[j].x);
                    const float4 rj = *reinterpret_cast<const float4 *>(a.r_in + jdx);
                    const float4 pj = *reinterpret_cast<const float4 *>(a.p_in + jdx);
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        const float dv = (float)vc[v] - fmaf(f4(b4, v), f4(pj, v), dj * f4(rj, v));
                        if constexpr (MODE == MODE_A_DOT) q[v] = fmaf(0.5f * g * dv, dv, (float)q[v]);
                        else q[v] = fmaf(g, dv, (float)q[v]);
                    }
                }
            }
            if constexpr (R64) {
                const float dinv = fabsf(cfc.x);
                float ro[V];
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    ro[v] = q[v];
                    run[v] = fmaf(dinv * ro[v], ro[v], run[v]);
                }
                stv<float, float, V>(a.r_out + idx, ro);
            } else if constexpr (MODE == MODE_A_DOT) {
#pragma unroll
                for (int v = 0; v < V; ++v) run[v] += q[v];
            } else {
                const float dinv = fabsf(cfc.x);
                const float4 a4 = *reinterpret_cast<const float4 *>(s_alpha + lc * V);
                float rn[V];
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    rn[v] = fmaf(-f4(a4, v), q[v], rc[v]);
                    run[v] = fmaf(dinv * rn[v], rn[v], run[v]);
                }
                stv<float, float, V>(a.r_out + idx, rn);
            }
            {
                if (++nrun == 8) {
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        acc[v] = df_add(acc[v], run[v]);
                        run[v] = 0.f;
                    }
                    nrun = 0;
                }
            }
        }
        // publish the operand of row ri, rotate the registers
        {
            Cv *wr = ring + (ri & 1) * kNX * KB + xl * KB + lc * V;
            if constexpr (R64) {
                reinterpret_cast<float4 *>(wr)[0] = make_float4(vs[0].x, vs[0].y, vs[1].x, vs[1].y);
                reinterpret_cast<float4 *>(wr)[1] = make_float4(vs[2].x, vs[2].y, vs[3].x, vs[3].y);
            } else {
                *reinterpret_cast<float4 *>(wr) = make_float4(vs[0], vs[1], vs[2], vs[3]);
            }
        }
        gsn = cfc.z;
        cfc = cfs;
        gwc = gws;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            vn[v] = vc[v];
            vc[v] = vs[v];
            rc[v] = rs[v];

        }
        __syncthreads();
        if (threadIdx.x == 0 && ri + L::NS < nrow && !s_abort) issue(ri + L::NS);
    }
    // drain: after an expired wait, make sure no copy is still landing in shared memory
    if (threadIdx.x == 0 && s_abort) {
        for (int s = 0; s < L::NS && s < nrow; ++s) {
            int last = s;
            while (last + L::NS < nrow) last += L::NS;
            const uint32_t par = (uint32_t)(last / L::NS) & 1u;
            for (uint32_t n = 0; n < kSpinLimit && !mbar_try_wait(&bars[s], par); ++n) {
            }
        }
    }
    __syncthreads();
    // per column: the kNX node slots of the CTA summed in a fixed order, in double-float
    float2 *sdf = reinterpret_cast<float2 *>(smem);  // the stage ring is free now
#pragma unroll
    for (int v = 0; v < V; ++v) sdf[xl * KB + lc * V + v] = own ? df_add(acc[v], run[v]) : make_float2(0.f, 0.f);
    __syncthreads();
    double s_col = 0.0;
    if (threadIdx.x < KB) {
        float2 t = sdf[threadIdx.x];
        for (int xx = 1; xx < kNX; ++xx) {
            const float2 u = sdf[xx * KB + threadIdx.x];
            const float2 h = two_sum(t.x, u.x);
            t = two_sum(h.x, __fadd_rn(h.y, __fadd_rn(t.y, u.y)));
        }
        s_col = (double)t.x + (double)t.y;
    }
    __syncthreads();
    write_and_finalize<float, float, MODE, KB>(a, reinterpret_cast<double *>(smem), s_col, spatial, cb);
}

template <int MODE>
__global__ void __launch_bounds__(kThreads, MODE == MODE_A_DOT ? 4 : 3) k_tma(const __grid_constant__ TArgs ta) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    tma_pass<MODE>(ta.a, &ta.tm[0], &ta.tm[1], &ta.tm[2], &ta.tm[3], (int)blockIdx.x, smem_raw);
}

// ---------------------------------------------------------------------------------------
// streaming kernels of the FP32 form (same tiling, no halo)

template <int MODE>
__device__ __forceinline__ void fp32_stream_pass(const KArgs<float, float> &a, int block_id) {
    constexpr int V = 4, KB = kTPN * V;
    __shared__ double sred[kNX * KB];
    const int lc = threadIdx.x % kTPN, xl = threadIdx.x / kTPN;
    int tx, tyi, t, cb;
    decode_block(a, block_id, tx, tyi, t, cb);
    const int spatial = (t * a.tiles_y + tyi) * a.tiles_x + tx;
    const int x = tx * kTXI - 1 + xl;
    const int y0 = tyi * a.rows, y1 = min(y0 + a.rows, a.H);
    const int col = cb * KB + lc * V;
    const bool own = xl >= 1 && xl <= kNX - 2 && x < a.W && col < a.k;
    const int64_t tbase = (int64_t)t * a.W * a.H;
    Acc<float> acc[V];
    if (own) {
        for (int y = y0; y < y1; ++y) {
            const int64_t i = tbase + (int64_t)y * a.W + x;
            const int64_t idx = i * a.k + col;
            if constexpr (MODE == MODE_INIT) {  // r = b, x = 0, p = 0, xhl = 0; dot b.D^-1 b
                float b[V];
                const float z[V] = {0.f, 0.f, 0.f, 0.f};
                ldv<float, float, V>(a.b_in + idx, b);
                const float dinv = fabsf(a.coef[i].x);
                stv<float, float, V>(a.r_out + idx, b);
                stv<float, float, V>(a.x + idx, z);
                stv<float, float, V>(a.p_out + idx, z);
                *reinterpret_cast<float4 *>(a.xhl + idx) = make_float4(0.f, 0.f, 0.f, 0.f);
                *reinterpret_cast<float4 *>(a.xhl + idx + 2) = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int v = 0; v < V; ++v) acc[v].add(dinv * b[v], b[v]);
            } else if constexpr (MODE == MODE_ACCUM) {  // xhl += x (double-float); x = 0
                float c[V];
                const float z[V] = {0.f, 0.f, 0.f, 0.f};
                ldv<float, float, V>(a.x + idx, c);
                float4 *xp = reinterpret_cast<float4 *>(a.xhl + idx);
                const float4 c01 = xp[0], c23 = xp[1];
                const float2 x0 = df_add(make_float2(c01.x, c01.y), c[0]);
                const float2 x1 = df_add(make_float2(c01.z, c01.w), c[1]);
                const float2 x2 = df_add(make_float2(c23.x, c23.y), c[2]);
                const float2 x3 = df_add(make_float2(c23.z, c23.w), c[3]);
                xp[0] = make_float4(x0.x, x0.y, x1.x, x1.y);
                xp[1] = make_float4(x2.x, x2.y, x3.x, x3.y);
                stv<float, float, V>(a.x + idx, z);
            } else {  // MODE_UNSCALE: Z = hi + lo rounded to FP32
                const float4 *xp = reinterpret_cast<const float4 *>(a.xhl + idx);
                const float4 c01 = xp[0], c23 = xp[1];
                const float o[V] = {__fadd_rn(c01.x, c01.y), __fadd_rn(c01.z, c01.w), __fadd_rn(c23.x, c23.y),
                                    __fadd_rn(c23.z, c23.w)};
                stv<float, float, V>(a.x + idx, o);
            }
        }
    }
    if constexpr (MODE == MODE_INIT) {
#pragma unroll
        for (int v = 0; v < V; ++v) sred[xl * KB + lc * V + v] = own ? acc[v].val() : 0.0;
        __syncthreads();
        reduce_and_finalize<float, float, MODE_INIT, KB>(a, sred, spatial, cb);
    }
}

template <int MODE>
__global__ void __launch_bounds__(kThreads) k_fp32_stream(const KArgs<float, float> a) {
    fp32_stream_pass<MODE>(a, (int)blockIdx.x);
}

// ---------------------------------------------------------------------------------------
// batching form: one launch per pass covers the tiles of many networks.  The work list
// holds (network, block-within-network); each CTA copies its network's arguments into
// shared memory and runs the same pass as the single-network kernels.  With `sel`, only the
// networks c with sel[c] != 0 run (the other CTAs return at once).

template <int MODE>
__device__ __forceinline__ void batch_args(const BatchItem &it, int cur, int rmode, KArgs<float, float> &a) {
    a = it.a;
    a.rmode = rmode;
    if constexpr (MODE == MODE_R) {
        a.xhl = it.xhl;
        a.r_out = it.r[cur];
    } else if constexpr (MODE == MODE_INIT) {
        a.b_in = it.b; a.r_out = it.r[0]; a.x = it.c; a.p_out = it.p[0]; a.xhl = it.xhl;
    } else if constexpr (MODE == MODE_ACCUM || MODE == MODE_UNSCALE) {
        a.x = it.c; a.xhl = it.xhl;
    } else {
        a.r_in = it.r[cur]; a.p_in = it.p[cur]; a.x = it.c;
        a.r_out = it.r[1 - cur]; a.p_out = it.p[1 - cur];
    }
}

template <int MODE>
__global__ void __launch_bounds__(kThreads, MODE == MODE_A_DOT ? 4 : 3)
    k_tma_batch(const BatchItem *__restrict__ items, const int2 *__restrict__ work, int cur, int rmode,
                const int *__restrict__ sel) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ KArgs<float, float> s_a;
    const int2 wk = work[blockIdx.x];
    if (sel && !sel[wk.x]) return;
    const BatchItem &it = items[wk.x];
    if (threadIdx.x == 0) batch_args<MODE>(it, cur, rmode, s_a);
    __syncthreads();
    if constexpr (MODE == MODE_R)
        tma_pass<MODE>(s_a, &it.tm[5], &it.tm[6], nullptr, &it.tm[7], wk.y, smem_raw);
    else
        tma_pass<MODE>(s_a, &it.tm[cur], &it.tm[2 + cur], &it.tm[4], &it.tm[7], wk.y, smem_raw);
}

template <int MODE>
__global__ void __launch_bounds__(kThreads) k_stream_batch(const BatchItem *__restrict__ items,
                                                           const int2 *__restrict__ work, const int *__restrict__ sel) {
    __shared__ KArgs<float, float> s_a;
    const int2 wk = work[blockIdx.x];
    if (sel && !sel[wk.x]) return;
    if (threadIdx.x == 0) batch_args<MODE>(items[wk.x], 0, 0, s_a);
    __syncthreads();
    fp32_stream_pass<MODE>(s_a, wk.y);
}

// ---------------------------------------------------------------------------------------
// host side

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// 4-D map over [T][H][W][d0] (d0 innermost) with a box of d0box x 32 nodes x 1 x 1.
static er_status make_map(CUtensorMap *m, CUtensorMapDataType dt, int esize, const void *base, int64_t d0, int box0,
                          const GridDev &g) {
    auto fn = encode_fn();
    if (!fn) return fail(ER_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
    cuuint64_t dims[4] = {(cuuint64_t)d0, (cuuint64_t)g.W, (cuuint64_t)g.H, (cuuint64_t)g.T};
    cuuint64_t strides[3] = {(cuuint64_t)d0 * esize, (cuuint64_t)d0 * esize * g.W, (cuuint64_t)d0 * esize * g.W * g.H};
    cuuint32_t box[4] = {(cuuint32_t)box0, (cuuint32_t)kNX, 1, 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = fn(m, dt, 4, const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(ER_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return ER_OK;
}

er_status fp32_make_map(CUtensorMap *m, bool f64, const void *base, int64_t d0, int box0, const GridDev &g) {
    return f64 ? make_map(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 8, base, d0, box0, g)
               : make_map(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, d0, box0, g);
}

static std::atomic<bool> g_attr_done{false};  // set once; solves may run on several host threads
static std::atomic<bool> g_battr_done{false};

er_status fp32_batch_pass(int mode, const BatchItem *items, const int2 *work, int n_work, int cur, int rmode,
                          cudaStream_t s, const int *sel) {
    if (!g_battr_done.load()) {
        ER_CUDA(cudaFuncSetAttribute(k_tma_batch<MODE_A_DOT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     dyn_smem<MODE_A_DOT>()));
        ER_CUDA(cudaFuncSetAttribute(k_tma_batch<MODE_B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     dyn_smem<MODE_B>()));
        ER_CUDA(cudaFuncSetAttribute(k_tma_batch<MODE_B0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     dyn_smem<MODE_B0>()));
        ER_CUDA(cudaFuncSetAttribute(k_tma_batch<MODE_R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     dyn_smem<MODE_R>()));
        g_battr_done.store(true);
    }
    if (n_work <= 0) return ER_OK;
    const unsigned nb = (unsigned)n_work;
    switch (mode) {
        case MODE_A_DOT: k_tma_batch<MODE_A_DOT><<<nb, kThreads, dyn_smem<MODE_A_DOT>(), s>>>(items, work, cur, rmode, sel); break;
        case MODE_B: k_tma_batch<MODE_B><<<nb, kThreads, dyn_smem<MODE_B>(), s>>>(items, work, cur, rmode, sel); break;
        case MODE_B0: k_tma_batch<MODE_B0><<<nb, kThreads, dyn_smem<MODE_B0>(), s>>>(items, work, cur, rmode, sel); break;
        case MODE_R: k_tma_batch<MODE_R><<<nb, kThreads, dyn_smem<MODE_R>(), s>>>(items, work, cur, rmode, sel); break;
        case MODE_INIT: k_stream_batch<MODE_INIT><<<nb, kThreads, 0, s>>>(items, work, sel); break;
        case MODE_ACCUM: k_stream_batch<MODE_ACCUM><<<nb, kThreads, 0, s>>>(items, work, sel); break;
        case MODE_UNSCALE: k_stream_batch<MODE_UNSCALE><<<nb, kThreads, 0, s>>>(items, work, sel); break;
        default: return fail(ER_ERR_INVALID_ARG, "bad batch pass");
    }
    ER_CUDA(cudaGetLastError());
    return ER_OK;
}

er_status fp32_prepare(const GridDev &g, Workspace &w, const void *Yt, void *Z) {
    const auto F32 = CU_TENSOR_MAP_DATA_TYPE_FLOAT32, F64 = CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
    if (!w.tm_c_ptr) {  // workspace vectors: once per workspace
        for (int i = 0; i < 2; ++i) {
            er_status s = make_map(&w.tm_r[i], F32, 4, w.r[i], w.k, 32, g);
            if (s == ER_OK) s = make_map(&w.tm_p[i], F32, 4, w.p[i], w.k, 32, g);
            if (s != ER_OK) return s;
        }
        er_status s = make_map(&w.tm_xhl, F64, 8, w.xhl, w.k, 32, g);  // 8-byte {hi, lo} pairs, copied as bytes
        if (s == ER_OK) s = make_map(&w.tm_coef, F32, 4, g.coef32, 4, 4, g);
        if (s != ER_OK) return s;
    }
    if (w.tm_c_ptr != Z) {
        er_status s = make_map(&w.tm_c, F32, 4, Z, w.k, 32, g);
        if (s != ER_OK) return s;
        w.tm_c_ptr = Z;
    }
    if (w.tm_b_ptr != Yt) {
        er_status s = make_map(&w.tm_b, F32, 4, Yt, w.k, 32, g);
        if (s != ER_OK) return s;
        w.tm_b_ptr = Yt;
    }
    if (!g_attr_done.load()) {
        ER_CUDA(cudaFuncSetAttribute(k_tma<MODE_A_DOT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     dyn_smem<MODE_A_DOT>()));
        ER_CUDA(cudaFuncSetAttribute(k_tma<MODE_B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     dyn_smem<MODE_B>()));
        ER_CUDA(cudaFuncSetAttribute(k_tma<MODE_B0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     dyn_smem<MODE_B0>()));
        ER_CUDA(cudaFuncSetAttribute(k_tma<MODE_R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     dyn_smem<MODE_R>()));
        g_attr_done.store(true);
    }
    return ER_OK;
}

template <int MODE>
static void launch_tma(const TArgs &ta, Workspace &w, Prof *pf, int kind) {
    prof_begin(w, pf, kind);
    k_tma<MODE><<<(unsigned)w.til.n_ctas(), kThreads, dyn_smem<MODE>(), w.s>>>(ta);
    prof_end(w, pf, kind);
}

template <int MODE>
static void launch_stream(const KArgs<float, float> &a, Workspace &w, Prof *pf, int kind) {
    prof_begin(w, pf, kind);
    k_fp32_stream<MODE><<<(unsigned)w.til.n_ctas(), kThreads, 0, w.s>>>(a);
    prof_end(w, pf, kind);
}

er_status fp32_workspace_item(const GridDev &g, Workspace &w, const void *Yt, void *Z, double tol, BatchItem *it) {
    er_status st = fp32_prepare(g, w, Yt, Z);
    if (st != ER_OK) return st;
    std::memset(it, 0, sizeof(*it));
    it->tm[0] = w.tm_r[0];
    it->tm[1] = w.tm_r[1];
    it->tm[2] = w.tm_p[0];
    it->tm[3] = w.tm_p[1];
    it->tm[4] = w.tm_c;
    it->tm[5] = w.tm_xhl;
    it->tm[6] = w.tm_b;
    it->tm[7] = w.tm_coef;
    it->a = base_args<float, float>(g, w, tol);
    for (int i = 0; i < 2; ++i) {
        it->r[i] = (float *)w.r[i];
        it->p[i] = (float *)w.p[i];
    }
    it->c = (float *)Z;
    it->xhl = w.xhl;
    it->b = (const float *)Yt;
    return ER_OK;
}

void fp32_init(const GridDev &g, Workspace &w, const void *Yt, void *Z, double tol, Prof *pf) {
    auto a = base_args<float, float>(g, w, tol);
    a.b_in = (const float *)Yt;
    a.r_out = (float *)w.r[0];
    a.x = (float *)Z;
    a.p_out = (float *)w.p[0];
    a.xhl = w.xhl;
    launch_stream<MODE_INIT>(a, w, pf, ER_PASS_OTHER);
}

int fp32_iterate(const GridDev &g, Workspace &w, void *Z, double tol, int cur, Prof *pf) {
    TArgs ta;
    std::memset(&ta, 0, sizeof(ta));
    ta.a = base_args<float, float>(g, w, tol);
    ta.a.r_in = (const float *)w.r[cur];
    ta.a.p_in = (const float *)w.p[cur];
    ta.tm[0] = w.tm_r[cur];
    ta.tm[1] = w.tm_p[cur];
    ta.tm[3] = w.tm_coef;
    launch_tma<MODE_A_DOT>(ta, w, pf, ER_PASS_A);
    ta.a.x = (float *)Z;
    ta.a.r_out = (float *)w.r[1 - cur];
    ta.a.p_out = (float *)w.p[1 - cur];
    ta.a.freeze = 0;
    if (cur == 1) {  // odd iteration: x gains this and the previous iteration's steps
        ta.tm[2] = w.tm_c;
        launch_tma<MODE_B>(ta, w, pf, ER_PASS_B);
    } else {
        launch_tma<MODE_B0>(ta, w, pf, ER_PASS_B0);
    }
    return 1 - cur;
}

void fp32_accum(const GridDev &g, Workspace &w, void *Z, Prof *pf) {
    auto a = base_args<float, float>(g, w, 0.0);
    a.x = (float *)Z;
    a.xhl = w.xhl;
    launch_stream<MODE_ACCUM>(a, w, pf, ER_PASS_OTHER);
}

void fp32_residual(const GridDev &g, Workspace &w, const void *Yt, double tol, int cur_buf, int rmode, Prof *pf) {
    TArgs ta;
    std::memset(&ta, 0, sizeof(ta));
    ta.a = base_args<float, float>(g, w, tol);
    ta.a.xhl = w.xhl;
    ta.a.r_out = (float *)w.r[cur_buf];
    ta.a.rmode = rmode;
    ta.tm[0] = w.tm_xhl;
    ta.tm[1] = w.tm_b;
    ta.tm[3] = w.tm_coef;
    (void)Yt;
    launch_tma<MODE_R>(ta, w, pf, ER_PASS_R);
}

void fp32_final(const GridDev &g, Workspace &w, void *Z, Prof *pf) {
    auto a = base_args<float, float>(g, w, 0.0);
    a.x = (float *)Z;
    a.xhl = w.xhl;
    launch_stream<MODE_UNSCALE>(a, w, pf, ER_PASS_OTHER);
}

}  // namespace er
