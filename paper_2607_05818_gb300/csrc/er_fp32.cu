// FP32 form of the multi-RHS Jacobi-PCG solve, with TMA row staging (sm_103a).
//
// The FP32 iterations apply the network operator in edge-difference form,
//   (G v)_i = pad_i v_i + sum_{j ~ i} g_ij (v_i - v_j),
// with every conductance rounded to FP32 once at grid creation.  The FP64 residual
// b - G x uses exactly the same FP32 conductances (promoted), so the FP32 recursion and
// the FP64 residual see one operator, and the Laplacian structure (zero row sums apart
// from the pads) is exact.  Rounding each conductance by at most a relative u = 2^-24
// keeps every effective resistance within [R/(1+u), R/(1-u)] (Rayleigh monotonicity:
// the perturbed network lies between the original scaled by 1-u and by 1+u).
//
// Jacobi preconditioning: z = D^-1 r with D = diag(G) from the same conductances.
// Passes per iteration (vectors [n][k] FP32, k innermost):
//   A  p' = z + beta p; q = G p'; dot p'.q                          reads r, p
//   B  recompute p', q; x += alpha p'; r' = r - alpha q; dot r'.z'  reads r, p, x;
//                                                                  writes x, r', p'
// Every `replace_every` iterations the correction x is folded into an FP64 iterate
// (x64 += x, x = 0) and the FP64 residual r = b - G x64 replaces the recursive one
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
struct Layout<MODE_R> {  // stage: x64 (FP64), b, coef
    static constexpr int NS = 4, OFF_R = 8192, OFF_P = -1, OFF_X = 0, OFF_COEF = 12288, BYTES = 12800;
};
// dynamic shared memory: NS stages, then a two-row ring of the per-node operand
// (p' in FP32, x64 in FP64), plus slack for 128-byte alignment
template <int MODE>
constexpr int ring_bytes() { return MODE == MODE_R ? 2 * kNX * 256 : 2 * kNX * 128; }
template <int MODE>
constexpr int dyn_smem() { return Layout<MODE>::NS * Layout<MODE>::BYTES + ring_bytes<MODE>() + 128; }

__device__ __forceinline__ float4 lds4(const unsigned char *p) { return *reinterpret_cast<const float4 *>(p); }

// component v of a float4 (v is a compile-time constant after unrolling)
__device__ __forceinline__ float f4(const float4 &f, int v) { return v == 0 ? f.x : v == 1 ? f.y : v == 2 ? f.z : f.w; }

// One pass over a CTA's tile.  Step ri (row y = y0 - 1 + ri) waits for its stage, reads the
// thread's own node from it into registers (r, p or x64, x, coefficients), forms the
// operand v = p' (or x64) and, for row y - 1, finishes q = G v from registers (north,
// centre, south) and the ring (x-neighbours of the centre row); then it publishes v in the
// ring, synchronises once, and the stage is refilled NS rows ahead.
template <int MODE>
__device__ __forceinline__ void tma_pass(const KArgs<float, float> &a, const CUtensorMap *tm0, const CUtensorMap *tm1,
                                         const CUtensorMap *tm2, const CUtensorMap *tm3, int block_id,
                                         unsigned char *smem_raw) {
    using L = Layout<MODE>;
    constexpr int V = 4, KB = kTPN * V;  // 32 columns per CTA
    constexpr bool R64 = MODE == MODE_R;
    using Cv = typename std::conditional<R64, double, float>::type;  // operand type
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
            tma_load4(st + L::OFF_X, tm0, &bars[s], c0, xb, y, t);  // x64
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
    double acc[V] = {0.0, 0.0, 0.0, 0.0};
    int nrun = 0;
#pragma unroll
    for (int v = 0; v < V; ++v) vn[v] = vc[v] = (Cv)0, rc[v] = 0.f;

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
            const double2 lo = *reinterpret_cast<const double2 *>(st + L::OFF_X + xl * 256 + lc * 32);
            const double2 hi = *reinterpret_cast<const double2 *>(st + L::OFF_X + xl * 256 + lc * 32 + 16);
            vs[0] = lo.x; vs[1] = lo.y; vs[2] = hi.x; vs[3] = hi.y;
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
            Cv vw[V], ve[V], q[V];
            if constexpr (R64) {
                const double2 *pw = reinterpret_cast<const double2 *>(rw + (xl - 1) * KB + lc * V);
                const double2 *pe = reinterpret_cast<const double2 *>(rw + (xl + 1) * KB + lc * V);
                vw[0] = pw[0].x; vw[1] = pw[0].y; vw[2] = pw[1].x; vw[3] = pw[1].y;
                ve[0] = pe[0].x; ve[1] = pe[0].y; ve[2] = pe[1].x; ve[3] = pe[1].y;
            } else {
                const float4 w4 = *reinterpret_cast<const float4 *>(rw + (xl - 1) * KB + lc * V);
                const float4 e4 = *reinterpret_cast<const float4 *>(rw + (xl + 1) * KB + lc * V);
                vw[0] = w4.x; vw[1] = w4.y; vw[2] = w4.z; vw[3] = w4.w;
                ve[0] = e4.x; ve[1] = e4.y; ve[2] = e4.z; ve[3] = e4.w;
            }
            const Cv gp = cfc.w, ge = cfc.y, gs = cfc.z, gw = gwc, gn = gsn;
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
                // diagonal form: d v - sum_j g_j v_j, d summed exactly in FP64 from the FP32 g's
                Cv d = gp + ge + gw + gs + gn;
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    Cv qq = -ge * ve[v];
                    qq = fma(-gw, vw[v], qq);
                    qq = fma(-gs, vs[v], qq);
                    qq = fma(-gn, vn[v], qq);
                    q[v] = qq;
                }
                if (cfc.x < 0.f) {
                    const int e1 = a.tsv_ptr[i + 1];
                    for (int e = a.tsv_ptr[i]; e < e1; ++e) {
                        const int64_t jdx = (int64_t)a.tsv_nbr[e] * a.k + col;
                        const double g = a.tsv_g32[e];
                        const double2 lo = *reinterpret_cast<const double2 *>(a.x64 + jdx);
                        const double2 hi = *reinterpret_cast<const double2 *>(a.x64 + jdx + 2);
                        d += g;
                        q[0] = fma(-g, lo.x, q[0]);
                        q[1] = fma(-g, lo.y, q[1]);
                        q[2] = fma(-g, hi.x, q[2]);
                        q[3] = fma(-g, hi.y, q[3]);
                    }
                }
#pragma unroll
                for (int v = 0; v < V; ++v) q[v] = fma(d, vc[v], q[v]);
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
            if (!R64 && cfc.x < 0.f) {  // node with TSV segments (FP32 passes)
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
                    ro[v] = (float)((double)rc[v] - q[v]);
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
                        acc[v] += (double)run[v];
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
                reinterpret_cast<double2 *>(wr)[0] = make_double2(vs[0], vs[1]);
                reinterpret_cast<double2 *>(wr)[1] = make_double2(vs[2], vs[3]);
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
    double *sred = reinterpret_cast<double *>(smem);  // the stage ring is free now
#pragma unroll
    for (int v = 0; v < V; ++v) sred[xl * KB + lc * V + v] = own ? acc[v] + (double)run[v] : 0.0;
    __syncthreads();
    reduce_and_finalize<float, float, MODE, KB>(a, sred, spatial, cb);
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
            if constexpr (MODE == MODE_INIT) {  // r = b, x = 0, p = 0, x64 = 0; dot b.D^-1 b
                float b[V];
                const float z[V] = {0.f, 0.f, 0.f, 0.f};
                ldv<float, float, V>(a.b_in + idx, b);
                const float dinv = fabsf(a.coef[i].x);
                stv<float, float, V>(a.r_out + idx, b);
                stv<float, float, V>(a.x + idx, z);
                stv<float, float, V>(a.p_out + idx, z);
                *reinterpret_cast<double2 *>(a.x64 + idx) = make_double2(0.0, 0.0);
                *reinterpret_cast<double2 *>(a.x64 + idx + 2) = make_double2(0.0, 0.0);
#pragma unroll
                for (int v = 0; v < V; ++v) acc[v].add(dinv * b[v], b[v]);
            } else if constexpr (MODE == MODE_ACCUM) {  // x64 += x; x = 0
                float c[V];
                const float z[V] = {0.f, 0.f, 0.f, 0.f};
                ldv<float, float, V>(a.x + idx, c);
                double2 lo = *reinterpret_cast<const double2 *>(a.x64 + idx);
                double2 hi = *reinterpret_cast<const double2 *>(a.x64 + idx + 2);
                lo.x += (double)c[0]; lo.y += (double)c[1]; hi.x += (double)c[2]; hi.y += (double)c[3];
                *reinterpret_cast<double2 *>(a.x64 + idx) = lo;
                *reinterpret_cast<double2 *>(a.x64 + idx + 2) = hi;
                stv<float, float, V>(a.x + idx, z);
            } else {  // MODE_UNSCALE: Z = x64 rounded to FP32
                const double2 lo = *reinterpret_cast<const double2 *>(a.x64 + idx);
                const double2 hi = *reinterpret_cast<const double2 *>(a.x64 + idx + 2);
                const float o[V] = {(float)lo.x, (float)lo.y, (float)hi.x, (float)hi.y};
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
// shared memory and runs the same pass as the single-network kernels.

template <int MODE>
__device__ __forceinline__ void batch_args(const BatchItem &it, int cur, int rmode, KArgs<float, float> &a) {
    a = it.a;
    a.rmode = rmode;
    if constexpr (MODE == MODE_R) {
        a.x64 = it.x64;
        a.r_out = it.r[cur];
    } else if constexpr (MODE == MODE_INIT) {
        a.b_in = it.b; a.r_out = it.r[0]; a.x = it.c; a.p_out = it.p[0]; a.x64 = it.x64;
    } else if constexpr (MODE == MODE_ACCUM || MODE == MODE_UNSCALE) {
        a.x = it.c; a.x64 = it.x64;
    } else {
        a.r_in = it.r[cur]; a.p_in = it.p[cur]; a.x = it.c;
        a.r_out = it.r[1 - cur]; a.p_out = it.p[1 - cur];
    }
}

template <int MODE>
__global__ void __launch_bounds__(kThreads, MODE == MODE_A_DOT ? 4 : 3)
    k_tma_batch(const BatchItem *__restrict__ items, const int2 *__restrict__ work, int cur, int rmode) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ KArgs<float, float> s_a;
    const int2 wk = work[blockIdx.x];
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
                                                           const int2 *__restrict__ work) {
    __shared__ KArgs<float, float> s_a;
    const int2 wk = work[blockIdx.x];
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

static bool g_attr_done = false;
static bool g_battr_done = false;

er_status fp32_batch_pass(int mode, const BatchItem *items, const int2 *work, int n_work, int cur, int rmode,
                          cudaStream_t s) {
    if (!g_battr_done) {
        ER_CUDA(cudaFuncSetAttribute(k_tma_batch<MODE_A_DOT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     dyn_smem<MODE_A_DOT>()));
        ER_CUDA(cudaFuncSetAttribute(k_tma_batch<MODE_B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     dyn_smem<MODE_B>()));
        ER_CUDA(cudaFuncSetAttribute(k_tma_batch<MODE_B0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     dyn_smem<MODE_B0>()));
        ER_CUDA(cudaFuncSetAttribute(k_tma_batch<MODE_R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     dyn_smem<MODE_R>()));
        g_battr_done = true;
    }
    if (n_work <= 0) return ER_OK;
    const unsigned nb = (unsigned)n_work;
    switch (mode) {
        case MODE_A_DOT: k_tma_batch<MODE_A_DOT><<<nb, kThreads, dyn_smem<MODE_A_DOT>(), s>>>(items, work, cur, rmode); break;
        case MODE_B: k_tma_batch<MODE_B><<<nb, kThreads, dyn_smem<MODE_B>(), s>>>(items, work, cur, rmode); break;
        case MODE_B0: k_tma_batch<MODE_B0><<<nb, kThreads, dyn_smem<MODE_B0>(), s>>>(items, work, cur, rmode); break;
        case MODE_R: k_tma_batch<MODE_R><<<nb, kThreads, dyn_smem<MODE_R>(), s>>>(items, work, cur, rmode); break;
        case MODE_INIT: k_stream_batch<MODE_INIT><<<nb, kThreads, 0, s>>>(items, work); break;
        case MODE_ACCUM: k_stream_batch<MODE_ACCUM><<<nb, kThreads, 0, s>>>(items, work); break;
        case MODE_UNSCALE: k_stream_batch<MODE_UNSCALE><<<nb, kThreads, 0, s>>>(items, work); break;
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
        er_status s = make_map(&w.tm_x64, F64, 8, w.x64, w.k, 32, g);
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
    if (!g_attr_done) {
        ER_CUDA(cudaFuncSetAttribute(k_tma<MODE_A_DOT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     dyn_smem<MODE_A_DOT>()));
        ER_CUDA(cudaFuncSetAttribute(k_tma<MODE_B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     dyn_smem<MODE_B>()));
        ER_CUDA(cudaFuncSetAttribute(k_tma<MODE_B0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     dyn_smem<MODE_B0>()));
        ER_CUDA(cudaFuncSetAttribute(k_tma<MODE_R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     dyn_smem<MODE_R>()));
        g_attr_done = true;
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

void fp32_init(const GridDev &g, Workspace &w, const void *Yt, void *Z, double tol, Prof *pf) {
    auto a = base_args<float, float>(g, w, tol);
    a.b_in = (const float *)Yt;
    a.r_out = (float *)w.r[0];
    a.x = (float *)Z;
    a.p_out = (float *)w.p[0];
    a.x64 = w.x64;
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
    a.x64 = w.x64;
    launch_stream<MODE_ACCUM>(a, w, pf, ER_PASS_OTHER);
}

void fp32_residual(const GridDev &g, Workspace &w, const void *Yt, double tol, int cur_buf, int rmode, Prof *pf) {
    TArgs ta;
    std::memset(&ta, 0, sizeof(ta));
    ta.a = base_args<float, float>(g, w, tol);
    ta.a.x64 = w.x64;
    ta.a.r_out = (float *)w.r[cur_buf];
    ta.a.rmode = rmode;
    ta.tm[0] = w.tm_x64;
    ta.tm[1] = w.tm_b;
    ta.tm[3] = w.tm_coef;
    (void)Yt;
    launch_tma<MODE_R>(ta, w, pf, ER_PASS_R);
}

void fp32_final(const GridDev &g, Workspace &w, void *Z, Prof *pf) {
    auto a = base_args<float, float>(g, w, 0.0);
    a.x = (float *)Z;
    a.x64 = w.x64;
    launch_stream<MODE_UNSCALE>(a, w, pf, ER_PASS_OTHER);
}

}  // namespace er
