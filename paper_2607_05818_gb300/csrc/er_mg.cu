// Aggregation-multigrid preconditioned CG for the FP32 form (sm_103a).
//
// Jacobi-PCG needs about a thousand iterations on 512^2-tier stacks whose upper tiers reach
// the supply only through TSVs.  Here the preconditioner is one V-cycle of an aggregation
// multigrid whose levels are themselves PDN networks:
//   * level l+1 aggregates 2 x 2 nodes of every tier of level l (piecewise-constant
//     prolongation P).  For a graph Laplacian P^T G P is again a graph Laplacian: a segment
//     between two aggregates keeps its conductance (parallel ones add), a segment inside an
//     aggregate vanishes, TSV segments and pads move to their aggregate.  So every coarse
//     operator (the Galerkin product, exactly) is a grid of the same kind, built by
//     er_grid_create from the aggregated network, and every level runs the same stencil;
//   * V-cycle on level l with right-hand side r: z0 = w D^-1 r (one damped-Jacobi sweep
//     from zero), r_c = P^T (r - G z0), z_c = V-cycle on level l+1, z = z0 + s P z_c, and
//     one damped-Jacobi post-sweep z += w D^-1 (r - G z); the coarsest level is solved
//     exactly.  Every step is a fixed linear map and the pre- and post-sweeps are each
//     other's adjoints, so the V-cycle is a symmetric positive definite operator, as CG
//     requires;
//   * the pre-sweep and restriction are one kernel per level, and prolongation and post-sweep
//     another: a CTA owns 16 x 4 aggregates (32 x 8 nodes of the finer level) and 32 RHS
//     columns, staged with a one-node halo by cp.async.bulk.tensor (on the finest level with the
//     rows of its TSV partners on other tiers too); z0 is never stored, it is recomputed from r;
//     the coarsest level (at most 1,024 nodes) is solved exactly by its dense inverse.
// The CG recursion is the FP32 form's (FP32 vectors, double-float dot sums, double-float
// iterate with the accurate residual substituted every replace_every iterations, and whenever
// every column's recursive residual meets tol; a column stops only when that accurate residual
// meets tol, and a column whose recursion ran past its attainable accuracy restarts its search
// direction), in three stages per iteration: the V-cycle (whose last kernel also forms r.z),
// p' = z + beta p with the energy p'.G p', and r -= alpha G p' with G p' recomputed from p'
// (never stored) and r.D^-1 r; x takes two iterations' steps every second iteration.  The
// direction and update passes stage their stencil operand per 32 x 4 node tile the same way.
// Small per-column folds sum per-CTA partials in a fixed order (results are identical from
// run to run).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include <cudaTypedefs.h>

#include "er_common.cuh"

namespace er {

namespace {

constexpr float kOmega = 0.9f;    // damped-Jacobi weight of the smoother (below 1: omega lambda_max(D^-1 G) < 2)
constexpr float kScale = 1.3f;    // over-correction of the coarse-grid correction
constexpr int kCoarseTarget = kMgCoarseNodes;  // coarsen until a level has at most this many nodes
constexpr int kCoarseMax = 2048;     // largest coarsest level (solved by its dense inverse)
constexpr int kMaxSteps = 16;        // node steps per CTA in the streaming layout
constexpr int kMinCtas = 1216;       // small levels: fewer steps, so at least 8 CTAs per SM

struct Lvl {  // one level's device arrays (kernel argument)
    int T, W, H;
    int cb_outer;        // launch order of the tiled kernels: 0 column blocks of a tile adjacent,
                         // 1 column blocks outermost (the same arithmetic either way)
    int64_t n;
    const float4 *coef;  // {+-1/d, gE, gS, pad}; sign < 0: the node has TSV segments
    const int32_t *tsv_ptr, *tsv_nbr;
    const float *tsv_g;
    // TSV segments of the tile pass from this level to the next, grouped by tile (the tiles of
    // 16 x 4 aggregates): tile q's entries are tent[tent_ptr[q] .. tent_ptr[q + 1]), each
    // {i, j, aggregate of j, CSR index e}, node by node in CSR order; null where not built
    const int32_t *tent_ptr;
    const int4 *tent;
};

// Thread layout shared by the node-by-RHS kernels: TPN threads per node (one group of 4
// columns each), NPS nodes per step, `steps` steps per CTA (fewer on small levels, which
// would otherwise run on a handful of CTAs); blockIdx.y picks TPN groups.
struct Lay {
    int KG = 0, TPN = 1, NPS = 256, steps = kMaxSteps;
    int64_t chunks = 0;
    int ncb = 0;
};

Lay make_lay(int64_t n, int k) {
    Lay l;
    l.KG = k / 4;
    while (l.TPN < l.KG && l.TPN < 32) l.TPN <<= 1;
    l.NPS = 256 / l.TPN;
    l.ncb = (l.KG + l.TPN - 1) / l.TPN;
    const int64_t per_cta = (n + (int64_t)kMinCtas / l.ncb - 1) / std::max<int64_t>(1, kMinCtas / l.ncb);
    l.steps = (int)std::max<int64_t>(1, std::min<int64_t>(kMaxSteps, (per_cta + l.NPS - 1) / l.NPS));
    l.chunks = (n + (int64_t)l.NPS * l.steps - 1) / ((int64_t)l.NPS * l.steps);
    return l;
}

__device__ __forceinline__ float4 f4ld(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void f4st(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }
// Four-column arithmetic on the packed FP32 pipe: every float4 operation is two f32x2
// instructions (each lane rounded exactly as the scalar operation), so the stencil bodies
// issue half the FP32 instructions.  a - b is formed as fma(b, -1, a), which rounds once.
__device__ __forceinline__ float2 f2lo(float4 a) { return make_float2(a.x, a.y); }
__device__ __forceinline__ float2 f2hi(float4 a) { return make_float2(a.z, a.w); }
__device__ __forceinline__ float4 f4of(float2 l, float2 h) { return make_float4(l.x, l.y, h.x, h.y); }
__device__ __forceinline__ float4 operator+(float4 a, float4 b) {
    return f4of(__fadd2_rn(f2lo(a), f2lo(b)), __fadd2_rn(f2hi(a), f2hi(b)));
}
__device__ __forceinline__ float4 operator-(float4 a, float4 b) {
    const float2 m = make_float2(-1.f, -1.f);
    return f4of(__ffma2_rn(f2lo(b), m, f2lo(a)), __ffma2_rn(f2hi(b), m, f2hi(a)));
}
__device__ __forceinline__ float4 operator*(float s, float4 a) {
    const float2 s2 = make_float2(s, s);
    return f4of(__fmul2_rn(s2, f2lo(a)), __fmul2_rn(s2, f2hi(a)));
}
__device__ __forceinline__ float4 operator*(float4 a, float4 b) {
    return f4of(__fmul2_rn(f2lo(a), f2lo(b)), __fmul2_rn(f2hi(a), f2hi(b)));
}
__device__ __forceinline__ float4 fma4(float s, float4 a, float4 c) {  // s * a + c
    const float2 s2 = make_float2(s, s);
    return f4of(__ffma2_rn(s2, f2lo(a), f2lo(c)), __ffma2_rn(s2, f2hi(a), f2hi(c)));
}
__device__ __forceinline__ float4 fma4v(float4 a, float4 b, float4 c) {  // a * b + c per column
    return f4of(__ffma2_rn(f2lo(a), f2lo(b), f2lo(c)), __ffma2_rn(f2hi(a), f2hi(b), f2hi(c)));
}
__device__ __forceinline__ float4 zero4() { return make_float4(0.f, 0.f, 0.f, 0.f); }

// ---- TMA-tiled restriction and prolongation ------------------------------------------------
//
// A CTA owns a tile of 16 x 4 aggregates of one tier (32 x 8 nodes of the finer level) and 32
// RHS columns.  One thread issues three cp.async.bulk.tensor loads into shared memory: the
// finer level's r and coefficients over the tile plus a one-node halo (34 x 10 nodes; the box's
// zero fill is the mesh edge) and, for the prolongation, the coarse correction over the tile's
// aggregates plus a one-aggregate halo (18 x 6).  The threads then work from shared memory:
// thread item = (aggregate, group of 4 columns), 8 column groups of 4 aggregates per warp, so
// every quarter-warp reads 128 contiguous bytes.  Only TSV partners (other tiers) are read from
// global memory.  The wait on the loads is bounded: on expiry the CTA raises the error word,
// waits (bounded) for its own copies and returns.

constexpr int TAX = 16, TAY = 4;                 // aggregates per tile
constexpr int TFX = 2 * TAX + 2, TFY = 2 * TAY + 2;  // finer-level nodes per tile, with halo
constexpr int TZX = TAX + 2, TZY = TAY + 2;      // aggregates per tile, with halo
constexpr int TCB = 32;                          // RHS columns per CTA
constexpr int T_R = TFY * TFX * TCB * 4;         // 43,520 bytes
constexpr int T_C = ((TFY * TFX * 16 + 127) / 128) * 128;
constexpr int T_Z = TZY * TZX * TCB * 4;         // 13,824 bytes
constexpr int T_SMEM = T_R + T_C + T_Z + 128;
constexpr int T_SMEM_DOWN = T_R + T_C + 128;     // the restriction stages no coarse correction
// er_solve's tile passes also stage the TSV partners of up to TCAP segments per tile: per entry
// {node, g, w/d of the partner} and the partner's row of r (and of the coarse correction, UP)
constexpr int TCAP = 32;
constexpr int T_SI = TCAP * 16, T_SR = TCAP * TCB * 4;
constexpr int T_SMEM_TS = T_R + T_C + T_Z + T_SI + 2 * T_SR + 128;
constexpr int T_SMEM_DOWN_TS = T_R + T_C + T_SI + T_SR + 128;
constexpr uint32_t kTileSpin = 1u << 22;

int64_t n_tiles(const Lvl &C) {
    return (int64_t)((C.W + TAX - 1) / TAX) * ((C.H + TAY - 1) / TAY) * C.T;
}

dim3 tile_grid(const Lvl &C, int k) { return dim3((unsigned)(n_tiles(C) * ((k + TCB - 1) / TCB))); }

__device__ __forceinline__ uint32_t mg_saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mg_tma4(void *dst, const CUtensorMap *m, uint64_t *bar, int c0, int c1, int c2,
                                        int c3) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(mg_saddr(dst)),
        "l"(reinterpret_cast<uint64_t>(m)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(mg_saddr(bar))
        : "memory");
}

__device__ __forceinline__ bool mg_try_wait(uint64_t *b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(mg_saddr(b)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Issue the tile's loads and wait for them.  Returns false (error word raised) on expiry.
// `init`: the barrier is initialised here (one tile per CTA); otherwise the caller initialised
// it once and `parity` is the phase this tile completes (a CTA looping over tiles).  The
// issuing thread runs `hook` while the copies are in flight.
// Issue the tile's loads and wait for them.  Returns false (error word raised) on expiry.
// `init`: the barrier is initialised here (one tile per CTA); otherwise the caller initialised
// it once and `parity` is the phase this tile completes (a CTA looping over tiles).  The
// issuing thread runs `hook` while the copies are in flight; warp 1 runs `stage` meanwhile
// (extra copies on a barrier of their own, and shared values the CTA barrier below publishes).
template <class Hook, class Stage>
__device__ __forceinline__ bool tile_load(unsigned char *sm, uint64_t *bar, uint32_t parity, bool init,
                                          const CUtensorMap *mr, const CUtensorMap *mc, const CUtensorMap *mz, int c0,
                                          int X0, int Y0, int t, int *err, const Hook &hook, const Stage &stage) {
    if (threadIdx.x == 0) {
        if (init) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mg_saddr(bar)), "r"(1) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        const uint32_t bytes = (uint32_t)(T_R + TFY * TFX * 16 + (mz ? T_Z : 0));
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mg_saddr(bar)), "r"(bytes)
                     : "memory");
        mg_tma4(sm, mr, bar, c0, 2 * X0 - 1, 2 * Y0 - 1, t);
        mg_tma4(sm + T_R, mc, bar, 0, 2 * X0 - 1, 2 * Y0 - 1, t);
        if (mz) mg_tma4(sm + T_R + T_C, mz, bar, c0, X0 - 1, Y0 - 1, t);
        hook();
    } else if (threadIdx.x >= 32 && threadIdx.x < 64) {
        stage();
    }
    // thread 0 waits (bounded) while the other warps wait at the CTA barrier; the vote makes
    // the outcome uniform, and thread 0's acquire plus the barrier make the data visible
    bool done = true;
    if (threadIdx.x == 0)
        for (uint32_t spins = 0; !mg_try_wait(bar, parity);) {
            if (++spins > kTileSpin) {
                done = false;
                break;
            }
        }
    if (__syncthreads_and(done ? 1 : 0)) return true;
    if (threadIdx.x == 0) {  // raise the error word and let this CTA's own copies land first
        atomicExch(err, 1);
        for (uint32_t q = 0; q < kTileSpin && !mg_try_wait(bar, parity); ++q) {
        }
    }
    return false;
}

// 1-D bulk copy global -> shared completing on `bar` (addresses 16-byte aligned, bytes % 16 == 0)
__device__ __forceinline__ void mg_bulk(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            mg_saddr(dst)),
        "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(mg_saddr(bar))
        : "memory");
}

struct TileGeo {
    int X0, Y0, t, c0;
};

// Block -> (tile, column block).  The column blocks of one tile are adjacent in launch order, so
// the CTAs that read the same node rows (each takes a 128-byte slice of them) run together and
// the L2's 256-byte fills are used by both neighbours.
__device__ __forceinline__ TileGeo tile_geo(const Lvl &C, int k, int blk, int &tile) {
    const int ncb = (k + TCB - 1) / TCB;
    const int tx = (C.W + TAX - 1) / TAX, ty = (C.H + TAY - 1) / TAY;
    TileGeo g;
    const int ntile = tx * ty * C.T;
    int b = C.cb_outer ? blk % ntile : blk / ncb;
    tile = b;
    g.c0 = (C.cb_outer ? blk / ntile : blk % ncb) * TCB;
    g.X0 = (b % tx) * TAX;
    b /= tx;
    g.Y0 = (b % ty) * TAY;
    g.t = b / ty;
    return g;
}

// Per-column CTA partials of the CG dot products.  Thread q holds FP32 runs for the 4
// columns of group q % 8; the 32 threads that share a group are summed in a fixed tree order
// in double-float arithmetic (TwoSum, Knuth: s + e = a + b exactly), first across the four
// lanes of a warp (shuffles), then across the 8 warps; one {hi, lo} pair per column is written.
// FP64 arithmetic runs at 1/64 of the FP32 rate on this GPU: an FP64 sum here cost a large
// share of each tile kernel's duration.
__device__ __forceinline__ float2 mg_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return make_float2(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}
__device__ __forceinline__ float2 df_plus(float2 a, float2 b) {  // (hi, lo) + (hi, lo)
    const float2 t = mg_two_sum(a.x, b.x);
    return mg_two_sum(t.x, __fadd_rn(t.y, __fadd_rn(a.y, b.y)));
}
__device__ __forceinline__ void cta_col_partials(const float2 (&run)[4], int k, int c0, int tile, float2 *part) {
    __shared__ float2 sred[8][32];  // [warp][column within the CTA's 32]
    float2 v4[4] = {run[0], run[1], run[2], run[3]};
#pragma unroll
    for (int off = 8; off <= 16; off <<= 1)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const float2 o = make_float2(__shfl_xor_sync(0xffffffffu, v4[v].x, off),
                                         __shfl_xor_sync(0xffffffffu, v4[v].y, off));
            v4[v] = (threadIdx.x & off) ? df_plus(o, v4[v]) : df_plus(v4[v], o);  // same order on both lanes
        }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane < 8)
#pragma unroll
        for (int v = 0; v < 4; ++v) sred[w][lane * 4 + v] = v4[v];
    __syncthreads();
    if (threadIdx.x < TCB) {
        float2 acc = sred[0][threadIdx.x];
#pragma unroll
        for (int q = 1; q < 8; ++q) acc = df_plus(acc, sred[q][threadIdx.x]);
        const int col = c0 + threadIdx.x;
        if (col < k) part[(int64_t)tile * k + col] = acc;
    }
}
__device__ __forceinline__ void ctile_partials(float4 run, int k, int c0, int tile, float2 *part) {
    const float2 r2[4] = {make_float2(run.x, 0.f), make_float2(run.y, 0.f), make_float2(run.z, 0.f),
                          make_float2(run.w, 0.f)};
    cta_col_partials(r2, k, c0, tile, part);
}

// The arrays of one tile pass: finer level F, coarser level C, the finer level's residual r,
// the coarse correction zc (UP), the output (UP: z of F; !UP: the restricted residual of C),
// the dot partials (UP with DOT) and the error word.
struct TileArgs {
    Lvl F, C;
    const float *r, *zc;
    float *out;
    float2 *part;
    int *err;
};

struct NoHook {
    __device__ void operator()() const {}
};

// One item of the tile pass between levels F (finer) and C: aggregate (X, Y) of tier t and the
// 4 columns from `col`.  The accessors take a finer-level node by its offset (dy, dx) from the
// aggregate's first node (-1 .. 2 each: the aggregate's four nodes and the ring around them;
// after unrolling every offset is a constant, so each shared-memory access is a base address
// plus an immediate): the coefficients csm(dy, dx), the residual rsm(dy, dx) and the smoothed
// field sval(dy, dx) (w D^-1 r, for UP plus the scaled coarse correction); tsvt(i, vi, gv) adds
// the TSV terms of node i, g_e (vi - v_j) for its segments e in CSR order (v_j the smoothed
// field at the partner j on another tier), to gv.  UP: z = v + w D^-1
// (r - G v) at the aggregate's four nodes is written to `out` and r.z added to `run`; !UP:
// returns the restricted residual P^T (r - G v) of the aggregate.  An in-plane coupling that is
// 0 (no segment, or the mesh edge, where the staged values are 0) adds exactly 0, so no term
// is skipped.
template <bool UP, bool DOT, class CS, class RS, class SV, class VT>
__device__ __forceinline__ float4 mg_agg(const Lvl &F, int k, int t, int X, int Y, int col, const CS &csm,
                                         const RS &rsm, const SV &sval, const VT &tsvt, float *out, float4 &run) {
    float4 acc = zero4();
    // the smoothed field at the aggregate's own four nodes, computed once: each is the
    // centre of one stencil and a neighbour in two others (only the ring outside the
    // aggregate is evaluated per use, once each)
    float4 sv[2][2];
#pragma unroll
    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
        for (int dx = 0; dx < 2; ++dx) sv[dy][dx] = sval(dy, dx);
    const int64_t i0 = ((int64_t)t * F.H + 2 * Y) * F.W + 2 * X;
#pragma unroll
    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
        for (int dx = 0; dx < 2; ++dx) {
            if (2 * X + dx >= F.W || 2 * Y + dy >= F.H) continue;
            const float4 c = csm(dy, dx);
            const int i = (int)(i0 + (int64_t)dy * F.W + dx);
            if (c.x == 0.f) {  // floating node: not in P, z = 0
                if constexpr (UP) f4st(out + (int64_t)i * k + col, zero4());
                continue;
            }
            const float4 ri = rsm(dy, dx);
            const float4 vi = sv[dy][dx];
            float4 gv = c.w * vi;
            gv = fma4(c.y, vi - (dx == 0 ? sv[dy][1] : sval(dy, dx + 1)), gv);                // east
            gv = fma4(csm(dy, dx - 1).y, vi - (dx == 1 ? sv[dy][0] : sval(dy, dx - 1)), gv);  // west
            gv = fma4(c.z, vi - (dy == 0 ? sv[1][dx] : sval(dy + 1, dx)), gv);                // south
            gv = fma4(csm(dy - 1, dx).z, vi - (dy == 1 ? sv[0][dx] : sval(dy - 1, dx)), gv);  // north
            if (c.x < 0.f) gv = tsvt(i, vi, gv);
            if constexpr (UP) {
                const float4 zo = fma4(kOmega * fabsf(c.x), ri - gv, vi);
                f4st(out + (int64_t)i * k + col, zo);
                if constexpr (DOT) run = fma4v(ri, zo, run);
            } else {
                acc = acc + (ri - gv);
            }
        }
    return acc;
}

// prolongation + post-sweep (UP) or pre-sweep + restriction (!UP) over tile block `blk` of the
// level pair (ta.F, ta.C); false if the wait on the tile's loads expired (error word raised).
// `ta` may live in shared memory (read where used) or be built from kernel parameters.  TS (one
// tile per CTA): while the tile is in flight, warp 1 stages the tile's TSV partners (ta.F.tent)
// by bulk copies on a second barrier `bar2`, and the TSV terms read them from shared memory
// after waiting on it; a tile with more than TCAP segments, or a level without the table,
// reads them from global memory.  The values are the same either way.
template <bool UP, bool DOT, bool TS = false, class TA, class Hook>
__device__ __forceinline__ bool mg_tile_body(unsigned char *sm, uint64_t *bar, uint32_t parity, bool init, int blk,
                                             const CUtensorMap *mr, const CUtensorMap *mc, const CUtensorMap *mz,
                                             const TA &ta, int k, const Hook &hook, uint64_t *bar2 = nullptr) {
    const Lvl &F = ta.F, &C = ta.C;
    const float *rs = reinterpret_cast<const float *>(sm);
    const float4 *cs = reinterpret_cast<const float4 *>(sm + T_R);
    const float *zs = reinterpret_cast<const float *>(sm + T_R + T_C);
    // TS: the staged entries after the tile's regions
    unsigned char *st = sm + T_R + T_C + (UP ? T_Z : 0);
    float4 *s_info = reinterpret_cast<float4 *>(st);              // {node i (bits), g, w/d_j, 0}
    float *s_rr = reinterpret_cast<float *>(st + T_SI);            // partner rows of r
    float *s_rz = reinterpret_cast<float *>(st + T_SI + T_SR);     // partner rows of the coarse correction
    __shared__ int s_ne;                                           // staged entries, -1: not staged
    int tile;
    const TileGeo g = tile_geo(C, k, blk, tile);
    const auto stage = [&]() {  // warp 1
        if constexpr (TS) {
            const int lane = (int)threadIdx.x - 32;
            if (lane == 0) {
                asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mg_saddr(bar2)), "r"(1) : "memory");
                asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            }
            __syncwarp();
            const int p0 = F.tent_ptr ? F.tent_ptr[tile] : 0, p1 = F.tent_ptr ? F.tent_ptr[tile + 1] : 0;
            const int ne = F.tent_ptr && p1 - p0 <= TCAP ? p1 - p0 : -1;
            if (lane == 0) s_ne = ne;
            if (lane < ne) {
                const int4 en = F.tent[p0 + lane];  // {i, j, aggregate of j, e}
                const uint32_t bytes = (uint32_t)(min(TCB, k - g.c0) * 4);
                asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(mg_saddr(bar2)),
                             "r"(UP ? 2 * bytes : bytes)
                             : "memory");
                mg_bulk(s_rr + lane * TCB, ta.r + (int64_t)en.y * k + g.c0, bytes, bar2);
                if constexpr (UP) mg_bulk(s_rz + lane * TCB, ta.zc + (int64_t)en.z * k + g.c0, bytes, bar2);
                s_info[lane] = make_float4(__int_as_float(en.x), F.tsv_g[en.w], kOmega * fabsf(F.coef[en.y].x), 0.f);
            }
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mg_saddr(bar2)) : "memory");
        }
    };
    const bool ok = tile_load(sm, bar, parity, init, mr, mc, UP ? mz : nullptr, g.c0, g.X0, g.Y0, g.t, ta.err, hook,
                              stage);
    if (!ok) return false;
    const int Wc = C.W, WcHc = C.W * C.H;
    float4 run[2] = {zero4(), zero4()};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int item = threadIdx.x + 256 * h;
        const int cg = item & 7, a = item >> 3;
        const int ax = a % TAX, ay = a / TAX;
        const int X = g.X0 + ax, Y = g.Y0 + ay;
        const int col = g.c0 + cg * 4;
        if (X >= C.W || Y >= C.H || col >= k) continue;
        const int J = (g.t * C.H + Y) * Wc + X;
        // the aggregate's first node is tile node (1 + 2 ay, 1 + 2 ax); its coarse correction
        // is at (ay + 1, ax + 1) of the coarse tile (one-aggregate halo)
        const float4 *cb = cs + (1 + 2 * ay) * TFX + (1 + 2 * ax);
        const float *rb = rs + ((1 + 2 * ay) * TFX + (1 + 2 * ax)) * TCB + cg * 4;
        const float *zb = zs + ((ay + 1) * TZX + (ax + 1)) * TCB + cg * 4;
        const auto csm = [&](int dy, int dx) { return cb[dy * TFX + dx]; };
        const auto rsm = [&](int dy, int dx) { return *reinterpret_cast<const float4 *>(rb + (dy * TFX + dx) * TCB); };
        const auto sval = [&](int dy, int dx) {
            float4 v = (kOmega * fabsf(csm(dy, dx).x)) * rsm(dy, dx);
            if constexpr (UP)  // node offset -1 lies in the aggregate before, 2 in the one after
                v = fma4(kScale,
                         *reinterpret_cast<const float4 *>(zb + ((((dy + 2) >> 1) - 1) * TZX + (((dx + 2) >> 1) - 1)) *
                                                                    TCB),
                         v);
            return v;
        };
        const auto tsvt = [&](int i, float4 vi, float4 gv) {
            int ne = TS ? s_ne : -1;
            if (ne > 0) {  // the staged rows have landed (bounded wait; on expiry: global memory)
                bool ok = false;
                for (uint32_t q = 0; q < kTileSpin && !(ok = mg_try_wait(bar2, 0u));) ++q;
                if (!ok) {
                    atomicExch(ta.err, 1);
                    ne = -1;
                }
            }
            if (ne >= 0) {  // staged: node i's entries, in CSR order
                for (int q = 0; q < ne; ++q) {
                    const float4 in = s_info[q];
                    if (__float_as_int(in.x) != i) continue;
                    float4 v = in.z * *reinterpret_cast<const float4 *>(s_rr + q * TCB + cg * 4);
                    if constexpr (UP) v = fma4(kScale, *reinterpret_cast<const float4 *>(s_rz + q * TCB + cg * 4), v);
                    gv = fma4(in.y, vi - v, gv);
                }
                return gv;
            }
            const int32_t e1 = F.tsv_ptr[i + 1];
            for (int32_t e = F.tsv_ptr[i]; e < e1; ++e) {  // TSV partner on another tier (global memory)
                const int j = F.tsv_nbr[e];
                float4 v = (kOmega * fabsf(F.coef[j].x)) * f4ld(ta.r + (int64_t)j * k + col);
                if constexpr (UP) v = fma4(kScale, f4ld(ta.zc + (int64_t)(J + (j > i ? WcHc : -WcHc)) * k + col), v);
                gv = fma4(F.tsv_g[e], vi - v, gv);
            }
            return gv;
        };
        const float4 acc = mg_agg<UP, DOT>(F, k, g.t, X, Y, col, csm, rsm, sval, tsvt, ta.out, run[h]);
        if constexpr (!UP) f4st(ta.out + (int64_t)J * k + col, acc);
    }
    if constexpr (TS)  // no staged copy may still be landing when the CTA exits
        if (threadIdx.x == 0 && s_ne > 0)
            for (uint32_t q = 0; q < kTileSpin && !mg_try_wait(bar2, 0u); ++q) {
            }
    if constexpr (DOT) {
        // per column: the 64 items of the tile that share it (two per thread), summed in a fixed order
        const float2 r2[4] = {mg_two_sum(run[0].x, run[1].x), mg_two_sum(run[0].y, run[1].y),
                              mg_two_sum(run[0].z, run[1].z), mg_two_sum(run[0].w, run[1].w)};
        cta_col_partials(r2, k, g.c0, tile, ta.part);
    }
    return true;
}

template <bool UP, bool DOT, bool TS>
__global__ void __launch_bounds__(256, UP ? 3 : 4) k_mg_tile(const __grid_constant__ CUtensorMap mr,
                                                 const __grid_constant__ CUtensorMap mc,
                                                 const __grid_constant__ CUtensorMap mz, Lvl F, Lvl C, int k,
                                                 const float *__restrict__ r, const float *__restrict__ zc,
                                                 float *__restrict__ out, float2 *part, int *err) {
    extern __shared__ unsigned char mg_tile_raw[];
    __shared__ __align__(8) uint64_t bar, bar2;
    unsigned char *sm = mg_tile_raw + ((128u - (mg_saddr(mg_tile_raw) & 127u)) & 127u);
    const TileArgs a{F, C, r, zc, out, part, err};
    mg_tile_body<UP, DOT, TS>(sm, &bar, 0u, true, (int)blockIdx.x, &mr, &mc, &mz, a, k, NoHook{}, &bar2);
}

// ---- TMA-tiled CG passes on the finest level ---------------------------------------------
//
// A CTA owns 32 x 4 nodes of one tier and 32 RHS columns; the operands that the stencil needs
// at neighbours are staged by cp.async.bulk.tensor with a one-node halo (zero fill at the mesh
// edge): the direction pass loads z and p over x0..x0+32, y0..y0+4 (east and south halo only:
// its energy form needs those two neighbours), the update pass loads p' over x0-1..x0+32,
// y0-1..y0+4.  Operands needed only at the node itself (r, x, p'_prev) are plain coalesced
// float4 loads.  Items: (node, group of 4 columns), 8 column groups of 4 nodes per warp.

constexpr int CX = 32, CY = 4;                     // interior nodes per tile
constexpr int SPX = CX + 1, SPY = CY + 1;          // direction pass: east/south halo
constexpr int UPX = CX + 2, UPY = CY + 2;          // update pass: halo on every side
constexpr int S_V = SPY * SPX * TCB * 4;           // 21,120 bytes per vector
constexpr int S_C = ((SPY * SPX * 16 + 127) / 128) * 128;
constexpr int S_SMEM = 2 * S_V + S_C + 128;
constexpr int U_V = UPY * UPX * TCB * 4;           // 26,112 bytes
constexpr int U_C = ((UPY * UPX * 16 + 127) / 128) * 128;
constexpr int U_SMEM = U_V + U_C + 128;

int64_t n_ctiles(const Lvl &F) { return (int64_t)((F.W + CX - 1) / CX) * ((F.H + CY - 1) / CY) * F.T; }
dim3 ctile_grid(const Lvl &F, int k) { return dim3((unsigned)(n_ctiles(F) * ((k + TCB - 1) / TCB))); }

// After thread 0 issued the tile's loads: a bounded wait, made CTA-uniform.  Thread 0 alone
// polls the barrier (its acquire, then the CTA barrier, make the copied data visible to every
// thread); the other warps wait at the CTA barrier without taking issue slots from the
// co-resident CTAs' arithmetic.  The CTA barrier also publishes the shared values the threads
// wrote before the call.
__device__ __forceinline__ bool ctile_wait(uint64_t *bar, uint32_t parity, int *err) {
    bool done = true;
    if (threadIdx.x == 0)
        for (uint32_t spins = 0; !mg_try_wait(bar, parity);) {
            if (++spins > kTileSpin) {
                done = false;
                break;
            }
        }
    if (__syncthreads_and(done ? 1 : 0)) return true;
    if (threadIdx.x == 0) {
        atomicExch(err, 1);
        for (uint32_t q = 0; q < kTileSpin && !mg_try_wait(bar, parity); ++q) {
        }
    }
    return false;
}

// thread 0: (once per CTA, if `init`) initialise the barrier, then expect `bytes` on it
__device__ __forceinline__ void bar_init_expect(uint64_t *bar, uint32_t bytes, bool init) {
    if (init) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mg_saddr(bar)), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mg_saddr(bar)), "r"(bytes) : "memory");
}

struct CGeo {
    int x0, y0, t, c0;
};
__device__ __forceinline__ CGeo ctile_geo(const Lvl &F, int k, int blk, int &tile) {
    const int ncb = (k + TCB - 1) / TCB;
    const int tx = (F.W + CX - 1) / CX, ty = (F.H + CY - 1) / CY;
    CGeo g;
    const int ntile = tx * ty * F.T;
    int b = F.cb_outer ? blk % ntile : blk / ncb;
    tile = b;
    g.c0 = (F.cb_outer ? blk / ntile : blk % ncb) * TCB;
    g.x0 = (b % tx) * CX;
    b /= tx;
    g.y0 = (b % ty) * CY;
    g.t = b / ty;
    return g;
}

// p' = z + beta p over tile block `blk`; partials of p'.G p' in edge form (pad, east, south,
// half TSV).  False if the wait on the tile's loads expired (error word raised).  The issuing
// thread runs `hook` while the copies are in flight.
template <class Hook>
__device__ __forceinline__ bool mg_dir_body(unsigned char *sm, uint64_t *bar, uint32_t parity, bool init, int blk,
                                            const CUtensorMap *mzt, const CUtensorMap *mpt, const CUtensorMap *mct,
                                            const Lvl &F, int k, const float *__restrict__ z,
                                            const float *__restrict__ p, const double *__restrict__ beta,
                                            float *__restrict__ p_out, float2 *part, int *err, const Hook &hook) {
    const float *zs = reinterpret_cast<const float *>(sm);
    const float *ps = reinterpret_cast<const float *>(sm + S_V);
    const float4 *cs = reinterpret_cast<const float4 *>(sm + 2 * S_V);
    int tile;
    const CGeo g = ctile_geo(F, k, blk, tile);
    if (threadIdx.x == 0) {
        bar_init_expect(bar, (uint32_t)(2 * S_V + SPY * SPX * 16), init);
        mg_tma4(sm, mzt, bar, g.c0, g.x0, g.y0, g.t);
        mg_tma4(sm + S_V, mpt, bar, g.c0, g.x0, g.y0, g.t);
        mg_tma4(sm + 2 * S_V, mct, bar, 0, g.x0, g.y0, g.t);
        hook();
    }
    __shared__ __align__(16) float s_b[TCB];  // beta in FP32, one conversion per column
    if (threadIdx.x < TCB) s_b[threadIdx.x] = g.c0 + (int)threadIdx.x < k ? (float)beta[g.c0 + threadIdx.x] : 0.f;
    if (!ctile_wait(bar, parity, err)) return false;
    float4 run4 = zero4();
    const int cg = threadIdx.x & 7;
    const int col = g.c0 + cg * 4;
    const float4 b4 = *reinterpret_cast<const float4 *>(s_b + cg * 4);
    // this thread: tile column lx, rows 0..3; shared-memory bases so that every access below is
    // a base plus a constant offset
    const int lx = threadIdx.x >> 3, x = g.x0 + lx;
    const float4 *cb = cs + lx;
    const float *pb = ps + lx * TCB + cg * 4, *zb = zs + lx * TCB + cg * 4;
    auto sv = [&](int dy, int dx) {
        const int o = (dy * SPX + dx) * TCB;
        return fma4v(b4, *reinterpret_cast<const float4 *>(pb + o), *reinterpret_cast<const float4 *>(zb + o));
    };
    const int i0 = (g.t * F.H + g.y0) * F.W + x;
    float *po = p_out + (int64_t)i0 * k + col;
    const int64_t row_k = (int64_t)F.W * k;
    if (x < F.W && col < k)
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            if (g.y0 + h >= F.H) break;
            const float4 c = cb[h * SPX];
            float4 pv = zero4();
            if (c.x != 0.f) {
                pv = sv(h, 0);
                float4 en = c.w * (pv * pv);
                {  // east and south edges (a coupling of 0 adds exactly 0: the staged values are finite)
                    const float4 de = pv - sv(h, 1);
                    en = fma4(c.y, de * de, en);
                    const float4 ds = pv - sv(h + 1, 0);
                    en = fma4(c.z, ds * ds, en);
                }
                if (c.x < 0.f) {
                    const int i = i0 + h * F.W;
                    const int32_t e1 = F.tsv_ptr[i + 1];
                    for (int32_t e = F.tsv_ptr[i]; e < e1; ++e) {
                        const int64_t oj = (int64_t)F.tsv_nbr[e] * k + col;
                        const float4 d = pv - fma4v(b4, f4ld(p + oj), f4ld(z + oj));
                        en = fma4(0.5f * F.tsv_g[e], d * d, en);
                    }
                }
                run4 = run4 + en;
            }
            f4st(po + h * row_k, pv);
        }
    ctile_partials(run4, k, g.c0, tile, part);
    return true;
}

__global__ void __launch_bounds__(256, 4) k_mg_dir_tile(const __grid_constant__ CUtensorMap mzt,
                                                     const __grid_constant__ CUtensorMap mpt,
                                                     const __grid_constant__ CUtensorMap mct, Lvl F, int k,
                                                     const float *__restrict__ z, const float *__restrict__ p,
                                                     const double *__restrict__ beta, float *__restrict__ p_out,
                                                     float2 *part, int *err) {
    extern __shared__ unsigned char mg_dir_raw[];
    __shared__ __align__(8) uint64_t bar;
    unsigned char *sm = mg_dir_raw + ((128u - (mg_saddr(mg_dir_raw) & 127u)) & 127u);
    mg_dir_body(sm, &bar, 0u, true, (int)blockIdx.x, &mzt, &mpt, &mct, F, k, z, p, beta, p_out, part, err, NoHook{});
}

// q = G p' at one node in edge form: the pad term, then the east, west, south and north
// couplings (c.y, gw, c.z, gn; 0 where there is no segment, and p' there is a finite staged
// value, so such a term adds exactly 0), from p' at the node (pv) and at its in-plane
// neighbours pat(dy, dx); the TSV terms follow (mg_gq_tsv).
template <class PA>
__device__ __forceinline__ float4 mg_gq(float4 c, float gw, float gn, float4 pv, const PA &pat) {
    float4 q = c.w * pv;
    q = fma4(c.y, pv - pat(0, 1), q);
    q = fma4(gw, pv - pat(0, -1), q);
    q = fma4(c.z, pv - pat(1, 0), q);
    q = fma4(gn, pv - pat(-1, 0), q);
    return q;
}
// the TSV terms of node i (other tiers; p' read from global memory), in CSR order
__device__ __forceinline__ float4 mg_gq_tsv(const Lvl &F, int i, int k, int col, const float *__restrict__ p,
                                            float4 pv, float4 q) {
    const int32_t e1 = F.tsv_ptr[i + 1];
    for (int32_t e = F.tsv_ptr[i]; e < e1; ++e) q = fma4(F.tsv_g[e], pv - f4ld(p + (int64_t)F.tsv_nbr[e] * k + col), q);
    return q;
}

// r -= alpha G p' with G p' from the staged p' tile of block `blk`; partials of r.D^-1 r; with
// XPAIR also x += alpha_prev p'_prev + alpha p'.  False if the wait on the tile's loads expired.
// The issuing thread runs `hook` while the copies are in flight.
template <bool XPAIR, class Hook>
__device__ __forceinline__ bool mg_upd_body(unsigned char *sm, uint64_t *bar, uint32_t parity, bool init, int blk,
                                            const CUtensorMap *mpt, const CUtensorMap *mct, const Lvl &F, int k,
                                            const double *__restrict__ alpha, const double *__restrict__ alpha_prev,
                                            const float *__restrict__ p, const float *__restrict__ p_prev,
                                            float *__restrict__ x, float *__restrict__ r, float2 *part, int *err,
                                            const Hook &hook) {
    const float *ps = reinterpret_cast<const float *>(sm);
    const float4 *cs = reinterpret_cast<const float4 *>(sm + U_V);
    int tile;
    const CGeo g = ctile_geo(F, k, blk, tile);
    if (threadIdx.x == 0) {
        bar_init_expect(bar, (uint32_t)(U_V + UPY * UPX * 16), init);
        mg_tma4(sm, mpt, bar, g.c0, g.x0 - 1, g.y0 - 1, g.t);
        mg_tma4(sm + U_V, mct, bar, 0, g.x0 - 1, g.y0 - 1, g.t);
        hook();
    }
    // r (and for the x update x and p'_prev) are read straight from global memory after
    // the stencil; ask L2 for their 128-byte row slices now, so that the DRAM reads overlap
    // the wait for the tile's bulk copy (one thread per node row slice: column group 0)
    if ((threadIdx.x & 7) == 0 && g.c0 < k) {
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const int node = (threadIdx.x >> 3) + 32 * h;
            const int xg = g.x0 + node % CX, yg = g.y0 + node / CX;
            if (xg >= F.W || yg >= F.H) continue;
            const int64_t o = ((int64_t)(g.t * F.H + yg) * F.W + xg) * k + g.c0;
            asm volatile("prefetch.global.L2 [%0];" ::"l"(r + o));
            if constexpr (XPAIR) {
                asm volatile("prefetch.global.L2 [%0];" ::"l"(x + o));
                asm volatile("prefetch.global.L2 [%0];" ::"l"(p_prev + o));
            }
        }
    }
    // the CTA's 32 step lengths, converted to FP32 once per column (an FP64 -> FP32
    // conversion runs on the FP64 pipe: one per thread and column kept it 18% busy)
    __shared__ __align__(16) float s_a[TCB], s_ap[TCB];
    if (threadIdx.x < TCB) {
        const int j = g.c0 + threadIdx.x;
        s_a[threadIdx.x] = j < k ? (float)alpha[j] : 0.f;
        if constexpr (XPAIR) s_ap[threadIdx.x] = j < k ? (float)alpha_prev[j] : 0.f;
    }
    if (!ctile_wait(bar, parity, err)) return false;
    float4 run4 = zero4();
    const int cg = threadIdx.x & 7;
    const int col = g.c0 + cg * 4;
    const float4 a4 = *reinterpret_cast<const float4 *>(s_a + cg * 4);
    const float4 na4 = make_float4(-a4.x, -a4.y, -a4.z, -a4.w);
    const float4 ap4 = XPAIR ? *reinterpret_cast<const float4 *>(s_ap + cg * 4) : zero4();
    // this thread: tile column lx0, rows 0..3 (staged slot (1 + h, 1 + lx0)); shared-memory bases
    // so that every access below is a base plus a constant offset
    const int lx0 = threadIdx.x >> 3, xg = g.x0 + lx0;
    const float4 *cb = cs + UPX + 1 + lx0;
    const float *pb = ps + (UPX + 1 + lx0) * TCB + cg * 4;
    auto pv_at = [&](int dy, int dx) { return *reinterpret_cast<const float4 *>(pb + (dy * UPX + dx) * TCB); };
    const int i0 = (g.t * F.H + g.y0) * F.W + xg;
    const int64_t o0 = (int64_t)i0 * k + col, row_k = (int64_t)F.W * k;
    if (xg < F.W && col < k)
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            if (g.y0 + h >= F.H) break;
            const float4 c = cb[h * UPX];
            if (c.x == 0.f) continue;  // floating: r, x and p' stay 0
            const float4 pv = pv_at(h, 0);
            float4 q = mg_gq(c, cb[h * UPX - 1].y, cb[(h - 1) * UPX].z, pv,
                             [&](int dy, int dx) { return pv_at(h + dy, dx); });
            if (c.x < 0.f) q = mg_gq_tsv(F, i0 + h * F.W, k, col, p, pv, q);
            const int64_t o = o0 + h * row_k;
            const float4 rv = fma4v(na4, q, f4ld(r + o));
            f4st(r + o, rv);
            if constexpr (XPAIR) f4st(x + o, fma4v(a4, pv, fma4v(ap4, f4ld(p_prev + o), f4ld(x + o))));
            const float di = fabsf(c.x);
            run4 = fma4v(di * rv, rv, run4);
        }
    ctile_partials(run4, k, g.c0, tile, part);
    return true;
}

template <bool XPAIR>
__global__ void __launch_bounds__(256, 4) k_mg_upd_tile(const __grid_constant__ CUtensorMap mpt,
                                                     const __grid_constant__ CUtensorMap mct, Lvl F, int k,
                                                     const double *__restrict__ alpha,
                                                     const double *__restrict__ alpha_prev,
                                                     const float *__restrict__ p, const float *__restrict__ p_prev,
                                                     float *__restrict__ x, float *__restrict__ r, float2 *part,
                                                     int *err) {
    extern __shared__ unsigned char mg_upd_raw[];
    __shared__ __align__(8) uint64_t bar;
    unsigned char *sm = mg_upd_raw + ((128u - (mg_saddr(mg_upd_raw) & 127u)) & 127u);
    mg_upd_body<XPAIR>(sm, &bar, 0u, true, (int)blockIdx.x, &mpt, &mct, F, k, alpha, alpha_prev, p, p_prev, x, r,
                       part, err, NoHook{});
}

// coarsest level, solved exactly: z = G_c^-1 r with the dense inverse (FP32, symmetric,
// zero rows and columns at floating nodes) computed once on the host.  A dense product
// [n_c x ld] x [ld x k]: each CTA owns a 32-row x 32-column tile of z.  Per step it stages 128
// rows of the inverse restricted to the tile's 32 columns (by symmetry, the tile's 32 rows
// restricted to those 128 columns) and 128 rows of r restricted to the tile's 32 columns; the
// CTA's four thread groups each take 32 of the 128 (group q: 32 q .. 32 q + 31 of every step)
// and a thread accumulates a 4 x 4 block of z; the four groups' sums are added in a fixed
// order at the end.  ld % 4 == 0; the inverse's columns n_c .. ld-1 are zero and r has ld rows
// (rows n_c .. ld-1 zero).
constexpr int CI_T = 32, CI_J = 128;
dim3 cinv_grid(int64_t n, int k) { return dim3((unsigned)((n + CI_T - 1) / CI_T), (unsigned)((k + CI_T - 1) / CI_T)); }

// the tile of row block bx and column block by
__device__ __forceinline__ void mg_cinv_body(int bx, int by, int n, int ld, int k, const float *__restrict__ ainv,
                                             const float *__restrict__ r, float *__restrict__ z) {
    __shared__ __align__(16) float As[CI_J][CI_T];  // As[jj][i] = inverse (row0 + i, j0 + jj)
    __shared__ __align__(16) float Rs[CI_J][CI_T];  // Rs[jj][c] = r (j0 + jj, col0 + c)
    const int row0 = bx * CI_T, col0 = by * CI_T;
    const int grp = threadIdx.x >> 6, q = threadIdx.x & 63;
    const int ri = (q >> 3) * 4, ci = (q & 7) * 4;  // this thread: rows ri .. ri+3, columns ci .. ci+3
    float4 acc[4] = {zero4(), zero4(), zero4(), zero4()};
    for (int j0 = 0; j0 < ld; j0 += CI_J) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int e = threadIdx.x + 256 * u;  // staged row jj = e / 8, 4 values from (e % 8) * 4
            const int jj = e >> 3, c4 = (e & 7) * 4, j = j0 + jj;
            const bool oka = j < n && row0 + c4 < ld;
            const bool okr = j < ld && col0 + c4 < k;
            *reinterpret_cast<float4 *>(&As[jj][c4]) =
                oka ? *reinterpret_cast<const float4 *>(ainv + (int64_t)j * ld + row0 + c4) : zero4();
            *reinterpret_cast<float4 *>(&Rs[jj][c4]) = okr ? f4ld(r + (int64_t)j * k + col0 + c4) : zero4();
        }
        __syncthreads();
#pragma unroll 8
        for (int jj = grp * (CI_J / 4); jj < (grp + 1) * (CI_J / 4); ++jj) {
            const float4 a = *reinterpret_cast<const float4 *>(&As[jj][ri]);
            const float4 b = *reinterpret_cast<const float4 *>(&Rs[jj][ci]);
            acc[0] = fma4(a.x, b, acc[0]);
            acc[1] = fma4(a.y, b, acc[1]);
            acc[2] = fma4(a.z, b, acc[2]);
            acc[3] = fma4(a.w, b, acc[3]);
        }
        __syncthreads();
    }
    float4 *red = reinterpret_cast<float4 *>(&As[0][0]);  // groups 1..3: [3][64][4] float4, 12 KiB
    if (grp > 0)
#pragma unroll
        for (int u = 0; u < 4; ++u) red[((grp - 1) * 64 + q) * 4 + u] = acc[u];
    __syncthreads();
    if (grp != 0) return;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const float4 s = ((acc[u] + red[q * 4 + u]) + red[(64 + q) * 4 + u]) + red[(128 + q) * 4 + u];
        const int row = row0 + ri + u;
        if (row < n && col0 + ci < k) f4st(z + (int64_t)row * k + col0 + ci, s);
    }
}

__global__ void __launch_bounds__(256) k_mg_cinv(int n, int ld, int k, const float *__restrict__ ainv,
                                                 const float *__restrict__ r, float *__restrict__ z) {
    mg_cinv_body((int)blockIdx.x, (int)blockIdx.y, n, ld, k, ainv, r, z);
}

// ---- per-column folds (one CTA per column, partials summed in a fixed tree order) -------

enum { FOLD_ALPHA = 0, FOLD_RR = 1, FOLD_BETA = 2 };

struct FoldArgs {
    const float2 *part;  // per-CTA partials as double-float {hi, lo}
    int64_t chunks;
    int k;
    double *alpha, *beta, *rho, *rho0;
    double *relrec;  // recursive residual ||r||_{D^-1} / ||b||_{D^-1} per column (FOLD_RR)
    double *alpha_prev;  // FOLD_ALPHA keeps the previous alpha (x is updated in pairs)
    int *active;
    int *nunc;  // columns still above tol (FOLD_RR adds, FOLD_BETA resets)
    double tol;
};

// column j of one network's fold
template <int KIND>
__device__ __forceinline__ void mg_fold_body(const FoldArgs &f, int j) {
    __shared__ float2 s[256];
    float2 acc = make_float2(0.f, 0.f);
    for (int64_t c = threadIdx.x; c < f.chunks; c += blockDim.x) acc = df_plus(acc, f.part[c * f.k + j]);
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) s[threadIdx.x] = df_plus(s[threadIdx.x], s[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    const double tot = (double)s[0].x + (double)s[0].y;
    const bool act = f.active[j] != 0;
    if constexpr (KIND == FOLD_ALPHA) {
        f.alpha_prev[j] = f.alpha[j];
        f.alpha[j] = (act && tot > 0.0 && isfinite(tot)) ? f.rho[j] / tot : 0.0;
    } else if constexpr (KIND == FOLD_RR) {
        const double rel = f.rho0[j] > 0.0 ? sqrt(tot / f.rho0[j]) : 0.0;
        f.relrec[j] = rel;
        if (act && rel > f.tol) atomicAdd(f.nunc, 1);
    } else {  // FOLD_BETA: rho' = r.z
        if (j == 0) *f.nunc = 0;
        if (act && f.rho[j] > 0.0 && tot > 0.0 && isfinite(tot)) {
            f.beta[j] = tot / f.rho[j];
            f.rho[j] = tot;
        } else {
            f.beta[j] = 0.0;
            if (act && tot > 0.0 && isfinite(tot)) f.rho[j] = tot;
        }
    }
}

template <int KIND>
__global__ void __launch_bounds__(256) k_mg_fold(FoldArgs f) {
    mg_fold_body<KIND>(f, (int)blockIdx.x);
}

// after an accurate residual replacement: freeze the columns whose accurate residual meets
// tol and count the rest.  A column whose recursive residual has run more than 100x below the
// accurate one, or claims tol while the accurate residual does not, has a stale search direction (the
// recursion went on past its attainable accuracy): rho = 0 makes the next beta fold
// restart it (beta = 0), as rescaling a stale direction stalls CG.
__device__ __forceinline__ void mg_freeze_col(int j, const double *resid, const double *relrec, double tol,
                                              int *active, double *rho, int *nact) {
    const double tr = resid[j], rec = relrec[j];
    if (active[j] && (!(rec > 0.0) || rec < 1e-2 * tr || (!(rec > tol) && tr > tol))) rho[j] = 0.0;
    if (active[j] && !(tr > tol)) active[j] = 0;
    if (active[j]) atomicAdd(nact, 1);
}

__global__ void k_mg_freeze(int k, const double *resid, const double *relrec, double tol, int *active, double *rho,
                            int *nact) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < k) mg_freeze_col(j, resid, relrec, tol, active, rho, nact);
}

unsigned ublocks(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

// ---- tensor maps of the tiled kernels ------------------------------------------------------

static PFN_cuTensorMapEncodeTiled_v12000 mg_encode() {
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

// 4-D FP32 map over [T][H][W][d0] (d0 innermost) with a box of b0 x bx x by x 1
static er_status mg_map(CUtensorMap *m, const void *base, int64_t d0, const Lvl &L, int b0, int bx, int by) {
    auto fn = mg_encode();
    if (!fn) return fail(ER_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
    cuuint64_t dims[4] = {(cuuint64_t)d0, (cuuint64_t)L.W, (cuuint64_t)L.H, (cuuint64_t)L.T};
    cuuint64_t strides[3] = {(cuuint64_t)d0 * 4, (cuuint64_t)d0 * 4 * L.W, (cuuint64_t)d0 * 4 * L.W * L.H};
    cuuint32_t box[4] = {(cuuint32_t)b0, (cuuint32_t)bx, (cuuint32_t)by, 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void *>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(ER_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return ER_OK;
}

// ---- hierarchy ---------------------------------------------------------------------------

struct MgHier {
    int k = 0;
    std::vector<er_grid *> grids;  // level l >= 1; grids[0] = nullptr (the fine grid)
    std::vector<Lvl> lv;
    std::vector<float *> r, z;     // per level [n][k]; r[0] is the CG residual (not owned)
    float *ainv = nullptr;         // dense inverse of the coarsest level [n_c][ld_inv], zero padded
    int ld_inv = 0;                // row stride of ainv: n_c rounded up to a multiple of 4
    double *msc = nullptr;         // per column: recursive residual, previous alpha [2][k]
    // tiled kernels, per level l: r_l (finer side), coefficients, z_l (coarser side of l - 1)
    std::vector<CUtensorMap> map_r, map_c, map_z;
    // tiled CG passes on the finest level: direction (z, p[0], p[1], coefficients; east/south
    // halo) and update (p[0], p[1], coefficients; halo on every side)
    CUtensorMap dmap_z, dmap_p[2], dmap_c, umap_p[2], umap_c;
    std::vector<int32_t *> tent_ptr;  // per level: its tile pass's TSV segments grouped by tile
    std::vector<int4 *> tent;
    float2 *part = nullptr;
    int64_t part_chunks = 0;
    int *cnt = nullptr;            // [0] unconverged columns, [1] active columns
    int *h_cnt = nullptr;          // pinned host copy
};

static Lvl level_of(const GridDev &d) {
    Lvl l;
    l.T = d.T; l.W = d.W; l.H = d.H; l.n = d.n;
    l.cb_outer = 0;
    l.coef = reinterpret_cast<const float4 *>(d.coef32);
    l.tsv_ptr = d.tsv_ptr; l.tsv_nbr = d.tsv_nbr; l.tsv_g = d.tsv_g32;
    l.tent_ptr = nullptr;
    l.tent = nullptr;
    return l;
}

// The TSV segments of level f's nodes grouped by the tile (16 x 4 aggregates of the next level,
// numbered as the tile passes number them) that holds the node: per tile, node by node in index
// order, each node's segments in CSR order, as {i, j, aggregate of j, e}.
static er_status build_tsv_tiles(const GridDev &f, int32_t **ptr_out, int4 **ent_out) {
    const int64_t n = f.n;
    const int W = f.W, H = f.H, Wc = (W + 1) / 2, Hc = (H + 1) / 2;
    const int tx = (Wc + TAX - 1) / TAX, ty = (Hc + TAY - 1) / TAY;
    const int64_t ntile = (int64_t)tx * ty * f.T;
    std::vector<int32_t> tp((size_t)n + 1), tn;
    ER_CUDA(cudaMemcpy(tp.data(), f.tsv_ptr, (size_t)(n + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost));
    tn.resize((size_t)tp[(size_t)n]);
    if (!tn.empty())
        ER_CUDA(cudaMemcpy(tn.data(), f.tsv_nbr, tn.size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
    auto tile_of = [&](int64_t i) {
        const int64_t x = i % W, y = (i / W) % H, t = i / ((int64_t)W * H);
        return (t * ty + (y / 2) / TAY) * tx + (x / 2) / TAX;
    };
    auto agg_of = [&](int64_t j) {
        const int64_t x = j % W, y = (j / W) % H, t = j / ((int64_t)W * H);
        return (int32_t)((t * Hc + y / 2) * Wc + x / 2);
    };
    std::vector<int32_t> ptr((size_t)ntile + 1, 0);
    for (int64_t i = 0; i < n; ++i)
        if (tp[(size_t)i + 1] > tp[(size_t)i]) ptr[(size_t)tile_of(i) + 1] += tp[(size_t)i + 1] - tp[(size_t)i];
    for (int64_t q = 0; q < ntile; ++q) ptr[(size_t)q + 1] += ptr[(size_t)q];
    std::vector<int4> ent((size_t)ptr[(size_t)ntile]);
    std::vector<int32_t> fill(ptr.begin(), ptr.end() - 1);
    for (int64_t i = 0; i < n; ++i) {
        if (tp[(size_t)i + 1] == tp[(size_t)i]) continue;
        int32_t &f = fill[(size_t)tile_of(i)];
        for (int32_t e = tp[(size_t)i]; e < tp[(size_t)i + 1]; ++e) {
            const int32_t j = tn[(size_t)e];
            ent[(size_t)f++] = make_int4((int)i, j, agg_of(j), e);
        }
    }
    ER_CUDA(cudaMalloc(ptr_out, ptr.size() * sizeof(int32_t)));
    ER_CUDA(cudaMemcpy(*ptr_out, ptr.data(), ptr.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    ER_CUDA(cudaMalloc(ent_out, std::max<size_t>(1, ent.size()) * sizeof(int4)));
    if (!ent.empty()) ER_CUDA(cudaMemcpy(*ent_out, ent.data(), ent.size() * sizeof(int4), cudaMemcpyHostToDevice));
    return ER_OK;
}

void free_mg(GridDev *g) {
    MgHier *h = g->mg;
    if (!h) return;
    for (size_t i = 1; i < h->grids.size(); ++i) er_grid_destroy(h->grids[i]);
    for (size_t i = 1; i < h->r.size(); ++i) cudaFree(h->r[i]);
    for (size_t i = 0; i < h->z.size(); ++i) cudaFree(h->z[i]);
    if (h->ainv) cudaFree(h->ainv);
    if (h->msc) cudaFree(h->msc);
    if (h->part) cudaFree(h->part);
    if (h->cnt) cudaFree(h->cnt);
    if (h->h_cnt) cudaFreeHost(h->h_cnt);
    for (int32_t *p : h->tent_ptr) cudaFree(p);
    for (int4 *p : h->tent) cudaFree(p);
    delete h;
    g->mg = nullptr;
}

// A level's network, copied back from its device arrays (raw FP64 conductances).
struct HostNet {
    std::vector<double> gxr, gyr, tg, pg;
    std::vector<int32_t> tptr, tnbr, pptr;
    std::vector<uint8_t> fl;
};

static er_status fetch_net(const GridDev &f, HostNet &h) {
    const int64_t n = f.n;
    h.gxr.resize(n);
    h.gyr.resize(n);
    h.tptr.resize(n + 1);
    h.pptr.resize(n + 1);
    h.fl.resize(n);
    ER_CUDA(cudaMemcpy(h.gxr.data(), f.gxr, n * sizeof(double), cudaMemcpyDeviceToHost));
    ER_CUDA(cudaMemcpy(h.gyr.data(), f.gyr, n * sizeof(double), cudaMemcpyDeviceToHost));
    ER_CUDA(cudaMemcpy(h.tptr.data(), f.tsv_ptr, (n + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost));
    ER_CUDA(cudaMemcpy(h.pptr.data(), f.pad_ptr, (n + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost));
    ER_CUDA(cudaMemcpy(h.fl.data(), f.floating, n, cudaMemcpyDeviceToHost));
    h.tnbr.resize(h.tptr[n]);
    h.tg.resize(h.tptr[n]);
    h.pg.resize(h.pptr[n]);
    if (h.tptr[n]) {
        ER_CUDA(cudaMemcpy(h.tnbr.data(), f.tsv_nbr, h.tptr[n] * sizeof(int32_t), cudaMemcpyDeviceToHost));
        ER_CUDA(cudaMemcpy(h.tg.data(), f.tsv_g, h.tptr[n] * sizeof(double), cudaMemcpyDeviceToHost));
    }
    if (h.pptr[n]) ER_CUDA(cudaMemcpy(h.pg.data(), f.pad_g, h.pptr[n] * sizeof(double), cudaMemcpyDeviceToHost));
    return ER_OK;
}

// Dense inverse of a (small) level's G in FP64 by Cholesky, G = L L^T, G^-1 = L^-T L^-1,
// rounded to FP32; rows and columns of floating nodes are zero.
// A barrier for the host threads of spd_inverse (they spin, yielding, on a generation count).
struct SpinBarrier {
    std::atomic<int> count{0}, gen{0};
    int n = 1;
    void wait() {
        const int g = gen.load(std::memory_order_acquire);
        if (count.fetch_add(1, std::memory_order_acq_rel) + 1 == n) {
            count.store(0, std::memory_order_relaxed);
            gen.fetch_add(1, std::memory_order_acq_rel);
        } else {
            while (gen.load(std::memory_order_acquire) == g) std::this_thread::yield();
        }
    }
};

// In-place inverse of the symmetric positive definite n x n matrix A (row-major, FP64):
// blocked right-looking Cholesky A = L L^T (panels of 32 columns: diagonal block, the panel
// below it, then the trailing lower triangle), the columns of M = L^-1 by forward substitution,
// and A^-1 = M^T M.  Every inner loop is a dot product over contiguous rows; the rows (columns of
// M) are shared cyclically among the host threads.  False if A is not positive definite.
static bool spd_inverse(std::vector<double> &A, int n) {
    const int NB = 32;
    int nt = (int)std::min<unsigned>(16u, std::max(1u, std::thread::hardware_concurrency()));
    if (n <= 256) nt = 1;
    std::vector<double> MT((size_t)n * n, 0.0);  // row j: column j of M = L^-1 (entries j .. n-1)
    std::atomic<bool> bad{false};
    SpinBarrier bar;
    bar.n = nt;
    auto dot = [](const double *x, const double *y, int len) {  // 8 independent partial sums
        double v[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        int q = 0;
        for (; q + 8 <= len; q += 8)
            for (int u = 0; u < 8; ++u) v[u] += x[q + u] * y[q + u];
        for (; q < len; ++q) v[q & 7] += x[q] * y[q];
        return ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]));
    };
    auto work = [&](int t) {
        double *L = A.data();
        for (int k0 = 0; k0 < n; k0 += NB) {
            const int k1 = std::min(n, k0 + NB);
            if (t == 0)  // the diagonal block, already updated by the earlier panels
                for (int j = k0; j < k1 && !bad.load(); ++j) {
                    double *lj = L + (size_t)j * n;
                    const double d = lj[j] - dot(lj + k0, lj + k0, j - k0);
                    if (!(d > 0.0)) {
                        bad.store(true);
                        break;
                    }
                    lj[j] = std::sqrt(d);
                    for (int i = j + 1; i < k1; ++i) {
                        double *li = L + (size_t)i * n;
                        li[j] = (li[j] - dot(li + k0, lj + k0, j - k0)) / lj[j];
                    }
                }
            bar.wait();
            if (bad.load()) return;
            for (int i = k1 + t; i < n; i += nt) {  // the panel's rows below the block
                double *li = L + (size_t)i * n;
                for (int j = k0; j < k1; ++j) {
                    const double *lj = L + (size_t)j * n;
                    li[j] = (li[j] - dot(li + k0, lj + k0, j - k0)) / lj[j];
                }
            }
            bar.wait();
            for (int i = k1 + t; i < n; i += nt) {  // trailing lower triangle
                double *li = L + (size_t)i * n;
                for (int j = k1; j <= i; ++j) li[j] -= dot(li + k0, L + (size_t)j * n + k0, k1 - k0);
            }
            bar.wait();
        }
        for (int j = t; j < n; j += nt) {  // L m = e_j, m zero above j
            double *m = MT.data() + (size_t)j * n;
            for (int i = j; i < n; ++i) {
                const double *li = L + (size_t)i * n;
                m[i] = ((i == j ? 1.0 : 0.0) - dot(li + j, m + j, i - j)) / li[i];
            }
        }
        bar.wait();
        for (int a = t; a < n; a += nt)  // (M^T M)_ab = sum over q >= max(a, b) of M_qa M_qb
            for (int b = a; b < n; ++b) {
                const double v = dot(MT.data() + (size_t)a * n + b, MT.data() + (size_t)b * n + b, n - b);
                L[(size_t)a * n + b] = v;
            }
        bar.wait();
        for (int a = t; a < n; a += nt)  // mirror into the lower triangle
            for (int b = 0; b < a; ++b) L[(size_t)a * n + b] = L[(size_t)b * n + a];
    };
    if (nt == 1) {
        work(0);
    } else {
        std::vector<std::thread> th;
        for (int t = 1; t < nt; ++t) th.emplace_back(work, t);
        work(0);
        for (auto &x : th) x.join();
    }
    return !bad.load();
}

static er_status dense_inverse(const GridDev &c, std::vector<float> &out) {
    HostNet h;
    er_status st = fetch_net(c, h);
    if (st != ER_OK) return st;
    const int n = (int)c.n, W = c.W;
    std::vector<double> G((size_t)n * n, 0.0);
    auto add_edge = [&](int a, int b, double g) {
        G[(size_t)a * n + a] += g;
        G[(size_t)b * n + b] += g;
        G[(size_t)a * n + b] -= g;
        G[(size_t)b * n + a] -= g;
    };
    for (int i = 0; i < n; ++i) {
        if (h.fl[i]) {
            G[(size_t)i * n + i] = 1.0;  // decoupled identity row; zeroed in the inverse
            continue;
        }
        if (h.gxr[i] > 0.0) add_edge(i, i + 1, h.gxr[i]);
        if (h.gyr[i] > 0.0) add_edge(i, i + W, h.gyr[i]);
        for (int32_t e = h.tptr[i]; e < h.tptr[i + 1]; ++e)
            if (h.tnbr[e] > i) add_edge(i, h.tnbr[e], h.tg[e]);
        for (int32_t e = h.pptr[i]; e < h.pptr[i + 1]; ++e) G[(size_t)i * n + i] += h.pg[e];
    }
    // G^-1 = L^-T L^-1 from the Cholesky factor G = L L^T, on the host cores
    if (!spd_inverse(G, n)) return fail(ER_ERR_INVALID_ARG, "multigrid: coarsest level is not positive definite");
    out.assign((size_t)n * n, 0.0f);
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b)
            out[(size_t)a * n + b] = (h.fl[a] || h.fl[b]) ? 0.0f : (float)G[(size_t)a * n + b];
    return ER_OK;
}

// The network of level l+1 from the device arrays of level l: aggregate 2 x 2 nodes per tier.
static er_status coarsen(const GridDev &f, cudaStream_t s, er_grid **out) {
    const int T = f.T, W = f.W, H = f.H;
    const int Wc = (W + 1) / 2, Hc = (H + 1) / 2;
    const int64_t n = f.n;
    HostNet hn;
    er_status fst = fetch_net(f, hn);
    if (fst != ER_OK) return fst;
    const std::vector<double> &gxr = hn.gxr, &gyr = hn.gyr, &tg = hn.tg, &pg = hn.pg;
    const std::vector<int32_t> &tptr = hn.tptr, &tnbr = hn.tnbr, &pptr = hn.pptr;
    const std::vector<uint8_t> &fl = hn.fl;
    (void)s;
    auto id = [&](int t, int y, int x) { return ((int64_t)t * H + y) * W + x; };
    std::vector<double> gx((size_t)T * Hc * std::max(Wc - 1, 0), 0.0), gy((size_t)T * std::max(Hc - 1, 0) * Wc, 0.0);
    for (int t = 0; t < T; ++t)
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                const int64_t i = id(t, y, x);
                if (fl[i]) continue;  // segments of floating islands join floating nodes only
                if ((x & 1) && x + 1 < W && gxr[i] > 0.0)  // crosses from aggregate x/2 to x/2 + 1
                    gx[((size_t)t * Hc + y / 2) * (Wc - 1) + x / 2] += gxr[i];
                if ((y & 1) && y + 1 < H && gyr[i] > 0.0)
                    gy[((size_t)t * (Hc - 1) + y / 2) * Wc + x / 2] += gyr[i];
            }
    // TSV segments and pads that land on one aggregate act in parallel: their conductances are
    // summed into one segment (one pad) per aggregate, so a coarse node has at most one TSV
    // segment up and one down however many fine TSVs it gathers
    const int64_t nc = (int64_t)T * Hc * Wc;
    std::vector<double> tsum((size_t)nc, 0.0), psum((size_t)nc, 0.0);
    for (int64_t i = 0; i < n; ++i) {
        if (fl[i]) continue;
        const int x = (int)(i % W), y = (int)((i / W) % H), t = (int)(i / ((int64_t)W * H));
        const int64_t J = ((int64_t)t * Hc + y / 2) * Wc + x / 2;
        for (int32_t e = tptr[i]; e < tptr[i + 1]; ++e)
            if (tnbr[e] > i && tg[e] > 0.0) tsum[J] += tg[e];  // each segment once, from its lower end
        for (int32_t e = pptr[i]; e < pptr[i + 1]; ++e)
            if (pg[e] > 0.0) psum[J] += pg[e];
    }
    std::vector<er_tsv> tsv;
    std::vector<er_pad> pads;
    for (int64_t J = 0; J < nc; ++J) {
        const int X = (int)(J % Wc), Y = (int)((J / Wc) % Hc), t = (int)(J / ((int64_t)Wc * Hc));
        if (tsum[J] > 0.0) tsv.push_back({t, X, Y, tsum[J]});
        if (psum[J] > 0.0) pads.push_back({t, X, Y, psum[J]});
    }
    std::vector<er_tier> tiers(T);
    for (int t = 0; t < T; ++t) {
        tiers[t].W = Wc;
        tiers[t].H = Hc;
        tiers[t].gx = Wc > 1 ? gx.data() + (size_t)t * Hc * (Wc - 1) : nullptr;
        tiers[t].gy = Hc > 1 ? gy.data() + (size_t)t * (Hc - 1) * Wc : nullptr;
    }
    er_options o{};
    o.device = f.device;
    const er_status st = grid_create(tiers.data(), T, tsv.data(), (int64_t)tsv.size(), pads.data(),
                                     (int64_t)pads.size(), &o, nullptr, out);
    return st == ER_WARN_FLOATING ? ER_OK : st;
}

static er_status get_mg(GridDev &g, int k, cudaStream_t s, MgHier **out) {
    MgHier *h = g.mg;
    if (!h) {
        h = new MgHier();
        g.mg = h;
        h->grids.push_back(nullptr);
        h->lv.push_back(level_of(g));
        const GridDev *cur = &g;
        while (cur->n > kCoarseTarget) {
            if (cur->W <= 1 && cur->H <= 1) break;
            er_grid *c = nullptr;
            er_status st = coarsen(*cur, s, &c);
            if (st != ER_OK) {
                free_mg(&g);
                return st;
            }
            h->grids.push_back(c);
            h->lv.push_back(level_of(c->d));
            cur = &c->d;
        }
        if (h->lv.size() < 2 || h->lv.back().n > kCoarseMax) {
            free_mg(&g);
            return fail(ER_ERR_INVALID_ARG, "multigrid: the grid does not coarsen to 2,048 nodes (too many tiers)");
        }
        std::vector<float> inv;
        er_status ist = dense_inverse(*cur, inv);
        if (ist != ER_OK) {
            free_mg(&g);
            return ist;
        }
        const int nc = (int)cur->n;
        h->ld_inv = (nc + 3) & ~3;
        std::vector<float> padded((size_t)nc * h->ld_inv, 0.0f);
        for (int a = 0; a < nc; ++a)
            std::memcpy(&padded[(size_t)a * h->ld_inv], &inv[(size_t)a * nc], (size_t)nc * sizeof(float));
        ER_CUDA(cudaMalloc(&h->ainv, padded.size() * sizeof(float)));
        ER_CUDA(cudaMemcpy(h->ainv, padded.data(), padded.size() * sizeof(float), cudaMemcpyHostToDevice));
        ER_CUDA(cudaMalloc(&h->cnt, 2 * sizeof(int)));
        ER_CUDA(cudaMallocHost(&h->h_cnt, 2 * sizeof(int)));
        // every tile pass's TSV segments by tile, for the staged partner rows
        const size_t L = h->lv.size();
        h->tent_ptr.assign(L - 1, nullptr);
        h->tent.assign(L - 1, nullptr);
        for (size_t l = 0; l + 1 < L; ++l) {
            const GridDev &fl = l == 0 ? g : h->grids[l]->d;
            er_status ts = build_tsv_tiles(fl, &h->tent_ptr[l], &h->tent[l]);
            if (ts != ER_OK) {
                free_mg(&g);
                return ts;
            }
            h->lv[l].tent_ptr = h->tent_ptr[l];
            h->lv[l].tent = h->tent[l];
        }
    }
    if (h->k != k) {
        for (size_t i = 1; i < h->r.size(); ++i) cudaFree(h->r[i]);
        for (size_t i = 0; i < h->z.size(); ++i) cudaFree(h->z[i]);
        if (h->part) cudaFree(h->part);
        h->r.assign(h->lv.size(), nullptr);
        h->z.assign(h->lv.size(), nullptr);
        h->part = nullptr;
        h->k = 0;
        for (size_t l = 0; l < h->lv.size(); ++l) {
            // the coarsest level's r has ld_inv rows; rows n_c .. ld_inv - 1 stay zero
            const int64_t rows = l + 1 == h->lv.size() ? h->ld_inv : h->lv[l].n;
            const size_t bytes = (size_t)h->lv[l].n * k * sizeof(float);
            if (l > 0) {
                ER_CUDA(cudaMalloc(&h->r[l], (size_t)rows * k * sizeof(float)));
                ER_CUDA(cudaMemset(h->r[l], 0, (size_t)rows * k * sizeof(float)));
            }
            ER_CUDA(cudaMalloc(&h->z[l], bytes));
        }
        h->part_chunks = std::max(std::max(make_lay(g.n, k).chunks, n_tiles(h->lv[1])), n_ctiles(h->lv[0]));
        if (h->msc) cudaFree(h->msc);
        ER_CUDA(cudaMalloc(&h->msc, (size_t)2 * k * sizeof(double)));
        ER_CUDA(cudaMalloc(&h->part, (size_t)h->part_chunks * k * sizeof(float2)));
        h->k = k;
    }
    *out = h;
    return ER_OK;
}

// ---- the solve ---------------------------------------------------------------------------

namespace {

struct MgRun {
    const GridDev *g;
    Workspace *w;
    MgHier *h;
    int k;
    double tol;
    void *Z;
    int *err;      // the solve's error word (a bounded wait expired)
    int cb_outer;  // launch order of the tiled kernels (Lvl::cb_outer)
};


template <class K, class... A>
void mg_launch(Workspace &w, Prof *pf, int kind, K kern, dim3 grid, int smem, A... args) {
    prof_begin(w, pf, kind);
    kern<<<grid, 256, smem, w.s>>>(args...);
    prof_end(w, pf, kind);
}

FoldArgs fold_args(const MgRun &m, int64_t chunks) {
    FoldArgs f;
    f.part = m.h->part;
    f.chunks = chunks;
    f.k = m.k;
    f.alpha = m.w->scal;
    f.beta = m.w->scal + m.k;
    f.rho = m.w->scal + 2 * m.k;
    f.rho0 = m.w->scal + 3 * m.k;
    f.relrec = m.h->msc;
    f.alpha_prev = m.h->msc + m.k;
    f.active = m.w->ints;
    f.nunc = m.h->cnt;
    f.tol = m.tol;
    return f;
}

// level l of the hierarchy with this solve's launch order
Lvl run_lv(const MgRun &m, int l) {
    Lvl x = m.h->lv[l];
    x.cb_outer = m.cb_outer;
    return x;
}

// z[0] = V-cycle(r0) with the partials of r.z, then the beta fold
void vcycle(const MgRun &m, const float *r0, Prof *pf) {
    MgHier &h = *m.h;
    const int L = (int)h.lv.size(), k = m.k;
    auto lv = [&](int l) { return run_lv(m, l); };
    for (int l = 0; l + 1 < L; ++l) {
        const float *rl = l == 0 ? r0 : h.r[l];
        // the finest level stages its tiles' TSV partners; on the coarse levels, whose launches
        // are short, the staging's start-up cost outweighed it
        if (l == 0)
            mg_launch(*m.w, pf, ER_PASS_MG_DOWN, k_mg_tile<false, false, true>, tile_grid(h.lv[l + 1], k),
                      T_SMEM_DOWN_TS, h.map_r[l], h.map_c[l], h.map_r[l], lv(l), lv(l + 1), k, rl,
                      (const float *)nullptr, h.r[l + 1], (float2 *)nullptr, m.err);
        else
            mg_launch(*m.w, pf, ER_PASS_MG, k_mg_tile<false, false, false>, tile_grid(h.lv[l + 1], k), T_SMEM_DOWN,
                      h.map_r[l], h.map_c[l], h.map_r[l], lv(l), lv(l + 1), k, rl, (const float *)nullptr,
                      h.r[l + 1], (float2 *)nullptr, m.err);
    }
    const Lvl &C = h.lv[L - 1];
    mg_launch(*m.w, pf, ER_PASS_MG, k_mg_cinv, cinv_grid(C.n, k), 0, (int)C.n, h.ld_inv, k, (const float *)h.ainv,
              (const float *)h.r[L - 1], h.z[L - 1]);
    for (int l = L - 2; l >= 0; --l) {
        const float *rl = l == 0 ? r0 : h.r[l];
        if (l == 0)
            mg_launch(*m.w, pf, ER_PASS_MG_UP, k_mg_tile<true, true, true>, tile_grid(h.lv[1], k), T_SMEM_TS, h.map_r[0],
                      h.map_c[0], h.map_z[1], lv(0), lv(1), k, rl, (const float *)h.z[1], h.z[0], h.part, m.err);
        else
            mg_launch(*m.w, pf, ER_PASS_MG, k_mg_tile<true, false, false>, tile_grid(h.lv[l + 1], k), T_SMEM, h.map_r[l],
                      h.map_c[l], h.map_z[l + 1], lv(l), lv(l + 1), k, rl, (const float *)h.z[l + 1], h.z[l],
                      (float2 *)nullptr, m.err);
    }
    mg_launch(*m.w, pf, ER_PASS_OTHER, k_mg_fold<FOLD_BETA>, dim3((unsigned)k), 0, fold_args(m, n_tiles(h.lv[1])));
}

// one PCG iteration from the current residual w.r[0]: z = M r, beta, p' = z + beta p and
// p'.G p', alpha, r -= alpha G p' with the recursive residual norms, and every second
// iteration x += alpha_prev p'_prev + alpha p'
int mg_iterate(const MgRun &m, int cur, Prof *pf) {
    MgHier &h = *m.h;
    Workspace &w = *m.w;
    const int k = m.k;
    float *r = (float *)w.r[0];
    vcycle(m, r, pf);
    Lvl L0 = h.lv[0];
    L0.cb_outer = m.cb_outer;
    const dim3 grid = ctile_grid(L0, k);
    const int64_t nct = n_ctiles(L0);
    mg_launch(w, pf, ER_PASS_A, k_mg_dir_tile, grid, S_SMEM, h.dmap_z, h.dmap_p[cur], h.dmap_c, L0, k,
              (const float *)h.z[0], (const float *)w.p[cur], (const double *)(w.scal + k), (float *)w.p[1 - cur],
              h.part, m.err);
    mg_launch(w, pf, ER_PASS_OTHER, k_mg_fold<FOLD_ALPHA>, dim3((unsigned)k), 0, fold_args(m, nct));
    if (cur == 1)  // second iteration of a pair: x += alpha_prev p'_prev + alpha p'
        mg_launch(w, pf, ER_PASS_B, k_mg_upd_tile<true>, grid, U_SMEM, h.umap_p[1 - cur], h.umap_c, L0, k,
                  (const double *)w.scal, (const double *)(h.msc + k), (const float *)w.p[1 - cur],
                  (const float *)w.p[cur], (float *)m.Z, r, h.part, m.err);
    else
        mg_launch(w, pf, ER_PASS_B0, k_mg_upd_tile<false>, grid, U_SMEM, h.umap_p[1 - cur], h.umap_c, L0, k,
                  (const double *)w.scal, (const double *)(h.msc + k), (const float *)w.p[1 - cur],
                  (const float *)w.p[cur], (float *)m.Z, r, h.part, m.err);
    mg_launch(w, pf, ER_PASS_OTHER, k_mg_fold<FOLD_RR>, dim3((unsigned)k), 0, fold_args(m, nct));
    return 1 - cur;
}

}  // namespace

// The grid's multigrid hierarchy for k columns (built and cached on the first call) and the
// tensor maps of the V-cycle and CG kernels over the workspace's vectors.
static er_status mg_prepare(GridDev &g, Workspace &w, MgHier **out) {
    const int k = w.k;
    MgHier *h = nullptr;
    er_status st = get_mg(g, k, w.s, &h);
    if (st != ER_OK) return st;
    {
        const int L = (int)h->lv.size();
        h->map_r.resize(L);
        h->map_c.resize(L);
        h->map_z.resize(L);
        for (int l = 0; l < L; ++l) {
            const void *rl = l == 0 ? w.r[0] : (const void *)h->r[l];
            er_status ms = mg_map(&h->map_r[l], rl, k, h->lv[l], TCB, TFX, TFY);
            if (ms == ER_OK) ms = mg_map(&h->map_c[l], h->lv[l].coef, 4, h->lv[l], 4, TFX, TFY);
            if (ms == ER_OK) ms = mg_map(&h->map_z[l], h->z[l], k, h->lv[l], TCB, TZX, TZY);
            if (ms != ER_OK) return ms;
        }
        const Lvl &L0 = h->lv[0];
        er_status ms = mg_map(&h->dmap_z, h->z[0], k, L0, TCB, SPX, SPY);
        for (int b = 0; b < 2 && ms == ER_OK; ++b) {
            ms = mg_map(&h->dmap_p[b], w.p[b], k, L0, TCB, SPX, SPY);
            if (ms == ER_OK) ms = mg_map(&h->umap_p[b], w.p[b], k, L0, TCB, UPX, UPY);
        }
        if (ms == ER_OK) ms = mg_map(&h->dmap_c, L0.coef, 4, L0, 4, SPX, SPY);
        if (ms == ER_OK) ms = mg_map(&h->umap_c, L0.coef, 4, L0, 4, UPX, UPY);
        if (ms != ER_OK) return ms;
        static std::atomic<bool> attr{false};  // solves of different grids may run on several threads
        if (!attr.load()) {
            ER_CUDA(cudaFuncSetAttribute(k_mg_tile<false, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         T_SMEM_DOWN_TS));
            ER_CUDA(cudaFuncSetAttribute(k_mg_tile<false, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         T_SMEM_DOWN));
            ER_CUDA(cudaFuncSetAttribute(k_mg_tile<true, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         T_SMEM));
            ER_CUDA(cudaFuncSetAttribute(k_mg_tile<true, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         T_SMEM_TS));
            ER_CUDA(cudaFuncSetAttribute(k_mg_dir_tile, cudaFuncAttributeMaxDynamicSharedMemorySize, S_SMEM));
            ER_CUDA(cudaFuncSetAttribute(k_mg_upd_tile<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, U_SMEM));
            ER_CUDA(cudaFuncSetAttribute(k_mg_upd_tile<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, U_SMEM));
            attr.store(true);
        }
    }
    *out = h;
    return ER_OK;
}

er_status mg_solve_core(GridDev &g, Workspace &w, const void *Yt, void *Z, const er_solve_opts &opt,
                        er_solve_stats *stats, std::chrono::steady_clock::time_point t0) {
    const int k = w.k;
    const double tol = opt.tol;
    MgHier *h = nullptr;
    er_status st = mg_prepare(g, w, &h);
    if (st != ER_OK) return st;
    MgRun m{&g, &w, h, k, tol, Z, w.ints + w.k + w.til.n_colblk, opt.block_order == 2 ? 1 : 0};
    Prof pf;
    pf.on = opt.profile != 0;
    pf.chained = true;  // one event per timed launch (the stream operations below break the chain)
    const bool use_graph = opt.use_graph && !pf.on;
    ER_CUDA(cudaMemsetAsync(w.ints + w.k + w.til.n_colblk, 0, sizeof(int), w.s));  // error word
    fp32_init(g, w, Yt, Z, tol, &pf);  // r = b, x = 0, p = 0, xhl = 0; rho0 = rho = b.D^-1 b; active
    ER_CUDA(cudaGetLastError());

    auto poll = [&](int *vals) -> er_status {
        ER_CUDA(cudaMemcpyAsync(h->h_cnt, h->cnt, 2 * sizeof(int), cudaMemcpyDeviceToHost, w.s));
        ER_CUDA(cudaMemcpyAsync(w.h_poll, w.ints + w.k + w.til.n_colblk, sizeof(int), cudaMemcpyDeviceToHost, w.s));
        ER_CUDA(cudaStreamSynchronize(w.s));
        flush_prof(w, pf);
        vals[0] = h->h_cnt[0];
        vals[1] = h->h_cnt[1];
        vals[2] = w.h_poll[0];
        return ER_OK;
    };
    // accurate residual replacement: xhl += x, x = 0, r = b - G xhl (double-float); freeze columns at tol
    auto replace = [&](int *n_active) -> er_status {
        fp32_accum(g, w, Z, &pf);
        fp32_residual(g, w, Yt, tol, 0, 0, &pf);
        ER_CUDA(cudaMemsetAsync(h->cnt + 1, 0, sizeof(int), w.s));
        pf.chain = -1;
        prof_begin(w, &pf, ER_PASS_OTHER);
        k_mg_freeze<<<ublocks(k, 128), 128, 0, w.s>>>(k, w.scal + 4 * k, h->msc, tol, w.ints,
                                                       w.scal + 2 * k, h->cnt + 1);
        prof_end(w, &pf, ER_PASS_OTHER);
        ER_CUDA(cudaGetLastError());
        int v[3];
        st = poll(v);
        if (st != ER_OK) return st;
        *n_active = v[1];
        return v[2] ? fail(ER_ERR_TIMEOUT, "a bounded wait on a bulk copy expired inside a solver kernel") : ER_OK;
    };

    int cur = 0, it = 0, replacements = 0, last_replace = 0, n_active = 1;
    const int block = std::max(2, opt.check_every + (opt.check_every & 1));
    bool done = false;
    cudaGraphExec_t gexec = nullptr;
    int g_parity = -1;
    while (!done && it < opt.maxit) {
        int todo = std::min(block, opt.maxit - it);
        if (todo & 1) ++todo;  // x is updated in iteration pairs
        if (use_graph && todo == block) {
            if (!gexec || g_parity != cur) {
                if (gexec) cudaGraphExecDestroy(gexec);
                gexec = nullptr;
                cudaGraph_t graph;
                ER_CUDA(cudaStreamBeginCapture(w.s, cudaStreamCaptureModeThreadLocal));
                int c = cur;
                for (int i = 0; i < block; ++i) c = mg_iterate(m, c, nullptr);
                ER_CUDA(cudaStreamEndCapture(w.s, &graph));
                const cudaError_t e = cudaGraphInstantiate(&gexec, graph, 0);
                cudaGraphDestroy(graph);
                if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
                g_parity = cur;
            }
            ER_CUDA(cudaGraphLaunch(gexec, w.s));
            const int L = (int)h->lv.size();
            pf.launches[ER_PASS_A] += block;
            pf.launches[ER_PASS_B] += block / 2;
            pf.launches[ER_PASS_B0] += block / 2;
            pf.launches[ER_PASS_MG] += block * (2 * L - 3);
            pf.launches[ER_PASS_MG_DOWN] += block;
            pf.launches[ER_PASS_MG_UP] += block;
            pf.launches[ER_PASS_OTHER] += block * 3;
            if (block & 1) cur = 1 - cur;
        } else {
            for (int i = 0; i < todo; ++i) cur = mg_iterate(m, cur, &pf);
        }
        it += todo;
        ER_CUDA(cudaGetLastError());
        int v[3];
        st = poll(v);
        if (st != ER_OK) break;
        if (v[2]) {
            st = fail(ER_ERR_TIMEOUT, "a bounded wait on a bulk copy expired inside a solver kernel");
            break;
        }
        if (v[0] == 0 || it - last_replace >= opt.replace_every) {
            st = replace(&n_active);
            ++replacements;
            last_replace = it;
            if (st != ER_OK) break;
            done = n_active == 0;
        }
    }
    if (gexec) cudaGraphExecDestroy(gexec);
    if (st != ER_OK) return st;
    if (last_replace != it) {
        st = replace(&n_active);
        ++replacements;
        if (st != ER_OK) return st;
        done = n_active == 0;
    }
    fp32_final(g, w, Z, &pf);
    ER_CUDA(cudaGetLastError());
    std::vector<double> resid((size_t)k);
    ER_CUDA(cudaMemcpyAsync(resid.data(), w.scal + 4 * k, (size_t)k * sizeof(double), cudaMemcpyDeviceToHost, w.s));
    ER_CUDA(cudaStreamSynchronize(w.s));
    flush_prof(w, pf);
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
    if (!done)
        return fail(ER_ERR_NOT_CONVERGED,
                    std::to_string(n_active) + " columns above tol after " + std::to_string(it) + " iterations");
    return ER_OK;
}

// ---- batching form: level-synchronous launches over all networks ---------------------------
//
// Hundreds of uneven networks, each with its own hierarchy, vectors and per-column scalars,
// advance through er_solve's multigrid iteration together: every pass of the iteration (each
// level's restriction and prolongation, the coarsest solves, the direction and update passes,
// the folds) is ONE launch over the blocks of all networks still running.  These launches are
// persistent: a grid of a few CTAs per SM walks a device-side work list, the prefix sums of
// the running networks' blocks per pass, so a launch costs the same whether 500 networks or
// one are left.  A CTA maps its item to (network, block) by a binary search of the prefix sums
// (staged in shared memory) and runs exactly the single-network kernel's body on it: the same
// tiles, the same arithmetic, the same partial sums, so every network's map is bitwise what
// er_solve gives it alone.
//
// One poll period (er_solve's check_every iterations) is the body of a device-side WHILE node
// of a CUDA graph.  After the iterations, a control kernel takes each running network's
// decision exactly where er_solve's host loop would (run the accurate residual replacement,
// stop on an error or maxit); the replacement passes run over the networks that chose it;
// then one CTA updates the states, rebuilds the work list of the networks still running
// (prefix sums per pass) and ends the loop when none is left.  No host thread polls: the host
// launches the graph once per group of up to kBmgMaxNets networks.

namespace {

constexpr int kBmgLv = 12;          // levels per network (2 x 2 aggregation: 4^11 x 1,024 nodes)
constexpr int kBmgMaxNets = 1024;   // networks per group: one thread each in the control kernels
// pass kinds of the work list: 0 .. kBmgLv - 2 the tile pass between levels l and l + 1
enum { BP_CT = kBmgLv - 1, BP_CINV, BP_N };

struct BmgNet {  // one network of a batch, device resident (the TMA reads the maps from here)
    CUtensorMap map_r[kBmgLv], map_c[kBmgLv], map_z[kBmgLv];
    CUtensorMap dmap_z, dmap_p[2], dmap_c, umap_p[2], umap_c;
    Lvl lv[kBmgLv];          // with the network's launch order in cb_outer
    float *r[kBmgLv];        // r[0]: the CG residual (the workspace's)
    float *z[kBmgLv];
    const float *ainv;       // coarsest level's dense inverse
    float *p[2], *x;         // search directions, iterate (the caller's Z)
    float2 *part;
    double *scal, *msc;
    int *cnt, *err;
    FoldArgs fold_beta, fold_ct;
    int L, ld_inv, nc, cinv_gx;
    int items[BP_N];         // blocks per pass kind (0: the pass does not reach this network)
};

struct BmgState {  // one network's loop state (device memory)
    int it, last_replace, replacements, leave, err, converged;
    double max_resid;
};

// list layout (ints): [0] running networks na, [1 .. cap] their indices, then per pass kind
// the exclusive prefix sums of their blocks, cap + 1 entries each
__device__ __forceinline__ const int *bmg_pre(const int *list, int cap, int pass) {
    return list + 1 + cap + pass * (cap + 1);
}

// stage a pass's prefix sums in shared memory; returns the number of running networks
__device__ __forceinline__ int bmg_stage(const int *list, int cap, int pass, int *spre) {
    const int na = list[0];
    const int *pre = bmg_pre(list, cap, pass);
    for (int i = threadIdx.x; i <= na; i += blockDim.x) spre[i] = pre[i];
    __syncthreads();
    return na;
}

// the running network whose blocks hold item i: the largest s with spre[s] <= i
__device__ __forceinline__ int bmg_slot(const int *spre, int na, int i) {
    int lo = 0, hi = na - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (spre[mid] <= i) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ void bmg_bar_init(uint64_t *bar) {
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mg_saddr(bar)), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
}

// The persistent pass kernels overlap each item's bookkeeping with the previous item's copies:
// right after issuing item i's bulk copies, the issuing thread finds item i + gridDim.x
// (network, block, arguments, tensor maps) and writes it to the other of two shared slots, so
// the next item's copies can start as soon as the CTA's threads are done with the tile.

__device__ __forceinline__ void bmg_prefetch_map(const CUtensorMap *m) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(m)) : "memory");
}

struct BmgTileSlot {
    TileArgs a;
    const CUtensorMap *mr, *mc, *mz;
    int blk;
};

template <bool UP, bool DOT>
__device__ __forceinline__ void bmg_tile_decode(const BmgNet *__restrict__ nets, const int *__restrict__ list,
                                                const int *spre, int na, int l, int i, BmgTileSlot &s) {
    const int q = bmg_slot(spre, na, i);
    const BmgNet &N = nets[list[1 + q]];
    s.blk = i - spre[q];
    s.a.F = N.lv[l];
    s.a.C = N.lv[l + 1];
    s.a.r = N.r[l];
    s.a.zc = UP ? N.z[l + 1] : nullptr;
    s.a.out = UP ? N.z[l] : N.r[l + 1];
    s.a.part = DOT ? N.part : nullptr;
    s.a.err = N.err;
    s.mr = &N.map_r[l];
    s.mc = &N.map_c[l];
    s.mz = UP ? &N.map_z[l + 1] : nullptr;
    bmg_prefetch_map(s.mr);
    bmg_prefetch_map(s.mc);
    if (UP) bmg_prefetch_map(s.mz);
}

// the tile pass between levels l and l + 1 of every running network (k_mg_tile's body)
template <bool UP, bool DOT>
__global__ void __launch_bounds__(256, 3) k_bmg_tile(const BmgNet *__restrict__ nets, const int *__restrict__ list,
                                                  int cap, int l, int k) {
    extern __shared__ unsigned char bmg_tile_raw[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ BmgTileSlot slot[2];
    unsigned char *sm = bmg_tile_raw + ((128u - (mg_saddr(bmg_tile_raw) & 127u)) & 127u);
    int *spre = reinterpret_cast<int *>(sm + T_R + T_C + T_Z);
    bmg_bar_init(&bar);
    const int na = bmg_stage(list, cap, l, spre);  // (its __syncthreads also publishes the barrier)
    const int total = na > 0 ? spre[na] : 0;
    if (threadIdx.x == 0 && (int)blockIdx.x < total)
        bmg_tile_decode<UP, DOT>(nets, list, spre, na, l, (int)blockIdx.x, slot[0]);
    __syncthreads();
    uint32_t parity = 0;
    int q = 0;
    for (int i = blockIdx.x; i < total; i += gridDim.x) {
        const BmgTileSlot &S = slot[q];
        const int nx = i + (int)gridDim.x;
        const auto next = [&]() {
            if (nx < total) bmg_tile_decode<UP, DOT>(nets, list, spre, na, l, nx, slot[q ^ 1]);
        };
        if (!mg_tile_body<UP, DOT>(sm, &bar, parity, false, S.blk, S.mr, S.mc, S.mz, S.a, k, next))
            return;  // error word raised, this CTA's copies drained
        parity ^= 1u;
        q ^= 1;
        __syncthreads();  // the tile buffers and this item's slot are free
    }
}

struct BmgDirSlot {
    Lvl F;
    const float *z, *p;
    const double *beta;
    float *p_out;
    float2 *part;
    int *err;
    const CUtensorMap *mz, *mp, *mc;
    int blk;
};

__device__ __forceinline__ void bmg_dir_decode(const BmgNet *__restrict__ nets, const int *__restrict__ list,
                                               const int *spre, int na, int cur, int k, int i, BmgDirSlot &s) {
    const int q = bmg_slot(spre, na, i);
    const BmgNet &N = nets[list[1 + q]];
    s.blk = i - spre[q];
    s.F = N.lv[0];
    s.z = N.z[0];
    s.p = N.p[cur];
    s.beta = N.scal + k;
    s.p_out = N.p[1 - cur];
    s.part = N.part;
    s.err = N.err;
    s.mz = &N.dmap_z;
    s.mp = &N.dmap_p[cur];
    s.mc = &N.dmap_c;
    bmg_prefetch_map(s.mz);
    bmg_prefetch_map(s.mp);
    bmg_prefetch_map(s.mc);
}

// p' = z + beta p on the finest level of every running network (k_mg_dir_tile's body)
__global__ void __launch_bounds__(256, 4) k_bmg_dir(const BmgNet *__restrict__ nets, const int *__restrict__ list,
                                                 int cap, int k, int cur) {
    extern __shared__ unsigned char bmg_dir_raw[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ BmgDirSlot slot[2];
    unsigned char *sm = bmg_dir_raw + ((128u - (mg_saddr(bmg_dir_raw) & 127u)) & 127u);
    int *spre = reinterpret_cast<int *>(sm + 2 * S_V + S_C);
    bmg_bar_init(&bar);
    const int na = bmg_stage(list, cap, BP_CT, spre);
    const int total = na > 0 ? spre[na] : 0;
    if (threadIdx.x == 0 && (int)blockIdx.x < total) bmg_dir_decode(nets, list, spre, na, cur, k, (int)blockIdx.x, slot[0]);
    __syncthreads();
    uint32_t parity = 0;
    int q = 0;
    for (int i = blockIdx.x; i < total; i += gridDim.x) {
        const BmgDirSlot &S = slot[q];
        const int nx = i + (int)gridDim.x;
        const auto next = [&]() {
            if (nx < total) bmg_dir_decode(nets, list, spre, na, cur, k, nx, slot[q ^ 1]);
        };
        if (!mg_dir_body(sm, &bar, parity, false, S.blk, S.mz, S.mp, S.mc, S.F, k, S.z, S.p, S.beta, S.p_out, S.part,
                         S.err, next))
            return;
        parity ^= 1u;
        q ^= 1;
        __syncthreads();
    }
}

struct BmgUpdSlot {
    Lvl F;
    const double *alpha, *alpha_prev;
    const float *p, *p_prev;
    float *x, *r;
    float2 *part;
    int *err;
    const CUtensorMap *mp, *mc;
    int blk;
};

__device__ __forceinline__ void bmg_upd_decode(const BmgNet *__restrict__ nets, const int *__restrict__ list,
                                               const int *spre, int na, int cur, int k, int i, BmgUpdSlot &s) {
    const int q = bmg_slot(spre, na, i);
    const BmgNet &N = nets[list[1 + q]];
    s.blk = i - spre[q];
    s.F = N.lv[0];
    s.alpha = N.scal;
    s.alpha_prev = N.msc + k;
    s.p = N.p[1 - cur];
    s.p_prev = N.p[cur];
    s.x = N.x;
    s.r = N.r[0];
    s.part = N.part;
    s.err = N.err;
    s.mp = &N.umap_p[1 - cur];
    s.mc = &N.umap_c;
    bmg_prefetch_map(s.mp);
    bmg_prefetch_map(s.mc);
}

// r -= alpha G p' (and with XPAIR the paired x update) of every running network (k_mg_upd_tile's body)
template <bool XPAIR>
__global__ void __launch_bounds__(256, 4) k_bmg_upd(const BmgNet *__restrict__ nets, const int *__restrict__ list,
                                              int cap, int k, int cur) {
    extern __shared__ unsigned char bmg_upd_raw[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ BmgUpdSlot slot[2];
    unsigned char *sm = bmg_upd_raw + ((128u - (mg_saddr(bmg_upd_raw) & 127u)) & 127u);
    int *spre = reinterpret_cast<int *>(sm + U_V + U_C);
    bmg_bar_init(&bar);
    const int na = bmg_stage(list, cap, BP_CT, spre);
    const int total = na > 0 ? spre[na] : 0;
    if (threadIdx.x == 0 && (int)blockIdx.x < total) bmg_upd_decode(nets, list, spre, na, cur, k, (int)blockIdx.x, slot[0]);
    __syncthreads();
    uint32_t parity = 0;
    int q = 0;
    for (int i = blockIdx.x; i < total; i += gridDim.x) {
        const BmgUpdSlot &S = slot[q];
        const int nx = i + (int)gridDim.x;
        const auto next = [&]() {
            if (nx < total) bmg_upd_decode(nets, list, spre, na, cur, k, nx, slot[q ^ 1]);
        };
        if (!mg_upd_body<XPAIR>(sm, &bar, parity, false, S.blk, S.mp, S.mc, S.F, k, S.alpha, S.alpha_prev, S.p,
                                S.p_prev, S.x, S.r, S.part, S.err, next))
            return;
        parity ^= 1u;
        q ^= 1;
        __syncthreads();
    }
}

// the coarsest level's exact solve of every running network (k_mg_cinv's body)
__global__ void __launch_bounds__(256) k_bmg_cinv(const BmgNet *__restrict__ nets, const int *__restrict__ list,
                                               int cap, int k) {
    extern __shared__ int bmg_cinv_pre[];
    const int na = bmg_stage(list, cap, BP_CINV, bmg_cinv_pre);
    const int total = na > 0 ? bmg_cinv_pre[na] : 0;
    for (int i = blockIdx.x; i < total; i += gridDim.x) {
        const int s = bmg_slot(bmg_cinv_pre, na, i);
        const BmgNet &N = nets[list[1 + s]];
        const int b = i - bmg_cinv_pre[s];
        mg_cinv_body(b % N.cinv_gx, b / N.cinv_gx, N.nc, N.ld_inv, k, N.ainv, N.r[N.L - 1], N.z[N.L - 1]);
        __syncthreads();
    }
}

// one per-column fold of every running network: item = (network, column)
template <int KIND>
__global__ void __launch_bounds__(256) k_bmg_fold(const BmgNet *__restrict__ nets, const int *__restrict__ list,
                                               int k) {
    const int na = list[0];
    for (int i = blockIdx.x; i < na * k; i += gridDim.x) {
        const BmgNet &N = nets[list[1 + i / k]];
        mg_fold_body<KIND>(KIND == FOLD_BETA ? N.fold_beta : N.fold_ct, i % k);
        __syncthreads();
    }
}

// after a poll period's iterations, per running network: count them and decide, as er_solve's
// host loop would, whether the accurate residual replacement runs (need[c]) or, if not,
// whether the network stops (an error or maxit)
__global__ void k_bmg_control(const BmgNet *__restrict__ nets, BmgState *st, int *need, int n, int block,
                              int replace_every, int maxit) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        BmgState &s = st[c];
        need[c] = 0;
        if (s.leave) continue;
        const BmgNet &N = nets[c];
        s.it += block;
        const int e = *N.err;
        if (e) s.err = 1;
        if (!e && (N.cnt[0] == 0 || s.it - s.last_replace >= replace_every)) {
            need[c] = 1;
            N.cnt[1] = 0;  // k_mg_freeze counts the columns still above tol here
        } else if (e || s.it >= maxit) {
            s.leave = 1;
        }
    }
}

// the replacement's freeze for every network with need[c] (all networks if need is null)
__global__ void k_bmg_freeze(const BmgNet *__restrict__ nets, const int *need, int n, int k, double tol) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)n * k) return;
    const int c = (int)(t / k), j = (int)(t % k);
    if (need && !need[c]) return;
    const BmgNet &N = nets[c];
    mg_freeze_col(j, N.scal + 4 * k, N.msc, tol, N.fold_ct.active, N.scal + 2 * k, N.cnt + 1);
}

// exclusive prefix sum over the CTA's threads (blockDim.x a multiple of 32, at most 1024)
__device__ __forceinline__ int bmg_scan(int v, int *total) {
    __shared__ int wsum[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
        int t = lane < nw ? wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) wsum[lane] = t;  // inclusive sums of the warps
    }
    __syncthreads();
    const int base = w > 0 ? wsum[w - 1] : 0;
    *total = wsum[nw - 1];
    __syncthreads();  // wsum is reused by the next scan
    return base + x - v;
}

// after the replacement passes: the states of the networks that ran one (as er_solve after its
// replacement: stop when no column is above tol, on an error or at maxit), then the work list
// of the networks still running, and the WHILE node's condition.  One CTA of kBmgMaxNets threads.
__global__ void __launch_bounds__(kBmgMaxNets) k_bmg_compact(const BmgNet *__restrict__ nets, BmgState *st,
                                                           const int *need, int *list, int n, int cap, int maxit,
                                                           cudaGraphConditionalHandle h_loop, int set_loop) {
    const int c = threadIdx.x;
    int run = 0;
    if (c < n) {
        BmgState &s = st[c];
        const BmgNet &N = nets[c];
        if (need && need[c]) {
            s.last_replace = s.it;
            s.replacements += 1;
            if (*N.err) s.err = 1;
            if (N.cnt[1] == 0 || s.err || s.it >= maxit) s.leave = 1;
        }
        run = !s.leave;
    }
    int na;
    const int pos = bmg_scan(run, &na);
    if (run) list[1 + pos] = c;
    if (c == 0) list[0] = na;
    for (int p = 0; p < BP_N; ++p) {
        int tot;
        const int e = bmg_scan(run ? nets[c].items[p] : 0, &tot);
        int *pre = list + 1 + cap + p * (cap + 1);
        if (run) pre[pos] = e;
        if (c == 0) pre[na] = tot;
    }
    if (set_loop && c == 0) cudaGraphSetConditional(h_loop, na > 0 ? 1u : 0u);
}

// before the loop: error words, states and replacement flags cleared
__global__ void k_bmg_reset(const BmgNet *__restrict__ nets, BmgState *st, int *need, int n) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    *nets[c].err = 0;
    st[c] = BmgState{};
    need[c] = 0;
}

// the final replacement: its freeze counts from zero
__global__ void k_bmg_zero_active_count(const BmgNet *__restrict__ nets, int n) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n) nets[c].cnt[1] = 0;
}

// after the final replacement: its bookkeeping, the largest accurate residual of the network's
// columns and whether all of them meet tol
__global__ void k_bmg_summary(const BmgNet *__restrict__ nets, BmgState *st, int n, int k, double tol) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const BmgNet &N = nets[c];
    BmgState &s = st[c];
    s.replacements += 1;
    if (*N.err) s.err = 1;
    double mx = 0.0;
    int ok = 1;
    for (int j = 0; j < k; ++j) {
        const double r = N.scal[4 * k + j];
        mx = fmax(mx, r);
        ok &= r <= tol;
    }
    s.max_resid = mx;
    s.converged = ok;
}

}  // namespace

namespace {

struct BmgBuf {  // a device buffer released on every return path
    void *p = nullptr;
    ~BmgBuf() {
        if (p) cudaFree(p);
    }
};

template <class K>
int bmg_grid(K kern, size_t smem, int nsm) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 256, smem) != cudaSuccess || occ < 1) occ = 1;
    return occ * nsm;
}

size_t bmg_tile_smem(int cap) { return (size_t)T_SMEM + 4 * (size_t)(cap + 1); }
size_t bmg_dir_smem(int cap) { return (size_t)S_SMEM + 4 * (size_t)(cap + 1); }
size_t bmg_upd_smem(int cap) { return (size_t)U_SMEM + 4 * (size_t)(cap + 1); }

er_status bmg_attributes() {
    static std::atomic<bool> done{false};
    if (done.load()) return ER_OK;
    const int t = (int)bmg_tile_smem(kBmgMaxNets), d = (int)bmg_dir_smem(kBmgMaxNets),
              u = (int)bmg_upd_smem(kBmgMaxNets);
    ER_CUDA(cudaFuncSetAttribute(k_bmg_tile<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, t));
    ER_CUDA(cudaFuncSetAttribute(k_bmg_tile<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, t));
    ER_CUDA(cudaFuncSetAttribute(k_bmg_tile<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, t));
    ER_CUDA(cudaFuncSetAttribute(k_bmg_dir, cudaFuncAttributeMaxDynamicSharedMemorySize, d));
    ER_CUDA(cudaFuncSetAttribute(k_bmg_upd<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, u));
    ER_CUDA(cudaFuncSetAttribute(k_bmg_upd<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, u));
    done.store(true);
    return ER_OK;
}

// What one group's solve reports back.
struct BmgOut {
    std::vector<BmgState> states;
    int64_t launches = 0;
};

// One group of at most kBmgMaxNets networks (indices `mem` into grids, each with a hierarchy):
// head (sketches, r = b, x = 0, the first work list), the graph of the poll-period loop, tail
// (the final replacement, Z, R, the per-network summary).
er_status bmg_group(er_grid *const *grids, const std::vector<int> &mem, int k, uint64_t seed,
                    const int32_t *tile_rows, double *const *R_out, const er_solve_opts &opt, float *const *Y,
                    float *const *Zs, cudaStream_t us, cudaStream_t cs, int nsm, BmgOut &out) {
    const int m = (int)mem.size(), cap = m;
    std::vector<BmgNet> hn((size_t)m);
    std::vector<BatchItem> items((size_t)m);
    std::vector<int2> work;
    int Lmax = 0;
    for (int i = 0; i < m; ++i) {
        const int c = mem[(size_t)i];
        GridDev &g = grids[c]->d;
        Workspace *w = nullptr;
        er_status st = get_workspace(&g, k, ER_FP32_REFINE, 0, opt.block_order, &w);
        if (st == ER_OK) st = fp32_workspace_item(g, *w, Y[i], Zs[i], opt.tol, &items[(size_t)i]);
        MgHier *h = nullptr;
        if (st == ER_OK) st = mg_prepare(g, *w, &h);
        if (st != ER_OK) return st;
        ER_CUDA(cudaStreamSynchronize(w->s));  // any hierarchy set-up done on the workspace's stream
        const int L = (int)h->lv.size();
        if (L < 2 || L > kBmgLv) return fail(ER_ERR_INVALID_ARG, "network outside the batching form's level range");
        const int cbo = ((tile_rows && tile_rows[c]) ? tile_rows[c] : opt.block_order) == 2 ? 1 : 0;
        BmgNet &N = hn[(size_t)i];
        std::memset(&N, 0, sizeof(N));
        for (int l = 0; l < L; ++l) {
            N.map_r[l] = h->map_r[(size_t)l];
            N.map_c[l] = h->map_c[(size_t)l];
            N.map_z[l] = h->map_z[(size_t)l];
            N.lv[l] = h->lv[(size_t)l];
            N.lv[l].cb_outer = cbo;
            N.r[l] = l == 0 ? static_cast<float *>(w->r[0]) : h->r[(size_t)l];
            N.z[l] = h->z[(size_t)l];
        }
        N.dmap_z = h->dmap_z;
        N.dmap_c = h->dmap_c;
        N.umap_c = h->umap_c;
        for (int b = 0; b < 2; ++b) {
            N.dmap_p[b] = h->dmap_p[b];
            N.umap_p[b] = h->umap_p[b];
            N.p[b] = static_cast<float *>(w->p[b]);
        }
        N.ainv = h->ainv;
        N.ld_inv = h->ld_inv;
        N.nc = (int)h->lv[(size_t)L - 1].n;
        const dim3 cg = cinv_grid(N.nc, k);
        N.cinv_gx = (int)cg.x;
        N.x = Zs[i];
        N.part = h->part;
        N.scal = w->scal;
        N.msc = h->msc;
        N.cnt = h->cnt;
        N.err = w->ints + w->k + w->til.n_colblk;
        const MgRun run{&g, w, h, k, opt.tol, Zs[i], N.err, cbo};
        N.fold_beta = fold_args(run, n_tiles(h->lv[1]));
        N.fold_ct = fold_args(run, n_ctiles(h->lv[0]));
        N.L = L;
        for (int l = 0; l + 1 < L; ++l) N.items[l] = (int)tile_grid(h->lv[(size_t)l + 1], k).x;
        N.items[BP_CT] = (int)ctile_grid(h->lv[0], k).x;
        N.items[BP_CINV] = (int)(cg.x * cg.y);
        for (int64_t b = 0; b < w->til.n_ctas(); ++b) work.push_back(make_int2(i, (int)b));
        Lmax = std::max(Lmax, L);
    }
    if ((int64_t)work.size() >= INT32_MAX) return fail(ER_ERR_INVALID_ARG, "batch too large");

    // device copies: networks, batch items, the static (network, block) list of the FP32-form
    // passes, the running list, replacement flags and states
    const size_t list_n = 1 + (size_t)cap + (size_t)BP_N * (cap + 1);
    BmgBuf b_nets, b_items, b_work, b_list, b_need, b_state;
    ER_CUDA(cudaMalloc(&b_nets.p, (size_t)m * sizeof(BmgNet)));
    ER_CUDA(cudaMalloc(&b_items.p, (size_t)m * sizeof(BatchItem)));
    ER_CUDA(cudaMalloc(&b_work.p, std::max<size_t>(work.size(), 1) * sizeof(int2)));
    ER_CUDA(cudaMalloc(&b_list.p, list_n * sizeof(int)));
    ER_CUDA(cudaMalloc(&b_need.p, (size_t)m * sizeof(int)));
    ER_CUDA(cudaMalloc(&b_state.p, (size_t)m * sizeof(BmgState)));
    ER_CUDA(cudaMemcpyAsync(b_nets.p, hn.data(), (size_t)m * sizeof(BmgNet), cudaMemcpyHostToDevice, us));
    ER_CUDA(cudaMemcpyAsync(b_items.p, items.data(), (size_t)m * sizeof(BatchItem), cudaMemcpyHostToDevice, us));
    if (!work.empty())
        ER_CUDA(cudaMemcpyAsync(b_work.p, work.data(), work.size() * sizeof(int2), cudaMemcpyHostToDevice, us));
    const BmgNet *dn = static_cast<const BmgNet *>(b_nets.p);
    const BatchItem *di = static_cast<const BatchItem *>(b_items.p);
    const int2 *dw = static_cast<const int2 *>(b_work.p);
    const int nw = (int)work.size();
    int *dl = static_cast<int *>(b_list.p);
    int *dneed = static_cast<int *>(b_need.p);
    BmgState *ds = static_cast<BmgState *>(b_state.p);
    const unsigned nb = (unsigned)((m + 255) / 256);
    const unsigned nfz = (unsigned)(((int64_t)m * k + 255) / 256);

    // head: network i's sketch uses seed + its index in the call; error words, states; r = b,
    // x = 0, p = 0, rho0 (er_solve's initialisation); the first work list (every network)
    for (int i = 0; i < m; ++i) {
        er_status st = sketch(grids[mem[(size_t)i]], k, seed + (uint64_t)mem[(size_t)i], ER_FP32_REFINE, Y[i], us);
        if (st != ER_OK) return st;
    }
    k_bmg_reset<<<nb, 256, 0, us>>>(dn, ds, dneed, m);
    er_status st = fp32_batch_pass(MODE_INIT, di, dw, nw, 0, 0, us);
    if (st != ER_OK) return st;
    k_bmg_compact<<<1, kBmgMaxNets, 0, us>>>(dn, ds, nullptr, dl, m, cap, opt.maxit, 0, 0);
    ER_CUDA(cudaGetLastError());

    // the loop: a graph holding one WHILE node whose body is one poll period
    const int block = std::max(2, opt.check_every + (opt.check_every & 1));
    const size_t tsm = bmg_tile_smem(cap), dsm = bmg_dir_smem(cap), usm = bmg_upd_smem(cap),
                 csm = 4 * (size_t)(cap + 1);
    const int g_down = bmg_grid(k_bmg_tile<false, false>, tsm, nsm), g_up = bmg_grid(k_bmg_tile<true, false>, tsm, nsm),
              g_up0 = bmg_grid(k_bmg_tile<true, true>, tsm, nsm), g_dir = bmg_grid(k_bmg_dir, dsm, nsm),
              g_upd1 = bmg_grid(k_bmg_upd<true>, usm, nsm), g_upd0 = bmg_grid(k_bmg_upd<false>, usm, nsm),
              g_cinv = bmg_grid(k_bmg_cinv, csm, nsm), g_fold = 8 * nsm;
    struct GraphGuard {
        cudaGraph_t g = nullptr;
        cudaGraphExec_t e = nullptr;
        ~GraphGuard() {
            if (e) cudaGraphExecDestroy(e);
            if (g) cudaGraphDestroy(g);
        }
    } gg;
    ER_CUDA(cudaGraphCreate(&gg.g, 0));
    cudaGraphConditionalHandle h_loop;
    ER_CUDA(cudaGraphConditionalHandleCreate(&h_loop, gg.g, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h_loop;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t loop_node;
    ER_CUDA(cudaGraphAddNode(&loop_node, gg.g, nullptr, nullptr, 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    ER_CUDA(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    for (int it = 0; it < block; ++it) {
        const int cur = it & 1;
        // V-cycle: restriction down the levels, coarsest solves, prolongation up
        for (int l = 0; l + 1 < Lmax; ++l) k_bmg_tile<false, false><<<g_down, 256, tsm, cs>>>(dn, dl, cap, l, k);
        k_bmg_cinv<<<g_cinv, 256, csm, cs>>>(dn, dl, cap, k);
        for (int l = Lmax - 2; l >= 1; --l) k_bmg_tile<true, false><<<g_up, 256, tsm, cs>>>(dn, dl, cap, l, k);
        k_bmg_tile<true, true><<<g_up0, 256, tsm, cs>>>(dn, dl, cap, 0, k);
        k_bmg_fold<FOLD_BETA><<<g_fold, 256, 0, cs>>>(dn, dl, k);
        // CG: direction, step length, update, recursive residual norms
        k_bmg_dir<<<g_dir, 256, dsm, cs>>>(dn, dl, cap, k, cur);
        k_bmg_fold<FOLD_ALPHA><<<g_fold, 256, 0, cs>>>(dn, dl, k);
        if (cur == 1)
            k_bmg_upd<true><<<g_upd1, 256, usm, cs>>>(dn, dl, cap, k, cur);
        else
            k_bmg_upd<false><<<g_upd0, 256, usm, cs>>>(dn, dl, cap, k, cur);
        k_bmg_fold<FOLD_RR><<<g_fold, 256, 0, cs>>>(dn, dl, k);
    }
    k_bmg_control<<<nb, 256, 0, cs>>>(dn, ds, dneed, m, block, opt.replace_every, opt.maxit);
    fp32_batch_pass(MODE_ACCUM, di, dw, nw, 0, 0, cs, dneed);
    fp32_batch_pass(MODE_R, di, dw, nw, 0, 0, cs, dneed);
    k_bmg_freeze<<<nfz, 256, 0, cs>>>(dn, dneed, m, k, opt.tol);
    k_bmg_compact<<<1, kBmgMaxNets, 0, cs>>>(dn, ds, dneed, dl, m, cap, opt.maxit, h_loop, 1);
    cudaGraph_t captured = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(cs, &captured);
    if (ce != cudaSuccess) return cuda_fail(ce, "graph capture (multigrid batch)");
    ER_CUDA(cudaGraphInstantiate(&gg.e, gg.g, 0));
    ER_CUDA(cudaGraphLaunch(gg.e, us));

    // tail: the final replacement (a no-op on the iterate when the loop ended on one), Z, R
    k_bmg_zero_active_count<<<nb, 256, 0, us>>>(dn, m);
    st = fp32_batch_pass(MODE_ACCUM, di, dw, nw, 0, 0, us);
    if (st == ER_OK) st = fp32_batch_pass(MODE_R, di, dw, nw, 0, 0, us);
    if (st != ER_OK) return st;
    k_bmg_freeze<<<nfz, 256, 0, us>>>(dn, nullptr, m, k, opt.tol);
    st = fp32_batch_pass(MODE_UNSCALE, di, dw, nw, 0, 0, us);
    for (int i = 0; i < m && st == ER_OK; ++i)
        st = reff_map(grids[mem[(size_t)i]], Zs[i], k, ER_FP32_REFINE, R_out[mem[(size_t)i]], us);
    if (st != ER_OK) return st;
    k_bmg_summary<<<nb, 256, 0, us>>>(dn, ds, m, k, opt.tol);
    ER_CUDA(cudaGetLastError());
    out.states.resize((size_t)m);
    ER_CUDA(cudaMemcpyAsync(out.states.data(), ds, (size_t)m * sizeof(BmgState), cudaMemcpyDeviceToHost, us));
    ER_CUDA(cudaStreamSynchronize(us));
    int max_it = 0;
    for (const BmgState &s : out.states) max_it = std::max(max_it, s.it);
    // head: sketches, reset, init, list; per period: the iterations' passes, control, two
    // replacement passes, freeze, list; tail: 5 passes, the maps, the summary
    out.launches = (int64_t)m + 3 + (int64_t)(max_it / block) * (block * (2 * Lmax + 4) + 5) + 5 + m + 1;
    return ER_OK;
}

}  // namespace

er_status mg_batch_solve(er_grid *const *grids, int32_t n, int32_t k, uint64_t seed, const int32_t *tile_rows,
                         double *const *R_out, const er_solve_opts &opt, er_batch_stats *stats, cudaStream_t us,
                         std::chrono::steady_clock::time_point t0) {
    // every grid is used by this call alone (address order, so concurrent callers cannot deadlock)
    std::vector<er_grid *> by_addr(grids, grids + n);
    std::sort(by_addr.begin(), by_addr.end());
    std::vector<std::unique_lock<std::mutex>> locks;
    locks.reserve((size_t)n);
    for (er_grid *g : by_addr) locks.emplace_back(g->mu);
    // largest networks first: their blocks lead every pass's work list
    std::vector<int> order((size_t)n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return grids[a]->d.n > grids[b]->d.n; });
    // every network's sketch Y and solution Z
    std::vector<size_t> off((size_t)n);
    size_t tot = 0;
    for (int c = 0; c < n; ++c) {
        off[(size_t)c] = tot;
        tot += ((size_t)grids[c]->d.n * k * sizeof(float) + 255) & ~(size_t)255;
    }
    BmgBuf yz;
    ER_CUDA(cudaMalloc(&yz.p, 2 * tot));
    auto Yof = [&](int c) { return reinterpret_cast<float *>(static_cast<char *>(yz.p) + off[(size_t)c]); };
    auto Zof = [&](int c) { return reinterpret_cast<float *>(static_cast<char *>(yz.p) + tot + off[(size_t)c]); };

    int32_t iters = 0, reps = 0, conv = 0;
    int64_t launches = 0, nodes = 0;
    double mx = 0.0;
    bool err = false, unconv = false;
    std::vector<int> big;
    for (int q = 0; q < n; ++q) {
        const int c = order[(size_t)q];
        GridDev &g = grids[c]->d;
        if (g.n > kMgCoarseNodes && std::max(g.W, g.H) > 1) {
            big.push_back(c);
            continue;
        }
        // a network that is its own coarsest level: er_solve runs it with Jacobi; so does this
        er_solve_stats ss{};
        er_status st = sketch(grids[c], k, seed + (uint64_t)c, ER_FP32_REFINE, Yof(c), us);
        if (st == ER_OK) st = solve_locked(grids[c], Yof(c), Zof(c), k, ER_FP32_REFINE, &opt, &ss, us);
        const bool nc = st == ER_ERR_NOT_CONVERGED;
        if (st != ER_OK && !nc) return st;
        st = reff_map(grids[c], Zof(c), k, ER_FP32_REFINE, R_out[c], us);
        if (st != ER_OK) return st;
        unconv |= nc;
        iters = std::max(iters, ss.iterations);
        reps = std::max(reps, ss.sweeps);
        conv += ss.converged_cols == k;
        nodes += g.n - g.n_floating;
        mx = std::max(mx, ss.max_rel_residual);
        for (int i = 0; i < ER_N_PASS; ++i) launches += ss.launches[i];
        launches += 2;
    }
    int graphs = 0;
    if (!big.empty()) {
        er_status st = bmg_attributes();
        if (st != ER_OK) return st;
        int nsm = 0;
        ER_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, grids[big[0]]->d.device));
        cudaStream_t cs = nullptr;
        ER_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        struct StreamGuard {
            cudaStream_t s;
            ~StreamGuard() { cudaStreamDestroy(s); }
        } sg{cs};
        for (size_t g0 = 0; g0 < big.size(); g0 += kBmgMaxNets) {
            const std::vector<int> mem(big.begin() + (ptrdiff_t)g0,
                                       big.begin() + (ptrdiff_t)std::min(big.size(), g0 + kBmgMaxNets));
            std::vector<float *> Y, Z;
            for (int c : mem) {
                Y.push_back(Yof(c));
                Z.push_back(Zof(c));
            }
            BmgOut out;
            st = bmg_group(grids, mem, k, seed, tile_rows, R_out, opt, Y.data(), Z.data(), us, cs, nsm, out);
            if (st != ER_OK) return st;
            ++graphs;
            launches += out.launches;
            for (size_t i = 0; i < mem.size(); ++i) {
                const BmgState &x = out.states[i];
                const GridDev &g = grids[mem[i]]->d;
                iters = std::max(iters, x.it);
                reps = std::max(reps, x.replacements);
                conv += x.converged;
                err |= x.err != 0;
                unconv |= !x.converged;
                nodes += g.n - g.n_floating;
                mx = std::max(mx, x.max_resid);
            }
        }
    } else {
        ER_CUDA(cudaStreamSynchronize(us));
    }
    if (stats) {
        stats->n_grids = n;
        stats->iterations = iters;
        stats->replacements = reps;
        stats->converged = conv;
        stats->nodes = nodes;
        stats->max_rel_residual = mx;
        stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        stats->launches = (int32_t)std::min<int64_t>(launches, INT32_MAX);
        stats->graph_captures = graphs;
    }
    if (err) return fail(ER_ERR_TIMEOUT, "a bounded wait on a bulk copy expired inside a solver kernel");
    if (unconv) return fail(ER_ERR_NOT_CONVERGED, "maxit reached with networks still above tol");
    return ER_OK;
}

}  // namespace er
