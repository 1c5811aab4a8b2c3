// Pairwise effective resistance and IR drop from a solved sketch (sm_103a).
//
// With the supply grounded, any two network nodes u, v have
//   R(u, v) = (e_u - e_v)^T G^-1 (e_u - e_v)          (Sec. II-B, Eq. 2; Eq. 4)
// and a current I_l drawn at each load node l lowers node i by
//   drop_i = (G^-1 I)_i                              (Sec. II-A, Eq. 1).
// The solved sketch Z = G^-1 Y^T satisfies E[Z Z^T] = G^-1, so both follow from Z:
//   R_JL(u, v) = ||Z_u - Z_v||^2,      drop_JL = Z w,  w = Z^T I.
//
// k_pair_reff: a CTA computes a 64 x 64 block of pairs; Z rows of its u's and v's are
// staged through shared memory in chunks of 32 columns (transposed, so a thread's four
// consecutive u and four consecutive v of one column are one vector load each), and each
// thread accumulates a 4 x 4 register block of squared differences.  FP32 Z: differences
// and squares in FP32 over runs of 64 columns, run sums in FP64; FP64 Z: FP64 throughout.
// Differences are formed before squaring, so no R_u + R_v - 2 Z_u.Z_v cancellation enters.
//
// IR drop: k_drop_partial folds the load rows of Z into per-CTA partial sums of w (one
// thread per column, loads in a fixed order), k_drop_fold adds the partials in CTA order
// (deterministic), and k_drop_apply streams Z once, one warp per node, against w held in
// shared memory.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "er_internal.h"

namespace er {

namespace {

constexpr int kPT = 64;   // pairs tile edge
constexpr int kKC = 32;   // columns per staged chunk
constexpr int kDropMaxS = 8;
constexpr int kPartBlocks = 152;  // one CTA per SM

__device__ __forceinline__ double inf64() { return __longlong_as_double(0x7ff0000000000000LL); }

template <typename T>
__device__ __forceinline__ void lds4(const T *p, T (&o)[4]) {
    if constexpr (sizeof(T) == 4) {
        const float4 t = *reinterpret_cast<const float4 *>(p);
        o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
    } else {
        const double2 t0 = *reinterpret_cast<const double2 *>(p);
        const double2 t1 = *reinterpret_cast<const double2 *>(p + 2);
        o[0] = t0.x; o[1] = t0.y; o[2] = t1.x; o[3] = t1.y;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_pair_reff(const T *__restrict__ Z, int k, const int64_t *__restrict__ us,
                                                   int m, const int64_t *__restrict__ vs, int nv,
                                                   const uint8_t *__restrict__ floating, double *__restrict__ out) {
    // rows padded by 4 scalars: 16-byte aligned, so a thread's 4 consecutive u (or v) of one
    // column are one vector load
    __shared__ __align__(16) T su[kKC][kPT + 4];
    __shared__ __align__(16) T sv[kKC][kPT + 4];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;  // pairs (u0 + 4ty + a, v0 + 4tx + b)
    const int u0 = blockIdx.y * kPT, v0 = blockIdx.x * kPT;
    double acc[4][4];
    T run[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.0, run[a][b] = 0;
    // loader mapping: 64 rows x 32 columns per tile = 2048 scalars, 8 per thread as 2 x 4
    const int lr = threadIdx.x >> 2;        // row 0..63
    const int lc = (threadIdx.x & 3) * 8;   // column 0, 8, 16, 24 within the chunk
    const int64_t ru = u0 + lr < m ? us[u0 + lr] : -1;
    const int64_t rv = v0 + lr < nv ? vs[v0 + lr] : -1;
    // FP32: squares summed in FP32 over runs of kRun columns, runs in FP64 (FP64 arithmetic is
    // a small fraction of the FP32 rate, so it is kept out of the inner loop)
    constexpr int kRun = sizeof(T) == 4 ? 64 : kKC;
    for (int c0 = 0; c0 < k; c0 += kKC) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int c = c0 + lc + 4 * h;  // k is a multiple of 4, so c < k covers all four
            T a4[4] = {0, 0, 0, 0}, b4[4] = {0, 0, 0, 0};
            if (c < k) {
                if (ru >= 0) lds4(Z + ru * k + c, a4);
                if (rv >= 0) lds4(Z + rv * k + c, b4);
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                su[lc + 4 * h + e][lr] = a4[e];
                sv[lc + 4 * h + e][lr] = b4[e];
            }
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < kKC; ++kk) {
            T ua[4], vb[4];
            lds4(&su[kk][4 * ty], ua);
            lds4(&sv[kk][4 * tx], vb);
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const T d = ua[a] - vb[b];
                    run[a][b] = fma(d, d, run[a][b]);
                }
        }
        if ((c0 + kKC) % kRun == 0 || c0 + kKC >= k) {
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] += (double)run[a][b], run[a][b] = 0;
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int iu = u0 + 4 * ty + a;
        if (iu >= m) continue;
        const bool fu = floating[us[iu]] != 0;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int iv = v0 + 4 * tx + b;
            if (iv >= nv) continue;
            out[(int64_t)iu * nv + iv] = (fu || floating[vs[iv]]) ? inf64() : acc[a][b];
        }
    }
}

// part[blk][s][j] = sum over this CTA's loads l of I[l][s] * Z[load_l][j]
template <typename T, int S>
__global__ void __launch_bounds__(256) k_drop_partial(const T *__restrict__ Z, int k, const int64_t *__restrict__ loads,
                                                      const double *__restrict__ I, int64_t L, int64_t per_blk,
                                                      double *__restrict__ part) {
    const int64_t l0 = blockIdx.x * per_blk, l1 = min(L, l0 + per_blk);
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        double acc[S];
#pragma unroll
        for (int s = 0; s < S; ++s) acc[s] = 0.0;
        for (int64_t l = l0; l < l1; ++l) {
            const double z = (double)Z[loads[l] * k + j];
#pragma unroll
            for (int s = 0; s < S; ++s) acc[s] = fma(I[l * S + s], z, acc[s]);
        }
#pragma unroll
        for (int s = 0; s < S; ++s) part[((int64_t)blockIdx.x * S + s) * k + j] = acc[s];
    }
}

// w[s][j] = sum over CTAs b (in order) of part[b][s][j]
__global__ void k_drop_fold(const double *__restrict__ part, int nblk, int sk, double *__restrict__ w) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= sk) return;
    double acc = 0.0;
    for (int b = 0; b < nblk; ++b) acc += part[(int64_t)b * sk + t];
    w[t] = acc;
}

// drop[i][s] = sum_j Z[i][j] w[s][j]; one warp per node, w in shared memory (as T).  The
// accumulation runs in T: with FP32 Z its rounding stays at a few units of 1e-7 of
// ||Z_i|| ||w_s||, the level at which the FP32 rows of Z are themselves rounded (FP64
// arithmetic runs at a small fraction of the FP32 rate and would bound the kernel).
template <typename T, int S>
__global__ void __launch_bounds__(256) k_drop_apply(const T *__restrict__ Z, int64_t n, int k,
                                                    const double *__restrict__ w, const uint8_t *__restrict__ floating,
                                                    double *__restrict__ drop) {
    extern __shared__ __align__(16) unsigned char drop_smem[];
    T *sw = reinterpret_cast<T *>(drop_smem);  // [S][k]
    for (int t = threadIdx.x; t < S * k; t += blockDim.x) sw[t] = (T)w[t];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    constexpr int V = 16 / sizeof(T);
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
        const T *row = Z + i * k;
        T tot[S];
#pragma unroll
        for (int s = 0; s < S; ++s) tot[s] = 0;
        for (int c0 = lane * V; c0 < k; c0 += 32 * V) {
            T z[V];
            if constexpr (sizeof(T) == 4) {
                const float4 t = *reinterpret_cast<const float4 *>(row + c0);
                z[0] = t.x; z[1] = t.y; z[2] = t.z; z[3] = t.w;
            } else {
                const double2 t = *reinterpret_cast<const double2 *>(row + c0);
                z[0] = t.x; z[1] = t.y;
            }
#pragma unroll
            for (int s = 0; s < S; ++s)
#pragma unroll
                for (int v = 0; v < V; ++v) tot[s] = fma(z[v], sw[s * k + c0 + v], tot[s]);
        }
#pragma unroll
        for (int s = 0; s < S; ++s) {
            T x = tot[s];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            tot[s] = x;
        }
        if (lane < S) {
            T x = tot[0];
#pragma unroll
            for (int s = 1; s < S; ++s)
                if (lane == s) x = tot[s];
            drop[i * S + lane] = floating[i] ? inf64() : (double)x;
        }
    }
}

// I_pad[idx][s] = g_pad * V[i][s] for every pad (input order idx) at node i: the current it
// carries from the supply into the network when node i's voltage drops by V[i][s]
template <typename T>
__global__ void k_pad_currents(const T *__restrict__ V, int S, int64_t n, const int32_t *__restrict__ pad_ptr,
                               const int64_t *__restrict__ pad_eid, const double *__restrict__ pad_g, int64_t base,
                               double *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int32_t e = pad_ptr[i]; e < pad_ptr[i + 1]; ++e) {
        const int64_t idx = pad_eid[e] - base;
        for (int s = 0; s < S; ++s) out[idx * S + s] = pad_g[e] * (double)V[i * S + s];
    }
}

int sm_count(int dev) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return n;
}

// Grow the grid's auxiliary device buffer to at least `bytes` (synchronises the stream first:
// a previous call's kernels may still read it).
er_status aux_reserve(GridDev &d, size_t bytes, cudaStream_t s) {
    if (d.aux_bytes >= bytes) return ER_OK;
    ER_CUDA(cudaStreamSynchronize(s));
    if (d.aux) ER_CUDA(cudaFree(d.aux));
    d.aux = nullptr;
    d.aux_bytes = 0;
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(ER_ERR_OOM, "auxiliary buffer of " + std::to_string(bytes) + " bytes");
    }
    d.aux = p;
    d.aux_bytes = bytes;
    return ER_OK;
}

size_t up256(size_t b) { return (b + 255) & ~(size_t)255; }

er_status check_nodes(const GridDev &d, const int64_t *ids, int64_t count, const char *name) {
    if (count > 0 && !ids) return fail(ER_ERR_INVALID_ARG, std::string(name) + " is NULL");
    for (int64_t i = 0; i < count; ++i)
        if (ids[i] < 0 || ids[i] >= d.n)
            return fail(ER_ERR_INVALID_ARG, std::string(name) + "[" + std::to_string(i) + "] = " +
                                                std::to_string(ids[i]) + " is not a node id");
    return ER_OK;
}

template <typename T, int S>
void launch_drop(const GridDev &d, const T *Z, int k, const int64_t *loads, const double *I, int64_t L,
                 double *part, int nblk, int64_t per_blk, double *w, double *drop, int nsm, cudaStream_t s) {
    k_drop_partial<T, S><<<nblk, 256, 0, s>>>(Z, k, loads, I, L, per_blk, part);
    k_drop_fold<<<(S * k + 255) / 256, 256, 0, s>>>(part, nblk, S * k, w);
    const size_t smem = (size_t)S * k * sizeof(T);
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_drop_apply<T, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int64_t want = (d.n + 7) / 8;
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)nsm * 8));
    k_drop_apply<T, S><<<blocks, 256, smem, s>>>(Z, d.n, k, w, d.floating, drop);
}

template <typename T>
er_status drop_dispatch(const GridDev &d, const T *Z, int k, const int64_t *loads, const double *I, int64_t L, int S,
                        double *part, int nblk, int64_t per_blk, double *w, double *drop, int nsm, cudaStream_t s) {
    switch (S) {
        case 1: launch_drop<T, 1>(d, Z, k, loads, I, L, part, nblk, per_blk, w, drop, nsm, s); break;
        case 2: launch_drop<T, 2>(d, Z, k, loads, I, L, part, nblk, per_blk, w, drop, nsm, s); break;
        case 3: launch_drop<T, 3>(d, Z, k, loads, I, L, part, nblk, per_blk, w, drop, nsm, s); break;
        case 4: launch_drop<T, 4>(d, Z, k, loads, I, L, part, nblk, per_blk, w, drop, nsm, s); break;
        case 5: launch_drop<T, 5>(d, Z, k, loads, I, L, part, nblk, per_blk, w, drop, nsm, s); break;
        case 6: launch_drop<T, 6>(d, Z, k, loads, I, L, part, nblk, per_blk, w, drop, nsm, s); break;
        case 7: launch_drop<T, 7>(d, Z, k, loads, I, L, part, nblk, per_blk, w, drop, nsm, s); break;
        default: launch_drop<T, 8>(d, Z, k, loads, I, L, part, nblk, per_blk, w, drop, nsm, s); break;
    }
    ER_CUDA(cudaGetLastError());
    return ER_OK;
}

}  // namespace

er_status pair_reff(er_grid *g, const void *Z, int32_t k, er_precision prec, const int64_t *u, int32_t m,
                    const int64_t *v, int32_t nv, double *Rp, cudaStream_t s) {
    er_status st = check_nk(g, k, Z, "Z");
    if (st != ER_OK) return st;
    if (prec != ER_FP64 && prec != ER_FP32_REFINE) return fail(ER_ERR_INVALID_ARG, "bad precision");
    if (m < 0 || nv < 0) return fail(ER_ERR_INVALID_ARG, "negative pair count");
    if (m == 0 || nv == 0) return ER_OK;
    if (!Rp) return fail(ER_ERR_INVALID_ARG, "Rp is NULL");
    std::lock_guard<std::mutex> lk(g->mu);
    GridDev &d = g->d;
    if ((st = check_nodes(d, u, m, "u")) != ER_OK) return st;
    if ((st = check_nodes(d, v, nv, "v")) != ER_OK) return st;
    ER_CUDA(cudaSetDevice(d.device));
    const size_t bu = up256((size_t)m * 8), bv = up256((size_t)nv * 8);
    if ((st = aux_reserve(d, bu + bv, s)) != ER_OK) return st;
    int64_t *du = reinterpret_cast<int64_t *>(d.aux);
    int64_t *dv = reinterpret_cast<int64_t *>(reinterpret_cast<unsigned char *>(d.aux) + bu);
    ER_CUDA(cudaMemcpyAsync(du, u, (size_t)m * 8, cudaMemcpyHostToDevice, s));
    ER_CUDA(cudaMemcpyAsync(dv, v, (size_t)nv * 8, cudaMemcpyHostToDevice, s));
    const dim3 grid((unsigned)((nv + kPT - 1) / kPT), (unsigned)((m + kPT - 1) / kPT));
    if (grid.y > 65535u) return fail(ER_ERR_INVALID_ARG, "too many u nodes (at most 4,194,240)");
    if (prec == ER_FP64)
        k_pair_reff<double><<<grid, 256, 0, s>>>((const double *)Z, k, du, m, dv, nv, d.floating, Rp);
    else
        k_pair_reff<float><<<grid, 256, 0, s>>>((const float *)Z, k, du, m, dv, nv, d.floating, Rp);
    ER_CUDA(cudaGetLastError());
    ER_CUDA(cudaStreamSynchronize(s));
    return ER_OK;
}

er_status ir_drop(er_grid *g, const void *Z, int32_t k, er_precision prec, const int64_t *loads, const double *I,
                  int64_t L, int32_t S, double *drop, cudaStream_t s) {
    er_status st = check_nk(g, k, Z, "Z");
    if (st != ER_OK) return st;
    if (prec != ER_FP64 && prec != ER_FP32_REFINE) return fail(ER_ERR_INVALID_ARG, "bad precision");
    if (S < 1 || S > kDropMaxS) return fail(ER_ERR_INVALID_ARG, "S must be 1..8 load scenarios");
    if ((int64_t)S * k > 8192) return fail(ER_ERR_INVALID_ARG, "S * k must not exceed 8192");
    if (L < 0) return fail(ER_ERR_INVALID_ARG, "negative load count");
    if (!drop) return fail(ER_ERR_INVALID_ARG, "drop is NULL");
    if (L > 0 && !I) return fail(ER_ERR_INVALID_ARG, "I is NULL");
    std::lock_guard<std::mutex> lk(g->mu);
    GridDev &d = g->d;
    if ((st = check_nodes(d, loads, L, "loads")) != ER_OK) return st;
    for (int64_t i = 0; i < L * S; ++i)
        if (!std::isfinite(I[i])) return fail(ER_ERR_INVALID_ARG, "non-finite current");
    ER_CUDA(cudaSetDevice(d.device));
    const int nsm = sm_count(d.device);
    if (nsm <= 0) return fail(ER_ERR_CUDA, "multiprocessor count");
    const int64_t Lp = std::max<int64_t>(L, 1);
    const int nblk = (int)std::min<int64_t>(kPartBlocks, (Lp + 15) / 16);
    const int64_t per_blk = (Lp + nblk - 1) / nblk;
    const size_t bl = up256((size_t)Lp * 8), bi = up256((size_t)Lp * S * 8);
    const size_t bp = up256((size_t)nblk * S * k * 8), bw = up256((size_t)S * k * 8);
    if ((st = aux_reserve(d, bl + bi + bp + bw, s)) != ER_OK) return st;
    unsigned char *base = reinterpret_cast<unsigned char *>(d.aux);
    int64_t *dl = reinterpret_cast<int64_t *>(base);
    double *dI = reinterpret_cast<double *>(base + bl);
    double *part = reinterpret_cast<double *>(base + bl + bi);
    double *w = reinterpret_cast<double *>(base + bl + bi + bp);
    if (L > 0) {
        ER_CUDA(cudaMemcpyAsync(dl, loads, (size_t)L * 8, cudaMemcpyHostToDevice, s));
        ER_CUDA(cudaMemcpyAsync(dI, I, (size_t)L * S * 8, cudaMemcpyHostToDevice, s));
    }
    if (prec == ER_FP64)
        st = drop_dispatch<double>(d, (const double *)Z, k, dl, dI, L, S, part, nblk, per_blk, w, drop, nsm, s);
    else
        st = drop_dispatch<float>(d, (const float *)Z, k, dl, dI, L, S, part, nblk, per_blk, w, drop, nsm, s);
    if (st != ER_OK) return st;
    ER_CUDA(cudaStreamSynchronize(s));
    return ER_OK;
}

er_status pad_currents(er_grid *g, const void *V, int32_t S, er_precision prec, double *Ipad, cudaStream_t s) {
    if (!g) return fail(ER_ERR_INVALID_ARG, "grid is NULL");
    if (prec != ER_FP64 && prec != ER_FP32_REFINE) return fail(ER_ERR_INVALID_ARG, "bad precision");
    if (S < 1) return fail(ER_ERR_INVALID_ARG, "S must be positive");
    if (!V || !Ipad) return fail(ER_ERR_INVALID_ARG, "V or I_pad is NULL");
    const GridDev &d = g->d;
    ER_CUDA(cudaSetDevice(d.device));
    const int64_t base = d.ex_slots + d.ey_slots + d.n_tsv;
    const unsigned blocks = (unsigned)((d.n + 255) / 256);
    if (prec == ER_FP64)
        k_pad_currents<double><<<blocks, 256, 0, s>>>((const double *)V, S, d.n, d.pad_ptr, d.pad_eid, d.pad_g, base,
                                                      Ipad);
    else
        k_pad_currents<float><<<blocks, 256, 0, s>>>((const float *)V, S, d.n, d.pad_ptr, d.pad_eid, d.pad_g, base,
                                                     Ipad);
    ER_CUDA(cudaGetLastError());
    return ER_OK;
}

}  // namespace er

extern "C" {

er_status er_pad_currents(er_grid *g, const void *V, int32_t S, er_precision prec, double *I_pad, void *stream) {
    return er::pad_currents(g, V, S, prec, I_pad, (cudaStream_t)stream);
}


er_status er_pair_reff(er_grid *g, const void *Z, int32_t k, er_precision prec, const int64_t *u, int32_t m,
                       const int64_t *v, int32_t nv, double *Rp, void *stream) {
    return er::pair_reff(g, Z, k, prec, u, m, v, nv, Rp, (cudaStream_t)stream);
}

er_status er_ir_drop(er_grid *g, const void *Z, int32_t k, er_precision prec, const int64_t *loads, const double *I,
                     int64_t n_loads, int32_t S, double *drop, void *stream) {
    return er::ir_drop(g, Z, k, prec, loads, I, n_loads, S, drop, (cudaStream_t)stream);
}

}  // extern "C"
