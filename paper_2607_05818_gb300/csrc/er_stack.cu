// The paper's bump-to-load effective-resistance pipeline on a uniform die stack (sm_103a).
//
// Setting (Sec. III-A/B): d stacked dies, die i a uniform M x N mesh with x-segments r_i and
// y-segments s_i; p TSV columns at (tx_k, ty_k), segment k between die i and i+1 of
// resistance Rt[i][k]; m bumps on die 0 and n loads on die d-1.  Steps, in the paper's order:
//
//  K3  cos((x + 1/2) theta_m) tables by the multiple-angle recursion
//      c(x+1) = 2 cos(theta) c(x) - c(x-1)            (Sec. III-E),
//      re-seeded from directly evaluated cosines every 32 steps, which bounds the recursion's
//      error growth (about x^2 eps for small theta) without giving up the recursion;
//  K1/K2  Wu's two-point resistance (Eq. 3) for every TSV pair of every die, every bump-TSV
//      pair of die 0 and every load-TSV pair of die d-1: the double sum over modes (m, n) is
//      split across the threads of a CTA (each thread a strided share of n for every m) and
//      reduced in the CTA; a CTA evaluates up to 8 pairs so that one read of 1/lambda_mn
//      serves all of them;
//  Eq. 13  the pair-independent system C x = b: C = [A~ + D, B; B^T, 0] with A~ block
//      tridiagonal (diagonal blocks -(R^i + R^{i+1})/2, off-diagonal blocks +R^{i+1}/2,
//      zero diagonals), D = diag(Rt), B = blkdiag(1_p);
//  K4  one LU factorisation of C with partial pivoting (blocked, right-looking: a one-CTA
//      panel factorisation, row interchanges, a triangular solve for the U12 block and an
//      FP64 tiled update of the trailing matrix);
//  Eq. 14 / K5  m + n right-hand sides b^1_i (bump i: -R^0_{bump,TSV}/2 in block 0) and
//      b^d_j (load j: -R^{d-1}_{load,TSV}/2 in block d-2), both with 1/2 in every
//      constraint row, solved with the one factorisation (one warp per right-hand side);
//  Eq. 15 / K6  R(i, j) = -(x^1_i + x^d_j)^T (b^1_i + b^d_j) for all m x n pairs, summed over
//      the rows where a right-hand side can be non-zero (blocks 0 and d-2, constraint rows).
//
// Readings of the garbled typesetting (Eq. 8 as defined beside it, off-diagonal blocks of A~,
// b's last block 1_{d-1} split as 1/2 + 1/2) are those under which R = -x^T b follows from
// Eq. 6; they are pinned on the CPU against full Cholesky solves.  Everything is FP64.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "er_internal.h"

namespace er {

namespace {

struct WuPair {
    int32_t x1, y1, x2, y2;
    int64_t o1, o2;  // output offsets (o2 < 0: one output)
};

constexpr int kCosSeed = 32;  // recursion steps between direct re-seeds

// T[x*M + m] = cos((x + 1/2) m pi / M) for x, m in [0, M)
__global__ void k_cos_half(int M, double *T) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    const double two_c = 2.0 * cospi((double)m / M);
    double prev = 0.0, cur = 0.0;
    for (int x = 0; x < M; ++x) {
        if (x % kCosSeed == 0) {
            // (x +- 1/2) m / M in units of pi, reduced exactly in integers modulo 2 (period)
            const int64_t den = 2LL * M;
            const int64_t jc = ((2LL * x + 1) * m) % (2 * den);
            const int64_t jp = ((2LL * x - 1) * m % (2 * den) + 2 * den) % (2 * den);
            cur = cospi((double)jc / (double)den);
            prev = cospi((double)jp / (double)den);
        } else {
            const double nxt = fma(two_c, cur, -prev);
            prev = cur;
            cur = nxt;
        }
        T[(int64_t)x * M + m] = cur;
    }
}

// inv[(m-1)(N-1) + n-1] = 1 / ((1 - cos theta_m) / r + (1 - cos phi_n) / s), with
// 1 - cos a = 2 sin^2(a/2) (no cancellation for small angles)
__global__ void k_inv_lambda(int M, int N, double r, double s, double *inv) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t tot = (int64_t)(M - 1) * (N - 1);
    if (t >= tot) return;
    const int m = 1 + (int)(t / (N - 1)), n = 1 + (int)(t % (N - 1));
    const double a = sinpi(0.5 * m / M), b = sinpi(0.5 * n / N);
    inv[t] = 1.0 / (2.0 * a * a / r + 2.0 * b * b / s);
}

// Eq. 3 for PB pairs per CTA: R = r/N |x1-x2| + s/M |y1-y2| + 2/(MN) sum_{m,n} t_mn^2 / lambda_mn,
// t_mn = c_m(x1) d_n(y1) - c_m(x2) d_n(y2).  The pairs' cosine rows are staged in shared memory.
template <int PB>
__global__ void k_wu(int M, int N, double r, double s, const double *__restrict__ cxT,
                     const double *__restrict__ cyT, const double *__restrict__ inv,
                     const WuPair *__restrict__ pairs, int npairs, double *__restrict__ out) {
    extern __shared__ __align__(16) double wsm[];
    double *cx = wsm;                // [PB][2][M]
    double *cy = wsm + PB * 2 * M;   // [PB][2][N]
    __shared__ double red[PB][8];
    const int p0 = blockIdx.x * PB;
    for (int t = threadIdx.x; t < PB * 2 * M; t += blockDim.x) {
        const int p = t / (2 * M), e = (t / M) & 1, mm = t % M;
        const WuPair q = pairs[min(p0 + p, npairs - 1)];
        cx[t] = cxT[(int64_t)(e ? q.x2 : q.x1) * M + mm];
    }
    for (int t = threadIdx.x; t < PB * 2 * N; t += blockDim.x) {
        const int p = t / (2 * N), e = (t / N) & 1, nn = t % N;
        const WuPair q = pairs[min(p0 + p, npairs - 1)];
        cy[t] = cyT[(int64_t)(e ? q.y2 : q.y1) * N + nn];
    }
    __syncthreads();
    double acc[PB];
#pragma unroll
    for (int p = 0; p < PB; ++p) acc[p] = 0.0;
    for (int m = 1; m < M; ++m) {
        double a[PB], b[PB];
#pragma unroll
        for (int p = 0; p < PB; ++p) a[p] = cx[(2 * p) * M + m], b[p] = cx[(2 * p + 1) * M + m];
        const double *invm = inv + (int64_t)(m - 1) * (N - 1) - 1;
        for (int n = 1 + threadIdx.x; n < N; n += blockDim.x) {
            const double w = invm[n];
#pragma unroll
            for (int p = 0; p < PB; ++p) {
                const double t = fma(a[p], cy[(2 * p) * N + n], -b[p] * cy[(2 * p + 1) * N + n]);
                acc[p] = fma(t * t, w, acc[p]);
            }
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int p = 0; p < PB; ++p) {
        double v = acc[p];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[p][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < PB && p0 + (int)threadIdx.x < npairs) {
        const int p = threadIdx.x;
        double sum = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += red[p][w];
        const WuPair q = pairs[p0 + p];
        const double R = r / N * abs(q.x1 - q.x2) + s / M * abs(q.y1 - q.y2) + 2.0 / ((double)M * N) * sum;
        out[q.o1] = R;
        if (q.o2 >= 0) out[q.o2] = R;
    }
}

// C of Eq. 13, row-major [NC][NC]; RT [d][p][p] intra-die TSV-TSV resistances
__global__ void k_build_c(int d, int p, const double *__restrict__ RT, const double *__restrict__ Rt,
                          double *__restrict__ C) {
    const int nI = (d - 1) * p, NC = nI + d - 1;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)NC * NC) return;
    const int a = (int)(t / NC), b = (int)(t % NC);
    double v = 0.0;
    if (a < nI && b < nI) {
        const int ia = a / p, ja = a % p, ib = b / p, jb = b % p;
        const int64_t pp = (int64_t)p * p;
        if (ia == ib) {
            v = -0.5 * (RT[ia * pp + (int64_t)ja * p + jb] + RT[(ia + 1) * pp + (int64_t)ja * p + jb]);
            if (ja == jb) v += Rt[(int64_t)ia * p + ja];
        } else if (ib == ia + 1 || ia == ib + 1) {
            v = 0.5 * RT[max(ia, ib) * pp + (int64_t)ja * p + jb];
        }
    } else if (a < nI && b >= nI) {
        v = (b - nI == a / p) ? 1.0 : 0.0;
    } else if (a >= nI && b < nI) {
        v = (a - nI == b / p) ? 1.0 : 0.0;
    }
    C[t] = v;
}

// right-hand sides, one contiguous column per RHS: Bm[c][NC]; bumps c < m, loads m <= c < m+n
__global__ void k_build_rhs(int d, int p, int m, int n, const double *__restrict__ RB, const double *__restrict__ RL,
                            double *__restrict__ Bm, double *__restrict__ X) {
    const int nI = (d - 1) * p, NC = nI + d - 1;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)(m + n) * NC) return;
    const int c = (int)(t / NC), row = (int)(t % NC);
    double v = 0.0;
    if (row >= nI) {
        v = 0.5;
    } else if (c < m) {
        if (row < p) v = -0.5 * RB[(int64_t)c * p + row];
    } else {
        const int lo = (d - 2) * p;
        if (row >= lo && row < lo + p) v = -0.5 * RL[(int64_t)(c - m) * p + (row - lo)];
    }
    Bm[t] = v;
    X[t] = v;
}

// ---- LU with partial pivoting, row-major A [NC][NC] ----------------------------------

constexpr int kNB = 32;

// factor columns [j0, j0+jb) over rows [j0, NC) (one CTA); ties in |pivot| go to the lower row
__global__ void __launch_bounds__(512) k_lu_panel(double *A, int NC, int j0, int jb, int *piv, int *err) {
    __shared__ double sv[16];
    __shared__ int si[16];
    __shared__ int s_p;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int c = j0; c < j0 + jb; ++c) {
        double best = -1.0;
        int bi = NC;
        for (int r = c + threadIdx.x; r < NC; r += blockDim.x) {
            const double v = fabs(A[(int64_t)r * NC + c]);
            if (v > best) best = v, bi = r;  // rows visited in increasing order per thread
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > best || (ov == best && oi < bi)) best = ov, bi = oi;
        }
        if (lane == 0) sv[warp] = best, si[warp] = bi;
        __syncthreads();
        if (threadIdx.x == 0) {
            double b = sv[0];
            int i = si[0];
            for (int w = 1; w < nw; ++w)
                if (sv[w] > b || (sv[w] == b && si[w] < i)) b = sv[w], i = si[w];
            if (!(b > 0.0)) *err = 1;  // singular (or NaN) pivot column
            s_p = i < NC ? i : c;
            piv[c] = s_p;
        }
        __syncthreads();
        const int pr = s_p;
        if (pr != c)
            for (int cc = j0 + threadIdx.x; cc < j0 + jb; cc += blockDim.x) {
                const double t = A[(int64_t)c * NC + cc];
                A[(int64_t)c * NC + cc] = A[(int64_t)pr * NC + cc];
                A[(int64_t)pr * NC + cc] = t;
            }
        __syncthreads();
        const double pv = A[(int64_t)c * NC + c];
        const double rp = pv != 0.0 ? 1.0 / pv : 0.0;
        for (int r = c + 1 + threadIdx.x; r < NC; r += blockDim.x) {
            const double l = A[(int64_t)r * NC + c] * rp;
            A[(int64_t)r * NC + c] = l;
            for (int cc = c + 1; cc < j0 + jb; ++cc) A[(int64_t)r * NC + cc] -= l * A[(int64_t)c * NC + cc];
        }
        __syncthreads();
    }
}

// row interchanges of the panel applied to every column outside it
__global__ void k_lu_swap(double *A, int NC, int j0, int jb, const int *piv) {
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= NC || (col >= j0 && col < j0 + jb)) return;
    for (int c = j0; c < j0 + jb; ++c) {
        const int pr = piv[c];
        if (pr != c) {
            const double t = A[(int64_t)c * NC + col];
            A[(int64_t)c * NC + col] = A[(int64_t)pr * NC + col];
            A[(int64_t)pr * NC + col] = t;
        }
    }
}

// U12 = L11^-1 A12 (L11 unit lower), one thread per column of A12
__global__ void k_lu_trsm(double *A, int NC, int j0, int jb) {
    __shared__ double L[kNB][kNB];
    for (int t = threadIdx.x; t < jb * jb; t += blockDim.x) L[t / jb][t % jb] = A[(int64_t)(j0 + t / jb) * NC + j0 + t % jb];
    __syncthreads();
    const int col = j0 + jb + blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= NC) return;
    double x[kNB];
#pragma unroll
    for (int rr = 0; rr < kNB; ++rr) x[rr] = rr < jb ? A[(int64_t)(j0 + rr) * NC + col] : 0.0;
#pragma unroll
    for (int rr = 1; rr < kNB; ++rr) {
        double v = x[rr];
#pragma unroll
        for (int q = 0; q < rr; ++q) v -= L[rr][q] * x[q];
        x[rr] = rr < jb ? v : 0.0;
    }
#pragma unroll
    for (int rr = 0; rr < kNB; ++rr)
        if (rr < jb) A[(int64_t)(j0 + rr) * NC + col] = x[rr];
}

// A22 -= L21 U12 on 64 x 64 tiles, each thread a 4 x 4 block
__global__ void __launch_bounds__(256) k_lu_gemm(double *A, int NC, int j0, int jb) {
    __shared__ double Ls[64][kNB + 1];
    __shared__ double Us[kNB][64 + 1];
    const int s0 = j0 + jb;
    const int r0 = s0 + blockIdx.y * 64, c0 = s0 + blockIdx.x * 64;
    for (int t = threadIdx.x; t < 64 * kNB; t += blockDim.x) {
        const int rr = t / kNB, q = t % kNB;
        Ls[rr][q] = (r0 + rr < NC && q < jb) ? A[(int64_t)(r0 + rr) * NC + j0 + q] : 0.0;
        const int qq = t / 64, cc = t % 64;
        Us[qq][cc] = (c0 + cc < NC && qq < jb) ? A[(int64_t)(j0 + qq) * NC + c0 + cc] : 0.0;
    }
    __syncthreads();
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[4][4] = {};
    for (int q = 0; q < jb; ++q) {
        double a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = Ls[ty + 16 * i][q], b[i] = Us[q][tx + 16 * i];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = r0 + ty + 16 * i;
        if (r >= NC) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = c0 + tx + 16 * j;
            if (c < NC) A[(int64_t)r * NC + c] -= acc[i][j];
        }
    }
}

// X[c][:] <- P X[c][:], then L^-1 and U^-1 applied to every right-hand side; one warp per RHS
__global__ void __launch_bounds__(256) k_lu_solve(const double *__restrict__ A, int NC, const int *__restrict__ piv,
                                                  double *X, int nrhs) {
    const int lane = threadIdx.x & 31;
    const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (c >= nrhs) return;
    double *x = X + (int64_t)c * NC;
    if (lane == 0)
        for (int i = 0; i < NC; ++i) {
            const int pr = piv[i];
            if (pr != i) {
                const double t = x[i];
                x[i] = x[pr];
                x[pr] = t;
            }
        }
    __syncwarp();
    for (int i = 1; i < NC; ++i) {  // forward, unit lower
        double sum = 0.0;
        for (int q = lane; q < i; q += 32) sum = fma(A[(int64_t)i * NC + q], x[q], sum);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if (lane == 0) x[i] -= sum;
        __syncwarp();
    }
    for (int i = NC - 1; i >= 0; --i) {  // backward, upper
        double sum = 0.0;
        for (int q = i + 1 + lane; q < NC; q += 32) sum = fma(A[(int64_t)i * NC + q], x[q], sum);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if (lane == 0) x[i] = (x[i] - sum) / A[(int64_t)i * NC + i];
        __syncwarp();
    }
}

// row t of the rows where a right-hand side can be non-zero: block 0, block d-2 (when
// distinct), then the d-1 constraint rows
__device__ __forceinline__ int dot_row(int t, int d, int p) {
    if (t < p) return t;
    if (d > 2) {
        if (t < 2 * p) return (d - 2) * p + (t - p);
        return (d - 1) * p + (t - 2 * p);
    }
    return (d - 1) * p + (t - p);
}

// R[i][j] = -(x1_i + xd_j) . (b1_i + bd_j); a CTA covers 16 bumps x 64 loads, each thread 4 x 1
__global__ void __launch_bounds__(256) k_pair_dot(const double *__restrict__ X, const double *__restrict__ Bm, int NC,
                                                  int d, int p, int m, int n, double *__restrict__ R) {
    __shared__ double xb[16][33], bb[16][33], xl[64][33], bl[64][33];
    const int nrows = (d > 2 ? 2 * p : p) + d - 1;
    const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;  // load tx, bumps 4 ty .. 4 ty + 3
    const int i0 = blockIdx.y * 16, j0 = blockIdx.x * 64;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int t0 = 0; t0 < nrows; t0 += 32) {
        for (int t = threadIdx.x; t < 16 * 32; t += blockDim.x) {
            const int bi = t / 32, q = t % 32;
            const bool ok = i0 + bi < m && t0 + q < nrows;
            const int64_t off = ok ? (int64_t)(i0 + bi) * NC + dot_row(t0 + q, d, p) : 0;
            xb[bi][q] = ok ? X[off] : 0.0;
            bb[bi][q] = ok ? Bm[off] : 0.0;
        }
        for (int t = threadIdx.x; t < 64 * 32; t += blockDim.x) {
            const int lj = t / 32, q = t % 32;
            const bool ok = j0 + lj < n && t0 + q < nrows;
            const int64_t off = ok ? (int64_t)(m + j0 + lj) * NC + dot_row(t0 + q, d, p) : 0;
            xl[lj][q] = ok ? X[off] : 0.0;
            bl[lj][q] = ok ? Bm[off] : 0.0;
        }
        __syncthreads();
#pragma unroll 4
        for (int q = 0; q < 32; ++q) {
            const double xv = xl[tx][q], bv = bl[tx][q];
#pragma unroll
            for (int a = 0; a < 4; ++a) acc[a] = fma(xb[4 * ty + a][q] + xv, bb[4 * ty + a][q] + bv, acc[a]);
        }
        __syncthreads();
    }
    if (j0 + tx >= n) return;
#pragma unroll
    for (int a = 0; a < 4; ++a)
        if (i0 + 4 * ty + a < m) R[(int64_t)(i0 + 4 * ty + a) * n + j0 + tx] = -acc[a];
}

struct DevBuf {
    std::vector<void *> ptrs;
    ~DevBuf() {
        for (void *p : ptrs) cudaFree(p);
    }
    template <typename T>
    er_status get(T **out, size_t count, const char *what) {
        void *p = nullptr;
        if (cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) {
            cudaGetLastError();
            return fail(ER_ERR_OOM, std::string("er_stack_pairs: ") + what);
        }
        ptrs.push_back(p);
        *out = reinterpret_cast<T *>(p);
        return ER_OK;
    }
};

unsigned nb(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

template <int PB>
cudaError_t launch_wu(int M, int N, double r, double s, const double *cxT, const double *cyT, const double *inv,
                      const WuPair *pairs, int npairs, double *out, cudaStream_t st) {
    if (npairs <= 0) return cudaSuccess;
    const size_t smem = (size_t)PB * 2 * (M + N) * sizeof(double);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_wu<PB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int threads = std::min(256, std::max(32, ((N - 1 + 31) / 32) * 32));
    k_wu<PB><<<nb(npairs, PB), threads, smem, st>>>(M, N, r, s, cxT, cyT, inv, pairs, npairs, out);
    return cudaGetLastError();
}

}  // namespace

er_status stack_pairs(const er_stack *st, const int32_t *bump_xy, int32_t m, const int32_t *load_xy, int32_t n,
                      double *R, er_stack_stats *stats, cudaStream_t s) {
    const auto t_start = std::chrono::steady_clock::now();
    if (!st) return fail(ER_ERR_INVALID_ARG, "stack is NULL");
    const int M = st->M, N = st->N, d = st->d, p = st->p;
    if (M < 1 || N < 1 || (int64_t)M * N > (1LL << 26)) return fail(ER_ERR_INVALID_ARG, "bad mesh size");
    if (M + N > 3200) return fail(ER_ERR_INVALID_ARG, "M + N must not exceed 3200");
    if (d < 2 || d > 64) return fail(ER_ERR_INVALID_ARG, "d must be 2..64 dies");
    if (p < 1) return fail(ER_ERR_INVALID_ARG, "at least one TSV column is needed (else R is infinite)");
    if ((int64_t)(p + 1) * (d - 1) > 46000) return fail(ER_ERR_INVALID_ARG, "reduced system too large");
    if (m < 0 || n < 0) return fail(ER_ERR_INVALID_ARG, "negative bump or load count");
    if (!st->r || !st->s || !st->tsv_xy || !st->Rt) return fail(ER_ERR_INVALID_ARG, "NULL stack array");
    if ((m > 0 && !bump_xy) || (n > 0 && !load_xy)) return fail(ER_ERR_INVALID_ARG, "NULL bump or load array");
    if (m > 0 && n > 0 && !R) return fail(ER_ERR_INVALID_ARG, "R is NULL");
    for (int i = 0; i < d; ++i)
        if (!(st->r[i] > 0.0) || !(st->s[i] > 0.0) || !std::isfinite(st->r[i]) || !std::isfinite(st->s[i]))
            return fail(ER_ERR_INVALID_ARG, "segment resistances must be positive and finite");
    for (int64_t i = 0; i < (int64_t)(d - 1) * p; ++i)
        if (!(st->Rt[i] > 0.0) || !std::isfinite(st->Rt[i]))
            return fail(ER_ERR_INVALID_ARG, "TSV resistances must be positive and finite");
    auto in_mesh = [&](const int32_t *xy, int64_t cnt) {
        for (int64_t i = 0; i < cnt; ++i)
            if (xy[2 * i] < 0 || xy[2 * i] >= M || xy[2 * i + 1] < 0 || xy[2 * i + 1] >= N) return false;
        return true;
    };
    if (!in_mesh(st->tsv_xy, p) || !in_mesh(bump_xy, m) || !in_mesh(load_xy, n))
        return fail(ER_ERR_INVALID_ARG, "a TSV, bump or load lies outside the mesh");
    if (m == 0 || n == 0) return ER_OK;

    const int nI = (d - 1) * p, NC = nI + d - 1, nrhs = m + n;
    const int64_t pp = (int64_t)p * p;
    // Wu pair lists per die: TSV pairs (both triangle entries of RT), bump-TSV on die 0,
    // load-TSV on die d-1.  Output layout: RT [d][p][p] | RB [m][p] | RL [n][p]
    const int64_t oRB = (int64_t)d * pp, oRL = oRB + (int64_t)m * p, nout = oRL + (int64_t)n * p;
    std::vector<std::vector<WuPair>> lists(d);
    for (int i = 0; i < d; ++i) {
        for (int j = 0; j < p; ++j)
            for (int k = j + 1; k < p; ++k)
                lists[i].push_back({st->tsv_xy[2 * j], st->tsv_xy[2 * j + 1], st->tsv_xy[2 * k], st->tsv_xy[2 * k + 1],
                                    i * pp + (int64_t)j * p + k, i * pp + (int64_t)k * p + j});
        if (i == 0)
            for (int b = 0; b < m; ++b)
                for (int j = 0; j < p; ++j)
                    lists[i].push_back({bump_xy[2 * b], bump_xy[2 * b + 1], st->tsv_xy[2 * j], st->tsv_xy[2 * j + 1],
                                        oRB + (int64_t)b * p + j, -1});
        if (i == d - 1)
            for (int l = 0; l < n; ++l)
                for (int j = 0; j < p; ++j)
                    lists[i].push_back({load_xy[2 * l], load_xy[2 * l + 1], st->tsv_xy[2 * j], st->tsv_xy[2 * j + 1],
                                        oRL + (int64_t)l * p + j, -1});
    }
    int64_t npairs_all = 0;
    for (auto &l : lists) npairs_all += (int64_t)l.size();
    for (auto &l : lists)
        if (l.size() > 0x7fffffff) return fail(ER_ERR_INVALID_ARG, "too many Wu pairs");

    DevBuf buf;
    double *cxT, *cyT, *inv, *wu, *Rt, *C, *Bm, *X;
    WuPair *dpairs;
    int *piv, *err;
    er_status e;
    if ((e = buf.get(&cxT, (size_t)M * M, "cos table")) != ER_OK) return e;
    if ((e = buf.get(&cyT, (size_t)N * N, "cos table")) != ER_OK) return e;
    if ((e = buf.get(&inv, (size_t)std::max(M - 1, 1) * std::max(N - 1, 1), "1/lambda")) != ER_OK) return e;
    if ((e = buf.get(&wu, (size_t)nout, "Wu output")) != ER_OK) return e;
    if ((e = buf.get(&Rt, (size_t)nI, "TSV resistances")) != ER_OK) return e;
    if ((e = buf.get(&C, (size_t)NC * NC, "reduced system")) != ER_OK) return e;
    if ((e = buf.get(&Bm, (size_t)nrhs * NC, "right-hand sides")) != ER_OK) return e;
    if ((e = buf.get(&X, (size_t)nrhs * NC, "solutions")) != ER_OK) return e;
    if ((e = buf.get(&dpairs, (size_t)npairs_all, "pair list")) != ER_OK) return e;
    if ((e = buf.get(&piv, (size_t)NC, "pivots")) != ER_OK) return e;
    if ((e = buf.get(&err, 1, "error word")) != ER_OK) return e;

    cudaEvent_t ev[6];
    for (auto &x : ev) ER_CUDA(cudaEventCreate(&x));
    struct EvFree {
        cudaEvent_t *e;
        ~EvFree() {
            for (int i = 0; i < 6; ++i) cudaEventDestroy(e[i]);
        }
    } evfree{ev};

    ER_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    ER_CUDA(cudaMemsetAsync(wu, 0, (size_t)d * pp * sizeof(double), s));  // RT diagonals stay 0
    ER_CUDA(cudaMemcpyAsync(Rt, st->Rt, (size_t)nI * sizeof(double), cudaMemcpyHostToDevice, s));
    {
        int64_t off = 0;
        for (auto &l : lists) {
            if (!l.empty())
                ER_CUDA(cudaMemcpyAsync(dpairs + off, l.data(), l.size() * sizeof(WuPair), cudaMemcpyHostToDevice, s));
            off += (int64_t)l.size();
        }
    }
    ER_CUDA(cudaEventRecord(ev[0], s));
    // K3: cosine tables (shared by all dies), then K1/K2 per die
    k_cos_half<<<nb(M, 128), 128, 0, s>>>(M, cxT);
    k_cos_half<<<nb(N, 128), 128, 0, s>>>(N, cyT);
    ER_CUDA(cudaGetLastError());
    {
        int64_t off = 0;
        for (int i = 0; i < d; ++i) {
            const int np_i = (int)lists[i].size();
            if (M > 1 && N > 1) {
                k_inv_lambda<<<nb((int64_t)(M - 1) * (N - 1), 256), 256, 0, s>>>(M, N, st->r[i], st->s[i], inv);
                ER_CUDA(cudaGetLastError());
            }
            cudaError_t ce = (M + N <= 1600)
                                 ? launch_wu<8>(M, N, st->r[i], st->s[i], cxT, cyT, inv, dpairs + off, np_i, wu, s)
                                 : launch_wu<4>(M, N, st->r[i], st->s[i], cxT, cyT, inv, dpairs + off, np_i, wu, s);
            if (ce != cudaSuccess) return cuda_fail(ce, "k_wu");
            off += np_i;
        }
    }
    ER_CUDA(cudaEventRecord(ev[1], s));
    // Eq. 13-14: C and the m + n right-hand sides
    k_build_c<<<nb((int64_t)NC * NC, 256), 256, 0, s>>>(d, p, wu, Rt, C);
    k_build_rhs<<<nb((int64_t)nrhs * NC, 256), 256, 0, s>>>(d, p, m, n, wu + oRB, wu + oRL, Bm, X);
    ER_CUDA(cudaGetLastError());
    ER_CUDA(cudaEventRecord(ev[2], s));
    // K4: LU
    for (int j0 = 0; j0 < NC; j0 += kNB) {
        const int jb = std::min(kNB, NC - j0);
        k_lu_panel<<<1, 512, 0, s>>>(C, NC, j0, jb, piv, err);
        k_lu_swap<<<nb(NC, 256), 256, 0, s>>>(C, NC, j0, jb, piv);
        const int rest = NC - j0 - jb;
        if (rest > 0) {
            k_lu_trsm<<<nb(rest, 128), 128, 0, s>>>(C, NC, j0, jb);
            k_lu_gemm<<<dim3(nb(rest, 64), nb(rest, 64)), 256, 0, s>>>(C, NC, j0, jb);
        }
        ER_CUDA(cudaGetLastError());
    }
    ER_CUDA(cudaEventRecord(ev[3], s));
    // K5: m + n solves with the one factorisation
    k_lu_solve<<<nb(nrhs, 8), 256, 0, s>>>(C, NC, piv, X, nrhs);
    ER_CUDA(cudaGetLastError());
    ER_CUDA(cudaEventRecord(ev[4], s));
    // K6: pair dot products
    k_pair_dot<<<dim3(nb(n, 64), nb(m, 16)), 256, 0, s>>>(X, Bm, NC, d, p, m, n, R);
    ER_CUDA(cudaGetLastError());
    ER_CUDA(cudaEventRecord(ev[5], s));
    ER_CUDA(cudaStreamSynchronize(s));
    int herr = 0;
    ER_CUDA(cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost));
    if (stats) {
        float ms[5];
        for (int i = 0; i < 5; ++i) ER_CUDA(cudaEventElapsedTime(&ms[i], ev[i], ev[i + 1]));
        stats->n_system = NC;
        stats->wu_pairs = npairs_all;
        stats->ms_wu = ms[0];
        stats->ms_build = ms[1];
        stats->ms_lu = ms[2];
        stats->ms_solve = ms[3];
        stats->ms_dot = ms[4];
        stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    }
    if (herr) return fail(ER_ERR_INVALID_ARG, "the reduced system is singular");
    return ER_OK;
}

}  // namespace er

extern "C" er_status er_stack_pairs(const er_stack *st, const int32_t *bump_xy, int32_t m, const int32_t *load_xy,
                                    int32_t n, double *R, er_stack_stats *stats, void *stream) {
    return er::stack_pairs(st, bump_xy, m, load_xy, n, R, stats, (cudaStream_t)stream);
}
