// Kernels of the BF16 U-Net surrogate (forward and backward), sm_103a.
//
// Tensors are NHWC (channels innermost).  3x3 convolutions are implicit GEMMs on the
// tensor cores (mma.sync m16n8k16, BF16 operands, FP32 accumulation):
//   forward  Y[m][co] = act(sum_k A[m][k] W[co][k] + b[co]),  m = (n, y, x), k = (ky, kx, ci)
//   dgrad    the same kernel on dY with W' [ci][ky][kx][co] = W[co][2-ky][2-kx][ci]
//   wgrad    dW[co][k] = sum_m dY[m][co] A[m][k]  (split over pixels, FP32 atomics)
// The input may be the channel concatenation of two tensors (a decoder's upsampled path and
// its skip connection), and the first of them may be stored at half resolution, read with
// nearest-neighbour upsampling on the fly, so neither the concatenation nor the upsampled
// tensor is ever written.  Operand tiles are staged with cp.async (zero fill outside the
// image) and fed to the tensor cores with ldmatrix from XOR-swizzled shared memory.
#include <cuda_bf16.h>

#include <cstdint>

#include "er_internal.h"
#include "er_unet.h"

namespace er {

namespace unet {

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp_async16(void *dst, const void *src, bool valid) {
    const int n = valid ? 16 : 0;  // n = 0 copies nothing and fills 16 zero bytes
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(saddr(dst)), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void *p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(saddr(p)));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], const void *p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(saddr(p)));
}
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// ---------------------------------------------------------------------------------------
// 3x3 convolution, implicit GEMM: CTA tile 128 pixels x 64 output channels x 32 of K,
// 8 warps as 4 (M) x 2 (N), each 32 x 32, three cp.async stages.
// Shared tiles have 64-byte rows (32 BF16); the four 16-byte chunks of row r are stored
// at chunk ^ ((r >> 1) & 3), which makes every 8-row ldmatrix conflict-free.

constexpr int CBM = 128, CBN = 64, CBK = 32, CSTAGES = 3;

__device__ __forceinline__ int swz64(int r, int c) { return r * 32 + ((c ^ ((r >> 1) & 3)) << 3); }

struct ConvArgs {
    const __nv_bfloat16 *x1, *x2;  // inputs: channels [0, c1) from x1, [c1, c1+c2) from x2
    int c1, c2, x1_half;           // x1_half: x1 is stored at (H/2, W/2), nearest upsampling
    const __nv_bfloat16 *w;        // [cout][3][3][c1+c2]
    const float *bias;             // [cout] or null
    int nb, h, wd, cout;
    int relu;                      // forward: ReLU in the epilogue
    __nv_bfloat16 *y;              // forward: output [n][h][w][cout]
    // dgrad mode: y is null; the result (a gradient w.r.t. the forward input) is written to
    // g1 (channels [0, c1o)) at full resolution and g2 (channels [c1o, cout)), multiplied by
    // the ReLU mask of the forward input tensors m1 (half resolution if m1_half) and m2
    __nv_bfloat16 *g1, *g2;
    const __nv_bfloat16 *m1, *m2;
    int c1o, m1_half;
};

__global__ void __launch_bounds__(256) k_conv3x3(const ConvArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    __nv_bfloat16 *As = reinterpret_cast<__nv_bfloat16 *>(smem);                       // [S][128][32]
    __nv_bfloat16 *Bs = reinterpret_cast<__nv_bfloat16 *>(smem + CSTAGES * CBM * CBK * 2);  // [S][64][32]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp & 3, wn = warp >> 2;
    const int64_t M = (int64_t)a.nb * a.h * a.wd;
    const int64_t m0 = (int64_t)blockIdx.x * CBM;
    const int n0 = blockIdx.y * CBN;
    const int cin = a.c1 + a.c2;
    const int kblocks = 9 * (cin / CBK);

    // this thread's two A rows (pixels) and one B row (output channel)
    const int ar = tid >> 2, ac = tid & 3;
    int py[2], px[2], pn[2];
    bool pv[2];
    for (int i = 0; i < 2; ++i) {
        const int64_t m = m0 + ar + i * 64;
        pv[i] = m < M;
        const int64_t mm = pv[i] ? m : 0;
        px[i] = (int)(mm % a.wd);
        py[i] = (int)((mm / a.wd) % a.h);
        pn[i] = (int)(mm / ((int64_t)a.wd * a.h));
    }
    const int bco = n0 + (tid >> 2);

    auto load_stage = [&](int kb, int s) {
        const int kk = kb / (cin / CBK);          // 0..8 = ky*3 + kx
        const int ci0 = (kb % (cin / CBK)) * CBK;  // channel block
        const int ky = kk / 3 - 1, kx = kk % 3 - 1;
        for (int i = 0; i < 2; ++i) {
            const int r = ar + i * 64;
            const int ys = py[i] + ky, xs = px[i] + kx;
            const bool in = pv[i] && ys >= 0 && ys < a.h && xs >= 0 && xs < a.wd;
            const __nv_bfloat16 *src = a.x1;
            if (in) {
                if (ci0 < a.c1) {
                    if (a.x1_half) {
                        const int hh = a.h >> 1, ww = a.wd >> 1;
                        src = a.x1 + (((int64_t)pn[i] * hh + (ys >> 1)) * ww + (xs >> 1)) * a.c1 + ci0 + ac * 8;
                    } else {
                        src = a.x1 + (((int64_t)pn[i] * a.h + ys) * a.wd + xs) * a.c1 + ci0 + ac * 8;
                    }
                } else {
                    src = a.x2 + (((int64_t)pn[i] * a.h + ys) * a.wd + xs) * a.c2 + (ci0 - a.c1) + ac * 8;
                }
            }
            cp_async16(As + s * CBM * CBK + swz64(r, ac), src, in);
        }
        {
            const bool in = bco < a.cout;
            const __nv_bfloat16 *src = in ? a.w + ((int64_t)bco * 9 + kk) * cin + ci0 + ac * 8 : a.w;
            cp_async16(Bs + s * CBN * CBK + swz64(tid >> 2, ac), src, in);
        }
    };

    float acc[2][4][4];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 4; ++j)
            for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;

    for (int s = 0; s < CSTAGES - 1; ++s) {
        if (s < kblocks) load_stage(s, s);
        cp_async_commit();
    }
    for (int kb = 0; kb < kblocks; ++kb) {
        cp_async_wait<CSTAGES - 2>();
        __syncthreads();
        const int nk = kb + CSTAGES - 1;
        if (nk < kblocks) load_stage(nk, nk % CSTAGES);
        cp_async_commit();
        const __nv_bfloat16 *At = As + (kb % CSTAGES) * CBM * CBK;
        const __nv_bfloat16 *Bt = Bs + (kb % CSTAGES) * CBN * CBK;
#pragma unroll
        for (int k16 = 0; k16 < CBK / 16; ++k16) {
            uint32_t af[2][4], bfr[2][4];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int r = wm * 32 + i * 16 + (lane & 7) + ((lane >> 3) & 1) * 8;
                const int c = k16 * 2 + (lane >> 4);
                ldsm_x4(af[i], At + swz64(r, c));
            }
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int r = wn * 32 + j * 16 + (lane & 7) + (lane >> 4) * 8;
                const int c = k16 * 2 + ((lane >> 3) & 1);
                ldsm_x4(bfr[j], Bt + swz64(r, c));
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    mma_bf16(acc[i][j], af[i], bfr[j >> 1][(j & 1) * 2], bfr[j >> 1][(j & 1) * 2 + 1]);
        }
    }
    cp_async_wait<0>();

    // epilogue
    const int g = lane >> 2, t4 = lane & 3;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int64_t m = m0 + wm * 32 + i * 16 + g + half * 8;
            if (m >= M) continue;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int co = n0 + wn * 32 + j * 8 + t4 * 2;
                if (co >= a.cout) continue;
                float v0 = acc[i][j][half * 2], v1 = acc[i][j][half * 2 + 1];
                if (a.y) {
                    if (a.bias) {
                        v0 += a.bias[co];
                        v1 += a.bias[co + 1];
                    }
                    if (a.relu) {
                        v0 = fmaxf(v0, 0.f);
                        v1 = fmaxf(v1, 0.f);
                    }
                    *reinterpret_cast<__nv_bfloat162 *>(a.y + m * a.cout + co) = __floats2bfloat162_rn(v0, v1);
                } else {
                    // gradient w.r.t. the forward input, masked by that input's ReLU
                    const int x = (int)(m % a.wd), y = (int)((m / a.wd) % a.h), nn = (int)(m / ((int64_t)a.wd * a.h));
                    if (co < a.c1o) {
                        const __nv_bfloat16 *mk =
                            a.m1_half ? a.m1 + (((int64_t)nn * (a.h >> 1) + (y >> 1)) * (a.wd >> 1) + (x >> 1)) * a.c1o + co
                                      : a.m1 + m * a.c1o + co;
                        const __nv_bfloat162 mv = *reinterpret_cast<const __nv_bfloat162 *>(mk);
                        if (!(__bfloat162float(mv.x) > 0.f)) v0 = 0.f;
                        if (!(__bfloat162float(mv.y) > 0.f)) v1 = 0.f;
                        *reinterpret_cast<__nv_bfloat162 *>(a.g1 + m * a.c1o + co) = __floats2bfloat162_rn(v0, v1);
                    } else {
                        const int c2o = a.cout - a.c1o, cc = co - a.c1o;
                        const __nv_bfloat162 mv = *reinterpret_cast<const __nv_bfloat162 *>(a.m2 + m * c2o + cc);
                        if (!(__bfloat162float(mv.x) > 0.f)) v0 = 0.f;
                        if (!(__bfloat162float(mv.y) > 0.f)) v1 = 0.f;
                        *reinterpret_cast<__nv_bfloat162 *>(a.g2 + m * c2o + cc) = __floats2bfloat162_rn(v0, v1);
                    }
                }
            }
        }
}

// ---------------------------------------------------------------------------------------
// weight gradient: dW[co][k] += sum over a pixel range of dY[m][co] * A[m][k]; CTA tile
// 64 output channels x 64 input channels of one (ky, kx), 32 pixels per step, 4 warps
// (2 x 2, each 32 x 32); tiles are stored with pixels as rows (128-byte rows, chunks at
// chunk ^ (row & 7)) and read with ldmatrix.trans.

constexpr int WBM = 64, WBN = 64, WBK = 32, WSTAGES = 3;
__device__ __forceinline__ int swz128(int r, int c) { return r * 64 + ((c ^ (r & 7)) << 3); }

struct WgradArgs {
    const __nv_bfloat16 *dy;       // [m][cout]
    const __nv_bfloat16 *x1, *x2;  // forward input (as in ConvArgs)
    int c1, c2, x1_half;
    int nb, h, wd, cout;
    float *dw;                     // [cout][3][3][cin], FP32, accumulated
    int64_t pix_per_split;
};

__global__ void __launch_bounds__(128) k_wgrad3x3(const WgradArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    __nv_bfloat16 *As = reinterpret_cast<__nv_bfloat16 *>(smem);                        // [S][32][64] dY
    __nv_bfloat16 *Bs = reinterpret_cast<__nv_bfloat16 *>(smem + WSTAGES * WBK * WBM * 2);  // [S][32][64] X
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp & 1, wn = warp >> 1;
    const int cin = a.c1 + a.c2;
    const int co0 = blockIdx.x * WBM;
    const int kk = blockIdx.y % 9, cib = (blockIdx.y / 9) * WBN;
    const int ky = kk / 3 - 1, kx = kk % 3 - 1;
    const int64_t M = (int64_t)a.nb * a.h * a.wd;
    const int64_t p0 = (int64_t)blockIdx.z * a.pix_per_split;
    const int64_t p1 = p0 + a.pix_per_split < M ? p0 + a.pix_per_split : M;
    const int nsteps = (int)((p1 - p0 + WBK - 1) / WBK);

    auto load_stage = [&](int st, int s) {
        // 32 pixel rows x 8 chunks for each tile: 256 chunks each, 2 per thread per tile
        for (int q = 0; q < 2; ++q) {
            const int idx = tid + q * 128;
            const int r = idx >> 3, c = idx & 7;
            const int64_t m = p0 + (int64_t)st * WBK + r;
            const bool mv = m < p1;
            {  // dY
                const int co = co0 + c * 8;
                const bool in = mv && co < a.cout;
                cp_async16(As + s * WBK * WBM + swz128(r, c), in ? a.dy + m * a.cout + co : a.dy, in);
            }
            {  // shifted input
                const int ci = cib + c * 8;
                bool in = mv && ci < cin;
                const __nv_bfloat16 *src = a.x1;
                if (in) {
                    const int64_t mm = m;
                    const int x = (int)(mm % a.wd), y = (int)((mm / a.wd) % a.h), nn = (int)(mm / ((int64_t)a.wd * a.h));
                    const int ys = y + ky, xs = x + kx;
                    in = ys >= 0 && ys < a.h && xs >= 0 && xs < a.wd;
                    if (in) {
                        if (ci < a.c1) {
                            src = a.x1_half ? a.x1 + (((int64_t)nn * (a.h >> 1) + (ys >> 1)) * (a.wd >> 1) + (xs >> 1)) * a.c1 + ci
                                            : a.x1 + (((int64_t)nn * a.h + ys) * a.wd + xs) * a.c1 + ci;
                        } else {
                            src = a.x2 + (((int64_t)nn * a.h + ys) * a.wd + xs) * a.c2 + (ci - a.c1);
                        }
                    }
                }
                cp_async16(Bs + s * WBK * WBN + swz128(r, c), src, in);
            }
        }
    };

    float acc[2][4][4];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 4; ++j)
            for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;
    for (int s = 0; s < WSTAGES - 1; ++s) {
        if (s < nsteps) load_stage(s, s);
        cp_async_commit();
    }
    for (int st = 0; st < nsteps; ++st) {
        cp_async_wait<WSTAGES - 2>();
        __syncthreads();
        const int ns = st + WSTAGES - 1;
        if (ns < nsteps) load_stage(ns, ns % WSTAGES);
        cp_async_commit();
        const __nv_bfloat16 *At = As + (st % WSTAGES) * WBK * WBM;
        const __nv_bfloat16 *Bt = Bs + (st % WSTAGES) * WBK * WBN;
#pragma unroll
        for (int k16 = 0; k16 < WBK / 16; ++k16) {
            uint32_t af[2][4], bfr[2][4];
#pragma unroll
            for (int i = 0; i < 2; ++i) {  // A = dY^T: stored [pixel][co]
                const int mat = lane >> 3;
                const int r = k16 * 16 + (lane & 7) + (mat >> 1) * 8;
                const int c = (wm * 32 + i * 16) / 8 + (mat & 1);
                ldsm_x4_t(af[i], At + swz128(r, c));
            }
#pragma unroll
            for (int j = 0; j < 2; ++j) {  // B = X: stored [pixel][ci]
                const int mat = lane >> 3;
                const int r = k16 * 16 + (lane & 7) + (mat & 1) * 8;
                const int c = (wn * 32 + j * 16) / 8 + (mat >> 1);
                ldsm_x4_t(bfr[j], Bt + swz128(r, c));
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    mma_bf16(acc[i][j], af[i], bfr[j >> 1][(j & 1) * 2], bfr[j >> 1][(j & 1) * 2 + 1]);
        }
    }
    cp_async_wait<0>();
    const int g = lane >> 2, t4 = lane & 3;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int co = co0 + wm * 32 + i * 16 + g + half * 8;
            if (co >= a.cout) continue;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int ci = cib + wn * 32 + j * 8 + t4 * 2;
                if (ci >= cin) continue;
                float *dst = a.dw + ((int64_t)co * 9 + kk) * cin + ci;
                atomicAdd(dst, acc[i][j][half * 2]);
                atomicAdd(dst + 1, acc[i][j][half * 2 + 1]);
            }
        }
}

// ---------------------------------------------------------------------------------------
// small kernels

// 2x2 max pooling (NHWC), and its backward (the gradient goes to the first maximum)
__global__ void k_maxpool(const __nv_bfloat16 *x, __nv_bfloat16 *y, int nb, int h, int w, int c) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)nb * (h / 2) * (w / 2) * c;
    if (i >= total) return;
    const int ch = (int)(i % c);
    const int64_t p = i / c;
    const int xo = (int)(p % (w / 2)), yo = (int)((p / (w / 2)) % (h / 2)), n = (int)(p / ((int64_t)(w / 2) * (h / 2)));
    float m = -3.0e38f;
    for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx)
            m = fmaxf(m, __bfloat162float(x[(((int64_t)n * h + 2 * yo + dy) * w + 2 * xo + dx) * c + ch]));
    y[i] = __float2bfloat16(m);
}

__global__ void k_maxpool_bwd(const __nv_bfloat16 *x, const __nv_bfloat16 *dy, __nv_bfloat16 *dx, int nb, int h,
                              int w, int c) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)nb * (h / 2) * (w / 2) * c;
    if (i >= total) return;
    const int ch = (int)(i % c);
    const int64_t p = i / c;
    const int xo = (int)(p % (w / 2)), yo = (int)((p / (w / 2)) % (h / 2)), n = (int)(p / ((int64_t)(w / 2) * (h / 2)));
    float m = -3.0e38f;
    int arg = 0;
    for (int q = 0; q < 4; ++q) {
        const float v = __bfloat162float(x[(((int64_t)n * h + 2 * yo + q / 2) * w + 2 * xo + q % 2) * c + ch]);
        if (v > m) {
            m = v;
            arg = q;
        }
    }
    for (int q = 0; q < 4; ++q)
        dx[(((int64_t)n * h + 2 * yo + q / 2) * w + 2 * xo + q % 2) * c + ch] = q == arg ? dy[i] : __float2bfloat16(0.f);
}

// accumulate a full-resolution gradient into its half-resolution source (nearest upsampling
// backward): dx[n][y][x][c] += sum of the 2x2 block; dx is also a pooled layer's output
// gradient, so the sum adds into what is there
__global__ void k_upsample_bwd(const __nv_bfloat16 *dup, __nv_bfloat16 *dx, int nb, int h, int w, int c, int add) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)nb * (h / 2) * (w / 2) * c;
    if (i >= total) return;
    const int ch = (int)(i % c);
    const int64_t p = i / c;
    const int xo = (int)(p % (w / 2)), yo = (int)((p / (w / 2)) % (h / 2)), n = (int)(p / ((int64_t)(w / 2) * (h / 2)));
    float s = add ? __bfloat162float(dx[i]) : 0.f;
    for (int q = 0; q < 4; ++q) s += __bfloat162float(dup[(((int64_t)n * h + 2 * yo + q / 2) * w + 2 * xo + q % 2) * c + ch]);
    dx[i] = __float2bfloat16(s);
}

// elementwise dst += src (BF16), masked by the ReLU of `act` when act is given
__global__ void k_add_grad(__nv_bfloat16 *dst, const __nv_bfloat16 *src, const __nv_bfloat16 *act, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float v = __bfloat162float(dst[i]) + __bfloat162float(src[i]);
    if (act && !(__bfloat162float(act[i]) > 0.f)) v = 0.f;
    dst[i] = __float2bfloat16(v);
}

// 1x1 head: out[m][t] = sum_c x[m][c] w[t][c] + b[t] (FP32 out)
__global__ void k_head_fwd(const __nv_bfloat16 *x, const float *w, const float *b, float *out, int64_t M, int c, int co) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M * co) return;
    const int64_t m = i / co;
    const int t = (int)(i % co);
    float s = b[t];
    for (int ch = 0; ch < c; ++ch) s = fmaf(__bfloat162float(x[m * c + ch]), w[t * c + ch], s);
    out[i] = s;
}

// loss: masked MSE over out vs target; writes d(loss)/d(out) and accumulates the loss sum
__global__ void k_mse(const float *out, const float *target, const uint8_t *mask, float *dout, double *loss_sum,
                      int64_t n, float inv_count) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double l = 0.0;
    if (i < n) {
        const bool on = !mask || mask[i];
        const float d = on ? out[i] - target[i] : 0.f;
        dout[i] = 2.f * d * inv_count;
        l = (double)d * d;
    }
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0 && l != 0.0) atomicAdd(loss_sum, l);
}

// head backward: dx[m][c] = relu'(x) * sum_t dout[m][t] w[t][c]; dw[t][c] += sum_m dout x; db[t] += sum_m dout
__global__ void k_head_bwd_x(const __nv_bfloat16 *x, const float *w, const float *dout, __nv_bfloat16 *dx, int64_t M,
                             int c, int co) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M * c) return;
    const int64_t m = i / c;
    const int ch = (int)(i % c);
    float s = 0.f;
    for (int t = 0; t < co; ++t) s = fmaf(dout[m * co + t], w[t * c + ch], s);
    if (!(__bfloat162float(x[i]) > 0.f)) s = 0.f;
    dx[i] = __float2bfloat16(s);
}

__global__ void k_head_bwd_w(const __nv_bfloat16 *x, const float *dout, float *dw, float *db, int64_t M, int c, int co) {
    // one block per (t, ch) pair plus one per t for the bias: grid = co * (c + 1)
    const int t = blockIdx.x / (c + 1), ch = blockIdx.x % (c + 1);
    float s = 0.f;
    for (int64_t m = threadIdx.x; m < M; m += blockDim.x)
        s += dout[m * co + t] * (ch < c ? __bfloat162float(x[m * c + ch]) : 1.f);
    __shared__ float red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (ch < c) dw[t * c + ch] += red[0];
        else db[t] += red[0];
    }
}

// per-channel bias gradient of a conv: db[co] += sum_m dy[m][co] (dy already masked)
__global__ void k_bias_grad(const __nv_bfloat16 *dy, float *db, int64_t M, int cout) {
    const int co = blockIdx.x;
    float s = 0.f;
    for (int64_t m = threadIdx.x; m < M; m += blockDim.x) s += __bfloat162float(dy[m * cout + co]);
    __shared__ float red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) db[co] += red[0];
}

// Adam (Kingma and Ba 2015) on FP32 master weights; refreshes the BF16 copy used by the
// forward pass and, for 3x3 convolutions, the flipped/transposed copy used by dgrad
__global__ void k_adam(float *w, float *m, float *v, const float *g, int64_t n, float lr, float b1, float b2, float eps,
                       float bc1, float bc2, __nv_bfloat16 *wb, __nv_bfloat16 *wt, int cout, int cin) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    w[i] = wi;
    if (wb) wb[i] = __float2bfloat16(wi);
    if (wt) {  // i = ((co * 9) + kk) * cin + ci  ->  wt[((ci * 9) + (8 - kk)) * cout + co]
        const int ci = (int)(i % cin);
        const int64_t q = i / cin;
        const int kk = (int)(q % 9), co = (int)(q / 9);
        wt[((int64_t)ci * 9 + (8 - kk)) * cout + co] = __float2bfloat16(wi);
    }
}

__global__ void k_to_bf16(const float *src, __nv_bfloat16 *dst, __nv_bfloat16 *dt, int64_t n, int cout, int cin) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    dst[i] = __float2bfloat16(src[i]);
    if (dt) {
        const int ci = (int)(i % cin);
        const int64_t q = i / cin;
        const int kk = (int)(q % 9), co = (int)(q / 9);
        dt[((int64_t)ci * 9 + (8 - kk)) * cout + co] = __float2bfloat16(src[i]);
    }
}

}  // namespace unet

// ---------------------------------------------------------------------------------------
// launchers

static unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

cudaError_t unet_conv3x3(const UConv &c, cudaStream_t s) {
    using namespace unet;
    static bool attr = false;
    const int smem = CSTAGES * (CBM + CBN) * CBK * 2;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_conv3x3, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    ConvArgs a{};
    a.x1 = c.x1; a.x2 = c.x2; a.c1 = c.c1; a.c2 = c.c2; a.x1_half = c.x1_half;
    a.w = c.w; a.bias = c.bias; a.nb = c.nb; a.h = c.h; a.wd = c.w_; a.cout = c.cout; a.relu = c.relu; a.y = c.y;
    a.g1 = c.g1; a.g2 = c.g2; a.m1 = c.m1; a.m2 = c.m2; a.c1o = c.c1o; a.m1_half = c.m1_half;
    const int64_t M = (int64_t)c.nb * c.h * c.w_;
    dim3 grid(nblk(M, CBM), (unsigned)((c.cout + CBN - 1) / CBN));
    k_conv3x3<<<grid, 256, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t unet_wgrad3x3(const UConv &c, const __nv_bfloat16 *dy, float *dw, cudaStream_t s) {
    using namespace unet;
    static bool attr = false;
    const int smem = WSTAGES * WBK * (WBM + WBN) * 2;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_wgrad3x3, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    WgradArgs a{};
    a.dy = dy; a.x1 = c.x1; a.x2 = c.x2; a.c1 = c.c1; a.c2 = c.c2; a.x1_half = c.x1_half;
    a.nb = c.nb; a.h = c.h; a.wd = c.w_; a.cout = c.cout; a.dw = dw;
    const int cin = c.c1 + c.c2;
    const int64_t M = (int64_t)c.nb * c.h * c.w_;
    const int gx = (c.cout + WBM - 1) / WBM, gy = 9 * ((cin + WBN - 1) / WBN);
    // split the pixels so the grid covers the GPU a few times over
    int64_t splits = (int64_t)(4 * 152) / ((int64_t)gx * gy) + 1;
    splits = std::min<int64_t>(splits, (M + WBK - 1) / WBK);
    a.pix_per_split = ((M + splits - 1) / splits + WBK - 1) / WBK * WBK;
    splits = (M + a.pix_per_split - 1) / a.pix_per_split;
    k_wgrad3x3<<<dim3(gx, gy, (unsigned)splits), 128, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t unet_maxpool(const __nv_bfloat16 *x, __nv_bfloat16 *y, int nb, int h, int w, int c, cudaStream_t s) {
    const int64_t n = (int64_t)nb * (h / 2) * (w / 2) * c;
    unet::k_maxpool<<<nblk(n, 256), 256, 0, s>>>(x, y, nb, h, w, c);
    return cudaGetLastError();
}
cudaError_t unet_maxpool_bwd(const __nv_bfloat16 *x, const __nv_bfloat16 *dy, __nv_bfloat16 *dx, int nb, int h, int w,
                             int c, cudaStream_t s) {
    const int64_t n = (int64_t)nb * (h / 2) * (w / 2) * c;
    unet::k_maxpool_bwd<<<nblk(n, 256), 256, 0, s>>>(x, dy, dx, nb, h, w, c);
    return cudaGetLastError();
}
cudaError_t unet_upsample_bwd(const __nv_bfloat16 *dup, __nv_bfloat16 *dx, int nb, int h, int w, int c, int add,
                              cudaStream_t s) {
    const int64_t n = (int64_t)nb * (h / 2) * (w / 2) * c;
    unet::k_upsample_bwd<<<nblk(n, 256), 256, 0, s>>>(dup, dx, nb, h, w, c, add);
    return cudaGetLastError();
}
cudaError_t unet_add_grad(__nv_bfloat16 *dst, const __nv_bfloat16 *src, const __nv_bfloat16 *act, int64_t n,
                          cudaStream_t s) {
    unet::k_add_grad<<<nblk(n, 256), 256, 0, s>>>(dst, src, act, n);
    return cudaGetLastError();
}
cudaError_t unet_head_fwd(const __nv_bfloat16 *x, const float *w, const float *b, float *out, int64_t M, int c, int co,
                          cudaStream_t s) {
    unet::k_head_fwd<<<nblk(M * co, 256), 256, 0, s>>>(x, w, b, out, M, c, co);
    return cudaGetLastError();
}
cudaError_t unet_mse(const float *out, const float *target, const uint8_t *mask, float *dout, double *loss_sum,
                     int64_t n, float inv_count, cudaStream_t s) {
    unet::k_mse<<<nblk(n, 256), 256, 0, s>>>(out, target, mask, dout, loss_sum, n, inv_count);
    return cudaGetLastError();
}
cudaError_t unet_head_bwd(const __nv_bfloat16 *x, const float *w, const float *dout, __nv_bfloat16 *dx, float *dw,
                          float *db, int64_t M, int c, int co, cudaStream_t s) {
    unet::k_head_bwd_x<<<nblk(M * c, 256), 256, 0, s>>>(x, w, dout, dx, M, c, co);
    unet::k_head_bwd_w<<<(unsigned)(co * (c + 1)), 256, 0, s>>>(x, dout, dw, db, M, c, co);
    return cudaGetLastError();
}
cudaError_t unet_bias_grad(const __nv_bfloat16 *dy, float *db, int64_t M, int cout, cudaStream_t s) {
    unet::k_bias_grad<<<(unsigned)cout, 256, 0, s>>>(dy, db, M, cout);
    return cudaGetLastError();
}
cudaError_t unet_adam(float *w, float *m, float *v, const float *g, int64_t n, float lr, float b1, float b2, float eps,
                      int step, __nv_bfloat16 *wb, __nv_bfloat16 *wt, int cout, int cin, cudaStream_t s) {
    const float bc1 = 1.f - powf(b1, (float)step), bc2 = 1.f - powf(b2, (float)step);
    unet::k_adam<<<nblk(n, 256), 256, 0, s>>>(w, m, v, g, n, lr, b1, b2, eps, bc1, bc2, wb, wt, cout, cin);
    return cudaGetLastError();
}
cudaError_t unet_to_bf16(const float *src, __nv_bfloat16 *dst, __nv_bfloat16 *dt, int64_t n, int cout, int cin,
                         cudaStream_t s) {
    unet::k_to_bf16<<<nblk(n, 256), 256, 0, s>>>(src, dst, dt, n, cout, cin);
    return cudaGetLastError();
}

}  // namespace er
