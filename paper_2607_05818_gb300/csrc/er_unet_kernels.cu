// Kernels of the BF16 U-Net surrogate (forward and backward), sm_103a.
//
// Tensors are NHWC (channels innermost).  3x3 convolutions are implicit GEMMs on the
// tensor cores with BF16 operands and FP32 accumulation.  Three kernels share the layout:
// k_conv_tc (persistent, warp-specialised: TMA boxes -> tcgen05.mma -> TMEM -> epilogue),
// used whenever 128 consecutive pixels form a box of the tensor and the input is stored at
// full resolution; k_conv3x3_tc (cp.async staging, tcgen05.mma, TMEM) for other image sizes
// and for inputs read with on-the-fly upsampling; and k_conv3x3 (mma.sync m16n8k16), kept as
// the legacy warp-level path:
//   forward  Y[m][co] = act(sum_k A[m][k] W[co][k] + b[co]),  m = (n, y, x), k = (ky, kx, ci)
//   dgrad    the same kernel on dY with W' [ci][ky][kx][co] = W[co][2-ky][2-kx][ci]
//   wgrad    dW[co][k] = sum_m dY[m][co] A[m][k]  (split over pixels, FP32 atomics)
// The input may be the channel concatenation of two tensors (a decoder's upsampled path and
// its skip connection), and the first of them may be stored at half resolution, read with
// nearest-neighbour upsampling on the fly, so neither the concatenation nor the upsampled
// tensor is ever written.  Operand tiles are staged with cp.async (zero fill outside the
// image) and fed to the tensor cores with ldmatrix from XOR-swizzled shared memory.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>
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
// 3x3 convolution on the 5th-generation tensor cores (tcgen05): the same implicit GEMM and
// epilogue as k_conv3x3, with the FP32 accumulator in tensor memory.
//
// CTA: 128 pixels (UMMA M = 128) x bn output channels (bn <= 256, a multiple of 16), 4 warps.
// K advances 32 input channels of one (ky, kx) per stage.  All threads stage A (im2col rows)
// and B (weight rows) with cp.async into 64-byte rows in the hardware's 64-byte swizzle
// (16-byte chunk c of row r at c ^ ((r >> 1) & 3), 1024-byte aligned tiles); thread 0
// issues two kind::f16 MMAs (K = 16 each) per stage and commits them to the stage's
// mbarrier, which the loaders wait on before refilling that stage.  The epilogue reads the
// accumulator rows with tcgen05.ld (warp w owns TMEM lanes 32w..32w+31 = pixels).
// Every wait is bounded in time; on expiry the kernel sets *err and exits cleanly.

constexpr int TBM = 128, TBK = 32, TSTAGES = 6;
__device__ int g_err;  // set by a bounded wait that expired; read and cleared by unet_take_error
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t *b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(saddr(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// wait for the phase of parity `parity` to complete; false after kWaitNs
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *b, uint32_t parity) {
    if (mbar_test(b, parity)) return true;
    const unsigned long long t0 = gtimer();
    while (!mbar_test(b, parity))
        if (gtimer() - t0 > kWaitNs) return false;
    return true;
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// shared-memory matrix descriptor: K-major, 64-byte swizzle, 64-byte rows, 8-row groups
// 512 bytes apart (stride byte offset), descriptor version 1, swizzle mode 4 (64B)
__device__ __forceinline__ uint64_t sdesc_k_sw64(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(512 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)4 << 61);
}
// instruction descriptor, kind::f16: D FP32, A and B BF16, both K-major, N >> 3, M >> 4
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}
__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__global__ void __launch_bounds__(128) k_conv3x3_tc(const ConvArgs a, int bn, int tcols, int *err) {
    extern __shared__ unsigned char tc_smem_raw[];
    __shared__ uint64_t bars[TSTAGES + 1];  // per stage: its MMAs done; [TSTAGES]: all MMAs done
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_s;
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    constexpr int ASZ = TBM * TBK * 2;  // 8 KiB
    const int bsz = bn * TBK * 2;
    unsigned char *As = smem;
    unsigned char *Bs = smem + TSTAGES * ASZ;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t M = (int64_t)a.nb * a.h * a.wd;
    const int64_t m0 = (int64_t)blockIdx.x * TBM;
    const int n0 = blockIdx.y * bn;
    const int cin = a.c1 + a.c2;
    const int cblk = cin / TBK;
    const int kblocks = 9 * cblk;

    if (tid == 0) {
        for (int s = 0; s <= TSTAGES; ++s) mbar_init(&bars[s], 1);
        abort_s = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_slot)),
                     "r"(tcols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    // this thread's four A rows (pixels r = tid/4 + 32 i) and its 16-byte chunk (tid % 4)
    const int ch = tid & 3;
    int py[4], px[4], pn[4];
    bool pv[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t m = m0 + (tid >> 2) + 32 * i;
        pv[i] = m < M;
        const int64_t mm = pv[i] ? m : 0;
        px[i] = (int)(mm % a.wd);
        py[i] = (int)((mm / a.wd) % a.h);
        pn[i] = (int)(mm / ((int64_t)a.wd * a.h));
    }

    auto load_stage = [&](int kb, int s) {
        const int kk = kb / cblk, ci0 = (kb % cblk) * TBK;
        const int ky = kk / 3 - 1, kx = kk % 3 - 1;
        unsigned char *at = As + s * ASZ;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int r = (tid >> 2) + 32 * i;
            const int ys = py[i] + ky, xs = px[i] + kx;
            const bool in = pv[i] && ys >= 0 && ys < a.h && xs >= 0 && xs < a.wd;
            const __nv_bfloat16 *src = a.x1;
            if (in) {
                if (ci0 < a.c1) {
                    src = a.x1_half
                              ? a.x1 + (((int64_t)pn[i] * (a.h >> 1) + (ys >> 1)) * (a.wd >> 1) + (xs >> 1)) * a.c1 + ci0 + ch * 8
                              : a.x1 + (((int64_t)pn[i] * a.h + ys) * a.wd + xs) * a.c1 + ci0 + ch * 8;
                } else {
                    src = a.x2 + (((int64_t)pn[i] * a.h + ys) * a.wd + xs) * a.c2 + (ci0 - a.c1) + ch * 8;
                }
            }
            cp_async16(at + r * 64 + ((ch ^ ((r >> 1) & 3)) << 4), src, in);
        }
        unsigned char *bt = Bs + s * bsz;
        for (int r = tid >> 2; r < bn; r += 32) {
            const int co = n0 + r;
            const bool in = co < a.cout;
            const __nv_bfloat16 *src = in ? a.w + ((int64_t)co * 9 + kk) * cin + ci0 + ch * 8 : a.w;
            cp_async16(bt + r * 64 + ((ch ^ ((r >> 1) & 3)) << 4), src, in);
        }
    };

    constexpr int PF = TSTAGES - 2;  // stages loaded ahead
    for (int s = 0; s < PF; ++s) {
        if (s < kblocks) load_stage(s, s);
        cp_async_commit();
    }
    const uint32_t idesc = idesc_bf16_f32(TBM, bn);
    bool ok = true;
    for (int kb = 0; kb < kblocks; ++kb) {
        const int s = kb % TSTAGES;
        cp_async_wait<PF - 1>();  // this thread's copies of stage kb have landed
        fence_proxy_async();      // make them visible to the tensor core's (async proxy) reads
        __syncthreads();
        if (abort_s) {
            ok = false;
            break;
        }
        if (tid == 0) {
            tc_fence_after();
            const uint32_t ab = saddr(As + s * ASZ), bb = saddr(Bs + s * bsz);
#pragma unroll
            for (int k16 = 0; k16 < TBK / 16; ++k16)
                tc_mma(tmem, sdesc_k_sw64(ab + k16 * 32), sdesc_k_sw64(bb + k16 * 32), idesc, (kb | k16) != 0);
            tc_commit(&bars[s]);
        }
        // refill the stage read by the MMAs of kb - 2 with stage kb + PF
        const int nk = kb + PF;
        if (nk < kblocks) {
            if (kb >= 2) {
                const int pk = kb - 2;
                if (!mbar_wait_bounded(&bars[pk % TSTAGES], (uint32_t)((pk / TSTAGES) & 1))) {
                    atomicExch(err, 1);
                    abort_s = 1;
                }
            }
            if (!abort_s) load_stage(nk, nk % TSTAGES);
        }
        cp_async_commit();
    }
    cp_async_wait<0>();
    if (tid == 0) tc_commit(&bars[TSTAGES]);  // arrives when every MMA issued above is done
    const bool done = mbar_wait_bounded(&bars[TSTAGES], 0);
    if (!done) atomicExch(err, 2);
    tc_fence_after();
    __syncthreads();
    ok = ok && done && !abort_s;

    if (ok) {
        const int row = warp * 32 + lane;
        const int64_t m = m0 + row;
        for (int c0 = 0; c0 < bn; c0 += 16) {
            float v[16];
            tc_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            const int co = n0 + c0;
            if (m >= M || co >= a.cout) continue;
            __align__(16) __nv_bfloat16 o[16];
            if (a.y) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    float x = v[j] + (a.bias ? a.bias[co + j] : 0.f);
                    if (a.relu) x = fmaxf(x, 0.f);
                    o[j] = __float2bfloat16(x);
                }
                uint4 *dst = reinterpret_cast<uint4 *>(a.y + m * a.cout + co);
                dst[0] = reinterpret_cast<const uint4 *>(o)[0];
                dst[1] = reinterpret_cast<const uint4 *>(o)[1];
            } else {
                const int x = (int)(m % a.wd), y = (int)((m / a.wd) % a.h), nn = (int)(m / ((int64_t)a.wd * a.h));
                const __nv_bfloat16 *mk;
                __nv_bfloat16 *dst;
                if (co < a.c1o) {
                    mk = a.m1_half ? a.m1 + (((int64_t)nn * (a.h >> 1) + (y >> 1)) * (a.wd >> 1) + (x >> 1)) * a.c1o + co
                                   : a.m1 + m * a.c1o + co;
                    dst = a.g1 + m * a.c1o + co;
                } else {
                    const int c2o = a.cout - a.c1o;
                    mk = a.m2 + m * c2o + (co - a.c1o);
                    dst = a.g2 + m * c2o + (co - a.c1o);
                }
                __align__(16) __nv_bfloat16 mv[16];
                reinterpret_cast<uint4 *>(mv)[0] = reinterpret_cast<const uint4 *>(mk)[0];
                reinterpret_cast<uint4 *>(mv)[1] = reinterpret_cast<const uint4 *>(mk)[1];
#pragma unroll
                for (int j = 0; j < 16; ++j) o[j] = __float2bfloat16(__bfloat162float(mv[j]) > 0.f ? v[j] : 0.f);
                reinterpret_cast<uint4 *>(dst)[0] = reinterpret_cast<const uint4 *>(o)[0];
                reinterpret_cast<uint4 *>(dst)[1] = reinterpret_cast<const uint4 *>(o)[1];
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols) : "memory");
    }
}

// ---------------------------------------------------------------------------------------
// 3x3 convolution, persistent and warp-specialised: TMA -> shared memory -> tcgen05.mma ->
// tensor memory -> epilogue.  One CTA per SM walks output tiles of 128 pixels x bn
// channels (tile t: pixel block t / tiles_n, channel block t % tiles_n).
//   warp 0 (one thread)  producer: per K step (BK channels of one tap (ky, kx)) one 4-D TMA
//                        box of the input [n][y][x][c] at (ci, x0+kx-1, y0+ky-1, n0) -- the
//                        tap's shifted pixel window, zero-filled outside the image -- and
//                        one 2-D box of the weights [cout][9 cin], into stage s of a ring
//   warp 1               allocates 2 x bnp TMEM columns; one thread issues BK/16 MMAs per
//                        stage (M = 128, N = bn, K = 16) into accumulator tile % 2 and
//                        commits them to the stage's "empty" barrier, and each finished
//                        tile to its accumulator's "full" barrier
//   warps 2-5            epilogue: tcgen05.ld of their TMEM lane quarter, bias + ReLU (or
//                        the dgrad masks), BF16 stores; then release the accumulator
// The pixel block (bimg images x by rows x bx columns = 128) is a box of the tensor, so the
// 128 accumulator rows are the consecutive pixels m0 .. m0+127.  Operands are K-major with
// the 64-byte (BK = 32) or 128-byte (BK = 64) swizzle, written so by the TMA.  Every wait
// is bounded in time; on expiry the kernel records *err, stops all roles and frees TMEM.

struct TcArgs {
    const float *bias;
    int relu;
    __nv_bfloat16 *y;
    __nv_bfloat16 *g1, *g2;
    const __nv_bfloat16 *m1, *m2;
    int c1o, m1_half;
    int nb, h, wd, cout;
    int c1, c2;                  // channels read through map 0 and map 1
    int bn, bnp;                 // output channels per tile; TMEM columns per accumulator
    int tiles_n, tiles;
    int stages;
    int *err;
};

__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(b)) : "memory");
}
__device__ __forceinline__ void tma_box4(void *dst, const CUtensorMap *m, uint64_t *bar, int c0, int c1, int c2, int c3) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(saddr(dst)),
        "l"(reinterpret_cast<uint64_t>(m)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(saddr(bar))
        : "memory");
}
__device__ __forceinline__ void tma_box2(void *dst, const CUtensorMap *m, uint64_t *bar, int c0, int c1) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            saddr(dst)),
        "l"(reinterpret_cast<uint64_t>(m)), "r"(c0), "r"(c1), "r"(saddr(bar))
        : "memory");
}
// bounded wait that also gives up when another role has aborted
__device__ __forceinline__ bool wait_or_abort(uint64_t *b, uint32_t parity, volatile int *abort_flag, int *err) {
    if (mbar_test(b, parity)) return true;
    const unsigned long long t0 = gtimer();
    while (!mbar_test(b, parity)) {
        if (*abort_flag) return false;
        if (gtimer() - t0 > kWaitNs) {
            atomicExch(err, 1);
            *abort_flag = 1;
            return false;
        }
    }
    return true;
}
// K-major operand descriptors: 64-byte swizzle (8-row groups 512 B apart, mode 4) or
// 128-byte swizzle (1024 B apart, mode 2)
template <int BK>
__device__ __forceinline__ uint64_t sdesc_k(uint32_t addr) {
    constexpr uint64_t sbo = BK == 64 ? 1024 : 512, mode = BK == 64 ? 2 : 4;
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((sbo >> 4) << 32) | ((uint64_t)1 << 46) |
           (mode << 61);
}

template <int BK>
__global__ void __launch_bounds__(192, 1)
    k_conv_tc(const __grid_constant__ CUtensorMap mx1, const __grid_constant__ CUtensorMap mx2,
              const __grid_constant__ CUtensorMap mw, const TcArgs a) {
    extern __shared__ unsigned char tcv_smem_raw[];
    constexpr int kMaxStages = 8;
    __shared__ uint64_t full[kMaxStages], empty[kMaxStages], tfull[2], tempty[2], mdone;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int abort_s;
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(tcv_smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    constexpr int ABYTES = TBM * BK * 2;
    const int bbytes = a.bn * BK * 2;
    const int stg = ABYTES + bbytes;
    const int S = a.stages;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cin = a.c1 + a.c2;
    const int cblk = cin / BK;
    const int kblocks = 9 * cblk;
    const int64_t HW = (int64_t)a.h * a.wd, M = (int64_t)a.nb * HW;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 4);
        }
        mbar_init(&mdone, 1);
        abort_s = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_slot)),
                     "r"(2 * a.bnp)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            int it = 0;
            int last[kMaxStages];
            for (int s = 0; s < kMaxStages; ++s) last[s] = -1;
            for (int tile = blockIdx.x; tile < a.tiles && !abort_s; tile += gridDim.x) {
                const int64_t m0 = (int64_t)(tile / a.tiles_n) * TBM;
                const int n0 = (tile % a.tiles_n) * a.bn;
                const int img = (int)(m0 / HW);
                const int y0 = (int)((m0 % HW) / a.wd), x0 = (int)(m0 % a.wd);
                for (int kb = 0; kb < kblocks; ++kb, ++it) {
                    const int s = it % S;
                    if (!wait_or_abort(&empty[s], (uint32_t)(((it / S) & 1) ^ 1), &abort_s, a.err)) break;
                    unsigned char *st = smem + s * stg;
                    mbar_expect_tx(&full[s], (uint32_t)stg);
                    const int kk = kb / cblk, ci0 = (kb % cblk) * BK;
                    const int xs = x0 + kk % 3 - 1, ys = y0 + kk / 3 - 1;
                    if (ci0 < a.c1) tma_box4(st, &mx1, &full[s], ci0, xs, ys, img);
                    else tma_box4(st, &mx2, &full[s], ci0 - a.c1, xs, ys, img);
                    tma_box2(st + ABYTES, &mw, &full[s], kk * cin + ci0, n0);
                    last[s] = it;
                }
            }
            // every load issued must land before the CTA exits
            for (int s = 0; s < S; ++s)
                if (last[s] >= 0) {
                    const unsigned long long t0 = gtimer();
                    while (!mbar_test(&full[s], (uint32_t)((last[s] / S) & 1)) && gtimer() - t0 < kWaitNs) {
                    }
                }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16_f32(TBM, a.bn);
            int it = 0, tc = 0;
            bool ok = true;
            for (int tile = blockIdx.x; tile < a.tiles && ok; tile += gridDim.x, ++tc) {
                const int buf = tc & 1;
                if (!wait_or_abort(&tempty[buf], (uint32_t)(((tc >> 1) & 1) ^ 1), &abort_s, a.err)) break;
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(buf * a.bnp);
                for (int kb = 0; kb < kblocks; ++kb, ++it) {
                    const int s = it % S;
                    if (!wait_or_abort(&full[s], (uint32_t)((it / S) & 1), &abort_s, a.err)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t ab = saddr(smem + s * stg), bb = ab + ABYTES;
#pragma unroll
                    for (int k16 = 0; k16 < BK / 16; ++k16)
                        tc_mma(d, sdesc_k<BK>(ab + k16 * 32), sdesc_k<BK>(bb + k16 * 32), idesc, (kb | k16) != 0);
                    tc_commit(&empty[s]);
                }
                if (ok) tc_commit(&tfull[buf]);
            }
            // all MMAs issued above complete before TMEM is released
            tc_commit(&mdone);
            const unsigned long long t0 = gtimer();
            while (!mbar_test(&mdone, 0) && gtimer() - t0 < kWaitNs) {
            }
        }
    } else {
        const int q = warp & 3;  // TMEM lane quarter this warp may read
        int tc = 0;
        for (int tile = blockIdx.x; tile < a.tiles; tile += gridDim.x, ++tc) {
            const int buf = tc & 1;
            if (!wait_or_abort(&tfull[buf], (uint32_t)((tc >> 1) & 1), &abort_s, a.err)) break;
            tc_fence_after();
            const int64_t m = (int64_t)(tile / a.tiles_n) * TBM + q * 32 + lane;
            const int n0 = (tile % a.tiles_n) * a.bn;
            const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * a.bnp);
            for (int c0 = 0; c0 < a.bn; c0 += 16) {
                float v[16];
                tc_ld16(tbase + (uint32_t)c0, v);
                const int co = n0 + c0;
                if (m >= M) continue;
                __align__(16) __nv_bfloat16 o[16];
                if (a.y) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        float x = v[j] + (a.bias ? a.bias[co + j] : 0.f);
                        if (a.relu) x = fmaxf(x, 0.f);
                        o[j] = __float2bfloat16(x);
                    }
                    uint4 *dst = reinterpret_cast<uint4 *>(a.y + m * a.cout + co);
                    dst[0] = reinterpret_cast<const uint4 *>(o)[0];
                    dst[1] = reinterpret_cast<const uint4 *>(o)[1];
                } else {
                    const int x = (int)(m % a.wd), y = (int)((m / a.wd) % a.h), nn = (int)(m / HW);
                    const __nv_bfloat16 *mk;
                    __nv_bfloat16 *dst;
                    if (co < a.c1o) {
                        mk = a.m1_half ? a.m1 + (((int64_t)nn * (a.h >> 1) + (y >> 1)) * (a.wd >> 1) + (x >> 1)) * a.c1o + co
                                       : a.m1 + m * a.c1o + co;
                        dst = a.g1 + m * a.c1o + co;
                    } else {
                        const int c2o = a.cout - a.c1o;
                        mk = a.m2 + m * c2o + (co - a.c1o);
                        dst = a.g2 + m * c2o + (co - a.c1o);
                    }
                    __align__(16) __nv_bfloat16 mv[16];
                    reinterpret_cast<uint4 *>(mv)[0] = reinterpret_cast<const uint4 *>(mk)[0];
                    reinterpret_cast<uint4 *>(mv)[1] = reinterpret_cast<const uint4 *>(mk)[1];
#pragma unroll
                    for (int j = 0; j < 16; ++j) o[j] = __float2bfloat16(__bfloat162float(mv[j]) > 0.f ? v[j] : 0.f);
                    reinterpret_cast<uint4 *>(dst)[0] = reinterpret_cast<const uint4 *>(o)[0];
                    reinterpret_cast<uint4 *>(dst)[1] = reinterpret_cast<const uint4 *>(o)[1];
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[buf]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * a.bnp) : "memory");
    }
}

// ---------------------------------------------------------------------------------------
// weight gradient on tcgen05: dW[o][tap][c] += sum over a pixel range of dY[p][o] X[p + tap][c],
// an MMA with M = 128 output channels, N = bn input channels of one tap and K = pixels.  Both
// operands are MN-major in memory (the channels of a pixel are contiguous), so the TMA lands
// 64-pixel boxes of 64 channels (128-byte rows, 128-byte swizzle) and the MMAs read them as
// MN-major operands: within a 1,024-byte swizzle atom 64 consecutive channels x 8 pixels,
// atoms of further channels 8 KB apart (leading byte offset), groups of 8 pixels 1 KB apart
// (stride byte offset).  The box of x is the dY box shifted by the tap, zero-filled outside the
// image, so the pixel rows of both operands correspond.  One tile per CTA:
//   warp 0 (one thread)  producer: per K step the M/64 boxes of dY and bn/64 boxes of x
//   warp 1               allocates bn TMEM columns; one thread issues 4 MMAs (K = 16) per stage
//   warps 2-5            epilogue: tcgen05.ld of their lane quarter, FP32 atomics into dW
// (split-K over pixel ranges: the CTAs of one output tile add their sums).  Every wait is
// bounded in time; on expiry the kernel records *err, stops every role and frees TMEM.
struct WgTcArgs {
    float *dw;
    int cin, c1, c2, cout, bn, tiles_c1, tiles_c, blocks_per_split, n_blocks;
    int nb, h, wd, bx, by, bimg;
    int stages;
    int vec4;  // dW rows start on 16-byte boundaries: the epilogue adds 4 columns per reduction
    int *err;
};

// dst[0..3] += v[0..3] as one 16-byte reduction in L2 (dst 16-byte aligned)
__device__ __forceinline__ void red_add_v4(float *dst, float a, float b, float c, float d) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(dst), "f"(a), "f"(b), "f"(c), "f"(d)
                 : "memory");
}

// MN-major operand descriptor, 128-byte swizzle: channel atoms (64 x 8) `lbo` bytes apart,
// groups of 8 pixels 1,024 bytes apart, descriptor version 1, swizzle mode 2 (128B)
__device__ __forceinline__ uint64_t sdesc_mn_sw128(uint32_t addr, uint32_t lbo) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

constexpr int WG_M = 128, WG_KP = 64;  // output channels per tile; pixels per K step

__global__ void __launch_bounds__(192, 1)
    k_wgrad_tc(const __grid_constant__ CUtensorMap mdy, const __grid_constant__ CUtensorMap mx1,
               const __grid_constant__ CUtensorMap mx2, const WgTcArgs a) {
    extern __shared__ unsigned char wg_smem_raw[];
    constexpr int kMaxStages = 8;
    __shared__ uint64_t full[kMaxStages], empty[kMaxStages], tfull, mdone;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int abort_s;
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(wg_smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    constexpr int BOX = WG_KP * 128;          // one 64-channel x 64-pixel box: 8 KB
    constexpr int ABYTES = (WG_M / 64) * BOX;  // 16 KB
    const int bbytes = (a.bn / 64) * BOX;
    const int stg = ABYTES + bbytes;
    const int S = a.stages;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // tile: output channel block, (tap, input channel block of x1 or of x2), pixel split; a
    // block's channels beyond its source (and output channels beyond cout) are zero-filled by
    // the TMA and not stored
    const int o0 = blockIdx.x * WG_M;
    const int kk = blockIdx.y / a.tiles_c, tci = blockIdx.y % a.tiles_c;
    const bool second = tci >= a.tiles_c1;
    const int cx = (second ? tci - a.tiles_c1 : tci) * a.bn;  // first channel within its source
    const int csrc = second ? a.c2 : a.c1;
    const int cbase = second ? a.c1 + cx : cx;                 // first channel within dW's cin
    const int b0 = blockIdx.z * a.blocks_per_split;
    const int b1 = min(b0 + a.blocks_per_split, a.n_blocks);
    const int nkb = b1 - b0;
    const int64_t HW = (int64_t)a.h * a.wd;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&tfull, 1);
        mbar_init(&mdone, 1);
        abort_s = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_slot)),
                     "r"(a.bn)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            int last[kMaxStages];
            for (int s = 0; s < kMaxStages; ++s) last[s] = -1;
            for (int it = 0; it < nkb && !abort_s; ++it) {
                const int s = it % S;
                if (!wait_or_abort(&empty[s], (uint32_t)(((it / S) & 1) ^ 1), &abort_s, a.err)) break;
                unsigned char *st = smem + s * stg;
                mbar_expect_tx(&full[s], (uint32_t)stg);
                const int64_t m0 = (int64_t)(b0 + it) * WG_KP;
                const int img = (int)(m0 / HW);
                const int y0 = (int)((m0 % HW) / a.wd), x0 = (int)(m0 % a.wd);
                for (int j = 0; j < WG_M / 64; ++j) tma_box4(st + j * BOX, &mdy, &full[s], o0 + 64 * j, x0, y0, img);
                const int xs = x0 + kk % 3 - 1, ys = y0 + kk / 3 - 1;
                for (int j = 0; j < a.bn / 64; ++j)
                    tma_box4(st + ABYTES + j * BOX, second ? &mx2 : &mx1, &full[s], cx + 64 * j, xs, ys, img);
                last[s] = it;
            }
            for (int s = 0; s < S; ++s)  // every load issued lands before the CTA exits
                if (last[s] >= 0) {
                    const unsigned long long t0 = gtimer();
                    while (!mbar_test(&full[s], (uint32_t)((last[s] / S) & 1)) && gtimer() - t0 < kWaitNs) {
                    }
                }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // kind::f16, D FP32, A and B BF16, both MN-major (transpose bits 15 and 16)
            const uint32_t idesc = idesc_bf16_f32(WG_M, a.bn) | (1u << 15) | (1u << 16);
            bool ok = true;
            for (int it = 0; it < nkb; ++it) {
                const int s = it % S;
                if (!wait_or_abort(&full[s], (uint32_t)((it / S) & 1), &abort_s, a.err)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t ab = saddr(smem + s * stg), bb = ab + ABYTES;
#pragma unroll
                for (int k16 = 0; k16 < WG_KP / 16; ++k16)  // 16 pixels = 2 groups of 8 rows = 2 KB
                    tc_mma(tmem, sdesc_mn_sw128(ab + k16 * 2048, BOX), sdesc_mn_sw128(bb + k16 * 2048, BOX), idesc,
                           (it | k16) != 0);
                tc_commit(&empty[s]);
            }
            if (ok) tc_commit(&tfull);
            tc_commit(&mdone);  // all MMAs issued above complete before TMEM is released
            const unsigned long long t0 = gtimer();
            while (!mbar_test(&mdone, 0) && gtimer() - t0 < kWaitNs) {
            }
        }
    } else if (nkb > 0) {
        const int q = warp & 3;  // TMEM lane quarter = output channels o0 + 32q ..
        if (wait_or_abort(&tfull, 0, &abort_s, a.err)) {
            tc_fence_after();
            const int o = o0 + q * 32 + lane;
            const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16);
            for (int cc = 0; cc < a.bn; cc += 16) {
                float v[16];
                tc_ld16(tbase + (uint32_t)cc, v);
                if (o < a.cout) {
                    float *dst = a.dw + ((int64_t)o * 9 + kk) * a.cin + cbase + cc;
                    if (a.vec4) {  // csrc % 32 == 0: a group of 4 columns is all in or all out
#pragma unroll
                        for (int j = 0; j < 16; j += 4)
                            if (cx + cc + j < csrc) red_add_v4(dst + j, v[j], v[j + 1], v[j + 2], v[j + 3]);
                    } else {
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            if (cx + cc + j < csrc) atomicAdd(dst + j, v[j]);
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.bn) : "memory");
    }
}

// nearest 2x upsampling [n][h/2][w/2][c] -> [n][h][w][c], 16 bytes per thread
__global__ void k_upsample2x(const __nv_bfloat16 *x, __nv_bfloat16 *y, int nb, int h, int w, int c) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // 8-channel chunk of y
    const int cc = c / 8;
    const int64_t total = (int64_t)nb * h * w * cc;
    if (i >= total) return;
    const int ch = (int)(i % cc);
    const int64_t p = i / cc;
    const int xx = (int)(p % w), yy = (int)((p / w) % h), n = (int)(p / ((int64_t)w * h));
    reinterpret_cast<uint4 *>(y)[i] =
        reinterpret_cast<const uint4 *>(x)[(((int64_t)n * (h >> 1) + (yy >> 1)) * (w >> 1) + (xx >> 1)) * cc + ch];
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

static int *err_word() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    static int *addr[64] = {};
    if (!addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, unet::g_err) == cudaSuccess) addr[dev] = static_cast<int *>(p);
    }
    return addr[dev];
}

cudaError_t unet_take_error(int *host, cudaStream_t s) {
    int *w = err_word();
    if (!w) return cudaErrorInvalidSymbol;
    cudaError_t e = cudaMemcpyAsync(host, w, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(w, 0, sizeof(int), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e;
}

// output-channel tile of the tensor-memory kernel: the widest of 256, 192, 128, 96, 64, 32
// that divides cout and still gives two CTAs per SM; else the narrowest that divides
static int tc_tile_n(int64_t mtiles, int cout) {
    const int cands[] = {256, 192, 128, 96, 64, 32};
    int pick = 0;
    for (int bn : cands) {
        if (bn > cout || cout % bn) continue;
        pick = bn;
        if (mtiles * (cout / bn) >= 2 * 152) break;
    }
    return pick;
}

// a requested N-tile width is honoured when it is one the kernels support and divides cout
static bool tile_n_ok(int bn, int cout) {
    return (bn == 32 || bn == 64 || bn == 96 || bn == 128 || bn == 192 || bn == 256) && bn <= cout && cout % bn == 0;
}

static std::atomic<long long> g_conv_counts[16];

static int width_slot(int bn) { return bn == 32 ? 0 : bn == 64 ? 1 : bn == 96 ? 2 : bn == 128 ? 3 : bn == 192 ? 4 : 5; }

void unet_conv_counts(int64_t *out, int n, int reset) {
    for (int i = 0; i < 16; ++i) {
        const long long v = reset ? g_conv_counts[i].exchange(0) : g_conv_counts[i].load();
        if (out && i < n) out[i] = (int64_t)v;
    }
}

static PFN_cuTensorMapEncodeTiled_v12000 encode_tiled() {
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

// BF16 tensor map, dims innermost first, byte strides of dims 1.., zero fill outside
static cudaError_t bf16_map(CUtensorMap *m, const void *base, int rank, const cuuint64_t *dims,
                            const cuuint64_t *strides, const cuuint32_t *box, CUtensorMapSwizzle swz) {
    auto fn = encode_tiled();
    if (!fn) return cudaErrorNotSupported;
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, (cuuint32_t)rank, const_cast<void *>(base), dims,
                          strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidResourceHandle;  // distinct from launch errors
}

static int sm_count() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) !=
                                                   cudaSuccess)
        return 0;
    return n;
}

// pixel box of 128 consecutive pixels: bimg images x by rows x bx columns
static bool tc_pixel_box(int h, int w, int &bx, int &by, int &bimg) {
    if (w >= 128) {
        if (w % 128) return false;
        bx = 128, by = 1, bimg = 1;
        return true;
    }
    if (128 % w) return false;
    bx = w;
    const int rows = 128 / w;
    if (h >= rows) {
        if (h % rows) return false;
        by = rows, bimg = 1;
        return true;
    }
    if (rows % h) return false;
    by = h, bimg = rows / h;
    return true;
}

template <int BK>
static cudaError_t launch_conv_tc(const UConv &c, int bx, int by, int bimg, cudaStream_t s) {
    using namespace unet;
    const int cin = c.c1 + c.c2;
    const int64_t M = (int64_t)c.nb * c.h * c.w_;
    const int64_t tiles_m = (M + TBM - 1) / TBM;
    const int nsm = sm_count();
    if (nsm <= 0) return cudaErrorUnknown;
    int bn = 0;
    for (int cand : {256, 192, 128, 96, 64, 32}) {
        if (cand > c.cout || c.cout % cand) continue;
        bn = cand;
        if (tiles_m * (c.cout / cand) >= nsm) break;
    }
    if (c.tile_n && tile_n_ok(c.tile_n, c.cout)) bn = c.tile_n;
    if (bn == 0) return cudaErrorInvalidValue;
    const int bnp = bn <= 32 ? 32 : bn <= 64 ? 64 : bn <= 128 ? 128 : 256;
    const int stg = TBM * BK * 2 + bn * BK * 2;
    const int stages = std::min(8, (200 * 1024) / stg);
    if (stages < 2) return cudaErrorInvalidValue;
    const int smem = stages * stg + 1024;
    // dynamic plus static shared memory must fit the opt-in limit; stages * stg <= 200 KiB
    constexpr int kMaxDyn = 200 * 1024 + 1024;
    static bool attr[2] = {false, false};
    if (!attr[BK == 64]) {
        cudaError_t e = cudaFuncSetAttribute(k_conv_tc<BK>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDyn);
        if (e != cudaSuccess) return e;
        attr[BK == 64] = true;
    }
    const CUtensorMapSwizzle swz = BK == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
    CUtensorMap mx1, mx2, mw;
    const cuuint32_t xbox[4] = {(cuuint32_t)BK, (cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bimg};
    {
        const cuuint64_t dims[4] = {(cuuint64_t)c.c1, (cuuint64_t)c.w_, (cuuint64_t)c.h, (cuuint64_t)c.nb};
        const cuuint64_t str[3] = {(cuuint64_t)c.c1 * 2, (cuuint64_t)c.c1 * 2 * c.w_, (cuuint64_t)c.c1 * 2 * c.w_ * c.h};
        cudaError_t e = bf16_map(&mx1, c.x1, 4, dims, str, xbox, swz);
        if (e != cudaSuccess) return e;
    }
    if (c.c2 > 0) {
        const cuuint64_t dims[4] = {(cuuint64_t)c.c2, (cuuint64_t)c.w_, (cuuint64_t)c.h, (cuuint64_t)c.nb};
        const cuuint64_t str[3] = {(cuuint64_t)c.c2 * 2, (cuuint64_t)c.c2 * 2 * c.w_, (cuuint64_t)c.c2 * 2 * c.w_ * c.h};
        cudaError_t e = bf16_map(&mx2, c.x2, 4, dims, str, xbox, swz);
        if (e != cudaSuccess) return e;
    } else {
        mx2 = mx1;
    }
    {
        const cuuint64_t dims[2] = {(cuuint64_t)9 * cin, (cuuint64_t)c.cout};
        const cuuint64_t str[1] = {(cuuint64_t)9 * cin * 2};
        const cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)bn};
        cudaError_t e = bf16_map(&mw, c.w, 2, dims, str, box, swz);
        if (e != cudaSuccess) return e;
    }
    TcArgs a{};
    a.bias = c.bias; a.relu = c.relu; a.y = c.y;
    a.g1 = c.g1; a.g2 = c.g2; a.m1 = c.m1; a.m2 = c.m2; a.c1o = c.c1o; a.m1_half = c.m1_half;
    a.nb = c.nb; a.h = c.h; a.wd = c.w_; a.cout = c.cout;
    a.c1 = c.c1; a.c2 = c.c2; a.bn = bn; a.bnp = bnp;
    a.tiles_n = c.cout / bn;
    const int64_t tiles = tiles_m * a.tiles_n;
    if (tiles > 0x7fffffff) return cudaErrorInvalidValue;
    a.tiles = (int)tiles;
    a.stages = stages;
    a.err = err_word();
    if (!a.err) return cudaErrorInvalidSymbol;
    const unsigned grid = (unsigned)std::min<int64_t>(tiles, nsm);
    k_conv_tc<BK><<<grid, 192, smem, s>>>(mx1, mx2, mw, a);
    const cudaError_t le = cudaGetLastError();
    if (le == cudaSuccess) {
        g_conv_counts[(BK == 64 ? 6 : 0) + width_slot(bn)].fetch_add(1);
        if (c.info) *c.info = UConvInfo{1, bn, BK};
    }
    return le;
}

cudaError_t unet_upsample2x(const __nv_bfloat16 *x, __nv_bfloat16 *y, int nb, int h, int w, int c, cudaStream_t s) {
    if (c % 8) return cudaErrorInvalidValue;
    const int64_t n = (int64_t)nb * h * w * (c / 8);
    unet::k_upsample2x<<<nblk(n, 256), 256, 0, s>>>(x, y, nb, h, w, c);
    return cudaGetLastError();
}

cudaError_t unet_conv3x3(const UConv &c, cudaStream_t s) {
    using namespace unet;
    const int cin = c.c1 + c.c2;
    int bx, by, bimg;
    if (!c.x1_half && cin % 32 == 0 && c.c1 % 32 == 0 && c.cout % 32 == 0 && tc_pixel_box(c.h, c.w_, bx, by, bimg)) {
        if (c.c1 % 64 == 0 && c.c2 % 64 == 0) return launch_conv_tc<64>(c, bx, by, bimg, s);
        return launch_conv_tc<32>(c, bx, by, bimg, s);
    }
    return unet_conv3x3_stage(c, s);
}

// the same convolution with cp.async staging and a synchronous pipeline (any image size,
// upsampled input read on the fly)
cudaError_t unet_conv3x3_stage(const UConv &c, cudaStream_t s) {
    using namespace unet;
    const int cin = c.c1 + c.c2;
    const int64_t M = (int64_t)c.nb * c.h * c.w_;
    const int64_t mtiles = (M + TBM - 1) / TBM;
    const int bn = c.tile_n && tile_n_ok(c.tile_n, c.cout) ? c.tile_n : tc_tile_n(mtiles, c.cout);
    if (cin % TBK || c.c1 % TBK || bn == 0) return cudaErrorInvalidValue;
    int *err = err_word();
    if (!err) return cudaErrorInvalidSymbol;
    static bool tc_attr = false;
    constexpr int kMaxSmem = TSTAGES * (TBM * TBK * 2 + 256 * TBK * 2) + 1024;
    if (!tc_attr) {
        cudaError_t e = cudaFuncSetAttribute(k_conv3x3_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
        if (e != cudaSuccess) return e;
        tc_attr = true;
    }
    ConvArgs a{};
    a.x1 = c.x1; a.x2 = c.x2; a.c1 = c.c1; a.c2 = c.c2; a.x1_half = c.x1_half;
    a.w = c.w; a.bias = c.bias; a.nb = c.nb; a.h = c.h; a.wd = c.w_; a.cout = c.cout; a.relu = c.relu; a.y = c.y;
    a.g1 = c.g1; a.g2 = c.g2; a.m1 = c.m1; a.m2 = c.m2; a.c1o = c.c1o; a.m1_half = c.m1_half;
    const int tcols = bn <= 32 ? 32 : bn <= 64 ? 64 : bn <= 128 ? 128 : 256;
    const int smem = TSTAGES * (TBM * TBK * 2 + bn * TBK * 2) + 1024;
    k_conv3x3_tc<<<dim3((unsigned)mtiles, (unsigned)(c.cout / bn)), 128, smem, s>>>(a, bn, tcols, err);
    const cudaError_t le = cudaGetLastError();
    if (le == cudaSuccess) {
        g_conv_counts[12].fetch_add(1);
        if (c.info) *c.info = UConvInfo{2, bn, TBK};
    }
    return le;
}

cudaError_t unet_conv3x3_mma(const UConv &c, cudaStream_t s) {
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

// pixel box of 64 consecutive pixels: bimg images x by rows x bx columns
static bool wg_pixel_box(int h, int w, int &bx, int &by, int &bimg) {
    using unet::WG_KP;
    if (w >= WG_KP) {
        if (w % WG_KP) return false;
        bx = WG_KP, by = 1, bimg = 1;
        return true;
    }
    if (WG_KP % w) return false;
    bx = w;
    const int rows = WG_KP / w;
    if (h >= rows) {
        if (h % rows) return false;
        by = rows, bimg = 1;
        return true;
    }
    if (rows % h) return false;
    by = h, bimg = rows / h;
    return true;
}

// the tcgen05 weight gradient; cudaErrorNotSupported for shapes it does not take (channel
// counts not multiples of 32, an input read at half resolution, pixel counts that do not tile
// into 64-pixel boxes).  Channel blocks of 64 whose channels run past their tensor (layers of
// 32 or 96 channels) are zero-filled and their extra rows and columns are not stored.
static cudaError_t unet_wgrad3x3_tc(const UConv &c, const __nv_bfloat16 *dy, float *dw, cudaStream_t s) {
    using namespace unet;
    const int cin = c.c1 + c.c2;
    int bx, by, bimg;
    if (c.x1_half || c.cout % 32 || c.c1 % 32 || c.c2 % 32 || c.c1 == 0 || !wg_pixel_box(c.h, c.w_, bx, by, bimg))
        return cudaErrorNotSupported;
    int bn = 64;
    for (int cand : {256, 128})
        if (c.c1 % cand == 0 && c.c2 % cand == 0) {
            bn = cand;
            break;
        }
    const int stg = (WG_M / 64 + bn / 64) * WG_KP * 128;
    const int stages = std::min(8, (200 * 1024) / stg);
    constexpr int kMaxDyn = 200 * 1024 + 1024;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDyn);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    CUtensorMap mdy, mx1, mx2;
    const cuuint32_t box[4] = {64, (cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bimg};
    {
        const cuuint64_t dims[4] = {(cuuint64_t)c.cout, (cuuint64_t)c.w_, (cuuint64_t)c.h, (cuuint64_t)c.nb};
        const cuuint64_t str[3] = {(cuuint64_t)c.cout * 2, (cuuint64_t)c.cout * 2 * c.w_,
                                   (cuuint64_t)c.cout * 2 * c.w_ * c.h};
        if (bf16_map(&mdy, dy, 4, dims, str, box, CU_TENSOR_MAP_SWIZZLE_128B) != cudaSuccess)
            return cudaErrorNotSupported;
    }
    {
        const cuuint64_t dims[4] = {(cuuint64_t)c.c1, (cuuint64_t)c.w_, (cuuint64_t)c.h, (cuuint64_t)c.nb};
        const cuuint64_t str[3] = {(cuuint64_t)c.c1 * 2, (cuuint64_t)c.c1 * 2 * c.w_, (cuuint64_t)c.c1 * 2 * c.w_ * c.h};
        if (bf16_map(&mx1, c.x1, 4, dims, str, box, CU_TENSOR_MAP_SWIZZLE_128B) != cudaSuccess)
            return cudaErrorNotSupported;
    }
    if (c.c2 > 0) {
        const cuuint64_t dims[4] = {(cuuint64_t)c.c2, (cuuint64_t)c.w_, (cuuint64_t)c.h, (cuuint64_t)c.nb};
        const cuuint64_t str[3] = {(cuuint64_t)c.c2 * 2, (cuuint64_t)c.c2 * 2 * c.w_, (cuuint64_t)c.c2 * 2 * c.w_ * c.h};
        if (bf16_map(&mx2, c.x2, 4, dims, str, box, CU_TENSOR_MAP_SWIZZLE_128B) != cudaSuccess)
            return cudaErrorNotSupported;
    } else {
        mx2 = mx1;
    }
    WgTcArgs a{};
    a.dw = dw; a.cin = cin; a.c1 = c.c1; a.c2 = c.c2; a.cout = c.cout; a.bn = bn;
    a.tiles_c1 = (c.c1 + bn - 1) / bn;
    a.tiles_c = a.tiles_c1 + (c.c2 + bn - 1) / bn;
    a.nb = c.nb; a.h = c.h; a.wd = c.w_; a.bx = bx; a.by = by; a.bimg = bimg;
    a.stages = stages;
    a.vec4 = (reinterpret_cast<uintptr_t>(dw) % 16 == 0) ? 1 : 0;  // cin % 32 == 0 keeps every row aligned
    a.err = err_word();
    if (!a.err) return cudaErrorInvalidSymbol;
    const int64_t M = (int64_t)c.nb * c.h * c.w_;
    a.n_blocks = (int)((M + WG_KP - 1) / WG_KP);
    const int tiles_o = (c.cout + WG_M - 1) / WG_M;
    const int tiles = tiles_o * 9 * a.tiles_c;
    const int nsm = sm_count();
    if (nsm <= 0) return cudaErrorUnknown;
    // split the pixels so that the grid covers every SM about twice
    int splits = std::max(1, std::min(a.n_blocks, (2 * nsm + tiles - 1) / tiles));
    a.blocks_per_split = (a.n_blocks + splits - 1) / splits;
    splits = (a.n_blocks + a.blocks_per_split - 1) / a.blocks_per_split;
    k_wgrad_tc<<<dim3((unsigned)tiles_o, (unsigned)(9 * a.tiles_c), (unsigned)splits), 192,
                 stages * stg + 1024, s>>>(mdy, mx1, mx2, a);
    const cudaError_t le = cudaGetLastError();
    if (le == cudaSuccess) g_conv_counts[14].fetch_add(1);
    return le;
}

cudaError_t unet_wgrad3x3(const UConv &c, const __nv_bfloat16 *dy, float *dw, cudaStream_t s) {
    {
        const cudaError_t e = unet_wgrad3x3_tc(c, dy, dw, s);
        if (e != cudaErrorNotSupported) return e;
    }
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
    const cudaError_t le = cudaGetLastError();
    if (le == cudaSuccess) g_conv_counts[13].fetch_add(1);
    return le;
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
