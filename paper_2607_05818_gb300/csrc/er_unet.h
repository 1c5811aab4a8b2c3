// Internal interface between the U-Net host code (er_surrogate.cu) and its kernels
// (er_unet_kernels.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace er {

// What a convolution launch ran: kernel 1 = persistent TMA kernel, 2 = cp.async-staged
// kernel; bn = output channels per tile (N of the MMA); bk = input channels per K step.
struct UConvInfo {
    int kernel = 0, bn = 0, bk = 0;
};

// One 3x3 convolution launch (forward, or dgrad when y is null; see er_unet_kernels.cu).
struct UConv {
    const __nv_bfloat16 *x1 = nullptr, *x2 = nullptr;
    int c1 = 0, c2 = 0, x1_half = 0;
    const __nv_bfloat16 *w = nullptr;
    const float *bias = nullptr;
    int nb = 0, h = 0, w_ = 0, cout = 0, relu = 0;
    __nv_bfloat16 *y = nullptr;
    __nv_bfloat16 *g1 = nullptr, *g2 = nullptr;
    const __nv_bfloat16 *m1 = nullptr, *m2 = nullptr;
    int c1o = 0, m1_half = 0;
    int tile_n = 0;             // requested output channels per tile (0: automatic)
    UConvInfo *info = nullptr;  // filled with what ran (nullable)
};

// 3x3 convolution (forward, or dgrad when y is null) on tcgen05 with the accumulator in
// tensor memory; needs c1 and c1 + c2 multiples of 32 and cout a multiple of 32.  Inputs
// stored at full resolution and image sizes that tile into 128-pixel boxes take the
// persistent TMA kernel, the rest the cp.async-staged one.
cudaError_t unet_conv3x3(const UConv &c, cudaStream_t s);
cudaError_t unet_conv3x3_stage(const UConv &c, cudaStream_t s);
// nearest 2x upsampling [n][h/2][w/2][c] -> [n][h][w][c] (c a multiple of 8)
cudaError_t unet_upsample2x(const __nv_bfloat16 *x, __nv_bfloat16 *y, int nb, int h, int w, int c, cudaStream_t s);
// the same on warp-level mma.sync
cudaError_t unet_conv3x3_mma(const UConv &c, cudaStream_t s);
// copy the kernels' error word (non-zero: a bounded wait expired) to *host, clear it, sync
cudaError_t unet_take_error(int *host, cudaStream_t s);
// launches of the convolution kernels since the last reset: [0..5] persistent TMA kernel with
// 32-channel K steps and N tiles of 32, 64, 96, 128, 192, 256; [6..11] the same with 64-channel
// K steps; [12] cp.async-staged kernel; [13] weight gradient on mma.sync; [14] weight gradient
// on tcgen05
void unet_conv_counts(int64_t *out, int n, int reset);
// weight gradient dW += sum_p dY[p][o] X[p + tap][c] (FP32 atomics): on tcgen05 when the output
// channels are a multiple of 128, the input channels of 64 and the input is at full
// resolution, else on mma.sync
cudaError_t unet_wgrad3x3(const UConv &c, const __nv_bfloat16 *dy, float *dw, cudaStream_t s);
cudaError_t unet_maxpool(const __nv_bfloat16 *x, __nv_bfloat16 *y, int nb, int h, int w, int c, cudaStream_t s);
cudaError_t unet_maxpool_bwd(const __nv_bfloat16 *x, const __nv_bfloat16 *dy, __nv_bfloat16 *dx, int nb, int h, int w,
                             int c, cudaStream_t s);
cudaError_t unet_upsample_bwd(const __nv_bfloat16 *dup, __nv_bfloat16 *dx, int nb, int h, int w, int c, int add,
                              cudaStream_t s);
cudaError_t unet_add_grad(__nv_bfloat16 *dst, const __nv_bfloat16 *src, const __nv_bfloat16 *act, int64_t n,
                          cudaStream_t s);
cudaError_t unet_head_fwd(const __nv_bfloat16 *x, const float *w, const float *b, float *out, int64_t M, int c, int co,
                          cudaStream_t s);
cudaError_t unet_mse(const float *out, const float *target, const uint8_t *mask, float *dout, double *loss_sum,
                     int64_t n, float inv_count, cudaStream_t s);
cudaError_t unet_head_bwd(const __nv_bfloat16 *x, const float *w, const float *dout, __nv_bfloat16 *dx, float *dw,
                          float *db, int64_t M, int c, int co, cudaStream_t s);
cudaError_t unet_bias_grad(const __nv_bfloat16 *dy, float *db, int64_t M, int cout, cudaStream_t s);
cudaError_t unet_adam(float *w, float *m, float *v, const float *g, int64_t n, float lr, float b1, float b2, float eps,
                      int step, __nv_bfloat16 *wb, __nv_bfloat16 *wt, int cout, int cin, cudaStream_t s);
cudaError_t unet_to_bf16(const float *src, __nv_bfloat16 *dst, __nv_bfloat16 *dt, int64_t n, int cout, int cin,
                         cudaStream_t s);

}  // namespace er
