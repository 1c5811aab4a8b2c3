// BF16 U-Net surrogate of the R map: host side (layer graph, memory, forward, backward,
// Adam) behind er_surrogate_*.
//
// Input: per-node maps [B][H][W][in_ch] (BF16, NHWC), e.g. 4 tiers x {x-conductance,
// y-conductance, TSV mask, pad mask} zero-padded to in_ch = 32.  Output: log R per node
// and tier [B][H][W][out_ch] (FP32).  Architecture (levels L, base channels C):
//   encoder level l (l = 0..L-1): two 3x3 conv + ReLU with C*2^l channels, 2x2 max pool
//   between levels; decoder level l (l = L-2..0): nearest 2x upsampling of the level below
//   (fused into the convolution's loads), channel concatenation with the encoder's level-l
//   output (also fused), two 3x3 conv + ReLU; a 1x1 FP32 head.
// Training: masked mean-squared error on log R, Adam on FP32 master weights with BF16
// copies for the tensor-core kernels.
#include <cmath>
#include <cstring>
#include <memory>
#include <vector>

#include "er_internal.h"
#include "er_unet.h"

namespace er {

namespace {

struct Conv {
    int cin = 0, cout = 0;
    float *w = nullptr, *b = nullptr;             // FP32 master
    __nv_bfloat16 *wb = nullptr, *wt = nullptr;    // BF16 copy, flipped/transposed copy (dgrad)
    float *mw = nullptr, *vw = nullptr, *mb = nullptr, *vb = nullptr;
    float *gw = nullptr, *gb = nullptr;
    int64_t nw() const { return (int64_t)cout * 9 * cin; }
};

struct Act {
    __nv_bfloat16 *a = nullptr, *g = nullptr;  // value and gradient, [B][h][w][c]
    int h = 0, w = 0, c = 0;
};

template <typename T>
cudaError_t dalloc(T **p, size_t n) {
    return cudaMalloc((void **)p, std::max<size_t>(n, 1) * sizeof(T));
}

uint64_t mix64(uint64_t z) {  // SplitMix64 output function, for the initial weights
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

}  // namespace

}  // namespace er

struct er_surrogate {
    er_unet_shape shape{};
    int device = 0;
    int L = 0;
    std::vector<er::Conv> enc, dec;  // enc[2l + i], dec[2l + i]
    float *hw = nullptr, *hb = nullptr, *hmw = nullptr, *hvw = nullptr, *hmb = nullptr, *hvb = nullptr;
    float *hgw = nullptr, *hgb = nullptr;
    int batch = 0;                       // activations allocated for this batch size
    std::vector<er::Act> ea, eb, pool, da, db;  // per level
    __nv_bfloat16 *scratch = nullptr;    // full-resolution gradient scratch
    float *out = nullptr, *dout = nullptr;
    double *loss = nullptr;
    int step = 0;
    int tile_n = 0;                      // requested N-tile width of the convolutions (0: automatic)
    std::vector<void *> owned;           // activation buffers
};

namespace er {

static er_status sur_fail_cuda(cudaError_t e, const char *what) { return cuda_fail(e, what); }

// synchronises `cs` and reports a kernel whose bounded wait expired
static er_status check_kernels(cudaStream_t cs) {
    int word = 0;
    cudaError_t e = unet_take_error(&word, cs);
    if (e != cudaSuccess) return cuda_fail(e, "unet_take_error");
    if (word) return fail(ER_ERR_TIMEOUT, "a U-Net kernel's bounded wait expired");
    return ER_OK;
}

#define SUR_CUDA(call)                                                  \
    do {                                                                \
        cudaError_t _e = (call);                                        \
        if (_e != cudaSuccess) return ::er::sur_fail_cuda(_e, #call);   \
    } while (0)

static er_status init_conv(Conv &c, int cin, int cout, uint64_t seed, std::vector<void *> &owned) {
    c.cin = cin;
    c.cout = cout;
    const int64_t n = c.nw();
    SUR_CUDA(dalloc(&c.w, n)); SUR_CUDA(dalloc(&c.b, cout)); SUR_CUDA(dalloc(&c.wb, n)); SUR_CUDA(dalloc(&c.wt, n));
    SUR_CUDA(dalloc(&c.mw, n)); SUR_CUDA(dalloc(&c.vw, n)); SUR_CUDA(dalloc(&c.mb, cout)); SUR_CUDA(dalloc(&c.vb, cout));
    SUR_CUDA(dalloc(&c.gw, n)); SUR_CUDA(dalloc(&c.gb, cout));
    for (void *p : {(void *)c.w, (void *)c.b, (void *)c.wb, (void *)c.wt, (void *)c.mw, (void *)c.vw, (void *)c.mb,
                    (void *)c.vb, (void *)c.gw, (void *)c.gb})
        owned.push_back(p);
    // He-normal initial weights (Box-Muller on a counter-based stream), zero biases
    std::vector<float> hw((size_t)n);
    const double sd = std::sqrt(2.0 / (9.0 * cin));
    for (int64_t i = 0; i < n; i += 2) {
        const double u1 = ((mix64(seed ^ (uint64_t)i) >> 11) + 1.0) * (1.0 / 9007199254740993.0);
        const double u2 = (mix64(seed ^ (uint64_t)(i + 1) ^ 0xABCDEFULL) >> 11) * (1.0 / 9007199254740992.0);
        const double r = std::sqrt(-2.0 * std::log(u1));
        hw[i] = (float)(sd * r * std::cos(6.283185307179586 * u2));
        if (i + 1 < n) hw[i + 1] = (float)(sd * r * std::sin(6.283185307179586 * u2));
    }
    SUR_CUDA(cudaMemcpy(c.w, hw.data(), n * 4, cudaMemcpyHostToDevice));
    SUR_CUDA(cudaMemset(c.b, 0, cout * 4));
    SUR_CUDA(cudaMemset(c.mw, 0, n * 4)); SUR_CUDA(cudaMemset(c.vw, 0, n * 4));
    SUR_CUDA(cudaMemset(c.mb, 0, cout * 4)); SUR_CUDA(cudaMemset(c.vb, 0, cout * 4));
    SUR_CUDA(unet_to_bf16(c.w, c.wb, c.wt, n, cout, cin, nullptr));
    return ER_OK;
}

static int lvl_ch(const er_surrogate *s, int l) { return s->shape.base << l; }

static er_status ensure_batch(er_surrogate *s, int B) {
    if (s->batch >= B) return ER_OK;
    for (void *p : s->owned) cudaFree(p);
    s->owned.clear();
    const int L = s->L, H = s->shape.H, W = s->shape.W;
    s->ea.assign(L, {}); s->eb.assign(L, {}); s->pool.assign(L, {}); s->da.assign(L, {}); s->db.assign(L, {});
    auto mk = [&](Act &a, int h, int w, int c) -> er_status {
        a.h = h; a.w = w; a.c = c;
        const size_t n = (size_t)B * h * w * c;
        SUR_CUDA(dalloc(&a.a, n));
        SUR_CUDA(dalloc(&a.g, n));
        s->owned.push_back(a.a);
        s->owned.push_back(a.g);
        return ER_OK;
    };
    size_t scratch = 0;
    for (int l = 0; l < L; ++l) {
        const int h = H >> l, w = W >> l, c = lvl_ch(s, l);
        er_status st = mk(s->ea[l], h, w, c);
        if (st == ER_OK) st = mk(s->eb[l], h, w, c);
        if (st == ER_OK && l + 1 < L) st = mk(s->pool[l], h / 2, w / 2, c);
        if (st == ER_OK && l + 1 < L) st = mk(s->da[l], h, w, c);
        if (st == ER_OK && l + 1 < L) st = mk(s->db[l], h, w, c);
        if (st != ER_OK) return st;
        scratch = std::max(scratch, (size_t)B * h * w * std::max(c, l + 1 < L ? lvl_ch(s, l + 1) : c));
    }
    SUR_CUDA(dalloc(&s->scratch, scratch));
    s->owned.push_back(s->scratch);
    SUR_CUDA(dalloc(&s->out, (size_t)B * H * W * s->shape.out_ch));
    SUR_CUDA(dalloc(&s->dout, (size_t)B * H * W * s->shape.out_ch));
    s->owned.push_back(s->out);
    s->owned.push_back(s->dout);
    s->batch = B;
    return ER_OK;
}

// the N-tile width requested by the surrogate whose pass runs on this thread (forward and
// backward set it from er_surrogate::tile_n)
static thread_local int g_tile_n = 0;

static UConv fwd_conv(const Conv &c, const __nv_bfloat16 *x1, int c1, int x1_half, const __nv_bfloat16 *x2, int c2,
                      int B, int h, int w, __nv_bfloat16 *y) {
    UConv u;
    u.tile_n = g_tile_n;
    u.x1 = x1; u.c1 = c1; u.x1_half = x1_half; u.x2 = x2; u.c2 = c2;
    u.w = c.wb; u.bias = c.b; u.nb = B; u.h = h; u.w_ = w; u.cout = c.cout; u.relu = 1; u.y = y;
    return u;
}

static er_status forward(er_surrogate *s, const __nv_bfloat16 *maps, int B, cudaStream_t st) {
    const int L = s->L;
    g_tile_n = s->tile_n;
    for (int l = 0; l < L; ++l) {
        const int h = s->ea[l].h, w = s->ea[l].w, c = s->ea[l].c;
        const __nv_bfloat16 *in = l == 0 ? maps : s->pool[l - 1].a;
        const int cin = l == 0 ? s->shape.in_ch : lvl_ch(s, l - 1);
        SUR_CUDA(unet_conv3x3(fwd_conv(s->enc[2 * l], in, cin, 0, nullptr, 0, B, h, w, s->ea[l].a), st));
        SUR_CUDA(unet_conv3x3(fwd_conv(s->enc[2 * l + 1], s->ea[l].a, c, 0, nullptr, 0, B, h, w, s->eb[l].a), st));
        if (l + 1 < L) SUR_CUDA(unet_maxpool(s->eb[l].a, s->pool[l].a, B, h, w, c, st));
    }
    for (int l = L - 2; l >= 0; --l) {
        const int h = s->da[l].h, w = s->da[l].w, c = s->da[l].c;
        const __nv_bfloat16 *below = l == L - 2 ? s->eb[L - 1].a : s->db[l + 1].a;
        // the upsampled path is written once at full resolution so that the convolution's
        // operand boxes can be fetched by the TMA
        SUR_CUDA(unet_upsample2x(below, s->scratch, B, h, w, lvl_ch(s, l + 1), st));
        SUR_CUDA(unet_conv3x3(fwd_conv(s->dec[2 * l], s->scratch, lvl_ch(s, l + 1), 0, s->eb[l].a, c, B, h, w, s->da[l].a), st));
        SUR_CUDA(unet_conv3x3(fwd_conv(s->dec[2 * l + 1], s->da[l].a, c, 0, nullptr, 0, B, h, w, s->db[l].a), st));
    }
    const int64_t M = (int64_t)B * s->shape.H * s->shape.W;
    SUR_CUDA(unet_head_fwd(s->db[0].a, s->hw, s->hb, s->out, M, s->shape.base, s->shape.out_ch, st));
    return ER_OK;
}

// dgrad of conv c whose forward input was (x1 [c1, half?] | x2 [c2]); the gradient w.r.t.
// x1 goes to g1 (full resolution) and w.r.t. x2 to g2, each masked by its input's ReLU
static UConv dgrad_conv(const Conv &c, const __nv_bfloat16 *dy, int B, int h, int w, __nv_bfloat16 *g1,
                        const __nv_bfloat16 *m1, int c1, int m1_half, __nv_bfloat16 *g2, const __nv_bfloat16 *m2) {
    UConv u;
    u.tile_n = g_tile_n;
    u.x1 = dy; u.c1 = c.cout; u.w = c.wt; u.nb = B; u.h = h; u.w_ = w; u.cout = c.cin;
    u.g1 = g1; u.m1 = m1; u.c1o = c1; u.m1_half = m1_half; u.g2 = g2; u.m2 = m2;
    return u;
}

static UConv wgrad_in(const __nv_bfloat16 *x1, int c1, int x1_half, const __nv_bfloat16 *x2, int c2, int B, int h,
                      int w, int cout) {
    UConv u;
    u.x1 = x1; u.c1 = c1; u.x1_half = x1_half; u.x2 = x2; u.c2 = c2; u.nb = B; u.h = h; u.w_ = w; u.cout = cout;
    return u;
}

static er_status backward(er_surrogate *s, const __nv_bfloat16 *maps, int B, cudaStream_t st) {
    const int L = s->L, H = s->shape.H, W = s->shape.W;
    g_tile_n = s->tile_n;
    const int64_t M0 = (int64_t)B * H * W;
    // zero the weight gradients
    for (auto *v : {&s->enc, &s->dec})
        for (Conv &c : *v) {
            if (!c.w) continue;
            SUR_CUDA(cudaMemsetAsync(c.gw, 0, c.nw() * 4, st));
            SUR_CUDA(cudaMemsetAsync(c.gb, 0, c.cout * 4, st));
        }
    SUR_CUDA(cudaMemsetAsync(s->hgw, 0, (size_t)s->shape.out_ch * s->shape.base * 4, st));
    SUR_CUDA(cudaMemsetAsync(s->hgb, 0, (size_t)s->shape.out_ch * 4, st));
    // head
    SUR_CUDA(unet_head_bwd(s->db[0].a, s->hw, s->dout, s->db[0].g, s->hgw, s->hgb, M0, s->shape.base, s->shape.out_ch, st));
    // decoder, level 0 upwards
    for (int l = 0; l <= L - 2; ++l) {
        const int h = s->da[l].h, w = s->da[l].w, c = s->da[l].c, cb = lvl_ch(s, l + 1);
        const int64_t M = (int64_t)B * h * w;
        Conv &c2 = s->dec[2 * l + 1], &c1 = s->dec[2 * l];
        // second conv: input da[l]
        SUR_CUDA(unet_wgrad3x3(wgrad_in(s->da[l].a, c, 0, nullptr, 0, B, h, w, c2.cout), s->db[l].g, c2.gw, st));
        SUR_CUDA(unet_bias_grad(s->db[l].g, c2.gb, M, c2.cout, st));
        SUR_CUDA(unet_conv3x3(dgrad_conv(c2, s->db[l].g, B, h, w, s->da[l].g, s->da[l].a, c, 0, nullptr, nullptr), st));
        // first conv: input (up(below) | eb[l])
        const __nv_bfloat16 *below = l == L - 2 ? s->eb[L - 1].a : s->db[l + 1].a;
        __nv_bfloat16 *below_g = l == L - 2 ? s->eb[L - 1].g : s->db[l + 1].g;
        // the upsampled path at full resolution (the scratch is free until the data gradient
        // below), so that the weight gradient's operand boxes can be fetched by the TMA
        SUR_CUDA(unet_upsample2x(below, s->scratch, B, h, w, cb, st));
        SUR_CUDA(unet_wgrad3x3(wgrad_in(s->scratch, cb, 0, s->eb[l].a, c, B, h, w, c1.cout), s->da[l].g, c1.gw, st));
        SUR_CUDA(unet_bias_grad(s->da[l].g, c1.gb, M, c1.cout, st));
        SUR_CUDA(unet_conv3x3(dgrad_conv(c1, s->da[l].g, B, h, w, s->scratch, below, cb, 1, s->eb[l].g, s->eb[l].a), st));
        SUR_CUDA(unet_upsample_bwd(s->scratch, below_g, B, h, w, cb, 0, st));
    }
    // encoder, bottom level downwards; eb[l].g holds the skip gradient (and, at the bottom,
    // the decoder's), to which the pooled path's gradient is added
    for (int l = L - 1; l >= 0; --l) {
        const int h = s->ea[l].h, w = s->ea[l].w, c = s->ea[l].c;
        const int64_t M = (int64_t)B * h * w;
        Conv &c2 = s->enc[2 * l + 1], &c1 = s->enc[2 * l];
        if (l + 1 < L) {
            // pool[l].g (from level l+1's first conv) back through the max pool, added to eb[l].g
            SUR_CUDA(unet_maxpool_bwd(s->eb[l].a, s->pool[l].g, s->scratch, B, h, w, c, st));
            SUR_CUDA(unet_add_grad(s->eb[l].g, s->scratch, s->eb[l].a, M * c, st));
        }
        SUR_CUDA(unet_wgrad3x3(wgrad_in(s->ea[l].a, c, 0, nullptr, 0, B, h, w, c2.cout), s->eb[l].g, c2.gw, st));
        SUR_CUDA(unet_bias_grad(s->eb[l].g, c2.gb, M, c2.cout, st));
        SUR_CUDA(unet_conv3x3(dgrad_conv(c2, s->eb[l].g, B, h, w, s->ea[l].g, s->ea[l].a, c, 0, nullptr, nullptr), st));
        const __nv_bfloat16 *in = l == 0 ? maps : s->pool[l - 1].a;
        const int cin = l == 0 ? s->shape.in_ch : lvl_ch(s, l - 1);
        SUR_CUDA(unet_wgrad3x3(wgrad_in(in, cin, 0, nullptr, 0, B, h, w, c1.cout), s->ea[l].g, c1.gw, st));
        SUR_CUDA(unet_bias_grad(s->ea[l].g, c1.gb, M, c1.cout, st));
        if (l > 0)
            SUR_CUDA(unet_conv3x3(dgrad_conv(c1, s->ea[l].g, B, h, w, s->pool[l - 1].g, s->pool[l - 1].a, cin, 0,
                                             nullptr, nullptr), st));
    }
    return ER_OK;
}

static er_status loss_and_grad(er_surrogate *s, const float *target, const uint8_t *mask, int B, double *loss,
                               cudaStream_t st) {
    const int64_t n = (int64_t)B * s->shape.H * s->shape.W * s->shape.out_ch;
    int64_t count = n;
    if (mask) {  // count the masked-in entries on the host side of the call
        std::vector<uint8_t> h((size_t)n);
        SUR_CUDA(cudaMemcpyAsync(h.data(), mask, n, cudaMemcpyDeviceToHost, st));
        SUR_CUDA(cudaStreamSynchronize(st));
        count = 0;
        for (uint8_t v : h) count += v != 0;
        if (count == 0) count = 1;
    }
    SUR_CUDA(cudaMemsetAsync(s->loss, 0, sizeof(double), st));
    SUR_CUDA(unet_mse(s->out, target, mask, s->dout, s->loss, n, 1.0f / (float)count, st));
    double h = 0.0;
    SUR_CUDA(cudaMemcpyAsync(&h, s->loss, sizeof(double), cudaMemcpyDeviceToHost, st));
    SUR_CUDA(cudaStreamSynchronize(st));
    if (loss) *loss = h / (double)count;
    return ER_OK;
}

static std::vector<std::pair<float *, int64_t>> param_list(er_surrogate *s) {
    std::vector<std::pair<float *, int64_t>> v;
    for (Conv &c : s->enc) v.push_back({c.w, c.nw()}), v.push_back({c.b, c.cout});
    for (int l = s->L - 2; l >= 0; --l)
        for (int i = 0; i < 2; ++i) {
            Conv &c = s->dec[2 * l + i];
            v.push_back({c.w, c.nw()});
            v.push_back({c.b, c.cout});
        }
    v.push_back({s->hw, (int64_t)s->shape.out_ch * s->shape.base});
    v.push_back({s->hb, s->shape.out_ch});
    return v;
}

static std::vector<std::pair<float *, int64_t>> grad_list(er_surrogate *s) {
    std::vector<std::pair<float *, int64_t>> v;
    for (Conv &c : s->enc) v.push_back({c.gw, c.nw()}), v.push_back({c.gb, c.cout});
    for (int l = s->L - 2; l >= 0; --l)
        for (int i = 0; i < 2; ++i) {
            Conv &c = s->dec[2 * l + i];
            v.push_back({c.gw, c.nw()});
            v.push_back({c.gb, c.cout});
        }
    v.push_back({s->hgw, (int64_t)s->shape.out_ch * s->shape.base});
    v.push_back({s->hgb, s->shape.out_ch});
    return v;
}

static er_status check_io(er_surrogate *s, const void *maps, int B) {
    if (!s) return fail(ER_ERR_INVALID_ARG, "surrogate is NULL");
    if (!maps || B < 1) return fail(ER_ERR_INVALID_ARG, "maps and B >= 1 are required");
    if (((uintptr_t)maps & 15u)) return fail(ER_ERR_INVALID_ARG, "maps must be 16-byte aligned");
    return ER_OK;
}

}  // namespace er

extern "C" {

er_status er_surrogate_create(const er_unet_shape *shape, uint64_t seed, er_surrogate **out) {
    using namespace er;
    if (!shape || !out) return fail(ER_ERR_INVALID_ARG, "shape and out are required");
    *out = nullptr;
    const er_unet_shape sh = *shape;
    if (sh.levels < 2 || sh.levels > 8 || sh.base < 32 || sh.base % 32 || sh.in_ch < 32 || sh.in_ch % 32 ||
        sh.out_ch < 1 || sh.H < 1 || sh.W < 1 || sh.H % (1 << (sh.levels - 1)) || sh.W % (1 << (sh.levels - 1)))
        return fail(ER_ERR_INVALID_ARG,
                    "need base and in_ch multiples of 32, 2 <= levels <= 8, H and W divisible by 2^(levels-1)");
    std::unique_ptr<er_surrogate> s(new er_surrogate());
    s->shape = sh;
    s->L = sh.levels;
    ER_CUDA(cudaGetDevice(&s->device));
    s->enc.resize(2 * s->L);
    s->dec.resize(2 * s->L);
    uint64_t sd = mix64(seed);
    std::vector<void *> owned;
    er_status st = ER_OK;
    for (int l = 0; l < s->L && st == ER_OK; ++l) {
        const int c = sh.base << l, cin = l == 0 ? sh.in_ch : (sh.base << (l - 1));
        st = init_conv(s->enc[2 * l], cin, c, sd = mix64(sd), owned);
        if (st == ER_OK) st = init_conv(s->enc[2 * l + 1], c, c, sd = mix64(sd), owned);
    }
    for (int l = s->L - 2; l >= 0 && st == ER_OK; --l) {
        const int c = sh.base << l;
        st = init_conv(s->dec[2 * l], (sh.base << (l + 1)) + c, c, sd = mix64(sd), owned);
        if (st == ER_OK) st = init_conv(s->dec[2 * l + 1], c, c, sd = mix64(sd), owned);
    }
    const int64_t nh = (int64_t)sh.out_ch * sh.base;
    for (float **p : {&s->hw, &s->hb, &s->hmw, &s->hvw, &s->hmb, &s->hvb, &s->hgw, &s->hgb}) {
        if (st != ER_OK) break;
        const int64_t n = (p == &s->hw || p == &s->hmw || p == &s->hvw || p == &s->hgw) ? nh : sh.out_ch;
        if (cudaMalloc((void **)p, n * 4) != cudaSuccess) st = fail(ER_ERR_OOM, "surrogate head");
        else cudaMemset(*p, 0, n * 4);
        owned.push_back(*p);
    }
    if (st == ER_OK) {
        std::vector<float> h((size_t)nh);
        const double sdh = std::sqrt(1.0 / sh.base);
        for (int64_t i = 0; i < nh; ++i) h[i] = (float)(sdh * (((mix64(sd ^ (uint64_t)i) >> 11) * (1.0 / 9007199254740992.0)) * 2.0 - 1.0) * 1.7320508);
        if (cudaMemcpy(s->hw, h.data(), nh * 4, cudaMemcpyHostToDevice) != cudaSuccess) st = fail(ER_ERR_CUDA, "head init");
    }
    if (st == ER_OK && cudaMalloc((void **)&s->loss, sizeof(double)) != cudaSuccess) st = fail(ER_ERR_OOM, "loss");
    if (st != ER_OK) {
        for (void *p : owned) cudaFree(p);
        return st;
    }
    // parameter buffers are reachable through enc/dec/head until er_surrogate_destroy;
    // s->owned holds only the per-batch activations
    *out = s.release();
    return ER_OK;
}

er_status er_surrogate_destroy(er_surrogate *s) {
    if (!s) return ER_OK;
    cudaSetDevice(s->device);
    for (void *p : s->owned) cudaFree(p);
    for (auto *v : {&s->enc, &s->dec})
        for (er::Conv &c : *v)
            for (void *p : {(void *)c.w, (void *)c.b, (void *)c.wb, (void *)c.wt, (void *)c.mw, (void *)c.vw,
                            (void *)c.mb, (void *)c.vb, (void *)c.gw, (void *)c.gb})
                if (p) cudaFree(p);
    for (float *p : {s->hw, s->hb, s->hmw, s->hvw, s->hmb, s->hvb, s->hgw, s->hgb})
        if (p) cudaFree(p);
    if (s->loss) cudaFree(s->loss);
    delete s;
    return ER_OK;
}

er_status er_surrogate_num_params(const er_surrogate *s, int64_t *n) {
    if (!s || !n) return er::fail(ER_ERR_INVALID_ARG, "surrogate and n are required");
    int64_t t = 0;
    for (auto &p : er::param_list(const_cast<er_surrogate *>(s))) t += p.second;
    *n = t;
    return ER_OK;
}

er_status er_surrogate_get_params(const er_surrogate *s, float *host, int64_t n) {
    int64_t need = 0;
    er_status st = er_surrogate_num_params(s, &need);
    if (st != ER_OK) return st;
    if (!host || n != need) return er::fail(ER_ERR_INVALID_ARG, "host buffer must hold exactly num_params floats");
    int64_t off = 0;
    for (auto &p : er::param_list(const_cast<er_surrogate *>(s))) {
        ER_CUDA(cudaMemcpy(host + off, p.first, p.second * 4, cudaMemcpyDeviceToHost));
        off += p.second;
    }
    return ER_OK;
}

er_status er_surrogate_set_params(er_surrogate *s, const float *host, int64_t n) {
    int64_t need = 0;
    er_status st = er_surrogate_num_params(s, &need);
    if (st != ER_OK) return st;
    if (!host || n != need) return er::fail(ER_ERR_INVALID_ARG, "host buffer must hold exactly num_params floats");
    int64_t off = 0;
    for (auto &p : er::param_list(s)) {
        ER_CUDA(cudaMemcpy(p.first, host + off, p.second * 4, cudaMemcpyHostToDevice));
        off += p.second;
    }
    for (auto *v : {&s->enc, &s->dec})
        for (er::Conv &c : *v)
            if (c.w) ER_CUDA(er::unet_to_bf16(c.w, c.wb, c.wt, c.nw(), c.cout, c.cin, nullptr));
    ER_CUDA(cudaDeviceSynchronize());
    return ER_OK;
}

er_status er_surrogate_infer(er_surrogate *s, const void *maps, int32_t B, float *logR, void *stream) {
    er_status st = er::check_io(s, maps, B);
    if (st != ER_OK) return st;
    if (!logR) return er::fail(ER_ERR_INVALID_ARG, "logR is NULL");
    ER_CUDA(cudaSetDevice(s->device));
    st = er::ensure_batch(s, B);
    if (st != ER_OK) return st;
    cudaStream_t cs = (cudaStream_t)stream;
    st = er::forward(s, (const __nv_bfloat16 *)maps, B, cs);
    if (st != ER_OK) return st;
    ER_CUDA(cudaMemcpyAsync(logR, s->out, (size_t)B * s->shape.H * s->shape.W * s->shape.out_ch * 4,
                            cudaMemcpyDeviceToDevice, cs));
    return er::check_kernels(cs);
}

er_status er_surrogate_grad(er_surrogate *s, const void *maps, const float *target, const uint8_t *mask, int32_t B,
                            float *grads_host, double *loss, void *stream) {
    er_status st = er::check_io(s, maps, B);
    if (st != ER_OK) return st;
    if (!target) return er::fail(ER_ERR_INVALID_ARG, "target is NULL");
    ER_CUDA(cudaSetDevice(s->device));
    st = er::ensure_batch(s, B);
    if (st != ER_OK) return st;
    cudaStream_t cs = (cudaStream_t)stream;
    st = er::forward(s, (const __nv_bfloat16 *)maps, B, cs);
    if (st == ER_OK) st = er::loss_and_grad(s, target, mask, B, loss, cs);
    if (st == ER_OK) st = er::backward(s, (const __nv_bfloat16 *)maps, B, cs);
    if (st != ER_OK) return st;
    if (grads_host) {
        int64_t off = 0;
        for (auto &p : er::grad_list(s)) {
            ER_CUDA(cudaMemcpyAsync(grads_host + off, p.first, p.second * 4, cudaMemcpyDeviceToHost, cs));
            off += p.second;
        }
    }
    return er::check_kernels(cs);
}

er_status er_surrogate_train_step(er_surrogate *s, const void *maps, const float *target, const uint8_t *mask,
                                  int32_t B, float lr, double *loss, void *stream) {
    er_status st = er_surrogate_grad(s, maps, target, mask, B, nullptr, loss, stream);
    if (st != ER_OK) return st;
    if (!(lr > 0.f)) return er::fail(ER_ERR_INVALID_ARG, "lr must be positive");
    cudaStream_t cs = (cudaStream_t)stream;
    const int step = ++s->step;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (auto *v : {&s->enc, &s->dec})
        for (er::Conv &c : *v) {
            if (!c.w) continue;
            ER_CUDA(er::unet_adam(c.w, c.mw, c.vw, c.gw, c.nw(), lr, b1, b2, eps, step, c.wb, c.wt, c.cout, c.cin, cs));
            ER_CUDA(er::unet_adam(c.b, c.mb, c.vb, c.gb, c.cout, lr, b1, b2, eps, step, nullptr, nullptr, 1, 1, cs));
        }
    const int64_t nh = (int64_t)s->shape.out_ch * s->shape.base;
    ER_CUDA(er::unet_adam(s->hw, s->hmw, s->hvw, s->hgw, nh, lr, b1, b2, eps, step, nullptr, nullptr, 1, 1, cs));
    ER_CUDA(er::unet_adam(s->hb, s->hmb, s->hvb, s->hgb, s->shape.out_ch, lr, b1, b2, eps, step, nullptr, nullptr, 1, 1, cs));
    ER_CUDA(cudaStreamSynchronize(cs));
    return ER_OK;
}

er_status er_surrogate_set_tile_n(er_surrogate *s, int32_t tile_n) {
    if (!s) return er::fail(ER_ERR_INVALID_ARG, "surrogate is NULL");
    if (tile_n != 0 && tile_n != 32 && tile_n != 64 && tile_n != 96 && tile_n != 128 && tile_n != 192 && tile_n != 256)
        return er::fail(ER_ERR_INVALID_ARG, "tile_n must be 0, 32, 64, 96, 128, 192 or 256");
    s->tile_n = tile_n;
    return ER_OK;
}

er_status er_conv_launch_counts(int64_t *counts, int32_t n, int32_t reset) {
    if (n < 0 || (n > 0 && !counts)) return er::fail(ER_ERR_INVALID_ARG, "counts is NULL");
    er::unet_conv_counts(counts, n, reset);
    return ER_OK;
}

}  // extern "C"

// ---- single convolution layers ----------------------------------------------------------

namespace er {

static er_status conv_layer_args(const void *a, const void *b, const void *out, int B, int H, int W, int cin,
                                 int cout, int tile_n) {
    if (!a || !b || !out) return fail(ER_ERR_INVALID_ARG, "input, weight/gradient and output pointers are required");
    if ((((uintptr_t)a) | ((uintptr_t)b) | ((uintptr_t)out)) & 15u)
        return fail(ER_ERR_INVALID_ARG, "device arrays must be 16-byte aligned");
    if (B < 1 || H < 1 || W < 1 || cin < 32 || cin % 32 || cout < 32 || cout % 32)
        return fail(ER_ERR_INVALID_ARG, "need B, H, W >= 1 and cin, cout positive multiples of 32");
    if ((int64_t)B * H * W > (int64_t)1 << 31) return fail(ER_ERR_INVALID_ARG, "B*H*W must be below 2^31");
    if (tile_n != 0 && tile_n != 32 && tile_n != 64 && tile_n != 96 && tile_n != 128 && tile_n != 192 && tile_n != 256)
        return fail(ER_ERR_INVALID_ARG, "tile_n must be 0, 32, 64, 96, 128, 192 or 256");
    return ER_OK;
}

// BF16 copies of FP32 weights [cout][3][3][cin]: as stored, and flipped and transposed for the
// data gradient; freed in stream order by the caller through conv_weights_free
static er_status conv_weights(const float *w, int cout, int cin, cudaStream_t s, __nv_bfloat16 **wb,
                              __nv_bfloat16 **wt) {
    const int64_t n = (int64_t)cout * 9 * cin;
    *wb = *wt = nullptr;
    ER_CUDA(cudaMallocAsync((void **)wb, (size_t)n * 2, s));
    ER_CUDA(cudaMallocAsync((void **)wt, (size_t)n * 2, s));
    ER_CUDA(unet_to_bf16(w, *wb, *wt, n, cout, cin, s));
    return ER_OK;
}

static er_status layer_done(cudaStream_t s, __nv_bfloat16 *wb, __nv_bfloat16 *wt, cudaError_t launch) {
    if (wb) cudaFreeAsync(wb, s);
    if (wt) cudaFreeAsync(wt, s);
    if (launch != cudaSuccess) return cuda_fail(launch, "convolution launch");
    return check_kernels(s);
}

}  // namespace er

extern "C" {

er_status er_conv3x3_forward(const void *x, const float *w, const float *bias, int32_t B, int32_t H, int32_t W,
                             int32_t cin, int32_t cout, int32_t relu, int32_t tile_n, void *y, er_conv_info *info,
                             void *stream) {
    using namespace er;
    er_status st = conv_layer_args(x, w, y, B, H, W, cin, cout, tile_n);
    if (st != ER_OK) return st;
    cudaStream_t cs = (cudaStream_t)stream;
    __nv_bfloat16 *wb = nullptr, *wt = nullptr;
    st = conv_weights(w, cout, cin, cs, &wb, &wt);
    if (st != ER_OK) return layer_done(cs, wb, wt, cudaSuccess), st;
    UConvInfo ui;
    UConv u;
    u.x1 = (const __nv_bfloat16 *)x; u.c1 = cin; u.w = wb; u.bias = bias; u.nb = B; u.h = H; u.w_ = W;
    u.cout = cout; u.relu = relu != 0; u.y = (__nv_bfloat16 *)y; u.tile_n = tile_n; u.info = &ui;
    const cudaError_t e = unet_conv3x3(u, cs);
    st = layer_done(cs, wb, wt, e);
    if (st == ER_OK && info) *info = er_conv_info{ui.kernel, ui.bn, ui.bk, 0};
    return st;
}

er_status er_conv3x3_dgrad(const void *dy, const float *w, const void *x, int32_t B, int32_t H, int32_t W,
                           int32_t cin, int32_t cout, int32_t tile_n, void *dx, er_conv_info *info, void *stream) {
    using namespace er;
    er_status st = conv_layer_args(dy, w, dx, B, H, W, cin, cout, tile_n);
    if (st != ER_OK) return st;
    if (!x || ((uintptr_t)x & 15u)) return fail(ER_ERR_INVALID_ARG, "x (the forward input) must be a 16-byte aligned device array");
    cudaStream_t cs = (cudaStream_t)stream;
    __nv_bfloat16 *wb = nullptr, *wt = nullptr;
    st = conv_weights(w, cout, cin, cs, &wb, &wt);
    if (st != ER_OK) return layer_done(cs, wb, wt, cudaSuccess), st;
    UConvInfo ui;
    UConv u;
    u.x1 = (const __nv_bfloat16 *)dy; u.c1 = cout; u.w = wt; u.nb = B; u.h = H; u.w_ = W; u.cout = cin;
    u.g1 = (__nv_bfloat16 *)dx; u.m1 = (const __nv_bfloat16 *)x; u.c1o = cin; u.tile_n = tile_n; u.info = &ui;
    const cudaError_t e = unet_conv3x3(u, cs);
    st = layer_done(cs, wb, wt, e);
    if (st == ER_OK && info) *info = er_conv_info{ui.kernel, ui.bn, ui.bk, 0};
    return st;
}

er_status er_conv3x3_wgrad(const void *x, const void *dy, int32_t B, int32_t H, int32_t W, int32_t cin, int32_t cout,
                           float *dw, void *stream) {
    using namespace er;
    er_status st = conv_layer_args(x, dy, dw, B, H, W, cin, cout, 0);
    if (st != ER_OK) return st;
    cudaStream_t cs = (cudaStream_t)stream;
    ER_CUDA(cudaMemsetAsync(dw, 0, (size_t)cout * 9 * cin * sizeof(float), cs));
    UConv u;
    u.x1 = (const __nv_bfloat16 *)x; u.c1 = cin; u.nb = B; u.h = H; u.w_ = W; u.cout = cout;
    const cudaError_t e = unet_wgrad3x3(u, (const __nv_bfloat16 *)dy, dw, cs);
    return layer_done(cs, nullptr, nullptr, e);
}

}  // extern "C"
