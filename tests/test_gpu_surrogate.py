"""The BF16 U-Net surrogate: forward pass and parameter gradients of the library's own
kernels against the FP64 reference (oracle/unet_ref.py) on small shapes, and a short
training run showing what the trained network gains over predicting the training mean."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle.unet_ref import UNetRef


@pytest.fixture(scope="module")
def er():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2607_05818_gb300 import er as mod
    return mod


def bf16(a):
    return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)


def ref_params(net, flat):
    """The GPU's effective parameters: 3x3 weights in BF16, biases and the head in FP32."""
    p = net.unflatten(flat)
    for name, _ in net.shapes:
        if name.endswith(".w") and not name.startswith("head"):
            p[name] = bf16(p[name])
    return net.flatten(p)


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def linf(a):
    return float(np.max(np.abs(a))) if np.size(a) else 0.0


# (levels, base, hw, tile_n): the last two reach the deep layers' wide N tiles: 256 output
# channels per tile with two 256-column TMEM accumulators (levels 4, base 64: 256 and 512
# channels) and 192 (base 96: 192 and 384 channels); both with 64-channel K steps on every
# layer but the first.
NET_CASES = [(2, 32, 16, 0), (3, 32, 32, 0), (2, 64, 8, 0), (4, 64, 16, 256), (3, 96, 16, 192)]


@pytest.mark.parametrize("levels,base,hw,tile_n", NET_CASES)
def test_forward_and_gradients_match_reference(er, levels, base, hw, tile_n):
    in_ch, out_ch, B = 32, 4, 2
    model = er.Surrogate(in_ch=in_ch, out_ch=out_ch, levels=levels, base=base, H=hw, W=hw, seed=5)
    model.set_tile_n(tile_n)
    net = UNetRef(in_ch, out_ch, levels, base)
    assert model.num_params() == net.num_params()
    rng = np.random.default_rng(levels * 100 + base)
    flat = model.get_params().astype(np.float64)
    flat[-out_ch:] = rng.normal(0, 0.1, out_ch)            # nonzero head bias
    model.set_params(flat.astype(np.float32))
    x = bf16(rng.normal(0, 1, (B, hw, hw, in_ch)))
    target = rng.normal(0, 1, (B, hw, hw, out_ch))
    mask = rng.random((B, hw, hw, out_ch)) > 0.1
    maps = torch.from_numpy(x.astype(np.float32)).to("cuda", torch.bfloat16)
    tg = torch.from_numpy(target.astype(np.float32)).cuda()
    mk = torch.from_numpy(mask.astype(np.uint8)).cuda()
    out = torch.empty((B, hw, hw, out_ch), dtype=torch.float32, device="cuda")
    er.conv_launch_counts(reset=True)
    model.infer(maps, B, out)
    loss_gpu, g_gpu = model.grad(maps, tg, mk, B)
    torch.cuda.synchronize()
    ran = {k: v for k, v in er.conv_launch_counts().items() if v}
    print(f"levels {levels} base {base} {hw}x{hw} tile_n {tile_n}: convolution launches {ran}")
    if tile_n:
        assert ran.get(f"tma_k64_n{tile_n}", 0) > 0, ran
    pe = ref_params(net, flat)
    # Activations and activation gradients are stored in BF16 between layers.  A difference
    # of one rounding anywhere (FP32 vs FP64 sums landing on either side of a BF16 boundary)
    # spreads through the later layers, so the reference is evaluated exactly in FP64, rounded
    # to BF16 where the kernels store BF16, and rounded after nudging every stored value by a
    # few parts in 1e6.  The nudged evaluations differ from the rounded one only by which side
    # of a BF16 boundary near-ties land on: their largest element-wise deviation is the noise
    # floor of each tensor.  Every element of every GPU tensor must lie within twice that floor
    # (plus 2e-3 of the tensor's largest value) of the rounded reference.
    loss_ref, g_ref, out_ref = net.loss_and_grad(pe, x, target, mask)
    loss_b, g_b, out_b = net.loss_and_grad(pe, x, target, mask, rnd=bf16)
    nudged = [net.loss_and_grad(pe, x, target, mask, rnd=lambda v, f=f: bf16(v * f))
              for f in (1 + 1e-6, 1 - 1e-6, 1 + 3e-6)]
    og = out.cpu().numpy().astype(np.float64)
    noise_out = max(linf(o - out_b) for _, _, o in nudged)
    e_out = linf(og - out_b)
    print(f"output: max |gpu - rounded| {e_out:.2e} (noise {noise_out:.2e}, scale {linf(out_b):.2e})")
    assert e_out <= 2 * noise_out + 2e-3 * linf(out_b)
    assert linf(og - out_ref) <= 2 * linf(out_b - out_ref) + 2e-3 * linf(out_ref)
    assert loss_gpu == pytest.approx(loss_b, rel=1e-2)
    off = 0
    for name, shape in net.shapes:
        n = int(np.prod(shape))
        sl = slice(off, off + n)
        gg = g_gpu[sl].astype(np.float64)
        noise = max(linf(g[sl] - g_b[sl]) for _, g, _ in nudged)
        scale = linf(g_b[sl])
        e_b, e_x, e_bx = linf(gg - g_b[sl]), linf(gg - g_ref[sl]), linf(g_b[sl] - g_ref[sl])
        print(f"{name}: max |gpu - rounded| {e_b:.2e} (noise {noise:.2e}, scale {scale:.2e}); "
              f"max |gpu - exact| {e_x:.2e} (rounded vs exact {e_bx:.2e})")
        assert e_b <= 2 * noise + 2e-3 * scale, name
        assert e_x <= 2 * e_bx + 2e-3 * linf(g_ref[sl]), name
        off += n
    model.destroy()


# ---- single convolution layers through er_conv3x3_*: element by element against the oracle's
# FP64 convolution of the same BF16 values.  The kernels form BF16 x BF16 products exactly in
# FP32 and add them in FP32; forward and data-gradient outputs are rounded to BF16 once.  So
# an element may differ from the BF16 rounding of the exact value by at most half a BF16 unit
# in the last place (2^-8 of its magnitude) plus the FP32 summation error, bounded by
# (terms) x 2^-24 x (sum of the absolute values of its terms); most elements equal it exactly.

FWD_CASES = [  # (B, H, W, cin, cout, tile_n, expected (kernel, tile_n, k_step))
    (20, 32, 32, 128, 256, 0, ("tma", 256, 64)),    # the library's own choice at a deep layer's size
    (4, 16, 16, 64, 384, 192, ("tma", 192, 64)),
    (4, 16, 16, 96, 256, 256, ("tma", 256, 32)),
    (4, 16, 16, 96, 384, 96, ("tma", 96, 32)),
    (3, 8, 8, 64, 128, 128, ("tma", 128, 64)),      # 192 pixels: a ragged last pixel tile
    (2, 16, 16, 32, 64, 64, ("tma", 64, 32)),
    (2, 16, 16, 32, 32, 32, ("tma", 32, 32)),
    (2, 24, 24, 64, 256, 256, ("staged", 256, 32)),  # 24 x 24 does not tile into 128-pixel boxes
    (2, 12, 20, 32, 96, 0, ("staged", None, 32)),
]
DGRAD_CASES = [  # (B, H, W, cin, cout, tile_n, expected); the data gradient has cin outputs
    (4, 16, 16, 256, 128, 256, ("tma", 256, 64)),
    (4, 16, 16, 384, 64, 192, ("tma", 192, 64)),
    (3, 8, 8, 128, 96, 128, ("tma", 128, 32)),
    (2, 24, 24, 256, 64, 256, ("staged", 256, 32)),
]
WGRAD_CASES = [  # (B, H, W, cin, cout, expected kernel)
    (4, 16, 16, 64, 128, "wgrad_tc"), (2, 16, 16, 256, 256, "wgrad_tc"), (20, 32, 32, 128, 256, "wgrad_tc"),
    (3, 8, 8, 192, 128, "wgrad_tc"), (8, 4, 4, 512, 256, "wgrad_tc"), (2, 64, 64, 64, 128, "wgrad_tc"),
    (3, 8, 8, 96, 64, "wgrad_tc"),      # a half-empty 64-channel block of input channels
    (2, 16, 16, 32, 32, "wgrad_tc"),    # 32 output channels: rows 32-127 of the tile are zero-filled
    (2, 32, 32, 32, 64, "wgrad_tc"),
    (2, 24, 24, 32, 32, "wgrad_mma")]   # 24 x 24 does not tile into 64-pixel boxes


def _bf16_dev(a):
    return torch.from_numpy(np.asarray(a, np.float32)).to("cuda", torch.bfloat16)


def _check_rounded(got, exact, absum, k_terms, what):
    """got: BF16 outputs; exact: FP64 value before rounding; absum: sum of |terms| per element."""
    tol = 2.0 ** -8 * np.abs(exact) + (1 + 2.0 ** -8) * k_terms * 2.0 ** -24 * absum + 1e-30
    err = np.abs(got - exact)
    same = float(np.mean(got == bf16(exact)))
    print(f"{what}: max err / bound {float(np.max(err / tol)):.3f}, equal to the rounded exact value: "
          f"{100 * same:.2f}%")
    assert np.all(err <= tol), what
    assert same >= 0.9, what


@pytest.mark.parametrize("B,H,W,cin,cout,tile_n,expect", FWD_CASES)
def test_conv_layer_forward_elementwise(er, B, H, W, cin, cout, tile_n, expect):
    from oracle.unet_ref import conv3x3
    rng = np.random.default_rng(B * 1000 + cin + cout + tile_n)
    x = bf16(rng.normal(0, 1, (B, H, W, cin)))
    w = bf16(rng.normal(0, 1 / np.sqrt(9 * cin), (cout, 3, 3, cin)))
    b = rng.normal(0, 0.1, cout).astype(np.float32).astype(np.float64)
    y = torch.empty((B, H, W, cout), dtype=torch.bfloat16, device="cuda")
    info = er.conv3x3_forward(_bf16_dev(x), torch.from_numpy(w.astype(np.float32)).cuda(),
                              torch.from_numpy(b.astype(np.float32)).cuda(), B, H, W, cin, cout, y, relu=True,
                              tile_n=tile_n)
    print(f"forward {B}x{H}x{W} {cin}->{cout} tile_n {tile_n}: ran {info}")
    kern, tn, ks = expect
    assert info["kernel"] == kern and info["k_step"] == ks and (tn is None or info["tile_n"] == tn), info
    got = y.float().cpu().numpy().astype(np.float64)
    pre = conv3x3(x, w, b)
    absum = conv3x3(np.abs(x), np.abs(w), np.abs(b))
    _check_rounded(got, np.maximum(pre, 0.0), absum, 9 * cin + 1, "forward")


@pytest.mark.parametrize("B,H,W,cin,cout,tile_n,expect", DGRAD_CASES)
def test_conv_layer_dgrad_elementwise(er, B, H, W, cin, cout, tile_n, expect):
    from oracle.unet_ref import conv3x3_bwd
    rng = np.random.default_rng(B * 2000 + cin + cout + tile_n)
    x = bf16(rng.normal(0, 1, (B, H, W, cin)))          # the forward input: its sign is the ReLU mask
    dy = bf16(rng.normal(0, 1, (B, H, W, cout)))
    w = bf16(rng.normal(0, 1 / np.sqrt(9 * cin), (cout, 3, 3, cin)))
    dx = torch.empty((B, H, W, cin), dtype=torch.bfloat16, device="cuda")
    info = er.conv3x3_dgrad(_bf16_dev(dy), torch.from_numpy(w.astype(np.float32)).cuda(), _bf16_dev(x), B, H, W,
                            cin, cout, dx, tile_n=tile_n)
    print(f"dgrad {B}x{H}x{W} {cin}<-{cout} tile_n {tile_n}: ran {info}")
    kern, tn, ks = expect
    assert info["kernel"] == kern and info["k_step"] == ks and info["tile_n"] == tn, info
    got = dx.float().cpu().numpy().astype(np.float64)
    ref = conv3x3_bwd(x, w, dy)[0] * (x > 0)
    absum = conv3x3_bwd(x, np.abs(w), np.abs(dy))[0] * (x > 0)
    _check_rounded(got, ref, absum, 9 * cout, "dgrad")


@pytest.mark.parametrize("B,H,W,cin,cout,kern", WGRAD_CASES)
def test_conv_layer_wgrad_elementwise(er, B, H, W, cin, cout, kern):
    from oracle.unet_ref import conv3x3_bwd
    rng = np.random.default_rng(B * 3000 + cin + cout)
    x = bf16(rng.normal(0, 1, (B, H, W, cin)))
    dy = bf16(rng.normal(0, 1, (B, H, W, cout)))
    dw = torch.full((cout, 3, 3, cin), float("nan"), dtype=torch.float32, device="cuda")
    er.conv_launch_counts(reset=True)
    er.conv3x3_wgrad(_bf16_dev(x), _bf16_dev(dy), B, H, W, cin, cout, dw)
    ran = {k_: v for k_, v in er.conv_launch_counts().items() if v}
    print(f"wgrad {B}x{H}x{W} {cin}x{cout}: ran {ran}")
    assert ran == {kern: 1}, ran
    got = dw.cpu().numpy().astype(np.float64)
    w0 = np.zeros((cout, 3, 3, cin))
    ref = conv3x3_bwd(x, w0, dy)[1]
    absum = conv3x3_bwd(np.abs(x), w0, np.abs(dy))[1]
    npix = B * H * W
    tol = npix * 2.0 ** -24 * absum + 1e-30
    err = np.abs(got - ref)
    print(f"wgrad {B}x{H}x{W} {cin}x{cout}: max err / bound {float(np.max(err / tol)):.3f}, "
          f"max rel err {float(np.max(err / np.maximum(absum, 1e-30))):.2e}")
    assert np.all(err <= tol)


def test_training_and_screening_gain(er):
    """Small surrogate workload (4 tiers x 64x64 candidates, seeded random TSV layouts and sheet
    resistances): after a short training run on solver labels the network predicts held-out
    log R maps far better than the training-set mean map; screening the held-out candidates by
    the surrogate finds most of the worst ones at a small fraction of the cost of solving them
    all, which is the method without the surrogate."""
    import time

    from paper_2607_05818_gb300 import surrogate as S
    rng = np.random.default_rng(2026)
    ntr, nte = 128, 32
    nets = [S.candidate(rng, T=4, W=64) for _ in range(ntr + nte)]
    S.label(nets[:4], k=64, seed=7)                      # warm-up (module load, pools)
    t0 = time.perf_counter()
    Rs = S.label(nets, k=64, seed=11)
    t_solve = (time.perf_counter() - t0) / len(nets)
    maps, tgt, msk = S.to_device(nets, Rs)
    model = er.Surrogate(in_ch=32, out_ch=4, levels=3, base=32, H=64, W=64, seed=3)
    hist = S.train(model, maps[:ntr], tgt[:ntr], msk[:ntr], epochs=60, batch=8, lr=2e-3,
                   lr_final=2e-4)
    assert hist[-1] < 0.5 * hist[0]
    S.predict(model, maps[ntr:ntr + 8], batch=8)          # warm-up
    t1 = time.perf_counter()
    pred = S.predict(model, maps[ntr:], batch=8)
    t_inf = (time.perf_counter() - t1) / nte
    mean_map = (tgt[:ntr] * msk[:ntr]).sum(0) / msk[:ntr].sum(0).clamp(min=1)
    m = msk[ntr:].bool()
    mse_net = float(((pred - tgt[ntr:])[m] ** 2).mean())
    mse_mean = float(((mean_map.expand_as(tgt[ntr:]) - tgt[ntr:])[m] ** 2).mean())
    # screening: the worst quarter of the held-out candidates by the exact labels, and by the
    # surrogate's prediction
    pn, tn, mn = pred.cpu().numpy(), tgt[ntr:].cpu().numpy(), msk[ntr:].cpu().numpy()
    s_true = np.array([S.score(tn[i], mn[i]) for i in range(nte)])
    s_pred = np.array([S.score(pn[i], mn[i]) for i in range(nte)])
    q = nte // 4
    worst = set(np.argsort(-s_true)[:q])
    recall = len(worst & set(np.argsort(-s_pred)[:q])) / q
    recall2 = len(worst & set(np.argsort(-s_pred)[:2 * q])) / q      # verifying twice as many
    rho = np.corrcoef(np.argsort(np.argsort(s_true)), np.argsort(np.argsort(s_pred)))[0, 1]
    print(f"held-out MSE(log R): network {mse_net:.4f}, training mean {mse_mean:.4f}; worst {q}: recall "
          f"{recall:.2f} in the surrogate's worst {q}, {recall2:.2f} in its worst {2 * q}; rank correlation "
          f"{rho:.3f}; solve {t_solve * 1e3:.2f} ms/candidate, forward {t_inf * 1e3:.3f} ms/candidate")
    assert mse_net < 0.5 * mse_mean
    assert rho >= 0.8
    assert recall2 >= 0.75
    assert t_inf < 0.2 * t_solve
    model.destroy()
