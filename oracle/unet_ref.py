"""FP64 reference of the U-Net surrogate's forward and backward passes (test infrastructure).

Plain numpy, written from the layer definitions: 3x3 convolution with zero padding
(y[b,h,w,o] = bias[o] + sum_{ky,kx,c} x[b,h+ky-1,w+kx-1,c] W[o,ky,kx,c]), ReLU, 2x2 max
pooling (the gradient goes to the first maximum in row-major order), nearest-neighbour 2x
upsampling, channel concatenation, a 1x1 head and the masked mean-squared error.  The
network graph and the parameter order match er_surrogate_*: encoder convolutions level by
level, decoder convolutions from the deepest level up, then the head; each layer's
weights [cout][3][3][cin] (head [out][base]) before its biases.  The backward pass is
pinned by central finite differences in tests/test_oracle_pins.py.
"""
from __future__ import annotations

import numpy as np


def conv3x3(x, w, b):
    B, H, W, C = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    y = np.broadcast_to(b, (B, H, W, w.shape[0])).astype(np.float64).copy()
    for ky in range(3):
        for kx in range(3):
            y += np.einsum("bhwc,oc->bhwo", xp[:, ky:ky + H, kx:kx + W, :], w[:, ky, kx, :])
    return y


def conv3x3_bwd(x, w, dy):
    """(dx, dw, db) of y = conv3x3(x, w, b) given dy = dL/dy."""
    B, H, W, C = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for ky in range(3):
        for kx in range(3):
            dw[:, ky, kx, :] = np.einsum("bhwo,bhwc->oc", dy, xp[:, ky:ky + H, kx:kx + W, :])
            dxp[:, ky:ky + H, kx:kx + W, :] += np.einsum("bhwo,oc->bhwc", dy, w[:, ky, kx, :])
    return dxp[:, 1:H + 1, 1:W + 1, :], dw, dy.sum(axis=(0, 1, 2))


def maxpool(x):
    B, H, W, C = x.shape
    blocks = x.reshape(B, H // 2, 2, W // 2, 2, C).transpose(0, 1, 3, 2, 4, 5).reshape(B, H // 2, W // 2, 4, C)
    arg = np.argmax(blocks, axis=3)  # first maximum in (dy, dx) row-major order
    return blocks.max(axis=3), arg


def maxpool_bwd(arg, dy, shape):
    B, H, W, C = shape
    d = np.zeros((B, H // 2, W // 2, 4, C))
    np.put_along_axis(d, arg[:, :, :, None, :], dy[:, :, :, None, :], axis=3)
    return d.reshape(B, H // 2, W // 2, 2, 2, C).transpose(0, 1, 3, 2, 4, 5).reshape(B, H, W, C)


def upsample(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def upsample_bwd(d):
    B, H, W, C = d.shape
    return d.reshape(B, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4))


class UNetRef:
    def __init__(self, in_ch, out_ch, levels, base):
        self.in_ch, self.out_ch, self.L, self.base = in_ch, out_ch, levels, base
        self.shapes = []  # (name, shape) in parameter order
        for l in range(levels):
            c = base << l
            cin = in_ch if l == 0 else base << (l - 1)
            self.shapes += [(f"enc{l}a.w", (c, 3, 3, cin)), (f"enc{l}a.b", (c,)),
                            (f"enc{l}b.w", (c, 3, 3, c)), (f"enc{l}b.b", (c,))]
        for l in range(levels - 2, -1, -1):
            c = base << l
            self.shapes += [(f"dec{l}a.w", (c, 3, 3, (base << (l + 1)) + c)), (f"dec{l}a.b", (c,)),
                            (f"dec{l}b.w", (c, 3, 3, c)), (f"dec{l}b.b", (c,))]
        self.shapes += [("head.w", (out_ch, base)), ("head.b", (out_ch,))]

    def num_params(self):
        return int(sum(np.prod(s) for _, s in self.shapes))

    def unflatten(self, flat):
        out, off = {}, 0
        for name, s in self.shapes:
            n = int(np.prod(s))
            out[name] = np.asarray(flat[off:off + n], dtype=np.float64).reshape(s)
            off += n
        return out

    def flatten(self, d):
        return np.concatenate([d[name].ravel() for name, _ in self.shapes])

    def forward(self, p, x, rnd=None):
        """rnd (optional) rounds each stored activation, modelling reduced-precision storage."""
        r = rnd or (lambda v: v)
        cache = {"x": x}
        h = x
        for l in range(self.L):
            a = r(np.maximum(conv3x3(h, p[f"enc{l}a.w"], p[f"enc{l}a.b"]), 0))
            b = r(np.maximum(conv3x3(a, p[f"enc{l}b.w"], p[f"enc{l}b.b"]), 0))
            cache[f"enc{l}in"], cache[f"ea{l}"], cache[f"eb{l}"] = h, a, b
            if l + 1 < self.L:
                h, cache[f"arg{l}"] = maxpool(b)
        cur = cache[f"eb{self.L - 1}"]
        for l in range(self.L - 2, -1, -1):
            xin = np.concatenate([upsample(cur), cache[f"eb{l}"]], axis=3)
            a = r(np.maximum(conv3x3(xin, p[f"dec{l}a.w"], p[f"dec{l}a.b"]), 0))
            b = r(np.maximum(conv3x3(a, p[f"dec{l}b.w"], p[f"dec{l}b.b"]), 0))
            cache[f"din{l}"], cache[f"da{l}"], cache[f"db{l}"] = xin, a, b
            cur = b
        out = np.einsum("bhwc,oc->bhwo", cur, p["head.w"]) + p["head.b"]
        cache["top"] = cur
        return out, cache

    @staticmethod
    def loss(out, target, mask=None):
        m = np.ones_like(out) if mask is None else mask.astype(np.float64)
        cnt = max(m.sum(), 1.0)
        d = (out - target) * m
        return float((d * d).sum() / cnt), 2.0 * d / cnt

    def backward(self, p, cache, dout, rnd=None):
        """rnd (optional) rounds each stored activation gradient (as forward's rnd)."""
        r = rnd or (lambda v: v)
        g = {}
        top = cache["top"]
        g["head.w"] = np.einsum("bhwo,bhwc->oc", dout, top)
        g["head.b"] = dout.sum(axis=(0, 1, 2))
        dcur = r(np.einsum("bhwo,oc->bhwc", dout, p["head.w"]) * (top > 0))
        dskip = {}
        for l in range(self.L - 1):
            # decoder level l: db{l} = relu(conv(da{l})), da{l} = relu(conv([up(below) | eb{l}]))
            dx, g[f"dec{l}b.w"], g[f"dec{l}b.b"] = conv3x3_bwd(cache[f"da{l}"], p[f"dec{l}b.w"], dcur)
            dda = r(dx * (cache[f"da{l}"] > 0))
            dx, g[f"dec{l}a.w"], g[f"dec{l}a.b"] = conv3x3_bwd(cache[f"din{l}"], p[f"dec{l}a.w"], dda)
            cb = self.base << (l + 1)
            below = cache[f"eb{self.L - 1}"] if l == self.L - 2 else cache[f"db{l + 1}"]
            dskip[l] = r(dx[..., cb:] * (cache[f"eb{l}"] > 0))
            dup = r(dx[..., :cb] * (upsample(below) > 0))
            dcur = r(upsample_bwd(dup))
        deb = dcur  # gradient w.r.t. the bottom encoder output
        for l in range(self.L - 1, -1, -1):
            if l < self.L - 1:
                deb = r(dskip[l] + maxpool_bwd(cache[f"arg{l}"], dpool, cache[f"eb{l}"].shape) * (cache[f"eb{l}"] > 0))
            dx, g[f"enc{l}b.w"], g[f"enc{l}b.b"] = conv3x3_bwd(cache[f"ea{l}"], p[f"enc{l}b.w"], deb)
            dea = r(dx * (cache[f"ea{l}"] > 0))
            dx, g[f"enc{l}a.w"], g[f"enc{l}a.b"] = conv3x3_bwd(cache[f"enc{l}in"], p[f"enc{l}a.w"], dea)
            if l > 0:
                dpool = r(dx * (cache[f"enc{l}in"] > 0))
        return g

    def loss_and_grad(self, flat, x, target, mask=None, rnd=None):
        p = self.unflatten(flat)
        out, cache = self.forward(p, x, rnd)
        loss, dout = self.loss(out, target, mask)
        return loss, self.flatten(self.backward(p, cache, dout, rnd)), out
