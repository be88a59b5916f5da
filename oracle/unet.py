"""FP64 CPU oracle of the surrogate network's pieces and of the whole U-Net (numpy).

TEST INFRASTRUCTURE: only tests import it.  It shares no code with the CUDA kernels; it spells
each operation out from its definition.  Layouts follow include/surrogate.h: activations NHWC
(batch, H, W, C), 3x3 weights [tap][Cin][Cout] with tap = 3*(dy+1) + (dx+1), images periodic.
"""
from __future__ import annotations

import numpy as np

TAPS = [(dy, dx) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def shift(x, dy, dx):
    """x[b, (y+dy) mod H, (x+dx) mod W, c] as an array over (b, y, x, c)."""
    return np.roll(np.roll(x, -dy, axis=1), -dx, axis=2)


def conv3x3(x, w, bias=None, relu=False):
    """y[p, n] = sum_tap sum_k x[p + off(tap), k] w[tap, k, n] (+ bias) (ReLU)."""
    y = np.zeros(x.shape[:3] + (w.shape[2],))
    for t, (dy, dx) in enumerate(TAPS):
        y += np.einsum("bhwk,kn->bhwn", shift(x, dy, dx), w[t])
    if bias is not None:
        y = y + bias
    return np.maximum(y, 0.0) if relu else y


def conv3x3_bwd_data(dy, w):
    """dL/dx[p, k] = sum_tap sum_n dy[p - off(tap), n] w[tap, k, n]."""
    dx = np.zeros(dy.shape[:3] + (w.shape[1],))
    for t, (oy, ox) in enumerate(TAPS):
        dx += np.einsum("bhwn,kn->bhwk", shift(dy, -oy, -ox), w[t])
    return dx


def conv3x3_bwd_weight(x, dy):
    """dL/dw[tap, k, n] = sum_p x[p + off(tap), k] dy[p, n]."""
    return np.stack([np.einsum("bhwk,bhwn->kn", shift(x, oy, ox), dy) for (oy, ox) in TAPS])


def pool2(x):
    b, h, w, c = x.shape
    return x.reshape(b, h // 2, 2, w // 2, 2, c).mean(axis=(2, 4))


def pool2_bwd(dy):
    return np.repeat(np.repeat(dy, 2, axis=1), 2, axis=2) / 4.0


def up2(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def up2_bwd(dy):
    b, h, w, c = dy.shape
    return dy.reshape(b, h // 2, 2, w // 2, 2, c).sum(axis=(2, 4))


# --------------------------------------------------------------------------------------------
# The U-Net: per level l, channels ch[l]; encoder two conv+ReLU per level, 2x2 average pooling
# between levels; decoder: 2x upsampling, conv (no activation) to the finer level's channels,
# add the encoder skip, conv+ReLU; output conv to C_in channels, added to the input (residual).

def unet_layers(cin, ch):
    """Names and shapes (Cin, Cout) of the 3x3 convolutions, in forward order."""
    L = len(ch)
    layers = [("e0a", cin, ch[0]), ("e0b", ch[0], ch[0])]
    for l in range(1, L):
        layers += [(f"e{l}a", ch[l - 1], ch[l]), (f"e{l}b", ch[l], ch[l])]
    for l in range(L - 2, -1, -1):
        layers += [(f"u{l}", ch[l + 1], ch[l]), (f"d{l}", ch[l], ch[l])]
    layers += [("out", ch[0], cin)]
    return layers


def flux_update(out, x):
    """Prediction from the network output: phi' = phi - [Jx(x) - Jx(x-1) + Jy(y) - Jy(y-1)],
    u' = u + du, with (Jx, Jy, dux, duy) = out[..., 0:4] and (phi, ux, uy) = x[..., 0:3]."""
    jx, jy = out[..., 0], out[..., 1]
    div = (jx - np.roll(jx, 1, axis=2)) + (jy - np.roll(jy, 1, axis=1))
    return np.stack([x[..., 0] - div, x[..., 1] + out[..., 2], x[..., 2] + out[..., 3]], axis=-1)


def flux_update_bwd(dpred, C):
    """Adjoint of flux_update with respect to `out` (C channels)."""
    dphi = dpred[..., 0]
    dout = np.zeros(dpred.shape[:3] + (C,))
    dout[..., 0] = np.roll(dphi, -1, axis=2) - dphi
    dout[..., 1] = np.roll(dphi, -1, axis=1) - dphi
    dout[..., 2] = dpred[..., 1]
    dout[..., 3] = dpred[..., 2]
    return dout


def bf16_round(x):
    """x rounded to the nearest BF16 value (8 significant bits, ties to even), as float64: with
    x = m 2^e, 1/2 <= |m| < 1, the value round(256 m) 2^(e - 8); a carry to 256 m = 256 gives
    2^e, the next binade's first value.  (Below BF16's normal range, 2^-126, it keeps 8 bits
    where BF16 has fewer; no activation of the network comes near it.)"""
    m, e = np.frexp(np.asarray(x, dtype=np.float64))
    return np.ldexp(np.round(m * 256.0), e - 8)


def unet_forward(x, params, ch, bf16=False):
    """Returns (prediction = flux_update(net(x), x), cache of activations).  bf16: every
    activation the network stores in BF16 is rounded to it, once, from its exact value (pooled
    maps; convolution outputs after bias and ReLU; the decoder's sum of convolution, bias and
    skip); the output convolution and the prediction stay exact."""
    r = bf16_round if bf16 else (lambda v: v)
    L = len(ch)
    cache = {"x": x}
    h = x
    skips = []
    for l in range(L):
        if l > 0:
            h = r(pool2(h))
            cache[f"p{l}"] = h
        h = r(conv3x3(h, params[f"e{l}a"][0], params[f"e{l}a"][1], relu=True))
        cache[f"e{l}a"] = h
        h = r(conv3x3(h, params[f"e{l}b"][0], params[f"e{l}b"][1], relu=True))
        cache[f"e{l}b"] = h
        skips.append(h)
    for l in range(L - 2, -1, -1):
        up = up2(h)
        cache[f"up{l}"] = up
        t = conv3x3(up, params[f"u{l}"][0], params[f"u{l}"][1], relu=False)
        s = r(t + skips[l])
        cache[f"s{l}"] = s
        h = r(conv3x3(s, params[f"d{l}"][0], params[f"d{l}"][1], relu=True))
        cache[f"d{l}"] = h
    cache["top"] = h
    out = conv3x3(h, params["out"][0], params["out"][1], relu=False)
    return flux_update(out, x), cache


def unet_loss_and_grads(x, target, params, ch, bf16=False):
    """Mean squared error of the prediction (phi, ux, uy) against target, and the gradients of
    every weight and bias (reverse mode, written out layer by layer).  bf16: the forward of
    unet_forward(bf16=True), and every activation gradient the network stores in BF16 rounded
    to it once from its exact value (the output's gradient, each convolution's input gradient,
    the sums of a skip's and the decoder's gradients and of the 2x2 upsampling's four pixels);
    weight and bias gradients stay exact."""
    r = bf16_round if bf16 else (lambda v: v)
    pred, c = unet_forward(x, params, ch, bf16)
    L = len(ch)
    err = pred - target
    n = err.size
    loss = float((err ** 2).sum() / n)
    dout = r(flux_update_bwd(2.0 * err / n, x.shape[-1]))
    g = {}
    g["out"] = (conv3x3_bwd_weight(c["top"], dout), dout.sum(axis=(0, 1, 2)))
    dh = r(conv3x3_bwd_data(dout, params["out"][0]))
    dskip = [None] * L
    for l in range(0, L - 1):
        dh = dh * (c[f"d{l}"] > 0)
        g[f"d{l}"] = (conv3x3_bwd_weight(c[f"s{l}"], dh), dh.sum(axis=(0, 1, 2)))
        ds = r(conv3x3_bwd_data(dh, params[f"d{l}"][0]))
        dskip[l] = ds
        g[f"u{l}"] = (conv3x3_bwd_weight(c[f"up{l}"], ds), ds.sum(axis=(0, 1, 2)))
        dh = r(up2_bwd(r(conv3x3_bwd_data(ds, params[f"u{l}"][0]))))
    for l in range(L - 1, -1, -1):
        if dskip[l] is not None and l < L - 1:
            dh = r(dh + dskip[l])
        dh = dh * (c[f"e{l}b"] > 0)
        g[f"e{l}b"] = (conv3x3_bwd_weight(c[f"e{l}a"], dh), dh.sum(axis=(0, 1, 2)))
        dh = r(conv3x3_bwd_data(dh, params[f"e{l}b"][0]))
        dh = dh * (c[f"e{l}a"] > 0)
        inp = c[f"p{l}"] if l > 0 else c["x"]
        g[f"e{l}a"] = (conv3x3_bwd_weight(inp, dh), dh.sum(axis=(0, 1, 2)))
        if l > 0:
            dh = r(conv3x3_bwd_data(dh, params[f"e{l}a"][0]))
            dh = pool2_bwd(dh)  # a quarter of a BF16 value is one
    return loss, g
