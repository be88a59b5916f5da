"""Pins of the surrogate network's FP64 oracle (oracle/unet.py): the periodic 3x3 convolution
against circular correlation by FFT, every backward pass against its forward by the adjoint
identity <A x, y> = <x, A^T y>, exact conservation of the flux update, and the whole U-Net's
gradient against central finite differences."""
import numpy as np
import pytest

from oracle import unet as U


def _rng(seed):
    return np.random.default_rng(seed)


def test_conv_equals_fft_circular_correlation():
    rng = _rng(1)
    B, H, W, K, N = 2, 8, 12, 3, 4
    x = rng.standard_normal((B, H, W, K))
    w = rng.standard_normal((9, K, N))
    y = U.conv3x3(x, w)
    # y(p) = sum_off x(p + off) w(off): circular cross-correlation, FFT(x) * conj(FFT(w_img)).
    want = np.zeros_like(y)
    X = np.fft.fft2(x, axes=(1, 2))
    for k in range(K):
        for n in range(N):
            img = np.zeros((H, W))
            for t, (dy, dx) in enumerate(U.TAPS):
                img[dy % H, dx % W] += w[t, k, n]
            want[..., n] += np.real(np.fft.ifft2(X[..., k] * np.conj(np.fft.fft2(img)), axes=(1, 2)))
    np.testing.assert_allclose(y, want, atol=1e-12)


def test_conv_backward_passes_are_adjoints():
    rng = _rng(2)
    B, H, W, K, N = 2, 6, 8, 5, 3
    x = rng.standard_normal((B, H, W, K))
    w = rng.standard_normal((9, K, N))
    dy = rng.standard_normal((B, H, W, N))
    lhs = np.sum(U.conv3x3(x, w) * dy)
    assert np.isclose(lhs, np.sum(x * U.conv3x3_bwd_data(dy, w)), rtol=1e-12)
    assert np.isclose(lhs, np.sum(w * U.conv3x3_bwd_weight(x, dy)), rtol=1e-12)


def test_pool_and_upsample_adjoints():
    rng = _rng(3)
    x = rng.standard_normal((2, 8, 6, 3))
    y = rng.standard_normal((2, 4, 3, 3))
    assert np.isclose(np.sum(U.pool2(x) * y), np.sum(x * U.pool2_bwd(y)), rtol=1e-12)
    assert np.isclose(np.sum(U.up2(y) * x), np.sum(y * U.up2_bwd(x)), rtol=1e-12)
    np.testing.assert_allclose(U.pool2(U.up2(y)), y, atol=1e-15)


def test_flux_update_conserves_phi_and_is_adjoint():
    rng = _rng(4)
    x = rng.standard_normal((2, 6, 10, 16))
    out = rng.standard_normal((2, 6, 10, 16))
    pred = U.flux_update(out, x)
    assert np.allclose(pred[..., 0].sum(axis=(1, 2)), x[..., 0].sum(axis=(1, 2)), atol=1e-12)
    d = rng.standard_normal(pred.shape)
    base = U.flux_update(np.zeros_like(out), x)
    assert np.isclose(np.sum((pred - base) * d), np.sum(out * U.flux_update_bwd(d, 16)), rtol=1e-12)


def _tiny_net(seed, ch=(4, 6, 8), cin=5):
    rng = _rng(seed)
    return {n: (rng.standard_normal((9, ci, co)) * 0.3, rng.standard_normal(co) * 0.1)
            for n, ci, co in U.unet_layers(cin, ch)}


def test_unet_gradient_against_finite_differences():
    ch, cin = (4, 6, 8), 5
    params = _tiny_net(5, ch, cin)
    rng = _rng(6)
    x = rng.standard_normal((2, 8, 8, cin))
    target = rng.standard_normal((2, 8, 8, 3))
    loss, g = U.unet_loss_and_grads(x, target, params, ch)
    assert set(g) == set(params)
    h = 1e-6
    for name in ("e0a", "e1b", "e2a", "u1", "d0", "out"):
        w, b = params[name]
        for idx in [(0, 0, 0), (4, w.shape[1] - 1, w.shape[2] - 1), (8, 1, 1)]:
            w2 = w.copy()
            w2[idx] += h
            lp, _ = U.unet_forward(x, {**params, name: (w2, b)}, ch)
            w2[idx] -= 2 * h
            lm, _ = U.unet_forward(x, {**params, name: (w2, b)}, ch)
            fd = (np.mean((lp - target) ** 2) - np.mean((lm - target) ** 2)) / (2 * h)
            assert np.isclose(g[name][0][idx], fd, rtol=2e-5, atol=1e-9), (name, idx)
        b2 = b.copy()
        b2[0] += h
        lp, _ = U.unet_forward(x, {**params, name: (w, b2)}, ch)
        b2[0] -= 2 * h
        lm, _ = U.unet_forward(x, {**params, name: (w, b2)}, ch)
        fd = (np.mean((lp - target) ** 2) - np.mean((lm - target) ** 2)) / (2 * h)
        assert np.isclose(g[name][1][0], fd, rtol=2e-5, atol=1e-9), name


def test_bf16_round_is_round_to_nearest_even():
    """The oracle's BF16 rounding against the library's single rounding of FP32 values to BF16
    (torch on the CPU): random FP32 values over 40 binades, exact ties (which go to the even
    8-bit significand) and the carry into the next binade; and idempotence."""
    import torch
    rng = np.random.default_rng(5)
    x32 = (rng.standard_normal(100000) * np.exp(rng.uniform(-20, 20, 100000))).astype(np.float32)
    ties = np.array([(128 + k + 0.5) * 2.0 ** -8 for k in range(128)], dtype=np.float32)  # m*256 = k + 1/2
    carry = np.array([255.5 * 2.0 ** -8, -255.75 * 2.0 ** -8, 255.25 * 2.0 ** -8], dtype=np.float32)
    for v in (x32, ties, carry):
        want = torch.from_numpy(v).to(torch.bfloat16).to(torch.float64).numpy()
        got = U.bf16_round(v.astype(np.float64))
        assert np.array_equal(got, want)
    assert np.array_equal(U.bf16_round(U.bf16_round(x32.astype(np.float64))), U.bf16_round(x32.astype(np.float64)))
    assert U.bf16_round(np.array([255.5 * 2.0 ** -8]))[0] == 1.0  # tie at 255.5 rounds to even 256: the carry
