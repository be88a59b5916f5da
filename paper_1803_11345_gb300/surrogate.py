"""Learned surrogate for the coupled Cahn-Hilliard--Navier-Stokes lattice Boltzmann solver.

A 4-level convolutional U-Net maps the macroscopic fields (phi, ux, uy) of a periodic lattice at
time t to time t + K (K solver steps).  Its phi update is the discrete divergence of a predicted
flux, so sum phi is conserved by construction (the Cahn-Hilliard equation, Eq. 1 of
arXiv:1803.11345, is a conservation law); velocities are updated additively.  Weights and
activations are BF16, accumulation FP32; every operation runs in the kernels behind
include/surrogate.h (3x3 convolutions on the BF16 tensor cores), trained with Adam on trajectories
the solver itself generates.  The solver stays the judge: a prediction is accepted only if its
sum phi drift and (where the solver is run to check it) its phi error stay under stated
thresholds; otherwise the solver advances the state instead.

PyTorch only allocates device memory and provides the stream.  The ctypes wrappers below keep the
C names of include/surrogate.h.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from . import lbm

_lib = lbm._lib

SUR_OK = 0
U_SCALE = 100.0  # velocities enter and leave the network multiplied by this (O(1) inputs)


def _sig(name, argtypes):
    f = getattr(_lib, name)
    f.argtypes = argtypes
    f.restype = ctypes.c_int
    return f


_vp, _i, _sz, _f = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t, ctypes.c_float
_sig("sur_conv3x3", [_vp, _vp, _vp, _vp, _i, _i, _i, _i, _i, _i, _i, _i, _i, _vp])
_sig("sur_conv3x3_wgrad", [_vp, _vp, _vp, _i, _i, _i, _i, _i, _vp])
_sig("sur_conv3x3_up_add", [_vp, _vp, _vp, _vp, _vp, _i, _i, _i, _i, _i, _vp])
_sig("sur_conv3x3_wgrad_up", [_vp, _vp, _vp, _i, _i, _i, _i, _i, _vp])
_sig("sur_relu_bwd", [_vp, _vp, _vp, _sz, _vp])
_sig("sur_bias_grad", [_vp, _vp, _i, _i, _vp])
for _n in ("sur_pool2", "sur_pool2_bwd", "sur_up2", "sur_up2_bwd"):
    _sig(_n, [_vp, _vp, _i, _i, _i, _i, _vp])
_sig("sur_add", [_vp, _vp, _vp, _sz, _vp])
_sig("sur_mse", [_vp, _vp, _vp, _vp, _vp, _i, _i, _i, _vp])
_sig("sur_adam", [_vp, _vp, _vp, _vp, _vp, _sz, _f, _f, _f, _f, _i, _vp])
_sig("sur_flux_update", [_vp, _vp, _vp, _i, _i, _i, _i, _vp])
_sig("sur_flux_update_bwd", [_vp, _vp, _i, _i, _i, _i, _vp])
_sig("sur_mse3", [_vp, _vp, _vp, _vp, _sz, _vp])
_sig("sur_zero", [_vp, _sz, _vp])
_sig("sur_cast_bf16", [_vp, _vp, _sz, _vp])
_sig("sur_pack_state", [_vp, _vp, _vp, _sz, _i, _f, _vp])
_sig("sur_unpack_state", [_vp, _vp, _sz, _f, _vp])
_sig("sur_phi_sums", [_vp, _i, _i, _i, _vp, _vp])
_sig("sur_phi_sq_diff", [_vp, _vp, _i, _i, _i, _vp, _vp])
_sig("sur_conv3x3_tc", [_vp, _vp, _vp, _vp, _vp, _i, _i, _i, _i, _i, _i, _i, _i, _vp])
_sig("sur_conv3x3_tc_supported", [_i, _i, _i, _i, _i, _i])
_sig("sur_transpose_taps", [_vp, _vp, _i, _i, _vp])
_sig("sur_check", [_vp])
SUR_ERR_TIMEOUT = -5


class SurError(RuntimeError):
    pass


def _ok(st, what):
    if st != SUR_OK:
        raise SurError(f"{what} failed with status {st}")


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


# Same-name wrappers (tensor arguments; the stream is an int handle).
def sur_conv3x3(x, w, bias, y, batch, H, W, K, N, transposed_weights, sgn, relu, out_f32, stream):
    _ok(_lib.sur_conv3x3(_p(x), _p(w), _p(bias), _p(y), batch, H, W, K, N, transposed_weights, sgn, relu, out_f32,
                         stream), "sur_conv3x3")


def sur_conv3x3_wgrad(x, dy, dw, batch, H, W, Cin, Cout, stream):
    _ok(_lib.sur_conv3x3_wgrad(_p(x), _p(dy), _p(dw), batch, H, W, Cin, Cout, stream), "sur_conv3x3_wgrad")


def sur_conv3x3_up_add(xc, w, bias, addend, y, batch, H, W, K, N, stream):
    _ok(_lib.sur_conv3x3_up_add(_p(xc), _p(w), _p(bias), _p(addend), _p(y), batch, H, W, K, N, stream),
        "sur_conv3x3_up_add")


def sur_conv3x3_wgrad_up(xc, dy, dw, batch, H, W, Cin, Cout, stream):
    _ok(_lib.sur_conv3x3_wgrad_up(_p(xc), _p(dy), _p(dw), batch, H, W, Cin, Cout, stream), "sur_conv3x3_wgrad_up")


def sur_relu_bwd(y, dy, dx, stream):
    _ok(_lib.sur_relu_bwd(_p(y), _p(dy), _p(dx), y.numel(), stream), "sur_relu_bwd")


def sur_bias_grad(dy, db, npix, C, stream):
    _ok(_lib.sur_bias_grad(_p(dy), _p(db), npix, C, stream), "sur_bias_grad")


def sur_pool2(x, y, batch, H, W, C, stream):
    _ok(_lib.sur_pool2(_p(x), _p(y), batch, H, W, C, stream), "sur_pool2")


def sur_pool2_bwd(dy, dx, batch, H, W, C, stream):
    _ok(_lib.sur_pool2_bwd(_p(dy), _p(dx), batch, H, W, C, stream), "sur_pool2_bwd")


def sur_up2(x, y, batch, H, W, C, stream):
    _ok(_lib.sur_up2(_p(x), _p(y), batch, H, W, C, stream), "sur_up2")


def sur_up2_bwd(dy, dx, batch, H, W, C, stream):
    _ok(_lib.sur_up2_bwd(_p(dy), _p(dx), batch, H, W, C, stream), "sur_up2_bwd")


def sur_add(a, b, y, stream):
    _ok(_lib.sur_add(_p(a), _p(b), _p(y), a.numel(), stream), "sur_add")


def sur_mse(out, xin, target, dout, loss, npix, C, used, stream):
    _ok(_lib.sur_mse(_p(out), _p(xin), _p(target), _p(dout), _p(loss), npix, C, used, stream), "sur_mse")


def sur_adam(w, grad, m, v, wb, lr, b1, b2, eps, step, stream):
    _ok(_lib.sur_adam(_p(w), _p(grad), _p(m), _p(v), _p(wb), w.numel(), lr, b1, b2, eps, step, stream), "sur_adam")


def sur_flux_update(out, base, pred, batch, H, W, C, stream):
    _ok(_lib.sur_flux_update(_p(out), _p(base), _p(pred), batch, H, W, C, stream), "sur_flux_update")


def sur_flux_update_bwd(dpred, dout, batch, H, W, C, stream):
    _ok(_lib.sur_flux_update_bwd(_p(dpred), _p(dout), batch, H, W, C, stream), "sur_flux_update_bwd")


def sur_mse3(pred, target, dpred, loss, stream):
    _ok(_lib.sur_mse3(_p(pred), _p(target), _p(dpred), _p(loss), pred.numel(), stream), "sur_mse3")


def sur_zero(t, stream):
    _ok(_lib.sur_zero(_p(t), t.numel() * t.element_size(), stream), "sur_zero")


def sur_cast_bf16(x, y, stream):
    _ok(_lib.sur_cast_bf16(_p(x), _p(y), x.numel(), stream), "sur_cast_bf16")


def sur_conv3x3_tc(x, wt, bias, addend, y, batch, H, W, K, N, relu, out_f32, upsampled, stream):
    _ok(_lib.sur_conv3x3_tc(_p(x), _p(wt), _p(bias), _p(addend), _p(y), batch, H, W, K, N, relu, out_f32,
                            upsampled, stream), "sur_conv3x3_tc")


def sur_conv3x3_tc_supported(batch, H, W, K, N, upsampled=0):
    return bool(_lib.sur_conv3x3_tc_supported(batch, H, W, K, N, upsampled))


def sur_transpose_taps(w, wt, K, N, stream):
    _ok(_lib.sur_transpose_taps(_p(w), _p(wt), K, N, stream), "sur_transpose_taps")


def sur_check(stream):
    """SUR_OK, or SUR_ERR_TIMEOUT if a bounded wait of a tensor-core kernel gave up (cleared)."""
    return _lib.sur_check(stream)


def sur_pack_state(state, x, base, npix, C, u_scale, stream):
    _ok(_lib.sur_pack_state(_p(state), _p(x), _p(base), npix, C, float(u_scale), stream), "sur_pack_state")


def sur_unpack_state(pred, state, npix, u_scale, stream):
    _ok(_lib.sur_unpack_state(_p(pred), _p(state), npix, float(u_scale), stream), "sur_unpack_state")


def sur_phi_sums(state, batch, npix, C, sums, stream):
    _ok(_lib.sur_phi_sums(_p(state), batch, npix, C, _p(sums), stream), "sur_phi_sums")


def sur_phi_sq_diff(a, b, batch, npix, C, sums, stream):
    _ok(_lib.sur_phi_sq_diff(_p(a), _p(b), batch, npix, C, _p(sums), stream), "sur_phi_sq_diff")


# ---------------------------------------------------------------------------------------------

def layer_specs(cin, ch):
    """(name, Cin, Cout) of every 3x3 convolution in forward order (same as the oracle)."""
    L = len(ch)
    layers = [("e0a", cin, ch[0]), ("e0b", ch[0], ch[0])]
    for l in range(1, L):
        layers += [(f"e{l}a", ch[l - 1], ch[l]), (f"e{l}b", ch[l], ch[l])]
    for l in range(L - 2, -1, -1):
        layers += [(f"u{l}", ch[l + 1], ch[l]), (f"d{l}", ch[l], ch[l])]
    layers += [("out", ch[0], cin)]
    return layers


class UNet:
    """The surrogate network on one CUDA device.  ``ch`` = channels per level (multiples of 16),
    ``cin`` = input/output channels (16; the first three carry phi, ux, uy)."""

    def __init__(self, ch=(32, 64, 128, 256), cin=16, seed=0, stream=None, device="cuda", tensor_cores=True):
        import torch
        self.torch = torch
        # forward convolutions on the tcgen05 kernel (sur_conv3x3_tc) where it serves the shape;
        # False: the mma.sync kernels only (the reference path of the same arithmetic)
        self.tensor_cores = tensor_cores
        self.sms = torch.cuda.get_device_properties(torch.device(device)).multi_processor_count
        self.autotune = True  # time each convolution shape on both kernels at its first use (outside capture)
        self._choice = {}
        self.ch, self.cin = tuple(ch), cin
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.s = self.stream.cuda_stream
        self.layers = layer_specs(cin, self.ch)
        rng = np.random.default_rng(seed)
        self.w, self.b, self.wb, self.gw, self.gb, self.mw, self.vw, self.mb, self.vb = ({} for _ in range(9))
        self.wt = {}  # K-major BF16 copies [tap][Cout][Cin] for the tcgen05 convolution
        f32 = dict(dtype=torch.float32, device=device)
        for name, ci, co in self.layers:
            scale = 0.0 if name == "out" else math.sqrt(2.0 / (9 * ci))  # He init; zero output layer
            w = rng.standard_normal((9, ci, co)) * scale
            self.w[name] = torch.tensor(w, **f32)
            self.b[name] = torch.empty(co, **f32)
            sur_zero(self.b[name], self.s)
            self.wb[name] = torch.empty((9, ci, co), dtype=torch.bfloat16, device=device)
            sur_cast_bf16(self.w[name], self.wb[name], self.s)
            self.wt[name] = torch.empty((9, co, ci), dtype=torch.bfloat16, device=device)
            sur_transpose_taps(self.wb[name], self.wt[name], ci, co, self.s)
            for d in (self.gw, self.mw, self.vw):
                d[name] = torch.empty((9, ci, co), **f32)
                sur_zero(d[name], self.s)
            for d in (self.gb, self.mb, self.vb):
                d[name] = torch.empty(co, **f32)
                sur_zero(d[name], self.s)
        self.step_count = 0
        self._bufs = {}

    # -- parameters as numpy (for checks) ------------------------------------------------------
    def params_numpy(self):
        """{name: (w FP64 from the BF16 copy, b FP64)} -- what the forward pass actually uses."""
        return {n: (self.wb[n].float().cpu().numpy().astype(np.float64), self.b[n].cpu().numpy().astype(np.float64))
                for n, _, _ in self.layers}

    def grads_numpy(self):
        return {n: (self.gw[n].cpu().numpy().astype(np.float64), self.gb[n].cpu().numpy().astype(np.float64))
                for n, _, _ in self.layers}

    # -- buffers -------------------------------------------------------------------------------
    def _buf(self, key, shape, dtype):
        t = self._bufs.get(key)
        if t is None or tuple(t.shape) != tuple(shape) or t.dtype != dtype:
            t = self.torch.empty(shape, dtype=dtype, device=self.w["out"].device)
            self._bufs[key] = t
        return t

    def _tc(self, B, H, W, ci, co, up=0):
        # Which kernel runs a convolution: the faster of the two on this GPU for the shape, timed
        # once outside graph capture (tune_layer) and cached.  Both give the same bits (same
        # accumulation order), so the choice changes only time.  Under capture, before a shape
        # was timed: the tcgen05 kernel on layers with at least one 128 x 128 output tile per SM
        # (its persistent CTAs take one SM each; smaller layers leave most SMs idle), which
        # measured within a few percent of the timed choice on the default network.
        if not self.tensor_cores or not sur_conv3x3_tc_supported(B, H, W, ci, co, up):
            return False
        key = (B, H, W, ci, co, up)
        if key not in self._choice and self.autotune and not self.torch.cuda.is_current_stream_capturing():
            self._choice[key] = self.tune_layer(B, H, W, ci, co, up)
        if key in self._choice:
            return self._choice[key]
        return B * H * W // 128 * max(1, co // 128) >= self.sms

    def tune_layer(self, B, H, W, ci, co, up=0, reps=10):
        """Time the tcgen05 and the mma.sync convolution of this shape (scratch tensors, the
        network's stream) and return True if the tcgen05 one is faster."""
        torch = self.torch
        dev = self.w["out"].device
        hs, ws = (H // 2, W // 2) if up else (H, W)
        x = torch.zeros((B, hs, ws, ci), dtype=torch.bfloat16, device=dev)
        wb = torch.zeros((9, ci, co), dtype=torch.bfloat16, device=dev)
        wt = torch.zeros((9, co, ci), dtype=torch.bfloat16, device=dev)
        b = torch.zeros(co, dtype=torch.float32, device=dev)
        y = torch.empty((B, H, W, co), dtype=torch.bfloat16, device=dev)
        add = torch.zeros((B, H, W, co), dtype=torch.bfloat16, device=dev) if up else None
        s = self.s
        runs = {
            True: lambda: sur_conv3x3_tc(x, wt, b, add, y, B, H, W, ci, co, 0 if up else 1, 0, up, s),
            False: ((lambda: sur_conv3x3_up_add(x, wb, b, add, y, B, H, W, ci, co, s)) if up else
                    (lambda: sur_conv3x3(x, wb, b, y, B, H, W, ci, co, 0, 1, 1, 0, s))),
        }
        ms = {}
        with torch.cuda.stream(self.stream):
            for k, fn in runs.items():
                for _ in range(3):
                    fn()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(self.stream)
                for _ in range(reps):
                    fn()
                e1.record(self.stream)
                e1.synchronize()
                ms[k] = e0.elapsed_time(e1)
        return ms[True] < ms[False]

    def _conv(self, x, name, B, H, W, relu, out_f32=False, key=None):
        _, ci, co = next(l for l in self.layers if l[0] == name)
        y = self._buf(key or name, (B, H, W, co), self.torch.float32 if out_f32 else self.torch.bfloat16)
        if self._tc(B, H, W, ci, co):
            sur_conv3x3_tc(x, self.wt[name], self.b[name], None, y, B, H, W, ci, co, int(relu), int(out_f32), 0, self.s)
        else:
            sur_conv3x3(x, self.wb[name], self.b[name], y, B, H, W, ci, co, 0, 1, int(relu), int(out_f32), self.s)
        return y

    # -- forward / backward --------------------------------------------------------------------
    def forward(self, x, base):
        """x: (B, H, W, cin) BF16 network input; base: (B, H, W, 3) FP32 state (phi, U_SCALE*ux,
        U_SCALE*uy) -> prediction (B, H, W, 3) FP32, the base advanced by the network."""
        bf = self.torch.bfloat16
        B, H, W, _ = x.shape
        L = len(self.ch)
        self._x = x
        self._shape = (B, H, W)
        h, hh, ww = x, H, W
        skips = []
        self._sizes = []
        for l in range(L):
            if l > 0:
                p = self._buf(f"p{l}", (B, hh // 2, ww // 2, self.ch[l - 1]), bf)
                sur_pool2(h, p, B, hh, ww, self.ch[l - 1], self.s)
                h, hh, ww = p, hh // 2, ww // 2
            self._sizes.append((hh, ww))
            h = self._conv(h, f"e{l}a", B, hh, ww, True)
            h = self._conv(h, f"e{l}b", B, hh, ww, True)
            skips.append(h)
        for l in range(L - 2, -1, -1):
            hh, ww = self._sizes[l]
            # s = conv(up2(h)) + skip in one kernel (upsampling read through the coarse index)
            sk = self._buf(f"s{l}", (B, hh, ww, self.ch[l]), bf)
            if self._tc(B, hh, ww, self.ch[l + 1], self.ch[l], 1):
                sur_conv3x3_tc(h, self.wt[f"u{l}"], self.b[f"u{l}"], skips[l], sk, B, hh, ww, self.ch[l + 1],
                               self.ch[l], 0, 0, 1, self.s)
            else:
                sur_conv3x3_up_add(h, self.wb[f"u{l}"], self.b[f"u{l}"], skips[l], sk, B, hh, ww, self.ch[l + 1],
                                   self.ch[l], self.s)
            h = self._conv(sk, f"d{l}", B, hh, ww, True)
        out = self._conv(h, "out", B, H, W, False, out_f32=True)
        pred = self._buf("pred", (B, H, W, 3), self.torch.float32)
        sur_flux_update(out, base, pred, B, H, W, self.cin, self.s)
        return pred

    def launches_per_forward(self):
        """Kernel launches of one forward pass: two convolutions per level, a pooling between
        levels, one fused decoder convolution and one convolution per decoder level, the output
        convolution and the flux update."""
        L = len(self.ch)
        return 2 * L + (L - 1) + 2 * (L - 1) + 2

    def capture_forward(self, x, base):
        """Capture one forward pass over the tensors x, base in a CUDA graph; returns (graph,
        pred).  Replaying the graph re-reads x and base in place and rewrites pred."""
        torch = self.torch
        self.forward(x, base)  # every buffer exists before the capture
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        old = self.s
        self.s = side.cuda_stream
        try:
            with torch.cuda.graph(g, stream=side):
                pred = self.forward(x, base)
        finally:
            self.s = old
        return g, pred

    def backward(self, dpred):
        """Accumulate the gradients of every weight and bias for dL/dpred (FP32, (B, H, W, 3))."""
        bf = self.torch.bfloat16
        B, H, W = self._shape
        L = len(self.ch)
        for n, _, _ in self.layers:
            sur_zero(self.gw[n], self.s)
            sur_zero(self.gb[n], self.s)
        dout = self._buf("dout", (B, H, W, self.cin), bf)
        sur_flux_update_bwd(dpred, dout, B, H, W, self.cin, self.s)

        def conv_back(name, inp, dy, hh, ww, want_dx=True, up=False):
            _, ci, co = next(l for l in self.layers if l[0] == name)
            (sur_conv3x3_wgrad_up if up else sur_conv3x3_wgrad)(inp, dy, self.gw[name], B, hh, ww, ci, co, self.s)
            sur_bias_grad(dy, self.gb[name], B * hh * ww, co, self.s)
            if not want_dx:
                return None
            dx = self._buf(f"dx_{name}", (B, hh, ww, ci), bf)
            sur_conv3x3(dy, self.wb[name], None, dx, B, hh, ww, co, ci, 1, -1, 0, 0, self.s)
            return dx

        bufs = self._bufs
        dh = conv_back("out", bufs["d0"] if L > 1 else bufs["e0b"], dout, H, W)
        dskip = [None] * L
        for l in range(0, L - 1):
            hh, ww = self._sizes[l]
            g = self._buf(f"gd{l}", dh.shape, bf)
            sur_relu_bwd(bufs[f"d{l}"], dh, g, self.s)
            ds = conv_back(f"d{l}", bufs[f"s{l}"], g, hh, ww)
            dskip[l] = ds
            src = bufs[f"d{l + 1}"] if l + 1 < L - 1 else bufs[f"e{L - 1}b"]  # coarse input of u{l}
            dup = conv_back(f"u{l}", src, ds, hh, ww, up=True)
            dc = self._buf(f"gup{l}", (B, hh // 2, ww // 2, self.ch[l + 1]), bf)
            sur_up2_bwd(dup, dc, B, hh // 2, ww // 2, self.ch[l + 1], self.s)
            dh = dc
        for l in range(L - 1, -1, -1):
            hh, ww = self._sizes[l]
            if dskip[l] is not None:
                t = self._buf(f"gsum{l}", dh.shape, bf)
                sur_add(dh, dskip[l], t, self.s)
                dh = t
            g = self._buf(f"geb{l}", dh.shape, bf)
            sur_relu_bwd(bufs[f"e{l}b"], dh, g, self.s)
            dh = conv_back(f"e{l}b", bufs[f"e{l}a"], g, hh, ww)
            g = self._buf(f"gea{l}", dh.shape, bf)
            sur_relu_bwd(bufs[f"e{l}a"], dh, g, self.s)
            inp = bufs[f"p{l}"] if l > 0 else self._x
            if l == 0:
                conv_back("e0a", inp, g, hh, ww, want_dx=False)
            else:
                dh = conv_back(f"e{l}a", inp, g, hh, ww)
                dp = self._buf(f"gp{l}", (B, hh * 2, ww * 2, self.ch[l - 1]), bf)
                sur_pool2_bwd(dh, dp, B, hh * 2, ww * 2, self.ch[l - 1], self.s)
                dh = dp

    def loss_and_grads(self, x, base, target):
        """Forward, MSE against target (B, H, W, 3) FP32, backward; returns the loss tensor."""
        pred = self.forward(x, base)
        loss = self._buf("loss", (1,), self.torch.float32)
        sur_zero(loss, self.s)
        dpred = self._buf("dpred", pred.shape, self.torch.float32)
        sur_mse3(pred, target, dpred, loss, self.s)
        self.backward(dpred)
        return loss

    def load_weights(self, name, w):
        """Set layer `name`'s FP32 weights, shape (9, Cin, Cout), and refresh its BF16 copy and the
        K-major copy the tcgen05 kernel reads."""
        _, ci, co = next(l for l in self.layers if l[0] == name)
        self.w[name].copy_(w)
        sur_cast_bf16(self.w[name], self.wb[name], self.s)
        sur_transpose_taps(self.wb[name], self.wt[name], ci, co, self.s)

    def adam_step(self, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.step_count += 1
        for n, ci, co in self.layers:
            sur_adam(self.w[n], self.gw[n], self.mw[n], self.vw[n], self.wb[n], lr, b1, b2, eps, self.step_count, self.s)
            sur_adam(self.b[n], self.gb[n], self.mb[n], self.vb[n], None, lr, b1, b2, eps, self.step_count, self.s)
            if self.tensor_cores:
                sur_transpose_taps(self.wb[n], self.wt[n], ci, co, self.s)


# ---------------------------------------------------------------------------------------------
# Solver <-> network data.

def pack_fields(phi, ux, uy, cin=16):
    """(B, H, W) phi, ux, uy -> (B, H, W, cin) FP32 network input (velocities scaled)."""
    phi = np.asarray(phi, dtype=np.float32)
    x = np.zeros(phi.shape + (cin,), dtype=np.float32)
    x[..., 0] = phi
    x[..., 1] = np.asarray(ux) * U_SCALE
    x[..., 2] = np.asarray(uy) * U_SCALE
    return x


def unpack_prediction(pred):
    """(B, H, W, 3) network prediction -> phi, ux, uy (FP64 numpy)."""
    p = np.asarray(pred, dtype=np.float64)
    return p[..., 0], p[..., 1] / U_SCALE, p[..., 2] / U_SCALE


def generate_trajectories(members, steps_per_window, windows, prec="fp32", stream=None):
    """Run the batched solver on `members` [(phi0, params)] and return the fields of every member
    at every window boundary: array (windows + 1, M, 3, H, W) of (phi, ux, uy)."""
    bat = lbm.Batch(members, prec=prec, stream=stream)
    M = len(members)
    ny, nx = members[0][0].shape
    out = np.zeros((windows + 1, M, 3, ny, nx), dtype=np.float32)

    def snap(k):
        for m in range(M):
            rho, ux, uy, phi = bat.fields(m)
            out[k, m, 0], out[k, m, 1], out[k, m, 2] = phi, ux, uy

    snap(0)
    for k in range(1, windows + 1):
        bat.step(steps_per_window)
        snap(k)
    st, flags = bat.check()
    bat.close()
    if st != lbm.LBM_OK:
        raise lbm.LbmError(st, f"non-finite members {flags}")
    return out


def generate_states(members, steps_per_window, windows, prec="fp32", stream=None, chunk=64):
    """Run the batched solver on `members` [(phi0, params)] and keep, on the device, the state of
    every member at every window boundary: tensor (windows + 1, M, H, W, 3) FP32 (phi, ux, uy).
    Members are stepped in batches of `chunk`; states go from the solver to the tensor with
    lbm_batch_get_state, so nothing crosses the host."""
    import torch
    M = len(members)
    ny, nx = members[0][0].shape
    out = torch.empty((windows + 1, M, ny, nx, 3), dtype=torch.float32, device="cuda")
    stream = stream if stream is not None else torch.cuda.Stream()
    for c0 in range(0, M, chunk):
        part = members[c0:c0 + chunk]
        bat = lbm.Batch(part, prec=prec, stream=stream)
        for k in range(windows + 1):
            if k:
                bat.step(steps_per_window)
            for m in range(len(part)):
                bat.get_state(m, out[k, c0 + m].data_ptr())
        st, flags = bat.check()
        bat.close()
        if st != lbm.LBM_OK:
            raise lbm.LbmError(st, f"non-finite members {flags}")
    torch.cuda.synchronize()
    return out


class Judge:
    """Decides whether the surrogate's prediction for a window is kept, with what is known while
    the model runs (rollout()):

    * every window, on the GPU in FP64 (sur_phi_sums): every phi finite and the sum-phi drift per
      node, |sum phi_pred - sum phi_in| / N, at most `drift`;
    * every `audit_every`-th window the solver also advances the window from the same input and
      the RMS phi difference between the prediction and the solver's result must stay at most
      `phi_err` (sur_phi_sq_diff).  The solver's result is kept in an audited window (it has been
      paid for); a failed audit hands the next `audit_every` windows to the solver.

    accept() applies the same thresholds offline, to a prediction whose solver result is known
    (evaluate()); a deployment has that result only in audited windows."""

    def __init__(self, phi_err=1e-2, drift=1e-6, audit_every=8):
        self.phi_err, self.drift, self.audit_every = phi_err, drift, int(audit_every)

    def accept(self, phi_in, phi_pred, phi_true=None):
        n = phi_in.size
        d = abs(float(np.sum(phi_pred, dtype=np.float64) - np.sum(phi_in, dtype=np.float64))) / n
        finite = bool(np.isfinite(phi_pred).all())
        err = None if phi_true is None or not finite else float(np.sqrt(np.mean((phi_pred - phi_true) ** 2)))
        ok = finite and d <= self.drift and (err is None or err <= self.phi_err)
        return ok, d, err


class SolverWindows:
    """The batched solver on a set of periodic lattices, advancing device states (B, H, W, 3) FP32
    (phi, ux, uy) by windows of K steps: each member restarts from the given fields (equilibrium
    populations, rho = 1, lbm_batch_set_state), runs K steps and writes its fields back
    (lbm_batch_get_state), all on `stream`."""

    def __init__(self, members, K, stream, prec="fp32"):
        self.bat = lbm.Batch(members, prec=prec, stream=stream)
        self.K, self.B = K, len(members)

    def advance(self, state, out, steps=None):
        for m in range(self.B):
            self.bat.set_state(m, state[m].data_ptr())
        self.bat.step(self.K if steps is None else steps)
        for m in range(self.B):
            self.bat.get_state(m, out[m].data_ptr())
        return out

    def close(self):
        self.bat.close()


def rollout(net, members, state0, windows, K, judge, stream=None, inject=None, graph=True):
    """Advance the lattices `members` [(phi0, params)] from state0 (torch (B, H, W, 3) FP32 on the
    device: phi, ux, uy) by `windows` windows of K solver steps with the surrogate, under `judge`,
    the solver advancing every window the judge does not keep.  Closed loop: each kept prediction
    is the next window's input.  Everything runs on one stream; the wall time includes the judge's
    reductions, its per-window read of 2B FP64 sums and every audit and fallback.  inject(w, pred)
    (optional) may alter the prediction of window w before it is judged (tests).  graph: the
    window's packing, network forward and unpacking replay as one CUDA graph over fixed buffers
    (captured before the timed loop; the states are copied, not swapped).
    While the host reads window w's sums, window w + 1 is already predicted from w's candidate
    (not next to an audit); if the judge rejects w, that speculation is dropped, w's saved input
    restored and the window handed to the solver, so the states are those of judging one window
    at a time.  Returns (state, stats)."""
    import time as _time

    import torch
    stream = stream if stream is not None else torch.cuda.Stream()
    B, H, W, _ = state0.shape
    npix = H * W
    net_stream = net.stream
    net.stream, net.s = stream, stream.cuda_stream
    solver = SolverWindows(members, K, stream)
    dev = state0.device
    x = torch.empty((B, H, W, net.cin), dtype=torch.bfloat16, device=dev)
    base = torch.empty((B, H, W, 3), dtype=torch.float32, device=dev)
    cand = torch.empty_like(base)
    solv = torch.empty_like(base)
    state = torch.empty_like(base)
    prev = torch.empty_like(base)  # input of the window being judged while the next is speculated
    sums = [torch.empty(2 * B, dtype=torch.float64, device=dev) for _ in range(2)]
    host = [torch.empty(2 * B, dtype=torch.float64, pin_memory=True) for _ in range(2)]
    done = [torch.cuda.Event() for _ in range(2)]
    aud = torch.empty(B, dtype=torch.float64, device=dev)
    s = stream.cuda_stream
    stats = dict(windows=windows, kept=0, solver=0, audits=0, audit_failed=0, drift_rejected=0, audit_rms=[])

    def is_audit(w):
        return judge.audit_every > 0 and w % judge.audit_every == judge.audit_every - 1

    try:
        with torch.cuda.stream(stream):
            state.copy_(state0)
            net.forward(x, base)  # buffers exist before timing

            def predict():  # state -> cand through the network
                sur_pack_state(state, x, base, B * npix, net.cin, U_SCALE, s)
                pred = net.forward(x, base)
                sur_unpack_state(pred, cand, B * npix, U_SCALE, s)

            g = None
            if graph:
                torch.cuda.synchronize()
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g, stream=stream):
                    predict()

            def launch(w):  # window w's prediction from state and its two sums, read back into host[w % 2]
                if g is not None:
                    g.replay()
                else:
                    predict()
                if inject is not None:
                    inject(w, cand)
                sb = sums[w % 2]
                sur_phi_sums(state, B, npix, 3, sb[:B], s)
                sur_phi_sums(cand, B, npix, 3, sb[B:], s)
                host[w % 2].copy_(sb, non_blocking=True)
                done[w % 2].record(stream)

            torch.cuda.synchronize()
            t0 = _time.perf_counter()
            suspended = 0
            pending = False
            for w in range(windows):
                if suspended:
                    solver.advance(state, solv)
                    state.copy_(solv)
                    stats["solver"] += 1
                    suspended -= 1
                    continue
                if not pending:
                    launch(w)
                spec = w + 1 < windows and not is_audit(w) and not is_audit(w + 1)
                if spec:  # assume w is kept: predict w + 1 from its candidate meanwhile
                    prev.copy_(state)
                    state.copy_(cand)
                    launch(w + 1)
                done[w % 2].synchronize()
                sv = host[w % 2].numpy()
                drift = np.abs(sv[B:] - sv[:B]) / npix
                if not (np.all(np.isfinite(sv)) and np.all(drift <= judge.drift)):
                    if spec:
                        state.copy_(prev)
                    solver.advance(state, solv)
                    state.copy_(solv)
                    stats["drift_rejected"] += 1
                    stats["solver"] += 1
                    pending = False
                    continue
                if is_audit(w):
                    solver.advance(state, solv)
                    sur_phi_sq_diff(cand, solv, B, npix, 3, aud, s)
                    rms = np.sqrt(aud.cpu().numpy() / npix)
                    stats["audits"] += 1
                    stats["audit_rms"].append(float(rms.max()))
                    if not rms.max() <= judge.phi_err:
                        stats["audit_failed"] += 1
                        suspended = judge.audit_every
                    state.copy_(solv)
                    pending = False
                    continue
                if not spec:
                    state.copy_(cand)
                stats["kept"] += 1
                pending = spec
            torch.cuda.synchronize()
            stats["seconds"] = _time.perf_counter() - t0
    finally:
        net.stream, net.s = net_stream, net_stream.cuda_stream
        solver.close()
    return state, stats


def solver_only(members, state0, windows, K, stream=None):
    """The same lattices advanced by the solver alone, windows * K steps from state0 (restarted from
    its fields as the rollout's solver windows are); returns (state, seconds)."""
    import time as _time

    import torch
    stream = stream if stream is not None else torch.cuda.Stream()
    solver = SolverWindows(members, K, stream)
    out = torch.empty_like(state0)
    try:
        with torch.cuda.stream(stream):
            torch.cuda.synchronize()
            t0 = _time.perf_counter()
            solver.advance(state0, out, steps=windows * K)
            torch.cuda.synchronize()
            dt = _time.perf_counter() - t0
    finally:
        solver.close()
    return out, dt


def phi_rms(a, b):
    """Per-lattice RMS phi difference of two device states (B, H, W, 3), reduced in FP64 on the GPU."""
    import torch
    B, H, W, _ = a.shape
    sums = torch.empty(B, dtype=torch.float64, device=a.device)
    stream = torch.cuda.current_stream()
    sur_phi_sq_diff(a, b, B, H * W, 3, sums, stream.cuda_stream)
    return np.sqrt(sums.cpu().numpy() / (H * W))


def states_from_trajectory(traj, window):
    """Device state (M, H, W, 3) FP32 of every member of traj at a window boundary."""
    import torch
    st = np.ascontiguousarray(np.moveaxis(traj[window], 1, -1)).astype(np.float32)
    return torch.from_numpy(st).cuda()


# ---------------------------------------------------------------------------------------------
# Training and evaluation on solver trajectories.

def spinodal_members(count, n, seed, nu_l=0.1, nu_g=0.01, a=0.04, gamma=0.04, M=0.1):
    """Periodic spinodal decomposition members (viscosity ratio nu_l/nu_g, tau linear in phi)."""
    from . import workloads as W
    tau = lambda nu: 3.0 * nu + 0.5  # noqa: E731
    return [(W.spinodal(n, n, seed=seed + k),
             dict(tau_l=tau(nu_l), tau_g=tau(nu_g), visc=lbm.LBM_TAU_LINEAR, a=a, gamma=gamma, M=M))
            for k in range(count)]


def to_device_batch(traj, idx, cin=16):
    """Network input (BF16), FP32 base state and FP32 target for (member, window) pairs."""
    import torch
    xs = np.stack([pack_fields(traj[k, m, 0], traj[k, m, 1], traj[k, m, 2], cin) for m, k in idx])
    ys = np.stack([pack_fields(traj[k + 1, m, 0], traj[k + 1, m, 1], traj[k + 1, m, 2], 3) for m, k in idx])
    xf = torch.from_numpy(xs).cuda()
    x = xf.to(torch.bfloat16)
    base = xf[..., :3].contiguous()
    y = torch.from_numpy(ys).cuda()
    return x, base, y


def train(net, traj, iters, batch, lr=1e-3, seed=0, log_every=0):
    """Adam on random (member, window) pairs of traj (windows+1, M, 3, H, W); cosine-decayed lr.
    Returns the loss history (one value per iteration, synchronised every log_every)."""
    rng = np.random.default_rng(seed)
    nwin, M = traj.shape[0] - 1, traj.shape[1]
    hist = []
    for it in range(iters):
        idx = [(int(rng.integers(M)), int(rng.integers(nwin))) for _ in range(batch)]
        x, base, y = to_device_batch(traj, idx, net.cin)
        loss = net.loss_and_grads(x, base, y)
        net.adam_step(lr=lr * 0.5 * (1 + math.cos(math.pi * it / max(1, iters))))
        if log_every and (it % log_every == 0 or it == iters - 1):
            hist.append((it, float(loss.item())))
    return hist


def trajectory_states(traj):
    """All snapshots of traj (windows+1, M, 3, H, W) as one device tensor (windows+1, M, H, W, 3)
    FP32 of solver states (phi, ux, uy), the layout the surrogate kernels read."""
    import torch
    return torch.from_numpy(np.ascontiguousarray(np.moveaxis(traj, 2, -1)).astype(np.float32)).cuda()


def train_states(net, states, iters, batch, lr=1e-3, seed=0, log_every=0):
    """Adam on random (window, member) pairs of device states (windows+1, M, H, W, 3): the input
    and its target (the state one window later) are packed on the GPU (sur_pack_state), so no
    training data crosses the host.  Cosine-decayed lr; returns the loss history."""
    import torch
    rng = np.random.default_rng(seed)
    nwin, M, H, W, _ = states.shape
    nwin -= 1
    npix = batch * H * W
    dev = states.device
    x = torch.empty((batch, H, W, net.cin), dtype=torch.bfloat16, device=dev)
    xt = torch.empty_like(x)
    base = torch.empty((batch, H, W, 3), dtype=torch.float32, device=dev)
    tgt = torch.empty_like(base)
    hist = []
    s = net.s
    for it in range(iters):
        ks = torch.from_numpy(rng.integers(nwin, size=batch)).to(dev)
        ms = torch.from_numpy(rng.integers(M, size=batch)).to(dev)
        inp = states[ks, ms].contiguous()
        out = states[ks + 1, ms].contiguous()
        sur_pack_state(inp, x, base, npix, net.cin, U_SCALE, s)
        sur_pack_state(out, xt, tgt, npix, net.cin, U_SCALE, s)
        loss = net.loss_and_grads(x, base, tgt)
        net.adam_step(lr=lr * 0.5 * (1 + math.cos(math.pi * it / max(1, iters))))
        if log_every and (it % log_every == 0 or it == iters - 1):
            hist.append((it, float(loss.item())))
    return hist


def one_window_errors(net, states, batch=4):
    """RMS phi error of one-window predictions from every true state of device states
    (windows+1, M, H, W, 3), and of persistence (phi(t+K) ~ phi(t)): two arrays (windows * M)."""
    import torch
    nwin, M, H, W, _ = states.shape
    nwin -= 1
    dev = states.device
    errs, pers = [], []
    pairs = [(k, m) for k in range(nwin) for m in range(M)]
    for i in range(0, len(pairs), batch):
        idx = pairs[i:i + batch]
        b = len(idx)
        inp = torch.stack([states[k, m] for k, m in idx]).contiguous()
        out = torch.stack([states[k + 1, m] for k, m in idx]).contiguous()
        x = torch.empty((b, H, W, net.cin), dtype=torch.bfloat16, device=dev)
        base = torch.empty((b, H, W, 3), dtype=torch.float32, device=dev)
        pred_state = torch.empty_like(base)
        sur_pack_state(inp, x, base, b * H * W, net.cin, U_SCALE, net.s)
        pred = net.forward(x, base)
        sur_unpack_state(pred, pred_state, b * H * W, U_SCALE, net.s)
        errs += phi_rms(pred_state, out).tolist()
        pers += phi_rms(inp, out).tolist()
    return np.array(errs), np.array(pers)


def evaluate(net, traj, judge, batch=4):
    """One-window predictions from every true state of traj: per window the RMS phi error of the
    network and of persistence (phi(t+K) ~ phi(t)), the sum-phi drift per node, and whether the
    judge accepts the prediction (a rejected window is advanced by the solver instead, so the
    state after fallback is exact)."""
    nwin, M = traj.shape[0] - 1, traj.shape[1]
    rows = []
    pairs = [(m, k) for k in range(nwin) for m in range(M)]
    for i in range(0, len(pairs), batch):
        idx = pairs[i:i + batch]
        x, base, _ = to_device_batch(traj, idx, net.cin)
        pred = net.forward(x, base).cpu().numpy()
        for j, (m, k) in enumerate(idx):
            phi_in = traj[k, m, 0].astype(np.float64)
            phi_true = traj[k + 1, m, 0].astype(np.float64)
            phi_pred = pred[j, ..., 0].astype(np.float64)
            ok, drift, err = judge.accept(phi_in, phi_pred, phi_true)
            pers = float(np.sqrt(np.mean((phi_in - phi_true) ** 2)))
            rows.append(dict(member=m, window=k, err=err, persistence=pers, drift=drift, accepted=bool(ok)))
    return rows


def time_forward(net, x, base, reps=5, graph=False):
    """Milliseconds per forward pass of the batch x (CUDA events on the stream that runs it:
    the network's stream, or with graph=True the current stream replaying a captured forward)."""
    import torch
    if graph:
        g, _ = net.capture_forward(x, base)
        stream = torch.cuda.current_stream()
        run = g.replay
    else:
        stream = net.stream
        run = lambda: net.forward(x, base)  # noqa: E731
    for _ in range(2):
        run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        run()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def _main(argv=None):
    """Time the forward pass of the default network on a random batch (eager and graph-replayed),
    or with --layer H,Cin,Cout[,up] one 3x3 convolution of that shape (up: read through the 2x
    upsampling of an H/2 image, with a skip addend) on the tcgen05 kernel and on the mma.sync one."""
    import argparse

    import torch
    ap = argparse.ArgumentParser(description=_main.__doc__)
    ap.add_argument("--batch", type=int, default=4)
    ap.add_argument("--n", type=int, default=256, help="image side")
    ap.add_argument("--reps", type=int, default=10)
    ap.add_argument("--layer", type=str, default="", help="H,Cin,Cout[,up]: time one convolution")
    ap.add_argument("--kernel", choices=["both", "tc", "mma"], default="both")
    ap.add_argument("--mma-sync", action="store_true", help="network forward on the mma.sync kernels only")
    a = ap.parse_args(argv)
    s = torch.cuda.current_stream().cuda_stream
    if a.layer:
        parts = [int(v) for v in a.layer.split(",")]
        H, ci, co = parts[:3]
        up = parts[3] if len(parts) > 3 else 0
        g = torch.Generator(device="cuda").manual_seed(1)
        hs = H // 2 if up else H
        x = torch.randn((a.batch, hs, hs, ci), device="cuda", generator=g).to(torch.bfloat16)
        w = (torch.randn((9, ci, co), device="cuda", generator=g) * 0.1).to(torch.bfloat16)
        wt = torch.empty((9, co, ci), dtype=torch.bfloat16, device="cuda")
        sur_transpose_taps(w, wt, ci, co, s)
        b = torch.zeros(co, device="cuda")
        y = torch.empty((a.batch, H, H, co), dtype=torch.bfloat16, device="cuda")
        add = torch.zeros((a.batch, H, H, co), dtype=torch.bfloat16, device="cuda") if up else None
        runs = {}
        if a.kernel in ("both", "tc"):
            runs["tcgen05"] = lambda: sur_conv3x3_tc(x, wt, b, add, y, a.batch, H, H, ci, co, 0 if up else 1, 0, up, s)
        if a.kernel in ("both", "mma"):
            runs["mma.sync"] = ((lambda: sur_conv3x3_up_add(x, w, b, add, y, a.batch, H, H, ci, co, s)) if up else
                                (lambda: sur_conv3x3(x, w, b, y, a.batch, H, H, ci, co, 0, 1, 1, 0, s)))
        flop = 2.0 * 9 * ci * co * a.batch * H * H
        for name, fn in runs.items():
            for _ in range(3):
                fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(a.reps):
                fn()
            e1.record()
            torch.cuda.synchronize()
            us = e0.elapsed_time(e1) / a.reps * 1e3
            print(f"{name}: batch {a.batch} {H}x{H} {ci}->{co}{' (upsampled, skip)' if up else ''}: {us:.1f} us, "
                  f"{flop / us / 1e6:.0f} TFLOP/s")
        if sur_check(s) != SUR_OK:
            raise SurError("a bounded wait of the tensor-core kernel gave up")
        return
    net = UNet(ch=(32, 64, 128, 256), cin=16, seed=1, tensor_cores=not a.mma_sync)
    g = torch.Generator(device="cuda").manual_seed(1)
    x = torch.randn((a.batch, a.n, a.n, 16), device="cuda", generator=g).to(torch.bfloat16)
    base = x[..., :3].float().contiguous()
    eager = time_forward(net, x, base, reps=a.reps)
    graph = time_forward(net, x, base, reps=a.reps, graph=True)
    print(f"batch {a.batch} image {a.n}x{a.n}: {eager:.4f} ms/forward eager, {graph:.4f} ms/forward graph "
          f"({net.launches_per_forward()} launches per forward, "
          f"{'mma.sync' if a.mma_sync else 'faster kernel per layer, timed'})")


if __name__ == "__main__":
    _main()
