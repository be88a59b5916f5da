"""Surrogate kernels (include/surrogate.h) against the FP64 network oracle (oracle/unet.py).
Inputs are rounded to BF16 first and handed to the oracle exactly, so the kernels' only
departures are FP32 accumulation order (and BF16 rounding of BF16 outputs)."""
import numpy as np
import pytest

from oracle import unet as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1803_11345_gb300 import build
    build.build()
    from paper_1803_11345_gb300 import surrogate as mod
    return mod


def _bf(rng, shape, scale=1.0):
    """Random BF16 tensor on the GPU and its exact FP64 value."""
    import torch
    t = torch.tensor(rng.standard_normal(shape) * scale, dtype=torch.float32).to(torch.bfloat16).cuda()
    return t, t.float().cpu().numpy().astype(np.float64)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))



@pytest.mark.parametrize("K,N", [(16, 16), (16, 32), (32, 64), (48, 96)])
def test_conv_forward_backward_match_oracle(S, K, N):
    import torch
    rng = np.random.default_rng(K * 100 + N)
    B, H, W = 2, 8, 12  # 192 pixels: not a multiple of the 128-pixel tile
    s = torch.cuda.current_stream().cuda_stream
    x, xn = _bf(rng, (B, H, W, K))
    w, wn = _bf(rng, (9, K, N), 0.2)
    bias = torch.tensor(rng.standard_normal(N), dtype=torch.float32).cuda()
    y = torch.empty((B, H, W, N), dtype=torch.float32, device="cuda")
    S.sur_conv3x3(x, w, bias, y, B, H, W, K, N, 0, 1, 1, 1, s)
    want = U.conv3x3(xn, wn, bias.cpu().numpy().astype(np.float64), relu=True)
    assert _rel(y.cpu().numpy(), want) < 1e-5
    dy, dyn = _bf(rng, (B, H, W, N))
    dx = torch.empty((B, H, W, K), dtype=torch.float32, device="cuda")
    S.sur_conv3x3(dy, w, None, dx, B, H, W, N, K, 1, -1, 0, 1, s)
    assert _rel(dx.cpu().numpy(), U.conv3x3_bwd_data(dyn, wn)) < 1e-5
    dw = torch.zeros((9, K, N), dtype=torch.float32, device="cuda")
    S.sur_conv3x3_wgrad(x, dy, dw, B, H, W, K, N, s)
    assert _rel(dw.cpu().numpy(), U.conv3x3_bwd_weight(xn, dyn)) < 1e-5
    ybf = torch.empty((B, H, W, N), dtype=torch.bfloat16, device="cuda")
    S.sur_conv3x3(x, w, bias, ybf, B, H, W, K, N, 0, 1, 1, 0, s)
    assert _rel(ybf.float().cpu().numpy(), want) < 4e-3


@pytest.mark.parametrize("K,N", [(16, 16), (64, 32), (32, 128), (256, 128)])
def test_fused_decoder_conv_matches_oracle(S, K, N):
    """conv3x3(up2(xc)) + bias + skip in one kernel, and its weight gradient read through the
    coarse image, against the oracle's separate up2 / conv3x3 / add."""
    import torch
    rng = np.random.default_rng(K * 7 + N)
    B, H, W = 2, 10, 14  # 280 fine pixels: three 128-pixel tiles, the last one ragged
    s = torch.cuda.current_stream().cuda_stream
    xc, xcn = _bf(rng, (B, H // 2, W // 2, K))
    w, wn = _bf(rng, (9, K, N), 0.2)
    bias = torch.tensor(rng.standard_normal(N), dtype=torch.float32).cuda()
    skip, skipn = _bf(rng, (B, H, W, N))
    y = torch.empty((B, H, W, N), dtype=torch.bfloat16, device="cuda")
    S.sur_conv3x3_up_add(xc, w, bias, skip, y, B, H, W, K, N, s)
    want = U.conv3x3(U.up2(xcn), wn, bias.cpu().numpy().astype(np.float64)) + skipn
    assert _rel(y.float().cpu().numpy(), want) < 4e-3
    y2 = torch.empty_like(y)
    S.sur_conv3x3_up_add(xc, w, None, None, y2, B, H, W, K, N, s)
    assert _rel(y2.float().cpu().numpy(), U.conv3x3(U.up2(xcn), wn)) < 4e-3
    dy, dyn = _bf(rng, (B, H, W, N))
    dw = torch.zeros((9, K, N), dtype=torch.float32, device="cuda")
    S.sur_conv3x3_wgrad_up(xc, dy, dw, B, H, W, K, N, s)
    assert _rel(dw.cpu().numpy(), U.conv3x3_bwd_weight(U.up2(xcn), dyn)) < 1e-5
    with pytest.raises(S.SurError):  # odd fine sizes have no coarse image
        S.sur_conv3x3_up_add(xc, w, None, None, y2, B, H - 1, W, K, N, s)


def test_elementwise_kernels_match_oracle(S):
    import torch
    rng = np.random.default_rng(7)
    B, H, W, C = 2, 8, 6, 16
    s = torch.cuda.current_stream().cuda_stream
    x, xn = _bf(rng, (B, H, W, C))
    p = torch.empty((B, H // 2, W // 2, C), dtype=torch.bfloat16, device="cuda")
    S.sur_pool2(x, p, B, H, W, C, s)
    assert _rel(p.float().cpu().numpy(), U.pool2(xn)) < 4e-3
    c, cn = _bf(rng, (B, H // 2, W // 2, C))
    u = torch.empty((B, H, W, C), dtype=torch.bfloat16, device="cuda")
    S.sur_up2(c, u, B, H // 2, W // 2, C, s)
    assert np.array_equal(u.float().cpu().numpy(), U.up2(cn))
    g = torch.empty_like(x)
    S.sur_pool2_bwd(c, g, B, H, W, C, s)
    assert _rel(g.float().cpu().numpy(), U.pool2_bwd(cn)) < 1e-12
    gc = torch.empty_like(c)
    S.sur_up2_bwd(x, gc, B, H // 2, W // 2, C, s)
    assert _rel(gc.float().cpu().numpy(), U.up2_bwd(xn)) < 4e-3
    y, yn = _bf(rng, (B, H, W, C))
    r = torch.empty_like(x)
    S.sur_relu_bwd(y, x, r, s)
    assert np.array_equal(r.float().cpu().numpy(), xn * (yn > 0))
    db = torch.zeros(C, dtype=torch.float32, device="cuda")
    S.sur_bias_grad(x, db, B * H * W, C, s)
    assert _rel(db.cpu().numpy(), xn.sum(axis=(0, 1, 2))) < 1e-5
    out = torch.tensor(rng.standard_normal((B, H, W, C)), dtype=torch.float32).cuda()
    base = torch.tensor(rng.standard_normal((B, H, W, 3)), dtype=torch.float32).cuda()
    bn = base.cpu().numpy().astype(np.float64)
    pred = torch.empty((B, H, W, 3), dtype=torch.float32, device="cuda")
    S.sur_flux_update(out, base, pred, B, H, W, C, s)
    want = U.flux_update(out.cpu().numpy().astype(np.float64), bn)
    assert _rel(pred.cpu().numpy(), want) < 1e-6
    assert abs(pred[..., 0].double().sum().item() - bn[..., 0].sum()) < 1e-4
    dpred = torch.tensor(rng.standard_normal((B, H, W, 3)), dtype=torch.float32).cuda()
    dout = torch.empty((B, H, W, C), dtype=torch.bfloat16, device="cuda")
    S.sur_flux_update_bwd(dpred, dout, B, H, W, C, s)
    assert _rel(dout.float().cpu().numpy(), U.flux_update_bwd(dpred.cpu().numpy().astype(np.float64), C)) < 4e-3


def test_adam_step_follows_the_published_rule(S):
    """Adam (Kingma & Ba 2015): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
    w -= lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps)."""
    import torch
    rng = np.random.default_rng(8)
    n = 1000
    w0, g = rng.standard_normal(n), rng.standard_normal(n)
    w = torch.tensor(w0, dtype=torch.float32).cuda()
    gr = torch.tensor(g, dtype=torch.float32).cuda()
    m = torch.zeros(n, dtype=torch.float32, device="cuda")
    v = torch.zeros_like(m)
    wb = torch.empty(n, dtype=torch.bfloat16, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    mn, vn, wn = np.zeros(n), np.zeros(n), w0.copy()
    for t in (1, 2, 3):
        S.sur_adam(w, gr, m, v, wb, 1e-2, 0.9, 0.999, 1e-8, t, s)
        mn = 0.9 * mn + 0.1 * g
        vn = 0.999 * vn + 0.001 * g * g
        wn = wn - 1e-2 * (mn / (1 - 0.9 ** t)) / (np.sqrt(vn / (1 - 0.999 ** t)) + 1e-8)
    np.testing.assert_allclose(w.cpu().numpy(), wn, rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(wb.float().cpu().numpy(), wn, rtol=1e-2, atol=1e-2)


def test_unet_gradients_match_oracle(S):
    """Whole-network forward and backward on the GPU (BF16 activations, FP32 accumulation)
    against the FP64 oracle with the same BF16 weights.  Each kernel is checked to 1e-5 above;
    here the network's wiring is checked.  The GPU rounds every activation and activation
    gradient to BF16 (2^-9 relative) about twenty times along the deepest path and ReLU masks
    flip on pre-activations within that rounding of zero, so the deepest layer's gradient is
    held to 10% relative and cosine > 0.99 (a wiring error gives cosine far from 1)."""
    import torch
    ch, cin = (16, 32, 32), 16
    net = S.UNet(ch=ch, cin=cin, seed=3)
    rng = np.random.default_rng(9)
    # a non-zero output layer, so every layer receives gradient
    net.load_weights("out", torch.tensor(rng.standard_normal((9, ch[0], cin)) * 0.1, dtype=torch.float32).cuda())
    B, H, W = 2, 16, 16
    x, xn = _bf(rng, (B, H, W, cin), 0.5)
    base = x[..., :3].float().contiguous()
    target = torch.tensor(rng.standard_normal((B, H, W, 3)) * 0.1, dtype=torch.float32).cuda()
    loss = net.loss_and_grads(x, base, target)
    torch.cuda.synchronize()
    params = net.params_numpy()
    lo, go = U.unet_loss_and_grads(xn, target.cpu().numpy().astype(np.float64), params, ch)
    assert abs(loss.item() - lo) / lo < 1e-2
    gg = net.grads_numpy()
    for name, _, _ in S.layer_specs(cin, ch):
        a, b = gg[name][0].ravel(), go[name][0].ravel()
        cos = float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-30))
        assert _rel(a, b) < 0.1 and cos > 0.99, (name, _rel(a, b), cos)
        assert _rel(gg[name][1], go[name][1]) < 0.1, name


# (channels, batch, H, W, per-layer relative error, 1 - cosine, loss relative error)
BF16_ORACLE_CASES = [((16, 32, 32), 2, 16, 16, 1e-2, 1e-4, 1e-5), ((32, 64, 128, 256), 2, 64, 64, 3e-2, 1e-3, 1e-3)]


@pytest.mark.parametrize("ch,B,H,W,rel_max,cos_gap,loss_rel", BF16_ORACLE_CASES)
def test_unet_gradients_match_bf16_oracle(S, ch, B, H, W, rel_max, cos_gap, loss_rel):
    """Whole-network forward and backward on the GPU against the FP64 oracle that rounds every
    stored activation and activation gradient to BF16 where the network stores them in BF16
    (oracle unet_loss_and_grads(bf16=True)): the two then differ only by the GPU's FP32
    accumulation, which can tip a value to the other side of a BF16 rounding or of a ReLU's
    zero.  Small network (K up to 9 x 32): measured worst layer 5e-7, loss 1e-7, against 4e-2
    for the unrounded oracle.  The surrogate's own four-level shape on 64^2 images (K up to
    9 x 256, so more values tip): worst layer 1.2e-2 (the first layer, whose gradient sums every
    tipped value downstream), 1 - cosine 7e-5, loss 1.6e-4, against 2.2e-2 and 2.3e-4."""
    import torch
    cin = 16
    net = S.UNet(ch=ch, cin=cin, seed=3)
    rng = np.random.default_rng(11)
    net.load_weights("out", torch.tensor(rng.standard_normal((9, ch[0], cin)) * 0.1, dtype=torch.float32).cuda())
    x, xn = _bf(rng, (B, H, W, cin), 0.5)
    base = x[..., :3].float().contiguous()
    target = torch.tensor(rng.standard_normal((B, H, W, 3)) * 0.1, dtype=torch.float32).cuda()
    loss = net.loss_and_grads(x, base, target)
    torch.cuda.synchronize()
    params = net.params_numpy()
    lo, go = U.unet_loss_and_grads(xn, target.cpu().numpy().astype(np.float64), params, ch, bf16=True)
    assert abs(loss.item() - lo) / lo < loss_rel, (loss.item(), lo)
    gg = net.grads_numpy()
    worst = 0.0
    for name, _, _ in S.layer_specs(cin, ch):
        a, b = gg[name][0].ravel(), go[name][0].ravel()
        cos = float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-30))
        rel = _rel(a, b)
        worst = max(worst, rel)
        assert rel < rel_max and cos > 1 - cos_gap, (name, rel, cos)
        assert _rel(gg[name][1], go[name][1]) < rel_max, (name, _rel(gg[name][1], go[name][1]))
    print(ch, "worst per-layer weight-gradient relative error against the BF16-rounding oracle:", worst)


def test_training_reduces_loss(S):
    """A few hundred Adam steps on a fixed batch fit it (the kernels learn)."""
    import torch
    ch, cin = (16, 32), 16
    net = S.UNet(ch=ch, cin=cin, seed=4)
    rng = np.random.default_rng(10)
    B, H, W = 4, 32, 32
    x, xn = _bf(rng, (B, H, W, cin), 0.5)
    # target: a smooth function of the input the network can represent
    tgt = xn[..., :3] + 0.1 * np.roll(xn[..., :3], 1, axis=2)
    target = torch.tensor(tgt, dtype=torch.float32).cuda()
    base = x[..., :3].float().contiguous()
    first = net.loss_and_grads(x, base, target).item()
    for _ in range(300):
        net.loss_and_grads(x, base, target)
        net.adam_step(lr=2e-3)
    last = net.loss_and_grads(x, base, target).item()
    assert last < 0.2 * first, (first, last)


def test_graph_replayed_forward_equals_eager(S):
    """The CUDA-graph capture of the forward pass reproduces the eager pass bit for bit, and
    re-reads its input tensors in place on every replay."""
    import torch
    ch, cin = (16, 32, 64), 16
    net = S.UNet(ch=ch, cin=cin, seed=5)
    rng = np.random.default_rng(11)
    net.load_weights("out", torch.tensor(rng.standard_normal((9, ch[0], cin)) * 0.1, dtype=torch.float32).cuda())
    B, H, W = 3, 32, 48
    x, _ = _bf(rng, (B, H, W, cin), 0.5)
    base = x[..., :3].float().contiguous()
    g, pred = net.capture_forward(x, base)
    x2, _ = _bf(rng, (B, H, W, cin), 0.5)
    for inp in (x, x2):
        x.copy_(inp)
        base.copy_(inp[..., :3].float())
        g.replay()
        torch.cuda.synchronize()
        got = pred.clone()
        want = net.forward(x, base).clone()
        torch.cuda.synchronize()
        assert torch.equal(got, want)
    assert net.launches_per_forward() == 2 * 3 + 2 + 4 + 2


# -------------------------------------------------------------------------------------------
# The surrogate as used: trained on the solver's own trajectories, advancing lattices window by
# window under the judge, with the solver as audit and fallback.

@pytest.fixture(scope="module")
def trained(S):
    """A U-Net (32/64/128/256 channels) trained for 800 Adam steps on 12 solver trajectories of
    256^2 periodic spinodal decomposition (viscosity ratio 10, 30 windows of K = 50 steps), and 8
    held-out trajectories of the same workload."""
    import torch
    ntr, nte, wins, K = 12, 8, 30, 50
    members = S.spinodal_members(ntr + nte, 256, seed=100)
    traj = S.generate_trajectories(members, K, wins)
    states = S.trajectory_states(traj)
    del traj
    net = S.UNet(ch=(32, 64, 128, 256), cin=16, seed=1)
    S.train_states(net, states[:, :ntr], 800, 8, lr=1e-3, seed=2)
    torch.cuda.synchronize()
    return dict(net=net, states=states, test_members=members[ntr:], ntr=ntr, K=K)


def test_trained_network_beats_persistence(S, trained):
    """On held-out trajectories the trained network's one-window phi error (median over every
    window and lattice) is well below that of persistence (phi(t+K) ~ phi(t)): it has learned the
    dynamics, not the identity (measured 1.7e-4 against 8.6e-4)."""
    e, p = S.one_window_errors(trained["net"], trained["states"][:, trained["ntr"]:])
    print("one-window phi RMS error: median", float(np.median(e)), "persistence", float(np.median(p)))
    assert np.median(e) < 0.5 * np.median(p), (np.median(e), np.median(p))


def test_judged_rollout_against_the_solver(S, trained):
    """Closed loop: 8 held-out lattices advanced by 16 windows (800 steps) from step 500, each
    kept prediction feeding the next window, the judge checking every window's sum-phi drift on
    the GPU and auditing every 8th window with the solver.  Every window is accounted for (kept,
    audited or handed to the solver), and the final phi stays within 1e-2 RMS of the solver run
    alone from the same state (measured ~1.3e-3; doing nothing would be 1.3e-2 off), and the whole
    judged rollout takes less wall time than the solver alone over the same windows."""
    net, K = trained["net"], trained["K"]
    st0 = trained["states"][10, trained["ntr"]:].contiguous()
    judge = S.Judge(phi_err=1e-2, drift=1e-6, audit_every=8)
    S.rollout(net, trained["test_members"], st0, 2, K, judge)  # warm-up (graphs, buffers)
    fin, stats = S.rollout(net, trained["test_members"], st0, 16, K, judge)
    ref, t_solver = S.solver_only(trained["test_members"], st0, 16, K)
    err = S.phi_rms(fin, ref)
    pers = S.phi_rms(st0, ref)
    print("rollout:", {k: v for k, v in stats.items()}, "solver alone %.4f s" % t_solver,
          "speed-up %.3f" % (t_solver / stats["seconds"]), "final phi RMS", err.tolist(), "persistence", pers.tolist())
    assert stats["kept"] + stats["solver"] + stats["audits"] == stats["windows"] == 16
    assert stats["audits"] == 2 and stats["audit_failed"] == 0 and stats["drift_rejected"] == 0, stats
    assert max(stats["audit_rms"]) <= 1e-2
    assert err.max() <= 1e-2, err
    assert err.max() < 0.5 * np.median(pers), (err, pers)
    # faster than the solver alone, every cost counted (measured 1.23 with the window's network
    # part replayed as one CUDA graph and the next window predicted while the host judges;
    # 1.06 to 1.09 launched eagerly one window at a time)
    assert t_solver / stats["seconds"] > 1.0, (t_solver, stats["seconds"])


def test_judge_rejects_a_drifting_prediction_and_falls_back_exactly(S, trained):
    """A prediction made to create order parameter (0.1 added to every phi of one lattice: a drift
    of 0.1 per node against the 1e-6 threshold) is rejected by the judge's FP64 sum check, and the
    window is advanced by the solver instead: the state after that window equals, bit for bit, the
    solver's own advance of the window's input, also when the next window had already been
    predicted speculatively from the rejected candidate."""
    import torch
    net, K = trained["net"], trained["K"]
    members = trained["test_members"][:4]
    st0 = trained["states"][10, trained["ntr"]:trained["ntr"] + 4].contiguous()
    judge = S.Judge(phi_err=1e-2, drift=1e-6, audit_every=0)
    mid, stats1 = S.rollout(net, members, st0, 1, K, judge)
    assert stats1["kept"] == 1

    def inject(w, pred):
        if w == 1:
            pred[2, ..., 0] += 0.1

    fin, stats = S.rollout(net, members, st0, 2, K, judge, inject=inject)
    assert stats["kept"] == 1 and stats["drift_rejected"] == 1 and stats["solver"] == 1, stats
    solver = S.SolverWindows(members, K, torch.cuda.Stream())
    want = torch.empty_like(mid)
    solver.advance(mid, want)
    torch.cuda.synchronize()
    solver.close()
    assert torch.equal(fin, want)
    # A third window: window 2 is predicted speculatively while window 1 is judged; the rejection
    # drops it and restores window 1's input, so the run equals one window of the surrogate from
    # the solver's advance of window 1.
    fin3, stats3 = S.rollout(net, members, st0, 3, K, judge, inject=inject)
    assert stats3["kept"] == 2 and stats3["drift_rejected"] == 1 and stats3["solver"] == 1, stats3
    want3, _ = S.rollout(net, members, want, 1, K, judge)
    assert torch.equal(fin3, want3)


# -------------------------------------------------------------------------------------------
# The tcgen05 convolution (sur_conv3x3_tc): tensor memory accumulators, TMA or cp.async staging.

TC_SHAPES = [  # (batch, H, W, Cin, Cout, upsampled): every staging mode and tile shape
    (1, 16, 32, 16, 16, 0),    # copy mode (W < 128), one channel chunk
    (2, 16, 64, 64, 64, 0),    # copy mode, four chunks
    (1, 8, 32, 32, 256, 0),    # copy mode, two output-channel tiles
    (2, 8, 128, 32, 32, 0),    # row mode by TMA, four rows per tile
    (1, 8, 256, 48, 96, 0),    # row mode by TMA, two tiles per row, 96 output channels (2 rows per tile)
    (2, 16, 32, 64, 32, 1),    # copy mode through the 2x upsampling, with the skip addend
    (2, 8, 256, 32, 16, 1),    # row mode through the upsampling (cp.async), with the addend
]


@pytest.mark.parametrize("shape", TC_SHAPES, ids=lambda s: "x".join(map(str, s)))
def test_tcgen05_conv_matches_oracle(S, shape):
    """The tcgen05 convolution against the FP64 oracle on BF16-exact inputs: FP32 output within
    1e-5 relative (accumulation order only), BF16 output with the addend within a BF16 rounding.
    The bounded waits of the kernel did not give up (sur_check)."""
    import torch
    B, H, W, K, N, up = shape
    rng = np.random.default_rng(B * 1000 + H * 10 + W + K + N + up)
    s = torch.cuda.current_stream().cuda_stream
    assert S.sur_conv3x3_tc_supported(B, H, W, K, N, up)
    if up:
        x, xc = _bf(rng, (B, H // 2, W // 2, K))
        xn = np.repeat(np.repeat(xc, 2, axis=1), 2, axis=2)
    else:
        x, xn = _bf(rng, (B, H, W, K))
    w, wn = _bf(rng, (9, K, N), 0.2)
    wt = torch.empty((9, N, K), dtype=torch.bfloat16, device="cuda")
    S.sur_transpose_taps(w, wt, K, N, s)
    bias = torch.tensor(rng.standard_normal(N), dtype=torch.float32).cuda()
    bn = bias.cpu().numpy().astype(np.float64)
    if up:
        add, addn = _bf(rng, (B, H, W, N))
        y = torch.empty((B, H, W, N), dtype=torch.bfloat16, device="cuda")
        S.sur_conv3x3_tc(x, wt, bias, add, y, B, H, W, K, N, 0, 0, 1, s)
        assert _rel(y.float().cpu().numpy(), U.conv3x3(xn, wn, bn, relu=False) + addn) < 4e-3
    else:
        y = torch.empty((B, H, W, N), dtype=torch.float32, device="cuda")
        S.sur_conv3x3_tc(x, wt, bias, None, y, B, H, W, K, N, 1, 1, 0, s)
        assert _rel(y.cpu().numpy(), U.conv3x3(xn, wn, bn, relu=True)) < 1e-5
    assert S.sur_check(s) == S.SUR_OK


def test_tcgen05_conv_refuses_shapes_it_cannot_tile(S):
    """Shapes outside the kernel's tiling are refused with SUR_ERR_PARAM and reported unsupported:
    a width neither a multiple of 128 nor a power of two dividing it, a height not a multiple of the
    tile's rows, channels not multiples of 16, more than 128 output channels not a multiple of 128."""
    import torch
    s = torch.cuda.current_stream().cuda_stream
    x = torch.zeros((1, 16, 96, 32), dtype=torch.bfloat16, device="cuda")
    wt = torch.zeros((9, 32, 32), dtype=torch.bfloat16, device="cuda")
    y = torch.zeros((1, 16, 96, 32), dtype=torch.bfloat16, device="cuda")
    for bad in ((1, 16, 96, 32, 32), (1, 6, 32, 32, 32), (1, 16, 32, 24, 32), (1, 16, 32, 32, 160)):
        assert not S.sur_conv3x3_tc_supported(*bad, 0)
    with pytest.raises(S.SurError):
        S.sur_conv3x3_tc(x, wt, None, None, y, 1, 16, 96, 32, 32, 0, 0, 0, s)


def test_network_forward_same_on_both_tensor_core_paths(S):
    """The U-Net forward with every convolution the tcgen05 kernel serves on it (TMA rows of 4 or
    8 output rows per tile, multi-accumulator shifted copies, upsampled rows), whatever the timed
    choice would be, equals the forward on the mma.sync kernels bit for bit: both accumulate every
    16-channel chunk tap by tap in the same order on the same tensor-core dot products."""
    import torch
    net = S.UNet(ch=(32, 64, 128, 256), cin=16, seed=1)
    g = torch.Generator(device="cuda").manual_seed(3)
    s = torch.cuda.current_stream().cuda_stream
    net.load_weights("out", torch.randn(net.w["out"].shape, device="cuda", generator=g) * 0.05)
    x = (torch.randn((2, 256, 256, 16), device="cuda", generator=g) * 0.5).to(torch.bfloat16)
    base = x[..., :3].float().contiguous()
    net.tensor_cores = True
    net._tc = lambda B, H, W, ci, co, up=0: S.sur_conv3x3_tc_supported(B, H, W, ci, co, up)
    p1 = net.forward(x, base).clone()
    net.tensor_cores = False
    net._tc = lambda *a, **k: False
    p0 = net.forward(x, base).clone()
    torch.cuda.synchronize()
    assert torch.equal(p1, p0)
    assert float((p0 - base).abs().max()) > 1e-3  # the network does change the state
    assert S.sur_check(s) == S.SUR_OK
