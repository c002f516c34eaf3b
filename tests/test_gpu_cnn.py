"""The learned background's CUDA kernels against the FP64 oracle of the
network (oracle/cnn.py), and what the trained network gains over the plain
estimator.

Inputs and weights are rounded to bfloat16 first so both sides see the same
numbers; the kernels then accumulate in FP32, so layer outputs agree to FP32
summation error (bf16 rounding of stored activations aside).
"""
import ctypes as C

import numpy as np
import pytest

from oracle import cnn as ocnn

torch = pytest.importorskip("torch")
gp = pytest.importorskip("paper_2609_32375_gb300")
from paper_2609_32375_gb300 import learned  # noqa: E402

pytestmark = pytest.mark.gpu

PAIRS = [(16, 32), (32, 48), (48, 48), (48, 32), (32, 32), (32, 16)]


def bf(a):
    return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).cuda()


def f64(t):
    return t.float().cpu().numpy().astype(np.float64)


def _stream():
    return torch.cuda.current_stream().cuda_stream or None


def _pack(W, b):
    co, ci = W.shape[:2]
    cip, cop = ci, co
    wt = torch.empty((cop, 9 * cip), dtype=torch.bfloat16, device="cuda")
    wtd = torch.empty((cip, 9 * cop), dtype=torch.bfloat16, device="cuda")
    bp = torch.empty(cop, dtype=torch.float32, device="cuda")
    Wt = torch.from_numpy(W.astype(np.float32)).cuda().contiguous()
    bt = torch.from_numpy(b.astype(np.float32)).cuda()
    st = gp.load_library().gp_cnn_pack(Wt.data_ptr(), bt.data_ptr(), ci, co, cip, cop, wt.data_ptr(),
                                       wtd.data_ptr(), bp.data_ptr(), _stream())
    assert st == gp.GP_OK
    return wt, wtd, bp


@pytest.mark.parametrize("cip,cop", PAIRS)
def test_conv_forward_matches_oracle(cip, cop):
    rng = np.random.default_rng(cip * 100 + cop)
    N, H, W = 2, 24, 40                                   # W < 64: ragged tile in x
    x = ocnn.bf16_round(rng.normal(size=(N, H, W, cip)))
    Wm = ocnn.bf16_round(rng.normal(size=(cop, cip, 3, 3)) * 0.2)
    b = rng.normal(size=cop) * 0.1
    wt, _, bp = _pack(Wm, b)
    y = torch.empty((N, H, W, cop), dtype=torch.float32, device="cuda")
    L = gp.load_library()
    assert L.gp_cnn_conv3x3(bf(x).data_ptr(), N, H, W, cip, wt.data_ptr(), bp.data_ptr(), cop, 0, y.data_ptr(),
                            1, cop, _stream()) == gp.GP_OK
    ref = ocnn.conv3x3(x, Wm, b.astype(np.float32).astype(np.float64))
    scale = ocnn.conv3x3(np.abs(x), np.abs(Wm), np.abs(b)) + 1e-6
    err = np.abs(f64(y) - ref) / scale
    assert err.max() < 2e-6, err.max()
    # bf16 output with ReLU: within one bf16 rounding of the oracle
    yb = torch.empty((N, H, W, cop), dtype=torch.bfloat16, device="cuda")
    assert L.gp_cnn_conv3x3(bf(x).data_ptr(), N, H, W, cip, wt.data_ptr(), bp.data_ptr(), cop, 1, yb.data_ptr(),
                            0, 0, _stream()) == gp.GP_OK
    refr = np.maximum(ref, 0)
    assert np.all(np.abs(f64(yb) - refr) <= np.abs(refr) * 2.0 ** -8 + scale * 2e-6)


@pytest.mark.parametrize("cip,cop", PAIRS)
def test_weight_and_data_gradients_match_oracle(cip, cop):
    rng = np.random.default_rng(cip * 7 + cop)
    N, H, W = 2, 20, 70                                   # two x tiles, the second ragged
    x = ocnn.bf16_round(rng.normal(size=(N, H, W, cip)))
    dp = ocnn.bf16_round(rng.normal(size=(N, H, W, cop)))
    Wm = ocnn.bf16_round(rng.normal(size=(cop, cip, 3, 3)) * 0.2)
    L = gp.load_library()
    nslot = 16
    partial = torch.empty(nslot * 9 * cop * cip, dtype=torch.float32, device="cuda")
    bpart = torch.empty(nslot * 64, dtype=torch.float32, device="cuda")
    dW = torch.empty((cop, cip, 3, 3), dtype=torch.float32, device="cuda")
    db = torch.empty(cop, dtype=torch.float32, device="cuda")
    assert L.gp_cnn_conv3x3_wgrad(bf(x).data_ptr(), bf(dp).data_ptr(), N, H, W, cip, cop, cip, cop, nslot,
                                  partial.data_ptr(), bpart.data_ptr(), dW.data_ptr(), db.data_ptr(),
                                  _stream()) == gp.GP_OK
    rdx, rdW, rdb = ocnn.conv3x3_backward(x, Wm, dp)
    _, sdW, sdb = ocnn.conv3x3_backward(np.abs(x), np.abs(Wm), np.abs(dp))
    assert (np.abs(f64(dW) - rdW) / (sdW + 1e-6)).max() < 2e-6
    assert (np.abs(f64(db) - rdb) / (sdb + 1e-6)).max() < 2e-6
    # data gradient: the forward kernel with the flipped, transposed weights
    _, wtd, _ = _pack(Wm, np.zeros(cop))
    if (cop, cip) in PAIRS:
        dx = torch.empty((N, H, W, cip), dtype=torch.float32, device="cuda")
        zero = torch.zeros(cip, dtype=torch.float32, device="cuda")
        assert L.gp_cnn_conv3x3(bf(dp).data_ptr(), N, H, W, cop, wtd.data_ptr(), zero.data_ptr(), cip, 0,
                                dx.data_ptr(), 1, cip, _stream()) == gp.GP_OK
        sdx, _, _ = ocnn.conv3x3_backward(np.abs(x), np.abs(Wm), np.abs(dp))
        assert (np.abs(f64(dx) - rdx) / (sdx + 1e-6)).max() < 2e-6


def test_network_gradients_match_oracle():
    """Whole network: forward, MSE and every layer's gradients against the
    FP64 oracle fed the same bf16 weights and inputs, with the oracle's
    hidden activations rounded to bf16 where the GPU stores them."""
    torch.manual_seed(0)
    net = learned.Network(seed=3)
    rng = np.random.default_rng(5)
    N, H, W = 3, 16, 24
    feat = np.zeros((N, H, W, 16))
    feat[..., :5] = ocnn.bf16_round(rng.normal(size=(N, H, W, 5)))
    target = rng.normal(size=(N, H, W, 2)).astype(np.float32)
    ft = bf(feat)
    tt = torch.from_numpy(target).cuda()
    acts, out = net.forward(ft)
    loss, grads = net.backward(acts, out, tt)
    torch.cuda.synchronize()
    params = [(ocnn.bf16_round(f64(net.W[l])), f64(net.b[l])) for l in range(6)]
    # oracle forward with bf16-rounded hidden activations
    x = feat[..., :5]
    oacts = [x]
    for l, (Wl, bl) in enumerate(params):
        y = ocnn.conv3x3(oacts[-1], Wl, bl)
        y = np.maximum(y, 0) if l < 5 else y
        oacts.append(ocnn.bf16_round(y) if l < 5 else y)
    assert np.allclose(f64(out), oacts[-1], rtol=2e-2, atol=2e-2 * np.abs(oacts[-1]).max())
    assert float(loss.item()) == pytest.approx(ocnn.mse(oacts[-1], target), rel=2e-2)
    ograds, _ = ocnn.backward(oacts, params, target.astype(np.float64))
    for l in range(6):
        for a, b in ((f64(grads[l][0]), ograds[l][0]), (f64(grads[l][1]), ograds[l][1])):
            rel = np.linalg.norm(a - b) / (np.linalg.norm(b) + 1e-12)
            cos = float((a * b).sum() / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-30))
            print(f"layer {l}: relative gradient error {rel:.3e}, cosine {cos:.6f}")
            assert rel < 5e-2 and cos > 0.998


def test_adamw_step_is_the_published_update():
    """One AdamW step (Loshchilov & Hutter: bias-corrected Adam moments,
    decoupled weight decay) on a few values."""
    p = torch.tensor([1.0, -2.0, 0.5], device="cuda")
    g = torch.tensor([0.1, 0.2, -0.3], device="cuda")
    m = torch.zeros(3, device="cuda")
    v = torch.zeros(3, device="cuda")
    lr, b1, b2, eps, wd = 0.01, 0.9, 0.999, 1e-8, 0.1
    assert gp.load_library().gp_cnn_adamw(p.data_ptr(), g.data_ptr(), m.data_ptr(), v.data_ptr(), 3, lr, b1, b2,
                                          eps, wd, 1, _stream()) == gp.GP_OK
    # first step: m_hat = g, v_hat = g^2, so the Adam term is g / (|g| + eps) = sign(g)
    expect = np.array([1.0, -2.0, 0.5]) - lr * (np.sign([0.1, 0.2, -0.3]) + wd * np.array([1.0, -2.0, 0.5]))
    assert np.allclose(p.cpu().numpy(), expect, atol=1e-6)


def test_training_reduces_loss_and_learns_the_plain_estimator():
    """Train briefly on GPU-drawn frames with the library's own forward and
    backward kernels: the loss falls and the network learns the plain
    estimator's meshes on held-out frames."""
    ctx = gp.Context(0, workspace_bytes=512 << 20)
    try:
        train = learned.build_dataset(ctx, 96, seed0=1_000_000, size=2048, mesh=64)
        held = learned.build_dataset(ctx, 24, seed0=2_000_000, size=2048, mesh=64)
        net = learned.Network(seed=0)
        hist = learned.train(net, train, epochs=40, batch=16, lr=3e-3)
        print("loss", hist[0], "->", hist[-1])
        assert hist[-1] < 0.2 * hist[0]
        ev = learned.evaluate(net, held)
        print(ev)
        assert ev["bkg_rmse_learned_vs_plain"] < 0.5
    finally:
        ctx.close()


def test_trained_network_gains_over_the_plain_estimator():
    """The committed network (trained on the GPU on 2,000 frames, mesh 64)
    on frames it never saw: its background is closer to the true sky than
    the plain clipped estimator's, by a margin, and its background stage
    (one histogram pass and the network, in place of iterative clipping and
    the median filter) is faster, by a margin."""
    import os
    path = os.path.join(os.path.dirname(learned.__file__), "weights", "learned_bkg.npz")
    net = learned.load(path)
    ctx = gp.Context(0, workspace_bytes=1 << 30)
    try:
        held = learned.build_dataset(ctx, 32, seed0=3_000_000, size=4096, mesh=64)
        ev = learned.evaluate(net, held)
        print(ev)
        assert ev["bkg_rmse_learned_vs_truth"] < 0.95 * ev["bkg_rmse_plain_vs_truth"]
        assert ev["rms_relerr_learned_vs_truth"] < 0.05
        frame = learned.training_frame(3_100_000, 4096)
        t = learned.time_background(ctx, frame.image, 64, net)
        print(t)
        assert t["learned_ms"] < 0.8 * t["plain_ms"]
    finally:
        ctx.close()


def test_mesh256_network_on_the_dense_recipe():
    """The committed mesh-256 network (trained on uint16 8192^2 frames up to
    1,500 stars per megapixel, 400 epochs) on a 4096^2 crop of the dense
    151 MP recipe: its meshes stay within the accuracy measured for it at
    full size (background 0.11 sigma RMS from the clipped mesh, noise 2.9 %),
    with a margin; a regression guard, not the clipped estimator's accuracy."""
    import synth
    path = learned.weights_for_mesh(256)
    assert path is not None, "no committed weights trained at mesh 256"
    net = learned.load(path)
    cfg = synth.scaled_config(synth.CONFIGS["dense_12288x12304_u16"], 4096, 4096)
    img, _ = synth.make_frame(cfg, 0)
    ctx = gp.Context(0, workspace_bytes=1 << 30)
    try:
        t = torch.from_numpy(img).cuda()
        plain = ctx.gp_background(t, 256)
        lrn = learned.background_learned(ctx, t, 256, net)
        ctx.sync()
        pr = plain["rms_mesh"].clamp_min(1e-6)
        dbk = float(((lrn["bkg_mesh"] - plain["bkg_mesh"]) / pr).pow(2).mean().sqrt())
        drm = float(((lrn["rms_mesh"] - plain["rms_mesh"]) / pr).pow(2).mean().sqrt())
        print(f"background {dbk:.3f} sigma, noise {drm:.3f} relative")
        assert dbk < 0.2 and drm < 0.06
    finally:
        ctx.close()
