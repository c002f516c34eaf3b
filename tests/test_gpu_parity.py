"""CUDA path against the oracle, element by element, through the C ABI.

Sizes are chosen so the oracle finishes in seconds while the frames span
several detection tiles (64 x 32) and mesh boxes with ragged tails.
"""
import numpy as np
import pytest

import oracle
import synth
from parity import assert_close, rel_report, segment_scales

torch = pytest.importorskip("torch")
gp = pytest.importorskip("paper_2609_32375_gb300")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = gp.Context(0, workspace_bytes=1 << 30)
    yield c
    c.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def frame(name, seed, w=None, h=None):
    cfg = synth.CONFIGS[name]
    if w is not None:
        cfg = synth.scaled_config(cfg, w, h)
    img, truth = synth.make_frame(cfg, seed, cache=False)
    return cfg, img


CASES = [
    ("plain_1024x1024_f32", 0, None, None, 64),
    ("plain_2048x2048_u16", 1, None, None, 128),
    ("plain_2048x2048_u16", 2, 1000, 777, 128),           # ragged in both axes
    ("dense_12288x12304_u16", 3, 1500, 1100, 256),       # dense field, partial last boxes
    ("plain_1024x1024_f32", 4, 333, 190, 64),
]


# ----------------------------------------------------------- background ---
@pytest.mark.parametrize("name,seed,w,h,mesh", CASES)
def test_background_meshes_and_maps(ctx, name, seed, w, h, mesh):
    cfg, img = frame(name, seed, w, h)
    vals, bad = oracle.pixel_values(img)
    bm, rm, st = oracle.background_meshes(vals, bad, mesh)
    out = ctx.gp_background(dev(img), mesh, maps=True)
    ctx.sync()
    print(f"\n{name} {img.shape} mesh {mesh}")
    assert_close("bkg_mesh", out["bkg_mesh"].cpu().numpy(), bm, np.abs(bm) + 1e-6)
    assert_close("rms_mesh", out["rms_mesh"].cpu().numpy(), rm, np.abs(rm) + 1e-6)
    H, W = img.shape
    bmap = oracle.spline_map(bm, W, H, mesh)
    rmap = oracle.spline_map(rm, W, H, mesh)
    assert_close("bkg_map", out["bkg_map"].cpu().numpy(), bmap, np.abs(bmap) + 1e-6)
    assert_close("rms_map", out["rms_map"].cpu().numpy(), rmap, np.abs(rmap) + 1e-6)


def test_background_with_mask_and_nan(ctx):
    cfg, img = frame("plain_1024x1024_f32", 5, 400, 300)
    img = img.copy()
    rng = np.random.default_rng(5)
    img[rng.random(img.shape) < 0.01] = np.nan
    mask = np.zeros(img.shape, np.uint8)
    mask[64:128, 64:128] = 1                       # one whole box masked: filled from neighbours
    mask[200:260, 10:40] = 1
    vals, bad = oracle.pixel_values(img, mask)
    bm, rm, st = oracle.background_meshes(vals, bad, 64)
    assert st["valid"].min() == 0
    out = ctx.gp_background(dev(img), 64, mask=dev(mask))
    ctx.sync()
    assert_close("bkg_mesh", out["bkg_mesh"].cpu().numpy(), bm, np.abs(bm) + 1e-6)
    assert_close("rms_mesh", out["rms_mesh"].cpu().numpy(), rm, np.abs(rm) + 1e-6)


def test_background_windowed_histogram_fallback(ctx):
    """uint16 boxes whose clip the 4,096-value window cannot serve go to the
    full histogram: in half of the boxes every 16th row (the rows the window
    is placed from) is bright, so the window sits far from the true median;
    the other boxes finish in the window, others again hold a wide range.
    All must match the oracle."""
    rng = np.random.default_rng(17)
    H, W, B = 512, 640, 128
    img = rng.poisson(1000.0, (H, W)).astype(np.float64)
    for bj in range(H // B):
        for bi in range(W // B):
            y0, x0 = bj * B, bi * B
            if (bi + bj) % 2 == 0:
                img[y0:y0 + B:16, x0:x0 + B] = rng.normal(40000.0, 30.0, (B // 16, B))
            if (bi, bj) == (1, 0):
                img[y0:y0 + B, x0:x0 + B] += rng.uniform(0, 20000, (B, B))      # wider than the window
    img = np.clip(np.round(img), 0, 65535).astype(np.uint16)
    vals, bad = oracle.pixel_values(img)
    bm, rm, st = oracle.background_meshes(vals, bad, B)
    out = ctx.gp_background(dev(img), B)
    ctx.sync()
    assert_close("bkg_mesh", out["bkg_mesh"].cpu().numpy(), bm, np.abs(bm) + 1e-6)
    assert_close("rms_mesh", out["rms_mesh"].cpu().numpy(), rm, np.abs(rm) + 1e-6)
    # The learned background takes its quantiles from the same windowed
    # histograms (with the same fallback); gp_box_quantiles always uses the
    # full histogram.  The network fed by either must give identical meshes.
    from paper_2609_32375_gb300 import learned
    net = learned.Network(seed=2)
    t = dev(img)
    a = learned.background_learned(ctx, t, B, net)
    q = learned.box_quantiles(ctx, t, B)
    feat, norm = learned.features(q[None])
    _, outp = net.forward(feat)
    bb, rr = learned.denorm(outp, norm)
    ctx.sync()
    assert torch.equal(a["bkg_mesh"], bb[0]) and torch.equal(a["rms_mesh"], rr[0])


# -------------------------------------------------------------- labelling ---
def random_masks():
    rng = np.random.default_rng(11)
    for (h, w) in [(1, 1), (1, 300), (300, 1), (31, 65), (64, 64), (97, 200), (257, 130)]:
        for d in (0.1, 0.41, 0.6, 1.0):
            yield (rng.random((h, w)) < d).astype(np.uint8)
    # adversarial: spiral, comb, anti-diagonals crossing tile corners, checkerboard
    s = np.zeros((150, 150), np.uint8)
    for k in range(0, 75, 2):
        s[k, k:150 - k] = 1; s[k:150 - k, 150 - k - 1] = 1; s[150 - k - 1, k + 2:150 - k] = 1
        if k + 2 < 150 - k: s[k + 2:150 - k, k + 2] = 1
    yield s
    c = np.zeros((100, 260), np.uint8); c[99, :] = 1; c[:, ::2] = 1
    yield c
    yield np.eye(200, dtype=np.uint8)[::-1].copy()
    yield np.eye(200, 300, dtype=np.uint8)
    chk = (np.indices((130, 140)).sum(0) % 2).astype(np.uint8)
    yield chk
    # diagonal pairs touching only at tile corners (64 x 32 tiles)
    d = np.zeros((96, 192), np.uint8)
    for ty in (32, 64):
        for tx in (64, 128):
            d[ty - 1, tx - 1] = d[ty, tx] = 1          # main diagonal across the corner
            d[ty - 1, tx] = d[ty, tx - 1] = 1 if tx == 128 else 0   # anti-diagonal
    yield d


def test_label_mask_bit_exact(ctx):
    for mask in random_masks():
        for minarea in (1, 5):
            seg, n = ctx.gp_label_mask(dev(mask), minarea)
            ctx.sync()
            ref, nref = oracle.label(mask, minarea)
            got = seg.cpu().numpy().view(np.uint32)
            assert np.array_equal(got, ref), (mask.shape, minarea)
            assert int(n.item()) == nref


# -------------------------------------------------------------- detection ---
def check_detect(ctx, cfg, img, mesh, capacity=100000, mask=None):
    ref = oracle.extract(img, mesh, cfg.kernel, cfg.thresh, cfg.minarea, cfg.radii, cfg.gain, mask=mask,
                         saturation=cfg.saturation)
    out = ctx.gp_extract(dev(img), mesh, cfg.kernel, cfg.thresh, cfg.minarea, cfg.radii, cfg.gain,
                         capacity=capacity, saturation=cfg.saturation, mask=None if mask is None else dev(mask),
                         mask_out=True, count_near=True)
    ctx.sync()
    gmask = out["mask"].cpu().numpy()
    diff = gmask != ref["fg"]
    print(f"\n{cfg.name} {img.shape}: fg {int(ref['fg'].sum())} px, near-threshold {int(ref['near'].sum())}, "
          f"mask disagreements {int(diff.sum())}, GPU near count {int(out['nnear'].item())}")
    assert not np.any(diff & ~ref["near"]), "mask differs outside the near-threshold set"
    seg = out["segmap"].cpu().numpy().view(np.uint32)
    lab, nlab = oracle.label(gmask, cfg.minarea)
    assert np.array_equal(seg, lab), "segmap differs from the oracle labelling of the same mask"
    n = int(out["catalog"]["n"].item())
    assert n == nlab
    cat = {k: v[:n].cpu().numpy() for k, v in out["catalog"].items() if k != "n"}
    # oracle catalog of the same segmentation (identical to ref["cat"] when
    # the masks agree; row-aligned with the GPU's when a near-threshold pixel
    # flipped)
    rc = oracle.moments(lab, ref["m"], ref["sat"])
    assert np.array_equal(cat["label"], rc["label"])
    assert np.array_equal(cat["npix"], rc["npix"])
    for k in ("xmin", "xmax", "ymin", "ymax"):
        assert np.array_equal(cat[k], rc[k]), k
    assert np.array_equal(cat["flags"], rc["flags"])
    s_abs, s_dx, s_dy, s_d2 = segment_scales(lab, ref["m"], rc)
    assert_close("flux_iso", cat["flux_iso"], rc["flux"], s_abs)
    assert_close("x", cat["x"], rc["x"], s_dx + 1e-3)
    assert_close("y", cat["y"], rc["y"], s_dy + 1e-3)
    for k in ("x2", "y2", "xy"):
        assert_close(k, cat[k], rc[k], s_d2 + 1e-3)
    assert_close("peak", cat["peak"], rc["peak"], np.abs(rc["peak"]) + 1.0)
    # apertures at the (common) centroids
    rf, re, rfl = oracle.apertures(ref["m"], ref["rms_map"] ** 2, ref["bad"], ref["sat"], rc["x"], rc["y"],
                                   cfg.radii, cfg.gain)
    fa, _, _ = oracle.apertures(np.abs(ref["m"]), ref["rms_map"] ** 2, ref["bad"], ref["sat"], rc["x"], rc["y"],
                                cfg.radii, 0.0)
    nr = len(cfg.radii)
    flux = out["flux"][:n, :nr].cpu().numpy()
    ferr = out["fluxerr"][:n, :nr].cpu().numpy()
    afl = out["apflags"][:n, :nr].cpu().numpy().astype(np.uint32)
    assert_close("ap_flux", flux, rf, fa + 1e-6)
    assert_close("ap_fluxerr", ferr, re, np.abs(re) + 1e-6)
    assert np.array_equal(afl, rfl)
    return out


@pytest.mark.parametrize("name,seed,w,h,mesh", CASES)
def test_extract_matches_oracle(ctx, name, seed, w, h, mesh):
    cfg, img = frame(name, seed, w, h)
    check_detect(ctx, cfg, img, mesh)


def test_extract_with_bad_pixels(ctx):
    cfg, img = frame("plain_2048x2048_u16", 8, 640, 480)
    mask = np.zeros(img.shape, np.uint8)
    rng = np.random.default_rng(8)
    mask[rng.random(img.shape) < 0.002] = 1
    mask[100:140, 300:303] = 1
    check_detect(ctx, cfg, img, 128, mask=mask)


def test_aperture_entry_point(ctx):
    cfg, img = frame("plain_2048x2048_u16", 9, 700, 500)
    vals, bad = oracle.pixel_values(img)
    bm, rm, _ = oracle.background_meshes(vals, bad, 128)
    bkg = ctx.gp_background(dev(img), 128)
    rng = np.random.default_rng(9)
    xs = np.concatenate([rng.uniform(-3, 703, 300), [0.0, 699.0, 350.5, -0.5, 699.49]])
    ys = np.concatenate([rng.uniform(-3, 503, 300), [0.0, 499.0, 250.5, 250.0, 0.5]])
    radii = (1.5, 4.0, 8.0, 12.5)
    flux, ferr, fl = ctx.gp_aperture(dev(img), bkg, torch.from_numpy(xs), torch.from_numpy(ys), radii, gain=1.5,
                                     saturation=cfg.saturation)
    ctx.sync()
    H, W = img.shape
    bmap = oracle.spline_map(bm, W, H, 128)
    rmap = oracle.spline_map(rm, W, H, 128)
    m = np.where(bad != 0, 0.0, vals - bmap)
    sat = oracle.saturated(img, cfg.saturation)
    rf, re, rfl = oracle.apertures(m, rmap ** 2, bad, sat, xs, ys, radii, 1.5)
    fa, _, _ = oracle.apertures(np.abs(m), rmap ** 2, bad, sat, xs, ys, radii, 0.0)
    assert_close("ap_flux", flux.cpu().numpy(), rf, fa + 1e-6)
    assert_close("ap_fluxerr", ferr.cpu().numpy(), re, np.abs(re) + 1e-6)
    assert np.array_equal(fl.cpu().numpy().astype(np.uint32), rfl)


def test_centroid_fallback_for_nonpositive_flux(ctx):
    """A segment whose own sum of m is <= 0 takes the unweighted centroid
    and moments (GP_FLAG_CENTROID_FALLBACK).  A one-tap kernel that is a
    shifted delta detects the pixels two columns and rows up-left of a bright
    square, where a dark square sits, so that segment's sum is negative."""
    rng = np.random.default_rng(5)
    img = (1000 + 20 * rng.standard_normal((256, 320))).round().astype(np.uint16)
    img[100:112, 150:162] = 9000           # bright: detected through the shifted tap
    img[98:110, 148:160] = 0               # dark: the detected pixels themselves
    img[40:48, 60:70] = 6000               # an ordinary positive source beside it
    k = np.zeros((5, 5), np.float32)
    k[4, 4] = 1.0                          # F(x, y) = m(x + 2, y + 2)

    class Cfg:
        name = "shifted-delta kernel"
        kernel = k
        thresh = 3.0
        minarea = 3
        radii = (3.0, 5.0)
        gain = 1.0
        saturation = 0.0

    out = check_detect(ctx, Cfg, img, 64)
    n = int(out["catalog"]["n"].item())
    flags = out["catalog"]["flags"][:n].cpu().numpy().astype(np.uint32)
    flux = out["catalog"]["flux_iso"][:n].cpu().numpy()
    assert np.any(flux <= 0) and np.any(flux > 0)
    assert np.all(((flags & gp.GP_FLAG_CENTROID_FALLBACK) != 0) == (flux <= 0))


def test_tiles_without_foreground_overwrite_stale_outputs(ctx):
    """Tiles with no foreground take a short path that writes zero map rows
    and empty edge records; outputs reused after a crowded frame must match
    a run into fresh buffers."""
    cfg, crowded = frame("dense_12288x12304_u16", 21, 1024, 768)
    sparse = crowded.copy()
    sky = np.median(crowded)
    sparse[:, 200:] = np.random.default_rng(3).normal(sky, 4.0, sparse[:, 200:].shape).round().astype(np.uint16)
    ex = gp.Extractor(ctx, crowded.shape, torch.uint16, 64, cfg.kernel, cfg.thresh, cfg.minarea, cfg.radii,
                      cfg.gain, 50000, saturation=cfg.saturation, device="cuda")
    ex.run(dev(crowded))
    ctx.sync()
    assert int((ex.out["segmap"][:, 512:] != 0).sum()) > 1000
    ex.run(dev(sparse))
    ctx.sync()
    fresh = ctx.gp_extract(dev(sparse), 64, cfg.kernel, cfg.thresh, cfg.minarea, cfg.radii, cfg.gain,
                           capacity=50000, saturation=cfg.saturation)
    ctx.sync()
    assert torch.equal(ex.out["segmap"], fresh["segmap"])
    n = int(fresh["catalog"]["n"].item())
    assert int(ex.out["catalog"]["n"].item()) == n
    for k, v in fresh["catalog"].items():
        if k != "n":
            assert torch.equal(ex.out["catalog"][k][:n], v[:n]), k
    # far from the crowded strip (the spline background blends across about
    # a mesh box there) the frame is plain sky: no segments, where the
    # crowded frame left many
    assert int((fresh["segmap"][:, 512:] != 0).sum()) == 0
    assert int((ex.out["segmap"][:, 512:] != 0).sum()) == 0


# ------------------------------------------------------------- edge cases ---
def test_constant_frame_has_no_detections(ctx):
    img = np.full((200, 300), 1234, np.uint16)
    k = synth.gaussian_kernel(5, 3.0)
    out = ctx.gp_extract(dev(img), 64, k, 1.5, 5, (3.0,), 1.0, capacity=16, mask_out=True)
    ctx.sync()
    assert np.all(out["bkg_mesh"].cpu().numpy() == 1234.0) and np.all(out["rms_mesh"].cpu().numpy() == 0.0)
    assert int(out["catalog"]["n"].item()) == 0 and int(out["mask"].sum()) == 0
    assert int(out["segmap"].abs().sum()) == 0


@pytest.mark.parametrize("shape", [(1, 1), (3, 5), (17, 16), (16, 17), (33, 65), (1, 700)])
def test_tiny_and_thin_frames(ctx, shape):
    rng = np.random.default_rng(sum(shape))
    img = (1000 + 30 * rng.standard_normal(shape)).astype(np.float32)
    img[shape[0] // 2, shape[1] // 2] += 5000
    k = synth.gaussian_kernel(3, 2.0)
    ref = oracle.extract(img, 16, k, 3.0, 1, (2.0,), 1.0)
    out = ctx.gp_extract(dev(img), 16, k, 3.0, 1, (2.0,), 1.0, capacity=64, mask_out=True)
    ctx.sync()
    assert_close("bkg_mesh", out["bkg_mesh"].cpu().numpy(), ref["bkg_mesh"], np.abs(ref["bkg_mesh"]) + 1e-6)
    gmask = out["mask"].cpu().numpy()
    assert not np.any((gmask != ref["fg"]) & ~ref["near"])
    lab, n = oracle.label(gmask, 1)
    assert np.array_equal(out["segmap"].cpu().numpy().view(np.uint32), lab)
    assert int(out["catalog"]["n"].item()) == n


def test_capacity_overflow_reports_true_count(ctx):
    cfg, img = frame("plain_2048x2048_u16", 1)
    full = ctx.gp_extract(dev(img), 128, cfg.kernel, cfg.thresh, cfg.minarea, cfg.radii, cfg.gain,
                          capacity=100000, saturation=cfg.saturation)
    ctx.sync()
    n = int(full["catalog"]["n"].item())
    cap = n // 3
    part = ctx.gp_extract(dev(img), 128, cfg.kernel, cfg.thresh, cfg.minarea, cfg.radii, cfg.gain,
                          capacity=cap, saturation=cfg.saturation)
    with pytest.raises(gp.GpError) as e:
        ctx.sync()
    assert e.value.status == gp.GP_ERR_CAPACITY
    assert int(part["catalog"]["n"].item()) == n
    for k in ("label", "x", "y", "flux_iso", "npix"):
        assert torch.equal(part["catalog"][k][:cap], full["catalog"][k][:cap]), k
    assert torch.equal(part["flux"][:cap], full["flux"][:cap])


def test_repeat_runs_bit_identical(ctx):
    cfg, img = frame("dense_12288x12304_u16", 12, 1024, 1024)
    t = dev(img)
    outs = []
    for rep in range(3):
        o = ctx.gp_extract(t, 256, cfg.kernel, cfg.thresh, cfg.minarea, cfg.radii, cfg.gain, capacity=50000,
                           saturation=cfg.saturation)
        ctx.sync()
        outs.append(o)
    for o in outs[1:]:
        assert torch.equal(o["segmap"], outs[0]["segmap"])
        for k, v in o["catalog"].items():
            assert torch.equal(v, outs[0]["catalog"][k]), k
        assert torch.equal(o["flux"], outs[0]["flux"]) and torch.equal(o["fluxerr"], outs[0]["fluxerr"])


def test_invalid_arguments_are_rejected_on_host(ctx):
    img = dev(np.zeros((64, 64), np.uint16))
    k = synth.gaussian_kernel(5, 3.0)
    with pytest.raises(gp.GpError) as e:
        ctx.gp_extract(img, 8, k, 1.5, 5, (3.0,), 1.0, capacity=10)        # mesh too small
    assert e.value.status == gp.GP_ERR_INVALID_ARG
    with pytest.raises(gp.GpError):
        ctx.gp_extract(img, 64, np.array([[1.0, -1.0, 0.0]]), 1.5, 5, (3.0,), 1.0, capacity=10)  # zero sum
    with pytest.raises(gp.GpError):
        ctx.gp_extract(img, 64, np.ones((4, 4)), 1.5, 5, (3.0,), 1.0, capacity=10)          # even kernel
    with pytest.raises(gp.GpError):
        ctx.gp_extract(img, 64, k, 1.5, 0, (3.0,), 1.0, capacity=10)                       # minarea
    ctx.sync()
