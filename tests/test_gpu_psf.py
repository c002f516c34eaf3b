"""The second detection pass with a spatially varying PSF (paper Section
3.2) through gp_detect_psf, against the oracle.

With minarea 1 every foreground pixel is kept, so the GPU's segmentation
map gives its threshold mask: it must agree with the oracle's mask outside
the near-threshold set (|S - k sigma| <= 1e-5 |k sigma|), and the map must be
the oracle's labelling of that mask, bit for bit.  Catalog rows are compared
with the oracle's moments of the same segments (the plain path's rules),
with the tolerance of the growth test: 1e-5 of the segment's absolute sums
plus the float32 error of m = I - B, 8 u sum|B| (u = 2^-24), which is
relative to the background; minarea 1 keeps one-pixel segments of small |m|.
"""
import numpy as np
import pytest

import oracle
import synth
from parity import REL, assert_close, segment_scales

torch = pytest.importorskip("torch")
gp = pytest.importorskip("paper_2609_32375_gb300")

pytestmark = pytest.mark.gpu

U8 = 8 * 2.0 ** -24


@pytest.fixture(scope="module")
def ctx():
    c = gp.Context(0, workspace_bytes=1 << 28)
    yield c
    c.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def psf_model(size, K, W, H, tile, seed):
    """A Gaussian reference and K smooth deviation patterns (the x and y
    derivatives of the reference, a ring), with per-tile coefficients."""
    h = size // 2
    yy, xx = np.mgrid[-h:h + 1, -h:h + 1].astype(np.float64)
    s = 3.0 / 2.3548
    g = np.exp(-(xx * xx + yy * yy) / (2 * s * s))
    p0 = g / g.sum()
    modes = [xx * p0, yy * p0, (xx * xx + yy * yy - 2 * s * s) * p0][:K]
    rng = np.random.default_rng(seed)
    coef = rng.uniform(-0.4, 0.4, (K, -(-H // tile), -(-W // tile)))
    return p0.astype(np.float32), np.array(modes, np.float32).reshape(K, size, size), coef.astype(np.float32)


CASES = [
    ("plain_2048x2048_u16", 41, 800, 600, 128, 7, 3, 200),
    ("plain_1024x1024_f32", 42, 333, 290, 64, 5, 2, 100),
    ("dense_12288x12304_u16", 43, 700, 520, 256, 11, 3, 250),
    ("plain_2048x2048_u16", 44, 500, 400, 128, 3, 0, 128),      # no modes: the plain filter with P0
]


@pytest.mark.parametrize("name,seed,w,h,mesh,size,K,tile", CASES)
def test_psf_detection_matches_the_oracle(ctx, name, seed, w, h, mesh, size, K, tile):
    cfg = synth.scaled_config(synth.CONFIGS[name], w, h)
    img, _ = synth.make_frame(cfg, seed, cache=False)
    H, W = img.shape
    p0, modes, coef = psf_model(size, K, W, H, tile, seed)
    oracle.set_threads(0)
    ref = oracle.detect_psf(img, mesh, p0.astype(np.float64), modes.astype(np.float64), coef.astype(np.float64), tile,
                            cfg.thresh, 1, saturation=cfg.saturation)
    dimg = dev(img)
    bkg = ctx.gp_background(dimg, mesh)
    out = ctx.gp_detect_psf(dimg, bkg, p0, modes, dev(coef) if K else None, tile, cfg.thresh, 1, capacity=200000,
                            saturation=cfg.saturation)
    ctx.sync()
    seg = out["segmap"].cpu().numpy().view(np.uint32)
    gmask = (seg != 0).astype(np.uint8)
    diff = gmask != ref["fg"]
    print(f"\n{name} {img.shape} K={K} {size}x{size} tile {tile}: fg {int(ref['fg'].sum())} px, "
          f"near {int(ref['near'].sum())}, disagreements {int(diff.sum())}")
    assert ref["fg"].sum() > 100
    assert not np.any(diff & ~ref["near"]), "mask differs outside the near-threshold set"
    lab, nlab = oracle.label(gmask, 1)
    assert np.array_equal(seg, lab)
    n = int(out["catalog"]["n"].item())
    assert n == nlab
    cat = {k: v[:n].cpu().numpy() for k, v in out["catalog"].items() if k != "n"}
    sat = oracle.saturated(img, cfg.saturation)
    rc = oracle.moments(lab, ref["m"], sat)
    for k in ("label", "npix", "xmin", "xmax", "ymin", "ymax", "flags"):
        assert np.array_equal(cat[k], rc[k]), k
    s_abs, s_dx, s_dy, s_d2 = segment_scales(lab, ref["m"], rc)
    b_abs, b_dx, b_dy, _ = segment_scales(lab, ref["bkg_map"], rc)
    f = U8 / REL
    assert_close("flux_iso", cat["flux_iso"], rc["flux"], s_abs + f * b_abs)
    assert_close("x", cat["x"], rc["x"], s_dx + f * b_dx + 1e-3)
    assert_close("y", cat["y"], rc["y"], s_dy + f * b_dy + 1e-3)
    # the same frame with minarea 5: the oracle's labelling of the same mask
    out5 = ctx.gp_detect_psf(dimg, bkg, p0, modes, dev(coef) if K else None, tile, cfg.thresh, 5, capacity=200000,
                             saturation=cfg.saturation)
    ctx.sync()
    lab5, n5 = oracle.label(gmask, 5)
    assert np.array_equal(out5["segmap"].cpu().numpy().view(np.uint32), lab5)
    assert int(out5["catalog"]["n"].item()) == n5


def test_psf_detection_without_modes_is_gp_detect_with_the_reference_kernel(ctx):
    """K = 0 and P0 of unit sum: the same statistic as the plain filter; the
    two passes must agree outside their own near-threshold pixels."""
    cfg = synth.scaled_config(synth.CONFIGS["plain_2048x2048_u16"], 640, 480)
    img, _ = synth.make_frame(cfg, 45, cache=False)
    p0, _, _ = psf_model(5, 0, 640, 480, 128, 45)
    dimg = dev(img)
    bkg = ctx.gp_background(dimg, 128)
    a = ctx.gp_detect_psf(dimg, bkg, p0, np.zeros((0, 5, 5), np.float32), None, 128, cfg.thresh, 1, capacity=100000)
    b = ctx.gp_detect(dimg, bkg, p0, cfg.thresh, 1, capacity=100000, count_near=True)
    ctx.sync()
    sa = a["segmap"].cpu().numpy() != 0
    sb = b["segmap"].cpu().numpy() != 0
    assert (sa != sb).sum() <= int(b["nnear"].item()) + 2


def test_psf_detection_rejects_bad_models(ctx):
    img = np.full((64, 64), 1000, np.uint16)
    dimg = dev(img)
    bkg = ctx.gp_background(dimg, 32)
    p0 = np.ones((5, 5), np.float32) / 25
    modes = np.zeros((9, 5, 5), np.float32)
    coef = torch.zeros((9, 2, 2), device="cuda")
    for args in ((np.ones((4, 5), np.float32), modes[:0], None, 32),     # even side
                 (p0, modes, coef, 32),                                   # too many modes
                 (p0, modes[:1], coef[:1], 0)):                           # tile 0
        with pytest.raises(gp.GpError):
            ctx.gp_detect_psf(dimg, bkg, *args, thresh=1.5, minarea=1, capacity=100)
