"""Growth curves by top-hat apertures (paper Section 3.4) through gp_growth,
against the oracle element by element.

Tolerances: |d flux| <= 1e-5 sum|m| + 8 u sum|B| over the top-hat, with
u = 2^-24.  The first term is the aperture rule (a sum whose terms carry
1e-5 relative error).  The second is the float32 error of m = I - B(p)
itself, which is relative to the background B (about 1e3 here), not to m: a
top-hat that keeps one or two in-frame pixels of small |m| (a source just
off the frame) would otherwise be held to a bound its own arithmetic cannot
meet.  |d fluxerr| <= 1e-5 |fluxerr|; flags bit-exact.  The centre pixel is
an integer decision taken from the same double positions on both sides.
"""
import numpy as np
import pytest

import oracle
import synth
from parity import REL, assert_close

torch = pytest.importorskip("torch")
gp = pytest.importorskip("paper_2609_32375_gb300")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = gp.Context(0, workspace_bytes=1 << 28)
    yield c
    c.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def positions(rng, W, H, n):
    xs = np.concatenate([rng.uniform(-20, W + 20, n),
                         [0.0, W - 1.0, 0.5 * W + 0.5, -0.5, W - 0.51, -0.51, W - 0.5, 3.4999999, 1e7, -1e7]])
    ys = np.concatenate([rng.uniform(-20, H + 20, n),
                         [0.0, H - 1.0, 0.5 * H, 0.5 * H, 0.5, 10.5, 20.0, 7.5, 5.0, 5.0]])
    return xs, ys


def oracle_side(img, mesh, mask, saturation):
    vals, bad = oracle.pixel_values(img, mask)
    bm, rm, _ = oracle.background_meshes(vals, bad, mesh)
    H, W = img.shape
    bmap = oracle.spline_map(bm, W, H, mesh)
    rmap = oracle.spline_map(rm, W, H, mesh)
    m = np.where(bad != 0, 0.0, vals - bmap)
    sat = oracle.saturated(img, saturation)
    return m, rmap ** 2, bad, sat, bmap


def check(ctx, img, mesh, radii, gain, mask=None, saturation=0.0, n=400, seed=0):
    H, W = img.shape
    rng = np.random.default_rng(seed)
    xs, ys = positions(rng, W, H, n)
    m, var, bad, sat, bmap = oracle_side(img, mesh, mask, saturation)
    oracle.set_threads(0)
    rf, re, rfl = oracle.growth(m, var, bad, sat, xs, ys, radii, gain)
    fa, _, _ = oracle.growth(np.abs(m), var, bad, sat, xs, ys, radii, 0.0)
    fb, _, _ = oracle.growth(np.abs(bmap), var, bad, sat, xs, ys, radii, 0.0)
    dimg = dev(img)
    dmask = dev(mask) if mask is not None else None
    bkg = ctx.gp_background(dimg, mesh, mask=dmask)
    tx, ty = torch.from_numpy(xs), torch.from_numpy(ys)
    f1, e1, l1 = ctx.gp_growth(dimg, bkg, tx, ty, radii, gain=gain, mask=dmask, saturation=saturation)
    f2, e2, l2 = ctx.gp_growth(dimg, bkg, tx, ty, radii, gain=gain, mask=dmask, saturation=saturation)
    ctx.sync()
    flux, ferr, fl = f1.cpu().numpy(), e1.cpu().numpy(), l1.cpu().numpy().astype(np.uint32)
    print(f"\n{img.dtype} {img.shape} radii {radii[0]}..{radii[-1]} ({len(radii)})")
    assert_close("growth_flux", flux, rf, fa + (8 * 2.0 ** -24 / REL) * fb + 1e-6)
    assert_close("growth_fluxerr", ferr, re, np.abs(re) + 1e-6)
    assert np.array_equal(fl, rfl)
    # reproducible bit for bit
    assert np.array_equal(flux, f2.cpu().numpy()) and np.array_equal(ferr, e2.cpu().numpy())
    assert np.array_equal(fl, l2.cpu().numpy().astype(np.uint32))
    # sources far outside the frame: empty sums, every radius truncated
    far = np.abs(xs) > 1e6
    assert np.all(flux[far] == 0) and np.all(fl[far] == gp.GP_FLAG_TRUNCATED)
    return flux, rf


def test_growth_paper_radii_u16_ragged(ctx):
    cfg = synth.scaled_config(synth.CONFIGS["plain_2048x2048_u16"], 700, 500)
    img, _ = synth.make_frame(cfg, 21, cache=False)
    radii = oracle.growth_radii(3.0)            # 3 .. 15
    check(ctx, img, 128, radii, gain=1.5, saturation=cfg.saturation, seed=21)


def test_growth_f32_mask_nan_and_radius_zero(ctx):
    cfg = synth.scaled_config(synth.CONFIGS["plain_1024x1024_f32"], 333, 190)
    img, _ = synth.make_frame(cfg, 22, cache=False)
    img = img.astype(np.float32).copy()
    rng = np.random.default_rng(22)
    img[rng.random(img.shape) < 0.001] = np.nan
    mask = np.zeros(img.shape, np.uint8)
    mask[rng.random(img.shape) < 0.003] = 1
    mask[50:60, 100:104] = 1
    img[rng.random(img.shape) < 0.0005] = 70000.0
    check(ctx, img, 64, np.array([0, 1, 2, 5, 9], np.int32), gain=0.0, mask=mask, saturation=65535.0, seed=22)


def test_growth_most_radii_and_largest_rings(ctx):
    cfg = synth.scaled_config(synth.CONFIGS["dense_12288x12304_u16"], 900, 640)
    img, _ = synth.make_frame(cfg, 23, cache=False)
    radii = np.concatenate([np.arange(1, 31), [45, 70]]).astype(np.int32)      # 32 radii, ring of 70
    assert radii.size == gp.GP_GROWTH_MAX_NR
    check(ctx, img, 256, radii, gain=2.0, saturation=cfg.saturation, n=120, seed=23)


def test_growth_tracks_the_exact_overlap_aperture(ctx):
    """At a source well inside the frame the top-hat of radius r and the
    exact-overlap disc of radius r differ only by the boundary pixels' partial
    areas: |difference| <= sum of |m| over pixels within 1/sqrt(2) of the
    circle.  Both come from the CUDA path here; the bound is what relates
    them."""
    cfg = synth.scaled_config(synth.CONFIGS["plain_2048x2048_u16"], 512, 512)
    img, _ = synth.make_frame(cfg, 24, cache=False)
    rng = np.random.default_rng(24)
    xs = np.floor(rng.uniform(40, 470, 200)).astype(np.float64)
    ys = np.floor(rng.uniform(40, 470, 200)).astype(np.float64)
    dimg = dev(img)
    bkg = ctx.gp_background(dimg, 128)
    radii = np.array([3, 6, 10], np.int32)
    gf, _, _ = ctx.gp_growth(dimg, bkg, torch.from_numpy(xs), torch.from_numpy(ys), radii)
    af, _, _ = ctx.gp_aperture(dimg, bkg, torch.from_numpy(xs), torch.from_numpy(ys), tuple(float(r) for r in radii))
    ctx.sync()
    m, _, _, _, _ = oracle_side(img, 128, None, 0.0)
    d = np.abs(gf.cpu().numpy() - af.cpu().numpy())
    for k, r in enumerate(radii):
        for i in range(len(xs)):
            xc, yc = int(xs[i]), int(ys[i])
            yy, xx = np.mgrid[yc - r - 2:yc + r + 3, xc - r - 2:xc + r + 3]
            rho = np.hypot(xx - xc, yy - yc)
            band = np.abs(rho - r) <= np.sqrt(0.5) + 1e-9
            bound = np.abs(m[yy[band], xx[band]]).sum()
            # plus the float32 error of m in both GPU sums (8 u |B| a pixel, B < 2e3)
            slack = 2 * 8 * 2.0 ** -24 * 2e3 * np.pi * (r + 1) ** 2
            assert d[i, k] <= bound * (1 + 1e-5) + slack


def test_growth_rejects_bad_radii(ctx):
    img = np.full((64, 64), 1000, np.uint16)
    dimg = dev(img)
    bkg = ctx.gp_background(dimg, 32)
    x = torch.zeros(1, dtype=torch.float64)
    for bad in ([3, 3], [5, 4], [-1, 2], [256], list(range(1, 34))):
        with pytest.raises(gp.GpError):
            ctx.gp_growth(dimg, bkg, x, x, bad)
