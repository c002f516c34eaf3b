"""Pins of the CPU oracle to things other than itself.

Each test ties one oracle step to a closed form, an invariant, a library
routine that computes a special case of the same definition, or brute force
on tiny inputs, so that a dropped term, a wrong sign or index, or a
transposed operand in the oracle fails here.  No GPU involved.
"""
import math
import os

import numpy as np
import pytest
from scipy import ndimage
from scipy.interpolate import CubicSpline
from scipy.stats import norm

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "closed_forms.txt")


def golden():
    vals = {}
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            name, v = line.split()[:2]
            vals[name] = float(v)
    return vals


# ------------------------------------------------------------------ CCL ---
def brute_label(fg, minarea=1):
    """Independent brute force: relax every pixel to the minimum linear index
    over its 8-neighbourhood until nothing changes."""
    H, W = fg.shape
    lab = np.where(fg, np.arange(H * W).reshape(H, W) + 1, 0).astype(np.int64)
    big = np.iinfo(np.int64).max
    while True:
        p = np.pad(np.where(lab > 0, lab, big), 1, constant_values=big)
        nb = np.min([p[1 + dy:1 + dy + H, 1 + dx:1 + dx + W] for dy in (-1, 0, 1) for dx in (-1, 0, 1)], axis=0)
        new = np.where(fg, np.minimum(lab, nb), 0)
        if np.array_equal(new, lab):
            break
        lab = new
    if minarea > 1:
        ids, cnt = np.unique(lab[lab > 0], return_counts=True)
        small = ids[cnt < minarea]
        lab[np.isin(lab, small)] = 0
    return lab.astype(np.uint32)


def scipy_label_minindex(fg, minarea=1):
    """scipy.ndimage.label with the 3x3 structure, relabelled by min index."""
    lab, n = ndimage.label(fg, structure=np.ones((3, 3), int))
    out = np.zeros(fg.shape, np.uint32)
    flat = lab.ravel()
    for k in range(1, n + 1):
        idx = np.flatnonzero(flat == k)
        if idx.size >= minarea:
            out.ravel()[idx] = idx.min() + 1
    return out


def test_label_exhaustive_4x4():
    """Every one of the 65,536 4x4 masks against brute-force relaxation."""
    bits = np.arange(65536, dtype=np.uint32)
    masks = ((bits[:, None] >> np.arange(16, dtype=np.uint32)) & 1).astype(np.uint8).reshape(-1, 4, 4)
    # brute force vectorised over all masks at once
    H = W = 4
    fg = masks.astype(bool)
    lab = np.where(fg, np.arange(16).reshape(4, 4)[None] + 1, 0).astype(np.int64)
    big = 1 << 40
    while True:
        p = np.pad(np.where(lab > 0, lab, big), ((0, 0), (1, 1), (1, 1)), constant_values=big)
        nb = np.min([p[:, 1 + dy:1 + dy + H, 1 + dx:1 + dx + W] for dy in (-1, 0, 1) for dx in (-1, 0, 1)], axis=0)
        new = np.where(fg, np.minimum(lab, nb), 0)
        if np.array_equal(new, lab):
            break
        lab = new
    for i in range(65536):
        seg, _ = oracle.label(masks[i], 1)
        assert np.array_equal(seg, lab[i]), i


@pytest.mark.parametrize("density", [0.2, 0.35, 0.41, 0.5, 0.7])
def test_label_random_vs_scipy(density):
    rng = np.random.default_rng(int(density * 100))
    for trial in range(40):
        h, w = rng.integers(1, 65, 2)
        fg = (rng.random((h, w)) < density).astype(np.uint8)
        minarea = int(rng.integers(1, 6))
        seg, n = oracle.label(fg, minarea)
        ref = scipy_label_minindex(fg, minarea)
        assert np.array_equal(seg, ref)
        assert n == len(np.unique(ref[ref > 0]))


def test_label_adversarial_shapes():
    shapes = []
    # spiral
    s = np.zeros((41, 41), np.uint8)
    x0, y0, x1, y1 = 0, 0, 40, 40
    while x0 <= x1 and y0 <= y1:
        s[y0, x0:x1 + 1] = 1; s[y0:y1 + 1, x1] = 1; s[y1, x0:x1 + 1] = 1
        if y0 + 2 <= y1: s[y0 + 2:y1 + 1, x0] = 1
        x0 += 2; y0 += 2; x1 -= 2; y1 -= 2
        if x0 <= x1: s[y0 - 1, x0 - 1] = 1 if x0 - 1 >= 0 else 0
    shapes.append(s)
    # comb hanging from the bottom row (min index far from the start)
    c = np.zeros((30, 33), np.uint8); c[29, :] = 1; c[:, ::2] = 1; shapes.append(c)
    # diagonal chain: only 8-connected
    shapes.append(np.eye(37, dtype=np.uint8)[::-1].copy())
    shapes.append(np.ones((17, 23), np.uint8))
    shapes.append(np.ones((1, 1), np.uint8))
    chk = (np.indices((16, 16)).sum(0) % 2).astype(np.uint8); shapes.append(chk)
    for fg in shapes:
        for minarea in (1, 5, 50):
            seg, _ = oracle.label(fg, minarea)
            assert np.array_equal(seg, brute_label(fg.astype(bool), minarea))
    # the anti-diagonal is one 8-connected component labelled at its top-right pixel
    seg, n = oracle.label(np.eye(37, dtype=np.uint8)[::-1].copy(), 1)
    assert n == 1 and set(np.unique(seg)) == {0, 36 + 1}


# -------------------------------------------------------- overlap areas ---
@pytest.mark.parametrize("r", [0.3, 0.5, 1.0, 1.7, 3.0, 5.0, 8.0, 10.0])
def test_overlap_sums_to_disc_area(r):
    rng = np.random.default_rng(int(r * 10))
    for _ in range(5):
        cx, cy = rng.uniform(-0.5, 0.5, 2)
        R = int(math.ceil(r)) + 2
        tot = 0.0
        for y in range(-R, R + 1):
            for x in range(-R, R + 1):
                tot += oracle.overlap_area(x - 0.5 - cx, x + 0.5 - cx, y - 0.5 - cy, y + 0.5 - cy, r)
        assert abs(tot - math.pi * r * r) < 1e-12 * max(1.0, r * r)


@pytest.mark.parametrize("r", [0.5, 1.0, 1.5, 2.5, 4.0, 8.0, 12.5])
def test_overlap_sums_to_disc_area_at_aligned_centres(r):
    """Centres on a pixel centre, an edge midpoint and a corner make the
    circle tangent to pixel edges (y = +-r); the sum must still be pi r^2."""
    for cx, cy in [(0.0, 0.0), (0.5, 0.0), (0.0, 0.5), (0.5, 0.5)]:
        R = int(math.ceil(r)) + 2
        tot = sum(oracle.overlap_area(x - 0.5 - cx, x + 0.5 - cx, y - 0.5 - cy, y + 0.5 - cy, r)
                  for y in range(-R, R + 1) for x in range(-R, R + 1))
        assert abs(tot - math.pi * r * r) < 1e-12 * max(1.0, r * r), (cx, cy)


def test_overlap_tangent_pixel_against_quadrature():
    """Pixel [-1/2, 1/2] x [r-1, r] under a disc of radius r tangent to its
    top edge: area = integral of min(h(x), r) - (r - 1) by quadrature."""
    from scipy.integrate import quad
    for r in (1.5, 4.0, 12.5):
        ref, _ = quad(lambda x: min(math.sqrt(r * r - x * x), r) - (r - 1.0), -0.5, 0.5, epsabs=1e-13)
        assert oracle.overlap_area(-0.5, 0.5, r - 1.0, r, r) == pytest.approx(ref, abs=1e-12)
        assert oracle.overlap_area(-0.5, 0.5, -r, 1.0 - r, r) == pytest.approx(ref, abs=1e-12)


def test_overlap_interior_exterior_and_small_disc():
    r = 5.0
    for y in range(-7, 8):
        for x in range(-7, 8):
            a = oracle.overlap_area(x - 0.5, x + 0.5, y - 0.5, y + 0.5, r)
            far = math.hypot(abs(x) + 0.5, abs(y) + 0.5)
            near = math.hypot(max(abs(x) - 0.5, 0), max(abs(y) - 0.5, 0))
            if far <= r:
                assert a == pytest.approx(1.0, abs=1e-14)
            if near >= r:
                assert a == 0.0
            assert 0.0 <= a <= 1.0 + 1e-15
    for r in (0.1, 0.25, 0.49):
        assert oracle.overlap_area(-0.5, 0.5, -0.5, 0.5, r) == pytest.approx(math.pi * r * r, rel=1e-13)


def test_overlap_symmetries_and_monte_carlo():
    rng = np.random.default_rng(7)
    for _ in range(30):
        x0, y0 = rng.uniform(-4, 3, 2)
        x1, y1 = x0 + rng.uniform(0.2, 1.5), y0 + rng.uniform(0.2, 1.5)
        r = rng.uniform(0.5, 4)
        a = oracle.overlap_area(x0, x1, y0, y1, r)
        assert a == pytest.approx(oracle.overlap_area(y0, y1, x0, x1, r), abs=1e-13)       # x <-> y
        assert a == pytest.approx(oracle.overlap_area(-x1, -x0, y0, y1, r), abs=1e-13)     # x -> -x
        assert a == pytest.approx(oracle.overlap_area(x0, x1, -y1, -y0, r), abs=1e-13)     # y -> -y
    # Monte Carlo on boundary pixels
    for (x0, y0, r) in [(2.5, 0.5, 3.0), (1.5, 1.5, 2.3), (-0.5, 2.5, 3.1), (3.5, -4.5, 5.2)]:
        pts = rng.uniform(0, 1, (1_000_000, 2))
        inside = ((x0 + pts[:, 0]) ** 2 + (y0 + pts[:, 1]) ** 2 <= r * r).mean()
        a = oracle.overlap_area(x0, x0 + 1, y0, y0 + 1, r)
        assert abs(a - inside) < 5 * math.sqrt(max(inside * (1 - inside), 1e-6) / 1e6) + 1e-6


# ---------------------------------------------------------- sigma clip ---
def test_sigma_clip_gaussian_fixed_point():
    g = golden()
    # the fixed point itself, from the truncated-normal variance
    var_trunc = lambda a: 1 - 2 * a * norm.pdf(a) / (2 * norm.cdf(a) - 1)
    s = g["clip3_fixed_point"]
    assert s == pytest.approx(math.sqrt(var_trunc(3 * s)), abs=1e-12)
    rng = np.random.default_rng(1)
    v = rng.normal(100.0, 7.0, 2_000_000)
    med, mean, sd, nk, passes = oracle.sigma_clip(v, 3.0, 50)
    assert sd / 7.0 == pytest.approx(s, abs=2.5e-3)
    assert mean == pytest.approx(100.0, abs=0.03)
    assert med == pytest.approx(100.0, abs=0.03)
    # a single pass clips at 3 sigma of the raw sample
    med1, _, sd1, _, p1 = oracle.sigma_clip(v, 3.0, 1)
    assert p1 == 1 and sd1 / 7.0 == pytest.approx(g["clip3_single_pass"], abs=2.5e-3)


def test_sigma_clip_special_cases():
    v = np.full(1000, 42.0)
    med, mean, sd, nk, passes = oracle.sigma_clip(v, 3.0, 10)
    assert (med, mean, sd, nk, passes) == (42.0, 42.0, 0.0, 1000, 0)
    rng = np.random.default_rng(3)
    w = rng.normal(0, 1, 4001)
    # no clipping pass: plain median / mean / population std (numpy routines)
    med, mean, sd, nk, passes = oracle.sigma_clip(w, 3.0, 0)
    assert med == np.median(w) and nk == w.size and passes == 0
    assert mean == pytest.approx(np.mean(w), abs=1e-13) and sd == pytest.approx(np.std(w), rel=1e-13)
    # even count: median is the mean of the two middle order statistics
    med, *_ = oracle.sigma_clip(np.array([4.0, 1.0, 3.0, 10.0]), 3.0, 0)
    assert med == 3.5


def test_sigma_clip_equivariance_and_outliers():
    rng = np.random.default_rng(5)
    v = np.round(rng.normal(1000, 30, 20000))
    a = oracle.sigma_clip(v, 3.0, 10)
    b = oracle.sigma_clip(4.0 * v + 1024.0, 3.0, 10)          # exact in binary
    assert b[3] == a[3] and b[4] == a[4]
    assert b[0] == 4 * a[0] + 1024 and b[1] == pytest.approx(4 * a[1] + 1024, rel=1e-15)
    assert b[2] == pytest.approx(4 * a[2], rel=1e-12)
    c = oracle.sigma_clip(-v, 3.0, 10)                         # reflection
    assert c[3] == a[3] and c[0] == -a[0] and c[2] == pytest.approx(a[2], rel=1e-12)
    # 5 % of far outliers are removed and the clean result comes back
    out = np.concatenate([v, np.full(1000, 60000.0)])
    d = oracle.sigma_clip(out, 3.0, 20)
    e = oracle.sigma_clip(v, 3.0, 20)
    assert d[3] == e[3] and d[0] == e[0] and d[2] == pytest.approx(e[2], rel=1e-12)
    # the final kept set is contiguous in value order and inside its bounds
    med, mean, sd, nk, _ = e
    kept = np.sort(v)[(np.sort(v) >= med - 3 * sd - 1e-9) & (np.sort(v) <= med + 3 * sd + 1e-9)]
    assert kept.size == nk


def test_mode_estimate_symmetric():
    assert oracle.mode_estimate(10.0, 10.0, 2.0) == 10.0      # symmetric: mode = median
    assert oracle.mode_estimate(10.0, 12.0, 2.0) == 10.0      # skewed > 0.3 sigma: median
    assert oracle.mode_estimate(10.0, 10.4, 2.0) == pytest.approx(9.4)
    assert oracle.mode_estimate(5.0, 7.0, 0.0) == 5.0


# ------------------------------------------------------- mesh and spline ---
def test_median_filter_interior_matches_scipy_and_edges():
    rng = np.random.default_rng(11)
    a = rng.normal(0, 1, (9, 12))
    out = oracle.median_filter(a, 3)
    ref = ndimage.median_filter(a, size=3, mode="nearest")
    assert np.array_equal(out[1:-1, 1:-1], ref[1:-1, 1:-1])
    # corner window is the 2x2 block: mean of its two middle values
    c = np.sort(a[:2, :2].ravel())
    assert out[0, 0] == pytest.approx(0.5 * (c[1] + c[2]), abs=1e-15)
    spike = np.ones((5, 5)); spike[2, 2] = 1e6
    assert np.all(oracle.median_filter(spike, 3) == 1.0)


def test_spline_reproduces_linear_and_constant():
    W, H, B = 300, 250, 64             # partial last boxes on both axes
    Mx, My = -(-W // B), -(-H // B)
    cx = np.array([i * B + (min((i + 1) * B, W) - i * B - 1) / 2 for i in range(Mx)])
    cy = np.array([j * B + (min((j + 1) * B, H) - j * B - 1) / 2 for j in range(My)])
    mesh = 3.0 + 0.25 * cx[None, :] - 0.5 * cy[:, None]
    m = oracle.spline_map(mesh, W, H, B)
    yy, xx = np.mgrid[0:H, 0:W]
    assert np.allclose(m, 3.0 + 0.25 * xx - 0.5 * yy, atol=1e-9, rtol=0)
    c = oracle.spline_map(np.full((My, Mx), 1234.5), W, H, B)
    assert np.all(c == 1234.5)            # exact, so m = I - B is exactly 0 on a flat sky


def test_spline_is_natural_cubic_tensor_product():
    W, H, B = 700, 520, 64
    Mx, My = -(-W // B), -(-H // B)
    cx = np.array([i * B + (min((i + 1) * B, W) - i * B - 1) / 2 for i in range(Mx)])
    cy = np.array([j * B + (min((j + 1) * B, H) - j * B - 1) / 2 for j in range(My)])
    rng = np.random.default_rng(2)
    mesh = rng.normal(0, 10, (My, Mx))
    m = oracle.spline_map(mesh, W, H, B)
    # interpolates the mesh at the box centres
    for j in range(My):
        for i in range(Mx):
            if float(cx[i]).is_integer() and float(cy[j]).is_integer():
                assert m[int(cy[j]), int(cx[i])] == pytest.approx(mesh[j, i], abs=1e-9)
    # inside the node range: scipy's natural CubicSpline along x, then y
    xs = np.arange(int(math.ceil(cx[0])), int(cx[-1]) + 1)
    ys = np.arange(int(math.ceil(cy[0])), int(cy[-1]) + 1)
    rows = CubicSpline(cx, mesh, axis=1, bc_type="natural")(xs)
    ref = CubicSpline(cy, rows, axis=0, bc_type="natural")(ys)
    assert np.allclose(m[np.ix_(ys, xs)], ref, atol=1e-9, rtol=0)
    # the other order gives the same surface (tensor product)
    cols = CubicSpline(cy, mesh, axis=0, bc_type="natural")(ys)
    ref2 = CubicSpline(cx, cols, axis=1, bc_type="natural")(xs)
    assert np.allclose(ref, ref2, atol=1e-9)
    # beyond the outer centres the map is linear in x (zero second difference)
    d2 = m[:, 2:int(cx[0])] - 2 * m[:, 1:int(cx[0]) - 1] + m[:, 0:int(cx[0]) - 2]
    assert np.abs(d2).max() < 1e-9
    # samples agree with the full map
    qx = rng.integers(0, W, 50); qy = rng.integers(0, H, 50)
    assert np.allclose(oracle.spline_at(mesh, W, H, B, qx, qy), m[qy, qx], atol=1e-12, rtol=0)


def test_spline_one_and_two_nodes():
    m = oracle.spline_map(np.array([[7.0]]), 40, 30, 64)
    assert np.all(m == 7.0)
    m = oracle.spline_map(np.array([[1.0, 3.0]]), 100, 20, 64)   # centres 31.5 and 81.5
    assert m[0, 31] == pytest.approx(1.0 - 0.5 * 2 / 50) and m[5, 99] == pytest.approx(1 + 2 * (99 - 31.5) / 50)


# ---------------------------------------------------------------- filter ---
def test_filter_matches_scipy_mirror_correlation():
    rng = np.random.default_rng(4)
    m = rng.normal(0, 1, (37, 53))
    K = rng.uniform(0.1, 1, (5, 3))                    # asymmetric, non-square
    F = oracle.matched_filter(m, K)
    ref = ndimage.correlate(m, K / K.sum(), mode="mirror")
    assert np.allclose(F, ref, atol=1e-12, rtol=0)
    # a delta reproduces the flipped, normalised kernel (correlation, not convolution)
    d = np.zeros((11, 11)); d[5, 5] = 1.0
    F = oracle.matched_filter(d, K)
    assert np.allclose(F[3:8, 4:7], (K / K.sum())[::-1, ::-1], atol=1e-15)
    with pytest.raises(ValueError):
        oracle.matched_filter(m, np.array([[1.0, -1.0, 0.0]]))


def test_filter_golden_kernel_taps():
    g = golden()
    K = synth.gaussian_kernel(5, 3.0).astype(np.float64)
    d = np.zeros((9, 9)); d[4, 4] = 1.0
    F = oracle.matched_filter(d, K)
    assert F[4, 4] == pytest.approx(g["gauss5_fwhm3_centre"], abs=1e-6)
    assert F[2, 2] == pytest.approx(g["gauss5_fwhm3_corner"], abs=1e-7)
    assert math.sqrt((F ** 2).sum()) == pytest.approx(g["gauss5_fwhm3_l2"], abs=1e-6)


# --------------------------------------------------------------- moments ---
def test_moments_closed_forms():
    seg = np.zeros((20, 30), np.uint32)
    m = np.zeros((20, 30))
    # uniform w x h rectangle: centroid at its centre, x2 = (w^2-1)/12
    seg[2:7, 3:12] = 2 * 30 + 3 + 1
    m[2:7, 3:12] = 5.0
    # single pixel
    seg[15, 25] = 15 * 30 + 25 + 1
    m[15, 25] = 3.0
    # diagonal pair with weights 1 and 3
    seg[10, 1] = seg[11, 2] = 10 * 30 + 1 + 1
    m[10, 1], m[11, 2] = 1.0, 3.0
    cat = oracle.moments(seg, m)
    assert list(cat["label"]) == sorted(cat["label"])
    r = 0
    assert cat["x"][r] == pytest.approx(7.0) and cat["y"][r] == pytest.approx(4.0)
    assert cat["x2"][r] == pytest.approx((81 - 1) / 12) and cat["y2"][r] == pytest.approx((25 - 1) / 12)
    assert cat["xy"][r] == pytest.approx(0.0, abs=1e-12) and cat["npix"][r] == 45
    assert cat["flux"][r] == pytest.approx(225.0)
    assert (cat["xmin"][r], cat["xmax"][r], cat["ymin"][r], cat["ymax"][r]) == (3, 11, 2, 6)
    r = 1
    assert cat["x"][r] == pytest.approx(1.75) and cat["y"][r] == pytest.approx(10.75)
    assert cat["x2"][r] == pytest.approx(0.1875) and cat["xy"][r] == pytest.approx(0.1875)
    assert (cat["xpeak"][r], cat["ypeak"][r], cat["peak"][r]) == (2, 11, 3.0)
    r = 2
    assert (cat["x"][r], cat["y"][r], cat["x2"][r]) == (25.0, 15.0, 0.0)
    # non-positive sum: unweighted centroid and the fallback flag
    m2 = m.copy(); m2[10, 1], m2[11, 2] = -1.0, -3.0
    cat = oracle.moments(seg, m2)
    assert cat["x"][1] == 1.5 and cat["flags"][1] & oracle.FLAG_CENTROID_FALLBACK
    assert cat["x2"][1] == pytest.approx(0.25)


# ------------------------------------------------------------- apertures ---
def test_aperture_moffat_encircled_energy():
    """Aperture sums of a rendered Moffat star against the closed-form
    encircled energy.  A pixelised aperture differs from the continuous
    integral by a pixel-integration error that falls as the square of the
    sampling, while EE(r; alpha) = EE(s r; s alpha); so the star is drawn s
    times finer (FWHM 3 s, radii r s) and compared with the golden FWHM-3
    values."""
    g = golden()
    beta, F, s = 2.5, 1e5, 6
    R = 10 * s + 4
    W = H = 2 * R + 1
    cx, cy = R + 0.3, R - 0.2
    img, _ = synth.render_moffat((H, W), np.array([cx]), np.array([cy]), np.array([F]),
                                 np.array([3.0 * s]), np.array([0.0]), np.array([0.0]), beta, R, 8)
    radii = np.array([3.0, 5.0, 8.0, 10.0]) * s
    flux, err, flags = oracle.apertures(img, np.zeros_like(img), np.zeros((H, W), np.uint8), None,
                                        [cx], [cy], radii, 0.0)
    for k, r in enumerate((3, 5, 8, 10)):
        assert flux[0, k] / F == pytest.approx(g[f"moffat_ee_r{r}"], rel=1e-3)
    assert np.all(flags == 0) and np.all(err == 0)


def test_aperture_constant_image_and_flags():
    W, H = 40, 30
    img = np.full((H, W), 2.0)
    var = np.full((H, W), 9.0)
    bad = np.zeros((H, W), np.uint8)
    flux, err, flags = oracle.apertures(img, var, bad, None, [20.2], [14.9], [3.0, 6.5], 2.0)
    area = math.pi * np.array([9.0, 42.25])
    assert np.allclose(flux[0], 2.0 * area, rtol=1e-12)
    assert np.allclose(err[0] ** 2, 9.0 * area + 2.0 * area / 2.0, rtol=1e-12)
    # disc leaving the frame is flagged and sums only in-frame area
    flux, err, flags = oracle.apertures(img, var, bad, None, [1.0], [14.0], [3.0], 0.0)
    assert flags[0, 0] & oracle.FLAG_TRUNCATED
    half = sum(oracle.overlap_area(x - 0.5 - 1.0, x + 0.5 - 1.0, y - 0.5, y + 0.5, 3.0)
               for x in range(0, 5) for y in range(-4, 5))
    assert flux[0, 0] == pytest.approx(2.0 * half, rel=1e-12)
    bad[14, 20] = 1
    flux, err, flags = oracle.apertures(img, var, bad, None, [20.0], [14.0], [2.0], 0.0)
    assert flags[0, 0] & oracle.FLAG_BAD and flux[0, 0] == pytest.approx(2.0 * (math.pi * 4 - 1), rel=1e-12)


def test_aperture_poisson_term_only_for_positive_flux_and_saturation_flag():
    """err^2 = sum A var + max(F, 0) / gain: a negative sky-subtracted disc
    adds no Poisson term; a saturated pixel inside a disc flags that disc
    (and every larger one) without changing the sums."""
    W, H = 40, 30
    var = np.full((H, W), 4.0)
    bad = np.zeros((H, W), np.uint8)
    img = np.full((H, W), -3.0)
    flux, err, flags = oracle.apertures(img, var, bad, None, [20.3], [15.1], [4.0], 1.5)
    area = math.pi * 16.0
    assert flux[0, 0] == pytest.approx(-3.0 * area, rel=1e-12)
    assert err[0, 0] ** 2 == pytest.approx(4.0 * area, rel=1e-12)
    sat = np.zeros((H, W), np.uint8)
    sat[15, 26] = 1                                   # 5.7 px from the centre: inside r = 7 only
    img = np.full((H, W), 2.0)
    f1, e1, fl1 = oracle.apertures(img, var, bad, sat, [20.3], [15.1], [3.0, 7.0], 1.5)
    f0, e0, fl0 = oracle.apertures(img, var, bad, None, [20.3], [15.1], [3.0, 7.0], 1.5)
    assert np.array_equal(f1, f0) and np.array_equal(e1, e0)
    assert not fl1[0, 0] & oracle.FLAG_SAT and fl1[0, 1] & oracle.FLAG_SAT


# ----------------------------------------------------- whole-path invariants ---
def test_constant_sky_has_no_detections():
    img = np.full((256, 320), 1500.0, np.float32)
    r = oracle.extract(img, 64, synth.gaussian_kernel(5, 3.0), 1.5, 5, (3.0,), 1.0)
    assert np.all(r["bkg_map"] == 1500.0) and np.all(r["rms_map"] == 0.0)
    assert np.all(r["F"] == 0.0) and r["fg"].sum() == 0 and len(r["cat"]["label"]) == 0


def test_pure_noise_background_and_rms():
    g = golden()
    rng = np.random.default_rng(9)
    mu, s = 1000.0, 20.0
    img = rng.normal(mu, s, (512, 512)).astype(np.float32)
    st = oracle.box_stats(img.astype(np.float64), np.zeros(img.shape, np.uint8), 128)
    n = 128 * 128
    assert np.all(np.abs(st["bkg"] - mu) < 6 * s / math.sqrt(n) * 2.5)
    assert np.all(np.abs(st["rms"] / s - g["clip3_fixed_point"]) < 0.02)
    r = oracle.extract(img, 128, synth.gaussian_kernel(5, 3.0), 1.5, 5, (3.0,), 1.0)
    assert len(r["cat"]["label"]) == 0        # 1.5 sigma on the filtered image is 6.2 filtered sigmas


def test_isolated_star_recovered():
    """Noiseless flat sky plus one Moffat star (drawn 4x finer than FWHM 3 so
    that pixel integration is negligible): one segment, centroid at the star,
    aperture fluxes equal to the encircled energy."""
    g = golden()
    W = H = 192
    cx, cy, F = 90.4, 100.7, 2e6
    star, _ = synth.render_moffat((H, W), np.array([cx]), np.array([cy]), np.array([F]),
                                  np.array([12.0]), np.array([0.0]), np.array([0.0]), 2.5, 90, 6)
    img = (500.0 + star).astype(np.float64)
    r = oracle.extract(img, 64, synth.gaussian_kernel(5, 3.0), 1.5, 5, (12.0, 20.0), 1.0)
    cat = r["cat"]
    assert len(cat["label"]) == 1
    assert cat["x"][0] == pytest.approx(cx, abs=0.05) and cat["y"][0] == pytest.approx(cy, abs=0.05)
    # the star lifts its boxes' statistics; measure against the known sky
    flux, _, _ = oracle.apertures(img - 500.0, np.zeros_like(img), np.zeros((H, W), np.uint8), None,
                                  [cx], [cy], [12.0, 20.0], 0.0)
    assert flux[0, 0] / F == pytest.approx(g["moffat_ee_r3"], rel=2e-3)
    assert flux[0, 1] / F == pytest.approx(g["moffat_ee_r5"], rel=2e-3)


def test_box_geometry_and_invalid_fill():
    """[R2] box bounds including partial last boxes, [R5] filling of boxes
    with fewer than half good pixels from their valid neighbours."""
    W, H, B = 150, 70, 32                    # 5 x 3 boxes, last ones 22 and 6 px
    Mx, My = 5, 3
    vals = np.arange(Mx * My, dtype=np.float64).reshape(My, Mx) * 10 + 100
    img = np.repeat(np.repeat(vals, B, 0), B, 1)[:H, :W]
    bad = np.zeros((H, W), np.uint8)
    st = oracle.box_stats(img, bad, B)
    assert np.array_equal(st["bkg"], vals) and np.all(st["rms"] == 0) and np.all(st["valid"] == 1)
    assert st["nkept"][2, 4] == 22 * 6 and st["nkept"][0, 0] == 32 * 32
    # mask more than half of box (1, 2): it takes the mean of its 8 neighbours
    bad[32:64, 64:96] = 1
    bad[32:40, 64:70] = 0                    # 48 good of 1024: invalid
    st = oracle.box_stats(img, bad, B)
    assert st["valid"][1, 2] == 0
    b, r = oracle.fill_invalid(st["bkg"], st["rms"], st["valid"])
    nb = [vals[j, i] for j in (0, 1, 2) for i in (1, 2, 3) if (j, i) != (1, 2)]
    assert b[1, 2] == pytest.approx(np.mean(nb)) and r[1, 2] == 0.0
    # two invalid neighbours: the inner one is filled in the second sweep
    valid = np.ones((1, 4), np.uint8); valid[0, 2:] = 0
    b, _ = oracle.fill_invalid(np.array([[1.0, 3.0, 0, 0]]), np.zeros((1, 4)), valid)
    assert b[0, 2] == 3.0 and b[0, 3] == 3.0


def test_threshold_is_strict_and_skips_bad():
    F = np.array([[3.0, 3.0000001, 2.9, 5.0]])
    rms = np.array([[2.0, 2.0, 2.0, 2.0]])
    bad = np.array([[0, 0, 0, 1]], np.uint8)
    assert list(oracle.threshold(F, rms, bad, 1.5)[0]) == [0, 1, 0, 0]


def test_oracle_threads_give_identical_results():
    """The oracle's parallel loops (boxes, map columns, filter rows, aperture
    sources) compute each output on one thread in a fixed order, so the whole
    path is bit-identical on one thread and on every core."""
    cfg = synth.scaled_config(synth.CONFIGS["plain_2048x2048_u16"], 400, 300)
    img, _ = synth.make_frame(cfg, 5, cache=False)
    outs = []
    try:
        for n in (1, 0):
            oracle.set_threads(n)
            outs.append(oracle.extract(img, 64, cfg.kernel, cfg.thresh, cfg.minarea, cfg.radii, cfg.gain,
                                       saturation=cfg.saturation))
    finally:
        oracle.set_threads(1)
    a, b = outs
    for k in ("bkg_mesh", "rms_mesh", "bkg_map", "rms_map", "F", "seg", "flux", "fluxerr", "apflags"):
        assert np.array_equal(a[k], b[k]), k
    for k, v in a["cat"].items():
        assert np.array_equal(v, b["cat"][k]), k


# ------------------------------------------------ top-hat growth curves ---
def _tophat(r):
    u = np.arange(-r, r + 1)
    return (u[:, None] ** 2 + u[None, :] ** 2 <= r * r).astype(np.float64)


def test_growth_radii_are_the_papers_range():
    """Section 3.4: integer radii from ceil(0.75 FWHM) to ceil(5 FWHM)."""
    assert oracle.growth_radii(3.0).tolist() == list(range(3, 16))
    assert oracle.growth_radii(2.0).tolist() == list(range(2, 11))
    assert oracle.growth_radii(4.1).tolist() == list(range(4, 22))


def test_growth_counts_lattice_points_on_a_constant_image():
    """A unit image: each sum is the number of pixels of the top-hat, the
    Gauss circle count N(r)."""
    g = golden()
    radii = [0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 15]
    m = np.ones((64, 70))
    f, e, fl = oracle.growth(m, np.zeros_like(m), np.zeros(m.shape, np.uint8), None, [35.3], [31.6], radii, 0.0)
    assert f[0].tolist() == [g[f"gauss_circle_r{r}"] for r in radii]
    assert np.all(fl == 0)


def test_growth_is_the_tophat_correlation_sampled_at_the_source_pixel():
    """The paper's formulation: the frame (bad pixels zeroed) correlated with
    a top-hat kernel, read at the pixel nearest the position; the variance
    map through the same kernel; Poisson term F / gain; flags from the
    pixels under the kernel."""
    rng = np.random.default_rng(3)
    H, W = 90, 120
    m = rng.normal(0, 20, (H, W))
    var = rng.uniform(10, 50, (H, W))
    bad = (rng.random((H, W)) < 0.01).astype(np.uint8)
    sat = (rng.random((H, W)) < 0.01).astype(np.uint8)
    xs = np.concatenate([rng.uniform(10, W - 10, 20), [0.2, W - 0.7, 3.49, 3.51]])
    ys = np.concatenate([rng.uniform(10, H - 10, 20), [45.0, 2.0, H - 1.2, 0.3]])
    radii = np.array([1, 3, 6, 9], np.int32)
    f, e, fl = oracle.growth(m, var, bad, sat, xs, ys, radii, 2.0)
    mz = np.where(bad != 0, 0.0, m)
    vz = np.where(bad != 0, 0.0, var)
    for k, r in enumerate(radii):
        T = _tophat(r)
        cf = ndimage.correlate(mz, T, mode="constant", cval=0.0)
        cv = ndimage.correlate(vz, T, mode="constant", cval=0.0)
        cb = ndimage.correlate(bad.astype(np.float64), T, mode="constant", cval=0.0)
        cs = ndimage.correlate((sat & (bad == 0)).astype(np.float64), T, mode="constant", cval=0.0)
        inside = ndimage.correlate(np.ones((H, W)), T, mode="constant", cval=0.0)
        for s in range(xs.size):
            xc, yc = int(np.floor(xs[s] + 0.5)), int(np.floor(ys[s] + 0.5))
            assert abs(f[s, k] - cf[yc, xc]) <= 1e-9 * (1 + abs(cf[yc, xc]))
            vv = cv[yc, xc] + (max(cf[yc, xc], 0.0) / 2.0)
            assert abs(e[s, k] - np.sqrt(vv)) <= 1e-9 * np.sqrt(vv)
            want = (oracle.FLAG_TRUNCATED if inside[yc, xc] < T.sum() else 0) | \
                   (oracle.FLAG_BAD if cb[yc, xc] > 0 else 0) | (oracle.FLAG_SAT if cs[yc, xc] > 0 else 0)
            assert fl[s, k] == want, (s, r)


def test_growth_of_a_delta_and_against_exact_overlap_sums():
    """A single bright pixel at the source pixel: every radius holds exactly
    its value.  A smooth star: the top-hat and the exact disc overlap of the
    same radius differ only through the pixels the circle crosses, so their
    difference is bounded by the boundary pixels' values."""
    m = np.zeros((41, 41))
    m[20, 20] = 1234.5
    z = np.zeros(m.shape, np.uint8)
    f, _, _ = oracle.growth(m, np.zeros_like(m), z, None, [20.3], [19.8], [0, 1, 5, 12], 0.0)
    assert np.all(f == 1234.5)
    # a Moffat star (FWHM 3, beta 2.5) of unit flux drawn 6x finer
    H = W = 61
    s = 6
    yy, xx = (np.mgrid[0:H * s, 0:W * s] + 0.5) / s - 0.5
    alpha = 3.0 / (2 * np.sqrt(2 ** (1 / 2.5) - 1))
    prof = (1.5 / (np.pi * alpha ** 2)) * (1 + ((xx - 30.0) ** 2 + (yy - 30.0) ** 2) / alpha ** 2) ** -2.5
    img = prof.reshape(H, s, W, s).mean(axis=(1, 3))
    zz = np.zeros(img.shape, np.uint8)
    radii = np.arange(3, 16, dtype=np.int32)
    ft, _, _ = oracle.growth(img, np.zeros_like(img), zz, None, [30.0], [30.0], radii, 0.0)
    fx, _, _ = oracle.apertures(img, np.zeros_like(img), zz, None, [30.0], [30.0], radii.astype(np.float64), 0.0)
    for k, r in enumerate(radii):
        T = _tophat(r)
        ring = ndimage.binary_dilation(T > 0) & ~ndimage.binary_erosion(np.pad(T > 0, 1))[1:-1, 1:-1]
        border = img[30 - r:30 + r + 1, 30 - r:30 + r + 1][ring].sum()
        assert abs(ft[0, k] - fx[0, k]) <= border
    assert np.all(np.diff(ft[0]) > 0)               # a non-negative image: the curve grows


# ------------------------------------------- optimal radius (Section 3.4) ---
def test_snr_argmax_finds_the_background_limited_gaussian_optimum():
    """For a Gaussian star of width s on flat noise, S/N(r) is proportional
    to (1 - exp(-r^2 / 2 s^2)) / r, whose maximum sits where e^x = 1 + 2x with
    x = r^2 / 2 s^2 (the derivative set to zero).  The root is found here by
    bracketing, independently of the oracle."""
    from scipy.optimize import brentq
    x = brentq(lambda t: np.exp(t) - 1.0 - 2.0 * t, 0.5, 5.0)
    for s in (1.3, 2.0, 3.4):
        r = np.arange(0.5, 12.0, 0.001)
        flux = 1e4 * (1.0 - np.exp(-r * r / (2 * s * s)))
        err = 7.0 * np.sqrt(np.pi) * r
        k, snr = oracle.snr_argmax(flux[None, :], err[None, :])
        assert abs(r[k[0]] - s * np.sqrt(2 * x)) <= 0.0011
        assert snr.shape == (1, r.size)


def test_snr_argmax_takes_the_first_of_equal_values_and_zero_error_as_no_signal():
    flux = np.array([[1.0, 2.0, 2.0, 1.0], [5.0, 5.0, 5.0, 5.0], [3.0, 1.0, 2.0, 4.0]])
    err = np.array([[1.0, 1.0, 1.0, 1.0], [0.0, 1.0, 0.5, 0.5], [1.0, 1.0, 1.0, 0.0]])
    k, snr = oracle.snr_argmax(flux, err)
    assert k.tolist() == [1, 2, 0]
    assert snr[1, 0] == 0.0 and snr[2, 3] == 0.0


def test_isolated_excludes_pairs_closer_than_the_distance():
    xs = np.array([0.0, 3.0, 20.0, 40.0, 50.0])
    ys = np.array([0.0, 4.0, 0.0, 0.0, 0.0])          # (0,0)-(3,4) at 5; (40,0)-(50,0) at 10 exactly
    assert oracle.isolated(xs, ys, 5.0).tolist() == [True, True, True, True, True]
    assert oracle.isolated(xs, ys, 5.0001).tolist() == [False, False, True, True, True]
    assert oracle.isolated(xs, ys, 10.5).tolist() == [False, False, True, False, False]


def test_power_law_fit_recovers_exact_laws_and_matches_polyfit():
    rng = np.random.default_rng(3)
    nu = 10 ** rng.uniform(0.5, 3.0, 200)
    a0, b0 = 0.21, 0.47
    r = 10 ** (a0 * np.log10(nu) + b0)
    sel = np.ones(nu.size, bool)
    a, b, n = oracle.power_law_fit(nu, r, sel)
    assert n == 200 and abs(a - a0) < 1e-12 and abs(b - b0) < 1e-12
    rn = r * 10 ** rng.normal(0, 0.05, nu.size)
    sel[::3] = False
    a, b, n = oracle.power_law_fit(nu, rn, sel)
    pa, pb = np.polyfit(np.log10(nu[sel]), np.log10(rn[sel]), 1)
    assert n == sel.sum() and abs(a - pa) < 1e-10 and abs(b - pb) < 1e-10
    a, b, n = oracle.power_law_fit(nu, rn, np.arange(nu.size) < 2)
    assert n == 2 and np.isnan(a) and np.isnan(b)
    a, b, n = oracle.power_law_fit(np.full(5, 7.0), np.arange(1.0, 6.0), np.ones(5, bool))
    assert np.isnan(a)                                  # no spread in nu


def test_assign_radius_rounds_onto_the_grid():
    radii = np.arange(3, 16, dtype=np.int32)
    # b alone sets r_fit when a = 0: r_fit = 10^b
    cases = [(4.2, 1), (4.5, 2), (4.49, 1), (100.0, 12), (0.5, 0), (15.0, 12), (2.9, 0)]
    for rfit, k in cases:
        got = oracle.assign_radius(np.array([10.0]), 0.0, np.log10(rfit), radii)
        assert got[0] == k, (rfit, got)
    assert oracle.assign_radius(np.array([0.0, -3.0]), 0.5, 0.1, radii).tolist() == [0, 0]
    assert oracle.assign_radius(np.array([10.0]), float("nan"), 0.1, radii).tolist() == [0]
    # a non-uniform grid: the nearest radius
    g = np.array([2, 5, 11], np.int32)
    for rfit, k in ((3.6, 1), (3.4, 0), (8.2, 2), (7.8, 1)):
        assert oracle.assign_radius(np.array([10.0]), 0.0, np.log10(rfit), g).tolist() == [k]
    # an exact tie (10^1 = 10 between 5 and 15) goes to the larger radius
    assert oracle.assign_radius(np.array([10.0]), 0.0, 1.0, np.array([5, 15], np.int32)).tolist() == [1]


def test_calibrators_need_every_condition():
    n = 6
    snr = np.array([[10, 60, 40]] * n, float)
    kopt = np.full(n, 1, np.int32)
    cat_flags = np.zeros(n, np.uint32)
    gfl = np.zeros((n, 3), np.uint32)
    iso = np.ones(n, bool)
    nu = np.full(n, 30.0)
    cat_flags[1] = 1
    gfl[2, 2] = 4
    iso[3] = False
    nu[4] = -1.0
    snr[5, 1] = 49.0
    cal = oracle.calibrators(cat_flags, gfl, snr, kopt, iso, nu, 50.0)
    assert cal.tolist() == [True, False, False, False, False, False]


def test_significance_is_the_filtered_value_over_sigma_at_the_peak():
    m = np.zeros((40, 50))
    m[20, 30] = 500.0
    m[5, 7] = -80.0
    K = np.outer([1, 2, 3, 2, 1], [1, 4, 6, 4, 1]).astype(float)
    K /= K.sum()
    F = oracle.matched_filter(m, K)
    rms = np.full(m.shape, 4.0)
    rms[5, 7] = 0.0
    nu = oracle.significance(F, rms, [30, 7, 31], [20, 5, 20])
    assert nu[0] == pytest.approx(500.0 * K[2, 2] / 4.0, rel=1e-15)
    assert nu[1] == 0.0                                      # sigma 0 gives no significance
    assert nu[2] == pytest.approx(500.0 * K[2, 1] / 4.0, rel=1e-15)   # F(p) takes m(p + u) with tap u


# --------------------------- spatially varying matched filter (Section 3.2) ---
def _psf_inputs(seed=5, K=3, kw=7, kh=5, W=90, H=70, tile=32):
    rng = np.random.default_rng(seed)
    m = rng.normal(0, 10, (H, W))
    p0 = rng.random((kh, kw))
    p0 /= p0.sum()
    modes = rng.normal(0, 0.05, (K, kh, kw))
    coef = rng.normal(0, 1, (K, -(-H // tile), -(-W // tile)))
    return m, p0, modes, coef, tile


def test_correlate_is_scipy_mirror_correlation_with_the_kernel_as_given():
    from scipy import ndimage
    m, p0, modes, _, _ = _psf_inputs()
    for K in (p0, modes[0], modes[1] - modes[1].mean()):        # unit sum, arbitrary, zero sum
        ref = ndimage.correlate(m, K, mode="mirror")
        assert np.allclose(oracle.correlate(m, K), ref, rtol=0, atol=1e-12)


def test_psf_filter_without_modes_is_the_plain_matched_filter():
    m, p0, modes, coef, tile = _psf_inputs()
    S = oracle.psf_filter(m, p0, modes[:0], coef[:0], tile)
    assert np.allclose(S, oracle.matched_filter(m, p0), rtol=0, atol=1e-12)


def test_psf_filter_with_constant_coefficients_is_one_kernel():
    """With every tile holding the same coefficients the filter is the
    correlation with the single kernel P0 + sum_k c_k e_k (linearity)."""
    from scipy import ndimage
    m, p0, modes, coef, tile = _psf_inputs()
    c = np.array([0.7, -1.3, 2.1])
    const = np.broadcast_to(c[:, None, None], coef.shape).copy()
    S = oracle.psf_filter(m, p0, modes, const, tile)
    ref = ndimage.correlate(m, p0 + np.tensordot(c, modes, axes=1), mode="mirror")
    assert np.allclose(S, ref, rtol=0, atol=1e-10)


def test_psf_filter_of_a_delta_reads_the_local_kernel():
    """m = delta at q: S(p) = P0[q - p + h] + sum_k c_k(p) e_k[q - p + h],
    the tap orientation of a correlation, with each pixel's own coefficients."""
    m, p0, modes, coef, tile = _psf_inputs()
    H, W = m.shape
    d = np.zeros_like(m)
    qy, qx = 33, 41
    d[qy, qx] = 1.0
    S = oracle.psf_filter(d, p0, modes, coef, tile)
    cm = oracle.coefficient_maps(coef, W, H, tile)
    kh, kw = p0.shape
    for py in range(qy - kh // 2, qy + kh // 2 + 1):
        for px in range(qx - kw // 2, qx + kw // 2 + 1):
            v, u = qy - py + kh // 2, qx - px + kw // 2
            want = p0[v, u] + sum(cm[k][py, px] * modes[k][v, u] for k in range(len(modes)))
            assert S[py, px] == pytest.approx(want, abs=1e-14)
    assert S[qy + kh // 2 + 1, qx] == 0.0


def test_coefficient_maps_are_linear_for_linear_tiles():
    W, H, tile = 200, 150, 40
    My, Mx = -(-H // tile), -(-W // tile)
    ax = oracle.spline_map(np.zeros((My, Mx)), W, H, tile)       # shape check
    assert ax.shape == (H, W)
    # tile centres (first pixel + (w - 1)/2); a mesh linear in them gives the same plane everywhere
    cx = np.array([min(i * tile + (min(tile, W - i * tile) - 1) / 2, W) for i in range(Mx)])
    cy = np.array([min(j * tile + (min(tile, H - j * tile) - 1) / 2, H) for j in range(My)])
    mesh = 0.25 + 0.01 * cx[None, :] - 0.02 * cy[:, None]
    c = oracle.coefficient_maps(mesh[None], W, H, tile)[0]
    yy, xx = np.mgrid[0:H, 0:W]
    assert np.allclose(c, 0.25 + 0.01 * xx - 0.02 * yy, rtol=0, atol=1e-10)


# ----------------------------------------- cosmetic filters (Section 3.1) ---
def test_window_median_is_scipy_median_filter_and_skips_bad_values():
    from scipy import ndimage
    rng = np.random.default_rng(8)
    a = rng.normal(0, 5, (37, 41))
    for size in (3, 5, 7):
        assert np.array_equal(oracle.window_median(a, size), ndimage.median_filter(a, size=size, mode="mirror"))
    b = np.arange(9.0).reshape(3, 3)
    b[0, 0] = np.nan                                   # 8 values 1..8 around the centre: median 4.5
    assert oracle.window_median(b, 3)[1, 1] == 4.5
    assert np.isnan(oracle.window_median(np.full((4, 4), np.nan), 3)).all()


def test_rtn_replaces_isolated_outliers_only():
    rng = np.random.default_rng(9)
    img = (1000 + 3 * rng.standard_normal((40, 50))).round()
    img[10, 10] += 300                    # isolated: replaced by its 3x3 median
    img[20, 20] += 300                    # a pair of neighbours: kept
    img[20, 21] += 300
    img[30, 5] -= 40                      # below the threshold: kept
    mask = np.zeros(img.shape, np.uint8)
    img[5, 40] += 500
    mask[5, 40] = 1                       # bad: never changed
    out, rep = oracle.rtn_filter(img, 100.0, mask=mask)
    assert rep.sum() == 1 and rep[10, 10]
    from scipy import ndimage
    assert out[10, 10] == ndimage.median_filter(img, size=3, mode="mirror")[10, 10]
    keep = ~rep
    assert np.array_equal(out[keep], img[keep])


def test_cr_filter_noise_ramp_star_and_hits():
    rng = np.random.default_rng(10)
    H, W = 200, 210
    sigma = np.sqrt(1000.0 + 25.0)
    noise = 1000 + sigma * rng.standard_normal((H, W))
    # the Laplacian of independent pixel noise has standard deviation sqrt(20) sigma
    L = 4 * noise[1:-1, 1:-1] - noise[:-2, 1:-1] - noise[2:, 1:-1] - noise[1:-1, :-2] - noise[1:-1, 2:]
    assert L.std() == pytest.approx(np.sqrt(20.0) * sigma, rel=0.02)
    _, fl = oracle.cr_filter(noise, 1.0, 5.0)
    assert fl.sum() <= 2
    yy, xx = np.mgrid[0:H, 0:W]
    _, fl = oracle.cr_filter(1000 + 0.5 * xx + 0.25 * yy, 1.0, 5.0)   # a noiseless ramp: L = 0
    assert not fl.any()
    img = noise + 5000 * np.exp(-((xx - 150) ** 2 + (yy - 40) ** 2) / (2 * 1.274 ** 2))   # FWHM 3 star
    img[50, 60] += 800
    img[120, 100] += 2000
    img[120, 101] += 1500
    out, fl = oracle.cr_filter(img, 1.0, 5.0)
    assert set(map(tuple, np.argwhere(fl))) == {(50, 60), (120, 100), (120, 101)}
    # a flagged pixel takes the median of the good unflagged pixels of its 5x5 window
    w = img[48:53, 58:63].copy().ravel()
    assert out[50, 60] == np.median(np.delete(w, 12))
    w = img[118:123, 98:103].ravel()
    keep = [i for i in range(25) if i not in (12, 13)]
    assert out[120, 100] == np.median(w[keep])
    assert np.array_equal(out[~fl], img[~fl])


# ------------------------------------------- multi-threshold deblending ---
def _blend(peaks, H=48, W=72, s=2.5):
    yy, xx = np.mgrid[0:H, 0:W]
    m = np.zeros((H, W))
    for x0, y0, a in peaks:
        m += a * np.exp(-((xx - x0) ** 2 + (yy - y0) ** 2) / (2 * s * s))
    return m


def _deblend_map(m, thresh=1.5, minarea=5, **kw):
    nu = m.copy()                                    # sigma 1 and an identity filter: nu = m
    seg, n = oracle.label((nu > thresh).astype(np.uint8), minarea)
    out, nsplit = oracle.deblend(seg, nu, m, thresh, minarea, **kw)
    return seg, out, nsplit


def _objects_are_connected_partitions(seg, out):
    for L in np.unique(seg[seg > 0]):
        inseg = seg == L
        labs = np.unique(out[inseg])
        assert 0 not in labs and np.all(out[~(seg > 0)] == 0)
        for k in labs:
            obj = out == k
            assert np.all(inseg[obj])
            assert oracle.label(obj.astype(np.uint8), 1)[1] == 1          # 8-connected
            assert k == 1 + np.flatnonzero(obj.ravel())[0]                # canonical label


def test_deblend_keeps_a_single_star():
    m = _blend([(30, 20, 200.0)])
    seg, out, nsplit = _deblend_map(m)
    assert nsplit == 0 and np.array_equal(out, seg)


def test_deblend_splits_a_touching_pair_at_their_peaks():
    m = _blend([(26, 24, 150.0), (40, 25, 110.0)])
    seg, out, nsplit = _deblend_map(m)
    assert len(np.unique(seg[seg > 0])) == 1 and nsplit == 1
    labs = np.unique(out[out > 0])
    assert len(labs) == 2
    assert out[24, 26] != out[25, 40]                  # each peak in its own object
    _objects_are_connected_partitions(seg, out)
    # a pixel on the line between the peaks goes to the nearer, brighter side
    assert out[24, 29] == out[24, 26] and out[25, 37] == out[25, 40]


def test_deblend_contrast_decides_a_faint_companion():
    """A sharp companion 10 px from a bright star, joined to it above the
    threshold (the saddle stays above 1.5): with 0.4 % of the segment's flux
    it stays part of the star, with 1.6 % it is split off (minarea 1, so the
    contrast alone decides)."""
    for amp, split in ((5.0, False), (20.0, True)):
        m = _blend([(30, 24, 200.0)], s=2.5) + _blend([(40, 24, amp)], s=1.0)
        seg, out, nsplit = _deblend_map(m, minarea=1)
        assert len(np.unique(seg[seg > 0])) == 1
        frac = amp * 2 * np.pi / m[seg > 0].sum()
        assert (frac > 0.005) == split
        assert (nsplit == 1) == split, (amp, nsplit)
        if split:
            assert out[24, 30] != out[24, 40]
            _objects_are_connected_partitions(seg, out)


def test_deblend_three_peaks_and_nested_levels():
    m = _blend([(20, 20, 180.0), (33, 21, 140.0), (27, 33, 120.0)])
    seg, out, nsplit = _deblend_map(m)
    assert nsplit == 1
    assert len({out[20, 20], out[21, 33], out[33, 27]}) == 3
    assert len(np.unique(out[seg > 0])) == 3
    _objects_are_connected_partitions(seg, out)
    # fewer levels cannot resolve more than they separate; one level never splits
    _, out1, ns1 = _deblend_map(m, nthresh=1)
    assert ns1 == 0
    # mincont 1: no branch carries the whole flux, nothing splits
    _, _, nsx = _deblend_map(m, mincont=1.0)
    assert nsx == 0


def test_deblend_leaves_isolated_segments_alone():
    m = _blend([(15, 15, 100.0)]) + _blend([(55, 30, 120.0), (62, 31, 90.0)])
    seg, out, nsplit = _deblend_map(m)
    L = seg[15, 15]
    assert np.array_equal(out[seg == L], seg[seg == L])
    assert nsplit == 1


def _moffat(H, W, stars, fwhm=3.0, beta=2.5):
    """Moffat stars (x0, y0, total flux) sampled at pixel centres."""
    alpha = fwhm / (2.0 * np.sqrt(2.0 ** (1.0 / beta) - 1.0))
    yy, xx = np.mgrid[0:H, 0:W]
    m = np.zeros((H, W))
    for x0, y0, f in stars:
        r2 = (xx - x0) ** 2 + (yy - y0) ** 2
        m += f * (beta - 1.0) / (np.pi * alpha * alpha) * (1.0 + r2 / (alpha * alpha)) ** (-beta)
    return m


def _bridged_pair(H=48, W=72):
    """Two well-separated Moffat stars (32 px apart, far below threshold
    between them) joined by a faint one-pixel bridge of 3 (threshold 1.5)."""
    m = _moffat(H, W, [(20, 24, 5000.0), (52, 24, 4000.0)])
    m[24, 20:53] = np.maximum(m[24, 20:53], 3.0)
    return m


def test_deblend_splits_moffats_joined_by_a_faint_bridge():
    m = _bridged_pair()
    seg, out, nsplit = _deblend_map(m)
    assert len(np.unique(seg[seg > 0])) == 1            # one segment through the bridge
    assert nsplit == 1
    assert len(np.unique(out[out > 0])) == 2
    assert out[24, 20] != out[24, 52]
    _objects_are_connected_partitions(seg, out)
    # the bridge goes to the nearer star on either side of the midpoint
    assert out[24, 30] == out[24, 20] and out[24, 44] == out[24, 52]


def test_deblend_keeps_a_single_moffat_with_a_faint_tail():
    m = _moffat(48, 72, [(20, 24, 5000.0)])
    m[24, 20:53] = np.maximum(m[24, 20:53], 3.0)         # the same bridge, no star at its far end
    seg, out, nsplit = _deblend_map(m)
    assert nsplit == 0 and np.array_equal(out, seg)


def test_deblend_is_invariant_to_flux_scaling():
    """Scaling m, nu and the threshold by one factor leaves every level set
    (t_i / thresh depends on nu_max / thresh only) and every contrast ratio
    unchanged.  By a power of two the arithmetic is exact, so the maps must be
    identical.  The frames sweep a companion's distance and brightness, so
    that for some of them whether a level falls between the saddle and the
    companion's peak decides the split: a ladder that is not anchored at the
    threshold (t_i = thresh * nu_max^(i/N), say) moves with the scale there
    and changes 13 of the sweep's 44 scaled maps."""
    m = _bridged_pair() + _moffat(48, 72, [(36, 8, 800.0)])
    frames = [m] + [_blend([(26, 24, 150.0), (26 + d, 24.5, a2)])
                    for d in np.arange(4.0, 9.01, 0.5) for a2 in (60.0, 120.0)]
    nsplit = 0
    for f in frames:
        _, ref, nref = _deblend_map(f, thresh=1.5)
        nsplit += nref
        for c in (4.0, 0.25):
            _, out, n = _deblend_map(c * f, thresh=1.5 * c)
            assert n == nref
            assert np.array_equal(out, ref), c
    assert 0 < nsplit < len(frames)         # the sweep crosses the split boundary
