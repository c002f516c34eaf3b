"""The seeded synthetic frames follow the recipes they stand for (no GPU):
the flux law, the blended pairs of the dense workload, the CCD defects of
the 4.2 MP workload, the sky levels, the sizes kept by scaling, and the
Poisson arrivals of the serving stream."""
import numpy as np
import pytest

import synth

scipy_stats = pytest.importorskip("scipy.stats")


def test_fluxes_follow_the_differential_power_law():
    """dN/dF ~ F^-1.5 on [lo, hi]: the drawn fluxes against the analytic CDF
    (F^-0.5 - lo^-0.5) / (hi^-0.5 - lo^-0.5), and the law's median."""
    lo, hi = 1e2, 1e5
    f = synth.power_law_fluxes(np.random.default_rng(3), 40_000, lo, hi, slope=-1.5)
    assert f.min() >= lo and f.max() <= hi
    a = -0.5
    cdf = lambda x: (np.asarray(x) ** a - lo ** a) / (hi ** a - lo ** a)
    assert scipy_stats.kstest(f, cdf).pvalue > 1e-3
    med = ((lo ** a + hi ** a) / 2) ** (1 / a)
    assert abs(np.median(f) / med - 1) < 0.02
    # a slope of -2.5 would give a different law: the test can tell them apart
    g = synth.power_law_fluxes(np.random.default_rng(3), 40_000, lo, hi, slope=-2.5)
    assert scipy_stats.kstest(g, cdf).pvalue < 1e-6


def test_dense_recipe_has_five_percent_blended_pairs():
    base = synth.CONFIGS["dense_12288x12304_u16"]
    cfg = synth.scaled_config(base, 1024, 1024)
    assert cfg.nsrc == round(134_000 * 1024 * 1024 / (12288 * 12304))      # the dense source density
    img, t = synth.make_frame(cfg, 11, cache=False)
    assert img.dtype == np.uint16 and img.shape == (1024, 1024)
    n = cfg.nsrc
    npair = int(round(n * 0.05 / 2))
    assert npair > 0 and len(t["x"]) == n
    # the pairs: the last npair sources are the companions of the npair before them
    a = slice(n - 2 * npair, n - npair)
    b = slice(n - npair, n)
    sep = np.hypot(t["x"][b] - t["x"][a], t["y"][b] - t["y"][a])
    fw = t["fwhm"][b]
    assert np.all(sep >= fw - 1e-9) and np.all(sep <= 2 * fw + 1e-9)
    assert 2 * npair / n == pytest.approx(0.05, abs=1.5 / n)
    # sky 2000 ADU plus a random field of 100 ADU standard deviation
    assert abs(float(np.median(img)) - 2000) < 300
    assert t["sky_mean"] == pytest.approx(2000, abs=300)


def test_ccd_recipe_has_hot_pixels_cosmic_rays_and_saturation():
    base = synth.CONFIGS["plain_2048x2048_u16"]
    cfg = synth.scaled_config(base, 512, 512)
    img, t = synth.make_frame(cfg, 4, cache=False)
    assert img.dtype == np.uint16
    nh = int(round(5e-4 * 512 * 512))
    hot = int((img >= 5000).sum())
    assert hot >= nh                                       # hot pixels U[5e3, 65535] (stars may add more)
    assert img.max() <= 65535
    # vignetting darkens the corners by up to 2 % of the 800 ADU sky
    c = np.median(img[240:272, 240:272].astype(np.float64))
    k = np.median(img[:32, :32].astype(np.float64))
    assert 0 < c - k < 0.04 * 800
    assert 1.5 <= t["fwhm"].min() and t["fwhm"].max() <= 5.0


def test_scaling_keeps_the_source_density():
    base = synth.CONFIGS["dense_12288x12304_u16"]
    for w, h in ((2048, 2048), (4096, 4096), (8192, 8192), (14200, 10650)):
        c = synth.scaled_config(base, w, h)
        assert c.nsrc == pytest.approx(134_000 * w * h / base.npix, abs=1)
        assert (c.mesh, c.thresh, c.radii) == (base.mesh, base.thresh, base.radii)


def test_poisson_arrivals_have_exponential_gaps():
    t = synth.poisson_arrivals(np.random.default_rng(0), 4.0, 20_000)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    assert gaps.mean() == pytest.approx(0.25, rel=0.03)
    assert scipy_stats.kstest(gaps, "expon", args=(0, 0.25)).pvalue > 1e-3
