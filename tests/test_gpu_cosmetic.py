"""The cosmetic corrections (paper Section 3.1) through gp_cosmetic, against
the oracle.

On integer frames the salt-and-pepper filter's medians and residuals are
exact in float32, so its decisions and values must be bit-exact.  The
cosmic-ray filter's decisions compare float values (S less its median,
L+ / F) with thresholds; they must agree except where the oracle's value
lies within 1e-4 (relative) of the threshold, and the corrected frame must
agree at every pixel whose 5 x 5 window holds no such pixel.
"""
import numpy as np
import pytest

import oracle
import synth

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


def frame_u16(seed, w=640, h=520):
    cfg = synth.scaled_config(synth.CONFIGS["plain_2048x2048_u16"], w, h)
    img, _ = synth.make_frame(cfg, seed, cache=False)
    rng = np.random.default_rng(seed)
    img = img.astype(np.int64)
    # telegraph-noise pixels (isolated jumps) and a few adjacent pairs
    for _ in range(60):
        y, x = rng.integers(0, h), rng.integers(0, w)
        img[y, x] += int(rng.choice([-1, 1])) * int(rng.integers(200, 900))
    for _ in range(5):
        y, x = rng.integers(1, h - 1), rng.integers(1, w - 2)
        img[y, x] += 600
        img[y, x + 1] += 600
    return np.clip(img, 0, 65535).astype(np.uint16), cfg


def widen(m, r):
    """True where a (2r+1)^2 window around the pixel holds a True."""
    out = np.zeros_like(m)
    H, W = m.shape
    for y, x in np.argwhere(m):
        out[max(0, y - r):y + r + 1, max(0, x - r):x + r + 1] = True
    return out


def test_rtn_bit_exact_on_integer_frames(ctx):
    img, _ = frame_u16(61)
    t = 150.5
    ref, rep = oracle.rtn_filter(img, t)
    out = ctx.gp_cosmetic(dev(img), rtn_t=t)
    ctx.sync()
    g = out["image"].cpu().numpy()
    fl = out["flags"].cpu().numpy()
    assert rep.sum() > 20
    assert np.array_equal(fl == 1, rep)
    assert np.array_equal(g.astype(np.float64), ref)
    assert out["counts"].cpu().numpy().tolist() == [int(rep.sum()), 0]


def test_cr_matches_the_oracle(ctx):
    img, cfg = frame_u16(62)
    gain, rn = cfg.gain, 8.0
    ref, flag, d = oracle.cr_filter(img, gain, rn, 4.5, 5.0, details=True)
    out = ctx.gp_cosmetic(dev(img), cr_gain=gain, cr_read_noise=rn, cr_sigclip=4.5, cr_objlim=5.0)
    ctx.sync()
    g = out["image"].cpu().numpy().astype(np.float64)
    gf = out["flags"].cpu().numpy() == 2
    amb = (np.abs(d["sp"] - 4.5) <= 1e-4 * 4.5) | (np.abs(d["ratio"] - 5.0) <= 1e-4 * 5.0)
    print(f"\n{img.shape}: oracle flagged {int(flag.sum())}, gpu {int(gf.sum())}, near a threshold {int(amb.sum())}")
    assert flag.sum() > 20
    assert np.array_equal(gf[~amb], flag[~amb])
    sure = ~widen(amb, 2)
    assert np.array_equal(g[sure], ref[sure])
    assert int(out["counts"].cpu().numpy()[1]) == int(gf.sum())


def test_both_filters_with_bad_pixels_float32(ctx):
    img, cfg = frame_u16(63, 500, 430)
    f = img.astype(np.float32)
    rng = np.random.default_rng(63)
    f[rng.random(f.shape) < 0.002] = np.nan
    mask = np.zeros(f.shape, np.uint8)
    mask[rng.random(f.shape) < 0.003] = 1
    mask[100:104, 200:230] = 1
    c1, fl1, d = oracle.cr_filter(f, cfg.gain, 8.0, 4.5, 5.0, mask=mask, details=True)
    ref, rep = oracle.rtn_filter(c1, 150.5, mask=mask)
    out = ctx.gp_cosmetic(dev(f), rtn_t=150.5, cr_gain=cfg.gain, cr_read_noise=8.0, mask=dev(mask))
    ctx.sync()
    g = out["image"].cpu().numpy().astype(np.float64)
    fl = out["flags"].cpu().numpy()
    amb = (np.abs(d["sp"] - 4.5) <= 1e-4 * 4.5) | (np.abs(d["ratio"] - 5.0) <= 1e-4 * 5.0)
    near = widen(amb, 3)
    assert np.array_equal(((fl & 2) != 0)[~amb], fl1[~amb])
    assert np.array_equal(((fl & 1) != 0)[~near], rep[~near])
    same = ~near
    both_nan = np.isnan(g) & np.isnan(ref)
    assert np.all(both_nan[same] | (g[same] == ref[same]))
    bad = (mask != 0) | ~np.isfinite(f)
    assert not (fl[bad] != 0).any()


def test_cosmetic_rejects_bad_parameters(ctx):
    img = dev(np.full((64, 64), 1000, np.uint16))
    for kw in ({}, {"cr_gain": 1.0, "cr_read_noise": 0.0}, {"rtn_t": float("inf")}):
        with pytest.raises(gp.GpError):
            ctx.gp_cosmetic(img, **kw)
