"""A float32 decision taken against a float64 threshold (no GPU).

The deblending kernel computes each level t_i in float64 once per
candidate, rounds it toward minus infinity to float32, and compares the
float32 significance nu of every pixel with that float.  For a float nu,
nu > t holds exactly when nu > rd(t): if t is a float the two are equal;
otherwise rd(t) < t < the next float above rd(t), so no float lies in
(rd(t), t].  Checked here on random thresholds over many binades, with the
floats adjacent to each threshold, where a rounding to nearest would flip
decisions."""
import numpy as np


def rd32(t):
    """float64 -> float32 rounded toward minus infinity."""
    f = t.astype(np.float32)
    over = f.astype(np.float64) > t
    f[over] = np.nextafter(f[over], np.float32(-np.inf))
    return f


def test_rounding_down_keeps_every_strict_comparison():
    rng = np.random.default_rng(5)
    t = np.exp(rng.uniform(np.log(1e-3), np.log(1e6), 200_000))
    t = np.concatenate([t, np.float32(t[:1000]).astype(np.float64)])      # thresholds that are floats
    r = rd32(t)
    assert np.all(r.astype(np.float64) <= t)
    assert np.all(np.nextafter(r, np.float32(np.inf)).astype(np.float64) > t)
    near = [r, np.nextafter(r, np.float32(np.inf)), np.nextafter(r, np.float32(-np.inf)),
            t.astype(np.float32)]
    for nu in near:
        assert np.array_equal(nu.astype(np.float64) > t, nu > r)


def test_rounding_to_nearest_would_not():
    rng = np.random.default_rng(6)
    t = np.exp(rng.uniform(np.log(1e-3), np.log(1e6), 200_000))
    rn = t.astype(np.float32)
    nu = rn                                                # the float nearest to t
    wrong = (nu.astype(np.float64) > t) != (nu > rn)
    assert wrong.sum() > 1000                              # about half the thresholds round up
