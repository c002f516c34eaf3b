"""Helpers shared by the GPU parity tests: running the CUDA path through the
C ABI, and the tolerance rules for comparing it with the oracle.

Tolerances (relative 1e-5, scaled by the conditioning of each quantity):
  meshes / maps    |d| <= 1e-5 |oracle| + 1e-6
  segment sums     |d| <= 1e-5 sum|m|            (flux_iso)
  centroids        |d| <= 1e-5 sum(|m| |x - xc|) / |S|
  second moments   |d| <= 1e-5 sum(|m| (x - xc)^2) / |S|
  aperture flux    |d| <= 1e-5 sum(A |m|)
  aperture error   |d| <= 1e-5 |oracle|
Each is the first-order error bound of a sum whose terms carry a 1e-5
relative error, so an ill-conditioned quantity (a faint segment whose sum
nearly cancels) is not held to a bound its own arithmetic cannot meet.
"""
import numpy as np

REL = 1e-5


def rel_report(name, got, ref, scale):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    scale = np.asarray(scale, np.float64)
    err = np.abs(got - ref) / np.maximum(scale, 1e-300)
    if err.size == 0:
        return 0.0, 0.0
    mx = float(err.max())
    p99 = float(np.quantile(err, 0.99))
    print(f"  {name:14s} max {mx:.3e}  p99 {p99:.3e}  (relative to the scale, n={err.size})")
    return mx, p99


def assert_close(name, got, ref, scale, rel=REL):
    mx, _ = rel_report(name, got, ref, scale)
    assert mx <= rel, f"{name}: max scaled error {mx:.3e} > {rel}"


def segment_scales(seg, m, cat):
    """sum|m|, sum|m||dx|, sum|m||dy|, sum|m|dx^2 ... per catalog row (oracle
    order), from the oracle's m and its centroids."""
    H, W = seg.shape
    lab = seg.ravel()
    idx = np.flatnonzero(lab)
    ls = lab[idx]
    order = np.searchsorted(cat["label"], ls)
    am = np.abs(m.ravel()[idx])
    x = (idx % W).astype(np.float64)
    y = (idx // W).astype(np.float64)
    n = len(cat["label"])
    dx = x - cat["x"][order]
    dy = y - cat["y"][order]
    s_abs = np.bincount(order, am, n)
    s_dx = np.bincount(order, am * np.abs(dx), n)
    s_dy = np.bincount(order, am * np.abs(dy), n)
    s_d2 = np.bincount(order, am * (dx * dx + dy * dy + np.abs(dx * dy)), n)
    S = np.abs(cat["flux"])
    S = np.where(S > 0, S, 1.0)
    return s_abs, s_dx / S, s_dy / S, s_d2 / S
