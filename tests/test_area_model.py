"""The exact-overlap arithmetic of the aperture kernels, restated in float32
on the host, against the oracle's float64 disc/pixel areas (Section 3.4).

The kernel computes the area of a pixel crossed by the circle by folding it
into the first quadrant, one rectangle plus one arc integral, with the
hardware's approximate square root and division and its own arctangent (a
degree-8 polynomial in u^2 fitted to atan(u)/u on [0, 1]).  This model runs
the same float32 steps; the approximate square root and division are modelled
as the correctly rounded result moved by up to one and two ulps.  It pins
the polynomial and the arrangement of the formula, not the GPU's bits (the
GPU parity tests compare those with the oracle).
"""
import numpy as np
import pytest

import oracle

f32 = np.float32
# coefficients of P in atan(u) = u P(u^2), lowest first (as in the kernel)
ATAN_P = [1.0, -0.33333093, 0.19993053, -0.14207125, 0.10654641, -0.07533597, 0.043038424, -0.01628242,
          0.002903404]


class Model:
    def __init__(self, seed):
        self.rng = np.random.default_rng(seed)
        self.c = [f32(c) for c in ATAN_P]

    def _pert(self, x, ulps):
        x = f32(x)
        k = int(self.rng.integers(-ulps, ulps + 1))
        if k == 0:
            return x
        return np.nextafter(x, f32(np.inf) if k > 0 else f32(-np.inf), dtype=f32)

    def sqrt(self, x):
        return self._pert(np.sqrt(f32(x)), 1)

    def div(self, a, b):
        return self._pert(f32(a) / f32(b), 2)

    @staticmethod
    def fma(a, b, c):
        return f32(np.float64(a) * np.float64(b) + np.float64(c))

    def atan_q1(self, y, x):
        sw = y > x
        u = self.div(x if sw else y, y if sw else x)
        s = f32(u * u)
        p = self.c[8]
        for c in self.c[7::-1]:
            p = self.fma(p, s, c)
        a = f32(u * p)
        return f32(f32(1.57079637) - a) if sw else a

    def chord_int(self, a, b, r2):
        d = f32(b - a)
        if not d > 0:
            return f32(0)
        ha = self.sqrt(max(self.fma(-a, a, r2), f32(0)))
        hb = self.sqrt(max(self.fma(-b, b, r2), f32(0)))
        s = f32(ha + hb)
        q = self.div(f32(d * f32(a + b)), s) if s > 0 else f32(0)
        sin_t = self.fma(d, ha, f32(a * q))
        cos_t = self.fma(ha, hb, f32(a * b))
        return f32(f32(0.5) * self.fma(r2, self.atan_q1(sin_t, cos_t), self.fma(d, hb, f32(-a * q))))

    def quadrant_area(self, x0, x1, y0, y1, r2):
        if not self.fma(x0, x0, f32(y0 * y0)) < r2:
            return f32(0)
        xa = self.sqrt(max(self.fma(-y1, y1, r2), f32(0)))
        xb = self.sqrt(max(self.fma(-y0, y0, r2), f32(0)))
        lo = min(max(xa, x0), x1)
        d = max(f32(min(x1, xb) - lo), f32(0))
        rect = f32(f32(y1 - y0) * f32(lo - x0))
        return f32(rect + self.fma(-y0, d, self.chord_int(lo, f32(lo + d), r2)))

    @staticmethod
    def fold(a):
        b = f32(a + f32(1))
        two = a < 0 and b > 0
        p0 = a if a >= 0 else (-b if b <= 0 else f32(0))
        p1 = b if a >= 0 else (-a if b <= 0 else b)
        return f32(p0), f32(p1), f32(-a), two

    def pixel_area(self, dx0, dy0, r):
        r2 = f32(r * r)
        fx, fy = self.fold(dx0), self.fold(dy0)
        A = self.quadrant_area(fx[0], fx[1], fy[0], fy[1], r2)
        if fx[3]:
            A = f32(A + self.quadrant_area(f32(0), fx[2], fy[0], fy[1], r2))
        if fy[3]:
            A = f32(A + self.quadrant_area(fx[0], fx[1], f32(0), fy[2], r2))
        if fx[3] and fy[3]:
            A = f32(A + self.quadrant_area(f32(0), fx[2], f32(0), fy[2], r2))
        return A


def test_atan_polynomial_relative_error():
    """atan(u) = u P(u^2) on [0, 1] within 1e-7 relative (float64 evaluation),
    and the quadrant angle of the model against arctan2 over all directions."""
    u = np.linspace(0.0, 1.0, 100001)[1:]
    p = np.polyval(np.array(ATAN_P[::-1]), u * u)
    assert np.max(np.abs(u * p - np.arctan(u)) / np.arctan(u)) < 1e-7
    m = Model(0)
    ang = np.linspace(1e-4, np.pi / 2 - 1e-4, 2001)
    got = np.array([m.atan_q1(f32(np.sin(a)), f32(np.cos(a))) for a in ang], np.float64)
    ref = np.arctan2(np.sin(ang).astype(f32).astype(np.float64), np.cos(ang).astype(f32).astype(np.float64))
    assert np.max(np.abs(got - ref) / ref) < 5e-7


@pytest.mark.parametrize("r,bound", [(0.3, 2e-7), (3.0, 1e-6), (10.0, 3e-6), (100.0, 3e-5)])
def test_pixel_area_model_against_oracle(r, bound):
    """Pixels near the circle (random centre, random direction): the float32
    model of the kernel's area within `bound` of the oracle's exact area."""
    m = Model(1)
    rng = np.random.default_rng(2)
    r32 = f32(r)
    worst = 0.0
    for _ in range(1500):
        cx, cy = rng.uniform(0, 1, 2)
        ang = rng.uniform(0, 2 * np.pi)
        rad = r + rng.uniform(-1.5, 1.5)
        dx0 = f32(np.floor(cx + rad * np.cos(ang)) - cx)
        dy0 = f32(np.floor(cy + rad * np.sin(ang)) - cy)
        g = float(m.pixel_area(dx0, dy0, r32))
        o = oracle.overlap_area(float(dx0), float(dx0) + 1.0, float(dy0), float(dy0) + 1.0, float(r32))
        worst = max(worst, abs(g - o))
    assert worst < bound, (r, worst)
