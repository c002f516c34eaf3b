"""Pins of the learned-background network oracle (oracle/cnn.py): the
convolution against scipy's 2-D correlation, and the hand-written backward
pass against central finite differences."""
import numpy as np
import pytest
from scipy.signal import correlate2d

from oracle import cnn


def test_conv3x3_is_zero_padded_correlation():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(2, 7, 9, 3))
    W = rng.normal(size=(4, 3, 3, 3))
    b = rng.normal(size=4)
    y = cnn.conv3x3(x, W, b)
    for n in range(2):
        for co in range(4):
            ref = sum(correlate2d(x[n, :, :, ci], W[co, ci], mode="same", boundary="fill") for ci in range(3))
            assert np.allclose(y[n, :, :, co], ref + b[co], atol=1e-12)


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, 5, 6, 3))
    params = [(rng.normal(size=(4, 3, 3, 3)) * 0.5, rng.normal(size=4) * 0.1),
              (rng.normal(size=(4, 4, 3, 3)) * 0.5, rng.normal(size=4) * 0.1),
              (rng.normal(size=(2, 4, 3, 3)) * 0.5, rng.normal(size=2) * 0.1)]
    target = rng.normal(size=(2, 5, 6, 2))
    acts = cnn.forward(x, params)
    grads, _ = cnn.backward(acts, params, target)
    eps = 1e-6

    def loss(ps):
        return cnn.mse(cnn.forward(x, ps)[-1], target)

    for li in range(3):
        W, b = params[li]
        for idx in [(0, 0, 0, 0), (1, 2, 1, 2), (3 if W.shape[0] > 3 else 1, 1, 2, 0)]:
            Wp, Wm = W.copy(), W.copy()
            Wp[idx] += eps
            Wm[idx] -= eps
            ps_p = [p if i != li else (Wp, b) for i, p in enumerate(params)]
            ps_m = [p if i != li else (Wm, b) for i, p in enumerate(params)]
            fd = (loss(ps_p) - loss(ps_m)) / (2 * eps)
            assert grads[li][0][idx] == pytest.approx(fd, rel=1e-5, abs=1e-9)
        for j in range(b.size):
            bp, bm = b.copy(), b.copy()
            bp[j] += eps
            bm[j] -= eps
            fd = (loss([p if i != li else (W, bp) for i, p in enumerate(params)]) -
                  loss([p if i != li else (W, bm) for i, p in enumerate(params)])) / (2 * eps)
            assert grads[li][1][j] == pytest.approx(fd, rel=1e-5, abs=1e-9)


def test_bf16_round_matches_definition():
    vals = np.array([1.0, 1.00390625, 1.005859375, 3.14159265, -2.5e-3, 65504.0])
    r = cnn.bf16_round(vals)
    # bfloat16 keeps 8 significant bits: the rounded value has a zero low half
    u = r.astype(np.float32).view(np.uint32)
    assert np.all((u & 0xFFFF) == 0)
    assert np.all(np.abs(r - vals) <= np.abs(vals) * 2.0 ** -8)
    assert r[1] == 1.0                  # 1 + 2^-8 is a tie -> even mantissa (1.0)
    assert r[2] == 1.0078125            # above the tie -> up
