"""Pins of the CPU reference convolution used by the pressure operator's GPU tests: against
scipy's 2-D correlation, and the adjoint identities that the weight- and input-gradient
passes must satisfy (<conv(x, w), g> = <x, conv(g, flip(w))> = <w, wgrad(x, g)>)."""
import numpy as np
import pytest

from _conv_ref import bf16_round, conv3x3, conv3x3_wgrad, flip

signal = pytest.importorskip("scipy.signal")


def test_conv_matches_scipy_correlation():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 9, 11, 3))
    w = rng.standard_normal((9, 4, 3))
    y = conv3x3(x, w)
    for n in range(2):
        for co in range(4):
            ref = np.zeros((9, 11))
            for ci in range(3):
                k = w[:, co, ci].reshape(3, 3)          # k[dy + 1, dx + 1]
                ref += signal.correlate2d(x[n, :, :, ci], k, mode="same", boundary="fill")
            assert np.allclose(y[n, :, :, co], ref, atol=1e-12)


def test_gradients_are_adjoints():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((1, 7, 6, 5))
    g = rng.standard_normal((1, 7, 6, 4))
    w = rng.standard_normal((9, 4, 5))
    lhs = np.sum(conv3x3(x, w) * g)
    assert np.isclose(lhs, np.sum(x * conv3x3(g, flip(w))), rtol=1e-12)
    assert np.isclose(lhs, np.sum(w * conv3x3_wgrad(x, g)), rtol=1e-12)


def test_bf16_rounding():
    v = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -2.5, 1e-3], dtype=np.float32)
    r = bf16_round(v)
    assert r[0] == 1.0 and r[1] == 1.0            # tie to even
    assert r[2] == 1.0 + 2 ** -7                  # rounds up
    assert r[3] == -2.5
    assert abs(r[4] - 1e-3) <= 1e-3 * 2 ** -8


def test_network_gradients_match_finite_differences():
    """The reference network's gradients (no BF16 rounding) against central differences of
    its loss, for a few weights and biases of every layer."""
    from _conv_ref import network_gradients
    rng = np.random.default_rng(2)
    feat = np.zeros((1, 6, 5, 16))
    feat[..., :4] = rng.standard_normal((1, 6, 5, 4))
    t = rng.standard_normal((1, 6, 5))
    layers = [(16, 32), (32, 32), (32, 32), (32, 32), (32, 16)]
    W = [rng.standard_normal((9, co, ci)) * 0.2 for ci, co in layers]
    B = [rng.standard_normal(co) * 0.1 for ci, co in layers]
    loss, dW, db = network_gradients(feat, t, W, B, rounding=False)
    h = 1e-6
    for l in range(5):
        for _ in range(3):
            idx = tuple(rng.integers(0, s) for s in W[l].shape)
            Wp = [w.copy() for w in W]
            Wm = [w.copy() for w in W]
            Wp[l][idx] += h
            Wm[l][idx] -= h
            fd = (network_gradients(feat, t, Wp, B, rounding=False)[0]
                  - network_gradients(feat, t, Wm, B, rounding=False)[0]) / (2 * h)
            assert fd == pytest.approx(dW[l][idx], rel=1e-5, abs=1e-7 * max(1.0, abs(loss)))
        j = int(rng.integers(0, B[l].size))
        Bp = [b.copy() for b in B]
        Bm = [b.copy() for b in B]
        Bp[l][j] += h
        Bm[l][j] -= h
        fd = (network_gradients(feat, t, W, Bp, rounding=False)[0]
              - network_gradients(feat, t, W, Bm, rounding=False)[0]) / (2 * h)
        assert fd == pytest.approx(db[l][j], rel=1e-5, abs=1e-7 * max(1.0, abs(loss)))
