"""Input generators: manufactured sources against symbolic differentiation and finite
differences; the Gaussian random field's statistics; wall trace geometry."""
import math

import numpy as np
import pytest

import workloads as W


def test_manufactured_sources_symbolic():
    sp = pytest.importorskip("sympy")
    x, y, t = sp.symbols("x y t", real=True)
    a = 2 * sp.pi
    mu_w, mu_n, phi, Ds, A = 1, 2, sp.Rational(1, 5), sp.Rational(1, 100), sp.Rational(7, 10)
    K = 1 + sp.Rational(1, 2) * sp.sin(a * x) * sp.sin(a * y)
    p = A * sp.sin(a * x) * sp.cos(a * y) * sp.exp(-t)
    S = sp.Rational(1, 2) + sp.Rational(1, 4) * sp.sin(a * x) * sp.sin(a * y) * sp.exp(-t)
    lw = S ** 2 / mu_w
    lt = lw + (1 - S) ** 2 / mu_n
    div = lambda c, f: sp.diff(c * sp.diff(f, x), x) + sp.diff(c * sp.diff(f, y), y)
    Fp = -div(K * lt, p)
    Fs = phi * sp.diff(S, t) - Ds * (sp.diff(S, x, 2) + sp.diff(S, y, 2)) - div(lw * K, p)
    fFp = sp.lambdify((x, y, t), Fp, "numpy")
    fFs = sp.lambdify((x, y, t), Fs, "numpy")
    X, Y = W.node_coords(9, 7, 0.11)
    m = W.manufactured_fields(X, Y, 0.37, p_amp=0.7)
    assert np.allclose(m["Fp"], fFp(X, Y, 0.37), rtol=1e-12, atol=1e-12)
    assert np.allclose(m["Fs"], fFs(X, Y, 0.37), rtol=1e-12, atol=1e-12)


def test_manufactured_sources_finite_difference():
    h = 1e-4
    X, Y = np.meshgrid(np.linspace(0.05, 0.95, 7), np.linspace(0.1, 0.9, 6))
    t = 0.2

    def fields(x, y, tt):
        return W.manufactured_fields(x, y, tt)

    m = fields(X, Y, t)

    def flux_div(coef_key):
        def flux(xx, yy):
            mm = fields(xx, yy, t)
            return mm[coef_key]
        return flux

    # D_p grad p and lambda_w K grad p by central differences of closed-form values
    def Dgradp(xx, yy, which):
        mm = fields(xx, yy, t)
        lw = mm["S"] ** 2
        lt = lw + (1 - mm["S"]) ** 2 / 2.0
        c = mm["K"] * (lt if which == "t" else lw)
        return c * mm["gradPx"], c * mm["gradPy"]

    for which, key, sign in (("t", "Fp", -1.0),):
        fx_p, _ = Dgradp(X + h, Y, which)
        fx_m, _ = Dgradp(X - h, Y, which)
        _, fy_p = Dgradp(X, Y + h, which)
        _, fy_m = Dgradp(X, Y - h, which)
        div = (fx_p - fx_m) / (2 * h) + (fy_p - fy_m) / (2 * h)
        assert np.allclose(m[key], sign * div, rtol=1e-6, atol=1e-6)


def test_grf_statistics_and_determinism():
    a = W.grf_lnK(128, 96, 1.0, 16.0, seed=2)
    b = W.grf_lnK(128, 96, 1.0, 16.0, seed=2)
    assert np.array_equal(a, b)
    assert abs(a.mean()) < 1e-12 and abs(a.std() - 1.0) < 1e-12
    c = W.grf_lnK(128, 96, 0.5, 16.0, seed=2)
    assert np.allclose(c, 0.5 * a)
    # correlation drops to ~exp(-1) at lag l for the Gaussian covariance exp(-r^2/l^2)
    g = W.grf_lnK(512, 512, 1.0, 16.0, seed=7)
    lag = 16
    corr = np.mean(g * np.roll(g, lag, axis=1))
    assert 0.2 < corr < 0.55


def test_wall_trace_geometry():
    x, y = W.wall_trace_points(W.XMIN, 8, 5, 0.1)
    assert x.shape == (11,) and np.all(x == 0.0) and y[0] == 0.0 and y[-1] == pytest.approx(0.5)
    x, y = W.wall_trace_points(W.YMAX, 8, 5, 0.1)
    assert x.shape == (17,) and np.all(y == pytest.approx(0.5)) and x[-1] == pytest.approx(0.8)


def test_quarter_five_spot_layout():
    p = W.quarter_five_spot(64, seed=2)
    assert p.bc == (W.NOFLUX,) * 4
    assert p.wells == [(0, 0, 1e-3, 0), (63, 63, 1e-3, 1)]
    assert p.dt == pytest.approx(4.0 / 64 ** 2)
    assert np.all(p.K > 0) and p.S0.min() == p.S0.max() == 0.2
