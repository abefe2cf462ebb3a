"""Pin: link-wise wall rules of Sec. 4 reproduce linear fields exactly.

Anti-bounce-back with the wall value taken where the link crosses the wall makes a linear
pressure an exact steady state of the pressure LBE for any tau_f: f_i = w_i (P - tau c_i.G)
is invariant under collision + streaming, and -f_opp^+ + 2 w_opp P(wall) equals it at the
boundary.  The same holds for a linear saturation when phi = beta (Gamma_i = w_i beta for
i >= 1).  Bounce-back conserves the totals (see the conservation tests).
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from _problems import constant_diffusivity


def traces(fun, nx, ny, dx):
    out = []
    for side in range(4):
        x, y = W.wall_trace_points(side, nx, ny, dx)
        out.append(fun(x, y))
    return out


@pytest.mark.parametrize("bc,grad", [((2, 2, 0, 0), (0.7, 0.0)), ((2, 2, 2, 2), (0.7, -0.4)),
                                     ((0, 0, 2, 2), (0.0, 1.3))])
@pytest.mark.parametrize("tau", [0.55, 1.0, 2.7])
def test_linear_pressure_is_exact(bc, grad, tau):
    nx, ny = 12, 10
    dx = 1.0 / nx
    a, b, c = 0.3, grad[0], grad[1]
    fun = lambda x, y: a + b * x + c * y
    Pb = traces(fun, nx, ny, dx)
    X, Y = W.node_coords(nx, ny, dx)
    p = constant_diffusivity(nx, ny, 0.02, tau, bc=bc, S0=0.0, P_b=Pb, S_b=[np.zeros_like(t) for t in Pb])
    o = O.Oracle(p, tol=1e-15, check_every=5, max_sub_iters=200000)
    fl = o.fields()
    o.close()
    assert np.max(np.abs(fl["P"] - fun(X, Y))) < 1e-11
    assert np.max(np.abs(fl["gradPx"] - b)) < 1e-9
    assert np.max(np.abs(fl["gradPy"] - c)) < 1e-9


def test_linear_saturation_is_steady_for_phi_equal_beta():
    nx, ny = 10, 8
    dx = 1.0 / nx
    Sfun = lambda x, y: 0.2 + 0.5 * x
    Sb = traces(Sfun, nx, ny, dx)
    Pb = [np.ones_like(t) for t in Sb]
    X, Y = W.node_coords(nx, ny, dx)
    p = constant_diffusivity(nx, ny, 0.02, 1.0, bc=(2, 2, 0, 0), phi=1.0, beta=1.0,
                             S0=Sfun(X, Y), P0=np.ones((ny, nx)), P_b=Pb, S_b=Sb)
    o = O.Oracle(p, tol=1e-14, check_every=2)
    st, k, r = o.step(25)
    S = o.fields()["S"]
    o.close()
    assert st == O.OK
    assert np.max(np.abs(S - Sfun(X, Y))) < 1e-12
