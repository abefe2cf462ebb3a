"""Pin: the initial saturation distribution of Sec. 4 (Eqs. gini, gneq).

Its non-equilibrium part must carry the Chapman-Enskog moments of Appendix B:
sum_i eps g_i^(1) = -dt F_s / 2 (Eq. Sgi) and
sum_i c_i eps g_i^(1) = -beta tau_g dt c_s^2 grad S + dt gamma c_s^2 grad P (Eq. CigiB1),
which in lattice units read -F~_s/2 and -(beta tau_g/3) grad_X S + (gamma~/3) grad_X P.
grad_X S is the central difference of S_0 (periodic wrap); grad_X P is the oracle's local
gradient (Eq. 3-10a); gamma~ = -3 lambda_w K dt / dx^2 (Eq. 3-8).
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from _problems import uniform


def test_initial_g_moments_match_appendix_b():
    prob = W.manufactured_periodic(24)
    o = O.Oracle(prob, tol=1e-11)
    g0 = o.get_pre()["g"]
    c = o.constants()
    sc = o.scalars()
    fl = o.fields()
    Fs_t = o.saturation_source()
    o.close()
    G = c["Gamma"]
    S0 = prob.S0
    eps = g0 - G[:, None, None] * S0[None]
    assert np.max(np.abs(eps.sum(0) - (-0.5 * Fs_t))) < 1e-13
    ex = c["ex"][:, None, None]
    ey = c["ey"][:, None, None]
    gSx = 0.5 * (np.roll(S0, -1, axis=1) - np.roll(S0, 1, axis=1))
    gSy = 0.5 * (np.roll(S0, -1, axis=0) - np.roll(S0, 1, axis=0))
    gPx = fl["gradPx"] * prob.dx
    gPy = fl["gradPy"] * prob.dx
    lw = S0 ** 2 / prob.mu_w
    gam = -3.0 * lw * prob.K * prob.dt / prob.dx ** 2
    tg = sc["tau_g"]
    ex_mom = (ex * eps).sum(0)
    ey_mom = (ey * eps).sum(0)
    assert np.max(np.abs(ex_mom - (-(prob.beta * tg / 3) * gSx + gam / 3 * gPx))) < 1e-13
    assert np.max(np.abs(ey_mom - (-(prob.beta * tg / 3) * gSy + gam / 3 * gPy))) < 1e-13
    # S recovered from g(t=0) with Eq. 3-9b is S_0
    assert np.max(np.abs(fl["S"] - S0)) < 1e-14


# Wall branches of grad S0 (reading R9: mirror image across a no-flux wall, one-sided second
# order at a Dirichlet wall, central differences inside).  Each rule is exact for a quadratic
# S0 that is even about the no-flux walls, so the first moment of eps g^(1) must equal
# Eq. CigiB1 with the EXACT derivative of the quadratic at every node, walls included.
# Box "low_mirror": no-flux at XMIN and YMAX, Dirichlet at XMAX and YMIN,
#   S0 = a + c x^2 + d (ny - y)^2 (x, y from the lower-left corner, nodes at half-integers);
# box "high_mirror": the reflection (no-flux at XMAX and YMIN, Dirichlet at XMIN and YMAX),
#   S0 = a + c (nx - x)^2 + d y^2.
def _box(kind, nx=12, ny=10):
    a, c, d = 0.25, 0.002, 0.0015
    x = np.arange(nx) + 0.5
    y = (np.arange(ny) + 0.5)[:, None]
    if kind == "low_mirror":
        bc = (W.NOFLUX, W.DIRICHLET, W.DIRICHLET, W.NOFLUX)
        S0 = a + c * x ** 2 + d * (ny - y) ** 2
        dSx = 2 * c * x + 0 * y
        dSy = -2 * d * (ny - y) + 0 * x
    else:
        bc = (W.DIRICHLET, W.NOFLUX, W.NOFLUX, W.DIRICHLET)
        S0 = a + c * (nx - x) ** 2 + d * y ** 2
        dSx = -2 * c * (nx - x) + 0 * y
        dSy = 2 * d * y + 0 * x
    # a pressure gradient from the Dirichlet walls, so the advective term is exercised too
    Pb = [None] * 4
    Sb = [None] * 4
    for s in range(4):
        if bc[s] == W.DIRICHLET:
            n = ny if s < 2 else nx
            Pb[s] = np.full(2 * n + 1, 0.05 * (s + 1))
            Sb[s] = np.full(2 * n + 1, 0.3)
    prob = uniform(nx, ny, bc=bc, S0=S0, P_b=Pb, S_b=Sb, P0=np.zeros((ny, nx)))
    return prob, dSx, dSy


@pytest.mark.parametrize("kind", ["low_mirror", "high_mirror"])
def test_initial_g_moments_at_walls(kind):
    prob, dSx, dSy = _box(kind)
    o = O.Oracle(prob, tol=1e-12)
    g0 = o.get_pre()["g"]
    c = o.constants()
    sc = o.scalars()
    fl = o.fields()
    Fs_t = o.saturation_source()
    o.close()
    G = c["Gamma"]
    S0 = prob.S0
    eps = g0 - G[:, None, None] * S0[None]
    assert np.max(np.abs(eps.sum(0) - (-0.5 * Fs_t))) < 1e-13
    ex = c["ex"][:, None, None]
    ey = c["ey"][:, None, None]
    gPx = fl["gradPx"] * prob.dx
    gPy = fl["gradPy"] * prob.dx
    assert np.max(np.abs(gPx)) > 1e-3          # the advective term is not trivially zero
    lw = S0 ** 2 / prob.mu_w
    gam = -3.0 * lw * prob.K * prob.dt / prob.dx ** 2
    tg = sc["tau_g"]
    want_x = -(prob.beta * tg / 3) * dSx + gam / 3 * gPx
    want_y = -(prob.beta * tg / 3) * dSy + gam / 3 * gPy
    assert np.max(np.abs((ex * eps).sum(0) - want_x)) < 1e-13
    assert np.max(np.abs((ey * eps).sum(0) - want_y)) < 1e-13
