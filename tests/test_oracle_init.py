"""Pin: the initial saturation distribution of Sec. 4 (Eqs. gini, gneq).

Its non-equilibrium part must carry the Chapman-Enskog moments of Appendix B:
sum_i eps g_i^(1) = -dt F_s / 2 (Eq. Sgi) and
sum_i c_i eps g_i^(1) = -beta tau_g dt c_s^2 grad S + dt gamma c_s^2 grad P (Eq. CigiB1),
which in lattice units read -F~_s/2 and -(beta tau_g/3) grad_X S + (gamma~/3) grad_X P.
grad_X S is the central difference of S_0 (periodic wrap); grad_X P is the oracle's local
gradient (Eq. 3-10a); gamma~ = -3 lambda_w K dt / dx^2 (Eq. 3-8).
"""
import numpy as np

import oracle as O
import workloads as W


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
