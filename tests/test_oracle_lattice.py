"""Pin: D2Q9 constants of the oracle and the equilibrium moment conditions, Eq. 3-7.

The oracle's tables are compared with the paper's definitions evaluated independently here
(Eq. 3-6 from its trigonometric form) and with the exact rational moments of Eq. 3-7.
"""
import math
from fractions import Fraction as F

import numpy as np
import pytest

import oracle as O
from _problems import uniform


def _fr(x):
    return F(float(x)).limit_denominator(100000)


@pytest.fixture(scope="module")
def consts():
    o = O.Oracle(uniform(4, 4, phi=0.2, beta=0.4), init_replay=0)
    c = o.constants()
    o.close()
    return c


def test_velocities_follow_eq_3_6(consts):
    # Eq. 3-6: i = 1..4 at angles (i-1) pi/2; i = 5..8 at (2i-9) pi/4 with length sqrt(2)
    for i in range(9):
        if i == 0:
            e = (0, 0)
        elif i <= 4:
            a = (i - 1) * math.pi / 2
            e = (round(math.cos(a)), round(math.sin(a)))
        else:
            a = (2 * i - 9) * math.pi / 4
            e = (round(math.sqrt(2) * math.cos(a)), round(math.sqrt(2) * math.sin(a)))
        assert (consts["ex"][i], consts["ey"][i]) == e
        o = consts["opp"][i]
        assert (consts["ex"][o], consts["ey"][o]) == (-e[0], -e[1])


def test_weights_eq_3_5(consts):
    assert [_fr(w) for w in consts["w"]] == [F(4, 9)] + [F(1, 9)] * 4 + [F(1, 36)] * 4
    assert [_fr(w) for w in consts["wbar"]] == [F(0)] + [F(1, 8)] * 8


def test_pressure_equilibrium_moments_eq_3_7a(consts):
    w = [_fr(v) for v in consts["w"]]
    ex, ey = consts["ex"], consts["ey"]
    feq = [w[0] - 1] + w[1:]           # Eq. 3-3 with P = 1
    assert sum(feq) == 0
    assert sum(feq[i] * int(ex[i]) for i in range(9)) == 0
    assert sum(feq[i] * int(ey[i]) for i in range(9)) == 0
    cs2 = F(1, 3)
    assert sum(feq[i] * int(ex[i]) ** 2 for i in range(9)) == cs2
    assert sum(feq[i] * int(ey[i]) ** 2 for i in range(9)) == cs2
    assert sum(feq[i] * int(ex[i]) * int(ey[i]) for i in range(9)) == 0
    # Eq. 3-9a reads P from f_1..f_8 only: sum_{i>=1} f_i^eq / (1 - w0) = P
    assert sum(feq[1:]) / (1 - w[0]) == 1


@pytest.mark.parametrize("phi,beta", [(0.2, 0.4), (1.0, 1.0), (0.5, 0.25), (0.5, 1.0), (0.3, 0.45)])
def test_saturation_equilibrium_moments_eq_3_7b(phi, beta):
    o = O.Oracle(uniform(4, 4, phi=phi, beta=beta), init_replay=0)
    c = o.constants()
    o.close()
    G = [_fr(v) for v in c["Gamma"]]    # g_i^eq / S
    ex, ey = c["ex"], c["ey"]
    phi_f, beta_f = _fr(phi), _fr(beta)
    assert sum(G) == phi_f
    assert sum(G[i] * int(ex[i]) for i in range(9)) == 0
    assert sum(G[i] * int(ey[i]) for i in range(9)) == 0
    assert sum(G[i] * int(ex[i]) ** 2 for i in range(9)) == beta_f / 3
    assert sum(G[i] * int(ey[i]) ** 2 for i in range(9)) == beta_f / 3
    assert sum(G[i] * int(ex[i]) * int(ey[i]) for i in range(9)) == 0
    # Sec. 3: phi/2 <= beta <= 2 phi keeps every g_i^eq non-negative
    assert all(g >= 0 for g in G) == (phi_f / 2 <= beta_f <= 2 * phi_f)


def test_relaxation_times_eq_3_11():
    # config rule: tau_s = 0.8 at dt = 4 dx^2, beta = 0.4, D_s = 0.01 (Eq. 3-11b)
    o = O.Oracle(uniform(8, 8, phi=0.2, beta=0.4, D_s=0.01), init_replay=0)
    sc = o.scalars()
    o.close()
    assert sc["tau_g"] == pytest.approx(0.8, rel=1e-14)
    # reference mode: tau_f equals tau_p where D_p equals the geometric-mean reference
    p = uniform(8, 8, K=np.full((8, 8), 2.5), S0=0.3, tau_p=1.0)
    o = O.Oracle(p, init_replay=0)
    st = o.get_state()
    sc = o.scalars()
    o.close()
    lt = 0.3 ** 2 / 1.0 + 0.7 ** 2 / 2.0
    assert sc["D_ref"] == pytest.approx(2.5 * lt, rel=1e-13)
    assert np.allclose(st["tau_f"], 1.0, rtol=1e-13)
