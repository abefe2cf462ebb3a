"""Pin: exact balance laws of the two LBEs under periodic and bounce-back walls.

Saturation: sum_i g_i^eq = phi S and sum_i w_i c_i = 0, so one collision changes
sum_i g_i by exactly dt F_s at every node (Eq. 2-1b with Eq. 3-9b), and streaming with
periodic or bounce-back walls moves populations without loss.  Hence the lattice total
grows by sum_x dt F_s per step, and with no source phi * sum S is constant.
Pressure: sum_i f_i^eq = 0 (Eq. 3-7a) and sum_i w_bar_i = 1, so with a uniform tau_f the
total T = sum_x sum_i f_i^+ obeys T' = (1 - 1/tau) T + sum_x s dx^2 F_p per sweep.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from _problems import constant_diffusivity, uniform


@pytest.mark.parametrize("bc", [(1, 1, 1, 1), (0, 0, 1, 1), (0, 0, 0, 0)])
def test_saturation_total_grows_by_source(bc):
    nx, ny = 23, 17
    rng = np.random.default_rng(5)
    lnK = W.grf_lnK(nx, ny, 1.0, 4.0, seed=11)
    Fs = 0.3 * rng.standard_normal((ny, nx))
    wells = [(0, 0, 1e-3, 0), (nx - 1, ny - 1, 1e-3, 1), (5, 9, 4e-4, 1)]
    p = uniform(nx, ny, bc=bc, K=np.exp(lnK), S0=0.2 + 0.1 * rng.random((ny, nx)), Fs=Fs,
                wells=wells)
    o = O.Oracle(p, tol=1e-9, init_replay=30)
    for _ in range(4):
        before = o.sums()["g"]
        st, k, r = o.step(1, replay=[20])
        after = o.sums()["g"]
        src = o.saturation_source().sum()
        assert abs((after - before) - src) <= 1e-12 * max(1.0, abs(after))
    o.close()


def test_zero_source_conserves_phi_S():
    nx, ny = 16, 12
    rng = np.random.default_rng(3)
    p = uniform(nx, ny, bc=(1, 1, 0, 0), K=np.exp(W.grf_lnK(nx, ny, 0.5, 3.0, seed=4)),
                S0=0.3 + 0.2 * rng.random((ny, nx)), P0=rng.standard_normal((ny, nx)))
    o = O.Oracle(p, tol=1e-9, init_replay=40)
    m0 = o.fields()["S"].sum()
    o.step(5, replay=[15] * 5)
    m1 = o.fields()["S"].sum()
    o.close()
    assert abs(m1 - m0) <= 1e-12 * abs(m0)


@pytest.mark.parametrize("bc", [(0, 0, 0, 0), (1, 1, 1, 1), (0, 0, 1, 1)])
def test_pressure_total_recursion(bc):
    nx, ny = 14, 9
    rng = np.random.default_rng(8)
    tau = 1.3
    Fp = rng.standard_normal((ny, nx))
    p = constant_diffusivity(nx, ny, 0.03, tau, bc=bc, S0=0.0, Fp=Fp,
                             P0=rng.standard_normal((ny, nx)))
    o = O.Oracle(p, init_replay=0)
    sc = o.scalars()
    srcsum = (sc["s"] * p.dx ** 2 * Fp).sum()
    T = o.sums()["f"]
    for _ in range(6):
        o.pressure(1)
        Tn = o.sums()["f"]
        assert abs(Tn - ((1 - 1 / tau) * T + srcsum)) <= 1e-12 * max(1.0, abs(Tn))
        T = Tn
    o.close()


def test_producer_takes_out_what_the_injector_puts_in_when_only_water_moves():
    """With the decoupled mobility of Sec. 4.1 (lambda_t = lambda_w) the water fraction
    f_w = lambda_w / lambda_t is 1 at any saturation, so a producer removes exactly what an
    injector of the same rate adds: in a closed box the lattice total of g stays put."""
    nx, ny = 18, 14
    rng = np.random.default_rng(12)
    wells = [(1, 2, 1e-3, 0), (nx - 2, ny - 3, 1e-3, 1)]
    p = constant_diffusivity(nx, ny, 0.03, 1.2, bc=(1, 1, 1, 1), wells=wells,
                             S0=0.3 + 0.2 * rng.random((ny, nx)))
    o = O.Oracle(p, tol=1e-9, init_replay=30)
    total0 = o.sums()["g"]
    for _ in range(4):
        st, k, r = o.step(1, replay=[16])
        src = o.saturation_source()
        assert src[2, 1] > 0.0 and src[ny - 3, nx - 2] == -src[2, 1]
        assert abs(o.sums()["g"] - total0) <= 1e-12 * abs(total0)
    o.close()


def test_balanced_wells_keep_the_mean_pressure():
    """An injector and a producer of the same rate in a closed box add no net pressure source
    (F_p = +q/dx^2 and -q/dx^2), so by the recursion of the population total the mean of P does
    not move from one converged step to the next, while P stands above its mean at the injector
    and below it at the producer."""
    nx, ny = 20, 16
    rng = np.random.default_rng(17)
    wells = [(2, 3, 1e-3, 0), (nx - 3, ny - 2, 1e-3, 1)]
    p = constant_diffusivity(nx, ny, 0.03, 1.2, bc=(1, 1, 1, 1), wells=wells,
                             S0=0.3 + 0.2 * rng.random((ny, nx)),
                             P0=0.01 * rng.standard_normal((ny, nx)))
    o = O.Oracle(p, tol=1e-10, check_every=8, max_sub_iters=20_000)
    assert o.init_status == O.OK
    P0 = o.fields()["P"]
    st, k, r = o.step(1)
    assert st == O.OK and k[0] > 0
    P1 = o.fields()["P"]
    o.close()
    span = P1.max() - P1.min()
    assert abs(P1.mean() - P0.mean()) <= 1e-10 * span
    assert P1[3, 2] > P1.mean() + 0.2 * span and P1[ny - 2, nx - 3] < P1.mean() - 0.2 * span
