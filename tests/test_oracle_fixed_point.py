"""Pin: the pressure sub-iteration converges to the exact fixed point of its own sweep, and
the stopping rule (checks every m sweeps on the relative increment) behaves as stated.

On a 6x6 lattice with heterogeneous tau_f, a source, and mixed walls (anti-bounce-back on
x, bounce-back on y), one sweep is an affine map f+ -> A f+ + b of the 324 stored values.
A and b are probed column by column; the fixed point of (I - A) f = b is solved with numpy
and compared with the iterated state.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from _problems import constant_diffusivity, uniform


def _problem(bc):
    nx = ny = 6
    rng = np.random.default_rng(21)
    Pb = [0.3 + 0.1 * rng.random(2 * ny + 1), -0.2 + 0.1 * rng.random(2 * ny + 1),
          np.zeros(2 * nx + 1), np.zeros(2 * nx + 1)]
    Sb = [np.full(2 * ny + 1, 0.5), np.full(2 * ny + 1, 0.5), np.full(2 * nx + 1, 0.5),
          np.full(2 * nx + 1, 0.5)]
    return uniform(nx, ny, bc=bc, K=np.exp(rng.standard_normal((ny, nx))),
                   S0=0.2 + 0.6 * rng.random((ny, nx)), Fp=rng.standard_normal((ny, nx)),
                   P_b=Pb, S_b=Sb, tau_p=1.2)


@pytest.mark.parametrize("bc", [(2, 2, 1, 1), (2, 2, 2, 2)])
def test_iteration_reaches_direct_fixed_point(bc):
    p = _problem(bc)
    o = O.Oracle(p, init_replay=0)
    n = 6 * 6 * 9
    st = o.get_state()
    tau = st["tau_f"]
    zero = np.zeros((9, 6, 6))
    o.set_state(f=zero, tau_f=tau)
    o.pressure(1)
    b = o.get_state()["f"].ravel().copy()
    A = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        o.set_state(f=e.reshape(9, 6, 6), tau_f=tau)
        o.pressure(1)
        A[:, j] = o.get_state()["f"].ravel() - b
    fstar = np.linalg.solve(np.eye(n) - A, b)
    o.set_state(f=zero, tau_f=tau)
    o.set_prev_pressure(np.zeros((6, 6)))
    status, k, r = o.pressure(-1)
    it = o.get_state()["f"].ravel()
    o.close()
    assert status == O.OK and r <= 1e-8
    # increment criterion: error ~ r / (1 - spectral radius)
    rho = max(abs(np.linalg.eigvals(A)))
    assert rho < 1.0
    assert np.max(np.abs(it - fstar)) <= 50.0 * 1e-8 / (1.0 - rho) * np.max(np.abs(fstar))


def test_stopping_rule_cadence_and_cap():
    prob = W.quarter_five_spot(20, seed=3)
    o = O.Oracle(prob, tol=1e-6, check_every=7)
    assert o.init_status == O.OK
    assert o.init_sub_iters % 7 == 0 and o.init_residual <= 1e-6
    o.close()
    o = O.Oracle(prob, tol=0.0, check_every=4, max_sub_iters=30)
    assert o.init_status == O.ENOTCONVERGED and o.init_sub_iters == 30
    st, k, r = o.step(2, replay=[5, 0])
    assert st == O.OK and list(k) == [5, 0]
    o.close()


def test_nan_source_is_reported():
    prob = W.quarter_five_spot(12, seed=3)
    Fp = np.zeros((12, 12))
    Fp[3, 4] = np.nan
    prob.Fp = Fp
    with pytest.raises(O.OracleError):
        O.Oracle(prob, tol=1e-8)


@pytest.mark.parametrize("bc", [(0, 0, 0, 0), (1, 1, 1, 1)])
def test_neutral_mode_does_not_block_convergence(bc):
    """With periodic or bounce-back walls on every side a constant added to P is neutral.
    Summing the collision over i >= 1 with Eq. 3-9a gives sum_i f_i^+ = sum_i f_i + F~ at
    every node, and such streaming keeps each population total, so a source with a nonzero
    total raises the mean of P by sum_x F~ / ((1 - w_0) n) every sweep while its shape
    settles.  The stopping rule's numerator is mean-free, so the solves still end (a raw
    increment would stay at the drift); between two solves the shape (mean-free P) stays put
    and the mean moves by exactly the drift of the sweeps run."""
    nx, ny = 16, 12
    rng = np.random.default_rng(31)
    Fp = 0.5 + rng.standard_normal((ny, nx))
    # decoupled mobility: tau_f does not depend on S, so the pressure shape cannot either
    prob = constant_diffusivity(nx, ny, 0.03, 1.2, bc=bc, Fp=Fp)
    o = O.Oracle(prob, tol=1e-10, check_every=8, max_sub_iters=20_000)
    assert o.init_status == O.OK, (o.init_status, o.init_sub_iters)
    P0 = o.fields()["P"]
    st, k, r = o.step(1)
    assert st == O.OK and 0 < k[0] < 20_000 and r[0] <= 1e-10
    P1 = o.fields()["P"]
    src = (o.scalars()["s"] * prob.dx ** 2 * Fp).sum()
    o.close()
    drift = int(k[0]) * src / ((1.0 - 4.0 / 9.0) * nx * ny)
    assert abs(drift) > 1e-2 * np.abs(P0 - P0.mean()).max()
    assert abs((P1.mean() - P0.mean()) - drift) <= 1e-9 * abs(drift)
    assert W.rel_l2(W.mean_free(P1), W.mean_free(P0)) < 1e-7
