"""Pin: second-order convergence on the manufactured periodic problem, and the local
pressure gradient of Eq. 3-10a against the exact gradient and a central difference of P.

The manufactured p and S (workloads.manufactured_fields) solve Eqs. 2-15 and 2-18 with the
closed-form sources; with tau fixed under refinement (dt proportional to dx^2) the errors of
P (mean-free), u and S fall as dx^2 (Sec. 4, Remark III).
"""
import math

import numpy as np

import oracle as O
import workloads as W


def _run(n, T, p_amp=1.0, tol=1e-10):
    prob = W.manufactured_periodic(n, p_amp=p_amp)
    steps = int(round(T / prob.dt))
    o, log = O.run_problem(prob, nsteps=steps, tol=tol)
    fl = o.fields()
    o.close()
    ex = prob.exact_at(steps * prob.dt)
    err = dict(P=W.rel_l2(W.mean_free(fl["P"]), W.mean_free(ex["P"])),
               ux=W.rel_l2(fl["ux"], ex["ux"]), uy=W.rel_l2(fl["uy"], ex["uy"]),
               S=W.rel_l2(fl["S"], ex["S"]))
    return err, fl, prob


def test_manufactured_second_order():
    # p amplitude 0.2 keeps the advective Courant number below 1/2 on the 16^2 grid
    T = 4 * 4.0 / 16 ** 2
    errs = [_run(n, T, p_amp=0.2, tol=1e-9)[0] for n in (16, 32, 64)]
    for k in ("P", "ux", "uy", "S"):
        order = math.log(errs[1][k] / errs[2][k]) / math.log(2.0)
        assert 1.7 < order < 2.6, (k, [e[k] for e in errs], order)


def test_local_gradient_matches_exact_and_finite_difference():
    T = 4.0 / 16 ** 2
    d = {}
    for n in (32, 64):
        err, fl, prob = _run(n, T)
        m = W.manufactured_fields(*W.node_coords(n, n, prob.dx), T, p_amp=1.0)
        P = fl["P"]
        fdx = (np.roll(P, -1, axis=1) - np.roll(P, 1, axis=1)) / (2 * prob.dx)
        fdy = (np.roll(P, -1, axis=0) - np.roll(P, 1, axis=0)) / (2 * prob.dx)
        d[n] = (W.rel_l2(fl["gradPx"], m["gradPx"]), W.rel_l2(fl["gradPy"], m["gradPy"]),
                W.rel_l2(fl["gradPx"], fdx), W.rel_l2(fl["gradPy"], fdy))
    for j in range(4):
        assert d[64][j] < 1e-2
        assert d[32][j] / d[64][j] > 3.0, (j, d)
