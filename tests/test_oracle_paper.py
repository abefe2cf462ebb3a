"""Pin: the paper's analytic examples (Sec. 4.1, 4.2) reproduced by the oracle.

The paper prints upper bounds on the global relative errors (Sec. 4) for Example 1 at 64^2
and Example 2 at 128^2, and second-order convergence in space.  Bounds and citations are
in tests/golden/paper_bounds.json.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
import workloads as W

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_bounds.json")))


def _errors(prob, tol):
    o, log = O.run_problem(prob, tol=tol)
    T = prob.steps * prob.dt
    fl = o.fields()
    ex = prob.exact_at(T)
    o.close()
    return {k: W.rel_l1(fl[k], ex[k]) for k in ("P", "ux", "uy", "S")}


def test_example1_error_bound():
    g = GOLD["example1"]
    prob = W.example1(g["n"], g["c"])
    assert prob.steps * prob.dt == pytest.approx(g["T"])
    err = _errors(prob, 1e-10)
    for k, e in err.items():
        assert e < g["bound"], (k, e)


def test_example1_second_order():
    errs = [_errors(W.example1(n, 1.0), 1e-10) for n in (32, 64, 128)]
    for k in ("P", "ux", "S"):
        order = math.log(errs[0][k] / errs[2][k]) / math.log(4.0)
        assert order > 1.8, (k, order)


def test_example2_error_bound():
    g = GOLD["example2"]
    prob = W.example2(g["n"], g["c"])
    assert prob.steps * prob.dt == pytest.approx(g["T"])
    err = _errors(prob, 1e-8)
    for k, e in err.items():
        assert e < g["bound"], (k, e)


def test_example2_errors_fall_with_beta_at_phi_half():
    g = GOLD["example2_beta_sweep"]
    errs = [_errors(W.example2(48, phi=g["phi"], beta=b), 1e-8) for b in g["betas"]]
    for k in ("P", "ux", "S"):
        seq = [e[k] for e in errs]
        assert all(a > b for a, b in zip(seq, seq[1:])), (k, seq)
