"""Pins for the warm start of each pressure solve (the iteration starts from the pressure
extrapolated linearly in time, 2 P^n - P^{n-1}, keeping the non-equilibrium part of f).

- The shift f_i^+ += f_i^eq(dP) adds nothing to sum_i f_i^+, because sum_i f_i^eq = 0
  (Eq. 3-3, Eq. 3-7a): the total of the pressure populations is unchanged by it.
- The warm start moves only the starting iterate, not the fixed point of a solve: solved to a
  tight tolerance, runs with and without it give the same fields.
- It reaches the paper's stopping rule in far fewer sweeps once two steps of history exist.
"""
import numpy as np

import oracle as O
import workloads as W


def test_warm_start_keeps_the_population_total():
    prob = W.quarter_five_spot(40, seed=5, corr_len=6.0)
    o = O.Oracle(prob, init_replay=300, warm_start=1)
    o.step(2, replay=[64, 64])
    # the pressure populations' total after the step's S refresh (no f change) and after the
    # warm start: sum f^eq(dP) = 0
    o.refresh()
    before = o.sums()["f"]
    o2 = O.Oracle(prob, init_replay=300, warm_start=1)
    o2.step(2, replay=[64, 64])
    st, k, r = o2.step(1, replay=[0])       # refresh + warm start + no sweep + saturation
    after = o2.sums()["f"]
    o.close()
    o2.close()
    assert abs(after - before) <= 1e-12 * max(1.0, abs(before))


def test_warm_start_keeps_the_fixed_point():
    prob = W.quarter_five_spot(48, seed=6, corr_len=8.0)
    runs = []
    for ws in (0, 1):
        o, log = O.run_problem(prob, nsteps=6, tol=1e-12, warm_start=ws)
        runs.append((o.fields(), log))
        o.close()
    (a, la), (b, lb) = runs
    assert W.rel_l2(W.mean_free(b["P"]), W.mean_free(a["P"])) < 1e-7
    assert W.rel_l2(b["S"], a["S"]) < 1e-9
    assert W.rel_l2(b["ux"], a["ux"]) < 1e-6


def test_warm_start_cuts_sweeps():
    prob = W.quarter_five_spot(64, seed=2)
    o0, plain = O.run_problem(prob, nsteps=10, tol=1e-8, warm_start=0)
    o1, warm = O.run_problem(prob, nsteps=10, tol=1e-8, warm_start=1)
    o0.close()
    o1.close()
    assert plain[:2] == warm[:2]                # no history yet at the first step
    assert sum(warm[4:]) < 0.25 * sum(plain[4:]), (plain, warm)
