"""Warm start of every pressure solve (params.warm_start = 1: the equilibrium part of f moved
to the pressure extrapolated linearly in time) and from a caller's field (lbm2p_warm_start),
against the FP64 oracle doing the same (its counts replayed), and its effect on the sweep
counts of the paper's stopping rule."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from test_gpu_parity import assert_parity, compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1808_07554_gb300 import build
    build.build()
    import paper_1808_07554_gb300 as pkg
    pkg.load_library()


def _pkg():
    import paper_1808_07554_gb300 as pkg
    return pkg


def _pair(prob, nsteps, storage=0):
    """Oracle and GPU, both warm-starting, the oracle's free-running counts replayed."""
    pkg = _pkg()
    orc = O.Oracle(prob, tol=1e-8, check_every=8, warm_start=1)
    gpu = pkg.Solver.from_problem(prob, tol=1e-8, check_every=8, init_replay=orc.init_sub_iters,
                                  warm_start=1, storage=storage)
    log = []
    for n in range(1, nsteps + 1):
        t = n * prob.dt
        if prob.sources_at is not None:
            Fp, Fs = prob.sources_at(t)
            orc.set_sources(Fp, Fs)
            gpu.set_sources(Fp, Fs)
        if prob.walls_at is not None:
            Pb, Sb = prob.walls_at(t)
            for s in range(4):
                if prob.bc[s] == W.DIRICHLET:
                    orc.set_dirichlet(s, Pb[s], Sb[s])
                    gpu.set_dirichlet(s, Pb[s], Sb[s])
        st, k, r = orc.step(1)
        assert st == O.OK
        log.append(int(k[0]))
        gst, stats = gpu.step(1, replay=[log[-1]])
        assert stats[0].sub_iters == log[-1]
    return orc, gpu, log


@pytest.mark.parametrize("name", ["five_spot_96", "example2_40"])
def test_warm_start_matches_oracle(name):
    prob = {"five_spot_96": lambda: W.quarter_five_spot(96, seed=14, corr_len=8.0),
            "example2_40": lambda: W.example2(40)}[name]()
    orc, gpu, log = _pair(prob, 10)
    err = compare(orc, gpu, gauge_free=W.DIRICHLET not in prob.bc)
    orc.close()
    gpu.close()
    assert_parity(err)


def test_warm_start_with_fp16_storage_matches_oracle():
    pkg = _pkg()
    prob = W.quarter_five_spot(96, seed=15, corr_len=8.0)
    orc, gpu, log = _pair(prob, 8, storage=pkg.STORE_FP16_DEV)
    err = compare(orc, gpu, gauge_free=True)
    orc.close()
    gpu.close()
    assert all(v <= 2e-3 for v in err.values()), err


def test_warm_start_cuts_free_running_sweeps():
    pkg = _pkg()
    prob = W.quarter_five_spot(128, seed=16, corr_len=12.0)
    plain = pkg.Solver.from_problem(prob, tol=1e-8)
    warm = pkg.Solver.from_problem(prob, tol=1e-8, warm_start=1)
    kp, kw = [], []
    for _ in range(8):
        st, s = plain.step(1)
        assert st == pkg.OK
        kp.append(s[0].sub_iters)
        st, s = warm.step(1)
        assert st == pkg.OK
        kw.append(s[0].sub_iters)
    assert kp[0] == kw[0]                        # no history at the first step
    assert sum(kw[3:]) < 0.3 * sum(kp[3:]), (kp, kw)
    # both meet the same stopping rule: the saturation fields agree closely
    assert W.rel_l2(warm.fields()[1], plain.fields()[1]) < 1e-5


def test_caller_warm_start_from_the_converged_pressure():
    """Starting a step from the pressure another run converged to for that very step needs
    only the first residual check."""
    pkg = _pkg()
    prob = W.quarter_five_spot(96, seed=17, corr_len=8.0)
    a = pkg.Solver.from_problem(prob, tol=1e-8)
    b = pkg.Solver.from_problem(prob, tol=1e-8)
    for _ in range(3):
        a.step(1)
        b.step(1)
    ka = a.step(1)[1][0].sub_iters
    Pa, Sa = a.fields()
    b.warm_start(Pa)
    st, s = b.step(1)
    assert st == pkg.OK
    assert s[0].sub_iters < 0.5 * ka, (ka, s[0].sub_iters)
    assert W.rel_l2(b.fields()[1], Sa) < 1e-5


def test_batch_with_warm_start_members_is_bit_identical():
    pkg = _pkg()
    probs = [W.quarter_five_spot(48, seed=18), W.quarter_five_spot(40, 24, seed=19),
             W.quarter_five_spot(32, seed=20)]
    ws = [1, 0, 1]
    alone = [pkg.Solver.from_problem(p, init_replay=100, warm_start=w) for p, w in zip(probs, ws)]
    inb = [pkg.Solver.from_problem(p, init_replay=100, warm_start=w) for p, w in zip(probs, ws)]
    counts = np.array([[16, 24, 8], [8, 8, 16], [40, 16, 24], [8, 32, 8]])
    with pkg.Batch(inb) as batch:
        for row in counts:
            for s, c in zip(alone, row):
                s.step(1, replay=[int(c)])
            batch.step(1, replay=row)
            for a, b in zip(alone, inb):
                assert np.array_equal(a.get_state(), b.get_state())
