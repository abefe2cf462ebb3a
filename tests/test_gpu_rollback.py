"""A step whose pressure residual is not a number (LBM2P_ENONFINITE) is rolled back: the
state after the failed step equals the state before it, bit for bit, on every path that runs
a step (the graph-resident loop with single or fused sweeps, the warm start, replayed counts
on the host, FP16 storage), and the solver steps on from that state exactly as a twin that
never saw the failure.  The failure is made on the host: a NaN in the dense pressure source
of one step (Eq. 3-1's F_p), nothing that faults the GPU."""
import numpy as np
import pytest

import workloads as W

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


MODES = {
    "graph_single": dict(fuse_sweeps=1),
    "graph_fused_direct": dict(fuse_sweeps=2, sweep_kernel=2),
    "graph_fused_rows": dict(fuse_sweeps=2, sweep_kernel=3),
    "graph_warm_start": dict(warm_start=1),
    "replayed": dict(),
    "fp16": dict(storage=1),
}


@pytest.mark.parametrize("mode", sorted(MODES))
def test_nonfinite_step_rolls_back(mode):
    import paper_1808_07554_gb300 as pkg
    prob = W.quarter_five_spot(96, 80, seed=12, corr_len=8.0)
    prob.Fp = np.zeros((80, 96))
    kw = dict(init_replay=200, **MODES[mode])
    replay = mode in ("replayed", "fp16")
    a = pkg.Solver.from_problem(prob, **kw)
    twin = pkg.Solver.from_problem(prob, **kw)
    for s in (a, twin):                      # two good steps (history for the warm start)
        for _ in range(2):
            st, _ = s.step(1, replay=[24]) if replay else s.step(1)
            assert st in (pkg.OK, pkg.ENOTCONVERGED)
    before = a.get_state()
    assert np.array_equal(before, twin.get_state())
    bad = np.zeros((80, 96))
    bad[20, 30] = np.nan
    a.set_sources(Fp=bad)
    with pytest.raises(pkg.LBM2PError) as ei:
        if replay:
            a.step(1, replay=[16])
        else:
            a.step(1)
    assert ei.value.status == pkg.ENONFINITE
    assert np.array_equal(a.get_state(), before), "the failed step changed the state"
    # the solver goes on from the restored state: the same sweeps give the same state
    a.set_sources(Fp=np.zeros((80, 96)))
    for s in (a, twin):
        st, _ = s.step(1, replay=[32])
        assert st == pkg.OK
    assert np.array_equal(a.get_state(), twin.get_state())
    a.close()
    twin.close()
