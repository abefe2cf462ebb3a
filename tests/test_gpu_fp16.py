"""FP16 storage of the pressure populations inside each sub-iteration (storage FP16_DEV)
against the FP64 oracle: the oracle decides the sweep counts, the GPU replays them, every
field within relative L2 2e-3 (the FP16 bar); on the five-spot (wells, no-flux walls),
Example 2 (Dirichlet walls, moving sources) and the periodic manufactured problem."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from test_gpu_parity import compare, run_pair

pytestmark = pytest.mark.gpu

TOL16 = 2e-3


@pytest.fixture(scope="module", autouse=True)
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1808_07554_gb300 import build
    build.build()
    import paper_1808_07554_gb300 as pkg
    pkg.load_library()


def _run_pair16(prob, nsteps, kernel=0):
    """run_pair with the GPU solver in FP16 storage: the oracle's counts replayed."""
    import paper_1808_07554_gb300 as pkg
    orc = O.Oracle(prob, tol=1e-8, check_every=8)
    gpu = pkg.Solver.from_problem(prob, tol=1e-8, check_every=8, init_replay=orc.init_sub_iters,
                                  storage=pkg.STORE_FP16_DEV, sweep_kernel=kernel)
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
        gst, stats = gpu.step(1, replay=[int(k[0])])
        assert stats[0].sub_iters == int(k[0])
    return orc, gpu


@pytest.mark.parametrize("kernel", [2, 3], ids=["scalar", "rows"])
@pytest.mark.parametrize("name", ["five_spot_96", "example2_48", "manufactured_32"])
def test_fp16_storage_matches_oracle(name, kernel):
    prob = {"five_spot_96": lambda: W.quarter_five_spot(96, seed=8, corr_len=8.0),
            "example2_48": lambda: W.example2(48),
            "manufactured_32": lambda: W.manufactured_periodic(32, p_amp=0.2)}[name]()
    orc, gpu = _run_pair16(prob, 8, kernel)
    err = compare(orc, gpu, gauge_free=W.DIRICHLET not in prob.bc)
    orc.close()
    gpu.close()
    assert all(v <= TOL16 for v in err.values()), err
    print(name, err)


@pytest.mark.parametrize("name", ["five_spot_300x140", "example2_40", "tiny_5x3"])
def test_fp16_kernels_agree_bit_for_bit(name):
    """The FP16 one-node-per-thread and staged-rows sweeps compute the same stored values."""
    import paper_1808_07554_gb300 as pkg
    from _problems import uniform
    rng = np.random.default_rng(12)
    prob = {"five_spot_300x140": lambda: W.quarter_five_spot(300, 140, seed=12, corr_len=6.0),
            "example2_40": lambda: W.example2(40),
            "tiny_5x3": lambda: uniform(5, 3, bc=(1, 1, 0, 0), Fp=rng.standard_normal((3, 5)),
                                        K=np.exp(rng.standard_normal((3, 5))))}[name]()
    a = pkg.Solver.from_problem(prob, init_replay=40, storage=pkg.STORE_FP16_DEV,
                                sweep_kernel=pkg.SWEEP_SCALAR)
    b = pkg.Solver.from_problem(prob, init_replay=40, storage=pkg.STORE_FP16_DEV,
                                sweep_kernel=pkg.SWEEP_ROWS)
    assert any(r[0] == "fp16_rows" for r in b.autotune_report())
    assert np.array_equal(a.get_state(), b.get_state())
    for n in (1, 7, 300):
        ra = a.pressure_sweeps(n)
        rb = b.pressure_sweeps(n)
        assert np.array_equal(a.get_state(), b.get_state()), (name, n)
        if n >= 2:
            assert rb == pytest.approx(ra, rel=1e-3, abs=1e-30)


def test_fp16_and_fp32_on_a_256_crop_of_the_4096_field():
    """The precision study at matching resolution: the 4096^2 five-spot's ln K field (same
    seed rule), cropped to its first 256 x 256 nodes, run with FP32 and with FP16 storage on
    the oracle's sweep counts; every field against the FP64 oracle, FP32 to 1e-5 and FP16 to
    2e-3."""
    import paper_1808_07554_gb300 as pkg
    big = W.quarter_five_spot(4096, seed=2)
    prob = W.quarter_five_spot(256, seed=2)
    prob.K = np.ascontiguousarray(big.K[:256, :256])
    del big
    # a fixed number of sweeps for the t = 0 solve and for each step (a converged start would
    # take ~2e5 oracle sweeps); both sides run the same counts
    log = [4000] + [400] * 6
    orc = O.Oracle(prob, tol=1e-8, check_every=8, init_replay=log[0])
    for c in log[1:]:
        orc.step(1, replay=[c])
    errs = {}
    for name, storage in (("fp32", pkg.STORE_FP32), ("fp16", pkg.STORE_FP16_DEV)):
        gpu = pkg.Solver.from_problem(prob, tol=1e-8, check_every=8, init_replay=log[0],
                                      storage=storage)
        for c in log[1:]:
            gst, stats = gpu.step(1, replay=[c])
            assert stats[0].sub_iters == c
        errs[name] = compare(orc, gpu, gauge_free=True)
        gpu.close()
    orc.close()
    print("256 crop of the 4096 field", errs)
    assert all(v <= 1e-5 for v in errs["fp32"].values()), errs
    assert all(v <= TOL16 for v in errs["fp16"].values()), errs


def test_fp16_and_fp32_storage_agree_on_the_same_counts():
    import paper_1808_07554_gb300 as pkg
    prob = W.quarter_five_spot(128, seed=9, corr_len=12.0)
    a = pkg.Solver.from_problem(prob, init_replay=3000)
    b = pkg.Solver.from_problem(prob, init_replay=3000, storage=pkg.STORE_FP16_DEV)
    counts = [512, 256, 256, 256]
    a.step(len(counts), replay=counts)
    b.step(len(counts), replay=counts)
    Pa, Sa = a.fields(mean_free_P=True)
    Pb, Sb = b.fields(mean_free_P=True)
    assert W.rel_l2(Pb, Pa) <= TOL16 and W.rel_l2(Sb, Sa) <= TOL16


def test_fp16_free_running_meets_a_loose_tolerance():
    """Free-running with FP16 storage stops on the same stopping rule; FP16 rounding floors r
    well above the FP32 1e-8, so a looser tolerance is used."""
    import paper_1808_07554_gb300 as pkg
    prob = W.quarter_five_spot(64, seed=10, corr_len=8.0)
    s = pkg.Solver.from_problem(prob, tol=1e-5, check_every=8, max_sub_iters=400_000,
                                storage=pkg.STORE_FP16_DEV)
    st, stats = s.step(3)
    assert st == pkg.OK
    assert all(x.residual <= 1e-5 for x in stats)


def test_fp16_member_is_refused_by_a_batch():
    import paper_1808_07554_gb300 as pkg
    prob = W.quarter_five_spot(32, seed=11)
    a = pkg.Solver.from_problem(prob, init_replay=16)
    b = pkg.Solver.from_problem(prob, init_replay=16, storage=pkg.STORE_FP16_DEV)
    with pytest.raises(pkg.LBM2PError) as e:
        pkg.Batch([a, b])
    assert e.value.status == pkg.EINVAL
