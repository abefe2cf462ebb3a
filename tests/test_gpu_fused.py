"""Pressure sweeps fused in time (several sweeps per kernel launch) against one sweep per
launch, and the single-sweep kernels against each other: identical populations bit for bit,
on every wall kind and on ragged and tiny lattices, and the same residual up to the grouping
of its partial sums."""
import numpy as np
import pytest

import workloads as W
from _problems import uniform

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


def _problem(kind):
    rng = np.random.default_rng(hash(kind) % 2 ** 32)
    if kind == "five_spot_ragged":
        return W.quarter_five_spot(300, 200, seed=5, corr_len=8.0)
    if kind == "wide_ragged":
        return W.quarter_five_spot(2049, 17, seed=6, corr_len=4.0)
    if kind == "periodic":
        return W.manufactured_periodic(96)
    # "wide_dirichlet": wide enough that the two-sweep row-walking kernels have blocks with
    # no wall and no well (their interior path), here with a dense pressure source
    nx, ny, bc = {"dirichlet": (97, 70, (2, 2, 2, 2)), "mixed": (65, 129, (0, 0, 2, 2)),
                  "wide_dirichlet": (523, 161, (2, 2, 1, 1)),
                  "tiny": (5, 3, (1, 1, 0, 0)), "column": (1, 7, (0, 0, 0, 0)),
                  "tall": (31, 300, (2, 2, 1, 1))}[kind]
    Pb = [rng.random(2 * (ny if s < 2 else nx) + 1) for s in range(4)]
    return uniform(nx, ny, bc=bc, K=np.exp(rng.standard_normal((ny, nx))),
                   S0=0.2 + 0.5 * rng.random((ny, nx)), Fp=rng.standard_normal((ny, nx)),
                   wells=[(0, 0, 1e-3, 0), (nx - 1, ny - 1, 1e-3, 1)] if nx * ny > 1 else [],
                   P_b=Pb, S_b=[0.3 + 0.0 * t for t in Pb])


@pytest.mark.parametrize("kind", ["five_spot_ragged", "wide_ragged", "periodic", "dirichlet",
                                  "mixed", "tiny", "column", "tall", "wide_dirichlet"])
@pytest.mark.parametrize("T", [2, 4, "2rows", "2direct"])
def test_fused_equals_single_sweeps(kind, T):
    """T = 2 or 4 sweeps on shared-memory stages; "2rows": two sweeps on rows staged by
    bulk copies; "2direct": two sweeps with direct loads (both for lattices with walls on every
    side only)."""
    import paper_1808_07554_gb300 as pkg
    prob = _problem(kind)
    single = pkg.Solver.from_problem(prob, init_replay=0, fuse_sweeps=1)
    if T in ("2rows", "2direct"):
        if W.PERIODIC in prob.bc:
            pytest.skip("the two-sweep row-walking kernels need walls on every side")
        pin = pkg.SWEEP_ROWS if T == "2rows" else pkg.SWEEP_SCALAR
        T = 2
        fused = pkg.Solver.from_problem(prob, init_replay=0, fuse_sweeps=2, sweep_kernel=pin)
        cfg = fused.sweep_config()
        assert cfg[0] == 2 and cfg[2] in (120, 240) and 1 <= cfg[3] <= 128
    else:
        fused = pkg.Solver.from_problem(prob, init_replay=0, fuse_sweeps=T)
        cfg = fused.sweep_config()
        assert cfg[0] == T and cfg[2] in (32, 64, 128, 120, 240) and 1 <= cfg[3] <= 128
    assert single.sweep_config()[0] == 1 and single.sweep_config()[1] in (1, 2, 3)
    rng = np.random.default_rng(3)
    state = single.get_state()
    state[:8] = 0.01 * rng.standard_normal(state[:8].shape)
    state[17] = 1.0 / (0.55 + 2.0 * rng.random(state[17].shape))
    state[19] = rng.standard_normal(state[19].shape)
    single.set_state(state)
    fused.set_state(state)
    for n in (3 * T + 1, T, 2 * T):
        r1 = single.pressure_sweeps(n)
        r2 = fused.pressure_sweeps(n)
        a, b = single.get_state(), fused.get_state()
        assert np.array_equal(a, b), (kind, T, n, float(np.max(np.abs(a - b))))
        # the residual is a sum of per-warp FP32 partials; fused launches group nodes into
        # warps differently, so near-cancelling sums may differ in the trailing digits
        assert r2 == pytest.approx(r1, rel=1e-3, abs=1e-30)
    # and through whole steps (graph-resident loop with fused bodies)
    s1 = single.step(2, replay=[4 * T, 2 * T])
    s2 = fused.step(2, replay=[4 * T, 2 * T])
    assert np.array_equal(single.get_state(), fused.get_state())
    single.close()
    fused.close()


ROWS2_SHAPES = [(4, 6), (4, 8), (8, 4), (8, 6), (4, 6 + 16)]


@pytest.mark.parametrize("kind", ["five_spot_ragged", "wide_dirichlet", "dirichlet", "tall"])
def test_every_pinned_two_sweep_shape_equals_single_sweeps(kind):
    """Each shape of the two two-sweep row-walking kernels (consumer warps x ring slots x rows
    per block for the staged-rows kernel, including the seven-blocks-per-SM register cap;
    warps x rows for the direct-load kernel), pinned with lbm2p_set_fused_shape, against one
    sweep per launch, bit for bit, in bare sweeps and through a graph-resident step."""
    import paper_1808_07554_gb300 as pkg
    prob = _problem(kind)
    single = pkg.Solver.from_problem(prob, init_replay=0, fuse_sweeps=1)
    fused = pkg.Solver.from_problem(prob, init_replay=0, fuse_sweeps=2, sweep_kernel=pkg.SWEEP_ROWS)
    rng = np.random.default_rng(11)
    state = single.get_state()
    state[:8] = 0.01 * rng.standard_normal(state[:8].shape)
    state[17] = 1.0 / (0.55 + 2.0 * rng.random(state[17].shape))
    state[19] = rng.standard_normal(state[19].shape)
    shapes = [(pkg.FUSED_STAGED_ROWS, w, s, H) for (w, s) in ROWS2_SHAPES for H in (16, 128)]
    shapes += [(pkg.FUSED_DIRECT, w, 0, H) for w in (4, 8) for H in (2, 32)]
    for form, w, sl, H in shapes:
        H = min(H, prob.ny)
        fused.set_fused_shape(form, w, sl, H)
        assert fused.fused_form() == form and fused.sweep_config()[2:] == (30 * w, H)
        single.set_state(state)
        fused.set_state(state)
        for n in (5, 2):
            single.pressure_sweeps(n)
            fused.pressure_sweeps(n)
            a, b = single.get_state(), fused.get_state()
            assert np.array_equal(a, b), (kind, form, w, sl, H, n, float(np.max(np.abs(a - b))))
        single.step(1, replay=[16])
        fused.step(1, replay=[16])
        assert np.array_equal(single.get_state(), fused.get_state()), (kind, form, w, sl, H)
    for bad in ((pkg.FUSED_STAGED_ROWS, 4, 7, 16), (pkg.FUSED_STAGED_ROWS, 4, 6, 24),
                (pkg.FUSED_DIRECT, 4, 6, 8), (pkg.FUSED_STAGES, 4, 6, 16)):
        with pytest.raises(pkg.LBM2PError) as e:
            fused.set_fused_shape(*bad)
        assert e.value.status == pkg.EINVAL
    single.close()
    fused.close()


@pytest.mark.parametrize("kind", ["five_spot_ragged", "wide_ragged", "periodic", "dirichlet",
                                  "mixed", "tiny", "column", "tall"])
def test_single_sweep_kernels_agree(kind):
    """VEC4, SCALAR and ROWS (strips staged in shared memory) give the same populations."""
    import paper_1808_07554_gb300 as pkg
    prob = _problem(kind)
    solvers = [pkg.Solver.from_problem(prob, init_replay=0, fuse_sweeps=1, sweep_kernel=k)
               for k in (pkg.SWEEP_VEC4, pkg.SWEEP_SCALAR, pkg.SWEEP_ROWS)]
    for k, s in zip((pkg.SWEEP_VEC4, pkg.SWEEP_SCALAR, pkg.SWEEP_ROWS), solvers):
        cfg = s.sweep_config()
        assert cfg[0] == 1 and cfg[1] == k
        if k == pkg.SWEEP_ROWS:
            assert cfg[2] in (128, 256, 512) and 1 <= cfg[3] <= prob.ny
    rng = np.random.default_rng(5)
    state = solvers[0].get_state()
    state[:8] = 0.01 * rng.standard_normal(state[:8].shape)
    state[17] = 1.0 / (0.55 + 2.0 * rng.random(state[17].shape))
    state[19] = rng.standard_normal(state[19].shape)
    for s in solvers:
        s.set_state(state)
    for n in (1, 2, 7, 8):
        rs = [s.pressure_sweeps(n) for s in solvers]
        ref = solvers[0].get_state()
        for s, r in zip(solvers[1:], rs[1:]):
            b = s.get_state()
            assert np.array_equal(ref, b), (kind, n, float(np.max(np.abs(ref - b))))
            if n >= 2:
                assert r == pytest.approx(rs[0], rel=1e-3, abs=1e-30)
    steps = [s.step(2, replay=[16, 8]) for s in solvers]
    ref = solvers[0].get_state()
    for s in solvers[1:]:
        assert np.array_equal(ref, s.get_state())
    for s in solvers:
        s.close()


def test_rows_kernel_free_running_graph_loop():
    """The staged-rows kernel inside the graph-resident loop: a free-running step agrees with
    the scalar kernel's (the same populations when the sweep counts agree; the counts may
    differ by one loop body when a residual sits on the tolerance)."""
    import paper_1808_07554_gb300 as pkg
    prob = W.quarter_five_spot(300, 140, seed=9, corr_len=8.0)
    a = pkg.Solver.from_problem(prob, init_replay=400, sweep_kernel=pkg.SWEEP_SCALAR,
                                fuse_sweeps=1)
    b = pkg.Solver.from_problem(prob, init_replay=400, sweep_kernel=pkg.SWEEP_ROWS,
                                fuse_sweeps=1)
    assert np.array_equal(a.get_state(), b.get_state())
    for _ in range(3):
        sa, ta = a.step(1)
        sb, tb = b.step(1)
        assert sa == pkg.OK and sb == pkg.OK
        ka, kb = ta[0].sub_iters, tb[0].sub_iters
        assert abs(ka - kb) <= 8
        if ka == kb:
            assert np.array_equal(a.get_state(), b.get_state())
        else:
            b.set_state(a.get_state())
