"""Batched realisations (lbm2p_batch_*) against the same handles stepped one at a time.

Each member of a batch runs the per-node arithmetic of the single-lattice kernels, so with
the same sweep counts its whole state (populations, saturation, 1/tau_f, S, R) must be
bit-identical to the state of an identical handle stepped alone.  The members differ in
size (lattices narrower than a block, ragged row segments, ragged row groups), boundary
kind, sources, wells and mobility law, so that every tile shape of the batch tile list is
exercised.  One test also replays the FP64 oracle's counts through the batch and compares
the fields with the oracle.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from _problems import uniform

pytestmark = pytest.mark.gpu

CHECK = 8


@pytest.fixture(scope="module", autouse=True)
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1808_07554_gb300 import build
    build.build()
    import paper_1808_07554_gb300 as pkg
    pkg.load_library()
    return pkg


def _pkg():
    import paper_1808_07554_gb300 as pkg
    return pkg


def _members():
    """Problems of different shapes; names say which tile shape each one exercises."""
    rng = np.random.default_rng(7)
    narrow = uniform(20, 70, bc=(W.NOFLUX,) * 4, K=np.exp(0.5 * rng.standard_normal((70, 20))),
                     S0=0.3, wells=[(0, 0, 2e-3, 0), (19, 69, 2e-3, 1)], tau_mode=W.TAU_PHYSICAL_DT)
    dense = uniform(48, 48, mobility=W.MOB_RATIONAL, Fp=0.1 * rng.standard_normal((48, 48)),
                    Fs=0.01 * rng.standard_normal((48, 48)), S0=0.4)
    dense.Fp -= dense.Fp.mean()
    return {
        "five_spot_96": W.quarter_five_spot(96, seed=11, sigma=1.0, corr_len=8),
        "five_spot_300x40": W.quarter_five_spot(300, 40, seed=12, sigma=0.7, corr_len=6),
        "narrow_20x70": narrow,
        "periodic_sources_48": dense,
        "example2_40": W.example2(n=40),
    }


def _solver(prob, **kw):
    return _pkg().Solver.from_problem(prob, check_every=CHECK, **kw)


def _drive(prob, solvers, n):
    """Time-dependent sources and wall values of step n, applied to every solver."""
    t = n * prob.dt
    if prob.sources_at is not None:
        Fp, Fs = prob.sources_at(t)
        for s in solvers:
            s.set_sources(Fp, Fs)
    if prob.walls_at is not None:
        Pb, Sb = prob.walls_at(t)
        for side in range(4):
            if prob.bc[side] == W.DIRICHLET:
                for s in solvers:
                    s.set_dirichlet(side, Pb[side], Sb[side])


def test_replay_bit_identical_to_single_handles():
    pkg = _pkg()
    probs = list(_members().values())
    alone = [_solver(p, init_replay=120) for p in probs]
    inb = [_solver(p, init_replay=120) for p in probs]
    for a, b in zip(alone, inb):
        assert np.array_equal(a.get_state(), b.get_state())
    counts = np.array([[16, 24, 8, 40, 0],
                       [0, 8, 32, 16, 24],
                       [48, 16, 16, 8, 8],
                       [8, 0, 24, 24, 56]])
    with pkg.Batch(inb) as batch:
        for n, row in enumerate(counts, start=1):
            for p, a, b in zip(probs, alone, inb):
                _drive(p, [a, b], n)
            for a, c in zip(alone, row):
                a.step(1, replay=[int(c)])
            st, stats = batch.step(1, replay=row)
            assert st == pkg.OK
            assert [s.sub_iters for s in stats[0]] == list(row)
            for m, (a, b) in enumerate(zip(alone, inb)):
                sa, sb = a.get_state(), b.get_state()
                assert np.array_equal(sa, sb), f"member {m} differs after step {n}: " \
                    f"max |d| = {np.abs(sa - sb).max()}"
        launches, tiles = batch.counters()
        assert launches >= 4 * len(counts)
        assert tiles > 0


def test_multistep_replay_and_counters():
    """nsteps > 1 in one call, step-major counts; equals two single-step calls."""
    pkg = _pkg()
    probs = list(_members().values())[:3]
    x = [_solver(p, init_replay=64) for p in probs]
    y = [_solver(p, init_replay=64) for p in probs]
    counts = np.array([[8, 16, 24], [24, 8, 16], [16, 16, 0]])
    with pkg.Batch(x) as bx, pkg.Batch(y) as by:
        bx.step(3, replay=counts)
        for row in counts:
            by.step(1, replay=row)
        for a, b in zip(x, y):
            assert np.array_equal(a.get_state(), b.get_state())
        for a in x:
            assert a.counters()[1] >= 0


def test_free_running_matches_single_handles():
    """Each member stops on its own residual or cap; counts agree with the handle alone (up to
    one body when a residual sits on the tolerance: the sums are grouped differently), the
    statuses agree, and equal counts give identical states."""
    pkg = _pkg()
    m = _members()
    probs = [W.quarter_five_spot(48, seed=11, sigma=1.0, corr_len=8),
             W.quarter_five_spot(40, 24, seed=13, sigma=0.8, corr_len=6), m["narrow_20x70"],
             m["example2_40"]]
    cap = 40_000
    alone = [_solver(p, max_sub_iters=cap) for p in probs]
    inb = [_solver(p, max_sub_iters=cap) for p in probs]
    with pkg.Batch(inb) as batch:
        for n in range(1, 4):
            for p, a, b in zip(probs, alone, inb):
                _drive(p, [a, b], n)
            ka, ra, sa = [], [], []
            for a in alone:
                st, s = a.step(1)
                ka.append(s[0].sub_iters)
                ra.append(s[0].residual)
                sa.append(s[0].status)
            st, stats = batch.step(1)
            kb = [s.sub_iters for s in stats[0]]
            assert sa[0] == pkg.OK, sa
            for i in range(len(probs)):
                assert abs(kb[i] - ka[i]) <= CHECK, (i, ka, kb)
                if kb[i] == ka[i]:
                    assert stats[0][i].status == sa[i]
                    assert stats[0][i].residual == pytest.approx(ra[i], rel=1e-3)
                    assert np.array_equal(alone[i].get_state(), inb[i].get_state())
                else:      # counts differ by one body: carry on from identical states
                    inb[i].set_state(alone[i].get_state())


def test_free_running_with_a_two_sweep_member():
    """A 512^2 member (swept two sweeps per launch by the batch's direct-load kernel over its
    blocks) beside a small one, free-running: each stops on its own residual, with the counts,
    statuses and residuals of its handle stepped alone (up to one body: the residual's partial
    sums are grouped by the batch's blocks), and equal counts give identical states."""
    pkg = _pkg()
    probs = [W.quarter_five_spot(512, seed=21, sigma=1.0, corr_len=16.0),
             W.quarter_five_spot(48, seed=22, sigma=1.0, corr_len=8)]
    cap = 40_000
    alone = [_solver(p, max_sub_iters=cap, init_replay=400) for p in probs]
    inb = [_solver(p, max_sub_iters=cap, init_replay=400) for p in probs]
    with pkg.Batch(inb) as batch:
        for _ in range(3):
            ka, ra, sa = [], [], []
            for a in alone:
                st, s = a.step(1)                   # a cap reached is a status, not an error
                ka.append(s[0].sub_iters)
                ra.append(s[0].residual)
                sa.append(s[0].status)
            st, stats = batch.step(1)
            for i in range(len(probs)):
                kb = stats[0][i].sub_iters
                assert abs(kb - ka[i]) <= CHECK, (i, ka, kb)
                assert stats[0][i].residual <= 1e-8 or kb == cap
                if kb == ka[i]:
                    assert stats[0][i].status == sa[i]
                    assert stats[0][i].residual == pytest.approx(ra[i], rel=1e-3)
                    assert np.array_equal(alone[i].get_state(), inb[i].get_state())
                else:      # counts differ by one body: carry on from identical states
                    inb[i].set_state(alone[i].get_state())


def test_batch_against_oracle():
    """The oracle decides the counts (free-running, FP64); the batch replays them."""
    pkg = _pkg()
    probs = [W.quarter_five_spot(64, seed=3, sigma=1.0, corr_len=8), W.example2(n=32)]
    orcs = [O.Oracle(p, tol=1e-8, check_every=CHECK) for p in probs]
    sols = [_solver(p, init_replay=o.init_sub_iters) for p, o in zip(probs, orcs)]
    with pkg.Batch(sols) as batch:
        for n in range(1, 6):
            row = []
            for p, o, s in zip(probs, orcs, sols):
                tt = n * p.dt
                if p.sources_at is not None:
                    Fp, Fs = p.sources_at(tt)
                    o.set_sources(Fp, Fs)
                    s.set_sources(Fp, Fs)
                if p.walls_at is not None:
                    Pb, Sb = p.walls_at(tt)
                    for side in range(4):
                        if p.bc[side] == W.DIRICHLET:
                            o.set_dirichlet(side, Pb[side], Sb[side])
                            s.set_dirichlet(side, Pb[side], Sb[side])
                st, k, r = o.step(1)
                assert st == O.OK
                assert k[0] % CHECK == 0
                row.append(int(k[0]))
            batch.step(1, replay=row)
    for p, o, s in zip(probs, orcs, sols):
        ref = o.fields()
        gauge_free = W.DIRICHLET not in p.bc
        P, S = s.fields(mean_free_P=gauge_free)
        Pref = W.mean_free(ref["P"]) if gauge_free else ref["P"]
        ux, uy = s.velocity()
        err = {"P": W.rel_l2(P, Pref), "S": W.rel_l2(S, ref["S"]),
               "ux": W.rel_l2(ux, ref["ux"]), "uy": W.rel_l2(uy, ref["uy"])}
        assert all(v <= 1e-5 for v in err.values()), err


def test_large_members_bit_identical():
    """Members of the sizes the batched workload draws from, up to 1024^2 (128^2, 256^2,
    512^2, 1024^2 and a ragged 1000 x 600), one replayed step: every member's state equals
    that of the same handle stepped alone."""
    pkg = _pkg()
    probs = [W.quarter_five_spot(n, seed=30 + n) for n in (128, 256, 512, 1024)]
    probs.append(W.quarter_five_spot(1000, 600, seed=31, corr_len=12.0))
    alone = [_solver(p, init_replay=50) for p in probs]
    inb = [_solver(p, init_replay=50) for p in probs]
    counts = [24, 40, 8, 64, 16]
    with pkg.Batch(inb) as batch:
        for s, c in zip(alone, counts):
            s.step(1, replay=[c])
        batch.step(1, replay=counts)
        for a, b in zip(alone, inb):
            assert np.array_equal(a.get_state(), b.get_state())
    for s in alone + inb:
        s.close()


def test_rejects_bad_members_and_counts():
    pkg = _pkg()
    p = W.quarter_five_spot(32, seed=4)
    a = _solver(p, init_replay=16)
    b = _solver(p, init_replay=16)
    odd = pkg.Solver.from_problem(p, check_every=7, init_replay=16)
    other = pkg.Solver.from_problem(p, check_every=10, max_sub_iters=1000, init_replay=16)
    capless = pkg.Solver.from_problem(p, check_every=CHECK, max_sub_iters=1001, init_replay=16)
    for bad in ([a, a], [a, odd], [a, other], [a, capless], []):
        with pytest.raises(pkg.LBM2PError) as e:
            pkg.Batch(bad)
        assert e.value.status == pkg.EINVAL
    with pkg.Batch([a, b]) as batch:
        before = a.get_state()
        with pytest.raises(pkg.LBM2PError) as e:
            batch.step(1, replay=[8, 12])
        assert e.value.status == pkg.EINVAL
        assert np.array_equal(a.get_state(), before)
        with pytest.raises(ValueError):
            batch.step(2, replay=[8, 8])
        a.step(1, replay=[8])               # stepped outside the batch
        with pytest.raises(pkg.LBM2PError) as e:
            batch.step(1, replay=[8, 8])
        assert e.value.status == pkg.EINVAL
    with pkg.Batch([a, b]) as batch:        # a new batch takes the current parities
        batch.step(1, replay=[8, 8])
        b.pressure_sweeps(1)                # odd sweep count flips b's f buffers
        with pytest.raises(pkg.LBM2PError) as e:
            batch.step(1, replay=[8, 8])
        assert e.value.status == pkg.EINVAL


def test_nonfinite_member_is_reported():
    pkg = _pkg()
    good = uniform(32, 32, Fp=np.zeros((32, 32)), S0=0.5)
    bad = uniform(40, 24, Fp=np.zeros((24, 40)), S0=0.5)
    g = _solver(good, init_replay=16)
    h = _solver(bad, init_replay=16)
    Fp = np.zeros((24, 40))
    Fp[5, 7] = np.nan
    h.set_sources(Fp, None)
    with pkg.Batch([g, h]) as batch:
        with pytest.raises(pkg.LBM2PError) as e:
            batch.step(1)
        assert e.value.status == pkg.ENONFINITE
    P, S = g.fields()
    assert np.isfinite(P).all() and np.isfinite(S).all()


def test_batch_against_oracle_with_a_1024_member():
    """A batch holding a 1024^2 five-spot member (the largest size of the batched workload)
    and a 128^2 one, both started from 64 t = 0 sweeps and stepped twice with 40 replayed
    sweeps: every field of both members within relative L2 1e-5 of the FP64 oracle run the
    same counts."""
    pkg = _pkg()
    probs = [W.quarter_five_spot(1024, seed=33), W.quarter_five_spot(128, seed=34)]
    orcs = [O.Oracle(p, tol=1e-8, check_every=CHECK, init_replay=64) for p in probs]
    sols = [_solver(p, init_replay=64) for p in probs]
    with pkg.Batch(sols) as batch:
        for _ in range(2):
            for o in orcs:
                st, k, r = o.step(1, replay=[40])
                assert st == O.OK
            batch.step(1, replay=[40, 40])
    for p, o, s in zip(probs, orcs, sols):
        ref = o.fields()
        P, S = s.fields(mean_free_P=True)
        ux, uy = s.velocity()
        err = {"P": W.rel_l2(P, W.mean_free(ref["P"])), "S": W.rel_l2(S, ref["S"]),
               "ux": W.rel_l2(ux, ref["ux"]), "uy": W.rel_l2(uy, ref["uy"])}
        o.close()
        assert all(v <= 1e-5 for v in err.values()), (p.nx, err)
