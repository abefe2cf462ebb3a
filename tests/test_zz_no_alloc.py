"""The pressure sweep for callers that cannot allocate device memory.

Host programs that give all device memory to their own pool, or that forbid allocation
once running, cannot create a solver handle; ``lbm2p_pressure_sweep_noalloc`` runs the
same fused pressure sweep and residual on planes they own, with the residual scratch in a
static device array.  Here it is called twice in a row (the second call chains on the
first call's pressure increment) and compared with the handle-based entry point,
``lbm2p_pressure_sweeps(h, 2)``, from the same state.  The file runs last so that a
failure here stops a first-failure run only after every other test.
"""
import numpy as np
import pytest

import workloads as W
from _problems import uniform

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1808_07554_gb300 import build
    build.build()
    import paper_1808_07554_gb300 as pkg
    pkg.load_library()
    return torch, pkg


def _problem():
    nx, ny = 1100, 96                       # two row tiles per row, ragged second tile
    rng = np.random.default_rng(31)
    K = np.exp(W.grf_lnK(nx, ny, 1.0, 8.0, seed=7))
    Pb = [0.2 * rng.random(2 * ny + 1), -0.1 * rng.random(2 * ny + 1), None, None]
    Sb = [np.full(2 * ny + 1, 0.6), np.full(2 * ny + 1, 0.2), None, None]
    return uniform(nx, ny, bc=(2, 2, 1, 1), K=K, S0=0.2 + 0.5 * rng.random((ny, nx)),
                   Fp=rng.standard_normal((ny, nx)), tau_mode=W.TAU_PHYSICAL_DT,
                   dt=0.3 / nx ** 2, P_b=Pb, S_b=Sb)


def test_noalloc_sweep_matches_handle_entry_point(env):
    torch, pkg = env
    prob = _problem()
    nx, ny = prob.nx, prob.ny
    solver = pkg.Solver.from_problem(prob, init_replay=40)
    solver.step(1, replay=[25])              # nonzero deviations and reference pressure
    state = solver.get_state()
    pitch = (nx + 31) // 32 * 32

    def plane(a):
        t = torch.zeros((ny, pitch), dtype=torch.float32, device="cuda")
        t[:, :nx] = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
        return t

    scale = (prob.dt / (prob.dx * prob.dx)) * prob.dx * prob.dx      # s dx^2 with s = dt/dx^2
    Fp = plane((scale * prob.Fp).astype(np.float32))
    n_a = [plane(state[i]) for i in range(8)]
    n_b = [torch.zeros_like(n_a[0]) for _ in range(8)]
    R = plane(state[19])
    inv_tau = plane(state[17])
    dP = torch.zeros_like(R)
    traces = [torch.from_numpy(t.astype(np.float32)).cuda() if t is not None else None
              for t in prob.P_b]
    tptr = [t.data_ptr() if t is not None else 0 for t in traces]
    stream = torch.cuda.current_stream().cuda_stream

    r_ref = solver.pressure_sweeps(2)
    ref = solver.get_state()[:8]
    solver.close()

    def call(src, dst):
        return pkg.lbm2p_pressure_sweep_noalloc(
            nx, ny, pitch, prob.bc, [t.data_ptr() for t in src], [t.data_ptr() for t in dst],
            R.data_ptr(), inv_tau.data_ptr(), Fp.data_ptr(), tptr, dP.data_ptr(), stream)

    call(n_a, n_b)
    r2 = call(n_b, n_a)
    torch.cuda.synchronize()
    got = np.stack([t[:, :nx].cpu().numpy() for t in n_a])
    scale_n = np.max(np.abs(ref))
    assert np.max(np.abs(got - ref)) <= 2e-6 * scale_n
    assert r2 == pytest.approx(r_ref, rel=1e-5)
    # the reference pressure was only read
    assert np.array_equal(R[:, :nx].cpu().numpy(), state[19])


def test_noalloc_rejects_lattices_beyond_its_scratch(env):
    """A lattice one row tile beyond the scratch is refused before any launch: every plane
    pointer is NULL, so no ordering of the argument checks can let a kernel start."""
    torch, pkg = env
    nx = pkg.NOALLOC_TILE_NODES + 1                 # two row tiles per row
    ny = pkg.NOALLOC_MAX_TILES // 2 + 1             # just beyond what the scratch holds
    assert 2 * ny == pkg.NOALLOC_MAX_TILES + 2
    pitch = (nx + 31) // 32 * 32
    torch.cuda.synchronize()
    with pytest.raises(pkg.LBM2PError) as ei:
        pkg.lbm2p_pressure_sweep_noalloc(nx, ny, pitch, (1, 1, 1, 1), [0] * 8, [0] * 8, 0, 0,
                                         0, None, 0)
    assert ei.value.status == pkg.EINVAL
    assert "row tiles" in str(ei.value)
    torch.cuda.synchronize()                        # nothing was queued, nothing failed
