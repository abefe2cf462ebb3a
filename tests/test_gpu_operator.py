"""The pressure operator's tensor-core kernels (tcgen05.mma, BF16 inputs, FP32 accumulators in
tensor memory) against the plain CPU reference convolution of tests/_conv_ref.py, on the
BF16-rounded inputs the kernels read.  Tolerances: a BF16 output is within half a BF16 ulp
(2^-8 relative) of the exact value plus FP32 accumulation error; FP32 outputs and gradients
within 1e-5 (forward) or 1e-4 (gradients, summed over many pixels by FP32 atomics) of the
largest magnitude.  Shapes span several 128-pixel tiles with a ragged last tile, images larger
than one wave of CTAs (several tiles per CTA), and every (C_in, C_out) the kernels build."""
import numpy as np
import pytest

from _conv_ref import bf16_round, conv3x3, conv3x3_wgrad, flip

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
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    return torch, pkg, err


def _bf16(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16).cuda()


def _f32(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _np(t):
    return t.float().cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("shape", [(2, 13, 21, 16, 32, 1), (2, 13, 21, 32, 32, 0),
                                   (1, 29, 7, 32, 16, 1), (1, 400, 400, 32, 32, 1)])
def test_conv_forward_against_cpu(env, shape):
    torch, pkg, err = env
    n, H, W, ci, co, act = shape
    rng = np.random.default_rng(hash(shape) % 2 ** 32)
    x = rng.standard_normal((n, H, W, ci))
    w = rng.standard_normal((9, co, ci)) / np.sqrt(9 * ci)
    b = 0.1 * rng.standard_normal(co)
    xd, wd, bd = _bf16(torch, x), _bf16(torch, w), _f32(torch, b)
    y = torch.empty((n, H, W, co), dtype=torch.bfloat16, device="cuda")
    y0 = torch.empty((n, H, W), dtype=torch.float32, device="cuda")
    err.zero_()
    pkg.lbm2p_op_conv3x3(xd.data_ptr(), wd.data_ptr(), bd.data_ptr(), 0, y.data_ptr(),
                         y0.data_ptr(), n, H, W, ci, co, act, err.data_ptr(),
                         torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    ref = conv3x3(bf16_round(x), bf16_round(w), bias=b.astype(np.float32).astype(np.float64))
    if act:
        ref = np.maximum(ref, 0.0)
    got = _np(y)
    scale = np.max(np.abs(ref))
    assert np.all(np.abs(got - ref) <= 2.0 ** -8 * np.abs(ref) + 1e-5 * scale)
    assert np.max(np.abs(_np(y0) - ref[..., 0])) <= 1e-5 * scale


def test_conv_mask_is_the_relu_derivative(env):
    torch, pkg, err = env
    n, H, W, ci, co = 1, 33, 45, 32, 32
    rng = np.random.default_rng(11)
    g = rng.standard_normal((n, H, W, ci))
    w = rng.standard_normal((9, co, ci)) / 17.0
    mask = np.maximum(rng.standard_normal((n, H, W, co)), 0.0)      # half zeros
    y = torch.empty((n, H, W, co), dtype=torch.bfloat16, device="cuda")
    # device copies kept alive until the kernel has run (a freed tensor's memory is handed to
    # the next allocation)
    gd, wd, md = _bf16(torch, g), _bf16(torch, w), _bf16(torch, mask)
    err.zero_()
    pkg.lbm2p_op_conv3x3(gd.data_ptr(), wd.data_ptr(), 0, md.data_ptr(), y.data_ptr(), 0, n, H,
                         W, ci, co, 0, err.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    ref = conv3x3(bf16_round(g), bf16_round(w)) * (bf16_round(mask) > 0)
    got = _np(y)
    assert np.all(got[bf16_round(mask) == 0] == 0.0)
    assert np.all(np.abs(got - ref) <= 2.0 ** -8 * np.abs(ref) + 1e-5 * np.max(np.abs(ref)))


@pytest.mark.parametrize("shape", [(1, 50, 70, 32, 32), (2, 19, 23, 16, 32),
                                   (1, 50, 70, 32, 16), (1, 400, 400, 32, 32)])
def test_weight_gradient_against_cpu(env, shape):
    torch, pkg, err = env
    n, H, W, ci, co = shape
    rng = np.random.default_rng(hash(shape) % 2 ** 32)
    x = rng.standard_normal((n, H, W, ci))
    g = rng.standard_normal((n, H, W, co))
    dw = torch.empty((9, co, ci), dtype=torch.float32, device="cuda")
    db = torch.empty(co, dtype=torch.float32, device="cuda")
    xd, gd = _bf16(torch, x), _bf16(torch, g)
    err.zero_()
    pkg.lbm2p_op_conv3x3_wgrad(xd.data_ptr(), gd.data_ptr(), dw.data_ptr(), db.data_ptr(), n, H,
                               W, ci, co, 0, err.data_ptr(),
                               torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    xr, gr = bf16_round(x), bf16_round(g)
    ref = conv3x3_wgrad(xr, gr)
    assert np.max(np.abs(_np(dw) - ref)) <= 1e-4 * np.max(np.abs(ref))
    refb = gr.reshape(-1, co).sum(0)
    assert np.max(np.abs(_np(db) - refb)) <= 1e-4 * np.max(np.abs(gr).reshape(-1, co).sum(0))


def test_flipped_weights_give_the_input_gradient(env):
    torch, pkg, err = env
    ci, co = 32, 16
    rng = np.random.default_rng(5)
    w = rng.standard_normal((9, co, ci))
    wd = _bf16(torch, w)
    wt = torch.empty((9, ci, co), dtype=torch.bfloat16, device="cuda")
    pkg.lbm2p_op_flip_weights(wd.data_ptr(), wt.data_ptr(), ci, co,
                              torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert np.array_equal(_np(wt), flip(bf16_round(w)))


def test_training_step_gradients_against_cpu(env):
    """One training step of the five-layer operator: the gradient of every weight and bias
    (before the Adam update) against the CPU reference network with the same BF16 roundings,
    within 1e-2 of each layer's largest gradient (BF16 activations near a rounding boundary
    may round the other way on one side), and the loss within 1e-4."""
    torch, pkg, err = env
    from paper_1808_07554_gb300.operator import LAYERS, PressureOperator
    from _conv_ref import network_gradients
    n, H, W = 2, 20, 24
    rng = np.random.default_rng(21)
    feat = np.zeros((n, H, W, 16))
    feat[..., :4] = rng.standard_normal((n, H, W, 4))
    target = rng.standard_normal((n, H, W))
    op = PressureOperator(seed=3)
    flat = op.p.cpu().numpy().astype(np.float64)
    weights, biases = [], []
    for (ci, co), (a, b, c) in zip(LAYERS, op.offsets):
        weights.append(flat[a:b].reshape(9, co, ci))
        biases.append(flat[b:c])
    fd = _bf16(torch, feat)
    td = _f32(torch, target)
    loss = op.train_step(fd, td, n, H, W, lr=1e-3)
    torch.cuda.synchronize()
    op.check()
    ref_loss, dW, db = network_gradients(feat, target, weights, biases)
    assert float(loss.item()) == pytest.approx(ref_loss, rel=1e-4)
    g = op.g.cpu().numpy().astype(np.float64)
    for l, ((ci, co), (a, b, c)) in enumerate(zip(LAYERS, op.offsets)):
        gw = g[a:b].reshape(9, co, ci)
        scale = max(np.max(np.abs(dW[l])), 1e-30)
        assert np.max(np.abs(gw - dW[l])) <= 1e-2 * scale, (l, np.max(np.abs(gw - dW[l])), scale)
        sb = max(np.max(np.abs(db[l])), 1e-30)
        assert np.max(np.abs(g[b:c] - db[l])) <= 1e-2 * sb, l


def test_training_reduces_a_learnable_loss(env):
    """A target that the operator can represent exactly (a fixed 3x3 filter of the pressure
    increment channel): twenty Adam steps lower the loss by more than half."""
    torch, pkg, err = env
    from paper_1808_07554_gb300.operator import PressureOperator
    from _conv_ref import conv3x3
    n, H, W = 4, 48, 40
    rng = np.random.default_rng(8)
    feat = np.zeros((n, H, W, 16))
    feat[..., :4] = rng.standard_normal((n, H, W, 4))
    k = np.zeros((9, 1, 16))
    k[4, 0, 3], k[1, 0, 3], k[7, 0, 0] = 0.8, 0.3, -0.5
    target = conv3x3(feat, k)[..., 0]
    op = PressureOperator(seed=4)
    fd, td = _bf16(torch, feat), _f32(torch, target)
    losses = [float(op.train_step(fd, td, n, H, W, lr=3e-3).item()) for _ in range(20)]
    op.check()
    assert losses[-1] < 0.5 * losses[0], losses


def test_learned_warm_start_loop_keeps_the_solution(env):
    """The whole learned warm start: training data recorded from the solver (two 64^2
    five-spot realisations), a short training, then a 128^2 five-spot stepped from the
    operator's predictions next to one stepped from the previous populations.  Both meet the
    same stopping rule, so their saturation fields agree closely (the prediction changes the
    sweep counts only)."""
    torch, pkg, err = env
    import workloads as W
    from paper_1808_07554_gb300.operator import (LearnedWarmStart, PressureOperator,
                                                 record_snapshots, train)
    runs = record_snapshots(pkg, [W.quarter_five_spot(64, seed=6000 + r, corr_len=8.0)
                                  for r in range(2)], 40)
    op = PressureOperator(seed=1)
    losses = train(op, runs, epochs=2, batch=8)
    assert len(losses) == 2 and np.all(np.isfinite(losses))
    prob = W.quarter_five_spot(128, seed=16, corr_len=12.0)
    plain = pkg.Solver.from_problem(prob, tol=1e-8)
    learned = pkg.Solver.from_problem(prob, tol=1e-8)
    lw = LearnedWarmStart(op, learned, np.log(prob.K))
    for _ in range(2):
        assert plain.step(1)[0] == pkg.OK
        assert learned.step(1)[0] == pkg.OK
        lw.prime()
    for _ in range(6):
        assert plain.step(1)[0] == pkg.OK
        st, stats = lw.step()
        assert st == pkg.OK and stats[0].sub_iters > 0
    op.check()
    assert W.rel_l2(learned.fields()[1], plain.fields()[1]) < 1e-5
    assert np.all(np.isfinite(lw.Ppred.cpu().numpy()))
