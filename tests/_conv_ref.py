"""Plain CPU reference of the pressure operator's layers (test infrastructure): 3x3
convolutions with zero padding on channels-last images, their weight and input gradients, in
FP64 on the BF16-rounded values the GPU kernels read."""
import numpy as np

TAPS = [(t // 3 - 1, t % 3 - 1) for t in range(9)]          # (dy, dx) of tap t


def bf16_round(a):
    """Round FP32/FP64 values to the nearest BF16 (ties to even), returned as float64."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def shifted(x, dy, dx):
    """x[:, y + dy, x + dx, :] with zeros outside the image; x is [n, H, W, C]."""
    n, H, W, C = x.shape
    out = np.zeros_like(x)
    ys = slice(max(0, -dy), min(H, H - dy))
    xs = slice(max(0, -dx), min(W, W - dx))
    yd = slice(max(0, dy), min(H, H + dy))
    xd = slice(max(0, dx), min(W, W + dx))
    out[:, ys, xs, :] = x[:, yd, xd, :]
    return out


def conv3x3(x, w, bias=None):
    """y[p][co] = bias[co] + sum_t sum_ci x[p + d_t][ci] w[t][co][ci]; w is [9, co, ci]."""
    y = np.zeros(x.shape[:3] + (w.shape[1],))
    for t, (dy, dx) in enumerate(TAPS):
        y += shifted(x, dy, dx) @ w[t].T
    if bias is not None:
        y += bias
    return y


def conv3x3_wgrad(x, g):
    """dw[t][co][ci] = sum_p x[p + d_t][ci] g[p][co]."""
    ci, co = x.shape[-1], g.shape[-1]
    dw = np.zeros((9, co, ci))
    gf = g.reshape(-1, co)
    for t, (dy, dx) in enumerate(TAPS):
        dw[t] = gf.T @ shifted(x, dy, dx).reshape(-1, ci)
    return dw


def flip(w):
    """wt[t][ci][co] = w[8 - t][co][ci]: the input gradient is conv3x3(g, flip(w))."""
    return np.transpose(w[::-1], (0, 2, 1)).copy()


def network_gradients(feat, target, weights, biases, rounding=True):
    """Loss and parameter gradients of the operator's five layers (ReLU after the first four,
    mean-squared error of output channel 0 against target), rounding to BF16 where the GPU
    stores BF16: weights, activations and the backpropagated gradients.
    feat [n, H, W, 16]; weights[l] [9, co, ci]; returns (loss, [dW_l], [db_l])."""
    rd = bf16_round if rounding else (lambda a: np.asarray(a, dtype=np.float64))
    L = len(weights)
    wb = [rd(w) for w in weights]
    acts = [rd(feat)]
    for l in range(L - 1):
        acts.append(rd(np.maximum(conv3x3(acts[l], wb[l]) + biases[l], 0.0)))
    y = conv3x3(acts[L - 1], wb[L - 1]) + biases[L - 1]
    npix = y[..., 0].size
    y0 = y[..., 0].astype(np.float32).astype(np.float64) if rounding else y[..., 0]
    e = y0 - target
    loss = np.sum(e * e) / npix
    g = np.zeros_like(y)
    g[..., 0] = rd(2.0 * e / npix)
    dW, db = [None] * L, [None] * L
    for l in range(L - 1, -1, -1):
        dW[l] = conv3x3_wgrad(acts[l], g)
        db[l] = g.reshape(-1, g.shape[-1]).sum(0)
        if l > 0:
            g = rd(conv3x3(g, flip(wb[l])) * (acts[l] > 0))
    return loss, dW, db
