"""Python binding of the lbm2p C ABI (``include/lbm2p.h``).

Argument marshalling only: every step of the solver runs in the CUDA kernels of
``liblbm2p.so``.  The functions below carry the C names; ``Solver`` is a small convenience
wrapper that owns a handle.  PyTorch, when used, only supplies device memory (its caching
allocator, through the allocation callback) and the CUDA stream the work is queued on.

The shared library is built in-tree by ``paper_1808_07554_gb300.build.build()`` (or the
repository's ``__graft_entry__.build()``).  Importing this package never falls back to
anything else: without the library every call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "liblbm2p.so")

OK, EINVAL, ENOMEM, ECUDA, ENOTCONVERGED, ENONFINITE, ENOTIMPL = range(7)
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENOTCONVERGED",
                5: "ENONFINITE", 6: "ENOTIMPL"}
PERIODIC, NOFLUX, DIRICHLET = 0, 1, 2
MOB_QUADRATIC, MOB_DECOUPLED, MOB_RATIONAL = 0, 1, 2
TAU_REFERENCE, TAU_PHYSICAL_DT = 0, 1
STORE_FP32, STORE_FP16_DEV = 0, 1
SWEEP_AUTO, SWEEP_VEC4, SWEEP_SCALAR, SWEEP_ROWS = 0, 1, 2, 3
MAX_WELLS = 16
NOALLOC_MAX_TILES = 65536   # LBM2P_NOALLOC_MAX_TILES: row tiles the static sweep scratch holds
NOALLOC_TILE_NODES = 1024   # nodes of one row tile of lbm2p_pressure_sweep_noalloc
STATE_PLANES = 20   # n_1..n_8 (f^+ - w_i R), g_0..g_8, 1/tau_f, S, R

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
RELEASE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p)


class lbm2p_well(C.Structure):
    _fields_ = [("i", C.c_int), ("j", C.c_int), ("q", C.c_double), ("is_producer", C.c_int)]


class lbm2p_params(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("dx", C.c_double), ("dt", C.c_double),
                ("phi", C.c_double), ("beta", C.c_double), ("mobility", C.c_int),
                ("mu_w", C.c_double), ("mu_n", C.c_double), ("D_s", C.c_double),
                ("tau_mode", C.c_int), ("tau_p", C.c_double), ("D_ref", C.c_double),
                ("tol", C.c_double), ("max_sub_iters", C.c_int), ("check_every", C.c_int),
                ("bc", C.c_int * 4), ("storage", C.c_int), ("fuse_sweeps", C.c_int),
                ("sweep_kernel", C.c_int), ("sat_lattice", C.c_int), ("D_c", C.c_double),
                ("warm_start", C.c_int),
                ("stream", C.c_void_p),
                ("alloc", ALLOC_FN), ("release", RELEASE_FN), ("alloc_ctx", C.c_void_p)]


class lbm2p_inputs(C.Structure):
    _fields_ = [("K", C.POINTER(C.c_double)), ("S0", C.POINTER(C.c_double)),
                ("P0", C.POINTER(C.c_double)), ("Fp", C.POINTER(C.c_double)),
                ("Fs", C.POINTER(C.c_double)), ("wells", C.POINTER(lbm2p_well)),
                ("n_wells", C.c_int), ("P_b", C.POINTER(C.c_double) * 4),
                ("S_b", C.POINTER(C.c_double) * 4), ("init_replay", C.POINTER(C.c_int))]


class lbm2p_step_stats(C.Structure):
    _fields_ = [("sub_iters", C.c_int), ("status", C.c_int), ("residual", C.c_double),
                ("sweep_ms", C.c_float), ("step_ms", C.c_float)]


class LBM2PError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load_library(path: str = LIB_PATH):
    """Load liblbm2p.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_1808_07554_gb300.build.build()")
    try:                      # let torch bind its CUDA runtime first when it is present
        import torch  # noqa: F401
    except ImportError:
        pass
    lib = C.CDLL(path)
    H = C.c_void_p
    fp = C.POINTER(C.c_float)
    sig = {
        "lbm2p_abi_version": (C.c_int, []),
        "lbm2p_default_params": (None, [C.POINTER(lbm2p_params)]),
        "lbm2p_create": (C.c_int, [C.POINTER(H), C.POINTER(lbm2p_params),
                                   C.POINTER(lbm2p_inputs), C.POINTER(lbm2p_step_stats)]),
        "lbm2p_set_sources": (C.c_int, [H, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
        "lbm2p_set_dirichlet": (C.c_int, [H, C.c_int, C.POINTER(C.c_double),
                                          C.POINTER(C.c_double)]),
        "lbm2p_step": (C.c_int, [H, C.c_int, C.POINTER(C.c_int), C.POINTER(lbm2p_step_stats)]),
        "lbm2p_pressure_sweeps": (C.c_int, [H, C.c_int, C.POINTER(C.c_double)]),
        "lbm2p_velocity": (C.c_int, [H, fp, fp, C.c_int]),
        "lbm2p_fields": (C.c_int, [H, fp, fp, C.c_int, C.c_int]),
        "lbm2p_state_count": (C.c_size_t, [H]),
        "lbm2p_get_state": (C.c_int, [H, fp, C.c_size_t, C.c_int]),
        "lbm2p_set_state": (C.c_int, [H, fp, C.c_size_t, C.c_int]),
        "lbm2p_set_timing": (C.c_int, [H, C.c_int]),
        "lbm2p_counters": (C.c_int, [H, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]),
        "lbm2p_sweep_config": (C.c_int, [H] + [C.POINTER(C.c_int)] * 4),
        "lbm2p_fused_form_of": (C.c_int, [H]),
        "lbm2p_set_fused_shape": (C.c_int, [H, C.c_int, C.c_int, C.c_int, C.c_int]),
        "lbm2p_autotune_report": (C.c_char_p, [H]),
        "lbm2p_warm_start": (C.c_int, [H, fp, C.c_int]),
        "lbm2p_pressure_sweep_noalloc": (C.c_int, [C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int),
                                                   C.POINTER(fp), C.POINTER(fp), fp, fp, fp,
                                                   C.POINTER(fp), fp, C.POINTER(C.c_double),
                                                   C.c_void_p]),
        "lbm2p_batch_create": (C.c_int, [C.POINTER(H), C.POINTER(H), C.c_int]),
        "lbm2p_batch_step": (C.c_int, [H, C.c_int, C.POINTER(C.c_int),
                                       C.POINTER(lbm2p_step_stats)]),
        "lbm2p_batch_counters": (C.c_int, [H, C.POINTER(C.c_longlong), C.POINTER(C.c_int)]),
        "lbm2p_batch_last_error": (C.c_char_p, [H]),
        "lbm2p_batch_destroy": (None, [H]),
        "lbm2p_last_error": (C.c_char_p, [H]),
        "lbm2p_destroy": (None, [H]),
        # the pressure operator (include/lbm2p_operator.h); device pointers as void *
        "lbm2p_op_conv3x3": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.c_void_p, C.c_void_p] + [C.c_int] * 6
                             + [C.c_void_p, C.c_void_p]),
        "lbm2p_op_conv3x3_wgrad": (C.c_int, [C.c_void_p] * 4 + [C.c_int] * 6
                                   + [C.c_void_p, C.c_void_p]),
        "lbm2p_op_flip_weights": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int,
                                            C.c_void_p]),
        "lbm2p_op_adam": (C.c_int, [C.c_void_p] * 5 + [C.c_longlong] + [C.c_float] * 4
                          + [C.c_int, C.c_void_p]),
        "lbm2p_op_diff_stats": (C.c_int, [C.c_void_p, C.c_void_p, C.c_longlong, C.c_void_p,
                                          C.c_void_p]),
        "lbm2p_op_features": (C.c_int, [C.c_void_p] * 8 + [C.c_int] * 2 + [C.c_float] * 2
                              + [C.c_void_p]),
        "lbm2p_op_target": (C.c_int, [C.c_void_p] * 5 + [C.c_int] * 2 + [C.c_void_p]),
        "lbm2p_op_predict": (C.c_int, [C.c_void_p] * 5 + [C.c_int] * 2 + [C.c_void_p]),
        "lbm2p_op_mse_grad": (C.c_int, [C.c_void_p] * 4 + [C.c_longlong, C.c_int, C.c_void_p]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _lib_or_raise():
    return load_library()


# ------------------------------------------------------------------------------------------
# C-named thin wrappers
# ------------------------------------------------------------------------------------------
def lbm2p_abi_version() -> int:
    return _lib_or_raise().lbm2p_abi_version()


def lbm2p_default_params() -> lbm2p_params:
    p = lbm2p_params()
    _lib_or_raise().lbm2p_default_params(C.byref(p))
    return p


def lbm2p_last_error(h=None) -> str:
    s = _lib_or_raise().lbm2p_last_error(h)
    return s.decode() if s else ""


def _check(st, h=None, allow=(OK,)):
    if st not in allow:
        raise LBM2PError(st, lbm2p_last_error(h))
    return st


def lbm2p_create(params: lbm2p_params, inputs: lbm2p_inputs, init_stats=None):
    h = C.c_void_p()
    st = _lib_or_raise().lbm2p_create(C.byref(h), C.byref(params), C.byref(inputs),
                                      C.byref(init_stats) if init_stats is not None else None)
    _check(st, None if not h.value else h, allow=(OK, ENOTCONVERGED))
    return h, st


def lbm2p_set_sources(h, Fp, Fs):
    return _check(_lib_or_raise().lbm2p_set_sources(h, _dp(Fp), _dp(Fs)), h)


def lbm2p_set_dirichlet(h, side, P_b, S_b):
    return _check(_lib_or_raise().lbm2p_set_dirichlet(h, side, _dp(P_b), _dp(S_b)), h)


def lbm2p_step(h, nsteps, replay=None, stats=None):
    rp = None
    if replay is not None:
        rp = (C.c_int * nsteps)(*[int(v) for v in replay])
    st = _lib_or_raise().lbm2p_step(h, nsteps, rp, stats)
    return _check(st, h, allow=(OK, ENOTCONVERGED))


def lbm2p_pressure_sweeps(h, nsweeps):
    r = C.c_double(0.0)
    _check(_lib_or_raise().lbm2p_pressure_sweeps(h, nsweeps, C.byref(r)), h)
    return r.value


def lbm2p_velocity(h, ux_ptr, uy_ptr, on_device):
    return _check(_lib_or_raise().lbm2p_velocity(h, ux_ptr, uy_ptr, on_device), h)


def lbm2p_fields(h, P_ptr, S_ptr, mean_free_P, on_device):
    return _check(_lib_or_raise().lbm2p_fields(h, P_ptr, S_ptr, mean_free_P, on_device), h)


def lbm2p_state_count(h) -> int:
    return int(_lib_or_raise().lbm2p_state_count(h))


def lbm2p_get_state(h, buf_ptr, count, on_device):
    return _check(_lib_or_raise().lbm2p_get_state(h, buf_ptr, count, on_device), h)


def lbm2p_set_state(h, buf_ptr, count, on_device):
    return _check(_lib_or_raise().lbm2p_set_state(h, buf_ptr, count, on_device), h)


def lbm2p_set_timing(h, enable):
    return _check(_lib_or_raise().lbm2p_set_timing(h, int(bool(enable))), h)


def lbm2p_counters(h):
    a, b = C.c_longlong(0), C.c_longlong(0)
    _check(_lib_or_raise().lbm2p_counters(h, C.byref(a), C.byref(b)), h)
    return a.value, b.value


def lbm2p_pressure_sweep_noalloc(nx, ny, pitch, bc, n_in, n_out, R, inv_tau, Fp, P_b, dP,
                                 stream=None):
    """Device pointers (ints) in, residual out; allocates nothing (see include/lbm2p.h)."""
    fp = C.POINTER(C.c_float)
    cast = lambda p: C.cast(C.c_void_p(p), fp) if p else None
    bcs = (C.c_int * 4)(*[int(b) for b in bc])
    nin = (fp * 8)(*[cast(p) for p in n_in])
    nout = (fp * 8)(*[cast(p) for p in n_out])
    pb = (fp * 4)(*[cast(p) for p in (P_b if P_b is not None else [0, 0, 0, 0])])
    r = C.c_double(0.0)
    st = _lib_or_raise().lbm2p_pressure_sweep_noalloc(
        int(nx), int(ny), int(pitch), bcs, nin, nout, cast(R), cast(inv_tau), cast(Fp), pb,
        cast(dP), C.byref(r), C.c_void_p(stream) if stream else None)
    _check(st, None)
    return r.value


# ---- the pressure operator (include/lbm2p_operator.h): device pointers as ints ----------
def lbm2p_op_conv3x3(x, w, bias, mask, y, y0, n_img, H, W, c_in, c_out, act, err, stream=0):
    _check(_lib_or_raise().lbm2p_op_conv3x3(x, w, bias or None, mask or None, y or None,
                                            y0 or None, n_img, H, W, c_in, c_out, act, err,
                                            stream or None))


def lbm2p_op_conv3x3_wgrad(x, g, dw, dbias, n_img, H, W, c_in, c_out, accumulate, err, stream=0):
    _check(_lib_or_raise().lbm2p_op_conv3x3_wgrad(x, g, dw, dbias or None, n_img, H, W, c_in,
                                                  c_out, int(bool(accumulate)), err,
                                                  stream or None))


def lbm2p_op_flip_weights(w, wt, c_in, c_out, stream=0):
    _check(_lib_or_raise().lbm2p_op_flip_weights(w, wt, c_in, c_out, stream or None))


def lbm2p_op_adam(p, g, m, v, pb, n, lr, beta1, beta2, eps, t, stream=0):
    _check(_lib_or_raise().lbm2p_op_adam(p, g, m, v, pb or None, n, lr, beta1, beta2, eps, t,
                                         stream or None))


def lbm2p_op_diff_stats(a, b, n, stats, stream=0):
    _check(_lib_or_raise().lbm2p_op_diff_stats(a, b, n, stats, stream or None))


def lbm2p_op_features(lnK, S, S_prev, P, P_prev, ds_stats, dp_stats, feat, H, W, s_mean, s_scale,
                      stream=0):
    _check(_lib_or_raise().lbm2p_op_features(lnK, S, S_prev, P, P_prev, ds_stats, dp_stats, feat,
                                             H, W, s_mean, s_scale, stream or None))


def lbm2p_op_target(P_next, P, P_prev, dp_stats, tgt, H, W, stream=0):
    _check(_lib_or_raise().lbm2p_op_target(P_next, P, P_prev, dp_stats, tgt, H, W, stream or None))


def lbm2p_op_predict(P, P_prev, d, dp_stats, P_pred, H, W, stream=0):
    _check(_lib_or_raise().lbm2p_op_predict(P, P_prev, d, dp_stats, P_pred, H, W, stream or None))


def lbm2p_op_mse_grad(y0, tgt, g, loss, npix, c_out, stream=0):
    _check(_lib_or_raise().lbm2p_op_mse_grad(y0, tgt, g, loss, npix, c_out, stream or None))


FUSED_NONE, FUSED_STAGES, FUSED_STAGED_ROWS, FUSED_DIRECT = 0, 1, 2, 3
ROWS2_DENSE = 16


def lbm2p_fused_form_of(h):
    """Which fused kernel runs the sweeps (FUSED_*)."""
    return _lib_or_raise().lbm2p_fused_form_of(h)


def lbm2p_set_fused_shape(h, form, warps, slots, rows):
    return _check(_lib_or_raise().lbm2p_set_fused_shape(h, int(form), int(warps), int(slots),
                                                        int(rows)), h)


def lbm2p_sweep_config(h):
    """(sweeps fused per launch, single-sweep kernel kind, fused tile threads, fused tile rows)"""
    v = [C.c_int(0) for _ in range(4)]
    _check(_lib_or_raise().lbm2p_sweep_config(h, *[C.byref(x) for x in v]), h)
    return tuple(x.value for x in v)


def lbm2p_autotune_report(h) -> str:
    s = _lib_or_raise().lbm2p_autotune_report(h)
    return s.decode() if s else ""


def lbm2p_destroy(h):
    if h:
        _lib_or_raise().lbm2p_destroy(h)


def lbm2p_batch_last_error(b=None) -> str:
    s = _lib_or_raise().lbm2p_batch_last_error(b)
    return s.decode() if s else ""


def lbm2p_batch_create(handles):
    arr = (C.c_void_p * len(handles))(*[h.value if isinstance(h, C.c_void_p) else h
                                        for h in handles])
    b = C.c_void_p()
    st = _lib_or_raise().lbm2p_batch_create(C.byref(b), arr, len(handles))
    if st != OK:
        raise LBM2PError(st, lbm2p_batch_last_error(None))
    return b


def lbm2p_batch_step(b, nsteps, count, replay=None, stats=None):
    """replay: None or nsteps*count sweep counts, step-major."""
    rp = None
    if replay is not None:
        flat = [int(v) for v in np.asarray(replay).reshape(-1)]
        if len(flat) != nsteps * count:
            raise ValueError(f"replay needs {nsteps * count} counts")
        rp = (C.c_int * len(flat))(*flat)
    st = _lib_or_raise().lbm2p_batch_step(b, nsteps, rp, stats)
    if st not in (OK, ENOTCONVERGED):
        raise LBM2PError(st, lbm2p_batch_last_error(b))
    return st


def lbm2p_batch_counters(b):
    a, t = C.c_longlong(0), C.c_int(0)
    st = _lib_or_raise().lbm2p_batch_counters(b, C.byref(a), C.byref(t))
    if st != OK:
        raise LBM2PError(st, lbm2p_batch_last_error(b))
    return a.value, t.value


def lbm2p_batch_destroy(b):
    if b:
        _lib_or_raise().lbm2p_batch_destroy(b)


# ------------------------------------------------------------------------------------------
# marshalling helpers
# ------------------------------------------------------------------------------------------
def _f64(a, n=None):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


def _dp(a):
    if a is None:
        return None
    a = _f64(a)
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _fp(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_float))


def _dev_fp(t):
    """A float32 device tensor's address as a float pointer (shape and dtype checked by the
    caller)."""
    return None if t is None else C.cast(C.c_void_p(t.data_ptr()), C.POINTER(C.c_float))


class _TorchMemory:
    """Device memory from torch's caching allocator on torch's current stream."""

    def __init__(self, device=None):
        import torch
        self.torch = torch
        self.device = torch.cuda.current_device() if device is None else device
        self.stream = torch.cuda.current_stream(self.device)
        self._live = {}

        def _alloc(nbytes, ctx):
            try:
                ptr = torch.cuda.caching_allocator_alloc(int(nbytes), self.device, self.stream)
            except Exception:       # out of memory: report NULL to the library
                return None
            self._live[int(ptr)] = int(nbytes)
            return int(ptr)

        def _release(ptr, nbytes, ctx):
            if ptr and int(ptr) in self._live:
                del self._live[int(ptr)]
                torch.cuda.caching_allocator_delete(int(ptr))

        self.alloc_fn = ALLOC_FN(_alloc)
        self.release_fn = RELEASE_FN(_release)


class Solver:
    """Owns one lbm2p handle.  Arrays are numpy [ny, nx]; FP64 in, FP32 out."""

    def __init__(self, *, nx, ny, dx, dt, phi, beta, mobility, mu_w, mu_n, D_s, tau_mode,
                 tau_p, bc, K, S0, P0=None, Fp=None, Fs=None, wells=(), P_b=None, S_b=None,
                 D_ref=0.0, tol=1e-8, max_sub_iters=10_000_000, check_every=8,
                 init_replay=None, use_torch=True, stream=None, fuse_sweeps=0,
                 sweep_kernel=0, sat_lattice=9, D_c=0.0, storage=0, warm_start=0):
        lib = _lib_or_raise()
        self.nx, self.ny = int(nx), int(ny)
        n = self.nx * self.ny
        p = lbm2p_params()
        lib.lbm2p_default_params(C.byref(p))
        p.nx, p.ny, p.dx, p.dt = self.nx, self.ny, float(dx), float(dt)
        p.phi, p.beta, p.mobility = float(phi), float(beta), int(mobility)
        p.mu_w, p.mu_n, p.D_s = float(mu_w), float(mu_n), float(D_s)
        p.tau_mode, p.tau_p, p.D_ref = int(tau_mode), float(tau_p), float(D_ref)
        p.tol, p.max_sub_iters, p.check_every = float(tol), int(max_sub_iters), int(check_every)
        p.fuse_sweeps = int(fuse_sweeps)
        p.sweep_kernel = int(sweep_kernel)
        p.sat_lattice = int(sat_lattice)
        p.storage = int(storage)
        p.warm_start = int(warm_start)
        p.D_c = float(D_c)
        for s in range(4):
            p.bc[s] = int(bc[s])
        self._mem = None
        if use_torch:
            self._mem = _TorchMemory()
            p.alloc = self._mem.alloc_fn
            p.release = self._mem.release_fn
            p.stream = self._mem.stream.cuda_stream if stream is None else stream
        elif stream is not None:
            p.stream = stream
        self.params = p
        keep = []
        inp = lbm2p_inputs()

        def put(a):
            a = _f64(a, n)
            keep.append(a)
            return a.ctypes.data_as(C.POINTER(C.c_double))

        inp.K = put(K)
        inp.S0 = put(S0)
        inp.P0 = put(P0) if P0 is not None else None
        inp.Fp = put(Fp) if Fp is not None else None
        inp.Fs = put(Fs) if Fs is not None else None
        wl = list(wells)
        if wl:
            arr = (lbm2p_well * len(wl))(*[lbm2p_well(int(i), int(j), float(q), int(bool(pr)))
                                           for (i, j, q, pr) in wl])
            keep.append(arr)
            inp.wells = C.cast(arr, C.POINTER(lbm2p_well))
        inp.n_wells = len(wl)
        for s in range(4):
            if P_b is not None and P_b[s] is not None:
                a = _f64(P_b[s])
                keep.append(a)
                inp.P_b[s] = a.ctypes.data_as(C.POINTER(C.c_double))
            if S_b is not None and S_b[s] is not None:
                a = _f64(S_b[s])
                keep.append(a)
                inp.S_b[s] = a.ctypes.data_as(C.POINTER(C.c_double))
        if init_replay is not None:
            ir = C.c_int(int(init_replay))
            keep.append(ir)
            inp.init_replay = C.pointer(ir)
        self.init_stats = lbm2p_step_stats()
        self.h, self.create_status = lbm2p_create(p, inp, self.init_stats)
        del keep

    @classmethod
    def from_problem(cls, prob, **kw):
        """Build from any object with the attributes of a problem description (nx, ny, dx,
        dt, phi, beta, mobility, mu_w, mu_n, D_s, tau_mode, tau_p, bc, K, S0, P0, Fp, Fs,
        wells, P_b, S_b, D_ref)."""
        return cls(nx=prob.nx, ny=prob.ny, dx=prob.dx, dt=prob.dt, phi=prob.phi, beta=prob.beta,
                   mobility=prob.mobility, mu_w=prob.mu_w, mu_n=prob.mu_n, D_s=prob.D_s,
                   tau_mode=prob.tau_mode, tau_p=prob.tau_p, bc=prob.bc, K=prob.K, S0=prob.S0,
                   P0=prob.P0, Fp=prob.Fp, Fs=prob.Fs, wells=prob.wells, P_b=prob.P_b,
                   S_b=prob.S_b, D_ref=prob.D_ref,
                   sat_lattice=getattr(prob, "sat_lattice", 9), D_c=getattr(prob, "D_c", 0.0),
                   **kw)

    # -- lifecycle ----------------------------------------------------------------------
    def close(self):
        if getattr(self, "h", None):
            lbm2p_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- inputs ---------------------------------------------------------------------------
    def set_sources(self, Fp=None, Fs=None):
        n = self.nx * self.ny
        lbm2p_set_sources(self.h, _f64(Fp, n), _f64(Fs, n))

    def warm_start(self, P_guess):
        """Start the next pressure solve from the pressure field P_guess ([ny, nx])."""
        buf = np.ascontiguousarray(P_guess, dtype=np.float32).reshape(self.ny, self.nx)
        _check(_lib_or_raise().lbm2p_warm_start(self.h, _fp(buf), 0), self.h)

    def set_dirichlet(self, side, P_b=None, S_b=None):
        lbm2p_set_dirichlet(self.h, side, P_b, S_b)

    # -- stepping -------------------------------------------------------------------------
    def step(self, nsteps=1, replay=None):
        """Advance nsteps; returns (status, stats list)."""
        stats = (lbm2p_step_stats * max(1, nsteps))()
        st = lbm2p_step(self.h, nsteps, replay, stats)
        return st, [stats[i] for i in range(nsteps)]

    def pressure_sweeps(self, nsweeps):
        return lbm2p_pressure_sweeps(self.h, nsweeps)

    def set_timing(self, enable=True):
        lbm2p_set_timing(self.h, enable)

    def counters(self):
        return lbm2p_counters(self.h)

    def set_fused_shape(self, form, warps, slots, rows):
        """Pin the two-sweep launch shape (see lbm2p_set_fused_shape)."""
        return lbm2p_set_fused_shape(self.h, form, warps, slots, rows)

    def sweep_config(self):
        return lbm2p_sweep_config(self.h)

    def fused_form(self):
        return lbm2p_fused_form_of(self.h)

    def autotune_report(self):
        """[(candidate, a1, a2, a3, a4, us per sweep)] as timed at create."""
        out = []
        for ln in lbm2p_autotune_report(self.h).splitlines():
            f = ln.split()
            out.append((f[0], *[int(v) for v in f[1:5]], float(f[5])))
        return out

    # -- outputs --------------------------------------------------------------------------
    def fields(self, mean_free_P=False, out=None):
        """P and S of the current time level as float32 [ny, nx] host arrays; ``out`` = a
        pair of C-contiguous float32 arrays of that shape to fill instead (page-locked ones
        make the copy a direct DMA)."""
        if out is None:
            P = np.empty((self.ny, self.nx), np.float32)
            S = np.empty((self.ny, self.nx), np.float32)
        else:
            P, S = out
            for a in (P, S):
                if a.dtype != np.float32 or a.shape != (self.ny, self.nx) or not a.flags.c_contiguous:
                    raise ValueError("out arrays must be C-contiguous float32 of shape (ny, nx)")
        lbm2p_fields(self.h, _fp(P), _fp(S), int(bool(mean_free_P)), 0)
        return P, S

    def fields_device(self, P, S, mean_free_P=False):
        """P and S of the current time level into float32 [ny, nx] contiguous device tensors
        (either may be None); the copy is queued on the solver's stream."""
        for t in (P, S):
            if t is not None and (str(t.dtype) != "torch.float32" or not t.is_cuda or
                                  tuple(t.shape) != (self.ny, self.nx) or not t.is_contiguous()):
                raise ValueError("fields_device wants contiguous float32 (ny, nx) CUDA tensors")
        lbm2p_fields(self.h, _dev_fp(P), _dev_fp(S), int(bool(mean_free_P)), 1)

    def warm_start_device(self, P_guess):
        """Start the next pressure solve from a float32 [ny, nx] device tensor."""
        if (str(P_guess.dtype) != "torch.float32" or not P_guess.is_cuda or
                tuple(P_guess.shape) != (self.ny, self.nx) or not P_guess.is_contiguous()):
            raise ValueError("warm_start_device wants a contiguous float32 (ny, nx) CUDA tensor")
        _check(_lib_or_raise().lbm2p_warm_start(self.h, _dev_fp(P_guess), 1), self.h)

    def velocity(self):
        ux = np.empty((self.ny, self.nx), np.float32)
        uy = np.empty((self.ny, self.nx), np.float32)
        lbm2p_velocity(self.h, _fp(ux), _fp(uy), 0)
        return ux, uy

    def get_state(self):
        n = lbm2p_state_count(self.h)
        buf = np.empty(n, np.float32)
        lbm2p_get_state(self.h, _fp(buf), n, 0)
        return buf.reshape(STATE_PLANES, self.ny, self.nx)

    def set_state(self, state):
        n = lbm2p_state_count(self.h)
        buf = np.ascontiguousarray(state, dtype=np.float32).reshape(-1)
        if buf.size != n:
            raise ValueError(f"state must hold {n} floats")
        lbm2p_set_state(self.h, _fp(buf), n, 0)


class Batch:
    """Steps several Solver objects together (lbm2p_batch_*).  Keep the solvers alive and
    step them only through the batch while it exists."""

    def __init__(self, solvers):
        self.solvers = list(solvers)
        self.b = lbm2p_batch_create([s.h for s in self.solvers])

    def close(self):
        if getattr(self, "b", None):
            lbm2p_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def step(self, nsteps=1, replay=None):
        """Advance every member nsteps; returns (status, stats[nsteps][count])."""
        n = len(self.solvers)
        stats = (lbm2p_step_stats * max(1, nsteps * n))()
        st = lbm2p_batch_step(self.b, nsteps, n, replay, stats)
        return st, [[stats[s * n + m] for m in range(n)] for s in range(nsteps)]

    def counters(self):
        """(kernels launched by the batch, tiles of one batched sweep)"""
        return lbm2p_batch_counters(self.b)
