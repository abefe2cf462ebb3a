"""FP64 CPU oracle (test infrastructure).

A thin ctypes front end for ``lbm2p_oracle.c``: the plain double-precision implementation
of the double-distribution LB model (arXiv 1808.07554, Secs. 3-4) that the GPU solver is
checked against.  Only the test-suite, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg use this package; the solver library never imports, links or runs it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm2p_oracle.c")
_LIB = os.path.join(_HERE, "liblbm2p_oracle.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, ENOMEM, ENOTCONVERGED, ENONFINITE = 0, 1, 2, 4, 5


# Another build of the oracle to load instead of this one (the pin tests' planted-mistake
# check compiles altered copies of the source and runs the pins against them)
LIB_ENV = "LBM2P_ORACLE_LIB"


def compile_source(src: str, out: str) -> str:
    """gcc with the oracle's flags (IEEE double, no fast-math, no FMA contraction)."""
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-fopenmp", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle (once, or again when the source is newer)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    return compile_source(_SRC, _LIB)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            alt = os.environ.get(LIB_ENV)
            if alt:
                lib = C.CDLL(alt)
            else:
                build()
                lib = C.CDLL(_LIB)
            dp = C.POINTER(C.c_double)
            ip = C.POINTER(C.c_int)
            lib.orc_create.restype = C.c_void_p
            lib.orc_create.argtypes = [ip, dp, dp, dp, dp, dp, dp, C.c_int, ip, dp,
                                       C.POINTER(dp), C.POINTER(dp), ip, ip, dp]
            lib.orc_destroy.argtypes = [C.c_void_p]
            lib.orc_set_sources.argtypes = [C.c_void_p, dp, dp]
            lib.orc_set_dirichlet.argtypes = [C.c_void_p, C.c_int, dp, dp]
            lib.orc_set_dirichlet.restype = C.c_int
            lib.orc_step.argtypes = [C.c_void_p, C.c_int, ip, ip, dp]
            lib.orc_step.restype = C.c_int
            lib.orc_refresh.argtypes = [C.c_void_p]
            lib.orc_pressure.argtypes = [C.c_void_p, C.c_int, ip, dp]
            lib.orc_pressure.restype = C.c_int
            lib.orc_saturation.argtypes = [C.c_void_p]
            lib.orc_fields.argtypes = [C.c_void_p] + [dp] * 6
            lib.orc_get_state.argtypes = [C.c_void_p, dp, dp, dp, dp]
            lib.orc_set_state.argtypes = [C.c_void_p, dp, dp, dp, dp]
            lib.orc_set_prev_pressure.argtypes = [C.c_void_p, dp]
            lib.orc_get_pre.argtypes = [C.c_void_p, dp, dp]
            lib.orc_scalars.argtypes = [C.c_void_p, dp]
            lib.orc_constants.argtypes = [C.c_void_p, dp]
            lib.orc_sums.argtypes = [C.c_void_p, dp]
            lib.orc_saturation_source.argtypes = [C.c_void_p, dp]
            lib.orc_set_threads.argtypes = [C.c_int]
            lib.orc_set_threads.restype = C.c_int
            _lib = lib
    return _lib


def _dptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a, shape=None):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None and a.shape != shape:
        a = a.reshape(shape)
    return a


def set_threads(n: int = 0) -> int:
    """Host threads the oracle's loops use from now on (n <= 0: leave as is); returns the
    count in effect."""
    return int(_load().orc_set_threads(int(n)))


class OracleError(RuntimeError):
    pass


class Oracle:
    """FP64 reference solver.  Arrays are [ny, nx] float64, row-major."""

    def __init__(self, prob, tol=1e-8, max_sub_iters=10_000_000, check_every=8,
                 init_replay=None, warm_start=0):
        lib = _load()
        self.lib = lib
        self.nx, self.ny = prob.nx, prob.ny
        self.prob = prob
        shape = (prob.ny, prob.nx)
        ip = (C.c_int * 13)(prob.nx, prob.ny, prob.mobility, prob.tau_mode, int(max_sub_iters),
                            int(check_every), *[int(b) for b in prob.bc],
                            -1 if init_replay is None else int(init_replay),
                            int(getattr(prob, "sat_lattice", 9)), int(warm_start))
        dpar = (C.c_double * 11)(prob.dx, prob.dt, prob.phi, prob.beta, prob.mu_w, prob.mu_n,
                                 prob.D_s, prob.tau_p, prob.D_ref, tol,
                                 float(getattr(prob, "D_c", 0.0)))
        self._keep = []
        K = _f64(prob.K, shape)
        S0 = _f64(prob.S0, shape)
        P0 = _f64(prob.P0, shape)
        Fp = _f64(prob.Fp, shape)
        Fs = _f64(prob.Fs, shape)
        nw = len(prob.wells)
        wint = np.zeros(max(1, 3 * nw), dtype=np.int32)
        wq = np.zeros(max(1, nw), dtype=np.float64)
        for m, (i, j, q, prod) in enumerate(prob.wells):
            wint[3 * m:3 * m + 3] = (i, j, 1 if prod else 0)
            wq[m] = q
        Pb_arr = (C.POINTER(C.c_double) * 4)()
        Sb_arr = (C.POINTER(C.c_double) * 4)()
        for s in range(4):
            if prob.P_b[s] is not None:
                a = _f64(prob.P_b[s])
                self._keep.append(a)
                Pb_arr[s] = _dptr(a)
            if prob.S_b[s] is not None:
                a = _f64(prob.S_b[s])
                self._keep.append(a)
                Sb_arr[s] = _dptr(a)
        status = C.c_int(0)
        k0 = C.c_int(0)
        r0 = C.c_double(0.0)
        h = lib.orc_create(ip, dpar, _dptr(K), _dptr(S0), _dptr(P0), _dptr(Fp), _dptr(Fs), nw,
                           wint.ctypes.data_as(C.POINTER(C.c_int)), _dptr(wq), Pb_arr, Sb_arr,
                           C.byref(status), C.byref(k0), C.byref(r0))
        if not h:
            raise OracleError(f"orc_create failed with status {status.value}")
        self.h = h
        self.init_status = status.value
        self.init_sub_iters = k0.value
        self.init_residual = r0.value

    def close(self):
        if getattr(self, "h", None):
            self.lib.orc_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    # -- inputs -----------------------------------------------------------------------
    def set_sources(self, Fp=None, Fs=None):
        shape = (self.ny, self.nx)
        Fp = _f64(Fp, shape)
        Fs = _f64(Fs, shape)
        self.lib.orc_set_sources(self.h, _dptr(Fp), _dptr(Fs))

    def set_dirichlet(self, side, Pb=None, Sb=None):
        Pb = _f64(Pb)
        Sb = _f64(Sb)
        st = self.lib.orc_set_dirichlet(self.h, side, _dptr(Pb), _dptr(Sb))
        if st != OK:
            raise OracleError(f"orc_set_dirichlet({side}) failed with status {st}")

    # -- stepping ---------------------------------------------------------------------
    def step(self, nsteps=1, replay=None):
        """Advance nsteps physical steps; returns (status, sub_iters[nsteps], r[nsteps])."""
        k = np.zeros(nsteps, dtype=np.int32)
        r = np.zeros(nsteps, dtype=np.float64)
        rp = None
        if replay is not None:
            rarr = np.ascontiguousarray(replay, dtype=np.int32)
            assert rarr.size == nsteps
            rp = rarr.ctypes.data_as(C.POINTER(C.c_int))
        st = self.lib.orc_step(self.h, nsteps, rp, k.ctypes.data_as(C.POINTER(C.c_int)),
                               r.ctypes.data_as(C.POINTER(C.c_double)))
        return st, k, r

    def refresh(self):
        self.lib.orc_refresh(self.h)

    def pressure(self, n=-1):
        k = C.c_int(0)
        r = C.c_double(0.0)
        st = self.lib.orc_pressure(self.h, int(n), C.byref(k), C.byref(r))
        return st, k.value, r.value

    def saturation(self):
        self.lib.orc_saturation(self.h)

    # -- outputs ----------------------------------------------------------------------
    def fields(self):
        shape = (self.ny, self.nx)
        out = {k: np.zeros(shape) for k in ("P", "S", "gradPx", "gradPy", "ux", "uy")}
        self.lib.orc_fields(self.h, *[_dptr(out[k]) for k in
                                      ("P", "S", "gradPx", "gradPy", "ux", "uy")])
        return out

    def get_state(self):
        n = self.nx * self.ny
        f = np.zeros((9, self.ny, self.nx))
        g = np.zeros((9, self.ny, self.nx))
        tau = np.zeros((self.ny, self.nx))
        S = np.zeros((self.ny, self.nx))
        self.lib.orc_get_state(self.h, _dptr(f), _dptr(g), _dptr(tau), _dptr(S))
        del n
        return dict(f=f, g=g, tau_f=tau, S=S)

    def set_state(self, f=None, g=None, tau_f=None, S=None):
        f = _f64(f, (9, self.ny, self.nx))
        g = _f64(g, (9, self.ny, self.nx))
        tau_f = _f64(tau_f, (self.ny, self.nx))
        S = _f64(S, (self.ny, self.nx))
        self.lib.orc_set_state(self.h, _dptr(f), _dptr(g), _dptr(tau_f), _dptr(S))

    def get_pre(self):
        """Most recent pulled populations (after creation: g(t=0) before its collision)."""
        f = np.zeros((9, self.ny, self.nx))
        g = np.zeros((9, self.ny, self.nx))
        self.lib.orc_get_pre(self.h, _dptr(f), _dptr(g))
        return dict(f=f, g=g)

    def set_prev_pressure(self, P):
        P = _f64(P, (self.ny, self.nx))
        self.lib.orc_set_prev_pressure(self.h, _dptr(P))

    def scalars(self):
        out = np.zeros(6)
        self.lib.orc_scalars(self.h, _dptr(out))
        return dict(s=out[0], tau_g=out[1], D_ref=out[2], step=int(out[3]), last_r=out[4],
                    last_k=int(out[5]))

    def constants(self):
        out = np.zeros(64)
        self.lib.orc_constants(self.h, _dptr(out))
        return dict(w=out[0:9], wbar=out[9:18], Gamma=out[18:27], wg=out[54:63], qs=int(out[63]),
                    ex=out[27:36].astype(int),
                    ey=out[36:45].astype(int), opp=out[45:54].astype(int))

    def sums(self):
        out = np.zeros(2)
        self.lib.orc_sums(self.h, _dptr(out))
        return dict(f=out[0], g=out[1])

    def saturation_source(self):
        out = np.zeros((self.ny, self.nx))
        self.lib.orc_saturation_source(self.h, _dptr(out))
        return out


def run_problem(prob, nsteps=None, tol=1e-8, check_every=8, max_sub_iters=10_000_000,
                replay=None, init_replay=None, warm_start=0):
    """Run a workloads.Problem through the oracle, updating time-dependent sources and
    wall values before each step.  Returns (oracle, sub_iters log [init, step1, ...])."""
    o = Oracle(prob, tol=tol, check_every=check_every, max_sub_iters=max_sub_iters,
               init_replay=init_replay, warm_start=warm_start)
    nsteps = prob.steps if nsteps is None else nsteps
    log = [o.init_sub_iters]
    for n in range(1, nsteps + 1):
        t = n * prob.dt
        if prob.sources_at is not None:
            o.set_sources(*prob.sources_at(t))
        if prob.walls_at is not None:
            Pb, Sb = prob.walls_at(t)
            for s in range(4):
                if prob.bc[s] == 2:
                    o.set_dirichlet(s, Pb[s], Sb[s])
        st, k, _ = o.step(1, None if replay is None else [replay[n]])
        if st not in (OK, ENOTCONVERGED):
            raise OracleError(f"oracle step {n} failed with status {st}")
        log.append(int(k[0]))
    return o, log
