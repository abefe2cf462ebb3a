"""Small problem builders shared by the tests (inputs only; no solver arithmetic)."""
import numpy as np

import workloads as W


def uniform(nx, ny, *, bc=(W.PERIODIC,) * 4, phi=0.2, beta=0.4, mobility=W.MOB_QUADRATIC,
            mu_w=1.0, mu_n=2.0, D_s=0.01, tau_mode=W.TAU_REFERENCE, tau_p=1.0, dx=None,
            dt=None, K=None, S0=0.5, P0=None, Fp=None, Fs=None, wells=(), P_b=None, S_b=None,
            D_ref=0.0):
    dx = 1.0 / nx if dx is None else dx
    dt = 4.0 * dx * dx if dt is None else dt
    K = np.ones((ny, nx)) if K is None else np.asarray(K, dtype=np.float64)
    S0 = np.full((ny, nx), float(S0)) if np.isscalar(S0) else np.asarray(S0, dtype=np.float64)
    return W.Problem(name="test", nx=nx, ny=ny, dx=dx, dt=dt, phi=phi, beta=beta,
                     mobility=mobility, mu_w=mu_w, mu_n=mu_n, D_s=D_s, tau_mode=tau_mode,
                     tau_p=tau_p, bc=tuple(bc), K=K, S0=S0, P0=P0, Fp=Fp, Fs=Fs,
                     wells=list(wells), P_b=list(P_b) if P_b is not None else [None] * 4,
                     S_b=list(S_b) if S_b is not None else [None] * 4, D_ref=D_ref)


def constant_diffusivity(nx, ny, D, tau, **kw):
    """Decoupled mobility (lambda_t = lambda_w = 1/mu_w), K = 1, pseudo-step = dt, with dt
    chosen so that the pressure relaxation time is `tau` for D_p = D."""
    dx = kw.pop("dx", 1.0 / nx)
    dt = (tau - 0.5) * dx * dx / (3.0 * D)
    return uniform(nx, ny, mobility=W.MOB_DECOUPLED, mu_w=1.0 / D, mu_n=0.0,
                   tau_mode=W.TAU_PHYSICAL_DT, dx=dx, dt=dt, **kw)
