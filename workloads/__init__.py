"""Seeded synthetic inputs for the two-phase Darcy LB solver and its oracle.

This module only *describes problems*: permeability fields, initial fields, closed-form
manufactured solutions with their source terms, well lists and Dirichlet wall traces. It
contains none of the lattice Boltzmann arithmetic (no equilibria, no collision, no streaming,
no relaxation-time mapping); both the CUDA path and the FP64 oracle receive these arrays as
inputs.

Problem statement (Chai, Liang, Du, Shi, arXiv 1808.07554, Sec. 2, Eqs. 2-15 and 2-18):
    div(D_p grad P) + F_p = 0,           D_p = K * lambda_t(S)
    phi dS/dt = div(D_s grad S) + F_s + div(lambda_w K grad P)

Grids are cell-centred: node (i, j) sits at x = (i + 1/2) dx, y = (j + 1/2) dx, with walls
half-way between the outermost nodes and the domain edge. Arrays are row-major [j, i]
(ny rows of nx values), FP64.

Dirichlet wall traces ("half-spaced traces") hold the prescribed value at the points
k * dx / 2, k = 0 .. 2n, along a side (n = ny for the x-sides, nx for the y-sides); a
boundary link of node j on an x-side crosses the wall at k = 2 j + 1 - e_y.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# side order used by the solver and the oracle: x-min, x-max, y-min, y-max
XMIN, XMAX, YMIN, YMAX = 0, 1, 2, 3
PERIODIC, NOFLUX, DIRICHLET = 0, 1, 2
# mobility laws (see the solver header for their definitions)
MOB_QUADRATIC, MOB_DECOUPLED, MOB_RATIONAL = 0, 1, 2
TAU_REFERENCE, TAU_PHYSICAL_DT = 0, 1


@dataclass
class Problem:
    """A complete problem instance: parameters plus the arrays both solvers need."""
    name: str
    nx: int
    ny: int
    dx: float
    dt: float
    phi: float
    beta: float
    mobility: int
    mu_w: float
    mu_n: float
    D_s: float
    tau_mode: int
    tau_p: float
    bc: tuple
    K: np.ndarray
    S0: np.ndarray
    P0: np.ndarray | None = None
    Fp: np.ndarray | None = None
    Fs: np.ndarray | None = None
    wells: list = field(default_factory=list)   # (i, j, q, is_producer)
    P_b: list = field(default_factory=lambda: [None] * 4)
    S_b: list = field(default_factory=lambda: [None] * 4)
    D_ref: float = 0.0                          # <= 0: geometric mean of D_p at t = 0
    sat_lattice: int = 9                        # saturation lattice: 9 (D2Q9) or 5 (D2Q5)
    D_c: float = 0.0                            # D_s(S) = D_s + D_c K lambda_w lambda_n / lambda_t
    # callables t -> arrays, for problems whose sources / wall values depend on time
    sources_at: object = None                   # t -> (Fp, Fs)
    walls_at: object = None                     # t -> (P_b list, S_b list)
    exact_at: object = None                     # t -> dict(P=, S=, ux=, uy=)
    steps: int = 0


def node_coords(nx: int, ny: int, dx: float, x0: float = 0.0, y0: float = 0.0):
    """Cell-centred node coordinates as [ny, nx] arrays."""
    x = x0 + (np.arange(nx) + 0.5) * dx
    y = y0 + (np.arange(ny) + 0.5) * dx
    return np.meshgrid(x, y, indexing="xy")


def wall_trace_points(side: int, nx: int, ny: int, dx: float, x0=0.0, y0=0.0):
    """Coordinates (x, y) of the 2n+1 half-spaced points of a side's wall trace."""
    if side in (XMIN, XMAX):
        k = np.arange(2 * ny + 1)
        y = y0 + 0.5 * k * dx
        x = np.full_like(y, x0 if side == XMIN else x0 + nx * dx)
    else:
        k = np.arange(2 * nx + 1)
        x = x0 + 0.5 * k * dx
        y = np.full_like(x, y0 if side == YMIN else y0 + ny * dx)
    return x, y


# --------------------------------------------------------------------------------------
# Gaussian random permeability fields
# --------------------------------------------------------------------------------------
def grf_lnK(nx: int, ny: int, sigma: float, corr_len: float, seed: int) -> np.ndarray:
    """Stationary Gaussian random field on the periodic nx-by-ny grid.

    White noise from ``numpy.random.default_rng(seed)`` is filtered with the square root of
    the spectrum of the Gaussian covariance C(r) = exp(-r^2 / l^2) (l in cells, wrapped
    distances), then standardised to sample mean 0 and standard deviation 1 and scaled by
    sigma.  Returns ln K.
    """
    rng = np.random.default_rng(seed)
    w = rng.standard_normal((ny, nx))
    ix = np.arange(nx)
    iy = np.arange(ny)
    dxw = np.minimum(ix, nx - ix).astype(np.float64)
    dyw = np.minimum(iy, ny - iy).astype(np.float64)
    C = np.exp(-(dyw[:, None] ** 2 + dxw[None, :] ** 2) / float(corr_len) ** 2)
    spec = np.fft.fft2(C).real
    spec[spec < 0.0] = 0.0
    fld = np.fft.ifft2(np.sqrt(spec) * np.fft.fft2(w)).real
    fld = (fld - fld.mean()) / fld.std()
    return sigma * fld


# --------------------------------------------------------------------------------------
# Manufactured periodic problem: 64^2 unit square, quadratic relative permeabilities
# --------------------------------------------------------------------------------------
def manufactured_fields(x, y, t, mu_w=1.0, mu_n=2.0, phi=0.2, D_s=0.01, p_amp=1.0, D_c=0.0):
    """Closed-form p, S, K on the periodic unit square and the sources that make them exact.

    p = A sin(2 pi x) cos(2 pi y) e^-t,  S = 1/2 + 1/4 sin(2 pi x) sin(2 pi y) e^-t,
    K = 1 + 1/2 sin(2 pi x) sin(2 pi y),  lambda_w = S^2/mu_w, lambda_n = (1-S)^2/mu_n.
    F_p = -div(K lambda_t grad p),  F_s = phi dS/dt - div(D grad S) - div(lambda_w K grad p)
    with D = D_s + D_c K h(S), h = lambda_w lambda_n / lambda_t (D_c = 0: constant D_s),
    expanded by the product rule with hand-derived first and second derivatives.
    The pressure amplitude A (p_amp) is 1 for the parity workload; smaller values lower the
    Darcy velocity, hence the advective Courant number on coarse grids.
    """
    a = 2.0 * math.pi
    sx, cx = np.sin(a * x), np.cos(a * x)
    sy, cy = np.sin(a * y), np.cos(a * y)
    e = math.exp(-t)
    K = 1.0 + 0.5 * sx * sy
    Kx = 0.5 * a * cx * sy
    Ky = 0.5 * a * sx * cy
    p = p_amp * sx * cy * e
    px = p_amp * a * cx * cy * e
    py = -p_amp * a * sx * sy * e
    lap_p = -2.0 * a * a * p
    S = 0.5 + 0.25 * sx * sy * e
    Sx = 0.25 * a * cx * sy * e
    Sy = 0.25 * a * sx * cy * e
    lap_S = -2.0 * a * a * (S - 0.5)
    dS_dt = -(S - 0.5)
    lw = S * S / mu_w
    ln = (1.0 - S) ** 2 / mu_n
    lt = lw + ln
    dlw = 2.0 * S / mu_w
    dlt = dlw - 2.0 * (1.0 - S) / mu_n
    gradS_gradp = Sx * px + Sy * py
    gradK_gradp = Kx * px + Ky * py
    div_Klt_gradp = lt * gradK_gradp + K * dlt * gradS_gradp + K * lt * lap_p
    div_Klw_gradp = lw * gradK_gradp + K * dlw * gradS_gradp + K * lw * lap_p
    Fp = -div_Klt_gradp
    # div(D grad S) = D lap S + grad D . grad S, grad D = D_c (h grad K + K h'(S) grad S)
    dln = -2.0 * (1.0 - S) / mu_n
    h = lw * ln / lt
    dh = (dlw * ln + lw * dln) / lt - lw * ln * dlt / (lt * lt)
    D = D_s + D_c * K * h
    gradS2 = Sx * Sx + Sy * Sy
    gradK_gradS = Kx * Sx + Ky * Sy
    div_D_gradS = D * lap_S + D_c * (h * gradK_gradS + K * dh * gradS2)
    Fs = phi * dS_dt - div_D_gradS - div_Klw_gradp
    u_x = -K * lt * px
    u_y = -K * lt * py
    return dict(K=K, P=p, S=S, Fp=Fp, Fs=Fs, ux=u_x, uy=u_y, gradPx=px, gradPy=py)


def manufactured_periodic(n: int = 64, steps: int = 500, tau_p: float = 1.0,
                          p_amp: float = 1.0, D_c: float = 0.0, sat_lattice: int = 9,
                          beta: float = 0.4) -> Problem:
    """64x64 periodic unit square with the manufactured p and S (closed-form sources).

    phi = 0.2, beta = 0.4 (the largest admissible value not above 1 for phi = 0.2),
    mu_w = 1, mu_n = 2, D_s = 0.01, tau_p = 1.0, tau_s = 0.8; dt = 4 dx^2 is the step
    at which the saturation relaxation time equals 0.8 for these beta and D_s.
    The discrete mean of F_p is removed at every time: on a periodic domain the pressure
    equation is solvable only for a zero-mean source.  Variants: D_c > 0 makes D_s depend
    on S and K (D_s + D_c K lambda_w lambda_n / lambda_t); sat_lattice = 5 carries S on
    D2Q5 (which needs beta <= 1.5 phi, e.g. beta = 0.3).
    """
    dx = 1.0 / n
    dt = 4.0 * dx * dx
    X, Y = node_coords(n, n, dx)
    f0 = manufactured_fields(X, Y, 0.0, p_amp=p_amp, D_c=D_c)

    def sources_at(t):
        m = manufactured_fields(X, Y, t, p_amp=p_amp, D_c=D_c)
        Fp = m["Fp"] - m["Fp"].mean()
        return Fp, m["Fs"]

    def exact_at(t):
        m = manufactured_fields(X, Y, t, p_amp=p_amp, D_c=D_c)
        return dict(P=m["P"], S=m["S"], ux=m["ux"], uy=m["uy"])

    Fp0, Fs0 = sources_at(0.0)
    return Problem(name=f"manufactured_periodic_{n}", nx=n, ny=n, dx=dx, dt=dt, phi=0.2,
                   beta=beta, mobility=MOB_QUADRATIC, mu_w=1.0, mu_n=2.0, D_s=0.01,
                   tau_mode=TAU_REFERENCE, tau_p=tau_p, bc=(PERIODIC,) * 4, K=f0["K"],
                   S0=f0["S"], P0=f0["P"], Fp=Fp0, Fs=Fs0, sources_at=sources_at,
                   exact_at=exact_at, steps=steps, sat_lattice=sat_lattice, D_c=D_c)


# --------------------------------------------------------------------------------------
# Quarter five-spot on a Gaussian-random-field permeability
# --------------------------------------------------------------------------------------
def quarter_five_spot(nx: int = 1024, ny: int | None = None, seed: int = 2,
                      sigma: float = 1.0, corr_len: float = 16.0, q: float = 1e-3,
                      mu_w: float = 1.0, mu_n: float = 2.0, S0: float = 0.2,
                      steps: int = 2000, tau_p: float = 1.0) -> Problem:
    """Quarter five-spot: injector at node (0, 0), producer at the opposite corner node.

    No-flux walls on all four sides; ln K is a seeded Gaussian random field (sigma, corr_len
    in cells); uniform initial saturation S0; P0 = 0; phi = 0.2, beta = 0.4, D_s = 0.01,
    tau_p = 1.0, tau_s = 0.8 (dt = 4 dx^2).  The domain is [0, nx dx] x [0, ny dx] with
    dx = 1/nx.  Each well is a point source of total rate q at one node: the solver spreads
    it over that node's cell (F = +-q / dx^2).
    """
    ny = nx if ny is None else ny
    dx = 1.0 / nx
    dt = 4.0 * dx * dx
    lnK = grf_lnK(nx, ny, sigma, corr_len, seed)
    K = np.exp(lnK)
    wells = [(0, 0, q, 0), (nx - 1, ny - 1, q, 1)]
    return Problem(name=f"quarter_five_spot_{nx}x{ny}", nx=nx, ny=ny, dx=dx, dt=dt, phi=0.2,
                   beta=0.4, mobility=MOB_QUADRATIC, mu_w=mu_w, mu_n=mu_n, D_s=0.01,
                   tau_mode=TAU_REFERENCE, tau_p=tau_p, bc=(NOFLUX,) * 4, K=K,
                   S0=np.full((ny, nx), float(S0)), P0=np.zeros((ny, nx)), wells=wells,
                   steps=steps)


# --------------------------------------------------------------------------------------
# The paper's analytic examples (Sec. 4.1 and 4.2), Dirichlet walls on all sides
# --------------------------------------------------------------------------------------
def example1(n: int = 64, c: float = 1.0) -> Problem:
    """Decoupled problem of Sec. 4.1 (Eqs. 4-1, 4-2) on [0, 2]^2.

    P = 1 + sin(pi x) sin(pi y),  S = t sin(pi x) sin(pi y),  phi = 1, D_p = D_s = 1e-3,
    lambda_t = lambda_w (so lambda_w K = D_p); F_p = 2 D_p pi^2 sin sin and
    Q = F_s - F_p = (2 D_s pi^2 t + phi) sin sin.  Lattice speed c, dt = dx / c; the
    pressure pseudo-step equals dt.  Initial and wall values from the exact solution.
    """
    L = 2.0
    dx = L / n
    dt = dx / c
    Dp = 1e-3
    Ds = 1e-3
    phi = 1.0
    X, Y = node_coords(n, n, dx)
    pi = math.pi

    def ssxy(x, y):
        return np.sin(pi * x) * np.sin(pi * y)

    def exact_at(t):
        s = ssxy(X, Y)
        ux = -Dp * pi * np.cos(pi * X) * np.sin(pi * Y)
        uy = -Dp * pi * np.sin(pi * X) * np.cos(pi * Y)
        return dict(P=1.0 + s, S=t * s, ux=ux, uy=uy)

    def sources_at(t):
        s = ssxy(X, Y)
        Fp = 2.0 * Dp * pi * pi * s
        Q = (2.0 * Ds * pi * pi * t + phi) * s
        return Fp, Q + Fp

    def walls_at(t):
        Pb, Sb = [], []
        for side in range(4):
            wx, wy = wall_trace_points(side, n, n, dx)
            s = ssxy(wx, wy)
            Pb.append(1.0 + s)
            Sb.append(t * s)
        return Pb, Sb

    Fp0, Fs0 = sources_at(0.0)
    Pb0, Sb0 = walls_at(0.0)
    e0 = exact_at(0.0)
    return Problem(name=f"example1_{n}", nx=n, ny=n, dx=dx, dt=dt, phi=phi, beta=1.0,
                   mobility=MOB_DECOUPLED, mu_w=1.0 / Dp, mu_n=0.0, D_s=Ds,
                   tau_mode=TAU_PHYSICAL_DT, tau_p=0.0, bc=(DIRICHLET,) * 4,
                   K=np.ones((n, n)), S0=e0["S"], P0=e0["P"], Fp=Fp0, Fs=Fs0, P_b=Pb0, S_b=Sb0,
                   sources_at=sources_at, walls_at=walls_at, exact_at=exact_at,
                   steps=int(round(1.0 / dt)))


def example2(n: int = 128, c: float = 10.0, phi: float = 1.0, beta: float = 1.0,
             T: float = 0.2) -> Problem:
    """Coupled benchmark of Sec. 4.2 (Eqs. 4-4, 4-5) on [0, 1]^2.

    D_p = 1/(0.5 - 0.2 S), lambda_w K = S D_p, D_s = 0.01, F_p = 0,
    F_s = 2 pi^2 D_s sin(pi xi) + 2 pi (1 - phi) cos(pi xi), xi = x + y - 2t;
    exact P = -cos(pi xi)/(5 pi) - (x + y)/2, u = (1, 1), S = sin(pi xi).
    """
    dx = 1.0 / n
    dt = dx / c
    Ds = 0.01
    X, Y = node_coords(n, n, dx)
    pi = math.pi

    def exact_xy(x, y, t):
        xi = x + y - 2.0 * t
        return -np.cos(pi * xi) / (5.0 * pi) - 0.5 * (x + y), np.sin(pi * xi)

    def exact_at(t):
        P, S = exact_xy(X, Y, t)
        return dict(P=P, S=S, ux=np.ones_like(P), uy=np.ones_like(P))

    def sources_at(t):
        xi = X + Y - 2.0 * t
        Fs = 2.0 * pi * pi * Ds * np.sin(pi * xi) + 2.0 * pi * (1.0 - phi) * np.cos(pi * xi)
        return np.zeros_like(Fs), Fs

    def walls_at(t):
        Pb, Sb = [], []
        for side in range(4):
            wx, wy = wall_trace_points(side, n, n, dx)
            P, S = exact_xy(wx, wy, t)
            Pb.append(P)
            Sb.append(S)
        return Pb, Sb

    Fp0, Fs0 = sources_at(0.0)
    Pb0, Sb0 = walls_at(0.0)
    e0 = exact_at(0.0)
    return Problem(name=f"example2_{n}", nx=n, ny=n, dx=dx, dt=dt, phi=phi, beta=beta,
                   mobility=MOB_RATIONAL, mu_w=1.0, mu_n=1.0, D_s=Ds,
                   tau_mode=TAU_PHYSICAL_DT, tau_p=0.0, bc=(DIRICHLET,) * 4,
                   K=np.ones((n, n)), S0=e0["S"], P0=e0["P"], Fp=Fp0, Fs=Fs0, P_b=Pb0, S_b=Sb0,
                   sources_at=sources_at, walls_at=walls_at, exact_at=exact_at,
                   steps=int(round(T / dt)))


# --------------------------------------------------------------------------------------
# Error measures
# --------------------------------------------------------------------------------------
def mean_free(a: np.ndarray) -> np.ndarray:
    return a - a.mean()


def rel_l2(a: np.ndarray, b: np.ndarray) -> float:
    """||a - b||_2 / ||b||_2 (b is the reference)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b.ravel())
    return float(np.linalg.norm((a - b).ravel()) / (nb if nb > 0 else 1.0))


def rel_l1(numeric: np.ndarray, exact: np.ndarray) -> float:
    """Global relative error of Sec. 4: sum|exact - numeric| / sum|exact|."""
    return float(np.abs(exact - numeric).sum() / np.abs(exact).sum())
