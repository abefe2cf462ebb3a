"""Initial pressure guess for the t = 0 solve of a five-spot (set-up on the host side).

The paper leaves the t = 0 guess free (Sec. 4 starts the pressure solve from the equilibrium
of a given P_0).  A cold start from P_0 = 0 relaxes the slowest modes of the lattice, which
takes of the order of the lattice area in sweeps; solving the same problem on a 4x coarser
lattice first and prolonging its pressure removes most of that.  This module only prepares
an input array; every solve runs in the library.
"""
from __future__ import annotations

import numpy as np

import workloads as W


def coarse_initial_pressure(prob, pkg, factor=4, min_n=64, log=None, **solver_kw):
    """Initial pressure guess for a five-spot from the same problem on a coarser lattice
    (set-up only; the paper leaves the t = 0 guess free).  K is averaged geometrically
    over factor x factor blocks, the wells stay at the corner nodes, dt scales with dx^2;
    the coarse solve itself starts from a still coarser guess, down to min_n nodes, and is
    only converged to a relative increment of 1e-6 (a guess, not a solution)."""
    if prob.wells == [] or prob.nx % factor or prob.ny % factor or prob.nx // factor < min_n:
        return None
    nx, ny = prob.nx // factor, prob.ny // factor
    lnK = np.log(prob.K).reshape(ny, factor, nx, factor).mean(axis=(1, 3))
    c = W.quarter_five_spot(nx, ny, seed=0)
    c.K = np.exp(lnK)
    c.dx, c.dt = prob.dx * factor, prob.dt * factor * factor
    c.mu_w, c.mu_n, c.tau_p = prob.mu_w, prob.mu_n, prob.tau_p
    c.wells = [(0, 0, prob.wells[0][2], 0), (nx - 1, ny - 1, prob.wells[1][2], 1)]
    c.S0 = prob.S0.reshape(ny, factor, nx, factor).mean(axis=(1, 3))
    c.P0 = coarse_initial_pressure(c, pkg, factor, min_n, log, **solver_kw)
    s = pkg.Solver.from_problem(c, tol=1e-6, max_sub_iters=200_000, **solver_kw)
    if log is not None:
        log.append({"n": nx, "sweeps": s.init_stats.sub_iters, "r": s.init_stats.residual})
    P, _ = s.fields()
    s.close()
    return np.kron(P.astype(np.float64), np.ones((factor, factor)))
