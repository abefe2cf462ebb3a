"""Pin: steady state of the pressure LBE for one Fourier mode (periodic, constant tau_f).

For F_p = A cos(k.x) on a periodic lattice the LBE (Eq. 3-1 with Eqs. 3-3, 3-9a) is linear
and shift invariant, so its steady state is one mode e^{ik.x} whose amplitudes solve an 8x8
complex system: after streaming f_i = e^{-ik.c_i} f_i^+ and f_i^+ = (1 - 1/tau) f_i
+ w_i P / tau + F/8 with P = (9/5) sum_i f_i.  For k -> 0 the amplitude tends to the
continuum solution of Eq. 2-15, P = F / (D |k|^2) with D = (tau - 1/2)/3 (Eq. 3-11a).
"""
import numpy as np
import pytest

import oracle as O
from _problems import constant_diffusivity

E = np.array([(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)])
Wt = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def closed_form_amplitude(k, tau, F):
    """P-hat of the steady mode, lattice units."""
    ph = np.exp(-1j * (E[1:] @ k))                 # e^{-i k.c_i}, i = 1..8
    A = np.eye(8, dtype=complex) - np.diag(ph) * (1.0 - 1.0 / tau)
    A -= np.outer(ph * Wt[1:], np.ones(8)) * (9.0 / 5.0) / tau
    b = ph * F / 8.0
    fhat = np.linalg.solve(A, b)
    return (9.0 / 5.0) * fhat.sum()


@pytest.mark.parametrize("nx,ny,m,tau", [(16, 16, (1, 2), 0.9), (12, 20, (2, 1), 1.7),
                                         (16, 8, (3, 0), 0.6)])
def test_oracle_matches_fourier_closed_form(nx, ny, m, tau):
    D = 0.05
    A = 2.0
    jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    k = np.array([2 * np.pi * m[0] / nx, 2 * np.pi * m[1] / ny])
    Fp_phys = A * np.cos(k[0] * ii + k[1] * jj)
    p = constant_diffusivity(nx, ny, D, tau, Fp=Fp_phys, S0=0.0)
    o = O.Oracle(p, tol=1e-14, check_every=2)
    assert o.init_status == O.OK
    sc = o.scalars()
    P = o.fields()["P"]
    o.close()
    # the source enters as s dx^2 F_p = dt F_p in lattice units
    Fl = sc["s"] * p.dx ** 2 * A
    Phat = closed_form_amplitude(k, tau, Fl)
    expect = np.real(Phat * np.exp(1j * (k[0] * ii + k[1] * jj)))
    assert np.max(np.abs(P - P.mean() - expect)) <= 1e-9 * np.max(np.abs(expect))


def test_closed_form_tends_to_continuum_poisson():
    tau, F = 1.1, 1e-3
    for nlat in (256, 1024):
        k = np.array([2 * np.pi / nlat, 0.0])
        D = (tau - 0.5) / 3.0
        ratio = closed_form_amplitude(k, tau, F) / (F / (D * k @ k))
        assert abs(ratio - 1.0) < 4.0 * (k @ k)        # second-order lattice correction
