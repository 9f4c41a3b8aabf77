"""Pins for the global spin-torque diagnostics (CPU only).

The torque formula (commutator i <[H, sigma]>: 2 int b x m dV for the 2x2 potential, Eq. GMT;
the L.S part of the projectors, Eq. SOtorque) is checked against the time derivative of the
magnetisation under the exact propagator of the same fixed Hamiltonian (Ehrenfest), taken by
central differences with Richardson extrapolation, and its parts against their special cases:
no torque from the spin-orbit term without SOC, 2 mu_B B x M from a uniform field (Eq. magrot),
zero XC torque in the locally collinear approximation (Eq. spincont2)."""
import numpy as np
import pytest

from oracle import System
from oracle.tddft import chebyshev_order, exp_chebyshev
from tests._systems import parity_system


def magnetisation(s, psi):
    _, m = System.n_m(s.rho_v(psi))
    return m.sum(axis=(1, 2, 3)) * s.grid.dV


@pytest.mark.parametrize("lam,Bvec,xc", [(0.3, (0.05, -0.02, 0.04), 1), (0.3, (0.0, 0.0, 0.0), 0),
                                         (0.0, (0.05, 0.0, 0.03), 1)])
def test_torque_is_the_time_derivative_of_M(lam, Bvec, xc):
    wl, s, psi = parity_system(n=12, nstates=3, nk=2, lam=lam, natoms=2, xc=xc)
    A = np.array([0.05, -0.02, 0.03])
    B = np.array(Bvec)
    rho = s.rho_v(psi)
    V, parts = s.potential(rho, B)
    tq = s.torques(psi, rho, V, parts, A, B)
    emin, emax = s.spectral_bounds(V, [A])

    def M_at(tau):
        K = chebyshev_order(abs(tau) * 0.5 * (emax - emin), 1e-16)
        return magnetisation(s, exp_chebyshev(lambda x: s.apply_h(x, V, A), psi, tau, emin, emax, K))

    d = {}
    for tau in (2e-3, 1e-3):
        d[tau] = (M_at(tau) - M_at(-tau)) / (2.0 * tau)
    dMdt = (4.0 * d[1e-3] - d[2e-3]) / 3.0
    scale = max(np.abs(tq["total"]).max(), 1e-4)
    assert np.abs(dMdt - tq["total"]).max() <= 1e-6 * scale, (dMdt, tq)
    if lam == 0.0:
        assert np.abs(tq["soc"]).max() <= 1e-16
    else:
        assert np.abs(tq["soc"]).max() > 1e-3 * scale  # the spin-orbit term does act
    M = magnetisation(s, psi)
    assert np.allclose(tq["zeeman"], 2 * 0.5 * np.cross(B, M), atol=1e-15)
    assert np.abs(tq["xc"]).max() <= 1e-14  # b_xc parallel to m at every point
