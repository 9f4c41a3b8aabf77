"""Pins for the collinear (Eq. SDFT / Eq. HSDFT, sigma_z-only potential) and spin-unpolarised
modes of the propagation step (CPU only).

Both modes are checked against an independent scalar propagation written here: every spinor
component psi_{i,alpha} is a scalar orbital with occupation f_i, propagated by the same ETRS
scheme with its channel's potential -- v_loc + v_H[n] + v^LSDA_alpha(n_up, n_dn) +
(-1)^alpha mu_B B_z with n_alpha = sum_i f_i |psi_{i,alpha}|^2 (collinear), or v_loc + v_H[n] +
v^LDA(n) for both components (unpolarised) -- so that tilted spinors, whose transverse
magnetisation the collinear Hamiltonian ignores, are covered too."""
import math

import numpy as np
import pytest

from oracle import System
from oracle import xc as oxc
from oracle.tddft import MU_B, exp_chebyshev, hartree_potential
from paper_2506_21908_gb300 import synthetic as S
from tests._systems import make_oracle


def tilted_system(mode, n=12, nstates=3):
    wl = S.small_parity(n=n, nstates=nstates, nk=1, lam=0.0, natoms=2, field=False)
    wl.spin_mode = mode
    s = System.from_workload(wl)
    psi = S.small_parity_states(wl)
    return wl, s, psi


def scalar_reference(s, psi, occ, pots, times, A, dt, nst, emin, emax, Kf, Kh):
    """ETRS with n_sc = 1 on the scalar components; pots(comps) -> [v_up, v_dn]."""
    comps = [(psi[0, i, a].copy(), occ[i], a) for i in range(psi.shape[1]) for a in (0, 1)]

    def hs(p, v, Avec):
        spin = np.zeros((1, 2) + p.shape, np.complex128)
        spin[0, 0] = p
        return s.apply_kinetic(spin, Avec)[0, 0] + v * p + s.apply_nonlocal(spin, Avec)[0, 0]

    def expo(cs, vs, Avec, tau, K):
        return [(exp_chebyshev(lambda x, a=a: hs(x, vs[a], Avec), p, tau, emin, emax, K), f, a) for p, f, a in cs]

    t = 0.0
    vs = pots(comps, t)
    for j in range(nst):
        A0, A1 = A[j], A[j + 1]
        pred = expo(comps, vs, A0, dt, Kf)
        v1 = pots(pred, t + dt)
        half = expo(comps, vs, A0, 0.5 * dt, Kh)
        new = expo(half, v1, A1, 0.5 * dt, Kh)
        v1 = pots(new, t + dt)
        new = expo(half, v1, A1, 0.5 * dt, Kh)
        comps = new
        t += dt
        vs = pots(comps, t)
    return comps


def channel_densities(comps):
    nu = sum(f * np.abs(p) ** 2 for p, f, a in comps if a == 0)
    nd = sum(f * np.abs(p) ** 2 for p, f, a in comps if a == 1)
    return nu, nd


@pytest.mark.parametrize("mode", [1, 2])
def test_spin_mode_equals_independent_scalar_propagation(mode):
    wl, s, psi = tilted_system(mode)
    nst, dt = 2, 0.05
    times = np.arange(nst + 1) * dt
    A = np.outer(times, [0.3, 0.1, 0.0])
    B = np.tile([0.15, -0.05, 0.2], (nst + 1, 1))  # transverse parts are ignored in both modes
    o = make_oracle(s, psi, times, A, B, dt, n_sc=1)
    emin, emax, Kf, Kh = o.emin, o.emax, o.K_full, o.K_half
    for _ in range(nst):
        o.step()

    def pots(comps, t):
        nu, nd = channel_densities(comps)
        vH = hartree_potential(s.grid, nu + nd)
        if mode == 1:
            _, vu, vd = oxc.lsda(nu, nd)
            Bz = B[0, 2]
            return [s.vloc + vH + vu + MU_B * Bz, s.vloc + vH + vd - MU_B * Bz]
        n = nu + nd
        _, v, _ = oxc.lsda(0.5 * n, 0.5 * n)
        return [s.vloc + vH + v, s.vloc + vH + v]

    comps = scalar_reference(s, psi, wl.occ[0], pots, times, A, dt, nst, emin, emax, Kf, Kh)
    for j, (p, f, a) in enumerate(comps):
        i = j // 2
        assert np.abs(o.psi[0, i, a] - p).max() < 1e-12 * np.abs(p).max()


def test_collinear_mode_matches_non_collinear_for_z_magnetisation():
    """With m along +-z at every point and B along z the two modes give the same potential."""
    wl, s1, psi = tilted_system(1)
    psi = psi.copy()
    for i, sg in enumerate([0, 1, 0]):
        psi[0, i, 1 - sg] = 0.0
    wl.spin_mode = 0
    s0 = System.from_workload(wl)
    rho = s0.rho_v(psi)
    V0, _ = s0.potential(rho, [0.0, 0.0, 0.2])
    V1, _ = s1.potential(rho, [0.0, 0.0, 0.2])
    assert np.abs(V0 - V1).max() <= 1e-13 * np.abs(V0).max()


def test_spin_modes_reject_spin_orbit_coupling():
    """L.S couples the spin channels, so it needs the non-collinear mode."""
    wl = S.small_parity(n=8, nstates=2, nk=1, lam=0.02, natoms=1, field=False)
    wl.spin_mode = 1
    with pytest.raises(ValueError):
        System.from_workload(wl)


def test_unpolarised_mode_has_no_spin_field():
    wl, s, psi = tilted_system(2)
    rho = s.rho_v(psi)
    V, parts = s.potential(rho, [0.3, 0.2, 0.1])
    assert np.array_equal(V[0], V[1]) and not V[2].any() and not V[3].any()
    n = rho[0] + rho[1]
    e, v, _ = oxc.lsda(0.5 * n, 0.5 * n)
    cx = (3.0 / math.pi) ** (1.0 / 3.0)
    ec, _, _ = oxc.pw92_correlation((3.0 / (4.0 * math.pi * n)) ** (1.0 / 3.0), np.zeros_like(n))
    assert np.allclose(parts["exc"], -0.75 * cx * n ** (4.0 / 3.0) + n * ec, rtol=1e-12, atol=0)
