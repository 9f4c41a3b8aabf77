"""Pins for the oracle's energy terms (System.energies), CPU only.

Two kinds of pin, both independent of how the terms are coded:

* conservation: for a Hamiltonian without explicit time dependence the exact dynamics conserves
  E = sum f <psi|T + V_NL|psi> + int v_loc n + 1/2 int v_H n + int n eps_xc + int mu_B B.m only when
  H is the functional derivative of E term by term (the Hartree factor 1/2, the XC functional value
  rather than its potential integral of Eq. xc_energy4, the sign of the Zeeman term of
  Eq. zeeman_potential).  The time-reversible ETRS step then conserves E up to O(dt^2) over a fixed
  time span, so the drift must fall fourfold when dt halves; a wrong weight or sign in any term
  adds a drift that does not fall with dt;
* closed forms: Hartree self-energy and erf-potential energy of a Gaussian charge in a periodic
  cubic cell with the G = 0 terms of reading P4 (Ewald sums with the simple-cubic Madelung
  constant), kinetic energy of plane waves, Zeeman energy of a uniform spin gas, and the non-local
  energy of a state equal to a projector.
"""
import math

import numpy as np
import pytest

from oracle.tddft import MU_B, System
from paper_2506_21908_gb300 import synthetic as S
from tests._systems import make_oracle, parity_system, uniform_gas

# Madelung constant of a simple cubic lattice of unit point charges in a uniform compensating
# background: the potential at a lattice site from all other charges and the background is -XI / L.
XI_SC = 2.8372974794806

TERMS = ("kin", "nl", "loc", "H", "xc", "Z")


def _energy_series(dt, T, lam, xc, natoms, B):
    """Energy terms at every step of a field-free (static B) run of duration T with converged
    self-consistency (time-reversible ETRS)."""
    wl, s, psi = parity_system(n=12, nstates=3, nk=1, lam=lam, field=False, natoms=natoms, xc=xc)
    nst = int(round(T / dt))
    times = np.arange(nst + 1) * dt
    Bt = np.tile(np.asarray(B, np.float64), (nst + 1, 1))
    o = make_oracle(s, psi, times, np.zeros((nst + 1, 3)), Bt, dt, n_sc=40, sc_tol=1e-13)
    out = [o.observables()[2]]
    for _ in range(nst):
        o.step()
        out.append(o.observables()[2])
    return {k: np.array([e[k] for e in out]) for k in TERMS + ("total", "xc_pot")}


def _drift(series, weights=None, xc_pot=False):
    """|E(T) - E(0)| of the total, optionally re-weighted term by term (planted mistakes)."""
    w = dict.fromkeys(TERMS, 1.0)
    if weights:
        w.update(weights)
    tot = sum(w[k] * series[k] for k in TERMS)
    if xc_pot:
        tot = tot - series["xc"] + series["xc_pot"]
    return abs(tot[-1] - tot[0])


CONFIGS = {
    # atoms with SOC, XC and a static Zeeman field: every term changes in time
    "full": dict(lam=0.02, xc=1, natoms=2, B=(0.05, -0.03, 0.08)),
    # no atoms: kinetic, Hartree, XC and Zeeman only
    "xc_only": dict(lam=0.0, xc=1, natoms=0, B=(0.0, 0.04, 0.06)),
    # atoms without XC or field: kinetic, local, non-local and Hartree
    "atoms_only": dict(lam=0.02, xc=0, natoms=2, B=(0.0, 0.0, 0.0)),
}


@pytest.fixture(scope="module")
def runs():
    return {name: {dt: _energy_series(dt, 0.4, **cfg) for dt in (0.1, 0.05, 0.025)} for name, cfg in CONFIGS.items()}


@pytest.mark.parametrize("name", list(CONFIGS))
def test_energy_conserved_to_second_order(runs, name):
    """Field-free total energy drift over a fixed span falls as dt^2 (ratio ~4 per halving), and at
    the smallest dt it is far below the change of every term that moves."""
    r = runs[name]
    d = {dt: _drift(s) for dt, s in r.items()}
    assert d[0.1] / d[0.05] > 3.3 and d[0.05] / d[0.025] > 3.3, d
    fine = r[0.025]
    moving = [abs(fine[k][-1] - fine[k][0]) for k in TERMS if abs(fine[k][-1] - fine[k][0]) > 1e-6]
    assert len(moving) >= 3
    assert d[0.025] < 0.02 * min(moving), (d, moving)
    # the reported total is the sum of the six terms
    assert np.allclose(fine["total"], sum(fine[k] for k in TERMS), rtol=0, atol=1e-13)


@pytest.mark.parametrize("mistake", [
    dict(weights={"H": 2.0}),         # Hartree energy without its 1/2
    dict(weights={"H": 0.0}),         # Hartree energy dropped
    dict(weights={"Z": -1.0}),        # Zeeman energy with the wrong sign
    dict(xc_pot=True),                # E_xc as the potential integral int <rho_v, V_xc> (Eq. xc_energy4)
    dict(weights={"nl": 2.0}),        # non-local energy counted twice
    dict(weights={"loc": -1.0}),      # local energy with the wrong sign
    dict(weights={"kin": 0.5}),       # kinetic energy with an extra 1/2
])
def test_conservation_detects_a_planted_mistake(runs, mistake):
    """Re-weighting one of the oracle's terms (a planted mistake in its energy) breaks the
    second-order convergence of the drift in the full configuration."""
    r = runs["full"]
    d = {dt: _drift(s, **mistake) for dt, s in r.items()}
    assert not (d[0.05] / d[0.025] > 3.3 and d[0.025] < 1e-6), (mistake, d)


def _gaussian_system(L, n, Q, with_atom):
    pos = np.array([[L / 2.0] * 3]) if with_atom else np.zeros((0, 3))
    return System([L] * 3, n, pos, np.zeros(len(pos), np.int32), [8.0], [0.8], [1.0], 0, np.zeros((1, 1)),
                  np.zeros((1, 1)), 5.0, np.zeros((1, 3)), np.ones(1), np.array([[Q]]), xc=0)


def _gaussian_state(s, L, sigma, Q):
    g = s.grid
    d = g.r - L / 2.0
    rho = Q * (2.0 * math.pi * sigma * sigma) ** -1.5 * np.exp(-(d * d).sum(-1) / (2.0 * sigma * sigma))
    psi = np.zeros((1, 1, 2) + rho.shape, np.complex128)
    psi[0, 0, 0] = np.sqrt(rho / Q)
    r4 = s.rho_v(psi)
    V, parts = s.potential(r4, np.zeros(3))
    return s.energies(psi, r4, V, parts, np.zeros(3), np.zeros(3))


@pytest.mark.parametrize("sigma,Q", [(1.0, 2.0), (0.8, 1.0)])
def test_hartree_energy_of_gaussian_charge(sigma, Q):
    """1/2 int v_H n of a Gaussian charge (per-axis width sigma) in a periodic cube with the G = 0
    term dropped: Q^2/(2 sigma sqrt(pi)) - Q^2 XI/(2L) + 2 pi Q^2 sigma^2 / L^3 (self-energy, Madelung
    energy of the lattice of images, and the background term of the Ewald sum)."""
    L, n = 20.0, 48
    E = _gaussian_state(_gaussian_system(L, n, Q, False), L, sigma, Q)
    expect = Q * Q / (2.0 * sigma * math.sqrt(math.pi)) - Q * Q * XI_SC / (2.0 * L) \
        + 2.0 * math.pi * Q * Q * sigma ** 2 / L ** 3
    assert E["H"] == pytest.approx(expect, rel=1e-12)


def test_local_energy_of_gaussian_charge_on_an_atom():
    """int v_loc n of a Gaussian charge centred on an atom with -Z erf(r/rc)/r (reading P4, G = 0 keeps
    pi Z rc^2 / Omega): -2 Z Q / sqrt(pi (rc^2 + 2 sigma^2)) + Z Q XI / L - 2 pi Z Q sigma^2 / L^3."""
    L, n, sigma, Q, Z, rc = 20.0, 48, 1.0, 2.0, 8.0, 0.8
    E = _gaussian_state(_gaussian_system(L, n, Q, True), L, sigma, Q)
    expect = -2.0 * Z * Q / math.sqrt(math.pi * (rc * rc + 2.0 * sigma * sigma)) + Z * Q * XI_SC / L \
        - 2.0 * math.pi * Z * Q * sigma ** 2 / L ** 3
    assert E["loc"] == pytest.approx(expect, rel=1e-12)


def test_kinetic_and_zeeman_energy_of_a_uniform_spin_gas():
    """Plane waves exp(i G_i.r) chi with occupations f_i at k-point k and vector potential A:
    E_kin = sum_i f_i |G_i + k + A|^2 / 2; the common spin direction u gives E_Z = mu_B B.u sum_i f_i."""
    theta, phi = 0.6, 0.2
    s, psi = uniform_gas(nstates=3, theta=theta, phi=phi, xc=0)
    occ = np.array([[1.0, 0.5, 0.25]])
    s.occ = occ
    k = np.array([0.1, -0.2, 0.05])
    A = np.array([0.03, 0.02, -0.04])
    s.kpts = k[None]
    B = np.array([0.3, -0.2, 0.1])
    r4 = s.rho_v(psi)
    V, parts = s.potential(r4, B)
    E = s.energies(psi, r4, V, parts, A, B)
    g = s.grid
    idx = [(0, 0, 0), (0, 1, 0), (2, 0, 1)]
    ekin = sum(f * 0.5 * ((g.G[i] + k + A) ** 2).sum() for f, i in zip(occ[0], idx))
    u = np.array([math.sin(theta) * math.cos(phi), math.sin(theta) * math.sin(phi), math.cos(theta)])
    assert E["kin"] == pytest.approx(ekin, rel=1e-12)
    assert E["Z"] == pytest.approx(MU_B * (B @ u) * occ.sum(), rel=1e-12)
    assert E["H"] == pytest.approx(0.0, abs=1e-12)  # uniform density: only G = 0, which is dropped


@pytest.mark.parametrize("D0", [1.0, -0.7])
def test_nonlocal_energy_of_a_projector_state(D0):
    """A state proportional to one atom's s projector, psi = beta / ||beta||: <psi|V_NL|psi> = D_0 ||beta||^2
    (the whole projector norm on the grid), in either spin channel."""
    L, n = 10.0, 32
    s = System([L] * 3, n, np.array([[5.0, 5.0, 5.0]]), np.zeros(1, np.int32), [8.0], [0.8], [1.0], 0,
               np.array([[D0]]), np.zeros((1, 1)), 4.0, np.zeros((1, 3)), np.ones(1), np.ones((1, 2)), xc=0)
    at = s.atoms[0]
    beta = np.zeros(s.grid.N)
    beta[at.idx] = at.beta[0]
    b2 = (beta * beta).sum() * s.grid.dV
    assert b2 == pytest.approx(1.0, abs=2e-3)  # continuum-normalised projector, sampled
    chi = S.spinor_along(1.1, -0.4)
    psi = np.zeros((1, 2, 2) + (n,) * 3, np.complex128)
    for i, c in enumerate((chi, S.spinor_along(1.1, -0.4, parallel=False))):
        psi[0, i, 0] = c[0] * beta.reshape((n,) * 3) / math.sqrt(b2)
        psi[0, i, 1] = c[1] * beta.reshape((n,) * 3) / math.sqrt(b2)
    r4 = s.rho_v(psi)
    V, parts = s.potential(r4, np.zeros(3))
    E = s.energies(psi, r4, V, parts, np.zeros(3), np.zeros(3))
    assert E["nl"] == pytest.approx(2.0 * D0 * b2, rel=1e-12)
