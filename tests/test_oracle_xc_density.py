"""Pins for the locally collinear LSDA and the spin-density bookkeeping (CPU only)."""
import math

import numpy as np
import pytest

from oracle import xc
from oracle.tddft import PAULI, System


def test_pw92_table_internal_relations():
    """PW92 rows satisfy beta2 = 2 A beta1^2, and A is the exact high-density coefficient:
    (1 - ln 2)/pi^2 for zeta = 0, half of it for zeta = 1, 1/(6 pi^2) for -alpha_c; f''(0) closed form."""
    for row in (xc.PW92_EC0, xc.PW92_EC1, xc.PW92_MAC):
        A, a1, b1, b2, b3, b4 = row
        assert b2 == pytest.approx(2 * A * b1 * b1, rel=2e-4)
    a0 = (1 - math.log(2)) / math.pi ** 2
    assert xc.PW92_EC0[0] == pytest.approx(a0, rel=1e-4)
    assert xc.PW92_EC1[0] == pytest.approx(a0 / 2, rel=1e-4)
    assert xc.PW92_MAC[0] == pytest.approx(1 / (6 * math.pi ** 2), rel=1e-4)
    assert xc.FPP0 == pytest.approx(8 / (9 * (2 ** (4 / 3) - 2)), rel=1e-6)


def test_pw92_high_density_limit():
    """eps_c -> A ln rs + const as rs -> 0: slope of eps_c vs ln rs tends to A."""
    for row, z in ((xc.PW92_EC0, 0.0), (xc.PW92_EC1, 1.0)):
        rs = np.array([1e-6, 2e-6])
        ec, _, _ = xc.pw92_correlation(rs, np.array([z, z]))
        slope = (ec[1] - ec[0]) / math.log(2)
        assert slope == pytest.approx(row[0], rel=2e-2)


@pytest.mark.parametrize("nu,nd", [(0.3, 0.1), (0.02, 0.05), (1.5, 1.5), (0.7, 0.0), (1e-3, 4e-4)])
def test_lsda_potentials_are_energy_derivatives(nu, nd):
    """v_sigma = d(n eps_xc)/d n_sigma by central finite differences."""
    e, vu, vd = xc.lsda(nu, nd)
    h = 1e-6 * (nu + nd)
    if nd > 0:
        fd_d = (xc.lsda(nu, nd + h)[0] - xc.lsda(nu, nd - h)[0]) / (2 * h)
        assert vd == pytest.approx(fd_d, rel=1e-7)
    fd_u = (xc.lsda(nu + h, nd)[0] - xc.lsda(nu - h, nd)[0]) / (2 * h)
    assert vu == pytest.approx(fd_u, rel=1e-7)


def test_slater_spin_scaling():
    """Exchange energy of a fully polarised gas is 2^(1/3) times the unpolarised one at equal n."""
    n = 0.37
    cx = 0.75 * (3 / math.pi) ** (1 / 3)
    ex_unpol = -cx * n ** (4 / 3)
    ex_pol = -0.75 * (6 / math.pi) ** (1 / 3) * n ** (4 / 3)
    assert ex_pol / ex_unpol == pytest.approx(2 ** (1 / 3))
    # unpolarised: v_up = v_dn and exchange part equals the textbook -(3 n / pi)^(1/3)
    e, vu, vd = xc.lsda(n / 2, n / 2)
    assert vu == pytest.approx(vd)
    ec, drs, _ = xc.pw92_correlation(np.array([(3 / (4 * math.pi * n)) ** (1 / 3)]), np.array([0.0]))
    assert e == pytest.approx(ex_unpol + n * ec[0], rel=1e-12)


def test_noncollinear_xc_zero_torque_and_collinear_limit():
    rng = np.random.default_rng(3)
    n = rng.uniform(0.01, 1.0, size=50)
    mdir = rng.normal(size=(3, 50))
    mdir /= np.linalg.norm(mdir, axis=0)
    m = mdir * n * rng.uniform(0, 0.9, size=50)
    e, vbar, b = xc.noncollinear_xc(n, m)
    assert np.allclose(np.cross(b.T, m.T), 0, atol=1e-15)  # local zero torque (Eq. spincont2)
    # collinear limit: m along +-z, V_up = v_up^LSDA(n_up, n_dn), V_dn = v_dn^LSDA
    for sgn in (1.0, -1.0):
        mz = sgn * n * 0.4
        e, vbar, b = xc.noncollinear_xc(n, np.stack([0 * n, 0 * n, mz]))
        nu, nd = 0.5 * (n + mz), 0.5 * (n - mz)
        e2, vu, vd = xc.lsda(nu, nd)
        assert np.allclose(vbar + b[2], vu, atol=1e-14)
        assert np.allclose(vbar - b[2], vd, atol=1e-14)
        assert np.allclose(e, e2, atol=1e-14)
    # thresholds: n below threshold gives zeros; |m| = 0 gives b = 0
    e, vbar, b = xc.noncollinear_xc(np.array([1e-15, 0.5]), np.zeros((3, 2)))
    assert e[0] == 0 and vbar[0] == 0 and np.all(b == 0)


def test_rho_v_and_magnetisation_identities():
    """m = Tr(sigma rho_s), n = Tr rho_s (Eqs. rho1-rho3) and the initial-density formula of Algorithm 1
    rho_v = n {(1+m_z)/2, (1-m_z)/2, m_x/2, -m_y/2} with m = M/n round-trips to (n, M)."""
    rng = np.random.default_rng(1)
    psi = rng.normal(size=(1, 3, 2, 4, 4, 4)) + 1j * rng.normal(size=(1, 3, 2, 4, 4, 4))
    occ = np.array([[1.0, 0.5, 0.25]])
    s = System.__new__(System)
    s.kw = np.ones(1)
    s.occ = occ
    rho = System.rho_v(s, psi)
    n, m = System.n_m(rho)
    rho_s = np.einsum("i,iazyx,ibzyx->abzyx", occ[0], psi[0], psi[0].conj())
    assert np.allclose(n, np.einsum("aazyx->zyx", rho_s).real)
    for a in range(3):
        assert np.allclose(m[a], np.einsum("ab,bazyx->zyx", PAULI[a], rho_s).real)
    # Algorithm 1 (ComputeSpinDensity) round trip
    M = m[:, 0, 0, 0]
    nn = n[0, 0, 0]
    mm = M / nn
    rv = nn * np.array([(1 + mm[2]) / 2, (1 - mm[2]) / 2, mm[0] / 2, -mm[1] / 2])
    n2, m2 = System.n_m(rv)
    assert n2 == pytest.approx(nn) and np.allclose(m2, M)


def test_voronoi_atom_moments_partition_the_totals():
    """Per-atom moments over nearest-atom cells (Algorithm 1's NearestAtom) add up to M and N;
    the ownership matches a brute-force nearest-atom search over all periodic images."""
    from tests._systems import parity_system
    wl, s, psi = parity_system(n=12, nstates=3, nk=1, natoms=3)
    rho = s.rho_v(psi)
    M, N = s.atom_moments(rho)
    n, m = System.n_m(rho)
    assert np.allclose(M.sum(axis=0), m.sum(axis=(1, 2, 3)) * s.grid.dV, atol=1e-13)
    assert N.sum() == pytest.approx(n.sum() * s.grid.dV, rel=1e-13)
    owner = s.voronoi_owner()
    r = s.grid.r.reshape(-1, 3)
    shifts = np.array([[i, j, k] for i in (-1, 0, 1) for j in (-1, 0, 1) for k in (-1, 0, 1)]) * s.grid.L
    dist = np.stack([np.min(np.linalg.norm(r[:, None, :] - (R + shifts)[None], axis=2), axis=1) for R in s.pos])
    assert np.all(dist[owner, np.arange(len(r))] <= dist.min(axis=0) + 1e-12)
