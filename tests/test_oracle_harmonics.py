"""Pins for real harmonics, angular momentum, the L.S block and the spinor-harmonic
KB form (Eq. Vps with the spinor spherical harmonics of Sec. 3.5)."""
import math

import numpy as np
import pytest
from scipy import integrate, special

from oracle.tddft import (PAULI, angular_momentum_complex, angular_momentum_real, complex_to_real,
                          radial_norm, real_ylm, soc_block)


def _sphere_quadrature(nt=24, nphi=48):
    x, w = np.polynomial.legendre.leggauss(nt)
    phi = np.arange(nphi) * 2 * math.pi / nphi
    ct, ph = np.meshgrid(x, phi, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    pts = np.stack([st * np.cos(ph), st * np.sin(ph), ct], axis=-1).reshape(-1, 3)
    wts = (w[:, None] * np.full(nphi, 2 * math.pi / nphi)[None, :]).reshape(-1)
    return pts, wts


@pytest.mark.parametrize("l", [0, 1, 2, 3])
def test_real_ylm_orthonormal(l):
    pts, wts = _sphere_quadrature()
    Y = real_ylm(l, pts)
    S = (Y * wts) @ Y.T
    assert np.allclose(S, np.eye(2 * l + 1), atol=1e-13)


def test_real_ylm_explicit_forms():
    """l = 1 ordering (y, z, x) and l = 2 forms with textbook prefactors."""
    rng = np.random.default_rng(0)
    d = rng.normal(size=(20, 3))
    r = np.linalg.norm(d, axis=1)
    x, y, z = (d / r[:, None]).T
    c1 = math.sqrt(3 / (4 * math.pi))
    assert np.allclose(real_ylm(1, d), c1 * np.stack([y, z, x]), atol=1e-14)
    c2 = 0.5 * math.sqrt(15 / math.pi)
    expect = np.stack([c2 * x * y, c2 * y * z, 0.25 * math.sqrt(5 / math.pi) * (3 * z * z - 1),
                       c2 * x * z, 0.5 * c2 * (x * x - y * y)])
    assert np.allclose(real_ylm(2, d), expect, atol=1e-14)
    assert np.allclose(real_ylm(0, d), 0.5 / math.sqrt(math.pi))


@pytest.mark.parametrize("l", [1, 2, 3])
def test_angular_momentum_real_matches_differential_operator(l):
    """(L_a y_nu)(p) = sum_mu y_mu(p) L[mu, nu] with L = -i r x grad applied by finite differences
    to the solid harmonics r^l y_nu (pins the complex-to-real transform and its conventions)."""
    Lr = angular_momentum_real(l)
    rng = np.random.default_rng(l)
    p = rng.normal(size=(15, 3))
    p /= np.linalg.norm(p, axis=1)[:, None]
    f = lambda q: np.linalg.norm(q, axis=1)[None, :] ** l * real_ylm(l, q)  # noqa: E731
    h = 1e-5
    grad = []
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        grad.append((f(p + e) - f(p - e)) / (2 * h))
    grad = np.array(grad)  # [axis][nu][pt]
    for a in range(3):
        b, c = (a + 1) % 3, (a + 2) % 3
        La_f = -1j * (p[:, b][None, :] * grad[c] - p[:, c][None, :] * grad[b])
        expect = np.einsum("mp,mn->np", f(p), Lr[a])
        assert np.allclose(La_f, expect, atol=1e-8)


@pytest.mark.parametrize("l", [1, 2, 3])
def test_angular_momentum_algebra(l):
    Lc = angular_momentum_complex(l)
    for L in (Lc, angular_momentum_real(l)):
        assert np.allclose(L[0] @ L[1] - L[1] @ L[0], 1j * L[2], atol=1e-13)
        L2 = sum(La @ La for La in L)
        assert np.allclose(L2, l * (l + 1) * np.eye(2 * l + 1), atol=1e-13)
    U = complex_to_real(l)
    assert np.allclose(U @ U.conj().T, np.eye(2 * l + 1), atol=1e-14)


@pytest.mark.parametrize("l", [0, 1, 2])
def test_soc_block_spectrum_and_rotation_invariance(l):
    """Spectrum {D + lam l/2 (x 2l+2), D - lam (l+1)/2 (x 2l)} and [D, J] = 0, J = L + S."""
    Dl, lam = 0.5, 0.02
    D = soc_block(l, Dl, lam)
    assert np.allclose(D, D.conj().T)
    ev = np.sort(np.linalg.eigvalsh(D))
    expect = np.sort([Dl + lam * l / 2] * (2 * l + 2) + [Dl - lam * (l + 1) / 2] * (2 * l))
    assert np.allclose(ev, expect, atol=1e-14)
    Lr = angular_momentum_real(l)
    for a in range(3):
        J = np.kron(Lr[a], np.eye(2)) + np.kron(np.eye(2 * l + 1), PAULI[a] / 2)
        assert np.allclose(D @ J - J @ D, 0, atol=1e-14)


def _spinor_harmonic_coeffs(l, j_plus, mj2):
    """Coefficients of Phi_{l,j}^{m_j} on Y_l^{m} chi_sigma in the complex basis, from the
    spinor spherical-harmonic formula of Sec. 3.5 (upper sign j = l + 1/2 with m = m_j - 1/2,
    lower sign j = l - 1/2 with m = m_j + 1/2); mj2 = 2 m_j."""
    v = np.zeros((2 * l + 1, 2), np.complex128)
    if j_plus:
        m = (mj2 - 1) // 2
        a = math.sqrt((l + m + 1) / (2 * l + 1))
        b = math.sqrt((l - m) / (2 * l + 1))
    else:
        m = (mj2 + 1) // 2
        a = math.sqrt((l - m + 1) / (2 * l + 1))
        b = -math.sqrt((l + m) / (2 * l + 1))
    up_m, dn_m = (mj2 - 1) // 2, (mj2 + 1) // 2
    if -l <= up_m <= l:
        v[up_m + l, 0] = a
    if -l <= dn_m <= l:
        v[dn_m + l, 1] = b
    return v


@pytest.mark.parametrize("l", [1, 2])
def test_ls_form_equals_spinor_harmonic_kb_form(l):
    """sum_j D_{l,j} sum_mj |Phi_lj^mj><Phi_lj^mj| (Eq. Vps with spinor harmonics) equals
    D_l + lam_l L.S when D_{l, l+1/2} - D_{l, l-1/2} = lam (2l+1)/2 (Eq. Vps-soc), after the
    transform to the real-harmonic basis."""
    Dl, lam = 0.5, 0.03
    Dp, Dm = Dl + lam * l / 2, Dl - lam * (l + 1) / 2
    assert Dp - Dm == pytest.approx(lam * (2 * l + 1) / 2)
    P = {True: np.zeros((2 * (2 * l + 1),) * 2, np.complex128), False: None}
    P[False] = np.zeros_like(P[True])
    for jp in (True, False):
        j2 = 2 * l + (1 if jp else -1)
        for mj2 in range(-j2, j2 + 1, 2):
            v = _spinor_harmonic_coeffs(l, jp, mj2).reshape(-1)
            assert np.vdot(v, v).real == pytest.approx(1.0)
            P[jp] += np.outer(v, v.conj())
    assert np.allclose(P[True] + P[False], np.eye(2 * (2 * l + 1)), atol=1e-14)
    Uk = np.kron(complex_to_real(l), np.eye(2))
    M_real = Uk.conj() @ (Dp * P[True] + Dm * P[False]) @ Uk.T
    assert np.allclose(M_real, soc_block(l, Dl, lam), atol=1e-14)


@pytest.mark.parametrize("l", [0, 1, 2])
def test_radial_normalisation(l):
    w = 1.3
    N = radial_norm(l, w)
    val, _ = integrate.quad(lambda r: (N * r ** l * math.exp(-r * r / (2 * w * w))) ** 2 * r * r, 0, 40)
    assert val == pytest.approx(1.0, abs=1e-12)


def test_sph_harm_condon_shortley():
    th, ph = 0.7, 0.3
    assert special.sph_harm_y(1, 1, th, ph) == pytest.approx(
        -math.sqrt(3 / (8 * math.pi)) * math.sin(th) * np.exp(1j * ph))
