"""Pins for the oracle's grid, FFT, kinetic, local and Hartree potentials (CPU only)."""
import math

import numpy as np
import pytest
from scipy import integrate, special

from oracle.tddft import Grid, hartree_potential, local_potential


@pytest.mark.parametrize("n", [6, 8, 12])
def test_fft_matches_bruteforce_dft(n):
    """Forward transform = sum_r f(r) exp(-i G.r) on the oracle's own G mesh (brute force O(N^2))."""
    g = Grid([7.0, 8.0, 9.0], n)
    rng = np.random.default_rng(n)
    f = rng.normal(size=(n, n, n)) + 1j * rng.normal(size=(n, n, n))
    r = g.r.reshape(-1, 3)
    G = g.G.reshape(-1, 3)
    dft = np.exp(-1j * G @ r.T) @ f.reshape(-1)
    assert np.allclose(g.fft(f).reshape(-1), dft, rtol=0, atol=1e-11 * np.abs(dft).max())
    back = (np.exp(1j * r @ G.T) @ dft) / g.N
    assert np.allclose(g.ifft(g.fft(f)).reshape(-1), back, atol=1e-12)
    # Nyquist index is negative (-n/2) on the mesh
    if n % 2 == 0:
        assert g.G[0, 0, n // 2, 0] == pytest.approx(-math.pi * n / 7.0)


def test_kinetic_on_plane_wave_is_exact():
    g = Grid([6.0, 7.0, 8.0], 12)
    shift = np.array([0.1, -0.2, 0.35])
    for idx in [(1, 2, 3), (0, 0, 6), (5, 11, 7)]:
        G0 = g.G[idx]
        pw = np.exp(1j * (g.r @ G0))
        out = np.fft.ifftn(g.kinetic(shift) * np.fft.fftn(pw))
        expect = 0.5 * np.sum((G0 + shift) ** 2)
        assert np.allclose(out, expect * pw, atol=1e-10)


def _erf_coulomb_ft(G, Z, rc):
    """Fourier transform of -Z erf(r/rc)/r by radial quadrature of its short-range part
    (the -Z/r part transforms to -4 pi Z / G^2)."""
    f = lambda r: r * special.erfc(r / rc) * (math.sin(G * r) / (G * r) if G * r > 0 else 1.0)  # noqa: E731
    val, _ = integrate.quad(f, 0.0, 12.0 * rc, limit=200, epsabs=1e-14)
    sr = 4.0 * math.pi * Z * val
    return sr if G == 0 else -4.0 * math.pi * Z / G ** 2 + sr


def test_local_potential_fourier_coefficients_match_quadrature():
    """Fourier coefficients of V_loc on the grid equal the radial-quadrature transform of
    -Z erf(r/rc)/r divided by the cell volume (G = 0 keeps only the non-Coulomb part)."""
    g = Grid([11.0, 11.0, 11.0], 16)
    R = np.array([2.0, 3.5, 5.0])
    Z, rc = 8.0, 0.8
    V = local_potential(g, [R], [Z], [rc])
    VG = np.fft.fftn(V) / g.N * g.omega
    for idx in [(0, 0, 0), (0, 0, 1), (1, 2, 3), (3, 1, 5), (7, 2, 2)]:
        G = g.G[idx]
        Gn = math.sqrt(float(np.sum(G * G)))
        expect = _erf_coulomb_ft(Gn, Z, rc) * np.exp(-1j * G @ R)
        assert abs(VG[idx] - expect) < 1e-8 * max(1.0, abs(expect))


def test_local_potential_near_atom_real_space():
    """Single atom in a large box: V(r) - V(0) = -Z [erf(r/rc)/r - 2/(sqrt(pi) rc)] - (2 pi/3)(Z/Omega) r^2
    near the atom (the quadratic term is the uniform compensating background)."""
    L = 30.0
    n = 96
    g = Grid([L, L, L], n)
    R = np.array([15.0, 15.0, 15.0])
    Z, rc = 8.0, 0.8
    V = local_potential(g, [R], [Z], [rc])
    c = n // 2
    v0 = V[c, c, c]
    for dx in [2, 4, 7, 9]:
        r = dx * L / n
        expect = -Z * (special.erf(r / rc) / r - 2.0 / (math.sqrt(math.pi) * rc)) \
            - 2.0 * math.pi / 3.0 * Z / L ** 3 * r * r
        assert V[c, c, c + dx] - v0 == pytest.approx(expect, abs=2e-4)


def test_hartree_of_gaussian_charge():
    """v_H of a normalised Gaussian charge Q: Q [erf(r/(sqrt2 s))/r - sqrt(2/pi)/s] + (2 pi/3)(Q/Omega) r^2
    relative to the centre, and zero mean (G = 0 dropped)."""
    L = 30.0
    n = 96
    g = Grid([L, L, L], n)
    s, Q = 1.0, 3.0
    d = g.r - 15.0
    r2 = (d * d).sum(-1)
    rho = Q * (2 * math.pi * s * s) ** -1.5 * np.exp(-r2 / (2 * s * s))
    vH = hartree_potential(g, rho)
    assert abs(vH.mean()) < 1e-12
    c = n // 2
    for dx in [2, 4, 7, 9]:
        r = dx * L / n
        expect = Q * (special.erf(r / (math.sqrt(2) * s)) / r - math.sqrt(2 / math.pi) / s) \
            + 2.0 * math.pi / 3.0 * Q / L ** 3 * r * r
        assert vH[c, c, c + dx] - vH[c, c, c] == pytest.approx(expect, abs=6e-5)
