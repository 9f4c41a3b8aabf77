"""Pins for the oracle's propagator: Chebyshev exponential, norm, time reversibility,
Larmor precession, spin conservation without SOC, second-order convergence and the
collinear limit (CPU only)."""
import math

import numpy as np
import pytest
from scipy.linalg import expm

from oracle import xc as oxc
from oracle.tddft import (MU_B, chebyshev_order, exp_chebyshev, exp_taylor)
from paper_2506_21908_gb300 import synthetic as S
from tests._systems import make_oracle, parity_system, rotate, uniform_gas


def test_chebyshev_exponential_matches_expm():
    rng = np.random.default_rng(0)
    X = rng.normal(size=(30, 30)) + 1j * rng.normal(size=(30, 30))
    H = 0.5 * (X + X.conj().T)
    ev = np.linalg.eigvalsh(H)
    emin, emax = ev[0] - 0.3, ev[-1] + 0.2
    v = rng.normal(size=30) + 1j * rng.normal(size=30)
    for tau in (0.05, -0.3, 1.1):
        K = chebyshev_order(tau * 0.5 * (emax - emin))
        got = exp_chebyshev(lambda x: H @ x, v, tau, emin, emax, K)
        assert np.allclose(got, expm(-1j * tau * H) @ v, atol=1e-13 * np.abs(v).max())
    tau = 0.01
    got = exp_taylor(lambda x: H @ x, v, tau, 12)
    assert np.allclose(got, expm(-1j * tau * H) @ v, atol=1e-13 * np.abs(v).max())


def test_norm_conservation_and_n_electrons():
    wl, s, psi = parity_system(n=12, nstates=3, nk=2)
    o = make_oracle(s, psi, wl.times, wl.A, wl.B, wl.dt)
    for _ in range(3):
        o.step()
    n, m, E, norms = o.observables()
    assert np.allclose(norms, 1.0, atol=1e-12)
    assert E["N"] == pytest.approx((wl.kw[:, None] * wl.occ).sum(), rel=1e-12)


def test_time_reversibility_with_converged_self_consistency():
    wl, s, psi = parity_system(n=12, nstates=3, nk=1)
    kw = dict(n_sc=60, sc_tol=1e-14)
    o = make_oracle(s, psi, wl.times, wl.A, wl.B, wl.dt, **kw)
    for _ in range(2):
        o.step()
    assert np.abs(o.psi - psi).max() > 1e-3
    o.dt = -o.dt
    for _ in range(2):
        o.step()
    assert abs(o.t) < 1e-14
    assert np.abs(o.psi - psi).max() < 1e-10 * np.abs(psi).max()


def test_larmor_precession_uniform_gas_closed_form():
    """Uniform gas in a static uniform B without XC torque: M precesses about B at
    omega = 2 mu_B |B| (Eq. magrot / Eq. MOmega) exactly."""
    s, psi = uniform_gas(nstates=3, xc=0)
    B = np.array([0.4, 0.0, 0.3])
    times, A, Bt = S.zero_fields(10, 0.1)
    Bt[:] = B
    o = make_oracle(s, psi, times, A, Bt, 0.1)
    M0 = o.observables()[2]["M"]
    for k in range(1, 9):
        o.step()
        M = o.observables()[2]["M"]
        expect = rotate(M0, B, 2 * MU_B * np.linalg.norm(B) * k * 0.1)
        assert np.allclose(M, expect, atol=1e-11)


def test_larmor_with_xc_converges_second_order():
    """With the XC field on, the uniform gas still precesses at 2 mu_B |B| (zero torque); the ETRS
    error against the closed form falls as dt^2."""
    B = np.array([0.0, 0.5, 0.0])
    errs = []
    T = 1.2
    for dt in (0.2, 0.1, 0.05):
        s, psi = uniform_gas(nstates=3, xc=1)
        nst = int(round(T / dt))
        times, A, Bt = S.zero_fields(nst, dt)
        Bt[:] = B
        o = make_oracle(s, psi, times, A, Bt, dt, n_sc=30, sc_tol=1e-14)
        M0 = o.observables()[2]["M"]
        for _ in range(nst):
            o.step()
        M = o.observables()[2]["M"]
        errs.append(np.linalg.norm(M - rotate(M0, B, np.linalg.norm(B) * T)))
    assert errs[0] < 1e-2
    assert errs[0] / errs[1] == pytest.approx(4.0, rel=0.1)
    assert errs[1] / errs[2] == pytest.approx(4.0, rel=0.1)


def test_laser_without_soc_leaves_magnetisation_constant():
    """Without SOC and XC torque a laser cannot change M: the Hamiltonian is spin independent."""
    wl, s, psi = parity_system(n=12, nstates=3, nk=1, lam=0.0, xc=0)
    wl.B[:] = 0.0
    o = make_oracle(s, psi, wl.times, wl.A, wl.B, wl.dt)
    M0 = o.observables()[2]["M"]
    for _ in range(3):
        o.step()
    assert np.allclose(o.observables()[2]["M"], M0, atol=1e-12)


def test_etrs_is_second_order():
    wl, s, psi = parity_system(n=12, nstates=2, nk=1)
    T = 0.4
    finals = []
    for nst in (4, 8, 16):
        dt = T / nst
        times = np.arange(nst + 1) * dt
        A = np.outer(times, [0.2, 0.0, -0.1])
        B = np.tile([0.05, 0.0, 0.02], (nst + 1, 1))
        o = make_oracle(s, psi, times, A, B, dt, n_sc=20, sc_tol=1e-14)
        for _ in range(nst):
            o.step()
        finals.append(o.psi)
    e1 = np.abs(finals[0] - finals[1]).max()
    e2 = np.abs(finals[1] - finals[2]).max()
    assert e1 / e2 == pytest.approx(4.0, rel=0.15)


def test_collinear_limit_equals_two_decoupled_lsda_channels():
    """Spinors purely up or down, no SOC, B along z: the non-collinear step reproduces a scalar
    collinear-LSDA propagation of the two spin channels (Eq. SDFT / Eq. HSDFT), written here
    independently with v_sigma = v^LSDA_sigma(n_up, n_dn) + (-1)^sigma mu_B B_z."""
    wl, s, psi = parity_system(n=12, nstates=4, nk=1, lam=0.0)
    psi = psi.copy()
    spins = [0, 1, 0, 0]
    for i, sg in enumerate(spins):
        psi[0, i, 1 - sg] = 0.0
        psi[0, i, sg] /= math.sqrt(np.vdot(psi[0, i, sg], psi[0, i, sg]).real * s.grid.dV)
    nst = 2
    dt = 0.05
    times = np.arange(nst + 1) * dt
    A = np.outer(times, [0.3, 0.1, 0.0])
    B = np.tile([0.0, 0.0, 0.2], (nst + 1, 1))
    o = make_oracle(s, psi, times, A, B, dt, n_sc=1)
    emin, emax, Kf, Kh = o.emin, o.emax, o.K_full, o.K_half
    for _ in range(nst):
        o.step()

    # scalar reference
    from oracle.tddft import hartree_potential
    occ = wl.occ[0]
    phis = [psi[0, i, sg].copy() for i, sg in enumerate(spins)]

    def chan_pots(ph, Bz):
        nu = sum(occ[i] * np.abs(p) ** 2 for i, (p, sg) in enumerate(zip(ph, spins)) if sg == 0)
        nd = sum(occ[i] * np.abs(p) ** 2 for i, (p, sg) in enumerate(zip(ph, spins)) if sg == 1)
        vH = hartree_potential(s.grid, nu + nd)
        _, vu, vd = oxc.lsda(nu, nd)
        return [s.vloc + vH + vu + MU_B * Bz, s.vloc + vH + vd - MU_B * Bz]

    def hs(p, v, Avec, sg):
        spin = np.zeros((1, 2) + p.shape, np.complex128)
        spin[0, sg] = p
        shift = Avec
        kin = s.apply_kinetic(spin, shift)[0, sg]
        nl = s.apply_nonlocal(spin, shift)[0, sg]
        return kin + v * p + nl

    def expo(ph, pots, Avec, tau, K):
        return [exp_chebyshev(lambda x, sg=sg: hs(x, pots[sg], Avec, sg), p, tau, emin, emax, K)
                for p, sg in zip(ph, spins)]

    t = 0.0
    pots = chan_pots(phis, B[0, 2])
    for _ in range(nst):
        A0, A1 = A[int(round(t / dt))], A[int(round(t / dt)) + 1]
        pred = expo(phis, pots, A0, dt, Kf)
        pots1 = chan_pots(pred, B[0, 2])
        half = expo(phis, pots, A0, 0.5 * dt, Kh)
        new = expo(half, pots1, A1, 0.5 * dt, Kh)
        pots1 = chan_pots(new, B[0, 2])
        new = expo(half, pots1, A1, 0.5 * dt, Kh)
        phis = new
        pots = chan_pots(phis, B[0, 2])
        t += dt
    for i, sg in enumerate(spins):
        assert np.abs(o.psi[0, i, sg] - phis[i]).max() < 1e-12
        assert np.abs(o.psi[0, i, 1 - sg]).max() < 1e-14


def test_magnetic_pulse_uniform_gas_closed_form():
    """Uniform gas, XC off, the paper's magnetic pulse B(t) = b(t) eps (delta_B along eps): all
    H(t) commute, and the ETRS step is exact for the linearly interpolated field table, so M
    turns about eps by 2 mu_B times the trapezoidal integral of b over the table (Eq. magrot)."""
    s, psi = uniform_gas(nstates=3, xc=0)
    eps = np.array([1.0, 0.0, 1.0]) / math.sqrt(2.0)
    dt, nst = 0.1, 30
    times, A, Bt = S.magnetic_pulse_table(nst, dt, amp=0.6, eps=eps, omega0=2.0, t0=0.45, tau=0.8,
                                          phi=0.3, delta_B=0.2 * eps)
    b = Bt @ eps
    assert np.allclose(Bt, b[:, None] * eps[None, :], atol=1e-15)
    assert b[0] == 0.0 and b[5] != 0.0
    o = make_oracle(s, psi, times, A, Bt, dt)
    M0 = o.observables()[2]["M"]
    theta = 0.0
    for k in range(1, nst + 1):
        o.step()
        theta += 2 * MU_B * 0.5 * dt * (b[k - 1] + b[k])
        M = o.observables()[2]["M"]
        assert np.allclose(M, rotate(M0, eps, theta), atol=1e-11), k


def _dense_h(s, V, A, shape):
    """H as a dense matrix on a tiny system, column by column."""
    nvec = int(np.prod(shape))
    H = np.empty((nvec, nvec), np.complex128)
    e = np.zeros(nvec, np.complex128)
    for j in range(nvec):
        e[j] = 1.0
        H[:, j] = s.apply_h(e.reshape(shape), V, A).reshape(-1)
        e[j] = 0.0
    return H


def test_crank_nicolson_is_the_cayley_transform():
    """The oracle's Crank-Nicolson step equals (1 + i tau H/2)^{-1} (1 - i tau H/2) psi from a
    dense solve, is unitary, and differs from exp(-i tau H) psi by O(tau^3) per step."""
    from oracle.tddft import exp_crank_nicolson
    wl, s, psi = parity_system(n=6, nstates=1, nk=1, lam=0.2, natoms=1)
    A = np.array([0.1, -0.05, 0.02])
    V, _ = s.potential(s.rho_v(psi), [0.02, 0.0, 0.05])
    H = _dense_h(s, V, A, psi.shape)
    assert np.abs(H - H.conj().T).max() <= 1e-12 * np.abs(H).max()
    I = np.eye(H.shape[0])
    x = psi.reshape(-1)
    err = {}
    for tau in (0.04, 0.02):
        cn = exp_crank_nicolson(lambda y: s.apply_h(y, V, A), psi, tau).reshape(-1)
        ref = np.linalg.solve(I + 0.5j * tau * H, (I - 0.5j * tau * H) @ x)
        assert np.abs(cn - ref).max() <= 1e-11 * np.abs(ref).max()
        assert abs(np.vdot(cn, cn).real - np.vdot(x, x).real) <= 1e-11 * np.vdot(x, x).real
        err[tau] = np.abs(cn - expm(-1j * tau * H) @ x).max()
    assert 7.0 < err[0.04] / err[0.02] < 9.0
