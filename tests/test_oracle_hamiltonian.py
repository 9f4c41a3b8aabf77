"""Pins for the oracle's Hamiltonian: Hermiticity, rotation symmetry, spin-rotation
invariance and the Zeeman splitting (CPU only)."""
import math

import numpy as np
import pytest
from scipy.linalg import expm

from oracle.tddft import MU_B, PAULI, System
from tests._systems import parity_system, uniform_gas


def test_hamiltonian_hermitian_with_soc_kpoints_and_fields():
    """<phi|H psi> = <H phi|psi> on random spinors (equivalently <phi|H psi> = <psi|H phi>*)."""
    wl, s, psi = parity_system(n=12, nstates=3, nk=2)
    rho = s.rho_v(psi)
    A, B = np.array([0.05, -0.1, 0.2]), np.array([0.3, 0.1, -0.2])
    V, _ = s.potential(rho, B)
    rng = np.random.default_rng(5)
    phi = rng.normal(size=psi.shape) + 1j * rng.normal(size=psi.shape)
    hp = s.apply_h(psi, V, A)
    hf = s.apply_h(phi, V, A)
    for ik in range(psi.shape[0]):
        for i in range(psi.shape[1]):
            a = np.vdot(phi[ik, i], hp[ik, i])
            b = np.vdot(hf[ik, i], psi[ik, i])
            assert abs(a - b) < 1e-12 * abs(a)


def _single_atom(n=16, lam=0.05, lmax=2):
    L = 8.0
    c = n // 2
    R = np.array([c, c, c]) * L / n
    return System([L] * 3, n, R[None], np.zeros(1, np.int32), [8.0], [0.8], [0.9], lmax,
                  np.array([[1.0, 0.5, 0.25][:lmax + 1]]), np.array([[0.0, lam, lam][:lmax + 1]]),
                  3.0, np.zeros((1, 3)), np.ones(1), np.ones((1, 2))), c


def _rotate_grid(f, c, axis):
    """(R f)(r) = f(R^-1 r) for +90 deg rotations about the atom at grid point (c,c,c)."""
    n = f.shape[-1]
    iz, iy, ix = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    X, Y, Z = ix - c, iy - c, iz - c
    if axis == "z":      # R^-1 (x,y,z) = (y,-x,z)
        sx, sy, sz = Y, -X, Z
    else:                # about x: R^-1 (x,y,z) = (x, z, -y)
        sx, sy, sz = X, Z, -Y
    return f[..., (sz + c) % n, (sy + c) % n, (sx + c) % n]


@pytest.mark.parametrize("axis", ["z", "x"])
def test_nonlocal_commutes_with_joint_space_spin_rotation(axis):
    """A 90-degree rotation of space together with the spinor rotation exp(-i pi/4 n.sigma) commutes
    with V_NL including L.S (J = L + S is conserved by one atom); space alone does not."""
    s, c = _single_atom()
    rng = np.random.default_rng(2)
    psi = rng.normal(size=(1, 2, 2, 16, 16, 16)) + 1j * rng.normal(size=(1, 2, 2, 16, 16, 16))
    nvec = np.array([0, 0, 1.0]) if axis == "z" else np.array([1.0, 0, 0])
    Us = expm(-1j * math.pi / 4 * np.einsum("a,aij->ij", nvec, PAULI))
    rot = lambda p: np.einsum("st,kbtzyx->kbszyx", Us, _rotate_grid(p, c, axis))  # noqa: E731
    zero = np.zeros(3)
    lhs = s.apply_nonlocal(rot(psi)[0], zero)
    rhs = rot(s.apply_nonlocal(psi[0], zero)[None])[0]
    assert np.abs(lhs - rhs).max() < 1e-13 * np.abs(rhs).max()
    # spatial rotation alone must fail when SOC is on
    rot_sp = lambda p: _rotate_grid(p, c, axis)  # noqa: E731
    bad = np.abs(s.apply_nonlocal(rot_sp(psi)[0], zero) - rot_sp(s.apply_nonlocal(psi[0], zero)[None])[0]).max()
    assert bad > 1e-4 * np.abs(rhs).max()


def test_global_spin_rotation_invariance_without_soc():
    """Without SOC and B: n invariant, m rotated by the SO(3) image of U, every energy term invariant."""
    wl, s, psi = parity_system(n=12, nstates=3, nk=1, lam=0.0)
    U = expm(-1j * 0.7 * np.einsum("a,aij->ij", np.array([0.3, -0.5, 0.81]) / 1.0, PAULI))
    R = np.array([[0.5 * np.trace(PAULI[a] @ U @ PAULI[b] @ U.conj().T).real for b in range(3)]
                  for a in range(3)])
    psi_r = np.einsum("st,kbtzyx->kbszyx", U, psi)
    A = np.array([0.1, 0.0, -0.05])
    zeroB = np.zeros(3)
    out = []
    for p in (psi, psi_r):
        rho = s.rho_v(p)
        V, parts = s.potential(rho, zeroB)
        out.append((parts, s.energies(p, rho, V, parts, A, zeroB)))
    (p0, e0), (p1, e1) = out
    assert np.allclose(p0["n"], p1["n"], atol=1e-13)
    assert np.allclose(np.einsum("ab,bzyx->azyx", R, p0["m"]), p1["m"], atol=1e-12)
    for key in ("kin", "nl", "loc", "H", "xc", "total"):
        assert e1[key] == pytest.approx(e0[key], rel=1e-12, abs=1e-13)


def test_zeeman_splitting_uniform_gas():
    """Spin-up/down splitting along B equals 2 mu_B |B| (tables of Zeeman splittings, Sec. 4.2)."""
    s, psi = uniform_gas(nstates=1, xc=0)
    B = np.array([0.2, -0.1, 0.35])
    V, _ = s.potential(s.rho_v(psi), B)
    bh = B / np.linalg.norm(B)
    w, vec = np.linalg.eigh(np.einsum("a,aij->ij", bh, PAULI))
    pw = psi[0, 0, 0] / np.abs(psi[0, 0, 0]).max()
    E = []
    for j in range(2):
        p = psi.copy()
        p[0, 0, 0] = vec[0, j] * pw
        p[0, 0, 1] = vec[1, j] * pw
        nrm = np.vdot(p, p).real * s.grid.dV
        E.append((np.vdot(p, s.apply_h(p, V, np.zeros(3))) * s.grid.dV / nrm).real)
    assert E[1] - E[0] == pytest.approx(2 * MU_B * np.linalg.norm(B), rel=1e-12)


def test_spectral_window_contains_the_exact_spectrum():
    """The non-local bound dominates ||V_NL|| and the window of reading P2 contains every
    eigenvalue of H (dense, tiny system with overlapping SOC projectors of two atoms)."""
    from tests._systems import parity_system
    wl, s, psi = parity_system(n=8, nstates=1, nk=1, lam=0.3, natoms=2)
    s.pos[1] = s.pos[0] + np.array([1.5, 0.7, -0.9])  # strongly overlapping projector spheres
    s.__init__(wl.L, wl.n, s.pos, wl.species, wl.Z, wl.rc_loc, wl.width, wl.lmax, wl.D, wl.lam,
               wl.r_cut, wl.kpts, wl.kw, wl.occ)
    A = np.array([0.1, -0.2, 0.05])
    V, _ = s.potential(s.rho_v(psi), [0.05, 0.0, 0.1])
    shape = psi.shape
    nvec = int(np.prod(shape))
    H = np.empty((nvec, nvec), np.complex128)
    NL = np.empty((nvec, nvec), np.complex128)
    e = np.zeros(nvec, np.complex128)
    for j in range(nvec):
        e[j] = 1.0
        x = e.reshape(shape)
        H[:, j] = s.apply_h(x, V, A).reshape(-1)
        NL[:, j] = s.apply_nonlocal(x[0], wl.kpts[0] + A).reshape(-1)
        e[j] = 0.0
    nl_norm = np.abs(np.linalg.eigvalsh(0.5 * (NL + NL.conj().T))).max()
    bound = s.nl_norm_bound()
    assert nl_norm <= bound
    assert bound <= 4.0 * nl_norm  # and is not loose by more than a small factor here
    ev = np.linalg.eigvalsh(0.5 * (H + H.conj().T))
    lo, hi = s.spectral_bounds(V, [A], margin=0.0)
    assert lo <= ev.min() and ev.max() <= hi


def test_zeeman_splitting_matches_the_papers_table():
    """Lowest eigenvalue of each spin channel of an atom's Hamiltonian (local pseudopotential, no
    SOC, no XC, static B along z) against the paper's printed Zeeman splittings of the H 1s level
    (tests/golden/zeeman_splitting_h_1s.txt): b_ext is the Zeeman energy mu_B B of one spin
    state, so B = b_ext / mu_B and the splitting is 2 b_ext."""
    import os
    from scipy.sparse.linalg import LinearOperator, eigsh
    from tests._systems import parity_system
    rows = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "zeeman_splitting_h_1s.txt"))
    wl, s, psi = parity_system(n=12, nstates=1, nk=1, lam=0.0, natoms=1)
    s.xc = 0
    ev = 27.211386245988  # eV per hartree
    n3 = s.grid.n ** 3
    for b_ev, split_ev in rows:
        B = np.array([0.0, 0.0, b_ev / ev / MU_B])
        V, _ = s.potential(np.zeros((4,) + (s.grid.n,) * 3), B)
        lows = []
        for spin in (0, 1):
            def mv(x, spin=spin):
                p = np.zeros(psi.shape, np.complex128)
                p[0, 0, spin] = x.reshape((s.grid.n,) * 3)
                return s.apply_h(p, V, np.zeros(3))[0, 0, spin].reshape(-1)
            op = LinearOperator((n3, n3), matvec=mv, dtype=np.complex128)
            w = eigsh(op, k=1, which="SA", tol=1e-12, v0=np.ones(n3, np.complex128))[0]
            lows.append(w[0])
        assert (lows[0] - lows[1]) * ev == pytest.approx(split_ev, abs=5e-5)

