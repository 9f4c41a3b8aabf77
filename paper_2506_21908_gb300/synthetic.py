"""Seeded synthetic workloads for the spinor real-time propagation step.

This module only builds inputs: cell, grid, atoms, projector constants,
k-points, occupations, field tables and initial spinors.  It holds none of
the propagation arithmetic, so both the CUDA library and the FP64 oracle can
be fed the very same arrays.

Workloads stand in for the paper's systems (Fe2/Fe6 clusters and bcc Fe
supercells, Sec. 4), which need pseudopotential files that are not
available: synthetic Z=8 atoms with an erf-screened local potential,
Gaussian Kleinman-Bylander projectors (Eq. Vps) and an L.S coupling of
0.02 Ha (Eq. Vps-soc).

Array conventions (shared by every consumer):
  * grid arrays are indexed [z][y][x] (x fastest); r = (x*hx, y*hy, z*hz)
  * spinors are complex128 arrays [nk][nstates][2][nz][ny][nx], normalised
    with the grid inner product  <a|b> = sum_r conj(a) b dV
  * field tables hold A(t) and B(t) in atomic units at given times
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

FS_AU = 41.341373335  # atomic units of time per femtosecond
BOHR_PER_ANGSTROM = 1.0 / 0.529177210903


@dataclasses.dataclass
class Workload:
    name: str
    L: np.ndarray            # (3,) orthorhombic cell lengths, bohr
    n: int                   # grid points per axis (cubic grid)
    pos: np.ndarray          # (natoms, 3) bohr
    species: np.ndarray      # (natoms,) int32
    Z: np.ndarray            # (nspecies,)
    rc_loc: np.ndarray       # (nspecies,)  local potential -Z erf(r/rc)/r
    width: np.ndarray        # (nspecies,)  projector Gaussian width
    lmax: int
    D: np.ndarray            # (nspecies, lmax+1) Ha, KB channel energies
    lam: np.ndarray          # (nspecies, lmax+1) Ha, L.S coefficient
    r_cut: float
    kpts: np.ndarray         # (nk, 3) cartesian, 1/bohr
    kw: np.ndarray           # (nk,)
    occ: np.ndarray          # (nk, nstates)
    dt: float
    nsteps: int
    seed: int
    times: np.ndarray = None  # (nt,) field table times
    A: np.ndarray = None      # (nt, 3) vector potential
    B: np.ndarray = None      # (nt, 3) magnetic field
    xc: int = 1
    n_sc: int = 1
    exp_order: int = 0
    spin_mode: int = 0        # 0 non-collinear, 1 collinear (sigma_z only), 2 unpolarised

    @property
    def nk(self):
        return self.kpts.shape[0]

    @property
    def nstates(self):
        return self.occ.shape[1]

    @property
    def ng(self):
        return self.n ** 3

    @property
    def updates_per_step(self):
        """Spinor-grid-point updates per step: N_k * N_occ * N_g."""
        return self.nk * self.nstates * self.ng


# ----------------------------------------------------------------------------
# fields

def gauss_laser_E(t, E0, omega, t0, tau, pol):
    """E(t) = E0 pol cos(omega (t - t0)) exp(-(t-t0)^2 / (2 tau^2)) (Sec. 4.4 pulse form)."""
    t = np.asarray(t, dtype=np.float64)
    env = np.exp(-((t - t0) ** 2) / (2.0 * tau * tau))
    return (E0 * np.cos(omega * (t - t0)) * env)[..., None] * np.asarray(pol, np.float64)


def vector_potential_table(times, efield, nquad=16):
    """A(t) = -int_{t_0}^{t} E dt' on the given (sorted) times, Gauss-Legendre per interval."""
    x, w = np.polynomial.legendre.leggauss(nquad)
    A = np.zeros((len(times), 3))
    for i in range(1, len(times)):
        a, b = times[i - 1], times[i]
        tq = 0.5 * (b - a) * x + 0.5 * (b + a)
        integral = (0.5 * (b - a) * w[:, None] * efield(tq)).sum(axis=0)
        A[i] = A[i - 1] - integral
    return A


def laser_table(nsteps, dt, E0=0.01, omega=0.057, fwhm_fs=10.0, pol=(1.0, 0.0, 0.0),
                t0=None, B_static=(0.0, 0.0, 0.0)):
    """Field table at every step time for a Gaussian laser in velocity gauge.

    The FWHM refers to the field envelope; the pulse peak sits at the middle
    of the run unless t0 is given."""
    times = np.arange(nsteps + 1, dtype=np.float64) * dt
    tau = fwhm_fs * FS_AU / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    if t0 is None:
        t0 = 0.5 * nsteps * dt
    A = vector_potential_table(times, lambda t: gauss_laser_E(t, E0, omega, t0, tau, pol))
    B = np.tile(np.asarray(B_static, np.float64), (len(times), 1))
    return times, A, B


def magnetic_pulse_B(t, amp, eps, omega0, t0, tau, phi=0.0, delta_B=(0.0, 0.0, 0.0)):
    """Uniform magnetic pulse of the paper's magnetic-drive experiments:
    B(t) = amp eps [cos(omega0 (t - t0) + phi) exp(-(t - t0)^2 / (2 tau^2)) - 1] Theta(t - t0)
           + delta_B Theta(t - t0),
    with eps normalised to a unit vector and Theta(0) = 1."""
    t = np.asarray(t, dtype=np.float64)
    e = np.asarray(eps, np.float64)
    e = e / np.linalg.norm(e)
    step = (t >= t0).astype(np.float64)
    env = np.cos(omega0 * (t - t0) + phi) * np.exp(-((t - t0) ** 2) / (2.0 * tau * tau)) - 1.0
    return (amp * env * step)[..., None] * e + step[..., None] * np.asarray(delta_B, np.float64)


def magnetic_pulse_table(nsteps, dt, amp=0.01, eps=(1.0, 0.0, 1.0), omega0=0.05, t0=None, tau=20.0, phi=0.0,
                         delta_B=(0.0, 0.0, 0.0), A_table=None):
    """Field table at every step time for the magnetic pulse (no laser unless A_table is
    given); the pulse starts at a tenth of the run unless t0 is given."""
    times = np.arange(nsteps + 1, dtype=np.float64) * dt
    if t0 is None:
        t0 = 0.1 * nsteps * dt
    A = np.zeros((len(times), 3)) if A_table is None else np.asarray(A_table, np.float64)
    return times, A, magnetic_pulse_B(times, amp, eps, omega0, t0, tau, phi, delta_B)


def zero_fields(nsteps, dt):
    times = np.arange(nsteps + 1, dtype=np.float64) * dt
    return times, np.zeros((len(times), 3)), np.zeros((len(times), 3))


# ----------------------------------------------------------------------------
# geometry

def icosahedron(center, radius):
    """13-atom cluster: centre atom plus the 12 vertices of an icosahedron at the given radius."""
    phi = (1.0 + math.sqrt(5.0)) / 2.0
    v = []
    for a in (-1.0, 1.0):
        for b in (-phi, phi):
            v += [(0.0, a, b), (a, b, 0.0), (b, 0.0, a)]
    v = np.array(v)
    v *= radius / np.linalg.norm(v[0])
    return np.vstack([np.asarray(center)[None, :], np.asarray(center)[None, :] + v])


def bcc_supercell(a, reps, jitter=0.0, rng=None):
    pos = []
    for i in range(reps):
        for j in range(reps):
            for k in range(reps):
                base = np.array([i, j, k], dtype=np.float64) * a
                pos.append(base)
                pos.append(base + 0.5 * a)
    pos = np.array(pos)
    if jitter > 0.0:
        pos = pos + rng.normal(0.0, jitter, size=pos.shape)
    L = a * reps
    return np.mod(pos, L)


def min_image(d, L):
    return d - L * np.round(d / L)


def grid_coords(L, n):
    h = np.asarray(L, np.float64) / n
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    return np.stack([x * h[0], y * h[1], z * h[2]], axis=-1)  # [z][y][x][3]


# ----------------------------------------------------------------------------
# initial spinors

def _gram_schmidt(phis, dV):
    """Modified Gram-Schmidt in index order with the grid inner product."""
    out = []
    for p in phis:
        q = p.copy()
        for o in out:
            q = q - (np.vdot(o, q) * dV) * o
        q = q / math.sqrt((np.vdot(q, q).real) * dV)
        out.append(q)
    return np.array(out)


def random_tilted_states(L, n, nstates, seed, polar_deg=30.0):
    """Seeded complex Gaussian orbitals, orthonormalised, each times the spinor
    (cos(theta/2), sin(theta/2)) with the spin tilted polar_deg from z."""
    rng = np.random.default_rng(seed)
    dV = float(np.prod(L)) / n ** 3
    phis = rng.normal(size=(nstates, n, n, n)) + 1j * rng.normal(size=(nstates, n, n, n))
    phis = _gram_schmidt(phis.reshape(nstates, -1), dV).reshape(nstates, n, n, n)
    th = math.radians(polar_deg)
    chi = np.array([math.cos(th / 2.0), math.sin(th / 2.0)])
    psi = phis[:, None, :, :, :] * chi[None, :, None, None, None]
    return psi[None].astype(np.complex128)


def spinor_along(theta, phi, parallel=True):
    if parallel:
        return np.array([math.cos(theta / 2.0), np.exp(1j * phi) * math.sin(theta / 2.0)])
    return np.array([-np.exp(-1j * phi) * math.sin(theta / 2.0), math.cos(theta / 2.0)])


def lowdin(psi_k, dV):
    """Loewdin orthonormalisation of the rows of psi_k (nstates, npts)."""
    S = (psi_k.conj() @ psi_k.T) * dV
    w, U = np.linalg.eigh(S)
    Sm = (U * (1.0 / np.sqrt(w))) @ U.conj().T
    return Sm.T @ psi_k


# The 9 atomic basis functions as sums of separable terms c * d_x^px d_y^py d_z^pz * Gaussian:
# s; p_x, p_y, p_z; d_xy, d_yz, d_zx, d_(x^2-y^2), d_(3z^2-r^2) = 2 z^2 - x^2 - y^2.
_BASIS_TERMS = [[(1.0, 0, 0, 0)], [(1.0, 1, 0, 0)], [(1.0, 0, 1, 0)], [(1.0, 0, 0, 1)], [(1.0, 1, 1, 0)],
                [(1.0, 0, 1, 1)], [(1.0, 1, 0, 1)], [(1.0, 2, 0, 0), (-1.0, 0, 2, 0)],
                [(2.0, 0, 0, 2), (-1.0, 2, 0, 0), (-1.0, 0, 2, 0)]]
# distinct power triples (px, py, pz) of those terms
_TRIPLES = sorted({(t[1], t[2], t[3]) for m in _BASIS_TERMS for t in m})


def _axis_factors(n, h, Lax, R, kax, sigma):
    """Per-axis factors d^p exp(-d^2 / (2 sigma^2)) exp(-i k (R + d)), p = 0, 1, 2, on the n grid
    coordinates of one axis (d the minimum-image displacement from R): (3, n)."""
    d = min_image(np.arange(n) * h - R, Lax)
    g = np.exp(-d * d / (2.0 * sigma * sigma))
    if kax != 0.0:
        g = g * np.exp(-1j * kax * (R + d))
    return np.stack([g, d * g, d * d * g])


def atomic_orbital_states(L, n, pos, kpts, axes, per_atom=8, n_par=5, sigma=1.0, seed=0, select=None,
                          dtype=np.complex128):
    """8 orbitals per atom: seeded random complex combinations of the s, p and d
    Gaussians (width sigma) on that atom; n_par parallel and the rest
    antiparallel to the atom's spin axis; Bloch phase folded into u_k;
    Loewdin-orthonormalised per k-point.

    The basis functions (and the Bloch phase) are products of one-dimensional factors on the
    orthorhombic grid, so the Gram matrix of the basis on the grid is a sum of products of
    one-dimensional sums; the spinor overlap S follows from it and the spinor products, and the
    orthonormalised states psi_i = sum_j (S^-1/2)_{ji} chi_j phi_j are formed as one coefficient
    matrix times the separable basis, one z-plane at a time (in the precision of `dtype`:
    complex128, or complex64 with single-precision products).  `select` picks the state indices
    to return (all by default)."""
    rng = np.random.default_rng(seed)
    L = np.asarray(L, np.float64)
    pos = np.asarray(pos, np.float64)
    h = L / n
    dV = float(np.prod(L)) / n ** 3
    natoms = len(pos)
    ns = natoms * per_atom
    coef = rng.normal(size=(natoms, per_atom, 9)) + 1j * rng.normal(size=(natoms, per_atom, 9))
    sel = np.arange(ns) if select is None else np.asarray(select)
    chi = np.array([spinor_along(axes[a][0], axes[a][1], parallel=(j < n_par))
                    for a in range(natoms) for j in range(per_atom)])  # (ns, 2)
    nt = len(_TRIPLES)
    tindex = {t: i for i, t in enumerate(_TRIPLES)}
    # T[m, tau]: weight of triple tau in basis function m
    T = np.zeros((9, nt))
    for m, terms in enumerate(_BASIS_TERMS):
        for c, px, py, pz in terms:
            T[m, tindex[(px, py, pz)]] += c
    real = np.dtype(dtype) == np.complex64
    out = np.empty((len(kpts), len(sel), 2, n, n, n), dtype)
    for ik, kv in enumerate(np.asarray(kpts, np.float64)):
        F = [np.stack([_axis_factors(n, h[ax], L[ax], pos[a, ax], kv[ax], sigma) for a in range(natoms)])
             for ax in range(3)]  # F[ax]: (natoms, 3, n)
        # one-dimensional overlaps O[ax][a, p, b, q] = sum_j conj(F_ap(j)) F_bq(j)
        O = [np.einsum("apj,bqj->apbq", f.conj(), f) for f in F]
        # Gram of the triples: Gt[a tau, b tau'] = prod_ax O[ax][a, p_ax, b, q_ax] dV
        Gt = np.empty((natoms, nt, natoms, nt), np.complex128)
        for i, (px, py, pz) in enumerate(_TRIPLES):
            for j, (qx, qy, qz) in enumerate(_TRIPLES):
                Gt[:, i, :, j] = O[0][:, px, :, qx] * O[1][:, py, :, qy] * O[2][:, pz, :, qz] * dV
        # orbital coefficients on the triples: Ct[a, tau, s] for the states s on atom a
        Ct = np.zeros((natoms, nt, ns), np.complex128)
        for a in range(natoms):
            Ct[a, :, a * per_atom:(a + 1) * per_atom] = (coef[a] @ T).T
        Ct = Ct.reshape(natoms * nt, ns)
        S = (chi.conj() @ chi.T) * (Ct.conj().T @ Gt.reshape(natoms * nt, natoms * nt) @ Ct)
        w, U = np.linalg.eigh(S)
        Sm = (U * (1.0 / np.sqrt(w))) @ U.conj().T
        # W[a tau, i, sigma] = sum_s Sm[s, i] Ct[a tau, s] chi[s, sigma]
        W = np.stack([(Ct * chi[None, :, x]) @ Sm[:, sel] for x in range(2)], axis=-1)
        W = W.reshape(natoms * nt, 2 * len(sel)).T
        # plane factors P[a tau](y, x) = F_y(a, py) F_x(a, px)
        P = np.stack([np.einsum("ay,ax->ayx", F[1][:, py], F[0][:, px]) for (px, py, pz) in _TRIPLES], axis=1)
        P = P.reshape(natoms * nt, n * n)
        Fz = np.stack([F[2][:, pz] for (px, py, pz) in _TRIPLES], axis=1).reshape(natoms * nt, n)
        if np.isrealobj(P) and np.isrealobj(Fz):
            # real basis (k = 0): real and imaginary parts as two real products
            ft = np.float32 if real else np.float64
            if real:
                # single-precision products: factors below 1e-12 (their contributions lie far below
                # complex64 resolution) are set to zero, so that no product underflows into the
                # slow subnormal range
                P = np.where(np.abs(P) < 1e-12, 0.0, P)
                Fz = np.where(np.abs(Fz) < 1e-12, 0.0, Fz)
            Wr, Wi = np.ascontiguousarray(W.real, dtype=ft), np.ascontiguousarray(W.imag, dtype=ft)
            P = np.ascontiguousarray(P, dtype=ft)
            for z in range(n):
                fz = Fz[:, z].astype(ft)[None, :]
                blk = out[ik, :, :, z].reshape(2 * len(sel), n * n)
                blk.real = (Wr * fz) @ P
                blk.imag = (Wi * fz) @ P
        else:
            if real:
                W, P = W.astype(np.complex64), P.astype(np.complex64)
            for z in range(n):
                out[ik, :, :, z] = ((W * Fz[:, z][None, :].astype(W.dtype)) @ P).reshape(len(sel), 2, n, n)
    return out


# ----------------------------------------------------------------------------
# workloads

def _species_block(nspecies, lmax, Z=8.0, rc=0.8, width=1.0, lam=0.0):
    D_all = np.array([1.0, 0.5, 0.25, 0.125])[: lmax + 1]
    D = np.tile(D_all, (nspecies, 1))
    lam_arr = np.full((nspecies, lmax + 1), lam)
    lam_arr[:, 0] = 0.0
    return (np.full(nspecies, Z), np.full(nspecies, rc), np.full(nspecies, width), D, lam_arr)


def tiny(seed=20250621):
    """Tiny oracle case: 10 bohr cube, 24^3, one Z=8 atom, l=0,1 projectors without SOC,
    4 random spinors tilted 30 deg, 10 steps of dt=0.05, no field."""
    L = np.array([10.0, 10.0, 10.0])
    n = 24
    Z, rc, w, D, lam = _species_block(1, 1)
    times, A, B = zero_fields(10, 0.05)
    return Workload("tiny", L, n, np.array([[5.0, 5.0, 5.0]]), np.zeros(1, np.int32), Z, rc, w, 1,
                    D, lam, 5.0, np.zeros((1, 3)), np.ones(1), np.ones((1, 4)), 0.05, 10, seed,
                    times, A, B)


def tiny_states(wl):
    return random_tilted_states(wl.L, wl.n, wl.nstates, wl.seed)


def cluster(n=64, nsteps=2000, seed=20250622, lam=0.02, laser=True):
    """13-atom icosahedral cluster (centre-vertex 4.7 bohr) in a 24 bohr cube; Z=8 atoms with
    l=0,1,2 projectors and L.S coefficient 0.02 Ha; 104 occupied spinors of 112
    (only occupied ones are propagated); Gaussian x-polarised laser in velocity gauge."""
    L = np.array([24.0, 24.0, 24.0])
    pos = icosahedron(L / 2.0, 4.7)
    Z, rc, w, D, lam_arr = _species_block(1, 2, lam=lam)
    dt = 0.04
    if laser:
        times, A, B = laser_table(nsteps, dt)
    else:
        times, A, B = zero_fields(nsteps, dt)
    return Workload("cluster%d" % n, L, n, pos, np.zeros(13, np.int32), Z, rc, w, 2, D, lam_arr, 5.0,
                    np.zeros((1, 3)), np.ones(1), np.ones((1, 104)), dt, nsteps, seed, times, A, B)


def cluster_axes(natoms, tilted=1, tilt_deg=20.0):
    axes = [(0.0, 0.0)] * natoms
    axes[tilted] = (math.radians(tilt_deg), 0.0)
    return axes


def cluster_states(wl, per_atom=8):
    return atomic_orbital_states(wl.L, wl.n, wl.pos, wl.kpts, cluster_axes(len(wl.pos)),
                                 per_atom=per_atom, seed=wl.seed)


def bcc(nsteps=1000, seed=20250623):
    """2x2x2 bcc supercell (a=5.42 bohr, 16 Z=8 atoms with L.S 0.02 Ha) on 48^3; 2x2x2
    Monkhorst-Pack k-points; 128 occupied spinors of 144 per k; static B_x = 0.001 plus laser."""
    a = 5.42
    L = np.array([2 * a] * 3)
    pos = bcc_supercell(a, 2)
    Z, rc, w, D, lam = _species_block(1, 2, lam=0.02)
    q = 0.25 * 2.0 * math.pi / L[0]
    kpts = np.array([[sx * q, sy * q, sz * q] for sx in (-1, 1) for sy in (-1, 1) for sz in (-1, 1)])
    dt = 0.04
    times, A, B = laser_table(nsteps, dt, B_static=(0.001, 0.0, 0.0))
    return Workload("bcc48", L, 48, pos, np.zeros(16, np.int32), Z, rc, w, 2, D, lam, 5.0,
                    kpts, np.full(8, 1.0 / 8.0), np.ones((8, 128)), dt, nsteps, seed, times, A, B)


def bcc_states(wl):
    return atomic_orbital_states(wl.L, wl.n, wl.pos, wl.kpts, [(0.0, 0.0)] * len(wl.pos), seed=wl.seed)


def large(nsteps=200, seed=20250625, nstates=1024):
    """4x4x4 bcc-like supercell (a = 5.425 bohr, 128 Z=8 atoms jittered by N(0, 0.1^2) bohr, L.S
    0.02 Ha) in a 21.7 bohr cube on 96^3; Gamma point; `nstates` occupied spinors (1024 of
    1088 in the full case); laser as in the cluster case."""
    rng = np.random.default_rng(seed)
    a = 5.425
    pos = bcc_supercell(a, 4, jitter=0.1, rng=rng)
    L = np.array([4 * a] * 3)
    Z, rc, w, D, lam = _species_block(1, 2, lam=0.02)
    dt = 0.04
    times, A, B = laser_table(nsteps, dt)
    return Workload("large96", L, 96, pos, np.zeros(len(pos), np.int32), Z, rc, w, 2, D, lam, 5.0,
                    np.zeros((1, 3)), np.ones(1), np.ones((1, nstates)), dt, nsteps, seed, times, A, B)


def large_axes(natoms, tilted=1, tilt_deg=20.0):
    """Spin axes of the large supercell's atoms: along z, one atom tilted as in the cluster."""
    return cluster_axes(natoms, tilted, tilt_deg)


def large_states(wl, select=None, dtype=np.complex64):
    """The large supercell's atomic-orbital spinors (8 per atom), complex64 by default (the
    FP32-mixed storage; the complex128 array of all 1024 is 29 GB)."""
    return atomic_orbital_states(wl.L, wl.n, wl.pos, wl.kpts, large_axes(len(wl.pos)), seed=wl.seed,
                                 select=select, dtype=dtype)


def small_parity(n=16, nstates=5, nk=2, seed=7, lam=0.02, lmax=2, field=True, natoms=3):
    """Small multi-feature case for element-wise parity: several atoms with SOC, two k-points,
    an odd number of states, laser plus static B."""
    rng = np.random.default_rng(seed)
    L = np.array([9.0, 9.0, 9.0])
    pos = rng.uniform(0.0, 9.0, size=(natoms, 3))
    Z, rc, w, D, lam_arr = _species_block(1, lmax, lam=lam, Z=3.0)
    kpts = rng.uniform(-0.3, 0.3, size=(nk, 3)) if nk > 1 else np.zeros((1, 3))
    kw = np.full(nk, 1.0 / nk)
    occ = np.ones((nk, nstates))
    occ[:, -1] = 0.5
    dt = 0.05
    nsteps = 4
    if field:
        times, A, B = laser_table(nsteps, dt, E0=0.3, omega=0.3, fwhm_fs=0.2, pol=(0.6, 0.0, 0.8),
                                  B_static=(0.02, -0.01, 0.03))
    else:
        times, A, B = zero_fields(nsteps, dt)
    return Workload("parity%d" % n, L, n, pos, np.zeros(natoms, np.int32), Z, rc, w, lmax, D, lam_arr,
                    4.0, kpts, kw, occ, dt, nsteps, seed, times, A, B)


def small_parity_states(wl):
    rng = np.random.default_rng(wl.seed + 1)
    n = wl.n
    dV = float(np.prod(wl.L)) / n ** 3
    out = np.empty((wl.nk, wl.nstates, 2, n, n, n), np.complex128)
    for ik in range(wl.nk):
        raw = rng.normal(size=(wl.nstates, 2 * n ** 3)) + 1j * rng.normal(size=(wl.nstates, 2 * n ** 3))
        # smooth the states a little so the kinetic energy stays moderate
        raw = raw.reshape(wl.nstates, 2, n, n, n)
        f = np.fft.fftn(raw, axes=(-3, -2, -1))
        g = np.fft.fftfreq(n) * n
        gz, gy, gx = np.meshgrid(g, g, g, indexing="ij")
        f *= np.exp(-(gx ** 2 + gy ** 2 + gz ** 2) / (0.08 * n * n))
        raw = np.fft.ifftn(f, axes=(-3, -2, -1)).reshape(wl.nstates, -1)
        out[ik] = lowdin(raw, dV).reshape(wl.nstates, 2, n, n, n)
    return out
