"""Oracle: spinor Kohn-Sham Hamiltonian and real-time propagation step (FP64, numpy).

Follows arXiv 2506.21908:
  * non-collinear KS Hamiltonian, Eq. HNC-SDFT:
        H = [-1/2 nabla^2 + v_ext + v_H + vbar_xc] I_2 + b_s . sigma,  b_s = mu_B b_ext + b_xc
    with mu_B = 1/2 (Sec. 2.1) and the spin Zeeman matrix of Eq. zeeman_potential;
  * time-dependent KS equation, Eq. TDSDFT, with the adiabatic locally collinear XC
    (Eqs. LC+ALDA2, LC+ALDA) evaluated at the instantaneous n, m;
  * spin density matrix and its 4-vector storage, Eqs. rho1-rho3 and density4;
    the 4-vector potential, Eq. potential4;
  * Kleinman-Bylander projectors with spin-orbit coupling, Eq. Vps, Eq. Vps-soc and the
    L.S form of the pseudopotential in Sec. 4.4 (|lm;a>[V_l + V_l^SO <lm|L|lm'>.S]<lm';a|).

Readings where the paper is silent (each one is a constant of this module or a
parameter, and the CUDA library takes the same reading):
  P1  propagator: enforced time-reversal symmetry (ETRS),
          psi(t+dt) = Exp(-i dt/2 H[rho~, t+dt]) Exp(-i dt/2 H[rho(t), t]) psi(t),
      rho~ from a predictor psi~ = Exp(-i dt H[rho(t), t]) psi(t), then n_sc corrector passes;
      Exp as a Chebyshev series (default) or a Taylor series;
  P2  Chebyshev spectral window from the potential extrema, kinetic maximum and a
      projector norm bound, widened by 5 %;
  P3  velocity gauge: kinetic 1/2 |G+k+A(t)|^2, projector phase exp(-i (k+A).d);
  P4  local potential -Z erf(r/rc)/r summed in reciprocal space; at G = 0 only the
      non-Coulomb part pi Z rc^2 / Omega is kept, the Hartree G = 0 term is dropped;
  P5  projector radial part N_l r^l exp(-r^2/(2 w^2)) times real Y_lm, cut at |d| < r_cut
      (minimum image), continuum-normalised;
  P6  coupling block on the (l, m, sigma) space D_l I + lambda_l L.S;
  P9  E_xc reported as the functional value int e_xc; int <rho_v, V_v^xc> is reported
      separately as the potential-weighted integral of Eq. xc_energy4.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import special

from .xc import collinear_xc, noncollinear_xc, unpolarised_xc

MU_B = 0.5
PAULI = np.array([[[0, 1], [1, 0]], [[0, -1j], [1j, 0]], [[1, 0], [0, -1]]], dtype=np.complex128)


# =============================================================================
# grid and FFT  (plane-wave basis on a periodic real-space grid)

class Grid:
    """Cubic-mesh orthorhombic cell.  Arrays are [z][y][x]; G follows the fftfreq
    convention with the Nyquist index at -n/2.  Forward FFT is unnormalised,
    inverse carries 1/N."""

    def __init__(self, L, n):
        self.L = np.asarray(L, np.float64)
        self.n = int(n)
        self.N = self.n ** 3
        self.omega = float(np.prod(self.L))
        self.dV = self.omega / self.N
        g = np.fft.fftfreq(self.n) * self.n
        gx = 2.0 * math.pi / self.L[0] * g
        gy = 2.0 * math.pi / self.L[1] * g
        gz = 2.0 * math.pi / self.L[2] * g
        Gz, Gy, Gx = np.meshgrid(gz, gy, gx, indexing="ij")
        self.G = np.stack([Gx, Gy, Gz], axis=-1)
        self.G2 = (self.G ** 2).sum(-1)
        h = self.L / self.n
        iz, iy, ix = np.meshgrid(np.arange(self.n), np.arange(self.n), np.arange(self.n), indexing="ij")
        self.r = np.stack([ix * h[0], iy * h[1], iz * h[2]], axis=-1)

    def fft(self, f):
        return np.fft.fftn(f, axes=(-3, -2, -1))

    def ifft(self, f):
        return np.fft.ifftn(f, axes=(-3, -2, -1))

    def kinetic(self, shift):
        """1/2 |G + k + A|^2 on the G mesh."""
        q = self.G + np.asarray(shift, np.float64)
        return 0.5 * (q ** 2).sum(-1)

    def kinetic_max(self, shift):
        """max over the G mesh of 1/2 |G + shift|^2 (corners of the box)."""
        g = np.fft.fftfreq(self.n) * self.n
        tot = 0.0
        for a in range(3):
            ga = 2.0 * math.pi / self.L[a] * np.array([g.min(), g.max()])
            tot += np.max((ga + shift[a]) ** 2)
        return 0.5 * tot


def local_potential(grid, pos, Zs, rcs):
    """V_loc(r) for atoms with potential -Z erf(r/rc)/r, periodic, reading P4.

    V(G) = sum_a -4 pi Z / G^2 exp(-G^2 rc^2/4) exp(-i G.R_a) / Omega, V(0) = sum_a pi Z rc^2 / Omega,
    V(r) = sum_G V(G) exp(i G.r), real part (symmetric treatment of the Nyquist planes)."""
    G2 = grid.G2
    VG = np.zeros(G2.shape, np.complex128)
    nz = G2 > 0
    for R, Z, rc in zip(pos, Zs, rcs):
        phase = np.exp(-1j * (grid.G @ np.asarray(R, np.float64)))
        term = np.zeros(G2.shape, np.complex128)
        term[nz] = -4.0 * math.pi * Z / G2[nz] * np.exp(-G2[nz] * rc * rc / 4.0)
        term[~nz] = math.pi * Z * rc * rc
        VG += term * phase
    VG /= grid.omega
    return (grid.ifft(VG) * grid.N).real


def hartree_potential(grid, n):
    """v_H(G) = 4 pi n(G) / G^2, v_H(G=0) = 0 (Eq. KSpot, Hartree term)."""
    nG = grid.fft(n)
    vG = np.zeros_like(nG)
    nz = grid.G2 > 0
    vG[nz] = 4.0 * math.pi * nG[nz] / grid.G2[nz]
    return grid.ifft(vG).real


# =============================================================================
# real spherical harmonics, angular momentum, spin-orbit block

def real_ylm(l, d):
    """Real Y_lm for mu = -l..l on displacement vectors d (npts, 3), from the complex
    Condon-Shortley Y_l^m:  mu>0: sqrt2 (-1)^mu Re Y_l^mu, mu=0: Y_l^0, mu<0: sqrt2 (-1)^mu Im Y_l^|mu|."""
    d = np.atleast_2d(d)
    r = np.sqrt((d * d).sum(-1))
    safe = np.where(r > 0, r, 1.0)
    theta = np.arccos(np.clip(d[:, 2] / safe, -1.0, 1.0))
    phi = np.arctan2(d[:, 1], d[:, 0])
    out = np.empty((2 * l + 1, d.shape[0]))
    for mu in range(-l, l + 1):
        Y = special.sph_harm_y(l, abs(mu), theta, phi)
        if mu > 0:
            out[mu + l] = math.sqrt(2.0) * (-1) ** mu * Y.real
        elif mu == 0:
            out[l] = Y.real
        else:
            out[mu + l] = math.sqrt(2.0) * (-1) ** mu * Y.imag
    return out


def complex_to_real(l):
    """U with y_mu = sum_m U[mu, m] Y_l^m (rows mu = -l..l, columns m = -l..l)."""
    U = np.zeros((2 * l + 1, 2 * l + 1), np.complex128)
    s2 = math.sqrt(2.0)
    for mu in range(-l, l + 1):
        if mu > 0:
            U[mu + l, mu + l] = (-1) ** mu / s2
            U[mu + l, -mu + l] = 1.0 / s2
        elif mu == 0:
            U[l, l] = 1.0
        else:
            a = -mu
            U[mu + l, a + l] = (-1) ** a / (s2 * 1j)
            U[mu + l, -a + l] = -1.0 / (s2 * 1j)
    return U


def angular_momentum_complex(l):
    """L_x, L_y, L_z in the |l m> basis, m = -l..l (ladder operators)."""
    m = np.arange(-l, l + 1)
    Lz = np.diag(m.astype(np.complex128))
    Lp = np.zeros((2 * l + 1, 2 * l + 1), np.complex128)
    for i, mm in enumerate(m[:-1]):
        Lp[i + 1, i] = math.sqrt(l * (l + 1) - mm * (mm + 1))
    Lm = Lp.T.copy()
    return np.array([(Lp + Lm) / 2.0, (Lp - Lm) / 2j, Lz])


def angular_momentum_real(l):
    """<y_mu| L_alpha |y_nu> in the real-harmonic basis: U* L^C U^T."""
    U = complex_to_real(l)
    return np.array([U.conj() @ La @ U.T for La in angular_momentum_complex(l)])


def soc_block(l, Dl, lam):
    """D_l I + lambda_l L.S on the (mu, sigma) space, index 2*(mu+l) + sigma (reading P6)."""
    Lr = angular_momentum_real(l)
    LS = sum(np.kron(Lr[a], PAULI[a] / 2.0) for a in range(3))
    return Dl * np.eye(2 * (2 * l + 1)) + lam * LS


def radial_norm(l, w):
    """N_l with int_0^inf (N_l r^l exp(-r^2/(2 w^2)))^2 r^2 dr = 1."""
    return math.sqrt(2.0 / (math.gamma(l + 1.5) * w ** (2 * l + 3)))


# =============================================================================
# system

class FieldTable:
    """Tabulated A(t), B(t) with linear interpolation, clamped outside the table."""

    def __init__(self, times, A, B):
        self.t = np.asarray(times, np.float64)
        self.A = np.asarray(A, np.float64)
        self.B = np.asarray(B, np.float64)

    def _interp(self, arr, t):
        return np.array([np.interp(t, self.t, arr[:, a]) for a in range(3)])

    def at(self, t):
        return self._interp(self.A, t), self._interp(self.B, t)


class AtomProjectors:
    """Sphere of grid points around one atom (|d| < r_cut, minimum image, surface points
    excluded with a 1e-10 relative margin) with the real projector values
    beta[(l,mu), point] (reading P5)."""

    def __init__(self, grid, R, w, lmax, r_cut):
        r = grid.r.reshape(-1, 3)
        d = r - R
        d = d - grid.L * np.round(d / grid.L)
        dist = np.sqrt((d * d).sum(-1))
        # points on the cut-off sphere itself (|d| = r_cut in exact arithmetic, common when the
        # grid is commensurate with r_cut) are excluded with a 1e-10 relative margin, so that the
        # set does not depend on the rounding of |d|
        sel = (d * d).sum(-1) < r_cut * r_cut * (1.0 - 1e-10)
        self.idx = np.nonzero(sel)[0]
        self.d = d[sel]
        dd = dist[sel]
        rows = []
        for l in range(lmax + 1):
            rad = radial_norm(l, w) * dd ** l * np.exp(-dd * dd / (2.0 * w * w))
            rows.append(rad[None, :] * real_ylm(l, self.d))
        self.beta = np.vstack(rows)  # ((lmax+1)^2, npts)


class System:
    def __init__(self, L, n, pos, species, Z, rc_loc, width, lmax, D, lam, r_cut,
                 kpts, kw, occ, xc=1, spin_mode=0):
        self.grid = Grid(L, n)
        self.pos = np.asarray(pos, np.float64)
        self.species = np.asarray(species, np.int64)
        self.Z = np.asarray(Z, np.float64)
        self.rc = np.asarray(rc_loc, np.float64)
        self.width = np.asarray(width, np.float64)
        self.lmax = int(lmax)
        self.D = np.asarray(D, np.float64)
        self.lam = np.asarray(lam, np.float64)
        self.r_cut = float(r_cut)
        self.kpts = np.asarray(kpts, np.float64)
        self.kw = np.asarray(kw, np.float64)
        self.occ = np.asarray(occ, np.float64)
        self.xc = int(xc)
        # 0: non-collinear (Eq. HNC-SDFT); 1: collinear, sigma_z-only potential (Eq. HSDFT);
        # 2: spin-unpolarised (no spin field at all)
        self.spin_mode = int(spin_mode)
        if self.spin_mode not in (0, 1, 2):
            raise ValueError("spin_mode must be 0, 1 or 2")
        if self.spin_mode != 0 and np.any(self.lam != 0.0):
            raise ValueError("spin-orbit coupling couples the spin channels: it needs the non-collinear mode")
        self.vloc = local_potential(self.grid, self.pos, self.Z[self.species], self.rc[self.species])
        self.atoms = [AtomProjectors(self.grid, R, self.width[s], self.lmax, self.r_cut)
                      for R, s in zip(self.pos, self.species)]
        self.blocks = [[soc_block(l, self.D[s, l], self.lam[s, l]) for l in range(self.lmax + 1)]
                       for s in self.species]

    @classmethod
    def from_workload(cls, wl):
        return cls(wl.L, wl.n, wl.pos, wl.species, wl.Z, wl.rc_loc, wl.width, wl.lmax, wl.D, wl.lam,
                   wl.r_cut, wl.kpts, wl.kw, wl.occ, wl.xc, getattr(wl, "spin_mode", 0))

    def effective_B(self, B):
        """External field seen by the spin: all of B (non-collinear), its z component along the
        quantisation axis (collinear, Eq. HSDFT), none (unpolarised)."""
        B = np.asarray(B, np.float64)
        if self.spin_mode == 1:
            return np.array([0.0, 0.0, B[2]])
        if self.spin_mode == 2:
            return np.zeros(3)
        return B

    # ------------------------------------------------------------------ density
    def rho_v(self, psi):
        """Spin-density 4-vector {rho_uu, rho_dd, Re rho_ud, Im rho_ud}, Eqs. rho1-rho3, density4,
        rho_s = sum_i f_i psi_i psi_i^dagger with k-point weights."""
        wf = self.kw[:, None] * self.occ
        up = psi[:, :, 0]
        dn = psi[:, :, 1]
        wfe = wf[:, :, None, None, None]
        ud = (wfe * up * dn.conj()).sum(axis=(0, 1))
        return np.stack([(wfe * np.abs(up) ** 2).sum(axis=(0, 1)),
                         (wfe * np.abs(dn) ** 2).sum(axis=(0, 1)), ud.real, ud.imag])

    @staticmethod
    def n_m(rho):
        """n = rho_uu + rho_dd; m_x = 2 Re rho_ud, m_y = -2 Im rho_ud, m_z = rho_uu - rho_dd."""
        return rho[0] + rho[1], np.stack([2.0 * rho[2], -2.0 * rho[3], rho[0] - rho[1]])

    # ---------------------------------------------------------------- potential
    def potential(self, rho, B):
        """V_v = [v + b_z, v - b_z, 2 b_x, -2 b_y] (Eq. potential4) with v = v_loc + v_H + vbar_xc and
        b = b_xc + mu_B B (Eq. HNC-SDFT, Eq. zeeman_potential).  Also returns the parts."""
        n, m = self.n_m(rho)
        vH = hartree_potential(self.grid, n)
        if not self.xc:
            exc, vbar, bxc = np.zeros_like(n), np.zeros_like(n), np.zeros_like(m)
        elif self.spin_mode == 1:
            exc, vbar, bz = collinear_xc(rho[0], rho[1])
            bxc = np.stack([np.zeros_like(n), np.zeros_like(n), bz])
        elif self.spin_mode == 2:
            exc, vbar = unpolarised_xc(n)
            bxc = np.zeros_like(m)
        else:
            exc, vbar, bxc = noncollinear_xc(n, m)
        v = self.vloc + vH + vbar
        b = bxc + MU_B * self.effective_B(B)[:, None, None, None]
        V = np.stack([v + b[2], v - b[2], 2.0 * b[0], -2.0 * b[1]])
        return V, dict(vH=vH, exc=exc, vbar=vbar, bxc=bxc, n=n, m=m)

    # ------------------------------------------------------------------ H apply
    def apply_local(self, V, psi):
        """2x2 spin-matrix potential [[v+b_z, b_x - i b_y], [b_x + i b_y, v - b_z]]."""
        up, dn = psi[..., 0, :, :, :], psi[..., 1, :, :, :]
        bm = 0.5 * (V[2] + 1j * V[3])  # b_x - i b_y
        bp = 0.5 * (V[2] - 1j * V[3])  # b_x + i b_y
        return np.stack([V[0] * up + bm * dn, bp * up + V[1] * dn], axis=-4)

    def apply_kinetic(self, psi_k, shift):
        return self.grid.ifft(self.grid.kinetic(shift) * self.grid.fft(psi_k))

    def projections(self, psi_k, shift):
        """c[a][l] = <beta~_{a,l,mu}|psi_sigma> (nb, 2l+1, 2) and D c, beta~ = exp(-i (k+A).d) beta."""
        nb = psi_k.shape[0]
        flat = psi_k.reshape(nb, 2, -1)
        out = []
        for a, at in enumerate(self.atoms):
            bt = at.beta * np.exp(-1j * (at.d @ shift))[None, :]
            c = np.einsum("pr,bsr->bps", bt.conj(), flat[:, :, at.idx]) * self.grid.dV
            per_l = []
            row = 0
            for l in range(self.lmax + 1):
                nl = 2 * l + 1
                cl = c[:, row:row + nl, :].reshape(nb, 2 * nl)
                dc = cl @ self.blocks[a][l].T
                per_l.append((cl, dc))
                row += nl
            out.append((bt, per_l))
        return out

    def apply_nonlocal(self, psi_k, shift):
        """V_NL psi = sum_a sum_pq beta~_p D_pq <beta~_q|psi>."""
        nb = psi_k.shape[0]
        res = np.zeros((nb, 2, self.grid.N), np.complex128)
        for at, (bt, per_l) in zip(self.atoms, self.projections(psi_k, shift)):
            dcs = np.concatenate([dc.reshape(nb, 2 * l + 1, 2) for l, (_, dc) in enumerate(per_l)], axis=1)
            res[:, :, at.idx] += np.einsum("pr,bps->bsr", bt, dcs)
        return res.reshape(psi_k.shape)

    def apply_h(self, psi, V, A):
        """H psi for all k-points: kinetic + 2x2 local + non-local (Eq. HNC-SDFT, Eq. Vps)."""
        out = np.empty_like(psi)
        loc = self.apply_local(V, psi)
        for ik in range(psi.shape[0]):
            shift = self.kpts[ik] + A
            out[ik] = self.apply_kinetic(psi[ik], shift) + loc[ik] + self.apply_nonlocal(psi[ik], shift)
        return out

    # ------------------------------------------------------- per-atom moments
    def voronoi_owner(self):
        """Nearest atom of every grid point (minimum image), Algorithm 1's NearestAtom rule;
        equal distances go to the lowest atom index.  |d|^2 = (dx^2 + dy^2) + dz^2."""
        r = self.grid.r.reshape(-1, 3)
        best = np.full(r.shape[0], np.inf)
        owner = np.zeros(r.shape[0], np.int64)
        for a, R in enumerate(self.pos):
            d = r - R
            d = d - self.grid.L * np.round(d / self.grid.L)
            d2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
            closer = d2 < best
            owner[closer] = a
            best = np.where(closer, d2, best)
        return owner

    def atom_moments(self, rho):
        """Integrals of m and n over each atom's Voronoi cell."""
        n, m = self.n_m(rho)
        owner = self.voronoi_owner()
        na = len(self.pos)
        M = np.zeros((na, 3))
        N = np.zeros(na)
        for a in range(na):
            sel = owner == a
            M[a] = m.reshape(3, -1)[:, sel].sum(axis=1) * self.grid.dV
            N[a] = n.reshape(-1)[sel].sum() * self.grid.dV
        return M, N

    # ---------------------------------------------------------------- torques
    def torques(self, psi, rho, V, parts, A, B):
        """Global spin torques, dM/dt = i <[H, sigma]> summed over the occupied spinors:
        the local 2x2 potential gives 2 int b x m dV (Eq. GMT), split into its XC part
        2 int b_xc x m dV (zero in the locally collinear approximation, Eq. spincont2) and the
        Zeeman part 2 mu_B B x M (Eq. magrot); the L.S projectors give the spin-orbit torque of
        Eq. SOtorque, sum_k w_k sum_i f_i sum_a 2 i c^dagger [D_a, S] c with S = sigma / 2 on the
        spin index of the projections c = <beta~|psi>.  The kinetic term and D_l I commute with
        the spin and give nothing."""
        g = self.grid
        n, m = parts["n"], parts["m"]
        bxc = parts["bxc"]
        xc = 2.0 * np.cross(bxc.reshape(3, -1).T, m.reshape(3, -1).T).sum(axis=0) * g.dV
        M = m.sum(axis=(1, 2, 3)) * g.dV
        zee = 2.0 * MU_B * np.cross(self.effective_B(B), M)
        wf = self.kw[:, None] * self.occ
        soc = np.zeros(3)
        for ik in range(psi.shape[0]):
            proj = self.projections(psi[ik], self.kpts[ik] + A)
            for a, (bt, per_l) in enumerate(proj):
                for l, (cl, _) in enumerate(per_l):
                    D = self.blocks[a][l]
                    for i in range(3):
                        Si = np.kron(np.eye(2 * l + 1), PAULI[i] / 2.0)
                        Ti = 2j * (D @ Si - Si @ D)
                        q = np.einsum("bp,pq,bq->b", cl.conj(), Ti, cl).real
                        soc[i] += (wf[ik] * q).sum()
        return dict(xc=xc, zeeman=zee, soc=soc, total=xc + zee + soc)

    # --------------------------------------------------------------- energies
    def inner(self, a, b):
        return np.vdot(a, b) * self.grid.dV

    def energies(self, psi, rho, V, parts, A, B):
        """Energy terms of the state (the quantity the exact dynamics conserves when H has no
        explicit time dependence): E_kin = sum w f <psi|1/2|G+k+A|^2|psi>, E_nl = sum w f <psi|V_NL|psi>,
        E_loc = int v_loc n, E_H = 1/2 int v_H n, E_xc = int n eps_xc (reading P9: the functional value,
        with int <rho_v, V_v^xc> of Eq. xc_energy4 reported as xc_pot), E_Z = int mu_B B.m
        (Eq. zeeman_potential); the ion-ion constant is excluded."""
        g = self.grid
        wf = self.kw[:, None] * self.occ
        ekin = 0.0
        enl = 0.0
        for ik in range(psi.shape[0]):
            shift = self.kpts[ik] + A
            tk = self.apply_kinetic(psi[ik], shift)
            nk = self.apply_nonlocal(psi[ik], shift)
            for i in range(psi.shape[1]):
                ekin += wf[ik, i] * np.vdot(psi[ik, i], tk[i]).real * g.dV
                enl += wf[ik, i] * np.vdot(psi[ik, i], nk[i]).real * g.dV
        n, m = parts["n"], parts["m"]
        eloc = (self.vloc * n).sum() * g.dV
        eH = 0.5 * (parts["vH"] * n).sum() * g.dV
        exc = parts["exc"].sum() * g.dV
        ez = MU_B * (self.effective_B(B)[:, None, None, None] * m).sum() * g.dV
        vxc4 = np.stack([parts["vbar"] + parts["bxc"][2], parts["vbar"] - parts["bxc"][2],
                         2.0 * parts["bxc"][0], -2.0 * parts["bxc"][1]])
        exc_pot = (rho * vxc4).sum() * g.dV
        tot = ekin + enl + eloc + eH + exc + ez
        return dict(kin=ekin, nl=enl, loc=eloc, H=eH, xc=exc, Z=ez, total=tot, xc_pot=exc_pot,
                    N=n.sum() * g.dV, M=m.sum(axis=(1, 2, 3)) * g.dV)

    # --------------------------------------------------------- spectral bound
    def nl_norm_bound(self):
        """Upper bound on ||V_NL|| = ||P D P^dagger|| <= max_a ||D_a|| ||P^dagger P||, with ||P^dagger P||
        bounded by the largest Gershgorin row sum of the Gram matrix of all projectors: within an
        atom the exact overlaps (the phases cancel), between atoms sum_r |beta_ap| |beta_bq| dV."""
        g = self.grid
        S = np.zeros(g.N)
        for at in self.atoms:
            np.add.at(S, at.idx, np.abs(at.beta).sum(axis=0))
        gmax = 0.0
        dmax = 0.0
        for a, at in enumerate(self.atoms):
            own = np.abs(at.beta).sum(axis=0)
            gram = (at.beta @ at.beta.T) * g.dV
            inter = (np.abs(at.beta) * (S[at.idx] - own)[None, :]).sum(axis=1) * g.dV
            if gram.size:
                gmax = max(gmax, (np.abs(gram).sum(axis=1) + inter).max())
            dmax = max(dmax, max(np.abs(np.linalg.eigvalsh(b)).max() for b in self.blocks[a]))
        return dmax * gmax

    def spectral_bounds(self, V, A_list, margin=0.05):
        """Reading P2: window [E_min, E_max] for the Chebyshev expansion."""
        v = 0.5 * (V[0] + V[1])
        b = np.sqrt((0.5 * (V[0] - V[1])) ** 2 + (0.5 * V[2]) ** 2 + (0.5 * V[3]) ** 2)
        nl = self.nl_norm_bound()
        kmax = max(self.grid.kinetic_max(k + A) for k in self.kpts for A in A_list)
        emin = v.min() - b.max() - nl
        emax = kmax + v.max() + b.max() + nl
        w = emax - emin
        return emin - 0.5 * margin * w, emax + 0.5 * margin * w


# =============================================================================
# propagators

def chebyshev_order(z, tol=1e-16, kmax=100000):
    """Smallest K with |J_k(z)| < tol for every k > K (J_k decreases monotonically for k > z)."""
    k = int(math.floor(abs(z))) + 1
    while k < kmax:
        if abs(special.jv(k, z)) < tol:
            return k - 1
        k += 1
    raise ValueError("Chebyshev order not found")


def chebyshev_coefficients(tau, emin, emax, K):
    """a_k = (2 - delta_k0) (-i)^k J_k(tau Delta) exp(-i tau c), so that
    exp(-i tau H) = sum_k a_k T_k((H - c)/Delta)  (Jacobi-Anger expansion)."""
    c = 0.5 * (emax + emin)
    dlt = 0.5 * (emax - emin)
    k = np.arange(K + 1)
    a = (2.0 - (k == 0)) * (-1j) ** k * special.jv(k, tau * dlt) * np.exp(-1j * tau * c)
    return a, c, dlt


def exp_chebyshev(apply_h, psi, tau, emin, emax, K):
    """Exp(-i tau H) psi by the Chebyshev recurrence T_{k+1} = 2 H~ T_k - T_{k-1}."""
    a, c, dlt = chebyshev_coefficients(tau, emin, emax, K)
    t_prev = psi
    acc = a[0] * psi
    if K == 0:
        return acc
    t_cur = (apply_h(psi) - c * psi) / dlt
    acc = acc + a[1] * t_cur
    for k in range(2, K + 1):
        t_next = 2.0 * (apply_h(t_cur) - c * t_cur) / dlt - t_prev
        acc = acc + a[k] * t_next
        t_prev, t_cur = t_cur, t_next
    return acc


def exp_crank_nicolson(apply_h, psi, tau, tol=1e-14):
    """Crank-Nicolson step (1 + i tau H / 2)^{-1} (1 - i tau H / 2) psi (the Cayley transform of
    -i tau H), the linear system solved by GMRES on the matrix-free H to relative residual tol."""
    from scipy.sparse.linalg import LinearOperator, gmres
    shape = psi.shape
    nvec = psi.size

    def amul(x):
        x = x.reshape(shape)
        return (x + 0.5j * tau * apply_h(x)).reshape(-1)

    A = LinearOperator((nvec, nvec), matvec=amul, dtype=np.complex128)
    rhs = (psi - 0.5j * tau * apply_h(psi)).reshape(-1)
    try:
        x, info = gmres(A, rhs, x0=psi.reshape(-1).copy(), rtol=tol, atol=0.0, restart=200, maxiter=50)
    except TypeError:  # scipy releases that name the relative tolerance `tol`
        x, info = gmres(A, rhs, x0=psi.reshape(-1).copy(), tol=tol, atol=0.0, restart=200, maxiter=50)
    if info != 0:
        raise RuntimeError("Crank-Nicolson solve did not converge (%d)" % info)
    return x.reshape(shape)


def exp_taylor(apply_h, psi, tau, K):
    """Exp(-i tau H) psi ~ sum_{k<=K} (-i tau H)^k / k! psi."""
    term = psi
    acc = psi.copy()
    for k in range(1, K + 1):
        term = (-1j * tau / k) * apply_h(term)
        acc = acc + term
    return acc


class Oracle:
    """Propagation state: psi(t), rho(t), V(t), and the ETRS step (reading P1)."""

    def __init__(self, system, fields, dt, psi0, t0=0.0, n_sc=1, sc_tol=0.0, exp_kind=0,
                 exp_order=0, bounds=None, cheb_tol=1e-16):
        self.s = system
        self.f = fields
        self.dt = float(dt)
        self.t = float(t0)
        self.n_sc = int(n_sc)
        self.sc_tol = float(sc_tol)
        self.exp_kind = int(exp_kind)
        self.psi = np.array(psi0, np.complex128)
        self.rho = self.s.rho_v(self.psi)
        A, B = self.f.at(self.t)
        self.V, self.parts = self.s.potential(self.rho, B)
        if bounds is None:
            bounds = self.s.spectral_bounds(self.V, [self.f.A[i] for i in range(len(self.f.t))])
        self.emin, self.emax = bounds
        dlt = 0.5 * (self.emax - self.emin)
        if self.exp_kind == 0:
            if exp_order > 0:
                self.K_full = self.K_half = int(exp_order)
            else:
                self.K_full = chebyshev_order(self.dt * dlt, cheb_tol)
                self.K_half = chebyshev_order(0.5 * self.dt * dlt, cheb_tol)
        elif self.exp_kind == 1:
            self.K_full = self.K_half = int(exp_order) if exp_order > 0 else 4
        else:
            self.K_full = self.K_half = 0  # Crank-Nicolson: an iterative solve, no fixed order

    def _exp(self, psi, V, t, tau, K):
        A, _ = self.f.at(t)
        h = lambda x: self.s.apply_h(x, V, A)  # noqa: E731
        if self.exp_kind == 0:
            return exp_chebyshev(h, psi, tau, self.emin, self.emax, K)
        if self.exp_kind == 2:
            return exp_crank_nicolson(h, psi, tau)
        return exp_taylor(h, psi, tau, K)

    def step(self):
        dt, t = self.dt, self.t
        _, B1 = self.f.at(t + dt)
        pred = self._exp(self.psi, self.V, t, dt, self.K_full)
        rho_p = self.s.rho_v(pred)
        V1, _ = self.s.potential(rho_p, B1)
        phi = self._exp(self.psi, self.V, t, 0.5 * dt, self.K_half)
        new = self._exp(phi, V1, t + dt, 0.5 * dt, self.K_half)
        rho_prev = rho_p
        for _ in range(self.n_sc):
            rho_c = self.s.rho_v(new)
            if self.sc_tol > 0.0 and np.abs(rho_c - rho_prev).max() < self.sc_tol:
                break
            V1, _ = self.s.potential(rho_c, B1)
            new = self._exp(phi, V1, t + dt, 0.5 * dt, self.K_half)
            rho_prev = rho_c
        self.psi = new
        self.t = t + dt
        self.rho = self.s.rho_v(self.psi)
        self.V, self.parts = self.s.potential(self.rho, B1)

    def observables(self):
        A, B = self.f.at(self.t)
        E = self.s.energies(self.psi, self.rho, self.V, self.parts, A, B)
        n, m = self.s.n_m(self.rho)
        norms = (np.abs(self.psi) ** 2).sum(axis=(2, 3, 4, 5)) * self.s.grid.dV
        return n, m, E, norms
