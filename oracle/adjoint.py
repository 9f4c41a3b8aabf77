"""Oracle: discrete adjoint of the ETRS propagation (FP64, numpy).  TEST INFRASTRUCTURE.

Differentiates L = sum_r dL/drho_v(r) . rho_v(r; T) (default: L = M_z(T) = int m_z) of
the exact discrete forward map of ``oracle.tddft.Oracle`` (fixed Chebyshev window and
orders, fixed number of corrector passes, sc_tol = 0) with respect to the field table
entries A(t_j), B(t_j).  The paper has no adjoint; this follows the reverse-mode
rules of the forward algorithm step by step:

  * complex cotangents: for real L, psibar = dL/dRe psi + i dL/dIm psi, so that
    dL = Re sum conj(psibar) dpsi (plain sum over the array, no dV);
  * Chebyshev series y = sum_k a_k T_k(H~) x, T_{k+1} = 2 H~ T_k - T_{k-1}: the cotangents
    S_k of T_k follow the Clenshaw-type recurrence
        S_k = conj(a_k) ybar + 2 H~ S_{k+1} - S_{k+2}  (k >= 1),
        S_0 = conj(a_0) ybar + H~ S_1 - S_2,  xbar = S_0,
    and dH~ enters through Re<S_{k+1}, 2 dH~ T_k> (k >= 1) and Re<S_1, dH~ T_0>;
  * dH/dV(r) for the 2x2 local potential, dH/dA = (G + k + A) for the kinetic term and
    the derivative of the projector phases exp(-i (k+A).d) for V_NL;
  * V = V[rho, B]: Hartree is a symmetric convolution, the locally collinear XC Jacobian
    is assembled by the chain rule from the LSDA Hessian (central differences of the
    pinned LSDA potentials), B enters V uniformly through mu_B B.sigma;
  * rho_v(psi) adjoint from its bilinear definition (Eqs. rho1-rho3, density4).
"""
import numpy as np

from . import xc as oxc
from .tddft import MU_B, chebyshev_coefficients, hartree_potential


def field_weights(times, t):
    """Linear-interpolation weights of table entries at time t (clamped), as used by FieldTable."""
    w = np.zeros(len(times))
    if t <= times[0]:
        w[0] = 1.0
    elif t >= times[-1]:
        w[-1] = 1.0
    else:
        j = int(np.searchsorted(times, t, side="right"))
        a = (t - times[j - 1]) / (times[j] - times[j - 1])
        w[j - 1], w[j] = 1.0 - a, a
    return w


def lsda_hessian(nu, nd, rel=1e-5):
    """d v_sigma / d n_sigma' by central differences of the LSDA potentials."""
    hu = rel * np.maximum(nu, 1e-300)
    hd = rel * np.maximum(nd, 1e-300)
    _, vu_p, vd_p = oxc.lsda(nu + hu, nd)
    _, vu_m, vd_m = oxc.lsda(nu - hu, nd)
    huu = (vu_p - vu_m) / (2 * hu)
    hdu = (vd_p - vd_m) / (2 * hu)
    _, vu_p, vd_p = oxc.lsda(nu, nd + hd)
    _, vu_m, vd_m = oxc.lsda(nu, nd - hd)
    hud = (vu_p - vu_m) / (2 * hd)
    hdd = (vd_p - vd_m) / (2 * hd)
    return huu, 0.5 * (hud + hdu), hdd


def xc_adjoint(n, m, gv, gb):
    """Given dL/dvbar (gv) and dL/db_xc (gb, shape (3,...)), return dL/dn and dL/dm through the
    locally collinear map vbar = (v_u + v_d)/2, b = (v_u - v_d)/2 m/|m| with n_u,d = (n +- |m|)/2."""
    nbar = np.zeros_like(n)
    mbar = np.zeros_like(m)
    mag = np.sqrt((m * m).sum(axis=0))
    ok = n >= oxc.N_THR
    if not np.any(ok):
        return nbar, mbar
    clamp = mag > n
    s = np.minimum(mag, n)
    nu, nd = 0.5 * (n + s), 0.5 * (n - s)
    huu, hud, hdd = [np.zeros_like(n) for _ in range(3)]
    a, b, c = lsda_hessian(nu[ok], nd[ok])
    huu[ok], hud[ok], hdd[ok] = a, b, c
    _, vu, vd = [np.zeros_like(n) for _ in range(3)]
    e_, vu_ok, vd_ok = oxc.lsda(nu[ok], nd[ok])
    vu[ok], vd[ok] = vu_ok, vd_ok
    # derivatives of v_u, v_d with respect to n and s (n_u = (n+s)/2, n_d = (n-s)/2)
    u_n, u_s = 0.5 * (huu + hud), 0.5 * (huu - hud)
    d_n, d_s = 0.5 * (hud + hdd), 0.5 * (hud - hdd)
    vbar_n, vbar_s = 0.5 * (u_n + d_n), 0.5 * (u_s + d_s)
    beta_n, beta_s = 0.5 * (u_n - d_n), 0.5 * (u_s - d_s)
    beta = 0.5 * (vu - vd)
    dirok = ok & (mag > oxc.M_THR)
    safe = np.where(dirok, mag, 1.0)
    mh = np.where(dirok[None], m / safe[None], 0.0)
    mg = (mh * gb).sum(axis=0)  # m^ . gb
    # ds/dn = 1 and ds/dm = 0 where |m| is clamped to n; otherwise ds/dm = m^
    s_n = np.where(clamp, 1.0, 0.0)
    s_m = np.where(clamp[None], 0.0, mh)
    gs = vbar_s * gv + np.where(dirok, beta_s * mg, 0.0)  # dL/ds
    nbar = np.where(ok, vbar_n * gv + np.where(dirok, beta_n * mg, 0.0) + gs * s_n, 0.0)
    perp = gb - mg[None] * mh
    mbar = np.where(ok[None], gs[None] * s_m + np.where(dirok[None], (beta / safe)[None] * perp, 0.0), 0.0)
    return nbar, mbar


def collinear_xc_adjoint(nu, nd, gv, gbz):
    """Cotangents of the channel densities through vbar = (v_u + v_d)/2 and b_z = (v_u - v_d)/2 of
    the collinear LSDA on (rho_uu, rho_dd) (Eq. SDFT / Eq. HSDFT)."""
    nubar, ndbar = np.zeros_like(nu), np.zeros_like(nd)
    ok = nu + nd >= oxc.N_THR
    if np.any(ok):
        huu, hud, hdd = lsda_hessian(nu[ok], nd[ok])
        nubar[ok] = 0.5 * (huu + hud) * gv[ok] + 0.5 * (huu - hud) * gbz[ok]
        ndbar[ok] = 0.5 * (hud + hdd) * gv[ok] + 0.5 * (hud - hdd) * gbz[ok]
    return nubar, ndbar


def unpolarised_xc_adjoint(n, gv):
    """Cotangent of n through v(n) = v_u(n/2, n/2) of the spin-unpolarised LDA:
    dv/dn = (d v_u/d n_u + d v_u/d n_d) / 2."""
    nbar = np.zeros_like(n)
    ok = n >= oxc.N_THR
    if np.any(ok):
        huu, hud, _ = lsda_hessian(0.5 * n[ok], 0.5 * n[ok])
        nbar[ok] = 0.5 * (huu + hud) * gv[ok]
    return nbar


def potential_adjoint(system, rho, Vbar):
    """Cotangent of rho_v and of B from the cotangent of V_v = [v+b_z, v-b_z, 2b_x, -2b_y].  In the
    collinear mode only B_z reaches the spinors and the XC field is along z; in the unpolarised
    mode neither B nor an XC field does."""
    gv = Vbar[0] + Vbar[1]
    gb = np.stack([2.0 * Vbar[2], -2.0 * Vbar[3], Vbar[0] - Vbar[1]])
    Bbar = MU_B * gb.sum(axis=(1, 2, 3))
    mode = getattr(system, "spin_mode", 0)
    n, m = system.n_m(rho)
    nbar = hartree_potential(system.grid, gv)  # symmetric convolution
    if mode == 1:
        Bbar = np.array([0.0, 0.0, Bbar[2]])
        xu, xd = collinear_xc_adjoint(rho[0], rho[1], gv, gb[2]) if system.xc else (0.0, 0.0)
        z = np.zeros_like(n)
        return np.stack([nbar + xu, nbar + xd, z, z]), Bbar
    if mode == 2:
        if system.xc:
            nbar = nbar + unpolarised_xc_adjoint(n, gv)
        z = np.zeros_like(n)
        return np.stack([nbar, nbar, z, z]), np.zeros(3)
    if system.xc:
        xn, xm = xc_adjoint(n, m, gv, gb)
        nbar = nbar + xn
    else:
        xm = np.zeros_like(m)
    rbar = np.stack([nbar + xm[2], nbar - xm[2], 2.0 * xm[0], -2.0 * xm[1]])
    return rbar, Bbar


def density_adjoint(system, psi, rbar):
    """psibar from the cotangent of rho_v (bilinear in psi)."""
    wf = (system.kw[:, None] * system.occ)[:, :, None, None, None]
    up, dn = psi[:, :, 0], psi[:, :, 1]
    r0, r1, r2, r3 = [rb[None, None] for rb in rbar]
    bu = wf * (2.0 * r0 * up + r2 * dn + 1j * r3 * dn)
    bd = wf * (2.0 * r1 * dn + r2 * up - 1j * r3 * up)
    return np.stack([bu, bd], axis=2)


def grad_V_bilinear(u, v):
    """dRe<u, dV v>/dV_v(r) for the 4-vector potential, summed over spinors."""
    uu, ud, vu, vd = u[:, :, 0], u[:, :, 1], v[:, :, 0], v[:, :, 1]
    g0 = (uu.conj() * vu).real.sum(axis=(0, 1))
    g1 = (ud.conj() * vd).real.sum(axis=(0, 1))
    g2 = 0.5 * (uu.conj() * vd + ud.conj() * vu).real.sum(axis=(0, 1))
    g3 = 0.5 * ((1j * uu.conj() * vd).real - (1j * ud.conj() * vu).real).sum(axis=(0, 1))
    return np.stack([g0, g1, g2, g3])


def grad_A(system, u, v, A):
    """dRe<u, H(A) v>/dA: kinetic (G + k + A) plus the projector-phase derivative."""
    g = np.zeros(3)
    grid = system.grid
    for ik in range(u.shape[0]):
        shift = system.kpts[ik] + A
        vf = grid.fft(v[ik])
        for a in range(3):
            pv = grid.ifft((grid.G[..., a] + shift[a]) * vf)
            g[a] += np.vdot(u[ik], pv).real
        nb = u.shape[1]
        fu = u[ik].reshape(nb, 2, -1)
        fv = v[ik].reshape(nb, 2, -1)
        for at, blocks in zip(system.atoms, system.blocks):
            bt = at.beta * np.exp(-1j * (at.d @ shift))[None, :]
            cu = np.einsum("pr,bsr->bps", bt.conj(), fu[:, :, at.idx]) * grid.dV
            cv = np.einsum("pr,bsr->bps", bt.conj(), fv[:, :, at.idx]) * grid.dV
            for a in range(3):
                dbt = -1j * at.d[:, a][None, :] * bt  # d beta~ / d A_a
                du = np.einsum("pr,bsr->bps", dbt.conj(), fu[:, :, at.idx]) * grid.dV  # <dbeta~|u>
                dv = np.einsum("pr,bsr->bps", dbt.conj(), fv[:, :, at.idx]) * grid.dV
                row = 0
                for l, D in enumerate(blocks):
                    nl = 2 * l + 1
                    sl = slice(row, row + nl)
                    cu_l = cu[:, sl].reshape(nb, -1)
                    cv_l = cv[:, sl].reshape(nb, -1)
                    du_l = du[:, sl].reshape(nb, -1)
                    dv_l = dv[:, sl].reshape(nb, -1)
                    # Re[ sum_r conj(u) dbeta D <beta|v> + sum_r conj(u) beta D <dbeta|v> ]; the
                    # projections carry dV, the outer sum over the array does not
                    g[a] += np.einsum("bp,pq,bq->", du_l.conj(), D, cv_l).real / grid.dV
                    g[a] += np.einsum("bp,pq,bq->", cu_l.conj(), D, dv_l).real / grid.dV
                    row += nl
    return g


def chebyshev_terms(apply_h, x, c, dlt, K):
    T = [x]
    if K >= 1:
        T.append((apply_h(x) - c * x) / dlt)
    for _ in range(2, K + 1):
        T.append(2.0 * (apply_h(T[-1]) - c * T[-1]) / dlt - T[-2])
    return T


def chebyshev_adjoint(apply_h, T, seeds, c, dlt, K, on_pair):
    """Reverse of y_s = sum_k a^s_k T_k for every seed (coefficients a^s, cotangent ybar_s).
    on_pair(S, Tk, factor) receives the pairs entering Re<S, factor dH~ Tk>; returns xbar."""
    def seed(k):
        out = 0.0
        for a, yb in seeds:
            if k < len(a):
                out = out + np.conj(a[k]) * yb
        return out

    S_next2 = 0.0
    S_next = 0.0
    for k in range(K, -1, -1):
        if k == K:
            S = seed(k) + 0.0 * T[0]
        elif k >= 1:
            S = seed(k) + 2.0 * (apply_h(S_next) - c * S_next) / dlt - S_next2
        else:
            S = seed(0) + (apply_h(S_next) - c * S_next) / dlt - S_next2
        if k < K:
            on_pair(S_next, T[k], (2.0 if k >= 1 else 1.0) / dlt)
        S_next2, S_next = S_next, S
    return S


class AdjointRun:
    """Forward ETRS run of ``Oracle`` with every step's internals, then the reverse sweep."""

    def __init__(self, oracle):
        self.o = oracle
        assert oracle.exp_kind == 0 and oracle.sc_tol == 0.0, "adjoint needs Chebyshev and fixed corrector passes"

    def _series(self, V, A):
        s = self.o.s
        return lambda x: s.apply_h(x, V, A)

    def run(self, nsteps, loss_rho_bar):
        o = self.o
        s = o.s
        tab = o.f
        c = 0.5 * (o.emax + o.emin)
        dlt = 0.5 * (o.emax - o.emin)
        aF, _, _ = chebyshev_coefficients(o.dt, o.emin, o.emax, o.K_full)
        aH, _, _ = chebyshev_coefficients(0.5 * o.dt, o.emin, o.emax, o.K_half)
        psis = [o.psi.copy()]
        t0 = o.t
        for _ in range(nsteps):
            o.step()
            psis.append(o.psi.copy())
        rho_T = s.rho_v(psis[-1])
        L = float((loss_rho_bar * rho_T).sum())
        gA_tab = np.zeros_like(tab.A)
        gB_tab = np.zeros_like(tab.B)
        psibar = density_adjoint(s, psis[-1], loss_rho_bar)
        for n in range(nsteps - 1, -1, -1):
            t = t0 + n * o.dt
            t1 = t + o.dt
            A0, B0 = tab.at(t)
            A1, B1 = tab.at(t1)
            w0, w1 = field_weights(tab.t, t), field_weights(tab.t, t1)
            # ---- recompute the step internals
            psi_n = psis[n]
            rho_n = s.rho_v(psi_n)
            V_n, _ = s.potential(rho_n, B0)
            h0 = self._series(V_n, A0)
            T1 = chebyshev_terms(h0, psi_n, c, dlt, max(o.K_full, o.K_half))
            pred = sum(aF[k] * T1[k] for k in range(o.K_full + 1))
            phi = sum(aH[k] * T1[k] for k in range(o.K_half + 1))
            rhos = [s.rho_v(pred)]
            Vs = [s.potential(rhos[0], B1)[0]]
            Ts = [chebyshev_terms(self._series(Vs[0], A1), phi, c, dlt, o.K_half)]
            outs = [sum(aH[k] * Ts[0][k] for k in range(o.K_half + 1))]
            srcs = [pred]
            for _ in range(o.n_sc):
                srcs.append(outs[-1])
                rhos.append(s.rho_v(outs[-1]))
                Vs.append(s.potential(rhos[-1], B1)[0])
                Ts.append(chebyshev_terms(self._series(Vs[-1], A1), phi, c, dlt, o.K_half))
                outs.append(sum(aH[k] * Ts[-1][k] for k in range(o.K_half + 1)))
            # ---- reverse through the corrector passes and the first half step at t+dt
            ybar = psibar
            phibar = 0.0
            gA1 = np.zeros(3)
            gB1 = np.zeros(3)
            for j in range(len(Ts) - 1, -1, -1):
                gV = np.zeros((4,) + rho_n.shape[1:])
                pairs = []

                def on_pair(S, Tk, f, pairs=pairs):
                    pairs.append((S, Tk, f))
                xbar = chebyshev_adjoint(self._series(Vs[j], A1), Ts[j], [(aH, ybar)], c, dlt, o.K_half, on_pair)
                for S, Tk, f in pairs:
                    gV += f * grad_V_bilinear(S, Tk)
                    gA1 += f * grad_A(s, S, Tk, A1)
                phibar = phibar + xbar
                rbar, Bb = potential_adjoint(s, rhos[j], gV)
                gB1 += Bb
                ybar = density_adjoint(s, srcs[j], rbar)  # cotangent of the previous pass (or pred)
            predbar = ybar
            # ---- reverse through series 1 (shared T_k for pred and phi) at time t
            gV = np.zeros((4,) + rho_n.shape[1:])
            gA0 = np.zeros(3)
            pairs = []
            xbar = chebyshev_adjoint(h0, T1, [(aF, predbar), (aH, phibar)], c, dlt, max(o.K_full, o.K_half),
                                     lambda S, Tk, f: pairs.append((S, Tk, f)))
            for S, Tk, f in pairs:
                gV += f * grad_V_bilinear(S, Tk)
                gA0 += f * grad_A(s, S, Tk, A0)
            rbar, gB0 = potential_adjoint(s, rho_n, gV)
            psibar = xbar + density_adjoint(s, psi_n, rbar)
            gA_tab += np.outer(w0, gA0) + np.outer(w1, gA1)
            gB_tab += np.outer(w0, gB0) + np.outer(w1, gB1)
        return L, gA_tab, gB_tab, psibar


def mz_loss_rho_bar(system):
    """dL/drho_v for L = M_z = int (rho_uu - rho_dd) dV."""
    shp = (system.grid.n,) * 3
    dV = system.grid.dV
    return np.stack([np.full(shp, dV), np.full(shp, -dV), np.zeros(shp), np.zeros(shp)])
