"""Oracle: locally collinear adiabatic LSDA exchange-correlation (FP64, plain numpy).

Paper passages: adiabatic approximation (Sec. 2.5, Eqs. ALSDA1/ALSDA2), locally
collinear approximation (Eqs. LC+ALDA2 and LC+ALDA: vbar_xc = vbar^LSDA[n,|m|],
b_xc = b^LSDA[n,|m|] m/|m|, b_xc = 0 where |m| vanishes), spin-matrix form of the
XC potential (Sec. 3.3).  b_xc = (v^0 - v^1)/2 and vbar = (v^0 + v^1)/2 as in Sec. 2.1.

The paper only says "LDA"; the reading taken here is Slater exchange with the
exact spin scaling plus the Perdew-Wang 1992 correlation fit.  The PW92 rows
are (A, alpha1, beta1, beta2, beta3, beta4) with p = 1.
Thresholds (paper: "below a given threshold", value unstated): n < 1e-14 gives
zero potential and energy; |m| <= 1e-14 gives b_xc = 0; zeta is clamped to 1.
"""
import math

import numpy as np

N_THR = 1e-14
M_THR = 1e-14

PW92_EC0 = (0.031091, 0.21370, 7.5957, 3.5876, 1.6382, 0.49294)
PW92_EC1 = (0.015545, 0.20548, 14.1189, 6.1977, 3.3662, 0.62517)
PW92_MAC = (0.016887, 0.11125, 10.357, 3.6231, 0.88026, 0.49671)  # gives -alpha_c
FPP0 = 1.709921


def pw92_G(rs, prm):
    """PW92 interpolation G(rs) and dG/drs."""
    A, a1, b1, b2, b3, b4 = prm
    srs = np.sqrt(rs)
    Q0 = -2.0 * A * (1.0 + a1 * rs)
    Q1 = 2.0 * A * (b1 * srs + b2 * rs + b3 * rs * srs + b4 * rs * rs)
    Q1p = A * (b1 / srs + 2.0 * b2 + 3.0 * b3 * srs + 4.0 * b4 * rs)
    lg = np.log1p(1.0 / Q1)
    G = Q0 * lg
    dG = -2.0 * A * a1 * lg - Q0 * Q1p / (Q1 * Q1 + Q1)
    return G, dG


def fzeta(z):
    den = 2.0 ** (4.0 / 3.0) - 2.0
    f = ((1.0 + z) ** (4.0 / 3.0) + (1.0 - z) ** (4.0 / 3.0) - 2.0) / den
    fp = (4.0 / 3.0) * ((1.0 + z) ** (1.0 / 3.0) - (1.0 - z) ** (1.0 / 3.0)) / den
    return f, fp


def pw92_correlation(rs, zeta):
    """eps_c(rs, zeta), d eps_c / d rs, d eps_c / d zeta (Hartree per electron)."""
    ec0, dec0 = pw92_G(rs, PW92_EC0)
    ec1, dec1 = pw92_G(rs, PW92_EC1)
    mac, dmac = pw92_G(rs, PW92_MAC)
    ac, dac = -mac, -dmac
    f, fp = fzeta(zeta)
    z3 = zeta ** 3
    z4 = zeta ** 4
    ec = ec0 + ac * f * (1.0 - z4) / FPP0 + (ec1 - ec0) * f * z4
    d_rs = dec0 + dac * f * (1.0 - z4) / FPP0 + (dec1 - dec0) * f * z4
    d_z = ac / FPP0 * (fp * (1.0 - z4) - 4.0 * z3 * f) + (ec1 - ec0) * (fp * z4 + 4.0 * z3 * f)
    return ec, d_rs, d_z


def lsda(nu, nd):
    """Collinear LSDA on spin densities (nu, nd) >= 0 with nu + nd > 0.

    Returns (energy density per volume, v_up, v_dn)."""
    nu = np.asarray(nu, np.float64)
    nd = np.asarray(nd, np.float64)
    n = nu + nd
    cx = 0.75 * (6.0 / math.pi) ** (1.0 / 3.0)
    ex = -cx * (nu ** (4.0 / 3.0) + nd ** (4.0 / 3.0))
    vxu = -(6.0 * nu / math.pi) ** (1.0 / 3.0)
    vxd = -(6.0 * nd / math.pi) ** (1.0 / 3.0)
    rs = (3.0 / (4.0 * math.pi * n)) ** (1.0 / 3.0)
    zeta = np.clip((nu - nd) / n, -1.0, 1.0)
    ec, d_rs, d_z = pw92_correlation(rs, zeta)
    common = ec - rs / 3.0 * d_rs
    vcu = common - (zeta - 1.0) * d_z
    vcd = common - (zeta + 1.0) * d_z
    return ex + n * ec, vxu + vcu, vxd + vcd


def noncollinear_xc(n, m):
    """Locally collinear XC on (n, m): returns (e_xc per volume, vbar, b_xc[3]).

    m has shape (3, ...) like n.  |m| is clamped to n (zeta <= 1)."""
    n = np.asarray(n, np.float64)
    m = np.asarray(m, np.float64)
    e = np.zeros_like(n)
    vbar = np.zeros_like(n)
    b = np.zeros_like(m)
    mag = np.sqrt((m * m).sum(axis=0))
    ok = n >= N_THR
    s = np.minimum(mag, n)
    nu = 0.5 * (n + s)
    nd = 0.5 * (n - s)
    if np.any(ok):
        ee, vu, vd = lsda(nu[ok], nd[ok])
        e[ok] = ee
        vbar[ok] = 0.5 * (vu + vd)
        bmag = np.zeros_like(n)
        bmag[ok] = 0.5 * (vu - vd)
        dirok = ok & (mag > M_THR)
        safe = np.where(dirok, mag, 1.0)
        b = np.where(dirok[None], bmag[None] * m / safe[None], 0.0)
    return e, vbar, b


def collinear_xc(nu, nd):
    """Collinear LSDA on the spin-channel densities (Eq. SDFT / Eq. HSDFT): returns (e_xc per
    volume, vbar = (v_up + v_dn)/2, b_z = (v_up - v_dn)/2); the field is along the quantisation
    axis only."""
    nu = np.asarray(nu, np.float64)
    nd = np.asarray(nd, np.float64)
    n = nu + nd
    e = np.zeros_like(n)
    vbar = np.zeros_like(n)
    bz = np.zeros_like(n)
    ok = n >= N_THR
    if np.any(ok):
        ee, vu, vd = lsda(nu[ok], nd[ok])
        e[ok] = ee
        vbar[ok] = 0.5 * (vu + vd)
        bz[ok] = 0.5 * (vu - vd)
    return e, vbar, bz


def unpolarised_xc(n):
    """Spin-unpolarised LDA, n_up = n_dn = n/2: returns (e_xc per volume, v_xc)."""
    n = np.asarray(n, np.float64)
    e = np.zeros_like(n)
    v = np.zeros_like(n)
    ok = n >= N_THR
    if np.any(ok):
        ee, vu, _ = lsda(0.5 * n[ok], 0.5 * n[ok])
        e[ok] = ee
        v[ok] = vu
    return e, v
