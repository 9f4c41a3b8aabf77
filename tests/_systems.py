"""Small oracle systems shared by the CPU pin tests (built from the seeded generators)."""
import math

import numpy as np

from oracle import Oracle, System
from oracle.tddft import FieldTable
from paper_2506_21908_gb300 import synthetic as S


def parity_system(n=12, nstates=3, nk=2, lam=0.02, field=True, natoms=2, xc=1, seed=7):
    wl = S.small_parity(n=n, nstates=nstates, nk=nk, lam=lam, field=field, natoms=natoms, seed=seed)
    wl.xc = xc
    return wl, System.from_workload(wl), S.small_parity_states(wl)


def uniform_gas(n=8, L=6.0, nstates=3, theta=0.6, phi=0.2, xc=0):
    """Plane-wave spinors exp(i G_i.r) chi / sqrt(Omega) with a common spin direction; no atoms."""
    s = System([L] * 3, n, np.zeros((0, 3)), np.zeros(0, np.int32), [8.0], [0.8], [1.0], 0,
               np.zeros((1, 1)), np.zeros((1, 1)), 5.0, np.zeros((1, 3)), np.ones(1),
               np.ones((1, nstates)), xc=xc)
    g = s.grid
    chi = S.spinor_along(theta, phi)
    psi = np.empty((1, nstates, 2, n, n, n), np.complex128)
    idx = [(0, 0, 0), (0, 1, 0), (2, 0, 1), (1, 1, 1), (0, 0, 3)]
    for i in range(nstates):
        pw = np.exp(1j * (g.r @ g.G[idx[i]])) / math.sqrt(g.omega)
        psi[0, i, 0] = chi[0] * pw
        psi[0, i, 1] = chi[1] * pw
    return s, psi


def rotate(M, axis, ang):
    k = np.asarray(axis, np.float64)
    k = k / np.linalg.norm(k)
    return M * math.cos(ang) + np.cross(k, M) * math.sin(ang) + k * (k @ M) * (1 - math.cos(ang))


def make_oracle(system, psi, times, A, B, dt, **kw):
    return Oracle(system, FieldTable(times, A, B), dt, psi, **kw)
