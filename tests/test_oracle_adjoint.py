"""Pin of the oracle's discrete adjoint against central finite differences of the oracle's
own forward map (CPU only)."""
import numpy as np
import pytest

from oracle.adjoint import AdjointRun, mz_loss_rho_bar
from tests._systems import make_oracle, parity_system


def _loss(s, psi, times, A, B, dt, nsteps, bounds, n_sc):
    o = make_oracle(s, psi, times, A, B, dt, bounds=bounds, n_sc=n_sc)
    for _ in range(nsteps):
        o.step()
    return float((mz_loss_rho_bar(s) * s.rho_v(o.psi)).sum())


@pytest.mark.parametrize("n_sc,xc", [(1, 1), (0, 0)])
def test_oracle_adjoint_matches_finite_differences(n_sc, xc):
    wl, s, psi = parity_system(n=8, nstates=2, nk=1, lam=0.05, natoms=2, xc=xc, seed=3)
    nst = 2
    dt = 0.1
    times = np.arange(nst + 1) * dt
    rng = np.random.default_rng(4)
    A = rng.normal(scale=0.3, size=(nst + 1, 3))
    B = rng.normal(scale=0.5, size=(nst + 1, 3))
    bounds = (-25.0, 80.0)
    o = make_oracle(s, psi, times, A, B, dt, bounds=bounds, n_sc=n_sc)
    L, gA, gB, _ = AdjointRun(o).run(nst, mz_loss_rho_bar(s))
    assert L == pytest.approx(_loss(s, psi, times, A, B, dt, nst, bounds, n_sc), rel=1e-13)
    h = 1e-5
    for (tab, g, name) in ((A, gA, "A"), (B, gB, "B")):
        for j in range(nst + 1):
            for a in range(3):
                tp, tm = tab.copy(), tab.copy()
                tp[j, a] += h
                tm[j, a] -= h
                if name == "A":
                    fd = (_loss(s, psi, times, tp, B, dt, nst, bounds, n_sc)
                          - _loss(s, psi, times, tm, B, dt, nst, bounds, n_sc)) / (2 * h)
                else:
                    fd = (_loss(s, psi, times, A, tp, dt, nst, bounds, n_sc)
                          - _loss(s, psi, times, A, tm, dt, nst, bounds, n_sc)) / (2 * h)
                scale = np.abs(g).max()
                assert abs(g[j, a] - fd) <= 1e-6 * scale, (name, j, a, g[j, a], fd)


def _loss_w(s, psi, times, A, B, dt, nsteps, bounds, n_sc, w):
    o = make_oracle(s, psi, times, A, B, dt, bounds=bounds, n_sc=n_sc)
    for _ in range(nsteps):
        o.step()
    return float((w * s.rho_v(o.psi)).sum())


@pytest.mark.parametrize("mode", [1, 2])
def test_oracle_adjoint_spin_modes_match_finite_differences(mode):
    """Collinear (sigma_z-only potential, only B_z acts) and spin-unpolarised modes: the adjoint's
    field-table derivatives against central finite differences of the oracle's forward, for a
    loss that weights every component of rho_v(T) with a fixed random field (M_z itself is a
    constant of motion in both modes)."""
    from oracle import System
    from paper_2506_21908_gb300 import synthetic as S
    wl = S.small_parity(n=8, nstates=2, nk=1, lam=0.0, natoms=2, field=False, seed=3)
    wl.spin_mode = mode
    s = System.from_workload(wl)
    psi = S.small_parity_states(wl)
    nst, dt = 2, 0.1
    times = np.arange(nst + 1) * dt
    rng = np.random.default_rng(5)
    A = rng.normal(scale=0.3, size=(nst + 1, 3))
    B = rng.normal(scale=0.5, size=(nst + 1, 3))
    bounds = (-25.0, 80.0)
    w = np.random.default_rng(6).normal(size=(4,) + (wl.n,) * 3)
    o = make_oracle(s, psi, times, A, B, dt, bounds=bounds, n_sc=1)
    L, gA, gB, _ = AdjointRun(o).run(nst, w)
    assert L == pytest.approx(_loss_w(s, psi, times, A, B, dt, nst, bounds, 1, w), rel=1e-13)
    h = 1e-5
    scale = max(np.abs(gA).max(), np.abs(gB).max())
    for tab, g, name in ((A, gA, "A"), (B, gB, "B")):
        for j in range(nst + 1):
            for a in range(3):
                tp, tm = tab.copy(), tab.copy()
                tp[j, a] += h
                tm[j, a] -= h
                args_p = (tp, B) if name == "A" else (A, tp)
                args_m = (tm, B) if name == "A" else (A, tm)
                fd = (_loss_w(s, psi, times, *args_p, dt, nst, bounds, 1, w)
                      - _loss_w(s, psi, times, *args_m, dt, nst, bounds, 1, w)) / (2 * h)
                assert abs(g[j, a] - fd) <= 1e-6 * scale, (name, j, a, g[j, a], fd)
    if mode == 1:
        assert not gB[:, :2].any()
    else:
        assert not gB.any()
