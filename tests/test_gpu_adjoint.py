"""GPU discrete adjoint (tddft_backward) against the oracle's adjoint (itself pinned by finite
differences) and against central finite differences of the GPU forward map.

Target: adjoint gradients within 1e-4 relative of central differences (h = 1e-5, FP64 path);
against the oracle's adjoint the agreement is limited by the oracle's finite-difference LSDA
Hessian (~1e-9 relative), so 1e-6 of the gradient's max-norm is asserted."""
import numpy as np
import pytest

from oracle.adjoint import AdjointRun, mz_loss_rho_bar
from tests._systems import make_oracle, parity_system

pytestmark = pytest.mark.gpu

BOUNDS = (-25.0, 80.0)


def _system(nk=1, xc=1, lam=0.05, n=12, nstates=2, n_sc=1, nst=2, seed=3):
    wl, s, psi = parity_system(n=n, nstates=nstates, nk=nk, lam=lam, natoms=2, xc=xc, seed=seed)
    wl.n_sc = n_sc
    dt = 0.1
    times = np.arange(nst + 1) * dt
    rng = np.random.default_rng(seed + 1)
    A = rng.normal(scale=0.3, size=(nst + 1, 3))
    B = rng.normal(scale=0.5, size=(nst + 1, 3))
    wl.dt = dt
    return wl, s, psi, times, A, B


def _gpu_backward(wl, psi, times, A, B, nst, ckpt=50, precision=0, exp_kind=0, bounds=BOUNDS):
    from paper_2506_21908_gb300 import _lib
    h = _lib.TDDFT.from_workload(wl, precision=precision, e_min=bounds[0], e_max=bounds[1], exp_kind=exp_kind)
    h.set_fields(times, A, B)
    h.set_states(psi)
    dV = float(np.prod(wl.L)) / wl.n ** 3
    seed = np.zeros((4,) + (wl.n,) * 3)
    seed[0], seed[1] = dV, -dV
    L, dA, dB = h.backward(nst, seed, ckpt_every=ckpt)
    _, _, E, _ = h.observables(fields=False)
    h.close()
    return L, dA, dB, E


def _gpu_loss(wl, psi, times, A, B, nst, exp_kind=0):
    from paper_2506_21908_gb300 import _lib
    h = _lib.TDDFT.from_workload(wl, e_min=BOUNDS[0], e_max=BOUNDS[1], exp_kind=exp_kind)
    h.set_fields(times, A, B)
    h.set_states(psi)
    h.step(nst)
    _, _, E, _ = h.observables(fields=False)
    h.close()
    return E["M"][2]


@pytest.mark.parametrize("nk,xc,n_sc", [(1, 1, 1), (2, 1, 0), (1, 0, 2)])
def test_gpu_adjoint_matches_oracle_adjoint(lib, nk, xc, n_sc):
    nst = 2
    wl, s, psi, times, A, B = _system(nk=nk, xc=xc, n_sc=n_sc, nst=nst)
    L, dA, dB, E = _gpu_backward(wl, psi, times, A, B, nst)
    o = make_oracle(s, psi, times, A, B, wl.dt, bounds=BOUNDS, n_sc=n_sc)
    Lo, gA, gB, _ = AdjointRun(o).run(nst, mz_loss_rho_bar(s))
    assert L == pytest.approx(Lo, rel=1e-11, abs=1e-13)
    assert E["M"][2] == pytest.approx(Lo, rel=1e-11, abs=1e-13)
    assert np.abs(dA - gA).max() <= 1e-6 * np.abs(gA).max()
    assert np.abs(dB - gB).max() <= 1e-6 * np.abs(gB).max()


@pytest.mark.parametrize("exp_kind", [0, 2])
def test_gpu_adjoint_matches_finite_differences(lib, exp_kind):
    """Chebyshev and Crank-Nicolson exponentials (the adjoint runs on the series coefficients)."""
    nst = 3
    wl, s, psi, times, A, B = _system(nk=1, xc=1, n_sc=1, nst=nst, seed=9)
    L, dA, dB, _ = _gpu_backward(wl, psi, times, A, B, nst, exp_kind=exp_kind)
    rng = np.random.default_rng(0)
    h = 1e-5
    picks = [(name, int(rng.integers(0, nst + 1)), int(rng.integers(0, 3))) for name in ("A", "B") for _ in range(4)]
    for name, j, a in picks:
        tab = A if name == "A" else B
        tp, tm = tab.copy(), tab.copy()
        tp[j, a] += h
        tm[j, a] -= h
        if name == "A":
            fd = (_gpu_loss(wl, psi, times, tp, B, nst, exp_kind) - _gpu_loss(wl, psi, times, tm, B, nst, exp_kind)) / (2 * h)
            g = dA[j, a]
            scale = np.abs(dA).max()
        else:
            fd = (_gpu_loss(wl, psi, times, A, tp, nst, exp_kind) - _gpu_loss(wl, psi, times, A, tm, nst, exp_kind)) / (2 * h)
            g = dB[j, a]
            scale = np.abs(dB).max()
        # per element: 1e-4 relative, above a floor of 1e-6 of the largest component (the central
        # difference's rounding, ~1e-15 |L| / h, lies far below it)
        assert abs(g - fd) <= 1e-4 * abs(fd) + 1e-6 * scale, (name, j, a, g, fd)


def test_checkpoint_segments_do_not_change_the_gradient(lib):
    nst = 5
    wl, s, psi, times, A, B = _system(nk=1, xc=1, n_sc=1, nst=nst, seed=5)
    L1, dA1, dB1, _ = _gpu_backward(wl, psi, times, A, B, nst, ckpt=2)
    L2, dA2, dB2, _ = _gpu_backward(wl, psi, times, A, B, nst, ckpt=5)
    assert L1 == L2
    assert np.abs(dA1 - dA2).max() <= 1e-13 * np.abs(dA2).max()
    assert np.abs(dB1 - dB2).max() <= 1e-13 * np.abs(dB2).max()


def test_fp32_mixed_adjoint_tracks_fp64(lib):
    nst = 2
    wl, s, psi, times, A, B = _system(nk=1, xc=1, n_sc=1, nst=nst, seed=11)
    L64, dA64, dB64, _ = _gpu_backward(wl, psi, times, A, B, nst, precision=0)
    L32, dA32, dB32, _ = _gpu_backward(wl, psi, times, A, B, nst, precision=1)
    assert L32 == pytest.approx(L64, rel=1e-5)
    assert np.abs(dA32 - dA64).max() <= 1e-3 * np.abs(dA64).max()
    assert np.abs(dB32 - dB64).max() <= 1e-3 * np.abs(dB64).max()


def test_differentiation_workload_envelope_gradient(lib):
    """Differentiation workload shape: the 13-atom cluster at 48^3 with 104 occupied spinors, a
    64-sample laser envelope seeded uniform in [0, 0.01] a.u., L = M_z(T), through the
    torch.autograd wrapper, FP64; horizon of 15 steps with checkpoints every 4 steps (four
    segments, three recomputed), central differences with h = 1e-5 on 8 random samples.  The
    differences are taken between the two m_z fields before the sum (so the rounding of the large
    M_z itself, about 20, does not enter), and each sample must agree to 1e-4 relative above a
    floor of 1e-3 of the largest gradient component."""
    import torch
    from paper_2506_21908_gb300 import _lib, synthetic as S
    from paper_2506_21908_gb300.autograd import MagnetizationFromPulse, PulseBasis, mz_seed
    nst = 15
    wl = S.cluster(n=48, nsteps=nst, laser=False)
    psi0 = S.cluster_states(wl)
    basis = PulseBasis(wl.times, 64, mode="laser", omega=0.057)
    rng = np.random.default_rng(20250624)
    a0 = rng.uniform(0.0, 0.01, 64)
    probe = _lib.TDDFT.from_workload(wl)
    At, Bt = basis.tables(a0)
    probe.set_fields(wl.times, At, Bt)
    probe.set_states(psi0)
    win = probe.info()
    probe.close()
    h = _lib.TDDFT.from_workload(wl, e_min=win["e_min"] - 1.0, e_max=win["e_max"] + 1.0)
    a = torch.tensor(a0, requires_grad=True)
    L = MagnetizationFromPulse.apply(a, h, psi0, basis, nst, mz_seed(48, wl.L), 4)
    L.backward()
    g = a.grad.numpy()
    dV = float(np.prod(wl.L)) / 48 ** 3

    def mz_field(av):
        At, Bt = basis.tables(av)
        h.set_fields(wl.times, At, Bt)
        h.set_states(psi0)
        h.step(nst)
        _, m, E, _ = h.observables()
        return m[2], E["M"][2]

    m0, L0 = mz_field(a0)
    assert float(L.detach()) == pytest.approx(L0, rel=1e-12)
    hstep = 1e-5
    scale = np.abs(g).max()
    for j in rng.choice(64, size=8, replace=False):
        ap, am = a0.copy(), a0.copy()
        ap[j] += hstep
        am[j] -= hstep
        fd = ((mz_field(ap)[0] - mz_field(am)[0]).sum() * dV) / (2 * hstep)
        assert abs(g[j] - fd) <= 1e-4 * abs(fd) + 1e-3 * scale, (j, g[j], fd)
    h.close()


def test_gpu_adjoint_matches_oracle_adjoint_cluster_24(lib):
    """The differentiation workload's cluster geometry at 24^3 (13 atoms with SOC, 16 of its 104
    spinors, laser-like random A and B tables), two steps: the GPU adjoint against the oracle's."""
    from paper_2506_21908_gb300 import synthetic as S
    from oracle import System
    nst = 2
    wl = S.cluster(n=24, nsteps=nst, laser=False)
    psi = np.ascontiguousarray(S.cluster_states(wl)[:, :16])
    wl.occ = wl.occ[:, :16]
    wl.dt = 0.04
    times = np.arange(nst + 1) * wl.dt
    rng = np.random.default_rng(24)
    A = rng.normal(scale=0.2, size=(nst + 1, 3))
    B = rng.normal(scale=0.3, size=(nst + 1, 3))
    s = System.from_workload(wl)
    o = make_oracle(s, psi, times, A, B, wl.dt, n_sc=1)  # spectral window of reading P2
    bounds = (o.emin, o.emax)
    L, dA, dB, E = _gpu_backward(wl, psi, times, A, B, nst, bounds=bounds)
    Lo, gA, gB, _ = AdjointRun(o).run(nst, mz_loss_rho_bar(s))
    assert L == pytest.approx(Lo, rel=1e-11, abs=1e-13)
    assert np.abs(dA - gA).max() <= 1e-6 * np.abs(gA).max()
    assert np.abs(dB - gB).max() <= 1e-6 * np.abs(gB).max()


def test_gpu_adjoint_at_the_xc_thresholds_matches_oracle(lib):
    """Adjoint through the locally collinear XC where m vanishes identically and in vacuum (the
    b_xc = 0 and no-XC branches of reading P8): GPU against the oracle, magnetic field table."""
    from oracle import System
    from tests.test_gpu_parity import xc_threshold_case
    nst = 2
    wl, psi = xc_threshold_case(n=16)
    wl.dt = 0.05
    times = np.arange(nst + 1) * wl.dt
    rng = np.random.default_rng(31)
    A = np.zeros((nst + 1, 3))
    B = rng.normal(scale=0.2, size=(nst + 1, 3))
    s = System.from_workload(wl)
    o = make_oracle(s, psi, times, A, B, wl.dt, n_sc=1)
    bounds = (o.emin, o.emax)
    L, dA, dB, E = _gpu_backward(wl, psi, times, A, B, nst, bounds=bounds)
    Lo, gA, gB, _ = AdjointRun(o).run(nst, mz_loss_rho_bar(s))
    assert L == pytest.approx(Lo, rel=1e-10, abs=1e-13)
    assert np.abs(dB - gB).max() <= 1e-6 * np.abs(gB).max()
    assert np.abs(dA - gA).max() <= 1e-6 * max(np.abs(gA).max(), np.abs(gB).max())
