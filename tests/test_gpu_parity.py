"""GPU parity: the CUDA library through its C ABI against the FP64 CPU oracle on the
same seeded inputs (element-wise), plus invariants at the full cluster size.

Tolerances (stated target): FP64 |dn|, |dm|, |dpsi| <= 1e-10 relative to the oracle's
max-norm and |dE| <= 1e-8 Ha per step.  FP32-mixed is compared at 2e-5 relative (spinor
storage and FFTs in FP32: a few ulp of 1.2e-7 accumulated over the Chebyshev terms)."""
import math

import numpy as np
import pytest

from oracle import Oracle, System
from oracle.tddft import FieldTable
from paper_2506_21908_gb300 import synthetic as S

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


def run_pair(lib, wl, psi0, nsteps, bounds, precision=0, **kw):
    from paper_2506_21908_gb300 import _lib
    h = _lib.TDDFT.from_workload(wl, precision=precision, e_min=bounds[0], e_max=bounds[1], **kw)
    h.set_fields(wl.times, wl.A, wl.B)
    h.set_states(psi0, 0.0)
    o = Oracle(System.from_workload(wl), FieldTable(wl.times, wl.A, wl.B), wl.dt, psi0, bounds=bounds,
               n_sc=kw.get("n_sc", wl.n_sc), exp_kind=kw.get("exp_kind", 0), exp_order=kw.get("exp_order", 0),
               cheb_tol=kw.get("cheb_tol", 0) or (1e-16 if precision == 0 else 1e-9))
    info = h.info()
    if kw.get("exp_kind", 0) != 2:  # the oracle's Crank-Nicolson is a linear solve, no fixed order
        assert (info["K_full"], info["K_half"]) == (o.K_full, o.K_half)
    rows = []
    for s in range(nsteps + 1):
        if s > 0:
            h.step(1)
            o.step()
        n_g, m_g, E_g, norms_g = h.observables()
        n_o, m_o, E_o, norms_o = o.observables()
        rows.append(dict(n=rel(n_g, n_o), m=rel(m_g, m_o), E=abs(E_g["total"] - E_o["total"]),
                         Eg=E_g, Eo=E_o, norms=np.abs(norms_g - norms_o).max()))
    psi_g = h.get_states()
    h.close()
    return rows, psi_g, o


def test_tiny_config_full_run_fp64(lib):
    """Tiny oracle case in full: 24^3, one atom, 4 spinors, 10 steps of dt = 0.05."""
    wl = S.tiny()
    psi0 = S.tiny_states(wl)
    rows, psi_g, o = run_pair(lib, wl, psi0, wl.nsteps, (-16.0, 96.0))
    for s, r in enumerate(rows):
        assert r["n"] <= 1e-10 and r["m"] <= 1e-10, (s, r["n"], r["m"])
        assert r["E"] <= 1e-8 * max(1, s), (s, r["E"])
        for key in ("kin", "nl", "loc", "H", "xc", "Z", "xc_pot", "N"):
            assert abs(r["Eg"][key] - r["Eo"][key]) <= 1e-8 * max(1, s) + 1e-12 * abs(r["Eo"][key]), key
    assert rel(psi_g, o.psi) <= 1e-10


@pytest.mark.parametrize("n,nstates,nk", [(16, 5, 2), (12, 3, 1), (24, 2, 1)])
def test_multi_atom_soc_kpoints_fields_fp64(lib, n, nstates, nk):
    """Several atoms with SOC, k-points, laser (velocity gauge) and static B; radix-2 and
    radix-3 grids; odd state counts."""
    wl = S.small_parity(n=n, nstates=nstates, nk=nk, natoms=3)
    psi0 = S.small_parity_states(wl)
    rows, psi_g, o = run_pair(lib, wl, psi0, 3, (-20.0, 0.6 * 3 * (math.pi * n / 9.0) ** 2 + 20.0))
    for s, r in enumerate(rows):
        assert r["n"] <= 1e-10 and r["m"] <= 1e-10, (s, r)
        assert r["E"] <= 1e-8 * max(1, s)
    assert rel(psi_g, o.psi) <= 1e-10


def test_auto_spectral_window_and_orders_match_oracle(lib):
    from paper_2506_21908_gb300 import _lib
    wl = S.small_parity(n=16, nstates=3, nk=2, natoms=3)
    psi0 = S.small_parity_states(wl)
    h = _lib.TDDFT.from_workload(wl)
    h.set_fields(wl.times, wl.A, wl.B)
    h.set_states(psi0)
    info = h.info()
    h.close()
    o = Oracle(System.from_workload(wl), FieldTable(wl.times, wl.A, wl.B), wl.dt, psi0)
    assert info["e_min"] == pytest.approx(o.emin, rel=1e-10)
    assert info["e_max"] == pytest.approx(o.emax, rel=1e-10)
    assert (info["K_full"], info["K_half"]) == (o.K_full, o.K_half)


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 2e-5)])
def test_hamiltonian_apply_and_hermiticity(lib, precision, tol):
    from paper_2506_21908_gb300 import _lib
    wl = S.small_parity(n=16, nstates=3, nk=2, natoms=3)
    psi0 = S.small_parity_states(wl)
    h = _lib.TDDFT.from_workload(wl, precision=precision, e_min=-20, e_max=100)
    h.set_fields(wl.times, wl.A, wl.B)
    h.set_states(psi0, 0.1)
    rng = np.random.default_rng(11)
    phi = (rng.normal(size=psi0.shape) + 1j * rng.normal(size=psi0.shape)) * 0.05
    hpsi = h.apply_hamiltonian(psi0)
    hphi = h.apply_hamiltonian(phi)
    V = h.get_potential()
    h.close()
    s = System.from_workload(wl)
    o = Oracle(s, FieldTable(wl.times, wl.A, wl.B), wl.dt, psi0, t0=0.1, bounds=(-20, 100))
    A, _ = o.f.at(0.1)
    assert rel(V, o.V) <= (1e-12 if precision == 0 else 1e-6)
    assert rel(hpsi, s.apply_h(psi0, o.V, A)) <= tol
    assert rel(hphi, s.apply_h(phi, o.V, A)) <= tol
    for ik in range(wl.nk):
        for i in range(wl.nstates):
            a = np.vdot(phi[ik, i], hpsi[ik, i])
            b = np.vdot(hphi[ik, i], psi0[ik, i])
            assert abs(a - b) <= 10 * tol * abs(a)


def test_fp32_mixed_step_tracks_oracle(lib):
    wl = S.small_parity(n=16, nstates=5, nk=2, natoms=3)
    psi0 = S.small_parity_states(wl)
    rows, psi_g, o = run_pair(lib, wl, psi0, 3, (-20.0, 100.0), precision=1)
    for r in rows:
        assert r["n"] <= 2e-5 and r["m"] <= 2e-5, r
        assert r["norms"] <= 1e-5


def test_taylor_variant_fp64(lib):
    wl = S.small_parity(n=12, nstates=3, nk=1, natoms=2)
    wl.dt = 0.01
    psi0 = S.small_parity_states(wl)
    rows, psi_g, o = run_pair(lib, wl, psi0, 2, (-20.0, 100.0), exp_kind=1, exp_order=4)
    for r in rows:
        assert r["n"] <= 1e-10 and r["m"] <= 1e-10
    assert rel(psi_g, o.psi) <= 1e-10


def test_larmor_uniform_gas_gpu_closed_form(lib):
    """No atoms (empty projector set), uniform spinor gas, static B, XC off: M precesses at
    2 mu_B |B| (Eq. magrot), on the GPU, against the closed form."""
    from paper_2506_21908_gb300 import _lib
    from tests._systems import rotate
    n, L = 8, 6.0
    B = np.array([0.4, 0.0, 0.3])
    times = np.arange(11) * 0.1
    g = np.fft.fftfreq(n) * n * 2 * math.pi / L
    iz, iy, ix = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    r = np.stack([ix, iy, iz], -1) * L / n
    chi = S.spinor_along(0.6, 0.2)
    psi = np.empty((1, 3, 2, n, n, n), np.complex128)
    for i, G in enumerate([(0, 0, 0), (g[1], 0, 0), (0, g[2], g[1])]):
        pw = np.exp(1j * (r @ np.array(G))) / math.sqrt(L ** 3)
        psi[0, i, 0], psi[0, i, 1] = chi[0] * pw, chi[1] * pw
    h = _lib.TDDFT([L] * 3, n, np.zeros((0, 3)), np.zeros(0, np.int32), [1.0], [1.0], [1.0], 0, [[0.0]], [[0.0]],
                   1.0, np.zeros((1, 3)), [1.0], np.ones((1, 3)), 0.1, xc=0)
    h.set_fields(times, np.zeros((11, 3)), np.tile(B, (11, 1)))
    h.set_states(psi)
    M0 = h.observables()[2]["M"]
    for k in range(1, 9):
        h.step(1)
        M = h.observables()[2]["M"]
        assert np.allclose(M, rotate(M0, B, np.linalg.norm(B) * k * 0.1), atol=1e-11)
    h.close()


def test_time_reversal_on_gpu(lib):
    from paper_2506_21908_gb300 import _lib
    wl = S.small_parity(n=12, nstates=3, nk=1, natoms=2)
    psi0 = S.small_parity_states(wl)
    kw = dict(e_min=-20, e_max=100, n_sc=60, sc_tol=1e-14)
    h = _lib.TDDFT.from_workload(wl, **kw)
    h.set_fields(wl.times, wl.A, wl.B)
    h.set_states(psi0, 0.0)
    h.step(2)
    psi2 = h.get_states()
    h.close()
    wl.dt = -wl.dt
    h = _lib.TDDFT.from_workload(wl, **kw)
    h.set_fields(wl.times, wl.A, wl.B)
    h.set_states(psi2, 2 * abs(wl.dt))
    h.step(2)
    back = h.get_states()
    h.close()
    assert rel(back, psi0) <= 1e-10


def test_error_paths_on_device(lib):
    from paper_2506_21908_gb300 import _lib
    wl = S.small_parity(n=8, nstates=1, nk=1, natoms=1)
    h = _lib.TDDFT.from_workload(wl)
    with pytest.raises(_lib.TddftError) as e:
        h.step(1)
    assert e.value.status == -4
    with pytest.raises(_lib.TddftError):
        h.get_states()
    h.close()


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 2e-5)])
def test_largest_grid_96(lib, precision, tol):
    """Maximum grid (96^3, the two-factor 8 x 12 FFT passes) in FP64 and FP32-mixed, one atom with
    SOC and one spinor with both components occupied, one step against the oracle."""
    wl = S.small_parity(n=96, nstates=1, nk=1, natoms=1, field=False)
    Lc = 24.0
    wl.L = np.array([Lc, Lc, Lc])
    wl.pos = np.array([[12.1, 11.9, 12.3]])
    wl.r_cut = 3.0
    wl.dt = 0.01
    g = np.fft.fftfreq(96) * 96 * 2 * math.pi / Lc
    rng = np.random.default_rng(2)
    psi0 = np.zeros((1, 1, 2, 96, 96, 96), np.complex128)
    iz, iy, ix = np.meshgrid(np.arange(96), np.arange(96), np.arange(96), indexing="ij")
    r = np.stack([ix, iy, iz], -1) * Lc / 96
    d2 = ((r - wl.pos[0]) ** 2).sum(-1)
    base = np.exp(-d2 / 4.0) * (1 + 0.3 * np.cos(r[..., 0] * g[3]))
    psi0[0, 0, 0] = base * (0.8 + 0.1j)
    psi0[0, 0, 1] = base * (0.3 - 0.5j) * np.exp(1j * r[..., 1] * g[2])
    psi0 /= math.sqrt((np.abs(psi0) ** 2).sum() * Lc ** 3 / 96 ** 3)
    # kinetic maximum 1/2 * 3 (pi / h)^2 = 237 Ha at h = 0.25 bohr
    rows, psi_g, o = run_pair(lib, wl, psi0, 1, (-30.0, 270.0), precision=precision)
    for r_ in rows:
        assert r_["n"] <= tol and r_["m"] <= tol
    assert rel(psi_g, o.psi) <= tol


TC_MODES = [(3, 2e-5), (5, 2e-5), (4, 1e-4), (2, 3e-3)]  # TF32x3, FP16x3, BF16x3, TF32


@pytest.mark.parametrize("proj_mode,tol", TC_MODES)
@pytest.mark.parametrize("nstates", [5, 40])
@pytest.mark.parametrize("n", [16, 32])
def test_tensor_core_projectors_apply_h(lib, proj_mode, tol, nstates, n):
    """Brick-by-brick tcgen05 projector contraction (gather and scatter) in the FP32-mixed
    Hamiltonian against the oracle: bricks of 16 (n = 16) and 32 (n = 32) x 8 x 8 points; 5 states
    give one ragged group of components, 40 states two groups per k-point; two k-points, laser and
    static B; the error budget of the split products is relative to the non-local part."""
    from paper_2506_21908_gb300 import _lib
    wl = S.small_parity(n=n, nstates=nstates, nk=2, natoms=3)
    psi0 = S.small_parity_states(wl)
    h = _lib.TDDFT.from_workload(wl, precision=1, proj_mode=proj_mode, e_min=-20, e_max=100)
    h.set_fields(wl.times, wl.A, wl.B)
    h.set_states(psi0, 0.1)
    hpsi = h.apply_hamiltonian(psi0)
    h.close()
    s = System.from_workload(wl)
    o = Oracle(s, FieldTable(wl.times, wl.A, wl.B), wl.dt, psi0, t0=0.1, bounds=(-20, 100))
    A, _ = o.f.at(0.1)
    ref = s.apply_h(psi0, o.V, A)
    vnl = np.stack([s.apply_nonlocal(psi0[ik], wl.kpts[ik] + A) for ik in range(wl.nk)])
    # the error budget is set by the non-local part
    assert np.abs(hpsi - ref).max() <= tol * np.abs(vnl).max() + 2e-5 * np.abs(ref).max()


def test_tensor_core_projectors_step_parity(lib):
    wl = S.small_parity(n=16, nstates=5, nk=2, natoms=3)
    psi0 = S.small_parity_states(wl)
    rows, psi_g, o = run_pair(lib, wl, psi0, 2, (-20.0, 100.0), precision=1, proj_mode=3)
    for r in rows:
        assert r["n"] <= 2e-5 and r["m"] <= 2e-5, r


def test_atom_moments_match_oracle_on_symmetric_cluster(lib):
    """Voronoi per-atom moments on the icosahedral cluster at 24^3 (many grid points are
    equidistant from several atoms: ties must resolve identically) against the oracle."""
    from paper_2506_21908_gb300 import _lib
    wl = S.cluster(n=24, nsteps=2, laser=False)
    psi0 = S.cluster_states(wl)
    h = _lib.TDDFT.from_workload(wl)
    h.set_states(psi0)
    M, N = h.atom_moments()
    _, _, E, _ = h.observables(fields=False)
    h.close()
    s = System.from_workload(wl)
    Mo, No = s.atom_moments(s.rho_v(psi0))
    assert np.abs(M - Mo).max() <= 1e-10 * np.abs(Mo).max()
    assert np.abs(N - No).max() <= 1e-10 * np.abs(No).max()
    assert np.allclose(M.sum(axis=0), E["M"], atol=1e-10)


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 2e-5)])
def test_torques_match_oracle(lib, precision, tol):
    """Global spin torques (Eq. GMT, Eq. magrot, Eq. SOtorque) at the current state against the
    oracle's commutator formula, with SOC, two k-points, laser and static B."""
    from paper_2506_21908_gb300 import _lib
    wl = S.small_parity(n=16, nstates=3, nk=2, natoms=3, lam=0.3)
    psi0 = S.small_parity_states(wl)
    h = _lib.TDDFT.from_workload(wl, precision=precision, e_min=-20, e_max=100)
    h.set_fields(wl.times, wl.A, wl.B)
    h.set_states(psi0, 0.1)
    tq = h.torques()
    h.step(1)
    tq1 = h.torques()
    psi1 = h.get_states()
    h.close()
    s = System.from_workload(wl)
    f = FieldTable(wl.times, wl.A, wl.B)
    for t, psi, g in ((0.1, psi0, tq), (0.1 + wl.dt, psi1, tq1)):
        A, B = f.at(t)
        rho = s.rho_v(psi)
        V, parts = s.potential(rho, B)
        ref = s.torques(psi, rho, V, parts, A, B)
        scale = np.abs(ref["total"]).max()
        for key in ("soc", "zeeman", "total"):
            assert np.abs(g[key] - ref[key]).max() <= tol * scale, (key, g[key], ref[key])
        assert np.abs(g["xc"]).max() <= 1e-10 * scale


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 2e-5)])
def test_collinear_and_unpolarised_modes_match_oracle(lib, mode, precision, tol):
    """sigma_z-only (Eq. HSDFT) and spin-unpolarised modes of the same step, with tilted spinors,
    two k-points, laser and a static field with transverse parts (ignored by both modes)."""
    wl = S.small_parity(n=16, nstates=3, nk=2, lam=0.0, natoms=2)
    wl.spin_mode = mode
    psi0 = S.small_parity_states(wl)
    rows, psi_g, o = run_pair(lib, wl, psi0, 2, (-20.0, 100.0), precision=precision)
    for s_, r in enumerate(rows):
        assert r["n"] <= tol and r["m"] <= tol, (s_, r["n"], r["m"])
        assert r["E"] <= (1e-8 * max(1, s_) if precision == 0 else 1e-4), (s_, r["E"])
        assert abs(r["Eg"]["Z"] - r["Eo"]["Z"]) <= 1e-8 + tol * abs(r["Eo"]["Z"])
    assert rel(psi_g, o.psi) <= (1e-10 if precision == 0 else 2e-5)


def test_magnetic_pulse_uniform_gas_gpu_closed_form(lib):
    """The paper's magnetic pulse on a uniform spinor gas (no atoms, XC off) on the GPU: M turns
    about eps by 2 mu_B times the trapezoidal integral of the field table (Eq. magrot)."""
    from paper_2506_21908_gb300 import _lib
    from tests._systems import rotate
    n, L, dt, nst = 8, 6.0, 0.1, 30
    eps = np.array([1.0, 0.0, 1.0]) / math.sqrt(2.0)
    times, A, Bt = S.magnetic_pulse_table(nst, dt, amp=0.6, eps=eps, omega0=2.0, t0=0.45, tau=0.8, phi=0.3,
                                          delta_B=0.2 * eps)
    b = Bt @ eps
    g = np.fft.fftfreq(n) * n * 2 * math.pi / L
    iz, iy, ix = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    r = np.stack([ix, iy, iz], -1) * L / n
    chi = S.spinor_along(0.6, 0.2)
    psi = np.empty((1, 3, 2, n, n, n), np.complex128)
    for i, G in enumerate([(0, 0, 0), (g[1], 0, 0), (0, g[2], g[1])]):
        pw = np.exp(1j * (r @ np.array(G))) / math.sqrt(L ** 3)
        psi[0, i, 0], psi[0, i, 1] = chi[0] * pw, chi[1] * pw
    for precision, tol in ((0, 1e-11), (1, 1e-5)):
        h = _lib.TDDFT([L] * 3, n, np.zeros((0, 3)), np.zeros(0, np.int32), [1.0], [1.0], [1.0], 0, [[0.0]],
                       [[0.0]], 1.0, np.zeros((1, 3)), [1.0], np.ones((1, 3)), dt, xc=0, precision=precision)
        h.set_fields(times, A, Bt)
        h.set_states(psi)
        M0 = h.observables()[2]["M"]
        theta = 0.0
        for k in range(1, nst + 1):
            h.step(1)
            theta += 0.5 * dt * (b[k - 1] + b[k])  # 2 mu_B = 1
            M = h.observables()[2]["M"]
            assert np.allclose(M, rotate(M0, eps, theta), atol=tol), (precision, k)
        h.close()


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 2e-5)])
def test_crank_nicolson_step_matches_oracle(lib, precision, tol):
    """Crank-Nicolson exponentials in the ETRS step: the library's Chebyshev expansion of the
    Cayley transform against the oracle's GMRES solve of (1 + i tau H/2) x = (1 - i tau H/2) psi."""
    wl = S.small_parity(n=16, nstates=3, nk=2, natoms=3)
    psi0 = S.small_parity_states(wl)
    rows, psi_g, o = run_pair(lib, wl, psi0, 2, (-20.0, 100.0), precision=precision, exp_kind=2)
    for s_, r in enumerate(rows):
        assert r["n"] <= tol and r["m"] <= tol, (s_, r["n"], r["m"])
        assert r["E"] <= (1e-8 * max(1, s_) if precision == 0 else 1e-4)
        assert r["norms"] <= (1e-12 if precision == 0 else 1e-5)
    assert rel(psi_g, o.psi) <= (1e-10 if precision == 0 else 2e-5)


@pytest.mark.parametrize("precision", [0, 1])
def test_pinned_host_buffers_match_pageable(lib, precision):
    """set_states / get_states from page-locked host memory (read and written by the conversion
    kernels through the mapped address) give the same bits as pageable numpy arrays."""
    import torch
    from paper_2506_21908_gb300 import _lib
    wl = S.small_parity(n=16, nstates=3, nk=2, natoms=2)
    psi0 = S.small_parity_states(wl)
    outs = []
    for pinned in (False, True):
        h = _lib.TDDFT.from_workload(wl, precision=precision, e_min=-20, e_max=100)
        h.set_fields(wl.times, wl.A, wl.B)
        src = torch.from_numpy(psi0.copy()).pin_memory() if pinned else psi0.copy()
        h.set_states(src.numpy() if pinned else src, 0.0)
        h.step(1)
        dst = torch.empty(psi0.shape, dtype=torch.complex128).pin_memory() if pinned else None
        got = h.get_states(dst.numpy() if pinned else None)
        outs.append(np.array(got))
        h.close()
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("precision", [0, 1])
def test_gather_overlap_gives_identical_bits(lib, precision, monkeypatch):
    """The projector gather on its second stream (beside the FFT passes) against the serial
    order (TDDFT_NO_OVERLAP=1): same kernels on the same data, so the states agree bit for bit."""
    from paper_2506_21908_gb300 import _lib
    wl = S.small_parity(n=16, nstates=5, nk=2, natoms=3)
    psi0 = S.small_parity_states(wl)
    outs = []
    for flag in ("0", "1"):
        monkeypatch.setenv("TDDFT_NO_OVERLAP", flag)
        h = _lib.TDDFT.from_workload(wl, precision=precision, e_min=-20, e_max=100)
        h.set_fields(wl.times, wl.A, wl.B)
        h.set_states(psi0, 0.0)
        h.step(3)
        outs.append(h.get_states())
        h.close()
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("n", [16, 24, 32, 48, 64])
def test_bulk_copy_xy_pass_gives_identical_bits(lib, n, monkeypatch):
    """FP32 xy passes fed by bulk asynchronous copies (double-buffered planes in shared memory)
    against the register-fed passes (TDDFT_NO_TMA=1): the same DFT arithmetic in the same order,
    so the states agree bit for bit, and no copy wait reports a timeout."""
    from paper_2506_21908_gb300 import _lib
    wl = S.small_parity(n=n, nstates=3, nk=2, natoms=2)
    psi0 = S.small_parity_states(wl)
    outs = []
    for flag in ("0", "1"):
        monkeypatch.setenv("TDDFT_NO_TMA", flag)
        h = _lib.TDDFT.from_workload(wl, precision=1)
        h.set_fields(wl.times, wl.A, wl.B)
        h.set_states(psi0, 0.0)
        h.step(2)
        h.observables()
        outs.append(h.get_states())
        h.close()
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("precision,tol", [(0, 1e-13), (1, 1e-6)])
def test_spinor_pair_epilogue_matches_single_spinor_form(lib, precision, tol, monkeypatch):
    """Epilogue threads holding one grid point of two spinors (the projector scatter walks the
    point's entries once for the pair) against two points of one spinor (TDDFT_NO_EPI_PAIRS=1):
    the same arithmetic per spinor and point, so the states agree to rounding."""
    from paper_2506_21908_gb300 import _lib
    wl = S.small_parity(n=16, nstates=4, nk=2, natoms=3)
    psi0 = S.small_parity_states(wl)
    outs = []
    for flag in ("0", "1"):
        monkeypatch.setenv("TDDFT_NO_EPI_PAIRS", flag)
        h = _lib.TDDFT.from_workload(wl, precision=precision)
        h.set_fields(wl.times, wl.A, wl.B)
        h.set_states(psi0, 0.0)
        h.step(3)
        outs.append(h.get_states())
        h.close()
    assert rel(outs[0], outs[1]) <= tol


@pytest.mark.parametrize("precision", [0, 1])
def test_complex64_state_calls(lib, precision):
    """tddft_set_states_c64 / tddft_get_states_c64: an FP32-mixed handle keeps complex64 spinors
    as they are, an FP64 handle widens them exactly; loading complex64 states (numpy, page-locked
    and device tensors) and loading the same values as complex128 give the same states and the
    same step."""
    import torch
    from paper_2506_21908_gb300 import _lib
    wl = S.small_parity(n=16, nstates=3, nk=2, natoms=2)
    psi64 = S.small_parity_states(wl).astype(np.complex64)
    outs = []
    for src in (psi64, psi64.astype(np.complex128), torch.from_numpy(psi64).pin_memory(),
                torch.from_numpy(psi64).to("cuda")):
        h = _lib.TDDFT.from_workload(wl, precision=precision)
        h.set_fields(wl.times, wl.A, wl.B)
        h.set_states(src, 0.0)
        assert np.array_equal(h.get_states(), psi64.astype(np.complex128))
        assert np.array_equal(h.get_states(np.empty(psi64.shape, np.complex64)), psi64)
        h.step(2)
        outs.append((h.get_states(), h.get_states(np.empty(psi64.shape, np.complex64))))
        h.close()
    for o128, o64 in outs[1:]:
        assert np.array_equal(o128, outs[0][0]) and np.array_equal(o64, outs[0][1])
    assert np.array_equal(outs[0][1], outs[0][0].astype(np.complex64))


def test_observables_without_energies_match_full_call(lib):
    """tddft_observables with E, M and norms NULL skips the energy passes; n and m agree bit for
    bit with the full call."""
    from paper_2506_21908_gb300 import _lib
    wl = S.small_parity(n=16, nstates=3, nk=2, natoms=2)
    psi0 = S.small_parity_states(wl)
    h = _lib.TDDFT.from_workload(wl, precision=1)
    h.set_fields(wl.times, wl.A, wl.B)
    h.set_states(psi0, 0.0)
    h.step(2)
    n_full, m_full, E, _ = h.observables()
    n = np.empty_like(n_full)
    m = np.empty_like(m_full)
    assert h.lib.tddft_observables(h.h, _lib._ptr(n), _lib._ptr(m), None, None, None) == 0
    h.close()
    assert np.array_equal(n, n_full) and np.array_equal(m, m_full)
    assert np.isfinite(E["total"])


@pytest.mark.parametrize("lmax", [0, 1])
@pytest.mark.parametrize("nstates", [3, 4])
@pytest.mark.parametrize("precision", [0, 1])
def test_lower_angular_momentum_projectors(lib, lmax, nstates, precision):
    """Projectors up to l = 0 and l = 1 (1 and 4 real harmonics per spin): H apply against the
    oracle, and three steps against the oracle's n and m, with an odd (two points of one spinor
    per epilogue thread) and an even (one point of two spinors) number of states."""
    from paper_2506_21908_gb300 import _lib
    wl = S.small_parity(n=16, nstates=nstates, nk=2, natoms=3, lmax=lmax)
    psi0 = S.small_parity_states(wl)
    h = _lib.TDDFT.from_workload(wl, precision=precision, e_min=-20, e_max=100)
    h.set_fields(wl.times, wl.A, wl.B)
    h.set_states(psi0, 0.1)
    hpsi = h.apply_hamiltonian(psi0)
    h.close()
    s = System.from_workload(wl)
    o = Oracle(s, FieldTable(wl.times, wl.A, wl.B), wl.dt, psi0, t0=0.1, bounds=(-20, 100))
    A, _ = o.f.at(0.1)
    assert rel(hpsi, s.apply_h(psi0, o.V, A)) <= (1e-12 if precision == 0 else 2e-5)
    rows, psi_g, o = run_pair(lib, wl, psi0, 3, (-20.0, 100.0), precision=precision)
    tol = 1e-10 if precision == 0 else 2e-5
    for r in rows:
        assert r["n"] <= tol and r["m"] <= tol, r


@pytest.mark.parametrize("proj_mode,tol", [(5, 2e-5), (3, 2e-5), (4, 1e-4)])
def test_tensor_core_projectors_step_matches_oracle(lib, proj_mode, tol):
    """Two ETRS steps with the tensor-core projector contraction (32^3, four SOC atoms, two
    k-points, laser and static B) against the FP64 oracle: n, m and psi."""
    wl = S.small_parity(n=32, nstates=6, nk=2, natoms=4)
    psi0 = S.small_parity_states(wl)
    rows, psi_g, o = run_pair(lib, wl, psi0, 2, (-20.0, 400.0), precision=1, proj_mode=proj_mode)
    for r in rows:
        assert r["n"] <= tol and r["m"] <= tol, (r["n"], r["m"])
    assert rel(psi_g, o.psi) <= tol


def xc_threshold_case(n=24):
    """States whose magnetisation vanishes identically over most of the cell: an orbital phi in
    spin up and the same phi in spin down with equal occupation (m = 0 wherever the third state is
    negligible), a third narrow orbital with a tilted spin and half occupation, and vacuum
    (n < 1e-14) near the cell corners.  No SOC and no field, so the first two states stay exact
    spin partners: the locally collinear XC takes its |m| <= 1e-14 branch (b_xc = 0) in most of the
    cell and its n < 1e-14 branch (no XC) in the corners (reading P8)."""
    wl = S.small_parity(n=n, nstates=3, nk=1, natoms=1, lam=0.0, field=False, seed=11)
    Lc = 12.0
    wl.L = np.array([Lc, Lc, Lc])
    wl.pos = np.array([[6.1, 5.9, 6.0]])
    wl.r_cut = 4.0
    wl.occ = np.array([[1.0, 1.0, 0.5]])
    g = np.arange(n) * Lc / n
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")

    def gauss(c, s):
        return np.exp(-((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2) / (2 * s * s))

    dV = Lc ** 3 / n ** 3
    phi = gauss((6.0, 6.0, 6.0), 1.2) * (1.0 + 0.3j * np.cos(2 * np.pi * X / Lc))
    phi /= np.sqrt((np.abs(phi) ** 2).sum() * dV)
    chi = (np.cos(0.5), np.sin(0.5) * np.exp(0.4j))
    phi3 = gauss((5.0, 6.5, 6.3), 0.7).astype(np.complex128)
    phi3 -= (np.vdot(phi, phi3) * dV) * phi
    phi3 /= np.sqrt((np.abs(phi3) ** 2).sum() * dV)
    psi = np.zeros((1, 3, 2, n, n, n), np.complex128)
    psi[0, 0, 0] = phi
    psi[0, 1, 1] = phi
    psi[0, 2, 0] = chi[0] * phi3
    psi[0, 2, 1] = chi[1] * phi3
    return wl, psi


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 2e-5)])
def test_xc_threshold_branches_match_oracle(lib, precision, tol):
    from oracle import xc as oxc
    wl, psi0 = xc_threshold_case()
    s = System.from_workload(wl)
    n0, m0 = s.n_m(s.rho_v(psi0))
    mag = np.sqrt((m0 ** 2).sum(axis=0))
    # both branches are taken at many points, and the ordinary path elsewhere
    assert ((mag <= oxc.M_THR) & (n0 >= oxc.N_THR)).mean() > 0.02
    assert (n0 < oxc.N_THR).mean() > 0.05 and (mag > oxc.M_THR).mean() > 0.3
    rows, psi_g, o = run_pair(lib, wl, psi0, 2, (-25.0, 120.0), precision=precision)
    for r in rows:
        assert r["n"] <= tol and r["m"] <= tol, (r["n"], r["m"])
    assert rel(psi_g, o.psi) <= tol


def test_fused_tensor_core_epilogue_matches_separate_kernels_and_oracle(lib, monkeypatch):
    """With the tensor-core projectors the Chebyshev epilogue runs inside the scatter kernel; the
    separate scatter + pointwise epilogue (TDDFT_NO_EPI_FUSE=1) computes the same arithmetic.  The
    cluster geometry at 32^3 leaves bricks that no projector sphere reaches (those take the fused
    path with V_NL = 0); both forms agree with each other and with the oracle."""
    from paper_2506_21908_gb300 import _lib
    wl = S.cluster(n=32, nsteps=4)
    psi0 = np.ascontiguousarray(S.cluster_states(wl)[:, :10])
    wl.occ = wl.occ[:, :10]
    outs = []
    for flag in ("0", "1"):
        monkeypatch.setenv("TDDFT_NO_EPI_FUSE", flag)
        h = _lib.TDDFT.from_workload(wl, precision=1, proj_mode=5, e_min=-30.0, e_max=60.0)
        h.set_fields(wl.times, wl.A, wl.B)
        h.set_states(psi0, 0.0)
        h.step(2)
        h.observables()
        outs.append(h.get_states())
        h.close()
    assert rel(outs[0], outs[1]) <= 1e-6
    o = Oracle(System.from_workload(wl), FieldTable(wl.times, wl.A, wl.B), wl.dt, psi0, bounds=(-30.0, 60.0),
               n_sc=1, cheb_tol=1e-9)
    o.step()
    o.step()
    assert rel(outs[0], o.psi) <= 2e-5
