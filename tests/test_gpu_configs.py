"""GPU checks at the full sizes of the benchmark configurations: the magnetic cluster (64^3,
104 spinors; the bench workload, in the launch configuration bench.py times), the bcc supercell
(48^3, 8 k-points x 128 spinors, static B plus laser) and the large supercell's grid and atoms
(96^3, 128 atoms with SOC; 16 of its 1024 spinors, so that the host-side inputs stay small).

The oracle cannot propagate these systems with all their spinors in seconds, so the checks take
outputs it computes one spinor at a time: the potential from the density of all spinors, H psi on
sampled spinors (Eq. HNC-SDFT with the 2x2 potential and the L.S projectors), and one full ETRS
step of the large and bcc supercells at full grid and with all atoms (and all 8 k-points) on a few
spinors, compared element by element.  A full step with all spinors is checked through properties
that hold at any size: norm and charge conservation, and agreement of the FP32-mixed step with the
FP64 step (itself pinned element-wise to the oracle) within the metric's |dM| <= 1e-5 mu_B per
atom."""
import numpy as np
import pytest

from oracle import System
from oracle.tddft import FieldTable
from paper_2506_21908_gb300 import synthetic as S

pytestmark = pytest.mark.gpu

T0 = 0.3  # a time inside the field tables with A(t) != 0


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


def oracle_potential(wl, psi, t0):
    s = System.from_workload(wl)
    f = FieldTable(wl.times, wl.A, wl.B)
    A, B = f.at(t0)
    V, _ = s.potential(s.rho_v(psi), B)
    return s, V, A


def gpu_apply(wl, psi, precision, bounds, t0=T0, proj_mode=None):
    from paper_2506_21908_gb300 import _lib
    h = _lib.TDDFT.from_workload(wl, precision=precision, proj_mode=proj_mode, e_min=bounds[0], e_max=bounds[1])
    h.set_fields(wl.times, wl.A, wl.B)
    h.set_states(psi, t0)
    hpsi = h.apply_hamiltonian(psi)
    V = h.get_potential()
    h.close()
    return hpsi, V


@pytest.fixture(scope="module")
def cluster_case():
    wl = S.cluster(64, nsteps=8)
    psi = S.cluster_states(wl)
    s, V, A = oracle_potential(wl, psi, T0)
    sample = [0, 51, 103]
    ref = s.apply_h(psi[:, sample], V, A)
    return wl, psi, V, sample, ref


@pytest.mark.parametrize("precision,tol_h,tol_v", [(0, 1e-11, 1e-11), (1, 2e-5, 1e-6)])
def test_cluster_full_size_potential_and_sampled_h(lib, cluster_case, precision, tol_h, tol_v):
    wl, psi, V, sample, ref = cluster_case
    hpsi, Vg = gpu_apply(wl, psi, precision, (-20.0, 140.0))
    assert rel(Vg, V) <= tol_v
    assert rel(hpsi[:, sample], ref) <= tol_h


def test_cluster_full_size_step_mixed_vs_fp64(lib, cluster_case):
    from paper_2506_21908_gb300 import _lib
    wl, psi, _, _, _ = cluster_case
    out = {}
    for prec in (_lib.FP64, _lib.FP32_MIXED):
        h = _lib.TDDFT.from_workload(wl, precision=prec)
        h.set_fields(wl.times, wl.A, wl.B)
        h.set_states(psi, 0.0)
        _, _, E0, _ = h.observables(fields=False)
        h.step(2)
        n, m, E, norms = h.observables()
        h.close()
        out[prec] = (n, m, E, norms, E0)
    n64, m64, E64, nrm64, E064 = out[_lib.FP64]
    n32, m32, E32, nrm32, _ = out[_lib.FP32_MIXED]
    assert np.abs(nrm64 - 1.0).max() <= 1e-11
    assert np.abs(nrm32 - 1.0).max() <= 1e-5
    assert abs(E64["N"] - E064["N"]) <= 1e-9 * E064["N"]
    dM = float(np.linalg.norm(E32["M"] - E64["M"])) / len(wl.pos)
    assert dM <= 1e-5
    assert rel(n32, n64) <= 1e-5
    assert rel(m32, m64) <= 1e-4
    assert abs(E32["total"] - E64["total"]) <= 1e-4


@pytest.fixture(scope="module")
def cluster_enl(cluster_case):
    """The oracle's nonlocal energy sum_i f_i <psi_i|V_NL|psi_i> of the cluster at t = 0."""
    wl, psi, _, _, _ = cluster_case
    s = System.from_workload(wl)
    A, _ = FieldTable(wl.times, wl.A, wl.B).at(0.0)
    wf = s.kw[0] * s.occ[0]
    nk = s.apply_nonlocal(psi[0], s.kpts[0] + A)
    return float(sum(wf[i] * np.vdot(psi[0, i], nk[i]).real for i in range(psi.shape[1])) * s.grid.dV)


# The tensor cores round each accumulation of a product into the FP32 accumulator with a bias
# toward zero; over the hundreds of MMAs of one brick sum this took a relative 1e-5 off every
# projection (E_nl low by 1e-5 relative with FP16 x3, 1.4e-5 with TF32 x3), which the grouped
# accumulation removes down to ~1.5e-6.  The tolerances are the bound for each contraction.
@pytest.mark.parametrize("precision,proj_mode,tol", [(0, None, 1e-10), (1, 1, 1e-6), (1, 3, 4e-6), (1, 4, 1e-5),
                                                     (1, 5, 4e-6)])
def test_cluster_nonlocal_energy_matches_oracle(lib, cluster_case, cluster_enl, precision, proj_mode, tol):
    from paper_2506_21908_gb300 import _lib
    wl, psi, _, _, _ = cluster_case
    h = _lib.TDDFT.from_workload(wl, precision=precision, proj_mode=proj_mode)
    h.set_fields(wl.times, wl.A, wl.B)
    h.set_states(psi, 0.0)
    _, _, E, _ = h.observables(fields=False)
    h.close()
    assert abs(E["nl"] - cluster_enl) <= tol * abs(cluster_enl), (E["nl"], cluster_enl)


# Norm conservation of the FP32-mixed propagation over 20 steps of the cluster.  The exact step is
# unitary, so an error repeated at every step drifts the norm (and the magnetisation with it):
# rounding the products of FP32 data with fixed FP32 series constants and the accumulator sums is
# biased for given constants, which drifted the norm by -6.1e-8 per step with only kinetic and
# Hartree terms and +5.4e-8 with all terms; the float-float accumulator updates bring this to
# ~3e-9 and ~1e-8.  Both bounds sit between the two.
@pytest.mark.parametrize("terms,proj_mode,bound", [("kinetic+hartree", 1, 1.5e-8), ("all", 1, 3e-8), ("all", 5, 3e-8)])
def test_cluster_fp32_norm_drift_per_step(lib, cluster_case, terms, proj_mode, bound):
    from paper_2506_21908_gb300 import _lib
    import copy
    wl, psi, _, _, _ = cluster_case
    wl = copy.deepcopy(wl)
    kw = {}
    if terms != "all":
        wl.D = wl.D * 0.0
        wl.lam = wl.lam * 0.0
        wl.Z = wl.Z * 0.0
        kw["xc"] = 0
    h = _lib.TDDFT.from_workload(wl, precision=_lib.FP32_MIXED, proj_mode=proj_mode, **kw)
    h.set_fields(wl.times, wl.A * 0.0, wl.B)
    h.set_states(psi.astype(np.complex64), 0.0)
    n0 = h.observables(fields=False)[3]
    h.step(20)
    n1 = h.observables(fields=False)[3]
    h.close()
    drift = float(np.mean(n1 - n0)) / 20
    assert abs(drift) <= bound, drift


def test_bcc_full_size_sampled_h_fp32_mixed(lib):
    wl = S.bcc(nsteps=8)
    psi = S.bcc_states(wl)
    s, V, A = oracle_potential(wl, psi, T0)
    hpsi, Vg = gpu_apply(wl, psi, 1, (-30.0, 400.0))
    assert rel(Vg, V) <= 1e-6
    sample = [0, 77, 127]
    ref = s.apply_h(psi[:, sample], V, A)  # every k-point, three spinors each
    assert rel(hpsi[:, sample], ref) <= 2e-5


@pytest.fixture(scope="module")
def large_case():
    wl = S.large(nsteps=8, nstates=16)
    psi = S.small_parity_states(wl)
    s, V, A = oracle_potential(wl, psi, T0)
    sample = [0, 9]
    ref = s.apply_h(psi[:, sample], V, A)
    vnl = s.apply_nonlocal(psi[0, sample], wl.kpts[0] + A)
    return wl, psi, sample, ref, vnl


@pytest.mark.parametrize("proj_mode,tol", [(1, 2e-5), (3, 2e-5), (5, 2e-5), (4, 1e-4), (2, 3e-3)])
def test_large_grid_and_atoms_sampled_h(lib, large_case, proj_mode, tol):
    """96^3 with all 128 atoms of the large supercell: CUDA-core FP32 and the tensor-core TF32x3,
    FP16x3, BF16x3 and TF32 projector contractions (bricks of 32 x 8 x 8 points with up to 24
    projector spheres each); the tensor-core error budget is relative to the non-local part."""
    wl, psi, sample, ref, vnl = large_case
    hpsi, _ = gpu_apply(wl, psi, 1, (-50.0, 450.0), proj_mode=proj_mode)
    err = np.abs(hpsi[:, sample] - ref).max()
    assert err <= tol * np.abs(vnl).max() + 2e-5 * np.abs(ref).max()


def _oracle_one_step(wl, psi, cheb_tol=1e-16):
    from oracle import Oracle
    o = Oracle(System.from_workload(wl), FieldTable(wl.times, wl.A, wl.B), wl.dt, psi, n_sc=wl.n_sc,
               cheb_tol=cheb_tol)
    o.step()
    n, m, E, _ = o.observables()
    return o, n, m, E


@pytest.fixture(scope="module")
def large_step_case():
    """The large supercell at full grid and with all 128 atoms, one of its 1024 spinors (the
    first Loewdin-orthonormalised atomic-orbital spinor), one ETRS step of dt = 0.04 with the laser
    table, by the oracle (FP64, window of reading P2)."""
    wl = S.large(nsteps=4, nstates=1)
    psi = S.large_states(wl, select=[0], dtype=np.complex128)
    o, n, m, E = _oracle_one_step(wl, psi)
    return wl, psi, o, n, m, E


@pytest.fixture(scope="module")
def bcc_step_case():
    """The bcc supercell at full grid and atoms with all 8 k-points (Bloch phases), one spinor per
    k-point, static B_x plus laser, one ETRS step by the oracle."""
    wl = S.bcc(nsteps=4)
    psi = np.ascontiguousarray(S.bcc_states(wl)[:, :1])
    wl.occ = wl.occ[:, :1]
    o, n, m, E = _oracle_one_step(wl, psi)
    return wl, psi, o, n, m, E


def _gpu_one_step(wl, psi, o, precision, proj_mode=None):
    from paper_2506_21908_gb300 import _lib
    h = _lib.TDDFT.from_workload(wl, precision=precision, proj_mode=proj_mode, e_min=o.emin, e_max=o.emax)
    h.set_fields(wl.times, wl.A, wl.B)
    h.set_states(psi, 0.0)
    h.step(1)
    n, m, E, _ = h.observables()
    out = h.get_states()
    h.close()
    return n, m, E, out


@pytest.mark.parametrize("precision,proj_mode,tol", [(0, None, 1e-10), (1, 5, 2e-5), (1, 1, 2e-5)])
def test_large_full_size_step_matches_oracle(lib, large_step_case, precision, proj_mode, tol):
    wl, psi, o, n_o, m_o, E_o = large_step_case
    n, m, E, out = _gpu_one_step(wl, psi, o, precision, proj_mode)
    assert rel(n, n_o) <= tol and rel(m, m_o) <= tol
    assert rel(out, o.psi) <= tol
    if precision == 0:
        assert abs(E["total"] - E_o["total"]) <= 1e-8


@pytest.mark.parametrize("precision,proj_mode,tol", [(0, None, 1e-10), (1, 5, 2e-5)])
def test_bcc_full_size_step_matches_oracle(lib, bcc_step_case, precision, proj_mode, tol):
    wl, psi, o, n_o, m_o, E_o = bcc_step_case
    n, m, E, out = _gpu_one_step(wl, psi, o, precision, proj_mode)
    assert rel(n, n_o) <= tol and rel(m, m_o) <= tol
    assert rel(out, o.psi) <= tol
    if precision == 0:
        assert abs(E["total"] - E_o["total"]) <= 1e-8


@pytest.fixture(scope="module")
def cluster_step_case():
    """The magnetic cluster at full grid and with all 13 atoms, 4 of its 104 spinors (two spin
    parallel and two antiparallel to their atom's axis), one ETRS step with the laser, by the oracle."""
    wl = S.cluster(64, nsteps=4)
    psi = np.ascontiguousarray(S.cluster_states(wl)[:, [0, 4, 51, 103]])
    wl.occ = wl.occ[:, :4]
    o, n, m, E = _oracle_one_step(wl, psi)
    return wl, psi, o, n, m, E


@pytest.mark.parametrize("precision,proj_mode,tol", [(0, None, 1e-10), (1, 5, 2e-5), (1, 1, 2e-5)])
def test_cluster_full_size_step_matches_oracle(lib, cluster_step_case, precision, proj_mode, tol):
    wl, psi, o, n_o, m_o, E_o = cluster_step_case
    n, m, E, out = _gpu_one_step(wl, psi, o, precision, proj_mode)
    assert rel(n, n_o) <= tol and rel(m, m_o) <= tol
    assert rel(out, o.psi) <= tol
    if precision == 0:
        assert abs(E["total"] - E_o["total"]) <= 1e-8
