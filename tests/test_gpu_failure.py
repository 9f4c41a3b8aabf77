"""Failure detection, tested without any GPU fault: every failure is made on the host (a
non-finite input, a spectral window that the potential leaves) or by the library's testing hook
that shortens the first try of its bounded mbarrier waits (the kernels then flag the error and
wait again with the full limit, so every copy and matrix product still completes).  Each test
checks the status the library returns and that the next handle works normally."""
import numpy as np
import pytest

from paper_2506_21908_gb300 import synthetic as S

pytestmark = pytest.mark.gpu

ERR_CUDA, ERR_DIVERGED, ERR_BOUND = -2, -5, -6


def _handle(wl, **kw):
    from paper_2506_21908_gb300 import _lib
    h = _lib.TDDFT.from_workload(wl, **kw)
    h.set_fields(wl.times, wl.A, wl.B)
    return h


@pytest.mark.parametrize("precision", [0, 1])
def test_non_finite_input_is_reported_as_diverged(lib, precision):
    wl = S.small_parity(n=16, nstates=3, nk=1, natoms=2)
    psi = S.small_parity_states(wl)
    bad = psi.copy()
    bad[0, 1, 0, 3, 4, 5] = np.nan
    h = _handle(wl, precision=precision, e_min=-20.0, e_max=100.0)
    h.set_states(bad, 0.0)
    _, _, E, _ = h.observables(fields=False, check=False)
    assert E["status"] == ERR_DIVERGED
    h.close()
    g = _handle(wl, precision=precision, e_min=-20.0, e_max=100.0)
    g.set_states(psi, 0.0)
    g.step(1)
    _, _, E, norms = g.observables(fields=False)
    assert E["status"] == 0 and np.abs(norms - 1.0).max() < 1e-5
    g.close()


def test_potential_outside_the_spectral_window_is_reported(lib):
    """A window narrower than the spectrum of the potential: the device check of every potential
    sets the flag and tddft_observables returns TDDFT_ERR_BOUND."""
    from paper_2506_21908_gb300 import _lib
    wl = S.small_parity(n=16, nstates=3, nk=1, natoms=2)
    psi = S.small_parity_states(wl)
    h = _handle(wl, precision=0, e_min=-0.5, e_max=0.5)
    h.set_states(psi, 0.0)
    h.step(1)
    with pytest.raises(_lib.TddftError) as e:
        h.observables(fields=False)
    assert e.value.status == ERR_BOUND
    h.close()


@pytest.mark.parametrize("proj_mode", [1, 5])
def test_expired_first_wait_sets_the_error_status(lib, proj_mode):
    """With the testing hook the first try of the bounded waits of the bulk-copy FFT pass (and, with
    proj_mode 5, of the tensor-core gather) gives up after one poll: the call reports
    TDDFT_ERR_CUDA; after the hook is reset, a fresh handle reproduces the reference run exactly."""
    from paper_2506_21908_gb300 import _lib
    wl = S.small_parity(n=32, nstates=4, nk=1, natoms=2)
    psi = S.small_parity_states(wl)

    def run():
        h = _handle(wl, precision=1, proj_mode=proj_mode, e_min=-20.0, e_max=400.0)
        h.set_states(psi, 0.0)
        h.step(1)
        n, m, E, _ = h.observables(check=False)
        out = h.get_states()
        msg = h.lib.tddft_last_error(h.h).decode()
        h.close()
        return E["status"], msg, n, out

    st0, _, n0, psi0 = run()
    assert st0 == 0
    assert lib.tddft_set_wait_test_limit(1) == 0
    try:
        st1, msg1, _, _ = run()
    finally:
        assert lib.tddft_set_wait_test_limit(0) == 0
    assert st1 == ERR_CUDA, (st1, msg1)
    assert "iteration limit" in msg1
    st2, _, n2, psi2 = run()
    assert st2 == 0
    assert np.array_equal(n2, n0) and np.array_equal(psi2, psi0)
