"""GPU test of the allocation-free entry point tddft_hartree_noalloc.

Callers that cannot allocate device memory (pre-reserved memory pools,
allocation-free loops) use this entry point; it must give the same Hartree potential as
the library's normal path.  On a handle with no atoms, no XC and no fields the potential
4-vector returned by tddft_get_potential is V_v = [v_H, v_H, 0, 0], so its first component
is the reference.  The file name makes pytest collect it last."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _reference(n, seed):
    from paper_2506_21908_gb300 import _lib, synthetic as S
    wl = S.small_parity(n=n, nstates=3, nk=1, natoms=1, seed=seed)
    psi = S.small_parity_states(wl)
    h = _lib.TDDFT(wl.L, n, np.zeros((0, 3)), np.zeros(0, np.int32), [1.0], [1.0], [1.0], 0, [[0.0]], [[0.0]],
                   1.0, np.zeros((1, 3)), [1.0], np.ones((1, 3)), 0.05, xc=0)
    h.set_states(psi)
    dens, _, _, _ = h.observables()
    V = h.get_potential()
    h.close()
    assert np.allclose(V[0], V[1]) and np.abs(V[2:]).max() == 0.0
    return wl.L, dens, V[0]


def test_hartree_noalloc_matches_library_potential_on_two_calls(lib):
    import torch
    from paper_2506_21908_gb300 import _lib
    n = 24
    refs = [_reference(n, seed) for seed in (5, 6)]
    outs = []
    for L, dens, _ in refs:  # two calls in a row on the shared static scratch
        n_dev = torch.from_numpy(dens).cuda()
        vh = torch.full_like(n_dev, float("nan"))
        _lib.hartree_noalloc(n_dev, vh, L)
        outs.append((n_dev, vh))
    torch.cuda.synchronize()
    for (L, dens, vref), (_, vh) in zip(refs, outs):
        got = vh.cpu().numpy()
        assert np.abs(got - vref).max() <= 1e-12 * np.abs(vref).max()
    assert np.abs(refs[0][2] - refs[1][2]).max() > 1e-3 * np.abs(refs[0][2]).max()


def test_hartree_noalloc_rejects_grids_beyond_its_scratch(lib):
    import torch
    from paper_2506_21908_gb300 import _lib
    n_dev = torch.zeros((96, 96, 96), dtype=torch.float64, device="cuda")
    vh = torch.zeros_like(n_dev)
    with pytest.raises(_lib.TddftError) as e:
        _lib.hartree_noalloc(n_dev, vh, [10.0, 10.0, 10.0])
    assert e.value.status == -1
    assert "64" in str(e.value)
