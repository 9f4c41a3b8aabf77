"""CPU checks of the C-ABI library: it loads, exports every entry point that
include/tddft.h declares, and reports errors without a GPU (no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "tddft.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tddft_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def cpu_lib():
    from paper_2506_21908_gb300 import _lib
    if not os.path.exists(_lib.LIB_PATH):
        from paper_2506_21908_gb300 import build
        build.build()
    return _lib.load()


def test_header_declares_binding_exports():
    from paper_2506_21908_gb300 import _lib
    assert _declared() == sorted(_lib.EXPORTS)


def test_library_exports_every_declared_symbol(cpu_lib):
    for name in _declared():
        assert hasattr(cpu_lib, name), name


def _gpu_present():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.mark.skipif(_gpu_present(), reason="checks the no-device error path")
def test_create_without_device_returns_error_not_crash(cpu_lib):
    from paper_2506_21908_gb300 import _lib, synthetic as S
    wl = S.small_parity(n=8, nstates=1, nk=1, natoms=1)
    with pytest.raises(_lib.TddftError) as e:
        _lib.TDDFT.from_workload(wl)
    assert e.value.status in (-2, -3)
    assert cpu_lib.tddft_last_error(None)


def test_argument_validation_before_device_use(cpu_lib):
    """Unsupported grids and cells are refused with a status, before any allocation."""
    from paper_2506_21908_gb300 import _lib, synthetic as S
    wl = S.small_parity(n=8, nstates=1, nk=1, natoms=1)
    with pytest.raises(_lib.TddftError) as e:
        _lib.TDDFT(wl.L, 10, wl.pos, wl.species, wl.Z, wl.rc_loc, wl.width, wl.lmax, wl.D, wl.lam, wl.r_cut,
                   wl.kpts, wl.kw, wl.occ, wl.dt)
    assert e.value.status == -7
    with pytest.raises(_lib.TddftError) as e:
        _lib.TDDFT(wl.L, 8, wl.pos, wl.species, wl.Z, wl.rc_loc, wl.width, wl.lmax, wl.D, wl.lam, 6.0,
                   wl.kpts, wl.kw, wl.occ, wl.dt)
    assert e.value.status == -1
    with pytest.raises(_lib.TddftError) as e:
        _lib.TDDFT(wl.L, 8, wl.pos, wl.species, wl.Z, wl.rc_loc, wl.width, 3, wl.D, wl.lam, wl.r_cut,
                   wl.kpts, wl.kw, wl.occ, wl.dt)
    assert e.value.status == -7


def _header_structs():
    """Field names, in order, of every `typedef struct { ... } name;` in include/tddft.h."""
    src = open(os.path.join(ROOT, "include", "tddft.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for body, name in re.findall(r"typedef struct\s*\{(.*?)\}\s*(tddft_[a-z]+)\s*;", src, flags=re.S):
        fields = []
        for decl in body.split(";"):
            decl = decl.strip()
            if decl:
                fields.append(re.findall(r"([A-Za-z_][A-Za-z_0-9]*)\s*(?:\[[^\]]*\])*\s*$", decl)[0])
        out[name] = fields
    return out


def test_binding_structs_match_the_header_layout():
    from paper_2506_21908_gb300 import _lib
    hs = _header_structs()
    pairs = {"tddft_cell": _lib.Cell, "tddft_grid": _lib.Grid, "tddft_atoms": _lib.Atoms,
             "tddft_projectors": _lib.Projectors, "tddft_params": _lib.Params}
    assert set(hs) == set(pairs)
    for name, cls in pairs.items():
        assert [f[0] for f in cls._fields_] == hs[name], name


def test_spin_mode_validation_before_device_use(cpu_lib):
    """An unknown spin mode, and spin-orbit coupling outside the non-collinear mode, are refused
    with TDDFT_ERR_ARG before any allocation."""
    from paper_2506_21908_gb300 import _lib, synthetic as S
    wl = S.small_parity(n=8, nstates=1, nk=1, natoms=1, lam=0.02)
    for mode in (1, 2, 3):
        with pytest.raises(_lib.TddftError) as e:
            _lib.TDDFT.from_workload(wl, spin_mode=mode)
        assert e.value.status == -1, mode


def test_binding_routes_complex64_to_the_c64_calls():
    """The binding passes complex64 host arrays through the *_c64 entry points without a copy and
    turns any other host array into contiguous complex128 (argument handling only, no GPU)."""
    import numpy as np
    from paper_2506_21908_gb300 import _lib
    h = object.__new__(_lib.TDDFT)
    h.nk, h.nstates, h.n = 1, 2, 4
    a64 = np.zeros(h.psi_shape, np.complex64)
    arr, dev, c64 = h._spinor_arg(a64)
    assert c64 and not dev and arr is a64
    a128 = np.zeros(h.psi_shape, np.complex128)
    arr, dev, c64 = h._spinor_arg(a128)
    assert not c64 and not dev and arr is a128
    arr, dev, c64 = h._spinor_arg(np.zeros(h.psi_shape))
    assert not c64 and arr.dtype == np.complex128
    with pytest.raises(AssertionError):
        h._spinor_arg(np.zeros(5, np.complex64))


@pytest.mark.parametrize("case", ["float32", "shape", "noncubic", "noncontig", "mismatch", "cpu"])
def test_hartree_noalloc_binding_rejects_bad_tensors_before_any_call(case):
    """The allocation-free Hartree binding checks dtype, shape, contiguity, equal shapes and the
    device of both tensors before it calls the library (no launch can see a wrong buffer)."""
    import torch
    from paper_2506_21908_gb300 import _lib
    good = torch.zeros((8, 8, 8), dtype=torch.float64)
    n, v = good, good.clone()
    if case == "float32":
        n = good.float()
    elif case == "shape":
        n = torch.zeros((8, 8), dtype=torch.float64)
    elif case == "noncubic":
        n, v = torch.zeros((8, 8, 16), dtype=torch.float64), torch.zeros((8, 8, 16), dtype=torch.float64)
    elif case == "noncontig":
        n = torch.zeros((8, 8, 16), dtype=torch.float64)[:, :, ::2]
    elif case == "mismatch":
        v = torch.zeros((16, 16, 16), dtype=torch.float64)
    with pytest.raises((TypeError, ValueError)):
        _lib.hartree_noalloc(n, v, [10.0, 10.0, 10.0])
