"""ctypes binding of libtddft.so (include/tddft.h): argument marshalling only.

Every step of the propagation runs inside the CUDA library; this module only
packs structs, passes pointers (numpy host arrays or torch CUDA tensors) and
turns status codes into exceptions.  There is no CPU fallback: if the library
is missing or cannot be loaded, ``load()`` raises.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtddft.so")

FP64, FP32_MIXED = 0, 1
SPIN_NONCOLLINEAR, SPIN_COLLINEAR, SPIN_UNPOLARISED = 0, 1, 2
PROJ_FP64, PROJ_FP32, PROJ_TF32, PROJ_TF32X3, PROJ_BF16X3, PROJ_F16X3 = 0, 1, 2, 3, 4, 5
EXP_CHEBYSHEV, EXP_TAYLOR, EXP_CRANK_NICOLSON = 0, 1, 2
E_NAMES = ["kin", "nl", "loc", "H", "xc", "Z", "total", "t", "xc_pot", "N"]
KERNEL_CLASSES = ["fft_xy", "fft_z_kinetic", "epilogue", "proj_gather", "density", "potential", "other",
                  "proj_scatter"]

# Every entry point declared in include/tddft.h (checked by the CPU tests).
EXPORTS = ["tddft_create", "tddft_set_fields", "tddft_set_states", "tddft_get_states", "tddft_step",
           "tddft_observables", "tddft_get_potential", "tddft_apply_hamiltonian", "tddft_set_stream",
           "tddft_info", "tddft_profile", "tddft_profile_read", "tddft_last_error", "tddft_destroy",
           "tddft_hartree_noalloc", "tddft_backward", "tddft_atom_moments", "tddft_torques",
           "tddft_set_states_c64", "tddft_get_states_c64", "tddft_set_wait_test_limit",
           "tddft_measure_peaks"]


class TddftError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("tddft status %d: %s" % (status, msg))
        self.status = status


class Cell(ctypes.Structure):
    _fields_ = [("a", (ctypes.c_double * 3) * 3)]


class Grid(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3)]


class Atoms(ctypes.Structure):
    _fields_ = [("natoms", ctypes.c_int), ("pos", ctypes.c_void_p), ("species", ctypes.c_void_p)]


class Projectors(ctypes.Structure):
    _fields_ = [("nspecies", ctypes.c_int), ("Z", ctypes.c_void_p), ("rc_loc", ctypes.c_void_p),
                ("width", ctypes.c_void_p), ("lmax", ctypes.c_int), ("D", ctypes.c_void_p),
                ("lambda_so", ctypes.c_void_p), ("r_cut", ctypes.c_double)]


class Params(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("proj_mode", ctypes.c_int), ("nk", ctypes.c_int),
                ("kpts", ctypes.c_void_p), ("kw", ctypes.c_void_p), ("nstates", ctypes.c_int),
                ("occ", ctypes.c_void_p), ("dt", ctypes.c_double), ("exp_kind", ctypes.c_int),
                ("exp_order", ctypes.c_int), ("cheb_tol", ctypes.c_double), ("n_sc", ctypes.c_int),
                ("sc_tol", ctypes.c_double), ("e_min", ctypes.c_double), ("e_max", ctypes.c_double),
                ("xc", ctypes.c_int), ("spin_mode", ctypes.c_int)]


_LIB = None


def load(path=LIB_PATH):
    """Load libtddft.so and declare its signatures; raises if it is absent."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(path):
        raise RuntimeError("libtddft.so not built (run __graft_entry__.build()): %s" % path)
    lib = ctypes.CDLL(path)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    sig = {
        "tddft_create": [vp, vp, vp, vp, vp, ctypes.POINTER(vp)],
        "tddft_set_fields": [vp, i, vp, vp, vp],
        "tddft_set_states": [vp, vp, i, d],
        "tddft_get_states": [vp, vp, i],
        "tddft_set_states_c64": [vp, vp, i, d],
        "tddft_get_states_c64": [vp, vp, i],
        "tddft_step": [vp, i],
        "tddft_observables": [vp, vp, vp, vp, vp, vp],
        "tddft_get_potential": [vp, vp],
        "tddft_apply_hamiltonian": [vp, vp, vp, i],
        "tddft_set_stream": [vp, vp],
        "tddft_info": [vp, vp, vp, vp, vp, vp],
        "tddft_profile": [vp, i],
        "tddft_profile_read": [vp, i, vp, vp, vp],
        "tddft_hartree_noalloc": [vp, vp, i, vp, vp],
        "tddft_backward": [vp, i, i, vp, vp, vp, vp],
        "tddft_atom_moments": [vp, vp, vp],
        "tddft_torques": [vp, vp, vp, vp],
        "tddft_set_wait_test_limit": [ctypes.c_uint],
        "tddft_measure_peaks": [vp, i],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.tddft_last_error.argtypes = [vp]
    lib.tddft_last_error.restype = ctypes.c_char_p
    lib.tddft_destroy.argtypes = [vp]
    lib.tddft_destroy.restype = None
    _LIB = lib
    return lib


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return a.ctypes.data_as(ctypes.c_void_p)


class TDDFT:
    """One propagation handle (owns the device state through the library)."""

    def __init__(self, L, n, pos, species, Z, rc_loc, width, lmax, D, lam, r_cut, kpts, kw, occ, dt,
                 precision=FP64, exp_kind=EXP_CHEBYSHEV, exp_order=0, cheb_tol=0.0, n_sc=1, sc_tol=0.0,
                 e_min=0.0, e_max=0.0, xc=1, proj_mode=None, stream=None, spin_mode=0):
        self.lib = load()
        self._keep = []
        L = _f64(L)
        cell = Cell()
        for a in range(3):
            for b in range(3):
                cell.a[a][b] = L[a] if a == b else 0.0
        grid = Grid()
        for a in range(3):
            grid.n[a] = int(n)
        pos = _f64(pos).reshape(-1, 3)
        species = np.ascontiguousarray(species, dtype=np.int32)
        self._keep += [pos, species]
        atoms = Atoms(len(pos), _ptr(pos).value if len(pos) else None, _ptr(species).value if len(pos) else None)
        arrs = [_f64(Z), _f64(rc_loc), _f64(width), _f64(D), _f64(lam)]
        self._keep += arrs
        proj = Projectors(len(arrs[0]), _ptr(arrs[0]).value, _ptr(arrs[1]).value, _ptr(arrs[2]).value, int(lmax),
                          _ptr(arrs[3]).value, _ptr(arrs[4]).value, float(r_cut))
        kpts = _f64(kpts).reshape(-1, 3)
        kw = _f64(kw)
        occ = _f64(occ).reshape(len(kpts), -1)
        self._keep += [kpts, kw, occ]
        if proj_mode is None:
            proj_mode = 0 if precision == FP64 else 1
        prm = Params(int(precision), int(proj_mode), len(kpts), _ptr(kpts).value, _ptr(kw).value, occ.shape[1],
                     _ptr(occ).value, float(dt), int(exp_kind), int(exp_order), float(cheb_tol), int(n_sc),
                     float(sc_tol), float(e_min), float(e_max), int(xc), int(spin_mode))
        h = ctypes.c_void_p()
        st = self.lib.tddft_create(ctypes.byref(cell), ctypes.byref(grid), ctypes.byref(atoms), ctypes.byref(proj),
                                   ctypes.byref(prm), ctypes.byref(h))
        if st != 0:
            raise TddftError(st, self.lib.tddft_last_error(None).decode())
        self.h = h
        self.n = int(n)
        self.N3 = self.n ** 3
        self.nk = len(kpts)
        self.nstates = occ.shape[1]
        self.precision = precision
        self._nt = 0
        self._L = L
        self._natoms = len(pos)
        if stream is not None:
            self.set_stream(stream)

    @classmethod
    def from_workload(cls, wl, **kw):
        return cls(wl.L, wl.n, wl.pos, wl.species, wl.Z, wl.rc_loc, wl.width, wl.lmax, wl.D, wl.lam, wl.r_cut,
                   wl.kpts, wl.kw, wl.occ, wl.dt, xc=kw.pop("xc", wl.xc), n_sc=kw.pop("n_sc", wl.n_sc),
                   spin_mode=kw.pop("spin_mode", getattr(wl, "spin_mode", 0)),
                   exp_order=kw.pop("exp_order", wl.exp_order), **kw)

    def _check(self, st):
        if st != 0:
            raise TddftError(st, self.lib.tddft_last_error(self.h).decode())

    @property
    def psi_shape(self):
        return (self.nk, self.nstates, 2, self.n, self.n, self.n)

    def set_stream(self, stream):
        self._check(self.lib.tddft_set_stream(self.h, ctypes.c_void_p(stream)))

    def set_fields(self, times, A, B):
        times, A, B = _f64(times), _f64(A).reshape(-1, 3), _f64(B).reshape(-1, 3)
        self._check(self.lib.tddft_set_fields(self.h, len(times), _ptr(times), _ptr(A), _ptr(B)))
        self._nt = len(times)

    @staticmethod
    def _is_dev(x):
        return hasattr(x, "data_ptr") and getattr(x, "is_cuda", False)

    def _spinor_arg(self, psi):
        """(array, on_device, complex64?) for a spinor array: CUDA tensors and complex64 host
        arrays are passed as they are (complex64 through the *_c64 calls); anything else is made
        a contiguous complex128 host array."""
        if self._is_dev(psi):
            c64 = str(psi.dtype) == "torch.complex64"
            assert psi.is_contiguous() and (c64 or str(psi.dtype) == "torch.complex128"), \
                "need a contiguous complex64 or complex128 tensor"
            assert psi.numel() == int(np.prod(self.psi_shape))
            return psi, 1, c64
        c64 = str(getattr(psi, "dtype", "")) in ("complex64", "torch.complex64")
        arr = np.ascontiguousarray(psi, dtype=np.complex64 if c64 else np.complex128)
        assert arr.size == int(np.prod(self.psi_shape)), "spinor array has the wrong size"
        return arr, 0, c64

    def set_states(self, psi, t0=0.0):
        arr, dev, c64 = self._spinor_arg(psi)
        fn = self.lib.tddft_set_states_c64 if c64 else self.lib.tddft_set_states
        self._check(fn(self.h, _ptr(arr), dev, float(t0)))

    def get_states(self, out=None):
        if out is None:
            out = np.empty(self.psi_shape, np.complex128)
        arr, dev, c64 = self._spinor_arg(out)
        fn = self.lib.tddft_get_states_c64 if c64 else self.lib.tddft_get_states
        self._check(fn(self.h, _ptr(arr), dev))
        if isinstance(out, np.ndarray) and arr is not out:
            np.copyto(out, arr.reshape(out.shape))
        return out

    def step(self, nsteps=1):
        self._check(self.lib.tddft_step(self.h, int(nsteps)))

    def observables(self, fields=True, check=True):
        n = np.empty((self.n,) * 3) if fields else None
        m = np.empty((3,) + (self.n,) * 3) if fields else None
        E = np.empty(10)
        M = np.empty(3)
        norms = np.empty((self.nk, self.nstates))
        st = self.lib.tddft_observables(self.h, _ptr(n), _ptr(m), _ptr(E), _ptr(M), _ptr(norms))
        if check:
            self._check(st)
        Ed = dict(zip(E_NAMES, E.tolist()))
        Ed["M"] = M
        Ed["status"] = st
        return n, m, Ed, norms

    def get_potential(self):
        V = np.empty((4,) + (self.n,) * 3)
        self._check(self.lib.tddft_get_potential(self.h, _ptr(V)))
        return V

    def apply_hamiltonian(self, psi, out=None):
        arr, dev, c64 = self._spinor_arg(psi)
        if c64 and not dev:
            arr = arr.astype(np.complex128)
        if out is None:
            out = np.empty(self.psi_shape, np.complex128)
        oarr, odev, oc64 = self._spinor_arg(out)
        assert odev == dev and not (dev and c64) and not oc64, "H apply takes complex128 arrays on one side"
        self._check(self.lib.tddft_apply_hamiltonian(self.h, _ptr(arr), _ptr(oarr), dev))
        return out

    def backward(self, nsteps, dL_drho, ckpt_every=50, nt=None):
        """Run nsteps forward and the discrete adjoint; returns (L, dL/dA table, dL/dB table)."""
        dL = _f64(dL_drho).reshape(4, -1)
        nt = self._nt if nt is None else nt
        dA = np.zeros((max(nt, 1), 3))
        dB = np.zeros((max(nt, 1), 3))
        L = ctypes.c_double()
        self._check(self.lib.tddft_backward(self.h, int(nsteps), int(ckpt_every), _ptr(dL), ctypes.byref(L),
                                            _ptr(dA), _ptr(dB)))
        return L.value, dA[:nt], dB[:nt]

    def atom_moments(self):
        """Per-atom (Voronoi cell) magnetic moments [natoms][3] and electron counts [natoms]."""
        na = self._natoms
        M = np.zeros((max(na, 1), 3))
        N = np.zeros(max(na, 1))
        self._check(self.lib.tddft_atom_moments(self.h, _ptr(M), _ptr(N)))
        return M[:na], N[:na]

    def torques(self):
        """Global spin torques at the current state: dict of 3-vectors soc (L.S projectors),
        xc (2 int b_xc x m dV), zeeman (2 mu_B B x M) and their sum total = dM/dt."""
        soc, xc, zee = np.zeros(3), np.zeros(3), np.zeros(3)
        self._check(self.lib.tddft_torques(self.h, _ptr(soc), _ptr(xc), _ptr(zee)))
        return dict(soc=soc, xc=xc, zeeman=zee, total=soc + xc + zee)

    def info(self):
        kf, kh = ctypes.c_int(), ctypes.c_int()
        lo, hi = ctypes.c_double(), ctypes.c_double()
        nl = ctypes.c_longlong()
        self._check(self.lib.tddft_info(self.h, ctypes.byref(kf), ctypes.byref(kh), ctypes.byref(lo),
                                        ctypes.byref(hi), ctypes.byref(nl)))
        return dict(K_full=kf.value, K_half=kh.value, e_min=lo.value, e_max=hi.value, launches=nl.value)

    def profile(self, enable=True):
        self._check(self.lib.tddft_profile(self.h, int(bool(enable))))

    def profile_read(self):
        ms = np.zeros(8)
        cnt = np.zeros(8, np.int64)
        by = np.zeros(8)
        self._check(self.lib.tddft_profile_read(self.h, 8, _ptr(ms), _ptr(cnt), _ptr(by)))
        return {name: dict(ms=float(ms[i]), launches=int(cnt[i]), bytes=float(by[i]))
                for i, name in enumerate(KERNEL_CLASSES)}

    def close(self):
        if getattr(self, "h", None):
            self.lib.tddft_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def measure_peaks():
    """Measured peak rates of the current GPU in TFLOP/s: FP64 and FP32 FMA on the CUDA cores,
    TF32, FP16 and BF16 tensor-core products (tddft_measure_peaks)."""
    lib = load()
    out = np.zeros(5)
    st = lib.tddft_measure_peaks(_ptr(out), 5)
    if st != 0:
        raise TddftError(st, "tddft_measure_peaks failed")
    return dict(zip(["fp64_fma", "fp32_fma", "tf32_mma", "fp16_mma", "bf16_mma"], out.tolist()))


def hartree_noalloc(n_dev, vH_dev, L, stream=None):
    """Allocation-free Hartree solve on device tensors: n_dev and vH_dev are contiguous float64
    CUDA tensors of one shape (n, n, n) on one device; the work is queued on ``stream`` (a raw
    cudaStream_t value; None = torch's current stream of that device).  Every argument is checked
    here, before the library is called, so a wrong tensor raises instead of reaching a kernel."""
    import torch
    for name, t in (("n_dev", n_dev), ("vH_dev", vH_dev)):
        if not isinstance(t, torch.Tensor):
            raise TypeError("%s must be a torch tensor" % name)
        if t.dtype != torch.float64:
            raise TypeError("%s must be float64, not %s" % (name, t.dtype))
        if t.dim() != 3 or not (t.shape[0] == t.shape[1] == t.shape[2]):
            raise ValueError("%s must have shape (n, n, n), not %s" % (name, tuple(t.shape)))
        if not t.is_contiguous():
            raise ValueError("%s must be contiguous" % name)
    if tuple(n_dev.shape) != tuple(vH_dev.shape):
        raise ValueError("n_dev and vH_dev differ in shape: %s, %s" % (tuple(n_dev.shape), tuple(vH_dev.shape)))
    if not (n_dev.is_cuda and vH_dev.is_cuda):
        raise ValueError("n_dev and vH_dev must be CUDA tensors")
    if n_dev.device != vH_dev.device:
        raise ValueError("n_dev and vH_dev are on different devices: %s, %s" % (n_dev.device, vH_dev.device))
    L = _f64(L)
    if L.shape != (3,):
        raise ValueError("L must hold the three cell lengths")
    lib = load()
    n = int(n_dev.shape[-1])
    with torch.cuda.device(n_dev.device):
        if stream is None:
            stream = torch.cuda.current_stream(n_dev.device).cuda_stream
        st = lib.tddft_hartree_noalloc(_ptr(n_dev), _ptr(vH_dev), n, _ptr(L), ctypes.c_void_p(stream or 0))
    if st != 0:
        raise TddftError(st, lib.tddft_last_error(None).decode())
