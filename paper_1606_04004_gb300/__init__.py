"""Python binding of libprunedq, the GB300 (sm_103a) pruned quantum-dynamics
library (Larsson, Hartke, Tannor, arXiv:1606.04004).

Thin ctypes marshalling over the C ABI in ``include/prunedq.h``: every
computational step runs in the library's CUDA kernels.  PyTorch is used only
for device memory and streams (tensors passed to ``State.apply_H``).  If the
shared library is missing, importing this package raises ImportError: there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# PQ_LIBRARY selects another build of the same library (e.g. the
# self-checking libprunedq_checked.so).
_LIB_PATH = os.environ.get("PQ_LIBRARY") or os.path.join(_HERE, "libprunedq.so")

if not os.path.exists(_LIB_PATH):
    raise ImportError(
        f"{_LIB_PATH} is missing: build it first (python -c 'import __graft_entry__ as g; g.build()')")
_lib = C.CDLL(_LIB_PATH)

# ----------------------------------------------------------------- enums
OK, EINVAL, ENOMEM, ECUDA, ECAPACITY, ENUMERIC, ETIMEOUT, EBREAKDOWN, ENOTSUP = range(9)
SINE_DVR, HO_DVR, PVB, PW, FGH_DVR = range(5)
FP64, FP32MIX = 0, 1
RADIUS_1, RADIUS_SQRT2, RADIUS_2 = 1, 2, 3   # neighbour rules of the adaption
SIL, RK4 = 0, 1                                # integrators of propagate
FACTOR_IDENTITY, FACTOR_KINETIC, FACTOR_DIAG = range(3)
_STATUS = {0: "PQ_OK", 1: "PQ_EINVAL", 2: "PQ_ENOMEM", 3: "PQ_ECUDA", 4: "PQ_ECAPACITY",
           5: "PQ_ENUMERIC", 6: "PQ_ETIMEOUT", 7: "PQ_EBREAKDOWN", 8: "PQ_ENOTSUP"}


class PQError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


# ----------------------------------------------------------------- structs
class ModeDesc(C.Structure):
    _fields_ = [("kind", C.c_int), ("n", C.c_int), ("xmin", C.c_double), ("xmax", C.c_double),
                ("mass", C.c_double), ("omega", C.c_double), ("nx_lattice", C.c_int),
                ("np_lattice", C.c_int), ("dvr", C.c_int)]


class Factor(C.Structure):
    _fields_ = [("kind", C.c_int), ("values", C.POINTER(C.c_double))]


class SopTerm(C.Structure):
    _fields_ = [("coef", C.c_double), ("factors", C.POINTER(Factor))]


class PropDesc(C.Structure):
    _fields_ = [("K", C.c_int), ("dt", C.c_double), ("theta", C.c_double), ("radius", C.c_int),
                ("reorth", C.c_int), ("rel_excl", C.c_double), ("integrator", C.c_int),
                ("sil_tol", C.c_double)]


class Observables(C.Structure):
    _fields_ = [("capacity", C.c_int64), ("count", C.POINTER(C.c_int64)),
                ("t", C.POINTER(C.c_double)), ("c_re", C.POINTER(C.c_double)),
                ("c_im", C.POINTER(C.c_double)), ("norm2", C.POINTER(C.c_double)),
                ("energy", C.POINTER(C.c_double)), ("n_active", C.POINTER(C.c_int64)),
                ("n_wasted", C.POINTER(C.c_int64))]


class ParamDesc(C.Structure):
    _fields_ = [("kind", C.c_int), ("mode", C.c_int), ("dterms", C.POINTER(SopTerm)),
                ("nterms", C.c_int)]


PARAM_POTENTIAL, PARAM_CENTRE = 0, 1

_vp = C.c_void_p
#: pq_alloc_fn / pq_free_fn of the C ABI
ALLOC_FN = C.CFUNCTYPE(_vp, C.c_size_t, _vp, _vp)
FREE_FN = C.CFUNCTYPE(None, _vp, _vp, _vp)
_SIGS = {
    "pq_set_allocator": [ALLOC_FN, FREE_FN, _vp],
    "pq_build_basis": [C.POINTER(ModeDesc), C.c_int, C.POINTER(_vp)],
    "pq_basis_free": [_vp],
    "pq_basis_grid": [_vp, C.c_int, _vp, _vp],
    "pq_basis_kinetic": [_vp, C.c_int, _vp],
    "pq_basis_transform": [_vp, C.c_int, _vp],
    "pq_set_sop": [_vp, C.POINTER(SopTerm), C.c_int],
    "pq_init_packet": [_vp, _vp, _vp, _vp, C.c_double, C.c_int, C.c_int, C.c_size_t,
                       C.POINTER(_vp)],
    "pq_state_free": [_vp],
    "pq_state_load": [_vp, _vp, C.c_int64, _vp],
    "pq_state_size": [_vp, C.POINTER(C.c_int64)],
    "pq_state_read": [_vp, _vp, _vp],
    "pq_state_psi_device": [_vp, C.POINTER(_vp)],
    "pq_apply_H": [_vp, _vp, _vp, C.c_int, _vp, _vp],
    "pq_apply_H_host": [_vp, _vp, _vp, C.c_int, _vp],
    "pq_prune": [_vp, C.c_double, C.c_int, C.c_double, _vp],
    "pq_set_potential_grid": [_vp, _vp, C.c_int64],
    "pq_propagate": [_vp, C.POINTER(PropDesc), C.c_int, _vp],
    "pq_observables_get": [_vp, C.POINTER(Observables)],
    "pq_set_timing": [_vp, C.c_int],
    "pq_timing_get": [_vp, C.POINTER(C.c_double), C.POINTER(C.c_int64), C.POINTER(C.c_double)],
    "pq_observe_noalloc": [_vp, C.c_double, _vp, _vp],
    "pq_survival_grad": [_vp, C.POINTER(PropDesc), C.c_int, C.c_int, C.POINTER(ParamDesc), C.c_int,
                         _vp, _vp, _vp],
    "pq_measure_peak": [C.c_int, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)],
    "pq_launch_count": [],
    "pq_last_error": [],
}
for _name, _args in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = C.c_int
_lib.pq_basis_free.restype = None
_lib.pq_state_free.restype = None
_lib.pq_launch_count.restype = C.c_int64
_lib.pq_last_error.restype = C.c_char_p

#: names the C ABI exports (checked against include/prunedq.h by the tests)
EXPORTS = tuple(_SIGS)


def _check(rc):
    if rc != OK:
        raise PQError(rc, _lib.pq_last_error().decode())


def launch_count() -> int:
    return int(_lib.pq_launch_count())


PEAK_FP32, PEAK_FP32X2, PEAK_FP64 = range(3)


def measure_peak(kind: int, iters: int = 4096) -> dict:
    """Measured arithmetic rate of the current device (pq_measure_peak):
    milliseconds, floating-point operations and TFLOP/s of one timed run."""
    ms, fl = C.c_double(), C.c_double()
    _check(_lib.pq_measure_peak(int(kind), int(iters), C.byref(ms), C.byref(fl)))
    return dict(ms=ms.value, flop=fl.value, tflops=fl.value / (ms.value * 1e-3) / 1e12)


_allocator = []   # keeps the ctypes callbacks alive while the library holds them


def set_allocator(alloc=None, free=None):
    """Route the library's device memory through alloc(bytes, stream, ctx) ->
    pointer and free(pointer, stream, ctx) (pq_set_allocator); no arguments
    restore cudaMalloc.  Only while no state exists."""
    if alloc is None:
        _check(_lib.pq_set_allocator(ALLOC_FN(), FREE_FN(), None))
        _allocator.clear()
        return
    fa, ff = ALLOC_FN(alloc), FREE_FN(free)
    _check(_lib.pq_set_allocator(fa, ff, None))
    _allocator[:] = [fa, ff]


def use_torch_allocator():
    """Let PyTorch's caching allocator own all of the library's device memory."""
    import torch

    def _alloc(n, stream, ctx):
        return torch.cuda.caching_allocator_alloc(int(n), stream=int(stream or 0))

    def _free(ptr, stream, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    set_allocator(_alloc, _free)


def lib_path() -> str:
    return _LIB_PATH


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_vp)


# ------------------------------------------------------------------ basis
class Basis:
    """Per-mode 1D DVR bases (pq_build_basis) plus an SoP Hamiltonian."""

    def __init__(self, modes):
        arr = (ModeDesc * len(modes))()
        for i, m in enumerate(modes):
            arr[i] = ModeDesc(int(m.get("kind", 0)), int(m["n"]), float(m.get("xmin", 0.0)),
                              float(m.get("xmax", 0.0)), float(m.get("mass", 1.0)),
                              float(m.get("omega", 1.0)), int(m.get("nx_lattice", 0)),
                              int(m.get("np_lattice", 0)), int(m.get("dvr", 0)))
        h = _vp()
        _check(_lib.pq_build_basis(arr, len(modes), C.byref(h)))
        self._h = h
        self.dims = tuple(int(m["n"]) for m in modes)
        self.D = len(modes)

    def __del__(self):
        if getattr(self, "_h", None):
            _lib.pq_basis_free(self._h)
            self._h = None

    def grid(self, mode):
        n = self.dims[mode]
        x, w = np.zeros(n), np.zeros(n)
        _check(_lib.pq_basis_grid(self._h, mode, _dptr(x), _dptr(w)))
        return x, w

    def kinetic(self, mode):
        n = self.dims[mode]
        T = np.zeros((n, n))
        _check(_lib.pq_basis_kinetic(self._h, mode, _dptr(T)))
        return T

    def transform(self, mode):
        """W of a phase-space mode (basis -> DVR coefficients); 1 for a DVR mode."""
        n = self.dims[mode]
        Wm = np.zeros((n, n))
        _check(_lib.pq_basis_transform(self._h, mode, _dptr(Wm)))
        return Wm

    def set_potential_grid(self, V):
        """A tabulated diagonal potential over the whole lattice (array of the
        lattice's shape or flat, row-major), added to the SoP potential;
        None removes it (pq_set_potential_grid)."""
        if V is None:
            _check(_lib.pq_set_potential_grid(self._h, None, 0))
            return
        v = np.ascontiguousarray(np.asarray(V, dtype=np.float64).ravel())
        _check(_lib.pq_set_potential_grid(self._h, _dptr(v), int(v.size)))

    def set_sop(self, terms):
        """terms: list of (coef, [factor per mode]) with factor None (identity),
        "T" (kinetic) or an array of n values (diagonal)."""
        keep = []
        carr = _marshal_terms(self.dims, terms, keep)
        _check(_lib.pq_set_sop(self._h, carr, len(terms)))


def _marshal_terms(dims, terms, keep):
    """SoP terms -> a ctypes pq_sop_term array (arrays kept alive in `keep`)."""
    D = len(dims)
    carr = (SopTerm * max(1, len(terms)))()
    for t, (coef, facs) in enumerate(terms):
        if len(facs) != D:
            raise ValueError("one factor per mode")
        fa = (Factor * D)()
        for k, f in enumerate(facs):
            if f is None:
                fa[k] = Factor(FACTOR_IDENTITY, None)
            elif isinstance(f, str) and f == "T":
                fa[k] = Factor(FACTOR_KINETIC, None)
            else:
                v = np.ascontiguousarray(f, dtype=np.float64)
                if v.shape != (dims[k],):
                    raise ValueError(f"factor of mode {k} needs {dims[k]} values")
                keep.append(v)
                fa[k] = Factor(FACTOR_DIAG, v.ctypes.data_as(C.POINTER(C.c_double)))
        keep.append(fa)
        carr[t] = SopTerm(float(coef), fa)
    return carr


# ------------------------------------------------------------------ state
def _cdtype(prec):
    return np.complex128 if prec == FP64 else np.complex64


class State:
    """Active set + coefficients on the device (pq_init_packet / pq_state_load)."""

    def __init__(self, basis: Basis, q0, p0, width, theta, precision=FP64, capacity=0, radius=1):
        D = basis.D
        q0 = np.ascontiguousarray(q0, dtype=np.float64).reshape(D)
        p0 = np.ascontiguousarray(p0, dtype=np.float64).reshape(D)
        w = np.ascontiguousarray(width, dtype=np.float64).reshape(D)
        h = _vp()
        _check(_lib.pq_init_packet(basis._h, _dptr(q0), _dptr(p0), _dptr(w), float(theta),
                                   int(radius), int(precision), int(capacity), C.byref(h)))
        self._h = h
        self.basis = basis          # the basis must outlive the state
        self.precision = precision
        self.dtype = _cdtype(precision)

    def __del__(self):
        if getattr(self, "_h", None):
            _lib.pq_state_free(self._h)
            self._h = None

    def free(self):
        self.__del__()

    def load(self, idx, psi=None):
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        p = None
        if psi is not None:
            p = np.ascontiguousarray(psi, dtype=self.dtype)
            if p.shape != idx.shape:
                raise ValueError("psi must match idx")
        _check(_lib.pq_state_load(self._h, _dptr(idx), len(idx), None if p is None else _dptr(p)))

    def size(self) -> int:
        n = C.c_int64()
        _check(_lib.pq_state_size(self._h, C.byref(n)))
        return int(n.value)

    def read(self):
        n = self.size()
        idx = np.zeros(n, dtype=np.int64)
        psi = np.zeros(n, dtype=self.dtype)
        _check(_lib.pq_state_read(self._h, _dptr(idx), _dptr(psi)))
        return idx, psi

    def psi_device_ptr(self) -> int:
        p = _vp()
        _check(_lib.pq_state_psi_device(self._h, C.byref(p)))
        return int(p.value or 0)

    def apply_H(self, x, out, precision=None, stream=None, vhv=None):
        """out = P_A H P_A x for torch CUDA tensors (complex64 or complex128);
        vhv (optional float64 CUDA tensor of 2) receives Re, Im of <x, out>."""
        import torch
        prec = precision if precision is not None else (FP64 if x.dtype == torch.complex128 else FP32MIX)
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        _check(_lib.pq_apply_H(self._h, _vp(x.data_ptr()), _vp(out.data_ptr()), int(prec),
                               _vp(vhv.data_ptr()) if vhv is not None else None, _vp(stream)))
        return out

    def apply_H_host(self, x: np.ndarray, precision=None) -> np.ndarray:
        """The same operator through host buffers (copies inside the call)."""
        prec = precision if precision is not None else (FP64 if x.dtype == np.complex128 else FP32MIX)
        xin = np.ascontiguousarray(x, dtype=_cdtype(prec))
        out = np.empty_like(xin)
        _check(_lib.pq_apply_H_host(self._h, _dptr(xin), _dptr(out), int(prec), None))
        return out

    def prune(self, theta, radius=1, rel_excl=0.0, stream=None):
        """Adaption (pq_prune); radius: RADIUS_1, RADIUS_SQRT2 or RADIUS_2."""
        _check(_lib.pq_prune(self._h, float(theta), int(radius), float(rel_excl),
                             _vp(stream or 0)))

    def propagate(self, K, dt, theta, nsteps, reorth=1, radius=1, rel_excl=0.0, integrator=0,
                  sil_tol=0.0, stream=None):
        d = PropDesc(int(K), float(dt), float(theta), int(radius), int(reorth), float(rel_excl),
                     int(integrator), float(sil_tol))
        _check(_lib.pq_propagate(self._h, C.byref(d), int(nsteps), _vp(stream or 0)))

    def observables(self) -> dict:
        cnt = C.c_int64()
        o = Observables(0, C.pointer(cnt))
        _check(_lib.pq_observables_get(self._h, C.byref(o)))
        n = int(cnt.value)
        arrs = {k: np.zeros(n) for k in ("t", "c_re", "c_im", "norm2", "energy")}
        ia = {k: np.zeros(n, dtype=np.int64) for k in ("n_active", "n_wasted")}
        o = Observables(n, C.pointer(cnt), *[arrs[k].ctypes.data_as(C.POINTER(C.c_double))
                                             for k in ("t", "c_re", "c_im", "norm2", "energy")],
                        *[ia[k].ctypes.data_as(C.POINTER(C.c_int64)) for k in ("n_active", "n_wasted")])
        _check(_lib.pq_observables_get(self._h, C.byref(o)))
        out = dict(arrs)
        out.update(ia)
        out["C"] = arrs["c_re"] + 1j * arrs["c_im"]
        return out

    def observe_noalloc(self, theta, stream=None):
        """C(t), ||psi||^2 and the small-coefficient count of the current state
        through pq_observe_noalloc (no device allocation; fixed scratch)."""
        out = np.zeros(4)
        _check(_lib.pq_observe_noalloc(self._h, float(theta), _dptr(out), _vp(stream or 0)))
        return dict(C=complex(out[0], out[1]), norm2=float(out[2]), n_wasted=int(round(out[3])))

    def survival_grad(self, K, dt, theta, nsteps, ckpt_every, params, reorth=1, radius=1,
                      rel_excl=0.0, stream=None):
        """P = |<Psi(0)|Psi(T)>|^2 and dP/dtheta (pq_survival_grad).  params:
        list of ("centre", mode) or ("potential", dH/dtheta SoP terms)."""
        keep = []
        parr = (ParamDesc * max(1, len(params)))()
        dims = self.basis.dims
        for i, (kind, arg) in enumerate(params):
            if kind == "centre":
                parr[i] = ParamDesc(PARAM_CENTRE, int(arg), None, 0)
            elif kind == "potential":
                terms = _marshal_terms(dims, arg, keep)
                keep.append(terms)
                parr[i] = ParamDesc(PARAM_POTENTIAL, 0, terms, len(arg))
            else:
                raise ValueError(kind)
        grad = np.zeros(max(1, len(params)))
        P = C.c_double()
        d = PropDesc(int(K), float(dt), float(theta), int(radius), int(reorth), float(rel_excl))
        _check(_lib.pq_survival_grad(self._h, C.byref(d), int(nsteps), int(ckpt_every), parr,
                                     len(params), _dptr(grad), C.byref(P), _vp(stream or 0)))
        return P.value, grad[:len(params)]

    def set_timing(self, enable=True):
        _check(_lib.pq_set_timing(self._h, int(enable)))

    def timing(self):
        ms, n, coef = C.c_double(), C.c_int64(), C.c_double()
        _check(_lib.pq_timing_get(self._h, C.byref(ms), C.byref(n), C.byref(coef)))
        return dict(apply_ms=ms.value, n_apply=int(n.value), coef_applied=coef.value)


from .hamiltonians import (build_model, henon_heiles_terms, coupled_morse_terms, double_well_terms,  # noqa: E402
                           modes_of, henon_heiles_param_derivs)
