"""Thin Python binding of the C ABI in include/pfc.h (argument marshalling only).

Every computation runs in libpfc.so's CUDA kernels; this module converts torch
tensors to device pointers, passes torch's current stream, and turns status
codes into exceptions.  If the library has not been built, the first call
raises: there is no CPU fallback.

    from paper_2103_04856_gb300 import pfc
    ctx = pfc.Context(pfc.Problem(nx=128, ny=128, nz=128, eps=2.0, a=(1, 0, 1, 0, 0, 0)))
    E, g = ctx.energy_and_grad(u)            # u: CUDA float32 tensor (nz, ny, nx)
    trace = ctx.run(u, nsteps=100, tau=1e-3)  # in place, mass conserved
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass, field

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# PFC_LIBRARY selects another build of the library (the debug build of
# paper_2103_04856_gb300.build --debug); the default is the in-tree libpfc.so
LIB_PATH = os.environ.get("PFC_LIBRARY") or os.path.join(_HERE, "libpfc.so")

PFC_OK, PFC_EINVAL, PFC_ENOMEM, PFC_ECUDA, PFC_ENONFINITE, PFC_ETIMEOUT, PFC_EUNSUPPORTED = 0, -1, -2, -3, -4, -5, -6
PFC_WELL_01, PFC_WELL_PM1 = 0, 1
PFC_FP32, PFC_FP64 = 0, 1
PFC_IMPL_FUSED, PFC_IMPL_PLAIN = 0, 1
FLAG_NO_DISCRIMINANT_REFINEMENT = 1

# every symbol include/pfc.h declares
EXPORTED = ("pfc_create", "pfc_destroy", "pfc_energy", "pfc_energy_and_grad", "pfc_step", "pfc_run",
            "pfc_curvatures", "pfc_batch_create", "pfc_batch_destroy", "pfc_batch_run", "pfc_batch_step",
            "pfc_batch_timing", "pfc_batch_last_timing", "pfc_hflow_create", "pfc_hflow_destroy",
            "pfc_hflow_field", "pfc_hflow_grad", "pfc_hflow_run", "pfc_energy_and_grad_noalloc", "pfc_b_to_a",
            "pfc_status_string", "pfc_last_error", "pfc_set_coefficient_field", "pfc_diagnostics",
            "pfc_hflow_set_coefficient_field", "pfc_hflow_set_mass_field", "pfc_surface_cells",
            "pfc_curvature_histogram", "pfc_batch_step_host", "pfc_batch_host_wait", "pfc_hflow_batch_create",
            "pfc_hflow_batch_destroy", "pfc_hflow_batch_field", "pfc_hflow_batch_run", "pfc_batch_step_lazy",
            "pfc_batch_lazy_finish", "pfc_slab_create", "pfc_slab_destroy", "pfc_slab_sweep", "pfc_slab_finish",
            "pfc_slab_apply_offset", "pfc_measure_fp32_peak", "pfc_diagnostics_dev")
SLAB_ENERGY, SLAB_GRAD, SLAB_STEP = 0, 1, 2
SLAB_NSUMS = 8


class PfcError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"pfc status {status}: {msg}")
        self.status = status


class NonFiniteError(PfcError):
    pass


class _CHFlow(ctypes.Structure):
    _fields_ = [("m0", ctypes.c_double), ("lr", ctypes.c_double), ("beta1", ctypes.c_double),
                ("beta2", ctypes.c_double), ("adam_eps", ctypes.c_double), ("blur_sigma", ctypes.c_double),
                ("blur_radius", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class _CProblem(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("well", ctypes.c_int32), ("prec", ctypes.c_int32), ("impl", ctypes.c_int32),
        ("h", ctypes.c_double), ("eps", ctypes.c_double), ("xi", ctypes.c_double),
        ("a", ctypes.c_double * 6),
        ("tile_y", ctypes.c_int32), ("tile_z", ctypes.c_int32),
        ("mu", ctypes.c_double), ("theta", ctypes.c_double * 3),
        ("proj", ctypes.c_int32), ("flags", ctypes.c_uint32),
    ]


@dataclass
class Problem:
    """Grid and parameters of eq. Feps; ``a`` in the paper's order (a20 a11 a02 a10 a01 a00),
    kappa1 >= kappa2.  ``prec`` is "fp32" or "fp64", ``impl`` "fused" or "plain".
    ``mu``, ``theta`` (x, y, z): the orientation term eps mu (theta . grad u)^2
    of Sec. 5.2 (mu = 0: none).  ``proj`` = 1: the tangent-projected
    M = -eps P Hess u P instead of eq. Meps.  ``flags``: PFC_FLAG_* bits
    (FLAG_NO_DISCRIMINANT_REFINEMENT turns the FP32 path's FP64
    re-evaluation of D off)."""
    nx: int
    ny: int
    nz: int
    eps: float
    a: tuple
    h: float = 1.0
    xi: float = 1e-6
    well: int = PFC_WELL_01
    prec: str = "fp32"
    impl: str = "fused"
    tile_y: int = 0
    tile_z: int = 0
    mu: float = 0.0
    theta: tuple = (0.0, 0.0, 0.0)
    proj: int = 0
    flags: int = 0

    @classmethod
    def from_shape(cls, shape, **kw):
        nz, ny, nx = shape
        return cls(nx=nx, ny=ny, nz=nz, **kw)

    @property
    def dtype(self):
        return torch.float64 if self.prec == "fp64" else torch.float32

    def _c(self) -> _CProblem:
        if self.prec not in ("fp32", "fp64"):
            raise ValueError("prec must be 'fp32' or 'fp64'")
        if self.impl not in ("fused", "plain"):
            raise ValueError("impl must be 'fused' or 'plain'")
        if len(self.a) != 6:
            raise ValueError("a needs 6 coefficients")
        if len(self.theta) != 3:
            raise ValueError("theta needs 3 components")
        return _CProblem(int(self.nx), int(self.ny), int(self.nz), int(self.well),
                         PFC_FP64 if self.prec == "fp64" else PFC_FP32,
                         PFC_IMPL_PLAIN if self.impl == "plain" else PFC_IMPL_FUSED,
                         float(self.h), float(self.eps), float(self.xi),
                         (ctypes.c_double * 6)(*[float(x) for x in self.a]),
                         int(self.tile_y), int(self.tile_z), float(self.mu),
                         (ctypes.c_double * 3)(*[float(x) for x in self.theta]), int(self.proj), int(self.flags))


_lib = None
_lock = threading.Lock()


def load_library():
    """Load libpfc.so; raises if it is missing (build it with python -m paper_2103_04856_gb300.build)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build the CUDA library first "
                               "(python -m paper_2103_04856_gb300.build)")
        lib = ctypes.CDLL(LIB_PATH)
        vp, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)
        P = ctypes.POINTER(_CProblem)
        sig = {
            "pfc_create": ([P, ctypes.POINTER(vp)], ctypes.c_int),
            "pfc_destroy": ([vp], None),
            "pfc_energy": ([vp, vp, dp, vp], ctypes.c_int),
            "pfc_energy_and_grad": ([vp, vp, vp, dp, vp], ctypes.c_int),
            "pfc_step": ([vp, vp, vp, ctypes.c_double, vp, vp], ctypes.c_int),
            "pfc_run": ([vp, vp, ctypes.c_int32, ctypes.c_double, dp, vp], ctypes.c_int),
            "pfc_curvatures": ([vp, vp, vp, vp, vp], ctypes.c_int),
            "pfc_batch_create": ([P, ctypes.c_int32, ctypes.POINTER(vp)], ctypes.c_int),
            "pfc_batch_destroy": ([vp], None),
            "pfc_batch_run": ([vp, ctypes.POINTER(vp), ctypes.c_int32, dp, dp, vp], ctypes.c_int),
            "pfc_batch_step": ([vp, ctypes.POINTER(vp), ctypes.POINTER(vp), dp, vp, vp], ctypes.c_int),
            "pfc_batch_timing": ([vp, ctypes.c_int], ctypes.c_int),
            "pfc_batch_step_host": ([vp, ctypes.POINTER(vp), ctypes.POINTER(vp), dp, vp], ctypes.c_int),
            "pfc_batch_step_lazy": ([vp, ctypes.POINTER(vp), ctypes.POINTER(vp), dp, ctypes.c_int32, vp], ctypes.c_int),
            "pfc_batch_lazy_finish": ([vp, ctypes.POINTER(vp), vp], ctypes.c_int),
            "pfc_batch_host_wait": ([vp, vp], ctypes.c_int),
            "pfc_hflow_batch_create": ([P, dp, ctypes.c_int32, ctypes.POINTER(_CHFlow), ctypes.POINTER(vp)],
                                       ctypes.c_int),
            "pfc_hflow_batch_destroy": ([vp], None),
            "pfc_hflow_batch_field": ([vp, ctypes.POINTER(vp), ctypes.POINTER(vp), vp], ctypes.c_int),
            "pfc_hflow_batch_run": ([vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.c_int32,
                                     ctypes.POINTER(ctypes.c_int32), dp, vp], ctypes.c_int),
            "pfc_batch_last_timing": ([vp, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)],
                                      ctypes.c_int),
            "pfc_energy_and_grad_noalloc": ([P, vp, vp, dp, vp], ctypes.c_int),
            "pfc_hflow_create": ([P, ctypes.POINTER(_CHFlow), ctypes.POINTER(vp)], ctypes.c_int),
            "pfc_hflow_destroy": ([vp], None),
            "pfc_hflow_field": ([vp, vp, vp, vp], ctypes.c_int),
            "pfc_hflow_grad": ([vp, vp, vp, dp, vp], ctypes.c_int),
            "pfc_hflow_run": ([vp, vp, vp, vp, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32), dp, vp],
                              ctypes.c_int),
            "pfc_b_to_a": ([dp, dp], ctypes.c_int),
            "pfc_set_coefficient_field": ([vp, vp, vp], ctypes.c_int),
            "pfc_diagnostics": ([vp, vp, dp, vp], ctypes.c_int),
            "pfc_diagnostics_dev": ([vp, vp, vp, vp], ctypes.c_int),
            "pfc_hflow_set_coefficient_field": ([vp, vp, vp], ctypes.c_int),
            "pfc_hflow_set_mass_field": ([vp, vp, vp], ctypes.c_int),
            "pfc_surface_cells": ([vp, vp, ctypes.c_double, vp, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64), vp],
                                  ctypes.c_int),
            "pfc_curvature_histogram": ([vp, vp, ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_double, vp,
                                         vp], ctypes.c_int),
            "pfc_slab_create": ([P, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(vp)], ctypes.c_int),
            "pfc_slab_destroy": ([vp], None),
            "pfc_slab_sweep": ([vp, vp, vp, vp, ctypes.c_int32, ctypes.c_double, vp, vp], ctypes.c_int),
            "pfc_slab_finish": ([vp, vp, ctypes.c_int32, vp, vp], ctypes.c_int),
            "pfc_slab_apply_offset": ([vp, vp, vp], ctypes.c_int),
            "pfc_measure_fp32_peak": ([dp, vp], ctypes.c_int),
            "pfc_status_string": ([ctypes.c_int], ctypes.c_char_p),
            "pfc_last_error": ([], ctypes.c_char_p),
        }
        for name, (args, res) in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
        return lib


def _check(rc: int):
    if rc != PFC_OK:
        lib = load_library()
        msg = lib.pfc_last_error().decode(errors="replace")
        raise (NonFiniteError if rc == PFC_ENONFINITE else PfcError)(rc, msg)


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _coef_field(t, prob: Problem):
    """a(x) (Sec. 5.2): a CUDA tensor shaped (6, nz, ny, nx) of the problem's
    dtype, a[k] the k-th coefficient in the order of Problem.a; None clears."""
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != prob.dtype:
        raise TypeError(f"a_field must be a CUDA {prob.dtype} tensor")
    if tuple(t.shape) != (6, prob.nz, prob.ny, prob.nx) or not t.is_contiguous():
        raise ValueError(f"a_field must be contiguous with shape {(6, prob.nz, prob.ny, prob.nx)}")
    return ctypes.c_void_p(t.data_ptr())


def _field(t: torch.Tensor, prob: Problem, name: str):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != prob.dtype:
        raise TypeError(f"{name} must be {prob.dtype}, got {t.dtype}")
    if tuple(t.shape) != (prob.nz, prob.ny, prob.nx) or not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous with shape {(prob.nz, prob.ny, prob.nx)}")
    return ctypes.c_void_p(t.data_ptr())


# ------------------------------------------------------------ C-named calls

def pfc_create(prob: Problem):
    lib = load_library()
    h = ctypes.c_void_p()
    _check(lib.pfc_create(ctypes.byref(prob._c()), ctypes.byref(h)))
    return h


def pfc_destroy(handle):
    if handle:
        load_library().pfc_destroy(handle)


def pfc_b_to_a(b) -> np.ndarray:
    b = np.ascontiguousarray(b, dtype=np.float64)
    if b.shape != (7,):
        raise ValueError("b needs 7 entries")
    a = np.empty(6, dtype=np.float64)
    _check(load_library().pfc_b_to_a(b.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                     a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return a


def energy_and_grad_noalloc(prob: Problem, u: torch.Tensor, g: torch.Tensor, stream=None, sync=True):
    """pfc_energy_and_grad_noalloc: the fused energy and gradient with no
    device allocation at all (for callers that may not allocate); g is filled
    in place.  Calls that overlap on the GPU race (one static scratch array)."""
    E = ctypes.c_double()
    _check(load_library().pfc_energy_and_grad_noalloc(ctypes.byref(prob._c()), _field(u, prob, "u"),
                                                      _field(g, prob, "g"), ctypes.byref(E) if sync else None,
                                                      _stream(stream)))
    return E.value if sync else None


def measure_fp32_peak(stream=None) -> float:
    """FP32 FMA throughput of the current GPU in TFLOP/s (pfc_measure_fp32_peak)."""
    t = ctypes.c_double()
    _check(load_library().pfc_measure_fp32_peak(ctypes.byref(t), _stream(stream)))
    return t.value


class Context:
    """A problem bound to the current CUDA device (owns the library's scratch)."""

    def __init__(self, prob: Problem):
        self.prob = prob
        self._h = pfc_create(prob)
        self._lib = load_library()

    def close(self):
        if getattr(self, "_h", None):
            pfc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def new_field(self):
        return torch.empty((self.prob.nz, self.prob.ny, self.prob.nx), dtype=self.prob.dtype, device="cuda")

    def energy(self, u: torch.Tensor, stream=None) -> float:
        E = ctypes.c_double()
        _check(self._lib.pfc_energy(self._h, _field(u, self.prob, "u"), ctypes.byref(E), _stream(stream)))
        return E.value

    def energy_and_grad(self, u: torch.Tensor, g: torch.Tensor | None = None, stream=None, sync=True):
        g = self.new_field() if g is None else g
        E = ctypes.c_double()
        _check(self._lib.pfc_energy_and_grad(self._h, _field(u, self.prob, "u"), _field(g, self.prob, "g"),
                                             ctypes.byref(E) if sync else None, _stream(stream)))
        return (E.value if sync else None), g

    def step(self, u_in: torch.Tensor, u_out: torch.Tensor, tau: float, scalars: torch.Tensor | None = None,
             stream=None):
        sp = None
        if scalars is not None:
            if scalars.dtype != torch.float64 or not scalars.is_cuda or scalars.numel() < 5:
                raise TypeError("scalars must be a CUDA float64 tensor with >= 5 entries")
            sp = ctypes.c_void_p(scalars.data_ptr())
        _check(self._lib.pfc_step(self._h, _field(u_in, self.prob, "u_in"), _field(u_out, self.prob, "u_out"),
                                  float(tau), sp, _stream(stream)))
        return u_out

    def run(self, u: torch.Tensor, nsteps: int, tau: float, trace: bool = True, stream=None):
        tr = np.empty((max(int(nsteps), 0), 5), dtype=np.float64) if trace else None
        _check(self._lib.pfc_run(self._h, _field(u, self.prob, "u"), int(nsteps), float(tau),
                                 tr.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if trace else None,
                                 _stream(stream)))
        return tr

    def set_coefficient_field(self, a_field, stream=None):
        """Spatialised coefficients a(x) (Sec. 5.2) for every later evaluation;
        None returns to the constant a.  The library keeps its own copy."""
        _check(self._lib.pfc_set_coefficient_field(self._h, _coef_field(a_field, self.prob), _stream(stream)))

    def diagnostics(self, u: torch.Tensor, stream=None) -> dict:
        """Sec. 4.5 viability quantities of u (discrepancy, Cahn-Hilliard
        energy, their ratio, max and min of u)."""
        out = np.empty(5)
        _check(self._lib.pfc_diagnostics(self._h, _field(u, self.prob, "u"),
                                         out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _stream(stream)))
        return {"discrepancy": float(out[0]), "cahn_hilliard": float(out[1]), "ratio": float(out[2]),
                "max": float(out[3]), "min": float(out[4])}

    def diagnostics_dev(self, u: torch.Tensor, out: torch.Tensor, stream=None) -> torch.Tensor:
        """The five diagnostics values written into out (a CUDA float64 tensor
        of 5 elements) without synchronising: discrepancy, Cahn-Hilliard
        energy, ratio, max u, min u."""
        if out.dtype != torch.float64 or not out.is_cuda or out.numel() < 5 or not out.is_contiguous():
            raise ValueError("out must be a contiguous CUDA float64 tensor of 5 elements")
        _check(self._lib.pfc_diagnostics_dev(self._h, _field(u, self.prob, "u"), ctypes.c_void_p(out.data_ptr()),
                                             _stream(stream)))
        return out

    def surface_cells(self, u: torch.Tensor, level: float | None = None, stream=None) -> torch.Tensor:
        """Cells (area, kappa1, kappa2) of the curvature diagram of {u = level}
        (Sec. 4.1); level defaults to the middle of the double well's two
        phases.  Returns a CUDA tensor shaped (n, 3)."""
        if level is None:
            level = 0.5 if self.prob.well == PFC_WELL_01 else 0.0
        n = ctypes.c_int64()
        up = _field(u, self.prob, "u")
        _check(self._lib.pfc_surface_cells(self._h, up, float(level), None, 0, ctypes.byref(n), _stream(stream)))
        cells = torch.empty((max(n.value, 1), 3), dtype=self.prob.dtype, device="cuda")
        _check(self._lib.pfc_surface_cells(self._h, up, float(level), ctypes.c_void_p(cells.data_ptr()), n.value,
                                           ctypes.byref(n), _stream(stream)))
        return cells[: n.value]

    def curvature_histogram(self, cells: torch.Tensor, nbins: int = 100, lo: float = -100.0, hi: float = 100.0,
                            stream=None) -> torch.Tensor:
        """Area-weighted (kappa1, kappa2) histogram of surface cells,
        (nbins, nbins) FP64 on the device; row = kappa1 bin."""
        if cells.dtype != self.prob.dtype or not cells.is_cuda or cells.dim() != 2 or cells.shape[1] != 3:
            raise TypeError("cells must be a CUDA tensor (n, 3) of the problem's dtype")
        cells = cells.contiguous()
        hist = torch.empty((nbins, nbins), dtype=torch.float64, device="cuda")
        _check(self._lib.pfc_curvature_histogram(self._h, ctypes.c_void_p(cells.data_ptr()) if cells.numel() else None,
                                                 cells.shape[0], int(nbins), float(lo), float(hi),
                                                 ctypes.c_void_p(hist.data_ptr()), _stream(stream)))
        return hist

    def curvatures(self, u: torch.Tensor, stream=None):
        k1, k2 = self.new_field(), self.new_field()
        _check(self._lib.pfc_curvatures(self._h, _field(u, self.prob, "u"), _field(k1, self.prob, "k1"),
                                        _field(k2, self.prob, "k2"), _stream(stream)))
        return k1, k2


class Batch:
    """Independent FP32 problems advanced together, one launch per step (pfc_batch_*)."""

    def __init__(self, probs):
        self.probs = list(probs)
        arr = (_CProblem * len(self.probs))(*[p._c() for p in self.probs])
        self._lib = load_library()
        self._h = ctypes.c_void_p()
        _check(self._lib.pfc_batch_create(arr, len(self.probs), ctypes.byref(self._h)))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.pfc_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, fields, nsteps: int, taus, trace: bool = True, stream=None, allow_nonfinite: bool = False):
        """Advance every field in place by nsteps steps.  Returns the trace
        (n, nsteps, 5).  With allow_nonfinite, a problem that diverged does not
        raise: (trace, finite) is returned, finite[k] False for those problems
        (read from their trace rows)."""
        if len(fields) != len(self.probs):
            raise ValueError("one field per problem")
        ptrs = (ctypes.c_void_p * len(fields))(*[_field(f, p, f"u[{k}]").value
                                                 for k, (f, p) in enumerate(zip(fields, self.probs))])
        taus = np.ascontiguousarray(np.broadcast_to(np.asarray(taus, dtype=np.float64), (len(fields),)))
        tr = np.empty((len(fields), max(int(nsteps), 0), 5), dtype=np.float64) if (trace or allow_nonfinite) else None
        rc = self._lib.pfc_batch_run(self._h, ptrs, int(nsteps), taus.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                     tr.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if tr is not None else None,
                                     _stream(stream))
        if allow_nonfinite and rc in (PFC_OK, PFC_ENONFINITE):
            return tr, np.all(np.isfinite(tr), axis=(1, 2))
        _check(rc)
        return tr

    def step(self, fields_in, fields_out, taus, scalars: torch.Tensor | None = None, stream=None):
        """One exact mass-projected step of every problem (enqueue only)."""
        n = len(self.probs)
        if len(fields_in) != n or len(fields_out) != n:
            raise ValueError("one input and one output field per problem")
        pin = (ctypes.c_void_p * n)(*[_field(f, p, f"u_in[{k}]").value for k, (f, p) in enumerate(zip(fields_in, self.probs))])
        pout = (ctypes.c_void_p * n)(*[_field(f, p, f"u_out[{k}]").value for k, (f, p) in enumerate(zip(fields_out, self.probs))])
        taus = np.ascontiguousarray(np.broadcast_to(np.asarray(taus, dtype=np.float64), (n,)))
        sp = None
        if scalars is not None:
            if scalars.dtype != torch.float64 or not scalars.is_cuda or scalars.numel() < 5 * n:
                raise TypeError("scalars must be a CUDA float64 tensor with >= 5 * n entries")
            sp = ctypes.c_void_p(scalars.data_ptr())
        _check(self._lib.pfc_batch_step(self._h, pin, pout, taus.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                        sp, _stream(stream)))

    def step_lazy(self, fields_in, fields_out, taus, first: bool, stream=None):
        """One chained step in the fused form of the mass projection (enqueue
        only): the stored result plus the pending per-problem offset is the
        projected field; ``first`` opens the chain; ``lazy_finish`` adds the
        offsets and closes it."""
        n = len(self.probs)
        if len(fields_in) != n or len(fields_out) != n:
            raise ValueError("one input and one output field per problem")
        pin = (ctypes.c_void_p * n)(*[_field(f, p, f"u_in[{k}]").value for k, (f, p) in enumerate(zip(fields_in, self.probs))])
        pout = (ctypes.c_void_p * n)(*[_field(f, p, f"u_out[{k}]").value for k, (f, p) in enumerate(zip(fields_out, self.probs))])
        taus = np.ascontiguousarray(np.broadcast_to(np.asarray(taus, dtype=np.float64), (n,)))
        _check(self._lib.pfc_batch_step_lazy(self._h, pin, pout, taus.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                             1 if first else 0, _stream(stream)))

    def lazy_finish(self, fields, stream=None):
        """Adds the pending offsets of a chain of ``step_lazy`` calls to the
        fields (its last outputs) and closes the chain (enqueue only)."""
        n = len(self.probs)
        if len(fields) != n:
            raise ValueError("one field per problem")
        pu = (ctypes.c_void_p * n)(*[_field(f, p, f"u[{k}]").value for k, (f, p) in enumerate(zip(fields, self.probs))])
        _check(self._lib.pfc_batch_lazy_finish(self._h, pu, _stream(stream)))

    def step_host(self, host_in, host_out, taus, wait: bool = True, stream=None):
        """One step of every problem from and to host memory (CPU float32
        tensors or arrays of the problems' shapes; pinned memory overlaps the
        copies with the steps).  With wait=False the call only enqueues and
        consecutive calls overlap; host_wait() then makes host_out final."""
        n = len(self.probs)
        if len(host_in) != n or len(host_out) != n:
            raise ValueError("one input and one output buffer per problem")

        def ptr(t, p, name):
            if isinstance(t, torch.Tensor):
                if t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
                    raise TypeError(f"{name} must be a contiguous CPU float32 tensor")
                if tuple(t.shape) != (p.nz, p.ny, p.nx):
                    raise ValueError(f"{name} must have shape {(p.nz, p.ny, p.nx)}")
                return t.data_ptr()
            if t.dtype != np.float32 or not t.flags.c_contiguous or t.shape != (p.nz, p.ny, p.nx):
                raise TypeError(f"{name} must be a C-contiguous float32 array of shape {(p.nz, p.ny, p.nx)}")
            return t.ctypes.data
        pin = (ctypes.c_void_p * n)(*[ptr(t, p, f"host_in[{k}]") for k, (t, p) in enumerate(zip(host_in, self.probs))])
        pout = (ctypes.c_void_p * n)(*[ptr(t, p, f"host_out[{k}]") for k, (t, p) in enumerate(zip(host_out, self.probs))])
        taus = np.ascontiguousarray(np.broadcast_to(np.asarray(taus, dtype=np.float64), (n,)))
        st = _stream(stream)
        _check(self._lib.pfc_batch_step_host(self._h, pin, pout, taus.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                             st))
        if wait:
            self.host_wait(stream)

    def host_wait(self, stream=None):
        _check(self._lib.pfc_batch_host_wait(self._h, _stream(stream)))

    def timing(self, enable: bool = True):
        _check(self._lib.pfc_batch_timing(self._h, 1 if enable else 0))

    def last_timing(self):
        """(step_ms, sweep_ms) of the most recent step; waits for it."""
        a, b = ctypes.c_float(), ctypes.c_float()
        _check(self._lib.pfc_batch_last_timing(self._h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value


class Slab:
    """One z-slab [z0, z0 + nz_local) of a periodic grid split across
    processes (pfc_slab_*): ``prob`` describes the WHOLE grid.  Fields of the
    slab are CUDA tensors (nz_local, ny, nx); its halo is (4, ny, nx): the two
    planes below the slab, then the two above (periodic), filled by the
    caller before every sweep (see paper_2103_04856_gb300.slab)."""

    def __init__(self, prob: Problem, z0: int, nz_local: int):
        self.prob = prob
        self.z0, self.nzl = int(z0), int(nz_local)
        self._lib = load_library()
        self._h = ctypes.c_void_p()
        _check(self._lib.pfc_slab_create(ctypes.byref(prob._c()), self.z0, self.nzl, ctypes.byref(self._h)))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.pfc_slab_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def shape(self):
        return (self.nzl, self.prob.ny, self.prob.nx)

    def new_field(self):
        return torch.empty(self.shape, dtype=self.prob.dtype, device="cuda")

    def new_halo(self):
        return torch.empty((4, self.prob.ny, self.prob.nx), dtype=self.prob.dtype, device="cuda")

    def _t(self, t, shape, name, dtype=None):
        dtype = dtype or self.prob.dtype
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != dtype:
            raise TypeError(f"{name} must be a CUDA {dtype} tensor")
        if tuple(t.shape) != tuple(shape) or not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous with shape {tuple(shape)}")
        return ctypes.c_void_p(t.data_ptr())

    def sweep(self, u, halo, out, mode: int, tau: float, sums_row, stream=None):
        """The fused sweep over the slab (enqueue only); sums_row: CUDA float64
        tensor of SLAB_NSUMS values receiving the slab's sums."""
        op = None if (mode == SLAB_ENERGY and out is None) else self._t(out, self.shape, "out")
        _check(self._lib.pfc_slab_sweep(self._h, self._t(u, self.shape, "u"),
                                        self._t(halo, (4, self.prob.ny, self.prob.nx), "halo"), op, int(mode),
                                        float(tau), self._t(sums_row, (SLAB_NSUMS,), "sums_row", torch.float64),
                                        _stream(stream)))

    def finish(self, sums_all, scalars=None, stream=None):
        """Combine every slab's sums (CUDA float64, (nslabs, SLAB_NSUMS), rank
        order) into the scalars; ``scalars``: optional CUDA float64 tensor of 5."""
        if sums_all.dim() != 2 or sums_all.shape[1] != SLAB_NSUMS:
            raise ValueError("sums_all must be shaped (nslabs, SLAB_NSUMS)")
        sp = None if scalars is None else self._t(scalars, (5,), "scalars", torch.float64)
        _check(self._lib.pfc_slab_finish(self._h, self._t(sums_all, tuple(sums_all.shape), "sums_all", torch.float64),
                                         int(sums_all.shape[0]), sp, _stream(stream)))

    def apply_offset(self, u, stream=None):
        """u += the pending offset of the mass projection; closes the chain."""
        _check(self._lib.pfc_slab_apply_offset(self._h, self._t(u, self.shape, "u"), _stream(stream)))


class HFlow:
    """The paper's generator (Alg. 1): Adam on a periodic vector field A with
    u = k * (div A + m0).  A, m, v: CUDA tensors shaped (3, nz, ny, nx)."""

    def __init__(self, prob: Problem, m0: float, lr: float = 1e-3, betas=(0.9, 0.999), adam_eps: float = 1e-8,
                 blur_sigma: float = 2.0, blur_radius: int = 0):
        self.prob = prob
        self._lib = load_library()
        self._h = ctypes.c_void_p()
        hp = _CHFlow(float(m0), float(lr), float(betas[0]), float(betas[1]), float(adam_eps), float(blur_sigma),
                     int(blur_radius), 0)
        _check(self._lib.pfc_hflow_create(ctypes.byref(prob._c()), ctypes.byref(hp), ctypes.byref(self._h)))
        self.t = 0

    def close(self):
        if getattr(self, "_h", None):
            self._lib.pfc_hflow_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _vec(self, t, name):
        p = self.prob
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != p.dtype:
            raise TypeError(f"{name} must be a CUDA {p.dtype} tensor")
        if tuple(t.shape) != (3, p.nz, p.ny, p.nx) or not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous with shape {(3, p.nz, p.ny, p.nx)}")
        return ctypes.c_void_p(t.data_ptr())

    def set_coefficient_field(self, a_field, stream=None):
        """a(x) of Sec. 5.2 for the flow's energy (None: the constant a)."""
        _check(self._lib.pfc_hflow_set_coefficient_field(self._h, _coef_field(a_field, self.prob), _stream(stream)))

    def set_mass_field(self, m_field, stream=None):
        """m(x) of Sec. 5.2: u = k * (div A + m(x)) (None: the constant m0)."""
        ptr = None if m_field is None else _field(m_field, self.prob, "m_field")
        _check(self._lib.pfc_hflow_set_mass_field(self._h, ptr, _stream(stream)))

    def field(self, A, stream=None):
        p = self.prob
        ut = torch.empty((p.nz, p.ny, p.nx), dtype=p.dtype, device="cuda")
        _check(self._lib.pfc_hflow_field(self._h, self._vec(A, "A"), _field(ut, p, "ut"), _stream(stream)))
        return ut

    def grad(self, A, stream=None):
        gA = torch.empty_like(A)
        G = ctypes.c_double()
        _check(self._lib.pfc_hflow_grad(self._h, self._vec(A, "A"), self._vec(gA, "gA"), ctypes.byref(G),
                                        _stream(stream)))
        return G.value, gA

    def run(self, A, m, v, nsteps: int, trace: bool = True, stream=None):
        tr = np.empty((max(int(nsteps), 0), 5)) if trace else None
        t = ctypes.c_int32(self.t)
        _check(self._lib.pfc_hflow_run(self._h, self._vec(A, "A"), self._vec(m, "m"), self._vec(v, "v"), int(nsteps),
                                       ctypes.byref(t), tr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
                                       if trace else None, _stream(stream)))
        self.t = t.value
        return tr


class HFlowBatch:
    """Many flows of Alg. 1 on grids of one size (FP32), advanced together:
    one launch per kernel of an iteration for all of them.  ``probs`` share
    nx, ny, nz; ``m0s`` are their masses; the blur and Adam's settings are
    shared.  Fields are lists of CUDA float32 tensors shaped (3, nz, ny, nx)."""

    def __init__(self, probs, m0s, lr: float = 1e-3, betas=(0.9, 0.999), adam_eps: float = 1e-8,
                 blur_sigma: float = 2.0, blur_radius: int = 0):
        self.probs = list(probs)
        self._lib = load_library()
        arr = (_CProblem * len(self.probs))(*[p._c() for p in self.probs])
        m0 = np.ascontiguousarray(np.broadcast_to(np.asarray(m0s, dtype=np.float64), (len(self.probs),)))
        hp = _CHFlow(0.0, float(lr), float(betas[0]), float(betas[1]), float(adam_eps), float(blur_sigma),
                     int(blur_radius), 0)
        self._h = ctypes.c_void_p()
        _check(self._lib.pfc_hflow_batch_create(arr, m0.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                                len(self.probs), ctypes.byref(hp), ctypes.byref(self._h)))
        self.t = 0

    def close(self):
        if getattr(self, "_h", None):
            self._lib.pfc_hflow_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ptrs(self, ts, name, shape3=True):
        if len(ts) != len(self.probs):
            raise ValueError(f"{name}: one tensor per instance")
        out = []
        for k, (t, p) in enumerate(zip(ts, self.probs)):
            want = (3, p.nz, p.ny, p.nx) if shape3 else (p.nz, p.ny, p.nx)
            if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32:
                raise TypeError(f"{name}[{k}] must be a CUDA float32 tensor")
            if tuple(t.shape) != want or not t.is_contiguous():
                raise ValueError(f"{name}[{k}] must be contiguous with shape {want}")
            out.append(t.data_ptr())
        return (ctypes.c_void_p * len(out))(*out)

    def field(self, As, stream=None):
        p = self.probs[0]
        uts = [torch.empty((p.nz, p.ny, p.nx), dtype=torch.float32, device="cuda") for _ in self.probs]
        _check(self._lib.pfc_hflow_batch_field(self._h, self._ptrs(As, "A"), self._ptrs(uts, "ut", False),
                                               _stream(stream)))
        return uts

    def run(self, As, ms, vs, nsteps: int, trace: bool = True, stream=None):
        """nsteps Adam steps of every instance in place; returns the trace
        (n, nsteps, 5) if asked."""
        tr = np.empty((len(self.probs), max(int(nsteps), 0), 5)) if trace else None
        t = ctypes.c_int32(self.t)
        _check(self._lib.pfc_hflow_batch_run(self._h, self._ptrs(As, "A"), self._ptrs(ms, "m"), self._ptrs(vs, "v"),
                                             int(nsteps), ctypes.byref(t),
                                             tr.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if trace else None,
                                             _stream(stream)))
        self.t = t.value
        return tr


class PhaseFieldEnergy(torch.autograd.Function):
    """E = F_eps(u) with the gradient from the library's fused adjoint sweep.

    ``PhaseFieldEnergy.apply(u, ctx)``: u a CUDA tensor shaped (nz, ny, nx) of
    the context's dtype; returns a 0-d float64 tensor on u's device."""

    @staticmethod
    def forward(fctx, u, ctx: Context):
        E, g = ctx.energy_and_grad(u.detach().contiguous())
        fctx.save_for_backward(g)
        return torch.tensor(E, dtype=torch.float64, device=u.device)

    @staticmethod
    def backward(fctx, grad_out):
        (g,) = fctx.saved_tensors
        return (grad_out.to(g.dtype) * g), None
