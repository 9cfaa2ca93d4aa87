"""FP64 CPU oracle of the phase-field curvature energy (Song, arXiv 2103.04856).

TEST INFRASTRUCTURE ONLY.  The oracle is the plain, single-threaded FP64
restatement of eq. Feps (Sec. 3.2) and of its exact discrete gradient that the
CUDA path is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import it; the product package never
does.  It shares no code with the CUDA library and imports nothing from it.

Every function takes float64 numpy arrays shaped (nz, ny, nx), C-contiguous,
periodic in all axes, and a problem dictionary with keys
``h, eps, xi, a (6 values: a20 a11 a02 a10 a01 a00, kappa1 >= kappa2), well``
(``well`` 0: W(u)=u^2(1-u)^2, wells 0/1; 1: the paper's W(s)=(1-s^2)^2/4).

Parity status per function (what pins it, in tests/test_oracle_pins.py):
  energy           closed forms (tanh sphere/cylinder/slab), Willmore and
                   Helfrich reductions, phase-swap and double-well identities
  energy_and_grad  central finite differences (all voxels of small grids) and
                   torch FP64 autograd of the forward formula
  grad_sampled     equals energy_and_grad at the sampled voxels
  step / run       mass conservation, lambda = mean(g), descent of E
  curvatures       kappa1 + kappa2 = H^eps, kappa1 kappa2 <= K^eps, tanh sphere
  b_to_a           the eight printed rows of the paper's two parameter tables
  mu, theta        (Sec. 5.2 orientation term) closed form on a sine field, the
                   axis-sum identity with the a00 term, central differences
  a_field          (Sec. 5.2 a(x)) linearity in a: E equals the sum of the
                   per-coefficient densities weighted by a(x); central differences
  diagnostics      (Sec. 4.5) constant field and tanh-slab closed forms
  proj (M_P)       planar profiles give M_P = 0 (closed form of E), tanh
                   sphere F/(sigma 8 pi) -> 1, axis permutations, central
                   differences of the gradient, torch autograd
  surface_cells    (Sec. 4.1) flat interfaces: exact area, zero curvature; tanh
                   sphere and cylinder: area and curvatures converge to the
                   sharp values; every triangle lies in its cube
  hflow_*          (Alg. 1) mass = m0 exactly, blur moments and symmetry, the
                   closed-form first Adam step, central differences of G(A)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pf_oracle.c")
_LIB = os.path.join(_HERE, "libpf_oracle.so")
_lock = threading.Lock()
_lib = None


class _HFlow(ctypes.Structure):
    _fields_ = [("m0", ctypes.c_double), ("lr", ctypes.c_double), ("beta1", ctypes.c_double),
                ("beta2", ctypes.c_double), ("adam_eps", ctypes.c_double), ("blur_sigma", ctypes.c_double),
                ("blur_radius", ctypes.c_int), ("m_field", ctypes.POINTER(ctypes.c_double))]


class _Problem(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("h", ctypes.c_double), ("eps", ctypes.c_double), ("xi", ctypes.c_double),
        ("a", ctypes.c_double * 6), ("well", ctypes.c_int),
        ("mu", ctypes.c_double), ("theta", ctypes.c_double * 3), ("a_field", ctypes.POINTER(ctypes.c_double)),
        ("proj", ctypes.c_int),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable flags: it also builds on aarch64)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER(_Problem)
            D = ctypes.POINTER(ctypes.c_double)
            for name, args in [
                ("pfo_energy", [P, D, D]),
                ("pfo_energy_and_grad", [P, D, D, D]),
                ("pfo_density", [P, D, D]),
                ("pfo_grad_sampled", [P, D, ctypes.c_int, ctypes.POINTER(ctypes.c_long), D]),
                ("pfo_step", [P, D, D, ctypes.c_double, D]),
                ("pfo_run", [P, D, ctypes.c_int, ctypes.c_double, D]),
                ("pfo_curvatures", [P, D, D, D]),
                ("pfo_diagnostics", [P, D, D]),
            ]:
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = ctypes.c_int
            H = ctypes.POINTER(_HFlow)
            for name, args in [
                ("pfo_blur", [P, H, D]),
                ("pfo_hflow_field", [P, H, D, D]),
                ("pfo_hflow_grad", [P, H, D, D, D]),
                ("pfo_hflow_run", [P, H, D, D, D, ctypes.c_int, ctypes.POINTER(ctypes.c_int), D]),
            ]:
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = ctypes.c_int
            lib.pfo_surface_cells.argtypes = [P, D, ctypes.c_double, ctypes.c_long, D, ctypes.POINTER(ctypes.c_long)]
            lib.pfo_surface_cells.restype = ctypes.c_int
            lib.pfo_gauss_weights.argtypes = [ctypes.c_double, ctypes.c_int, D]
            lib.pfo_gauss_weights.restype = None
            lib.pfo_b_to_a.argtypes = [D, D]
            lib.pfo_b_to_a.restype = None
            _lib = lib
    return _lib


def _prob(u: np.ndarray, p: dict) -> _Problem:
    """Problem keys: h, eps, xi, a, well; optional (Sec. 5.2) mu, theta (3
    values, x y z) and a_field (shape (6, nz, ny, nx): a(x)); proj = 1 for the
    tangent-projected M = -eps P Hess u P."""
    nz, ny, nx = u.shape
    a = p["a"]
    s = _Problem(nx, ny, nz, float(p.get("h", 1.0)), float(p["eps"]),
                 float(p.get("xi", 1e-6)), (ctypes.c_double * 6)(*[float(v) for v in a]),
                 int(p.get("well", 0)), float(p.get("mu", 0.0)),
                 (ctypes.c_double * 3)(*[float(v) for v in p.get("theta", (0.0, 0.0, 0.0))]), None,
                 int(p.get("proj", 0)))
    af = p.get("a_field")
    if af is not None:
        af = np.ascontiguousarray(af, dtype=np.float64)
        if af.shape != (6, nz, ny, nx):
            raise ValueError("a_field must be shaped (6, nz, ny, nx)")
        s.a_field = _ptr(af)
        s._keep = af          # the array must outlive the call
    return s


def _f64(u):
    u = np.ascontiguousarray(u, dtype=np.float64)
    if u.ndim != 3:
        raise ValueError("u must be a 3-D array shaped (nz, ny, nx)")
    return u


def _ptr(x):
    return x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ok(rc, name):
    if rc != 0:
        raise ValueError(f"{name}: invalid arguments")


def energy(u, p) -> float:
    u = _f64(u)
    E = ctypes.c_double()
    _ok(_load().pfo_energy(ctypes.byref(_prob(u, p)), _ptr(u), ctypes.byref(E)), "energy")
    return E.value


def density(u, p) -> np.ndarray:
    u = _f64(u)
    e = np.empty_like(u)
    _ok(_load().pfo_density(ctypes.byref(_prob(u, p)), _ptr(u), _ptr(e)), "density")
    return e


def energy_and_grad(u, p):
    u = _f64(u)
    g = np.empty_like(u)
    E = ctypes.c_double()
    _ok(_load().pfo_energy_and_grad(ctypes.byref(_prob(u, p)), _ptr(u), ctypes.byref(E), _ptr(g)),
        "energy_and_grad")
    return E.value, g


def grad_sampled(u, p, idx) -> np.ndarray:
    u = _f64(u)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    g = np.empty(idx.shape[0], dtype=np.float64)
    _ok(_load().pfo_grad_sampled(ctypes.byref(_prob(u, p)), _ptr(u), int(idx.shape[0]),
                                 idx.ctypes.data_as(ctypes.POINTER(ctypes.c_long)), _ptr(g)),
        "grad_sampled")
    return g


def step(u, p, tau):
    """Returns (u_next, scalars) with scalars = [E(u), mean(u), lambda, max|g|, mean|g|]."""
    u = _f64(u)
    out = np.empty_like(u)
    sc = np.empty(5, dtype=np.float64)
    _ok(_load().pfo_step(ctypes.byref(_prob(u, p)), _ptr(u), _ptr(out), float(tau), _ptr(sc)), "step")
    return out, sc


def run(u, p, nsteps, tau):
    """Returns (u_final, trace[nsteps, 5]) with the rows of ``step``."""
    u = _f64(u).copy()
    tr = np.empty((max(int(nsteps), 0), 5), dtype=np.float64)
    _ok(_load().pfo_run(ctypes.byref(_prob(u, p)), _ptr(u), int(nsteps), float(tau), _ptr(tr)), "run")
    return u, tr


def curvatures(u, p):
    u = _f64(u)
    k1 = np.empty_like(u)
    k2 = np.empty_like(u)
    _ok(_load().pfo_curvatures(ctypes.byref(_prob(u, p)), _ptr(u), _ptr(k1), _ptr(k2)), "curvatures")
    return k1, k2


def diagnostics(u, p) -> dict:
    """Sec. 4.5 viability quantities: discrepancy and Cahn-Hilliard integrals,
    their ratio, max and min of u."""
    u = _f64(u)
    out = np.empty(5)
    _ok(_load().pfo_diagnostics(ctypes.byref(_prob(u, p)), _ptr(u), _ptr(out)), "diagnostics")
    return {"discrepancy": out[0], "cahn_hilliard": out[1], "ratio": out[2], "max": out[3], "min": out[4]}


def surface_cells(u, p, level: float) -> np.ndarray:
    """Cells of the curvature diagram (Sec. 4.1): rows (area, kappa1, kappa2)
    of the triangles of {u = level}, in cube / tetrahedron / triangle order."""
    u = _f64(u)
    lib = _load()
    n = ctypes.c_long()
    _ok(lib.pfo_surface_cells(ctypes.byref(_prob(u, p)), _ptr(u), float(level), 0, None, ctypes.byref(n)),
        "surface_cells")
    cells = np.empty((max(n.value, 1), 3))
    _ok(lib.pfo_surface_cells(ctypes.byref(_prob(u, p)), _ptr(u), float(level), n.value, _ptr(cells),
                              ctypes.byref(n)), "surface_cells")
    return cells[: n.value]


def b_to_a(b) -> np.ndarray:
    b = np.ascontiguousarray(b, dtype=np.float64)
    if b.shape != (7,):
        raise ValueError("b must have 7 entries")
    a = np.empty(6, dtype=np.float64)
    _load().pfo_b_to_a(_ptr(b), _ptr(a))
    return a


# ---------------------------------------------------------------- Alg. 1

def _flow(fp: dict) -> _HFlow:
    """Flow keys: m0, lr, beta1, beta2, adam_eps, blur_sigma, blur_radius;
    optional m_field (shape (nz, ny, nx): the spatialised mass of Sec. 5.2)."""
    sigma = float(fp.get("blur_sigma", 0.0))
    R = int(fp.get("blur_radius", 0)) or (int(np.ceil(3.0 * sigma)) if sigma > 0 else 0)
    s = _HFlow(float(fp.get("m0", 0.0)), float(fp.get("lr", 1e-3)), float(fp.get("beta1", 0.9)),
               float(fp.get("beta2", 0.999)), float(fp.get("adam_eps", 1e-8)), sigma, R, None)
    mf = fp.get("m_field")
    if mf is not None:
        mf = np.ascontiguousarray(mf, dtype=np.float64)
        s.m_field = _ptr(mf)
        s._keep = mf
    return s


def _A(A):
    A = np.ascontiguousarray(A, dtype=np.float64)
    if A.ndim != 4 or A.shape[0] != 3:
        raise ValueError("A must be shaped (3, nz, ny, nx)")
    return A


def gauss_weights(sigma: float, R: int) -> np.ndarray:
    w = np.empty(2 * R + 1)
    _load().pfo_gauss_weights(float(sigma), int(R), _ptr(w))
    return w


def blur(a, p: dict, fp: dict) -> np.ndarray:
    """k * a (periodic separable Gaussian of std fp['blur_sigma'])."""
    a = _f64(a).copy()
    _ok(_load().pfo_blur(ctypes.byref(_prob(a, p)), ctypes.byref(_flow(fp)), _ptr(a)), "blur")
    return a


def hflow_field(A, p: dict, fp: dict) -> np.ndarray:
    """ut = k * (div A + m0) (Alg. 1, change of variable then blur)."""
    A = _A(A)
    ut = np.empty(A.shape[1:])
    _ok(_load().pfo_hflow_field(ctypes.byref(_prob(ut, p)), ctypes.byref(_flow(fp)), _ptr(A), _ptr(ut)), "hflow_field")
    return ut


def hflow_grad(A, p: dict, fp: dict):
    """(G, dG/dA) with G(A) = F_eps(k * (div A + m0))."""
    A = _A(A)
    gA = np.empty_like(A)
    G = ctypes.c_double()
    _ok(_load().pfo_hflow_grad(ctypes.byref(_prob(A[0], p)), ctypes.byref(_flow(fp)), _ptr(A), ctypes.byref(G),
                               _ptr(gA)), "hflow_grad")
    return G.value, gA


def hflow_run(A, m, v, p: dict, fp: dict, nsteps: int, t: int = 0):
    """nsteps Adam steps of Alg. 1; returns (A, m, v, t, trace[nsteps, 5])."""
    A, m, v = _A(A).copy(), _A(m).copy(), _A(v).copy()
    tt = ctypes.c_int(int(t))
    tr = np.empty((max(int(nsteps), 0), 5))
    _ok(_load().pfo_hflow_run(ctypes.byref(_prob(A[0], p)), ctypes.byref(_flow(fp)), _ptr(A), _ptr(m), _ptr(v),
                              int(nsteps), ctypes.byref(tt), _ptr(tr)), "hflow_run")
    return A, m, v, tt.value, tr
