"""Seeded synthetic inputs: initial fields, analytic shapes and workload specs.

This module holds no arithmetic of the energy or of its gradient.  It only
draws the fields the method is run on and names the workloads, so that the
CUDA path, the tests, the benchmark and the oracle all start from the same
numbers.  Everything is float64 numpy; callers round to float32 themselves.

Array layout: (nz, ny, nx), C-contiguous, u[z, y, x]; voxel (i, j, k) sits at
x = i*h, y = j*h, z = k*h.

Shapes follow the tanh profile of Sec. 3.1 (eq. tanh_profile): with d the
signed distance to the surface (positive inside),
  well 0 (wells 0 and 1):  u = (1 + tanh(d / (sqrt(2) eps))) / 2
  well 1 (wells -1 and 1): u = tanh(d / (sqrt(2) eps)).
Initial fields follow Sec. 4.1 (white noise) in the form u0 = m + s * N(0, 1)
drawn from numpy's PCG64 ``default_rng(seed)``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def noise(shape, mean: float, std: float, seed: int) -> np.ndarray:
    """u0 = mean + std * N(0,1), iid per voxel, float64, shape (nz, ny, nx)."""
    rng = np.random.default_rng(seed)
    return mean + std * rng.standard_normal(tuple(shape))


def _profile(d: np.ndarray, eps: float, well: int) -> np.ndarray:
    t = np.tanh(d / (math.sqrt(2.0) * eps))
    return t if well == 1 else 0.5 * (1.0 + t)


def _coords(shape, h):
    nz, ny, nx = shape
    z = np.arange(nz, dtype=np.float64)[:, None, None] * h
    y = np.arange(ny, dtype=np.float64)[None, :, None] * h
    x = np.arange(nx, dtype=np.float64)[None, None, :] * h
    return x, y, z


def tanh_sphere(shape, R: float, eps: float, h: float = 1.0, center=None, well: int = 0) -> np.ndarray:
    """Ball of radius R (centre at voxel index shape//2 unless given, in x,y,z order)."""
    nz, ny, nx = shape
    cx, cy, cz = center if center is not None else (nx // 2 * h, ny // 2 * h, nz // 2 * h)
    x, y, z = _coords(shape, h)
    d = R - np.sqrt((x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2)
    return _profile(d, eps, well)


def tanh_cylinder(shape, r: float, eps: float, h: float = 1.0, center=None, well: int = 0) -> np.ndarray:
    """z-periodic solid cylinder of radius r, axis parallel to z through (cx, cy)."""
    nz, ny, nx = shape
    cx, cy = center if center is not None else (nx // 2 * h, ny // 2 * h)
    x, y, z = _coords(shape, h)
    d = r - np.sqrt((x - cx) ** 2 + (y - cy) ** 2) + 0.0 * z
    return _profile(d, eps, well)


def tanh_slab(shape, width: float, eps: float, h: float = 1.0, well: int = 0) -> np.ndarray:
    """x,y-periodic slab |z - zc| < width/2 (two flat interfaces), periodic in z."""
    nz, ny, nx = shape
    L = nz * h
    x, y, z = _coords(shape, h)
    dz = np.abs(z - 0.5 * L)
    d = 0.5 * width - dz + 0.0 * x + 0.0 * y
    return _profile(d, eps, well)


# ---------------------------------------------------------------- workloads

def smaller_first_poly_to_a(a_, b_, c_, d_=0.0, e_=0.0):
    """Coefficients written with kappa1 the SMALLER curvature,
    a k1^2 + b k2^2 + c k1 k2 + d k1 + e k2, in the paper's order
    (a20, a11, a02, a10, a01, a00) with kappa1 the LARGER curvature."""
    return (float(b_), float(c_), float(a_), float(e_), float(d_), 0.0)


@dataclass
class Instance:
    """One problem: grid, parameters, initial field recipe."""
    name: str
    shape: tuple            # (nz, ny, nx)
    eps: float
    a: tuple
    h: float = 1.0
    xi: float = 1e-6
    well: int = 0
    tau: float = 1e-3
    init: dict = field(default_factory=dict)

    def problem(self) -> dict:
        return {"h": self.h, "eps": self.eps, "xi": self.xi, "a": tuple(self.a), "well": self.well}

    def field(self) -> np.ndarray:
        k = self.init["kind"]
        if k == "noise":
            return noise(self.shape, self.init["mean"], self.init["std"], self.init["seed"])
        if k == "sphere":
            return tanh_sphere(self.shape, self.init["R"], self.eps, self.h, well=self.well)
        if k == "cylinder":
            return tanh_cylinder(self.shape, self.init["r"], self.eps, self.h, well=self.well)
        if k == "slab":
            return tanh_slab(self.shape, self.init["width"], self.eps, self.h, well=self.well)
        raise ValueError(f"unknown init kind {k}")


def willmore_descent_32() -> Instance:
    """Plain FP64 method on a periodic 32^3 grid: h=1, eps=1.5, p = k1^2 + k2^2,
    W = u^2(1-u)^2, u0 = 0.3 + 0.1 N(0,1) (seed 0), 100 steps of size 1e-3."""
    return Instance("willmore_descent_32", (32, 32, 32), 1.5, (1.0, 0.0, 1.0, 0.0, 0.0, 0.0),
                    init={"kind": "noise", "mean": 0.3, "std": 0.1, "seed": 0})


def validation_128(shape_kind: str = "sphere", poly: str = "k1^2+k2^2", n: int = 128, eps: float = 2.0):
    """128^3 validation shapes: tanh sphere R = n/4 (32 at 128^3) or z-periodic
    cylinder r = 20 n/128, eps = 2; p = k1^2 + k2^2 or p = k1 k2."""
    a = {"k1^2+k2^2": (1.0, 0.0, 1.0, 0.0, 0.0, 0.0), "k1k2": (0.0, 1.0, 0.0, 0.0, 0.0, 0.0)}[poly]
    if shape_kind == "sphere":
        init = {"kind": "sphere", "R": n / 4.0}
    else:
        init = {"kind": "cylinder", "r": 20.0 * n / 128.0}
    return Instance(f"{shape_kind}_{n}_{poly}", (n, n, n), eps, a, init=init)


def validation_set_128():
    """The four 128^3 validation problems: {sphere, cylinder} x {k1^2+k2^2, k1 k2}."""
    return [validation_128(s, p) for s in ("sphere", "cylinder") for p in ("k1^2+k2^2", "k1k2")]


def tube_descent_256(n: int = 256) -> Instance:
    """256^3 FP32, p = k1^2 + 0.2 k2^2 - 0.5 k1 (k1 the smaller curvature),
    u0 = 0.25 + 0.1 N(0,1) (seed 1), eps = 1.5."""
    return Instance(f"tube_descent_{n}", (n, n, n), 1.5, smaller_first_poly_to_a(1.0, 0.2, 0.0, -0.5, 0.0),
                    init={"kind": "noise", "mean": 0.25, "std": 0.1, "seed": 1})


def membrane_descent_512(n: int = 512) -> Instance:
    """512^3 FP32, eps = 2, p = 0.2 k1^2 + k2^2 + 0.3 k1 k2 (k1 the smaller),
    u0 = 0.3 + 0.1 N(0,1) (seed 2)."""
    return Instance(f"membrane_descent_{n}", (n, n, n), 2.0, smaller_first_poly_to_a(0.2, 1.0, 0.3),
                    init={"kind": "noise", "mean": 0.3, "std": 0.1, "seed": 2})


def batch_instances(n_inst: int = 64, sizes=(64, 96, 128), seed: int = 12345):
    """Mixed-size batch: size uniform in ``sizes``; (a, b, c, d, e) uniform in
    [-1,1]^2 x [-0.5,0.5] x [-1,1]^2 (kappa1 the smaller curvature); volume
    fraction vf uniform in [0.15, 0.45]; u0 = vf + 0.1 N(0,1) with seed 100+k;
    eps = 1.5, tau = 1e-3."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_inst):
        n = int(sizes[int(rng.integers(len(sizes)))])
        a_, b_ = rng.uniform(-1.0, 1.0, 2)
        c_ = rng.uniform(-0.5, 0.5)
        d_, e_ = rng.uniform(-1.0, 1.0, 2)
        vf = rng.uniform(0.15, 0.45)
        out.append(Instance(f"batch_{k}", (n, n, n), 1.5, smaller_first_poly_to_a(a_, b_, c_, d_, e_),
                            init={"kind": "noise", "mean": float(vf), "std": 0.1, "seed": 100 + k}))
    return out


def paper_flow_100(seed: int = 0):
    """The generator's setting of Sec. 4.1 and Fig. cvg_1: a 100^3 grid with
    spacing 0.01, eps = 0.02, the paper's double well (wells -1 and 1),
    a = (1, 2.4, 9, 30, 170, -195), mass m0 = -0.66, blur of 2 voxels, Adam with
    lr 1e-3 and betas (0.9, 0.999).  A0 is white noise scaled so that div A0
    has a standard deviation of about 0.1 (the paper does not give the scale).
    Returns (problem dict, flow dict, A0 of shape (3, 100, 100, 100))."""
    n, h = 100, 0.01
    prob = {"shape": (n, n, n), "h": h, "eps": 0.02, "xi": 1e-6, "a": (1.0, 2.4, 9.0, 30.0, 170.0, -195.0), "well": 1}
    flow = {"m0": -0.66, "lr": 1e-3, "beta1": 0.9, "beta2": 0.999, "adam_eps": 1e-8, "blur_sigma": 2.0}
    scale = 2.0 * h * 0.1 / math.sqrt(6.0)
    rng = np.random.default_rng(seed)
    A0 = scale * rng.standard_normal((3, n, n, n))
    return prob, flow, A0


# The four generation parameters of the paper's spatialised example (Sec. 5.2,
# Table in_spatialized): a in the paper's order, and the mass m0.
SPATIALIZED_TABLE = (
    ((2.0, 2.0, 2.0, 0.0, 0.0, 0.0), -0.4),
    ((1.0, 2.0, 6.0, -40.0, -40.0, 400.0), -0.6),
    ((2.0, 2.0, 2.0, -75.0, -75.0, 937.5), -0.7),
    ((2.0, 2.0, 11.0, -180.0, -90.0, 4050.0), -0.7),
)


def spatialized_fields(n_cube: int, table=SPATIALIZED_TABLE):
    """a(x) and m(x) of the spatialised example (Sec. 5.2): six cubes of edge
    n_cube along x carry (p1, p1, p2, p3, p4, p4) at their mid-planes
    x = (k + 1/2) n_cube, linearly interpolated in between and periodically
    across the wrap.  Returns (a_field (6, n, n, 6n), m_field (n, n, 6n)),
    float64."""
    nodes = [table[0], table[0], table[1], table[2], table[3], table[3]]
    nx = 6 * n_cube
    xs = np.arange(nx, dtype=np.float64)
    a_line = np.empty((6, nx))
    m_line = np.empty(nx)
    for i, x in enumerate(xs):
        t = x / n_cube - 0.5                 # node coordinate
        k0 = int(math.floor(t)) % 6
        k1 = (k0 + 1) % 6
        w = t - math.floor(t)
        a_line[:, i] = (1 - w) * np.asarray(nodes[k0][0]) + w * np.asarray(nodes[k1][0])
        m_line[i] = (1 - w) * nodes[k0][1] + w * nodes[k1][1]
    shape = (n_cube, n_cube, nx)
    a_field = np.broadcast_to(a_line[:, None, None, :], (6,) + shape).copy()
    m_field = np.broadcast_to(m_line[None, None, :], shape).copy()
    return a_field, m_field
