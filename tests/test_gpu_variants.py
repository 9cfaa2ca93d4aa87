"""Extensions of Sec. 5.2 (orientation term, a(x), m(x)) and the viability
diagnostics of Sec. 4.5 on the GPU, against the FP64 oracle, through the C ABI.

Bars: FP64 1e-10 relative (energy, gradient 2-norm, trajectories), FP32 vs
FP64 on the same state 1e-4 relative energy and 1e-3 relative gradient
2-norm, as for the plain eq. Feps.  Diagnostics: FP64 1e-12 relative, FP32
1e-5 relative (sums of positive terms) and exact extremes.
"""
import ctypes
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2103_04856_gb300 import inputs as I

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2103_04856_gb300 import pfc


def P(shape, a, eps=1.5, prec="fp64", h=1.0, xi=1e-6, well=0, **kw):
    nz, ny, nx = shape
    return pfc.Problem(nx=nx, ny=ny, nz=nz, eps=eps, a=tuple(a), h=h, xi=xi, well=well, prec=prec, **kw)


def oprob(p, **kw):
    d = {"a": p.a, "eps": p.eps, "h": p.h, "xi": p.xi, "well": p.well, "mu": p.mu, "theta": p.theta}
    d.update(kw)
    return d


def dev(x, prec):
    return torch.tensor(x, dtype=torch.float64 if prec == "fp64" else torch.float32, device="cuda").contiguous()


def rel(g, gref):
    return float(np.linalg.norm(g - gref) / max(np.linalg.norm(gref), 1e-300))


SHAPES = [(7, 9, 11), (20, 24, 40), (33, 17, 64), (2, 3, 5)]


def _unit(rng):
    t = rng.normal(size=3)
    return tuple(t / np.linalg.norm(t))


# ------------------------------------------------------------ orientation

@pytest.mark.parametrize("shape", SHAPES)
def test_orientation_fp64_vs_oracle(shape):
    rng = np.random.default_rng(sum(shape))
    for well in (0, 1):
        p = P(shape, rng.uniform(-1, 1, 6), eps=1.3, h=0.9, well=well, mu=2.5, theta=_unit(rng))
        u = I.noise(shape, 0.3 if well == 0 else -0.1, 0.1 if well == 0 else 0.3, 5)
        Eo, go = oracle.energy_and_grad(u, oprob(p))
        ctx = pfc.Context(p)
        E, g = ctx.energy_and_grad(dev(u, "fp64"))
        assert E == pytest.approx(Eo, rel=1e-10, abs=1e-12)
        assert rel(g.cpu().numpy(), go) < 1e-10
        assert ctx.energy(dev(u, "fp64")) == pytest.approx(Eo, rel=1e-10, abs=1e-12)


def test_orientation_run_vs_oracle():
    shape = (12, 16, 20)
    rng = np.random.default_rng(4)
    p = P(shape, (1, 0, 1, 0, 0, 0), xi=1e-2, mu=1.5, theta=_unit(rng))
    u = I.noise(shape, 0.3, 0.1, 6)
    ud = dev(u, "fp64")
    tr = pfc.Context(p).run(ud, 70, 1e-3)          # graph replay + remainder
    uo, tro = oracle.run(u, oprob(p), 70, 1e-3)
    assert rel(ud.cpu().numpy(), uo) < 1e-10
    np.testing.assert_allclose(tr, tro, rtol=1e-9, atol=1e-12)


def test_orientation_fp32_vs_fp64():
    shape = (24, 40, 48)
    rng = np.random.default_rng(9)
    th = _unit(rng)
    u = I.noise(shape, 0.3, 0.1, 7).astype(np.float32).astype(np.float64)
    a = (0.2, 0, 1, 0, -0.5, 0)
    E64, g64 = pfc.Context(P(shape, a, mu=3.0, theta=th)).energy_and_grad(dev(u, "fp64"))
    E32, g32 = pfc.Context(P(shape, a, mu=3.0, theta=th, prec="fp32")).energy_and_grad(dev(u, "fp32"))
    assert abs(E32 - E64) / abs(E64) < 1e-4
    g32, g64 = g32.double().cpu().numpy(), g64.cpu().numpy()
    assert rel(g32, g64) < 1e-3
    # per voxel too: a voxel whose D the FP64-accurate refinement got wrong
    # (wrong constants or well) would stand out far above this bar
    assert np.abs(g32 - g64).max() <= 2e-3 * np.abs(g64).max()


def test_orientation_noalloc():
    shape = (10, 20, 36)
    rng = np.random.default_rng(10)
    p = P(shape, rng.uniform(-1, 1, 6), mu=0.8, theta=_unit(rng))
    u = I.noise(shape, 0.3, 0.1, 8)
    Eo, go = oracle.energy_and_grad(u, oprob(p))
    g = torch.empty(shape, dtype=torch.float64, device="cuda")
    E = pfc.energy_and_grad_noalloc(p, dev(u, "fp64"), g)
    assert E == pytest.approx(Eo, rel=1e-10)
    assert rel(g.cpu().numpy(), go) < 1e-10


# ------------------------------------------------------------ a(x)

@pytest.mark.parametrize("shape", SHAPES)
def test_coefficient_field_fp64_vs_oracle(shape):
    rng = np.random.default_rng(100 + sum(shape))
    af = rng.uniform(-1, 1, (6,) + shape)
    p = P(shape, (0,) * 6, eps=1.4, h=1.1)
    u = I.noise(shape, 0.3, 0.1, 11)
    Eo, go = oracle.energy_and_grad(u, oprob(p, a_field=af))
    ctx = pfc.Context(p)
    ctx.set_coefficient_field(dev(af, "fp64"))
    E, g = ctx.energy_and_grad(dev(u, "fp64"))
    assert E == pytest.approx(Eo, rel=1e-10, abs=1e-12)
    assert rel(g.cpu().numpy(), go) < 1e-10
    # cleared: the constant a again
    ctx.set_coefficient_field(None)
    E0 = ctx.energy(dev(u, "fp64"))
    assert E0 == pytest.approx(oracle.energy(u, oprob(p)), rel=1e-10, abs=1e-12)


def test_coefficient_field_with_orientation_and_run():
    """The paper's spatialised example (Table in_spatialized, h = 0.01,
    eps = 0.02) on 4-voxel cubes, with an orientation term: 40 steps (graph
    replays + remainder) against the oracle."""
    n = 4
    af, _ = I.spatialized_fields(n)
    shape = af.shape[1:]
    p = P(shape, (0,) * 6, eps=0.02, h=0.01, xi=1e-2, well=1, mu=50.0, theta=(0.0, 0.6, 0.8))
    u = I.noise(shape, -0.5, 0.3, 12)
    ctx = pfc.Context(p)
    ctx.set_coefficient_field(dev(af, "fp64"))
    ud = dev(u, "fp64")
    tr = ctx.run(ud, 40, 2e-6)
    uo, tro = oracle.run(u, oprob(p, a_field=af), 40, 2e-6)
    assert rel(ud.cpu().numpy(), uo) < 1e-10
    np.testing.assert_allclose(tr, tro, rtol=1e-9, atol=1e-12)


def test_coefficient_field_fp32_vs_fp64():
    n = 16
    af, _ = I.spatialized_fields(n)
    shape = af.shape[1:]
    u = I.noise(shape, -0.5, 0.3, 13).astype(np.float32).astype(np.float64)
    af32 = af.astype(np.float32).astype(np.float64)
    out = {}
    for prec in ("fp64", "fp32"):
        ctx = pfc.Context(P(shape, (0,) * 6, eps=0.02, h=0.01, well=1, prec=prec))
        ctx.set_coefficient_field(dev(af32, prec))
        E, g = ctx.energy_and_grad(dev(u, prec))
        out[prec] = (E, g.double().cpu().numpy())
    assert abs(out["fp32"][0] - out["fp64"][0]) / abs(out["fp64"][0]) < 1e-4
    assert rel(out["fp32"][1], out["fp64"][1]) < 1e-3
    assert np.abs(out["fp32"][1] - out["fp64"][1]).max() <= 2e-3 * np.abs(out["fp64"][1]).max()


# ------------------------------------------------------------ flow with a(x), m(x)

def test_flow_with_spatialised_parameters_vs_oracle():
    n = 4
    af, mf = I.spatialized_fields(n)
    shape = af.shape[1:]
    nz, ny, nx = shape
    p = pfc.Problem(nx=nx, ny=ny, nz=nz, eps=0.02, h=0.01, xi=1e-6, a=(0,) * 6, well=1, prec="fp64",
                    mu=20.0, theta=(1.0, 0.0, 0.0))
    flow = pfc.HFlow(p, m0=0.0, lr=1e-3, blur_sigma=1.0)
    flow.set_coefficient_field(dev(af, "fp64"))
    flow.set_mass_field(dev(mf, "fp64"))
    rng = np.random.default_rng(14)
    A = 2e-4 * rng.standard_normal((3,) + shape)
    Ad = dev(A, "fp64")
    op = {"a": (0,) * 6, "eps": 0.02, "h": 0.01, "xi": 1e-6, "well": 1, "mu": 20.0, "theta": (1.0, 0.0, 0.0),
          "a_field": af}
    fp = {"m0": 0.0, "lr": 1e-3, "blur_sigma": 1.0, "m_field": mf}
    ut = flow.field(Ad).cpu().numpy()
    assert np.max(np.abs(ut - oracle.hflow_field(A, op, fp))) < 1e-13
    assert abs(ut.mean() - mf.mean()) < 1e-13
    md, vd = torch.zeros_like(Ad), torch.zeros_like(Ad)
    tr = flow.run(Ad, md, vd, 5)
    Ao, mo, vo, to, tro = oracle.hflow_run(A, np.zeros_like(A), np.zeros_like(A), op, fp, 5)
    assert rel(Ad.cpu().numpy(), Ao) < 1e-10
    np.testing.assert_allclose(tr, tro, rtol=1e-10, atol=1e-14)
    # cleared: the constant m0 and a again
    flow.set_mass_field(None)
    flow.set_coefficient_field(None)
    assert abs(flow.field(Ad).cpu().numpy().mean()) < 1e-13


@pytest.mark.parametrize("sigma", [1.0, 2.0])
def test_flow_with_mass_field_fp32(sigma):
    """FP32 u = k * (div A + m(x)) (Sec. 5.2) on rows of 24 values, which take
    the kernel that forms div A + m and blurs it along x in one pass (radii 3
    and 6, the latter wider than the 4-voxel y and z axes): field, its mean
    and the trace's mass column against the oracle."""
    af, mf = I.spatialized_fields(4)
    shape = af.shape[1:]
    nz, ny, nx = shape
    a = (1.0, 0.4, 0.8, 0.3, -0.2, 0.1)
    p = pfc.Problem(nx=nx, ny=ny, nz=nz, eps=1.5, h=1.0, xi=1e-6, a=a, well=1, prec="fp32")
    flow = pfc.HFlow(p, m0=0.0, lr=1e-3, blur_sigma=sigma)
    flow.set_mass_field(dev(mf, "fp32"))
    rng = np.random.default_rng(15)
    A = (0.05 * rng.standard_normal((3,) + shape)).astype(np.float32).astype(np.float64)
    Ad = dev(A, "fp32")
    op = {"a": a, "eps": 1.5, "h": 1.0, "xi": 1e-6, "well": 1}
    fp = {"m0": 0.0, "lr": 1e-3, "blur_sigma": sigma, "m_field": mf.astype(np.float32).astype(np.float64)}
    ut = flow.field(Ad).double().cpu().numpy()
    uo = oracle.hflow_field(A, op, fp)
    assert np.max(np.abs(ut - uo)) < 1e-6
    assert abs(ut.mean() - uo.mean()) < 1e-6
    md, vd = torch.zeros_like(Ad), torch.zeros_like(Ad)
    tr = flow.run(Ad, md, vd, 5)
    _, _, _, _, tro = oracle.hflow_run(A, np.zeros_like(A), np.zeros_like(A), op, fp, 5)
    np.testing.assert_allclose(tr[:, 3], tro[:, 3], rtol=0, atol=1e-6)


# ------------------------------------------------------------ diagnostics

# the last five: FP32 rows of 128 to 512 voxels (the row kernel's float4
# path with several warps per row) with one to three tiles of 16 rows
@pytest.mark.parametrize("shape", [(7, 9, 11), (40, 33, 64), (1, 4, 8), (20, 17, 45), (6, 5, 33), (37, 8, 32),
                                   (3, 17, 132), (5, 3, 4), (9, 1, 260),
                                   (5, 16, 128), (9, 48, 256), (7, 32, 512), (1, 16, 512), (6, 24, 128)])
def test_diagnostics_vs_oracle(shape):
    for well in (0, 1):
        u = I.noise(shape, 0.3 if well == 0 else -0.1, 0.2, 15)
        p64 = P(shape, (1, 0, 1, 0, 0, 0), eps=1.7, h=0.8, well=well)
        want = oracle.diagnostics(u, oprob(p64))
        got = pfc.Context(p64).diagnostics(dev(u, "fp64"))
        for k in ("discrepancy", "cahn_hilliard", "ratio"):
            assert got[k] == pytest.approx(want[k], rel=1e-12), k
        assert got["max"] == want["max"] and got["min"] == want["min"]
        u32 = u.astype(np.float32).astype(np.float64)
        want = oracle.diagnostics(u32, oprob(p64))
        got = pfc.Context(P(shape, (1, 0, 1, 0, 0, 0), eps=1.7, h=0.8, well=well, prec="fp32")).diagnostics(
            dev(u32, "fp32"))
        for k in ("discrepancy", "cahn_hilliard", "ratio"):
            assert got[k] == pytest.approx(want[k], rel=1e-5), k
        assert got["max"] == want["max"] and got["min"] == want["min"]


def test_diagnostics_dev_matches_host_call():
    u = I.noise((20, 33, 64), 0.3, 0.2, 5)
    for prec in ("fp32", "fp64"):
        ctx = pfc.Context(P(u.shape, (1, 0, 1, 0, 0, 0), eps=1.7, h=0.8, prec=prec))
        d = dev(u, prec)
        want = ctx.diagnostics(d)
        out = torch.full((5,), float("nan"), dtype=torch.float64, device="cuda")
        got = ctx.diagnostics_dev(d, out).cpu().numpy()
        assert list(got) == [want[k] for k in ("discrepancy", "cahn_hilliard", "ratio", "max", "min")]
        with pytest.raises(ValueError):
            ctx.diagnostics_dev(d, torch.empty(5, dtype=torch.float64))
        # the library itself rejects a host pointer for out_dev
        host = np.zeros(5)
        rc = ctx._lib.pfc_diagnostics_dev(ctx._h, ctypes.c_void_p(d.data_ptr()),
                                          host.ctypes.data_as(ctypes.c_void_p), None)
        assert rc != 0 and not host.any()
        ctx.close()


def test_diagnostics_tanh_slab_and_constant():
    u = I.tanh_slab((64, 8, 8), 32.0, 4.0, 1.0, well=1)
    d = pfc.Context(P(u.shape, (0,) * 6, eps=4.0, well=1)).diagnostics(dev(u, "fp64"))
    sigma = 2 * math.sqrt(2) / 3
    assert d["ratio"] < 0.01
    assert d["cahn_hilliard"] / (sigma * 2 * 64) == pytest.approx(1.0, abs=0.005)
    c = np.full((5, 6, 7), 0.37)
    d = pfc.Context(P(c.shape, (0,) * 6, eps=1.3)).diagnostics(dev(c, "fp64"))
    assert d["ratio"] == pytest.approx(1.0, rel=1e-13)
    assert d["discrepancy"] == pytest.approx(210 * 0.37 ** 2 * 0.63 ** 2 / 1.3, rel=1e-13)


# ------------------------------------------------------------ curvature diagram

def _hist_ref(cells, nbins, lo, hi):
    w = (hi - lo) / nbins
    b1 = np.clip(np.floor((cells[:, 1] - lo) / w).astype(int), 0, nbins - 1)
    b2 = np.clip(np.floor((cells[:, 2] - lo) / w).astype(int), 0, nbins - 1)
    h = np.zeros((nbins, nbins))
    np.add.at(h, (b1, b2), cells[:, 0])
    return h


@pytest.mark.parametrize("case", ["sphere", "noise"])
def test_surface_cells_fp64_vs_oracle(case):
    if case == "sphere":
        n = 40
        u = I.tanh_sphere((n, n, n), 12.0, 2.0, 1.0, center=(20.31, 19.17, 20.23), well=1)
        p = P(u.shape, (0,) * 6, eps=2.0, well=1, h=0.5)
        level = 0.0
    else:
        u = I.noise((13, 17, 19), 0.5, 0.2, 16)
        p = P(u.shape, (0,) * 6, eps=1.5)
        level = 0.5
    want = oracle.surface_cells(u, oprob(p), level)
    ctx = pfc.Context(p)
    got = ctx.surface_cells(dev(u, "fp64"), level).cpu().numpy()
    assert got.shape == want.shape and len(want) > 100
    np.testing.assert_allclose(got[:, 0], want[:, 0], rtol=1e-12, atol=0)
    # curvatures: sqrt(D+) of a nearly umbilic point amplifies rounding (as for pfc_curvatures)
    scale = np.max(np.abs(want[:, 1:]))
    np.testing.assert_allclose(got[:, 1:], want[:, 1:], rtol=0, atol=1e-6 * scale)
    hist = ctx.curvature_histogram(torch.tensor(got, device="cuda"), 40, -2.0, 2.0).cpu().numpy()
    np.testing.assert_allclose(hist, _hist_ref(got, 40, -2.0, 2.0), rtol=1e-12, atol=1e-14)
    assert hist.sum() == pytest.approx(want[:, 0].sum(), rel=1e-12)
    # a short buffer gets the first records and the full count
    small = torch.zeros((10, 3), dtype=torch.float64, device="cuda")
    import ctypes
    cnt = ctypes.c_int64()
    lib = pfc.load_library()
    rc = lib.pfc_surface_cells(ctx._h, ctypes.c_void_p(dev(u, "fp64").data_ptr()), level,
                               ctypes.c_void_p(small.data_ptr()), 10, ctypes.byref(cnt), None)
    torch.cuda.synchronize()
    assert rc == 0 and cnt.value == len(want)
    np.testing.assert_allclose(small.cpu().numpy()[:, 0], want[:10, 0], rtol=1e-12)


def test_surface_cells_fp32():
    n = 48
    u = I.tanh_sphere((n, n, n), 14.0, 2.0, 1.0, center=(24.31, 23.17, 24.23), well=0)
    u = u.astype(np.float32).astype(np.float64)
    p64 = P(u.shape, (0,) * 6, eps=2.0)
    want = oracle.surface_cells(u, oprob(p64), 0.5)
    got = pfc.Context(P(u.shape, (0,) * 6, eps=2.0, prec="fp32")).surface_cells(dev(u, "fp32"), 0.5)
    got = got.double().cpu().numpy()
    assert got.shape == want.shape
    assert got[:, 0].sum() == pytest.approx(want[:, 0].sum(), rel=1e-5)
    assert np.max(np.abs(got[:, 0] - want[:, 0])) < 1e-4 * np.max(want[:, 0])
    A = want[:, 0].sum()
    for k in (1, 2):
        assert (got[:, 0] * got[:, k]).sum() / A == pytest.approx((want[:, 0] * want[:, k]).sum() / A, rel=1e-3)


# ------------------------------------------------------------ tangent-projected M

@pytest.mark.parametrize("shape", SHAPES)
def test_projected_fp64_vs_oracle(shape):
    rng = np.random.default_rng(200 + sum(shape))
    for well, mu in ((0, 0.0), (1, 1.3)):
        p = P(shape, rng.uniform(-1, 1, 6), eps=1.3, h=0.9, well=well, proj=1, mu=mu, theta=_unit(rng))
        u = I.noise(shape, 0.3 if well == 0 else -0.1, 0.1 if well == 0 else 0.3, 17)
        Eo, go = oracle.energy_and_grad(u, oprob(p, proj=1))
        ctx = pfc.Context(p)
        E, g = ctx.energy_and_grad(dev(u, "fp64"))
        assert E == pytest.approx(Eo, rel=1e-10, abs=1e-12)
        assert rel(g.cpu().numpy(), go) < 1e-10
        assert ctx.energy(dev(u, "fp64")) == pytest.approx(Eo, rel=1e-10, abs=1e-12)


def test_projected_with_coefficient_field_and_run():
    """70 steps with a(x) near p = k1^2 + k2^2 (a well-posed descent: with
    random-sign coefficients the field grows and the oracle itself moves by
    1e-3 under a 1e-13 perturbation of u0, so no two implementations agree)."""
    shape = (12, 16, 20)
    rng = np.random.default_rng(18)
    af = np.array([1, 0, 1, 0, 0, 0.0])[:, None, None, None] + 0.2 * rng.uniform(-1, 1, (6,) + shape)
    p = P(shape, (0,) * 6, xi=1e-2, proj=1)
    u = I.noise(shape, 0.3, 0.1, 19)
    ctx = pfc.Context(p)
    ctx.set_coefficient_field(dev(af, "fp64"))
    ud = dev(u, "fp64")
    tr = ctx.run(ud, 70, 1e-3)
    uo, tro = oracle.run(u, oprob(p, proj=1, a_field=af), 70, 1e-3)
    assert rel(ud.cpu().numpy(), uo) < 1e-10
    np.testing.assert_allclose(tr, tro, rtol=1e-9, atol=1e-12)


def test_projected_fp32_vs_fp64_and_sphere():
    """FP32 against FP64 on the same state (noise, asymmetric p), and the
    128^3 tanh sphere R = 32, eps = 2 (p = k1^2 + k2^2): FP32 energy against
    the oracle, whose ratio to sigma 8 pi is 1.0077."""
    shape = (24, 40, 48)
    u = I.noise(shape, 0.3, 0.1, 20).astype(np.float32).astype(np.float64)
    a = (0.2, 0, 1, 0, -0.5, 0)
    E64, g64 = pfc.Context(P(shape, a, proj=1)).energy_and_grad(dev(u, "fp64"))
    E32, g32 = pfc.Context(P(shape, a, proj=1, prec="fp32")).energy_and_grad(dev(u, "fp32"))
    assert abs(E32 - E64) / abs(E64) < 1e-4
    assert rel(g32.double().cpu().numpy(), g64.cpu().numpy()) < 1e-3
    n = 128
    s = I.tanh_sphere((n, n, n), 32.0, 2.0, 1.0, center=(64.3, 64.1, 64.2)).astype(np.float32).astype(np.float64)
    p32 = P(s.shape, (1, 0, 1, 0, 0, 0), eps=2.0, proj=1, prec="fp32")
    Eo = oracle.energy(s, oprob(p32, proj=1))
    assert pfc.Context(p32).energy(dev(s, "fp32")) == pytest.approx(Eo, rel=1e-4)


def test_projected_curvatures_and_flow_vs_oracle():
    shape = (10, 12, 14)
    u = I.noise(shape, 0.3, 0.15, 21)
    p = P(shape, (1.0, 0.4, 0.8, 0.3, -0.2, 0.1), proj=1)
    k1, k2 = pfc.Context(p).curvatures(dev(u, "fp64"))
    o1, o2 = oracle.curvatures(u, oprob(p, proj=1))
    sc = np.max(np.abs(o1))
    assert np.max(np.abs(k1.cpu().numpy() - o1)) < 1e-6 * sc
    assert np.max(np.abs(k2.cpu().numpy() - o2)) < 1e-6 * sc
    flow = pfc.HFlow(p, m0=0.3, lr=1e-3, blur_sigma=1.0)
    rng = np.random.default_rng(22)
    A = 0.04 * rng.standard_normal((3,) + shape)
    G, gA = flow.grad(dev(A, "fp64"))
    Go, gAo = oracle.hflow_grad(A, oprob(p, proj=1), {"m0": 0.3, "blur_sigma": 1.0})
    assert G == pytest.approx(Go, rel=1e-10)
    assert rel(gA.cpu().numpy(), gAo) < 1e-10
