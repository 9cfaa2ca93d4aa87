"""Alg. 1 on the GPU (pfc_hflow_*) against the oracle's restatement."""
import numpy as np
import pytest
import torch

import oracle
from paper_2103_04856_gb300 import inputs as I

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2103_04856_gb300 import pfc


def setup(shape, prec="fp64", sigma=1.5, xi=1e-6, a=(1.0, 0.4, 0.8, 0.3, -0.2, 0.1), seed=0, m0=0.3, lr=1e-3):
    nz, ny, nx = shape
    p = pfc.Problem(nx=nx, ny=ny, nz=nz, eps=1.5, a=a, xi=xi, prec=prec)
    rng = np.random.default_rng(seed)
    A = 0.04 * rng.standard_normal((3,) + tuple(shape))
    if prec == "fp32":
        A = A.astype(np.float32).astype(np.float64)
    op = {"a": a, "eps": 1.5, "xi": xi, "h": 1.0, "well": 0}
    fp = {"m0": m0, "blur_sigma": sigma, "lr": lr}
    flow = pfc.HFlow(p, m0=m0, lr=lr, blur_sigma=sigma)
    dt = torch.float64 if prec == "fp64" else torch.float32
    return flow, torch.tensor(A, dtype=dt, device="cuda"), A, op, fp


@pytest.mark.parametrize("shape,sigma", [((12, 10, 16), 1.5), ((7, 9, 11), 0.0), ((20, 24, 40), 2.0),
                                         ((20, 24, 40), 6.0), ((9, 13, 36), 5.4)])
def test_field_and_grad_vs_oracle(shape, sigma):
    flow, Ad, A, op, fp = setup(shape, sigma=sigma)
    ut = flow.field(Ad).cpu().numpy()
    uo = oracle.hflow_field(A, op, fp)
    assert np.max(np.abs(ut - uo)) < 1e-13
    assert abs(ut.mean() - 0.3) < 1e-14
    G, gA = flow.grad(Ad)
    Go, gAo = oracle.hflow_grad(A, op, fp)
    assert G == pytest.approx(Go, rel=1e-10)
    gA = gA.cpu().numpy()
    assert np.linalg.norm(gA - gAo) / np.linalg.norm(gAo) < 1e-10


def test_run_vs_oracle_short_horizon():
    """5 Adam steps (fresh moments), then 3 more continuing the step count."""
    shape = (12, 10, 16)
    flow, Ad, A, op, fp = setup(shape)
    md, vd = torch.zeros_like(Ad), torch.zeros_like(Ad)
    tr = flow.run(Ad, md, vd, 5)
    Ao, mo, vo, to, tro = oracle.hflow_run(A, np.zeros_like(A), np.zeros_like(A), op, fp, 5)
    assert flow.t == to == 5
    for d, o in ((Ad, Ao), (md, mo), (vd, vo)):
        assert np.linalg.norm(d.cpu().numpy() - o) / np.linalg.norm(o) < 1e-10
    np.testing.assert_allclose(tr, tro, rtol=1e-10, atol=1e-14)
    tr2 = flow.run(Ad, md, vd, 3)
    Ao, mo, vo, to, tro = oracle.hflow_run(Ao, mo, vo, op, fp, 3, t=5)
    assert flow.t == to == 8
    assert np.linalg.norm(Ad.cpu().numpy() - Ao) / np.linalg.norm(Ao) < 1e-10
    np.testing.assert_allclose(tr2, tro, rtol=1e-10, atol=1e-14)


def test_run_graph_replays_smooth_xi():
    """70 steps = two 32-step graph replays plus 6 direct steps (smooth xi, so
    the long trajectory is comparable)."""
    shape = (8, 12, 16)
    flow, Ad, A, op, fp = setup(shape, xi=1e-2, lr=2e-3)
    md, vd = torch.zeros_like(Ad), torch.zeros_like(Ad)
    tr = flow.run(Ad, md, vd, 70)
    Ao, mo, vo, to, tro = oracle.hflow_run(A, np.zeros_like(A), np.zeros_like(A), op, fp, 70)
    assert np.linalg.norm(Ad.cpu().numpy() - Ao) / np.linalg.norm(Ao) < 1e-8
    np.testing.assert_allclose(tr[:, 0], tro[:, 0], rtol=1e-8)
    np.testing.assert_allclose(tr[:, 3], 0.3, atol=1e-14)
    assert tr[-1, 0] < tr[0, 0]


def test_fp32_matches_fp64():
    shape = (20, 24, 32)
    f64, A64, A, op, fp = setup(shape, seed=3)
    f32, A32, _, _, _ = setup(shape, prec="fp32", seed=3)
    A64 = A32.double()
    G64, g64 = f64.grad(A64)
    G32, g32 = f32.grad(A32)
    assert abs(G32 - G64) / abs(G64) < 1e-4
    assert (torch.linalg.norm(g32.double() - g64) / torch.linalg.norm(g64)).item() < 1e-3
    assert torch.max(torch.abs(f32.field(A32).double() - f64.field(A64))).item() < 1e-6


def test_errors():
    shape = (8, 8, 8)
    flow, Ad, A, op, fp = setup(shape)
    with pytest.raises(ValueError):
        flow.field(Ad[:2].contiguous())
    with pytest.raises(pfc.PfcError):
        pfc.HFlow(pfc.Problem(nx=8, ny=8, nz=8, eps=1.5, a=(1, 0, 1, 0, 0, 0), prec="fp64"), m0=0.3,
                  blur_sigma=20.0)                                  # radius 60 > 32


def test_paper_setting_100():
    """Alg. 1 in the paper's own setting (Sec. 4.1, Fig. cvg_1 parameters at
    100^3, h = 0.01, eps = 0.02, the +-1 well, blur 2 voxels): FP32 against
    the FP64 oracle for 2 steps, then 300 steps stay finite, keep the mass
    and lower the energy."""
    pd, fd, A0 = I.paper_flow_100()
    nz, ny, nx = pd["shape"]
    prob = pfc.Problem(nx=nx, ny=ny, nz=nz, h=pd["h"], eps=pd["eps"], xi=pd["xi"], a=pd["a"], well=pd["well"],
                       prec="fp32")
    flow = pfc.HFlow(prob, m0=fd["m0"], lr=fd["lr"], blur_sigma=fd["blur_sigma"])
    A32 = A0.astype(np.float32)
    A = torch.tensor(A32, device="cuda")
    m, v = torch.zeros_like(A), torch.zeros_like(A)
    tr = flow.run(A, m, v, 2)
    op = {"a": pd["a"], "eps": pd["eps"], "xi": pd["xi"], "h": pd["h"], "well": pd["well"]}
    _, _, _, _, tro = oracle.hflow_run(A32.astype(np.float64), np.zeros_like(A0), np.zeros_like(A0), op, fd, 2)
    np.testing.assert_allclose(tr[:, 0], tro[:, 0], rtol=1e-4)
    np.testing.assert_allclose(tr[:, 1:3], tro[:, 1:3], rtol=1e-3)
    tr = flow.run(A, m, v, 300)
    assert np.all(np.isfinite(tr))
    assert np.max(np.abs(tr[:, 3] - fd["m0"])) < 1e-6
    assert tr[-1, 0] < tr[0, 0]


def test_paper_setting_generates_a_viable_shape():
    """The generator from white noise in the paper's setting (Sec. 4.1, Fig.
    cvg_1 parameters): within 2000 Adam iterations the field separates into
    the two phases and passes the paper's viability test (Sec. 4.5:
    normalised discrepancy below 0.75, max u > 0.1, min u < -0.1), the energy
    has dropped, the mass is kept and {u = 0} has a surface."""
    pd, fd, A0 = I.paper_flow_100()
    nz, ny, nx = pd["shape"]
    prob = pfc.Problem(nx=nx, ny=ny, nz=nz, h=pd["h"], eps=pd["eps"], xi=pd["xi"], a=pd["a"], well=pd["well"],
                       prec="fp32")
    flow = pfc.HFlow(prob, m0=fd["m0"], lr=fd["lr"], blur_sigma=fd["blur_sigma"])
    A = torch.tensor(A0.astype(np.float32), device="cuda")
    m, v = torch.zeros_like(A), torch.zeros_like(A)
    tr = flow.run(A, m, v, 2000)
    assert np.all(np.isfinite(tr))
    np.testing.assert_allclose(tr[:, 3], fd["m0"], atol=1e-6)
    assert tr[-1, 0] < 0.2 * tr[0, 0]
    ctx = pfc.Context(prob)
    ut = flow.field(A)
    d = ctx.diagnostics(ut)
    assert d["ratio"] < 0.75 and d["max"] > 0.1 and d["min"] < -0.1
    cells = ctx.surface_cells(ut)
    assert cells.shape[0] > 1000 and float(cells[:, 0].double().sum()) > 1.0


@pytest.mark.parametrize("shape,sigma", [((30, 26, 12), 2.0),    # x: 10 rows of 3 float4 per warp
                                         ((14, 40, 128), 1.0),   # x: one row of 32 float4 per warp
                                         ((17, 9, 100), 2.0),    # the paper's row length; y shorter than a window
                                         ((10, 28, 132), 2.0),   # x: rows above 128 values take the tiles
                                         ((13, 27, 18), 2.0),    # nx % 4 != 0: scalar windows
                                         ((9, 11, 20), 0.8)])    # radius 3 below a window on every axis
def test_fp32_blur_paths_vs_oracle(shape, sigma):
    """The FP32 blur passes (Alg. 1's Gaussian k) take float4 kernels when
    rows hold a multiple of 4 values: shuffles across a warp along x, register
    windows along y and z; the shapes above reach each variant, the tails of
    the windows and the wrap of every axis.  Field and gradient against the
    oracle in FP64.  The field is linear in A and checks the blur kernels
    alone; the gradient's bar grows with how far rounding the field to FP32
    moves the oracle's own dF/du (strongly blurred fields vary by a few 1e-3
    around m0, where the FP32 energy gradient is ill-conditioned)."""
    flow, Ad, A, op, fp = setup(shape, prec="fp32", sigma=sigma)
    ut = flow.field(Ad).double().cpu().numpy()
    uo = oracle.hflow_field(A, op, fp)
    assert np.max(np.abs(ut - uo)) < 1e-6
    G, gA = flow.grad(Ad)
    Go, gAo = oracle.hflow_grad(A, op, fp)
    assert G == pytest.approx(Go, rel=1e-4)
    _, gu = oracle.energy_and_grad(uo, op)
    _, gu32 = oracle.energy_and_grad(uo.astype(np.float32).astype(np.float64), op)
    sens = np.linalg.norm(gu32 - gu) / np.linalg.norm(gu)
    gA = gA.double().cpu().numpy()
    assert np.linalg.norm(gA - gAo) / np.linalg.norm(gAo) < max(1e-3, 10 * sens)


@pytest.mark.parametrize("shape", [(9, 10, 11), (8, 12, 20)])
def test_fp32_row_paths_and_misaligned_buffers(shape):
    """FP32 flow kernels take a float4 path when rows hold a multiple of 4
    voxels and the buffers are 16-byte aligned, else a scalar path: both
    against FP64, and a misaligned A (offset by one element) against an
    aligned copy of the same values."""
    f64, _, A, op, fp = setup(shape, seed=5)
    f32, A32, _, _, _ = setup(shape, prec="fp32", seed=5)
    G64, g64 = f64.grad(A32.double())
    G32, g32 = f32.grad(A32)
    assert abs(G32 - G64) / abs(G64) < 1e-4
    assert (torch.linalg.norm(g32.double() - g64) / torch.linalg.norm(g64)).item() < 1e-3
    store = torch.empty(A32.numel() + 1, dtype=torch.float32, device="cuda")
    Am = store[1:].view(A32.shape)
    Am.copy_(A32)
    assert Am.data_ptr() % 16 != 0
    Gm, gm = f32.grad(Am)
    assert Gm == pytest.approx(G32, rel=1e-5)
    assert (torch.linalg.norm(gm - g32) / torch.linalg.norm(g32)).item() < 1e-5
    md, vd = torch.zeros_like(Am), torch.zeros_like(Am)
    ma, va = torch.zeros_like(A32), torch.zeros_like(A32)
    Aa = A32.clone()
    f32.run(Am, md, vd, 3)
    f32.t = 0
    f32.run(Aa, ma, va, 3)
    assert (torch.linalg.norm(Am - Aa) / torch.linalg.norm(Aa)).item() < 1e-5


def _batch_problems(shape, wells=(0, 1, 0)):
    nz, ny, nx = shape
    rng = np.random.default_rng(17)
    probs, m0s = [], []
    for k, well in enumerate(wells):
        a = tuple(rng.uniform(-0.5, 0.5, 6) + np.array([1.0, 0, 1.0, 0, 0, 0]))
        probs.append(pfc.Problem(nx=nx, ny=ny, nz=nz, eps=1.5 + 0.1 * k, h=1.0 - 0.05 * k, a=a, well=well,
                                 prec="fp32"))
        m0s.append(0.3 if well == 0 else -0.4)
    return probs, m0s


@pytest.mark.parametrize("shape,sigma", [((12, 10, 16), 1.5), ((9, 13, 11), 2.0), ((28, 13, 20), 2.0)])
def test_flow_batch_matches_single_flows(shape, sigma):
    """A batch of flows (different coefficients, eps, h, wells and masses,
    one launch per kernel for all) gives each instance's single-flow result:
    40 steps = one 32-step graph replay plus 8 direct steps, twice."""
    probs, m0s = _batch_problems(shape)
    rng = np.random.default_rng(18)
    A0 = [torch.tensor((0.04 * rng.standard_normal((3,) + shape)).astype(np.float32), device="cuda")
          for _ in probs]
    fb = pfc.HFlowBatch(probs, m0s, lr=1e-3, blur_sigma=sigma)
    As = [a.clone() for a in A0]
    ms = [torch.zeros_like(a) for a in A0]
    vs = [torch.zeros_like(a) for a in A0]
    trb = fb.run(As, ms, vs, 40)
    trb2 = fb.run(As, ms, vs, 40)
    assert fb.t == 80
    for k, (p, m0) in enumerate(zip(probs, m0s)):
        fl = pfc.HFlow(p, m0=m0, lr=1e-3, blur_sigma=sigma)
        A, m, v = A0[k].clone(), torch.zeros_like(A0[k]), torch.zeros_like(A0[k])
        tr = fl.run(A, m, v, 40)
        tr2 = fl.run(A, m, v, 40)
        assert (torch.linalg.norm(As[k] - A) / torch.linalg.norm(A)).item() < 1e-6
        assert (torch.linalg.norm(vs[k] - v) / torch.linalg.norm(v)).item() < 1e-5
        for a, b in ((trb[k], tr), (trb2[k], tr2)):
            np.testing.assert_allclose(a[:, 0], b[:, 0], rtol=1e-5)
            np.testing.assert_allclose(a[:, 3], m0, atol=1e-6)
            np.testing.assert_allclose(a[:, 4], b[:, 4])
    ut = fb.field(As)
    for k, p in enumerate(probs):
        fl = pfc.HFlow(p, m0=m0s[k], lr=1e-3, blur_sigma=sigma)
        assert torch.allclose(ut[k], fl.field(As[k]), rtol=0, atol=1e-6)


def test_flow_batch_against_oracle_and_errors():
    shape = (8, 12, 16)
    probs, m0s = _batch_problems(shape, wells=(1, 0))
    rng = np.random.default_rng(19)
    A0 = [(0.04 * rng.standard_normal((3,) + shape)).astype(np.float32).astype(np.float64) for _ in probs]
    fb = pfc.HFlowBatch(probs, m0s, lr=1e-3, blur_sigma=1.0)
    As = [torch.tensor(a, dtype=torch.float32, device="cuda") for a in A0]
    ms = [torch.zeros_like(a) for a in As]
    vs = [torch.zeros_like(a) for a in As]
    tr = fb.run(As, ms, vs, 2)
    for k, p in enumerate(probs):
        op = {"a": p.a, "eps": p.eps, "h": p.h, "xi": p.xi, "well": p.well}
        fp = {"m0": m0s[k], "blur_sigma": 1.0, "lr": 1e-3}
        Ao, _, _, _, tro = oracle.hflow_run(A0[k], np.zeros_like(A0[k]), np.zeros_like(A0[k]), op, fp, 2)
        np.testing.assert_allclose(tr[k][:, 0], tro[:, 0], rtol=1e-4)
        d = As[k].double().cpu().numpy() - A0[k]
        do = Ao - A0[k]
        assert np.linalg.norm(d - do) / np.linalg.norm(do) < 1e-3
    # every instance must share the grid; the extensions are not batched
    nz, ny, nx = shape
    bad = probs + [pfc.Problem(nx=nx + 4, ny=ny, nz=nz, eps=1.5, a=(1, 0, 1, 0, 0, 0), prec="fp32")]
    with pytest.raises(pfc.PfcError):
        pfc.HFlowBatch(bad, m0s + [0.3])
    with pytest.raises(pfc.PfcError):
        pfc.HFlowBatch([pfc.Problem(nx=nx, ny=ny, nz=nz, eps=1.5, a=(1, 0, 1, 0, 0, 0), prec="fp32", mu=1.0,
                                    theta=(1, 0, 0))], [0.3])
    with pytest.raises(pfc.PfcError):
        pfc.HFlowBatch([pfc.Problem(nx=nx, ny=ny, nz=nz, eps=1.5, a=(1, 0, 1, 0, 0, 0), prec="fp64")], [0.3])


def test_flow_batch_64_instances_misaligned_and_limits():
    """The largest batch (64 flows, every descriptor slot in use) against single
    flows at both ends and in the middle (the batch runs another instantiation
    of the sweep, and Adam's m / sqrt(v) turns last-bit differences of
    near-zero gradients into visible ones: 1e-5); an A that is not 16-byte aligned
    sends the whole batch to the scalar div / Adam kernels, which must agree
    with the float4 ones; 65 flows and an empty batch are rejected."""
    shape = (9, 12, 16)
    nz, ny, nx = shape
    rng = np.random.default_rng(23)
    probs, m0s = [], []
    for k in range(64):
        a = tuple(rng.uniform(-0.3, 0.3, 6) + np.array([1.0, 0, 1.0, 0, 0, 0]))
        probs.append(pfc.Problem(nx=nx, ny=ny, nz=nz, eps=1.5, a=a, well=k % 2, prec="fp32"))
        m0s.append(0.3 if k % 2 == 0 else -0.4)
    A0 = [torch.tensor((0.04 * rng.standard_normal((3,) + shape)).astype(np.float32), device="cuda") for _ in probs]
    fb = pfc.HFlowBatch(probs, m0s, lr=1e-3, blur_sigma=2.0)
    As = [a.clone() for a in A0]
    ms = [torch.zeros_like(a) for a in A0]
    vs = [torch.zeros_like(a) for a in A0]
    tr = fb.run(As, ms, vs, 6)
    assert tr.shape == (64, 6, 5) and np.all(np.isfinite(tr))
    for k in (0, 31, 63):
        fl = pfc.HFlow(probs[k], m0=m0s[k], lr=1e-3, blur_sigma=2.0)
        A, m, v = A0[k].clone(), torch.zeros_like(A0[k]), torch.zeros_like(A0[k])
        trs = fl.run(A, m, v, 6)
        assert (torch.linalg.norm(As[k] - A) / torch.linalg.norm(A)).item() < 1e-5
        np.testing.assert_allclose(tr[k][:, 0], trs[:, 0], rtol=1e-5)
        np.testing.assert_allclose(tr[k][:, 3], m0s[k], atol=1e-6)
    # instance 5's A (and moments) one element off a 16-byte boundary
    stores = [torch.empty(A0[5].numel() + 1, dtype=torch.float32, device="cuda") for _ in range(3)]
    Am, mm, vm = (s[1:].view(A0[5].shape) for s in stores)
    Am.copy_(A0[5]); mm.zero_(); vm.zero_()
    assert Am.data_ptr() % 16 != 0
    fb2 = pfc.HFlowBatch(probs, m0s, lr=1e-3, blur_sigma=2.0)
    Bs = [a.clone() for a in A0]
    Bs[5] = Am
    mb = [torch.zeros_like(a) for a in A0]
    vb = [torch.zeros_like(a) for a in A0]
    mb[5], vb[5] = mm, vm
    tr2 = fb2.run(Bs, mb, vb, 6)
    for k in (0, 5, 63):
        assert (torch.linalg.norm(Bs[k] - As[k]) / torch.linalg.norm(As[k])).item() < 1e-5
        np.testing.assert_allclose(tr2[k][:, 0], tr[k][:, 0], rtol=1e-5)
    with pytest.raises(pfc.PfcError):
        pfc.HFlowBatch(probs + probs[:1], m0s + m0s[:1])
    with pytest.raises(pfc.PfcError):
        pfc.HFlowBatch([], [])


def test_flow_batch_field_bit_identical_to_single_at_paper_size():
    """At the paper's 100^3 (blur radius 6) a batch of 16 splits the y and z
    blur lines into long pieces (the unrolled register ring) and a single flow
    into short ones (the ring's tail loop); div + x pass, windows and taps are
    the same arithmetic in the same order, so the fields agree bit for bit."""
    from paper_2103_04856_gb300 import inputs as I
    pd, fd, _ = I.paper_flow_100()
    nz, ny, nx = pd["shape"]
    prob = pfc.Problem(nx=nx, ny=ny, nz=nz, h=pd["h"], eps=pd["eps"], xi=pd["xi"], a=pd["a"], well=pd["well"],
                       prec="fp32")
    n = 16
    fb = pfc.HFlowBatch([prob] * n, [fd["m0"]] * n, lr=fd["lr"], blur_sigma=fd["blur_sigma"])
    As = [torch.tensor(I.paper_flow_100(seed=s)[2].astype(np.float32), device="cuda") for s in range(n)]
    ub = fb.field(As)
    fl = pfc.HFlow(prob, m0=fd["m0"], lr=fd["lr"], blur_sigma=fd["blur_sigma"])
    for k in (0, 7, 15):
        assert torch.equal(ub[k], fl.field(As[k]))
