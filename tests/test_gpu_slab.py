"""One periodic grid split in z-slabs (pfc_slab_*), run in one process on one
GPU: the slabs' halos are filled from each other (paper_2103_04856_gb300.slab
.local_halos), each slab is swept by the library, and every slab combines
the rows of sums in rank order.

Bars: the gradient and the first stored step agree with the single-domain
sweep to a few units of rounding (1e-12 of max|g| in FP64, 1e-6 in FP32):
every voxel is evaluated by the same formulas, but the compiler contracts
multiply-adds differently in the z-march's phase instantiations (first
planes of a run, steady state, last plane), so a voxel's last bits depend on
where the CTA runs of its launch begin, and slabs split the planes
differently (with one slab the runs are the single domain's, and the fields
are equal bit for bit).  Energies within 1e-13 (FP64) / 1e-6 (FP32) of the
single-domain ones; FP64 against the oracle at 1e-10 (energy, gradient
2-norm) and 1e-12 (fields after chained steps)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2103_04856_gb300 import inputs as I

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2103_04856_gb300 import pfc
    from paper_2103_04856_gb300 import slab as S

A_GEN = (0.8, 0.3, 1.1, 0.4, -0.2, 0.1)


def _slabs(prob, u, R):
    parts = S.split_z(prob.nz, R)
    slabs = [pfc.Slab(prob, z0, n) for z0, n in parts]
    fields = [u[z0:z0 + n].clone() for z0, n in parts]
    return parts, slabs, fields


def _sweep_all(slabs, fields, outs, mode, tau):
    halos = [s.new_halo() for s in slabs]
    S.local_halos(fields, halos)
    rows = torch.zeros((len(slabs), S.SLAB_NSUMS), dtype=torch.float64, device="cuda")
    for k, s in enumerate(slabs):
        s.sweep(fields[k], halos[k], outs[k], mode, tau, rows[k])
    scal = []
    for s in slabs:
        sc = torch.zeros(5, dtype=torch.float64, device="cuda")
        s.finish(rows, sc)
        scal.append(sc)
    torch.cuda.synchronize()
    return [sc.cpu().numpy() for sc in scal]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("R", [1, 2, 3, 4])
def test_slab_gradient_equals_single_domain(prec, R):
    shape = (20, 24, 40) if prec == "fp64" else (64, 48, 64)
    a = A_GEN if prec == "fp64" else I.tube_descent_256().a
    dt = torch.float64 if prec == "fp64" else torch.float32
    u = torch.tensor(I.noise(shape, 0.3, 0.1, 21), dtype=dt, device="cuda")
    prob = pfc.Problem.from_shape(shape, eps=1.5, a=a, prec=prec)
    E1, g1 = pfc.Context(prob).energy_and_grad(u)
    parts, slabs, fields = _slabs(prob, u, R)
    outs = [s.new_field() for s in slabs]
    scal = _sweep_all(slabs, fields, outs, S.SLAB_GRAD, 0.0)
    g = torch.cat(outs)
    gscale = g1.abs().max().item()
    rnd = 1e-12 if prec == "fp64" else 1e-6
    if R == 1:
        assert torch.equal(g, g1)                   # the single domain's runs
    assert (g - g1).abs().max().item() <= rnd * gscale
    for sc in scal:
        assert np.array_equal(sc, scal[0])          # every slab holds the same scalars
    assert scal[0][0] == pytest.approx(E1, rel=1e-13 if prec == "fp64" else 1e-6)
    assert abs(scal[0][2] - float(g1.double().mean())) <= rnd * float(g1.double().abs().mean())
    if prec == "fp64":
        Eo, go = oracle.energy_and_grad(u.cpu().numpy(), {"a": a, "eps": 1.5, "h": 1.0, "xi": 1e-6, "well": 0})
        assert scal[0][0] == pytest.approx(Eo, rel=1e-10)
        gn = g.cpu().numpy()
        assert np.linalg.norm(gn - go) / np.linalg.norm(go) < 1e-10
    for s in slabs:
        s.close()


def test_slab_first_step_equals_single_domain_fp32():
    """The first stored step (the pending offset is 0) of 3 slabs agrees with
    the batch path's chained first step, the same sweep over the whole grid
    in one domain, to FP32 rounding (one ulp of the field); so do the fields
    once the offsets c = m - mean(v) are added (their FP32 per-thread sums
    are partitioned differently)."""
    shape = (48, 40, 64)
    u = torch.tensor(I.noise(shape, 0.3, 0.1, 22).astype(np.float32), device="cuda")
    prob = pfc.Problem.from_shape(shape, eps=1.5, a=A_GEN, prec="fp32")
    b = pfc.Batch([prob])
    out1 = torch.empty_like(u)
    b.step_lazy([u], [out1], [2e-3], first=True)
    parts, slabs, fields = _slabs(prob, u, 3)
    outs = [s.new_field() for s in slabs]
    _sweep_all(slabs, fields, outs, S.SLAB_STEP, 2e-3)
    ulp = 2.0 ** -23 * out1.abs().max().item()
    assert (torch.cat(outs) - out1).abs().max().item() <= ulp
    b.lazy_finish([out1])
    for s, o in zip(slabs, outs):
        s.apply_offset(o)
    torch.cuda.synchronize()
    assert (torch.cat(outs) - out1).abs().max().item() <= 1e-6


@pytest.mark.parametrize("R", [1, 2, 4])
def test_slab_chained_steps_vs_oracle_fp64(R):
    """Five chained slab steps (the projection in fused form, the offset
    combined from every slab's sums) against five exact oracle steps: fields
    to 1e-12, trace rows (E, mass, lambda, max|g|, mean|g|) to 1e-10."""
    shape = (16, 20, 24)
    u0 = I.noise(shape, 0.3, 0.1, 23)
    pr = {"a": A_GEN, "eps": 1.5, "h": 1.0, "xi": 1e-2, "well": 0}
    prob = pfc.Problem.from_shape(shape, eps=1.5, a=A_GEN, xi=1e-2, prec="fp64")
    uo, tro = oracle.run(u0, pr, 5, 5e-3)
    parts, slabs, fields = _slabs(prob, torch.tensor(u0, device="cuda"), R)
    nxt = [s.new_field() for s in slabs]
    tr = []
    for k in range(5):
        tr.append(_sweep_all(slabs, fields, nxt, S.SLAB_STEP, 5e-3)[0])
        fields, nxt = nxt, fields
    for s, f in zip(slabs, fields):
        s.apply_offset(f)
    torch.cuda.synchronize()
    got = torch.cat(fields).cpu().numpy()
    assert np.max(np.abs(got - uo)) < 1e-12
    np.testing.assert_allclose(np.array(tr), tro, rtol=1e-10, atol=1e-14)
    assert abs(got.mean() - u0.mean()) < 1e-14


def test_slab_descent_driver_single_rank_matches_oracle():
    """The descent driver of paper_2103_04856_gb300.slab without a process
    group (one slab: the halo wraps locally), FP64, against the oracle."""
    shape = (12, 16, 20)
    u0 = I.noise(shape, 0.3, 0.1, 24)
    pr = {"a": A_GEN, "eps": 1.5, "h": 1.0, "xi": 1e-2, "well": 0}
    prob = pfc.Problem.from_shape(shape, eps=1.5, a=A_GEN, xi=1e-2, prec="fp64")
    drv = S.SlabDescent(prob, torch.tensor(u0, device="cuda"), 0)
    tr = drv.run(4, 5e-3)
    uo, tro = oracle.run(u0, pr, 4, 5e-3)
    assert np.max(np.abs(drv.field().cpu().numpy() - uo)) < 1e-12
    np.testing.assert_allclose(tr, tro, rtol=1e-10, atol=1e-14)
    g = torch.empty_like(drv.field())
    E = drv.energy_and_grad(g)
    Eo, go = oracle.energy_and_grad(uo, pr)
    assert E == pytest.approx(Eo, rel=1e-10)
    assert np.linalg.norm(g.cpu().numpy() - go) / np.linalg.norm(go) < 1e-10


def test_slab_rejects_bad_arguments():
    prob = pfc.Problem.from_shape((8, 8, 8), eps=1.5, a=A_GEN, prec="fp32")
    for z0, n in ((0, 1), (-1, 4), (6, 4)):
        with pytest.raises(pfc.PfcError):
            pfc.Slab(prob, z0, n)
    s = pfc.Slab(prob, 0, 4)
    u = s.new_field()
    h = s.new_halo()
    row = torch.zeros(S.SLAB_NSUMS, dtype=torch.float64, device="cuda")
    with pytest.raises(pfc.PfcError):      # nothing swept yet
        s.finish(row.view(1, -1))
    with pytest.raises(pfc.PfcError):      # out aliases u
        s.sweep(u, h, u, S.SLAB_GRAD, 0.0, row)
    host = torch.zeros(S.SLAB_NSUMS, dtype=torch.float64)
    lib = pfc.load_library()
    import ctypes
    rc = lib.pfc_slab_sweep(s._h, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(h.data_ptr()),
                            ctypes.c_void_p(s.new_field().data_ptr()), 1, 0.0, ctypes.c_void_p(host.data_ptr()),
                            None)
    assert rc == pfc.PFC_EINVAL
    s.close()
