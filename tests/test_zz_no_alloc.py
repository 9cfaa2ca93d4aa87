"""pfc_energy_and_grad_noalloc against pfc_energy_and_grad, through the C ABI.

The no-allocation entry point serves callers that may not call cudaMalloc or
cudaFree (graph-capture regions, host callbacks, plugins whose host process
owns the device memory budget); its scratch is a static device array inside
the library.  Two calls in a row check that the shared scratch carries
nothing over from one call to the next.  This file sorts last so that a run
stopping at the first failure has already run every other test."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2103_04856_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,tol_e,tol_g", [("fp64", 1e-10, 1e-10), ("fp32", 1e-4, 1e-3)])
def test_noalloc_matches_context_path_twice(prec, tol_e, tol_g):
    from paper_2103_04856_gb300 import pfc
    lib = pfc.load_library()
    shape = (40, 24, 64)
    dt = torch.float64 if prec == "fp64" else torch.float32
    for call, (a, seed) in enumerate([((0.7, -0.2, 1.1, 0.3, -0.4, 0.2), 0), ((1.0, 0.0, 1.0, 0.0, 0.0, 0.0), 1)]):
        p = pfc.Problem.from_shape(shape, eps=1.5, a=a, prec=prec)
        u = torch.tensor(I.noise(shape, 0.3, 0.1, seed), dtype=dt, device="cuda")
        E_ref, g_ref = pfc.Context(p).energy_and_grad(u)
        g = torch.full_like(u, float("nan"))
        E = ctypes.c_double()
        rc = lib.pfc_energy_and_grad_noalloc(ctypes.byref(p._c()), ctypes.c_void_p(u.data_ptr()),
                                             ctypes.c_void_p(g.data_ptr()), ctypes.byref(E),
                                             ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == pfc.PFC_OK, (call, lib.pfc_last_error())
        assert abs(E.value - E_ref) <= tol_e * abs(E_ref), call
        err = torch.linalg.norm((g - g_ref).double()).item() / torch.linalg.norm(g_ref.double()).item()
        assert err <= tol_g, (call, err)


def test_noalloc_rejects_bad_input():
    from paper_2103_04856_gb300 import pfc
    lib = pfc.load_library()
    shape = (8, 8, 8)
    p = pfc.Problem.from_shape(shape, eps=1.5, a=(1, 0, 1, 0, 0, 0), prec="fp32", impl="plain")
    u = torch.zeros(shape, device="cuda")
    g = torch.zeros(shape, device="cuda")
    rc = lib.pfc_energy_and_grad_noalloc(ctypes.byref(p._c()), ctypes.c_void_p(u.data_ptr()),
                                         ctypes.c_void_p(g.data_ptr()), None, None)
    assert rc == pfc.PFC_EUNSUPPORTED
    p = pfc.Problem.from_shape(shape, eps=1.5, a=(1, 0, 1, 0, 0, 0), prec="fp32", tile_z=1)
    big = torch.zeros((128, 128, 128), device="cuda")      # 1 plane per CTA: 4096 CTAs
    gb = torch.empty_like(big)
    pb = pfc.Problem.from_shape(big.shape, eps=1.5, a=(1, 0, 1, 0, 0, 0), prec="fp32", tile_z=1)
    rc = lib.pfc_energy_and_grad_noalloc(ctypes.byref(pb._c()), ctypes.c_void_p(big.data_ptr()),
                                         ctypes.c_void_p(gb.data_ptr()), None, None)
    assert rc == pfc.PFC_EINVAL and b"1024" in lib.pfc_last_error()
    host = np.zeros(512, dtype=np.float32)
    rc = lib.pfc_energy_and_grad_noalloc(ctypes.byref(p._c()), ctypes.c_void_p(host.ctypes.data),
                                         ctypes.c_void_p(g.data_ptr()), None, None)
    assert rc == pfc.PFC_EINVAL
    # g aliasing u is refused before anything is launched
    p = pfc.Problem.from_shape(shape, eps=1.5, a=(1, 0, 1, 0, 0, 0), prec="fp32")
    rc = lib.pfc_energy_and_grad_noalloc(ctypes.byref(p._c()), ctypes.c_void_p(u.data_ptr()),
                                         ctypes.c_void_p(u.data_ptr()), None, None)
    assert rc == pfc.PFC_EINVAL and b"alias" in lib.pfc_last_error()
    # a non-finite field gives a non-finite energy, reported as such
    bad = torch.full(shape, float("nan"), device="cuda")
    E = ctypes.c_double()
    rc = lib.pfc_energy_and_grad_noalloc(ctypes.byref(p._c()), ctypes.c_void_p(bad.data_ptr()),
                                         ctypes.c_void_p(g.data_ptr()), ctypes.byref(E), None)
    assert rc == pfc.PFC_ENONFINITE
    # and the next call is correct again (the counters were left at zero)
    ok = torch.tensor(I.noise(shape, 0.3, 0.1, 3), dtype=torch.float32, device="cuda")
    E_ref, g_ref = pfc.Context(p).energy_and_grad(ok)
    rc = lib.pfc_energy_and_grad_noalloc(ctypes.byref(p._c()), ctypes.c_void_p(ok.data_ptr()),
                                         ctypes.c_void_p(g.data_ptr()), ctypes.byref(E), None)
    assert rc == pfc.PFC_OK and abs(E.value - E_ref) <= 1e-4 * abs(E_ref)
