"""Independent contexts driven from separate host threads on separate
streams at the same time: their step loops (captured and replayed as CUDA
graphs, trace buffers grown on demand) must neither fail nor change results.
This is how several shapes are generated concurrently."""
import threading

import numpy as np
import pytest
import torch

from paper_2103_04856_gb300 import inputs as I

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2103_04856_gb300 import pfc


def _in_threads(fns):
    errors = []

    def wrap(fn):
        try:
            fn()
        except Exception as e:          # reported after the join
            errors.append(e)
    ths = [threading.Thread(target=wrap, args=(fn,)) for fn in fns]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    torch.cuda.synchronize()
    assert not errors, errors


def test_concurrent_flows_match_sequential():
    shape = (16, 20, 24)
    prob = pfc.Problem.from_shape(shape, eps=1.5, a=(1.0, 0.4, 0.8, 0.3, -0.2, 0.1), prec="fp32")
    rng = np.random.default_rng(3)
    A0s = [torch.tensor((0.04 * rng.standard_normal((3,) + shape)).astype(np.float32), device="cuda")
           for _ in range(4)]

    def flows():
        return [pfc.HFlow(prob, m0=0.3, lr=1e-3, blur_sigma=1.5) for _ in A0s]

    # sequential reference
    ref = []
    for fl, A0 in zip(flows(), A0s):
        A, m, v = A0.clone(), torch.zeros_like(A0), torch.zeros_like(A0)
        fl.run(A, m, v, 40)
        fl.run(A, m, v, 300)            # grows the trace buffer
        ref.append(A)
    # the same four runs at once, each on its own stream and thread
    fls = flows()
    streams = [torch.cuda.Stream() for _ in fls]
    states = [(A0.clone(), torch.zeros_like(A0), torch.zeros_like(A0)) for A0 in A0s]

    def job(k):
        def f():
            A, m, v = states[k]
            fls[k].run(A, m, v, 40, stream=streams[k])
            fls[k].run(A, m, v, 300, stream=streams[k])
        return f
    _in_threads([job(k) for k in range(len(fls))])
    for (A, _, _), R in zip(states, ref):
        assert torch.equal(A, R)


def test_concurrent_descent_runs_match_sequential():
    shape = (24, 28, 32)
    prob = pfc.Problem.from_shape(shape, eps=1.5, a=(1, 0, 1, 0, 0, 0), prec="fp32")
    u0s = [torch.tensor(I.noise(shape, 0.3, 0.1, 40 + k).astype(np.float32), device="cuda") for k in range(3)]
    ref = []
    for u0 in u0s:
        u = u0.clone()
        ctx = pfc.Context(prob)
        ctx.run(u, 70, 1e-3)
        ctx.run(u, 200, 1e-3)
        ref.append(u)
    ctxs = [pfc.Context(prob) for _ in u0s]
    us = [u0.clone() for u0 in u0s]
    streams = [torch.cuda.Stream() for _ in u0s]

    def job(k):
        def f():
            ctxs[k].run(us[k], 70, 1e-3, stream=streams[k])
            ctxs[k].run(us[k], 200, 1e-3, stream=streams[k])
        return f
    _in_threads([job(k) for k in range(len(us))])
    for u, r in zip(us, ref):
        assert torch.equal(u, r)
