"""Multi-rank host logic of bench.py on CPU: two gloo ranks (127.0.0.1).

Independent problems shard across GPUs with no collective on the data path;
the only cross-rank step is the max of the per-rank step times, and the job's
value counts every rank's voxels (weak scaling)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import sys
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = [1.0 + rank, 10.0 - rank]           # rank 1 is slower on the first entry
        got = bench.max_over_ranks(mine)
        q.put((rank, got, bench.job_value(1000, world, got[0])))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_weak_value():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, value in res:
        assert got == [2.0, 10.0]
        assert value == pytest.approx(2 * 1000 / 2e-3)


def test_single_process_identity():
    import bench
    assert bench.max_over_ranks([3.0, 4.0]) == [3.0, 4.0]
    assert bench.job_value(10, 1, 1.0) == pytest.approx(1e4)


# ---------------------------------------------------------------- z-slabs
# The decomposition of one large grid across GPUs: rank r owns the z planes
# [z0, z1) and, before each sweep, receives the two planes below z0 and the
# two above z1 from its periodic neighbours (the stencil of eq. Feps reaches
# one plane, the transposed stencil of its gradient one more).  Emulated on
# CPU ranks with the oracle: everything outside a rank's slab and halo is
# NaN, so any dependency beyond two planes would show.

SLAB_SHAPE = (16, 10, 12)
SLAB_P = {"a": (0.8, 0.3, 1.1, 0.4, -0.2, 0.1), "eps": 1.5, "h": 1.0, "xi": 1e-6, "well": 0}


def _slab_bounds(nz, world):
    return [nz * r // world for r in range(world + 1)]


def _slab_worker(rank, world, port, q):
    import sys
    import numpy as np
    import torch
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import oracle
    from paper_2103_04856_gb300 import inputs as I
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        nz, ny, nx = SLAB_SHAPE
        b = _slab_bounds(nz, world)
        z0, z1 = b[rank], b[rank + 1]
        own = I.noise(SLAB_SHAPE, 0.3, 0.1, 7)[z0:z1].copy()      # this rank's planes only
        up, dn = (rank + 1) % world, (rank - 1) % world
        top, bot = torch.from_numpy(own[-2:].copy()), torch.from_numpy(own[:2].copy())
        below, above = torch.empty(2, ny, nx, dtype=torch.float64), torch.empty(2, ny, nx, dtype=torch.float64)
        reqs = [dist.isend(top, up, tag=0), dist.isend(bot, dn, tag=1),
                dist.irecv(below, dn, tag=0), dist.irecv(above, up, tag=1)]
        for r in reqs:
            r.wait()
        win = np.full(SLAB_SHAPE, np.nan)
        win[z0:z1] = own
        win[[(z0 - 2) % nz, (z0 - 1) % nz]] = below.numpy()
        win[[z1 % nz, (z1 + 1) % nz]] = above.numpy()
        dens = oracle.density(win, SLAB_P)[z0:z1]
        idx = np.arange(z0 * ny * nx, z1 * ny * nx)
        g = oracle.grad_sampled(win, SLAB_P, idx).reshape(z1 - z0, ny, nx)
        # the step's two global reductions: energy (fixed rank order) and sum g
        parts = [torch.zeros(2, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(parts, torch.tensor([float(dens.sum()), float(g.sum())], dtype=torch.float64))
        E = sum(float(pt[0]) for pt in parts)
        lam = sum(float(pt[1]) for pt in parts) / (nx * ny * nz)
        q.put((rank, z0, z1, dens, g, E, lam))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_zslab_halo_exchange_matches_single_domain(world):
    import numpy as np
    import oracle
    from paper_2103_04856_gb300 import inputs as I
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_slab_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=180) for _ in procs], key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    u = I.noise(SLAB_SHAPE, 0.3, 0.1, 7)
    dens_ref = oracle.density(u, SLAB_P)
    E_ref, g_ref = oracle.energy_and_grad(u, SLAB_P)
    E_slabs = sum(float(dens_ref[z0:z1].sum()) for _, z0, z1, *_ in res)
    for rank, z0, z1, dens, g, E, lam in res:
        assert np.all(np.isfinite(dens)) and np.all(np.isfinite(g))
        np.testing.assert_array_equal(dens, dens_ref[z0:z1])
        np.testing.assert_allclose(g, g_ref[z0:z1], rtol=0, atol=1e-14)
        assert E == E_slabs                                   # same partials, same order
        assert E == pytest.approx(E_ref, rel=1e-13)
        assert lam == pytest.approx(g_ref.sum() / u.size, rel=1e-10, abs=1e-15)


def test_zslab_one_halo_plane_is_not_enough():
    """The converse: with one halo plane per side the gradient of the planes
    next to the slab's faces reads beyond the halo (NaN), so two are needed."""
    import numpy as np
    import oracle
    from paper_2103_04856_gb300 import inputs as I
    nz, ny, nx = SLAB_SHAPE
    u = I.noise(SLAB_SHAPE, 0.3, 0.1, 7)
    z0, z1 = 4, 10
    win = np.full(SLAB_SHAPE, np.nan)
    win[z0 - 1:z1 + 1] = u[z0 - 1:z1 + 1]
    assert np.all(np.isfinite(oracle.density(win, SLAB_P)[z0:z1]))     # the energy needs one plane
    g = oracle.grad_sampled(win, SLAB_P, np.arange(z0 * ny * nx, z1 * ny * nx)).reshape(z1 - z0, ny, nx)
    assert np.all(np.isnan(g[0])) and np.all(np.isnan(g[-1]))
    assert np.all(np.isfinite(g[1:-1]))
