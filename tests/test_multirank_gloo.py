"""Multi-rank host logic on CPU: gloo ranks (127.0.0.1).

Independent problems shard across GPUs with no collective on the data path:
the benchmark's only cross-rank step is the max of the per-rank step times,
and the job's value counts every rank's voxels (weak scaling); the mixed
batch is partitioned by work and its traces gathered on rank 0.  One large
grid splits into z-slabs whose halos and sums the library's driver
exchanges (paper_2103_04856_gb300.slab)."""
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
# The decomposition of one large grid across GPUs, driven by the library's
# own host code (paper_2103_04856_gb300.slab: split_z, HaloExchange,
# gather_rows, SlabDescent) over gloo ranks on the CPU.  The arithmetic of a
# slab, which on a GPU is the library's sweep, is done here by the oracle on
# a grid that is NaN outside the rank's slab and the halo it received, so a
# plane delivered to the wrong place, or a dependency beyond two planes,
# shows in the results.

SLAB_SHAPE = (16, 10, 12)
SLAB_P = {"a": (0.8, 0.3, 1.1, 0.4, -0.2, 0.1), "eps": 1.5, "h": 1.0, "xi": 1e-6, "well": 0}
# a smooth softplus for trajectories (at xi = 1e-6 the descent map has kinks)
SLAB_P_SMOOTH = dict(SLAB_P, xi=1e-2)
SLAB_TAU = 5e-3


class OracleSlabBackend:
    """One slab's sweep and the combine of every slab's sums, on the CPU, for
    driving the multi-rank host code without a GPU.  Mirrors the library's
    slab entry points: the pending offset c is added to every loaded plane
    of a step, the row of sums is (energy, sum of u + c, sum g, sum |g|,
    max |g|, sum of the stored field), the combine runs in rank order."""

    def __init__(self, z0, nzl, shape, p):
        self.z0, self.nzl, self.shape, self.p = z0, nzl, shape, p
        self.N = shape[0] * shape[1] * shape[2]
        self.c, self.target, self.count, self.mode = 0.0, None, 0, None

    def sweep(self, u, halo, out, mode, tau, row):
        import numpy as np
        import torch
        import oracle
        nz, ny, nx = self.shape
        z0, z1 = self.z0, self.z0 + self.nzl
        add = self.c if mode == 2 else 0.0
        win = np.full(self.shape, np.nan)
        win[z0:z1] = u.numpy() + add
        h = halo.numpy() + add
        win[(z0 - 2) % nz], win[(z0 - 1) % nz] = h[0], h[1]
        win[z1 % nz], win[(z1 + 1) % nz] = h[2], h[3]
        dens = oracle.density(win, self.p)[z0:z1]
        g = oracle.grad_sampled(win, self.p, np.arange(z0 * ny * nx, z1 * ny * nx)).reshape(self.nzl, ny, nx)
        x = win[z0:z1]
        v = x - tau * g if mode == 2 else None
        if mode == 1:
            out.copy_(torch.from_numpy(g))
        elif mode == 2:
            out.copy_(torch.from_numpy(v))
        vals = [dens.sum(), x.sum() if mode == 2 else 0.0, g.sum(), np.abs(g).sum(), np.abs(g).max(),
                v.sum() if mode == 2 else 0.0, 0.0, 0.0]
        row.copy_(torch.tensor(vals, dtype=torch.float64))
        self.mode = mode

    def finish(self, rows, scalars=None):
        s = [0.0] * 6
        for r in rows.tolist():
            for i in range(6):
                s[i] = max(s[i], r[i]) if i == 4 else s[i] + r[i]
        mass = None
        if self.mode == 2:
            mass = s[1] / self.N
            if self.count == 0:
                self.target = mass
            self.c = self.target - s[5] / self.N
            self.count += 1
        if scalars is not None:
            import torch
            scalars.copy_(torch.tensor([s[0], mass or 0.0, s[2] / self.N, s[4], s[3] / self.N],
                                       dtype=torch.float64))

    def apply_offset(self, u):
        u += self.c
        self.c, self.count = 0.0, 0


def _slab_worker(rank, world, port, q):
    import sys
    import numpy as np
    import torch
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    from paper_2103_04856_gb300 import inputs as I
    from paper_2103_04856_gb300 import slab as S
    from test_multirank_gloo import OracleSlabBackend
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        z0, nzl = S.split_z(SLAB_SHAPE[0], world)[rank]
        own = torch.from_numpy(I.noise(SLAB_SHAPE, 0.3, 0.1, 7)[z0:z0 + nzl].copy())   # this rank's planes only
        # one evaluation at xi = 1e-6: densities and gradient of the initial field
        be = OracleSlabBackend(z0, nzl, SLAB_SHAPE, SLAB_P)
        drv = S.SlabDescent(None, own.clone(), z0, backend=be)
        g0 = torch.empty_like(own)
        E0 = drv.energy_and_grad(g0)
        # three chained descent steps at xi = 1e-2, then the final energy and gradient
        be = OracleSlabBackend(z0, nzl, SLAB_SHAPE, SLAB_P_SMOOTH)
        drv = S.SlabDescent(None, own.clone(), z0, backend=be)
        tr = drv.run(3, SLAB_TAU)
        u3 = drv.field().numpy().copy()
        g3 = torch.empty_like(own)
        E3 = drv.energy_and_grad(g3)
        q.put((rank, z0, nzl, E0, g0.numpy(), tr, u3, E3, g3.numpy()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_zslab_descent_over_gloo_ranks_matches_single_domain(world):
    import numpy as np
    import oracle
    from paper_2103_04856_gb300 import inputs as I
    from paper_2103_04856_gb300 import slab as S
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
    E_ref, g_ref = oracle.energy_and_grad(u, SLAB_P)
    u3_ref, tr_ref = oracle.run(u, SLAB_P_SMOOTH, 3, SLAB_TAU)
    E3_ref, g3_ref = oracle.energy_and_grad(u3_ref, SLAB_P_SMOOTH)
    assert [r[1] for r in res] == [z0 for z0, _ in S.split_z(SLAB_SHAPE[0], world)]
    for rank, z0, nzl, E0, g0, tr, u3, E3, g3 in res:
        z1 = z0 + nzl
        assert np.all(np.isfinite(g0)) and np.all(np.isfinite(u3))
        np.testing.assert_allclose(g0, g_ref[z0:z1], rtol=0, atol=1e-14)
        assert E0 == res[0][3]                                 # every rank combined the same rows
        assert E0 == pytest.approx(E_ref, rel=1e-13)
        np.testing.assert_allclose(tr, tr_ref, rtol=1e-11, atol=1e-15)
        np.testing.assert_allclose(u3, u3_ref[z0:z1], rtol=0, atol=1e-13)
        assert E3 == pytest.approx(E3_ref, rel=1e-12)
        np.testing.assert_allclose(g3, g3_ref[z0:z1], rtol=0, atol=1e-12)


def _partition_worker(rank, world, port, q):
    import sys
    import numpy as np
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    from paper_2103_04856_gb300 import inputs as I
    from paper_2103_04856_gb300 import slab as S
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        insts = I.batch_instances(64)
        parts = S.partition_instances([int(np.prod(i.shape)) for i in insts], world)
        mine = {k: np.full((2, 5), float(k) + 0.5 * rank) for k in parts[rank]}   # a per-problem "trace"
        q.put((rank, parts, S.gather_traces(mine, len(insts))))
    finally:
        dist.destroy_process_group()


def test_batch_partition_and_trace_gather_over_gloo_ranks():
    """The mixed batch split across ranks by work (voxels), each problem on
    exactly one rank, and the per-problem traces gathered on rank 0 in
    problem order."""
    import numpy as np
    from paper_2103_04856_gb300 import inputs as I
    from paper_2103_04856_gb300 import slab as S
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_partition_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=180) for _ in procs], key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    sizes = [int(np.prod(i.shape)) for i in I.batch_instances(64)]
    parts = res[0][1]
    assert res[1][1] == parts
    assert sorted(k for p in parts for k in p) == list(range(64))
    loads = [sum(sizes[k] for k in p) for p in parts]
    assert max(loads) - min(loads) <= max(sizes)
    owner = {k: r for r, p in enumerate(parts) for k in p}
    got = res[0][2]
    assert res[1][2] is None and len(got) == 64
    for k, t in enumerate(got):
        np.testing.assert_array_equal(t, np.full((2, 5), float(k) + 0.5 * owner[k]))
    assert S.partition_instances([5, 5, 5], 1) == [[0, 1, 2]]


def test_split_z_contiguous_and_balanced():
    from paper_2103_04856_gb300 import slab as S
    for nz, R in ((16, 2), (16, 3), (512, 8), (7, 3)):
        parts = S.split_z(nz, R)
        assert parts[0][0] == 0 and sum(n for _, n in parts) == nz
        assert all(parts[i][0] + parts[i][1] == parts[i + 1][0] for i in range(R - 1))
        assert max(n for _, n in parts) - min(n for _, n in parts) <= 1 and min(n for _, n in parts) >= 2
    with pytest.raises(ValueError):
        S.split_z(5, 3)


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
