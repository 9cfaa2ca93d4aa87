"""Work across several GPUs, one process per GPU (torch.distributed ranks).

Two ways the descent path spreads over ranks:

* One large periodic grid split in z into slabs (``SlabDescent``).  A slab
  holds planes [z0, z0 + nz_local); the fused sweep of a plane reads planes up
  to two away (the cotangents of a voxel's neighbours need their own stencils:
  Sec. 4.1 periodic central differences), so before every sweep each rank
  receives the two planes below and the two above its slab from its periodic
  neighbours into its own halo buffer.  After the sweep the ranks all-gather
  their FP64 sums (energy, mass, sum of g, ...) and every rank combines the
  rows in rank order, so all ranks hold the same multiplier and the same
  offset of the mass projection, bit for bit.  The arithmetic runs in the
  library (``pfc.Slab``); this module only moves planes and sums.
* Independent problems (the mixed-size batch) partitioned across ranks
  (``partition_instances``), with the per-problem traces gathered on rank 0
  (``gather_traces``): no communication on the data path.

Transport is torch.distributed: NCCL for CUDA tensors, gloo for CPU tensors
(the CPU tests drive the same code with an arithmetic backend of their own).
"""
from __future__ import annotations

import numpy as np
import torch
import torch.distributed as dist

SLAB_ENERGY, SLAB_GRAD, SLAB_STEP = 0, 1, 2
SLAB_NSUMS = 8
HALO = 2          # planes a sweep reads beyond each end of its slab


def split_z(nz: int, nranks: int):
    """(z0, nz_local) of each rank: contiguous slabs, sizes differing by at
    most one plane, each at least HALO planes (so that the two planes a
    neighbour needs are that neighbour's own)."""
    if nranks < 1 or nz < HALO * nranks:
        raise ValueError(f"{nz} planes cannot be split into {nranks} slabs of >= {HALO} planes")
    base, extra = divmod(nz, nranks)
    out, z0 = [], 0
    for r in range(nranks):
        n = base + (1 if r < extra else 0)
        out.append((z0, n))
        z0 += n
    return out


def local_halos(fields, halos):
    """Fill the halos of slabs held in one process (fields[r], halos[r] in rank
    order; with one slab its own planes wrap around): planes 0, 1 of halo r
    are the last two planes of slab r-1, planes 2, 3 the first two of slab
    r+1 (periodically)."""
    R = len(fields)
    for r in range(R):
        halos[r][0:HALO].copy_(fields[(r - 1) % R][-HALO:])
        halos[r][HALO:].copy_(fields[(r + 1) % R][:HALO])


class HaloExchange:
    """Halo planes between periodic neighbours over a process group.

    Each rank sends its top two planes up (they become the upper rank's lower
    halo) and its bottom two planes down (the lower rank's upper halo).  The
    operations are posted in the same order on every rank, (send up, receive
    from below, send down, receive from above), with one tag per direction,
    so that messages between the same two ranks (two ranks: both neighbours
    are the same rank) pair up correctly under in-order matching (NCCL) and
    tag matching (gloo) alike.  With one rank the planes wrap locally."""

    def __init__(self, group=None):
        self.group = group
        self.world = dist.get_world_size(group) if dist.is_initialized() else 1
        self.rank = dist.get_rank(group) if dist.is_initialized() else 0

    def __call__(self, u, halo):
        if self.world == 1:
            local_halos([u], [halo])
            return
        up = self._global((self.rank + 1) % self.world)
        down = self._global((self.rank - 1) % self.world)
        top = u[-HALO:].contiguous()
        bottom = u[:HALO].contiguous()
        lo = torch.empty_like(halo[:HALO])
        hi = torch.empty_like(halo[HALO:])
        ops = [dist.P2POp(dist.isend, top, up, self.group, tag=1),
               dist.P2POp(dist.irecv, lo, down, self.group, tag=1),
               dist.P2POp(dist.isend, bottom, down, self.group, tag=2),
               dist.P2POp(dist.irecv, hi, up, self.group, tag=2)]
        for w in dist.batch_isend_irecv(ops):
            w.wait()
        halo[:HALO].copy_(lo)
        halo[HALO:].copy_(hi)

    def _global(self, r):
        return dist.get_global_rank(self.group, r) if self.group is not None else r


def gather_rows(row, out, group=None):
    """All-gather one row per rank into out (world x len(row)), rank order."""
    if not dist.is_initialized() or dist.get_world_size(group) == 1:
        out[0].copy_(row)
        return out
    parts = list(out.unbind(0))
    dist.all_gather(parts, row, group=group)
    return out


class SlabDescent:
    """Mass-projected descent of one periodic grid split in z over the ranks
    of ``group``: this rank holds ``u_local`` (its slab, a tensor (nz_local,
    ny, nx)) of the whole grid described by ``prob``.

    ``backend`` does the arithmetic: by default a ``pfc.Slab`` (the library's
    fused sweep on this rank's GPU); any object with the same ``sweep``,
    ``finish``, ``apply_offset`` methods serves.  Steps chain the mass
    projection in fused form: ``field()`` adds the pending offset and returns
    the projected slab."""

    def __init__(self, prob, u_local, z0: int, group=None, backend=None):
        self.group = group
        self.world = dist.get_world_size(group) if dist.is_initialized() else 1
        self.rank = dist.get_rank(group) if dist.is_initialized() else 0
        nzl = int(u_local.shape[0])
        if backend is None:
            from . import pfc
            backend = pfc.Slab(prob, z0, nzl)
        self.backend = backend
        self.exchange = HaloExchange(group)
        dev, dt = u_local.device, u_local.dtype
        self.cur = u_local
        self.nxt = torch.empty_like(u_local)
        self.halo = torch.empty((2 * HALO,) + tuple(u_local.shape[1:]), dtype=dt, device=dev)
        self.row = torch.zeros(SLAB_NSUMS, dtype=torch.float64, device=dev)
        self.rows = torch.zeros((self.world, SLAB_NSUMS), dtype=torch.float64, device=dev)
        self.pending = False

    def _sweep(self, mode, out, tau):
        self.exchange(self.cur, self.halo)
        self.backend.sweep(self.cur, self.halo, out, mode, tau, self.row)
        gather_rows(self.row, self.rows, self.group)

    def step(self, tau: float, scalars=None):
        """One descent step of the whole grid (this rank's share); scalars
        (optional tensor of 5 float64 on the slab's device) receives E, mass,
        lambda, max|g|, mean|g| of the field the step evaluated."""
        self._sweep(SLAB_STEP, self.nxt, tau)
        self.backend.finish(self.rows, scalars)
        self.cur, self.nxt = self.nxt, self.cur
        self.pending = True

    def run(self, nsteps: int, tau: float):
        """nsteps steps; returns the trace (nsteps, 5) as a numpy array."""
        tr = torch.zeros((nsteps, 5), dtype=torch.float64, device=self.row.device)
        for k in range(nsteps):
            self.step(tau, tr[k])
        return tr.cpu().numpy()

    def energy_and_grad(self, g):
        """E of the whole grid and g on this slab (the projected field)."""
        self.field()
        self._sweep(SLAB_GRAD, g, 0.0)
        sc = torch.zeros(5, dtype=torch.float64, device=self.row.device)
        self.backend.finish(self.rows, sc)
        return float(sc[0])

    def field(self):
        """The projected field of this slab (adds a pending offset in place)."""
        if self.pending:
            self.backend.apply_offset(self.cur)
            self.pending = False
        return self.cur


def partition_instances(sizes, nranks: int):
    """Indices of independent problems per rank, balanced by work (voxels):
    largest first, each to the least loaded rank (ties: lowest rank);
    deterministic, so every rank computes the same split."""
    order = sorted(range(len(sizes)), key=lambda k: (-int(sizes[k]), k))
    load = [0] * nranks
    parts = [[] for _ in range(nranks)]
    for k in order:
        r = min(range(nranks), key=lambda j: (load[j], j))
        parts[r].append(k)
        load[r] += int(sizes[k])
    return [sorted(p) for p in parts]


def gather_traces(local: dict, n_total: int, group=None):
    """Per-problem results of every rank (``local``: problem index -> numpy
    array) gathered on rank 0 as a list in problem order (None elsewhere)."""
    if not dist.is_initialized() or dist.get_world_size(group) == 1:
        return [local[k] for k in range(n_total)]
    got = [None] * dist.get_world_size(group)
    dist.all_gather_object(got, {int(k): np.asarray(v) for k, v in local.items()}, group=group)
    if dist.get_rank(group) != 0:
        return None
    merged = {}
    for d in got:
        merged.update(d)
    return [merged[k] for k in range(n_total)]
