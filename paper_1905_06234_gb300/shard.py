"""Voxel-sharded SBB-NNLS: the host side of the exchange.

Each shard holds the Phi entries of one voxel range (``life_build_index_shard``),
its rows of the signal b, and replicated copies of w and the SBB state.  An
iteration is three phases on every shard (``life_sbb_shard_phase``) with two
exchanges between them, in which the fascicle-length vectors g = Σ_s M_s^T e_s
and u = Σ_s M_s^T M_s g~ and the scalars Σ e² and Σ (M g~)² are summed over all
shards.  This module decides which buffers are summed and when; the
arithmetic runs in the CUDA library, and the sums in torch.distributed (one
shard per process, NCCL on GPUs or gloo) or, for shards held by one process,
in an in-process sum.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import torch

from . import _native as N


@dataclass
class Shard:
    """One voxel range: its index, signal rows, the replicated w and state, the
    exchange buffers (g, u: Nf floats; scal: two doubles) and the workspace."""
    index: object
    D: torch.Tensor
    b: torch.Tensor
    w: torch.Tensor
    st: object
    workspace: object = None
    g: torch.Tensor = None
    u: torch.Tensor = None
    scal: torch.Tensor = None
    extra: dict = field(default_factory=dict)


class GpuPhases:
    """Phases run by liblife on the device that holds the shard."""

    def phase(self, s: Shard, k: int, tol: float, eq7_on_even: bool):
        N.life_sbb_shard_phase(s.index, s.D, s.b, s.w, s.g, s.u, s.scal, s.st, s.workspace, k, tol=tol,
                               eq7_on_even=eq7_on_even)


class ProcessGroupSum:
    """Exchange across processes, one shard per rank: an all-reduce (sum) of each
    buffer over the process group.  Every rank receives the same sums."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group

    def sum_(self, bufs):
        assert len(bufs) == 1, "one shard per rank"
        for t in bufs[0]:
            self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM, group=self.group)


class LocalSum:
    """Exchange among the shards one process holds (several shards on one device,
    the single-process stand-in for a multi-rank run): each buffer becomes the
    sum over shards, added in shard order, so every shard holds the same value."""

    def sum_(self, bufs):
        for i in range(len(bufs[0])):
            tot = bufs[0][i].clone()
            for sb in bufs[1:]:
                tot += sb[i]
            for sb in bufs:
                sb[i].copy_(tot)


class ShardedSBB:
    """SBB-NNLS iterations over voxel shards: phase 1, sum (g, Σe²), phase 2,
    sum (u, Σ v'²), phase 3."""

    def __init__(self, shards, phases, exchange, tol=0.0, eq7_on_even=True):
        self.shards = list(shards)
        self.phases = phases
        self.exchange = exchange
        self.tol = float(tol)
        self.eq7_on_even = bool(eq7_on_even)

    def step(self):
        for s in self.shards:
            self.phases.phase(s, 1, self.tol, self.eq7_on_even)
        self.exchange.sum_([[s.g, s.scal[0:1]] for s in self.shards])
        for s in self.shards:
            self.phases.phase(s, 2, self.tol, self.eq7_on_even)
        self.exchange.sum_([[s.u, s.scal[1:2]] for s in self.shards])
        for s in self.shards:
            self.phases.phase(s, 3, self.tol, self.eq7_on_even)

    def solve(self, max_iter: int):
        for _ in range(int(max_iter)):
            self.step()


def gpu_shard(index, D, b, w=None, st=None):
    """A Shard on the current CUDA device with fresh exchange buffers, workspace
    and (unless given) w = 1 and an initial state."""
    nf = index.n_fasc
    dev = D.device
    return Shard(index=index, D=D, b=b,
                 w=torch.ones(nf, dtype=torch.float32, device=dev) if w is None else w,
                 st=N.new_sbb_state() if st is None else st,
                 workspace=N.new_sbb_workspace(index),
                 g=torch.empty(nf, dtype=torch.float32, device=dev),
                 u=torch.empty(nf, dtype=torch.float32, device=dev),
                 scal=torch.zeros(2, dtype=torch.float64, device=dev))


def voxel_ranges(n_voxels: int, n_shards: int):
    """Contiguous voxel ranges [v0, v1) of nearly equal size."""
    q, r = divmod(int(n_voxels), int(n_shards))
    out, v = [], 0
    for k in range(int(n_shards)):
        n = q + (1 if k < r else 0)
        out.append((v, v + n))
        v += n
    return out
