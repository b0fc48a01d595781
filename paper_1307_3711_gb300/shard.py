"""One cluster spread over several GPUs by target records.

The step's cost is the direct sum over all pairs (Sec. II, particle mover
paragraph; Sec. III: time grows as N_part^2).  The paper parallelises its
force and mover loops over target particles on the cores of one node; here the
same split spreads one cluster over GPUs, one process per GPU:

  * every rank holds the whole cluster in a context of its own and pushes only
    its slice of target records (md_set_slice), summing the field of all
    sources at them;
  * after each step the ranks exchange their slices of the j-stream (the
    float4 (x, y, z, K_C w z) records the next step reads as sources, 16 bytes
    per record) with one all-gather, written into every rank's j-stream
    (md_get_jstream).

This module is marshalling and the collective only: the sums and pushes run in
the library's kernels.  The exchange works on any torch tensor of [n, 4]
records and any torch.distributed backend (NCCL between GPUs, gloo on CPU).
"""
from __future__ import annotations

import math

# slice bounds are multiples of this (a whole number of i-blocks of every
# kernel configuration of the library)
SLICE_ALIGN = 1024


def slice_bounds(n: int, world: int, rank: int, align: int = SLICE_ALIGN):
    """[b, e) of rank's target records in a cluster of n records split over
    `world` ranks, and the slice length `per` every rank sends (the last
    slices are shorter or empty).  per and b are multiples of align, except
    that an empty slice past the end has b = e = n."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    per = int(math.ceil(math.ceil(n / world) / align)) * align
    b = min(rank * per, n)
    e = min(b + per, n)
    return b, e, per


def exchange(jst, per: int, world: int, rank: int, group=None):
    """jst: [n, 4] records holding this rank's slice [rank per, rank per + per)
    (clipped to n) up to date.  After the call every slice is, from the rank
    that owns it: one all-gather of `per` records from each rank (a short or
    empty last slice is padded with zeros, which are not copied back)."""
    import torch
    import torch.distributed as dist
    n = jst.shape[0]
    b = min(rank * per, n)
    e = min(b + per, n)
    send = torch.zeros((per,) + tuple(jst.shape[1:]), dtype=jst.dtype, device=jst.device)
    send[: e - b] = jst[b:e]
    if dist.get_backend(group) == "nccl":
        out = torch.empty((world * per,) + tuple(jst.shape[1:]), dtype=jst.dtype,
                          device=jst.device)
        dist.all_gather_into_tensor(out, send, group=group)
    else:
        parts = [torch.empty_like(send) for _ in range(world)]
        dist.all_gather(parts, send, group=group)
        out = torch.cat(parts)
    jst.copy_(out[:n])
    return jst


class _DeviceRecords:
    """A device address seen by torch as float32 [n, 4] records, without a
    copy (the CUDA array interface)."""

    def __init__(self, ptr: int, n: int):
        self.__cuda_array_interface__ = {"shape": (n, 4), "typestr": "<f4",
                                         "data": (ptr, False), "version": 3, "strides": None}


def jstream_tensor(ctx, cluster: int = 0):
    """The context's current j-stream of `cluster` as a torch tensor that
    aliases the library's device buffer (valid until the next step)."""
    import torch
    ptr, n = ctx.jstream(cluster)
    return torch.as_tensor(_DeviceRecords(ptr, n), device="cuda")


class ShardedCluster:
    """One cluster pushed by `world` ranks, each on its own GPU: rank `rank`
    owns the targets slice_bounds(n, world, rank).  The context runs on
    `stream` (a cudaStream_t), which must be torch's current stream so that
    the all-gather is ordered between the steps."""

    def __init__(self, md, config, particles, world: int, rank: int, group=None, stream=None):
        self.world, self.rank, self.group = world, rank, group
        self.ctx = md.Context([config], [particles], stream=stream)
        self.b, self.e, self.per = slice_bounds(particles.n, world, rank)
        self.ctx.set_slice(0, self.b, self.e)

    def step(self, nsteps: int = 1):
        for _ in range(nsteps):
            self.ctx.step(1)
            if self.world > 1:
                exchange(jstream_tensor(self.ctx), self.per, self.world, self.rank, self.group)

    def close(self):
        self.ctx.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
