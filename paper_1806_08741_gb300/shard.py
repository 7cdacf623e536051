"""One image shared by several GPUs: each rank holds a slab of planes.

The paper's parallel SSLIC splits the image into non-overlapping regions;
every thread assigns and maps the pixels of its region, and a reduce merges
the regions' per-label sums before the centres are divided out (Sec. 3.1).
Across GPUs the regions are slabs of planes along the last axis, one per
rank, and the reduce is one collective sum per iteration:

  seeding   every rank seeds the lattice planes of its slab
            (sslic_shard_seed: perturbation reads two planes around them);
            the centre tables are summed, each row coming from one rank
  iterate   sslic_shard_map on the slab -> exact integer sums (K x (C+4))
            all-reduce (sum) of those sums over the ranks
            sslic_shard_finalize: every rank divides the same sums, so every
            rank holds the same centres, those of a single-GPU run
  connect   (Sec. 3.1 stage 3) rank 0 receives the ranks' label slabs in
            order and runs the slab form of connectivity
            (sslic_conn_slabs_*), then sends every rank its relabelled slab

This module only moves buffers between the library and the collective
library (torch.distributed: NCCL across GPUs, gloo on host tensors); every
step of the method runs in the library's kernels.
"""
from __future__ import annotations

from dataclasses import dataclass


def slab_align(ndim: int) -> int:
    """Slab bounds are multiples of this many planes (the assignment and
    connectivity tiles' extent along the last axis)."""
    return 8 if ndim == 3 else 64


def slab_bounds(n_planes: int, world: int, align: int) -> list:
    """Contiguous slabs [lo, hi) covering [0, n_planes), one per rank, as
    even as the alignment allows; every bound but the last is a multiple of
    ``align``.  Raises ValueError when a rank would get no plane."""
    units = -(-n_planes // align)
    if world < 1 or units < world:
        raise ValueError(f"{n_planes} planes in steps of {align} cannot give {world} ranks a slab each")
    out = []
    for r in range(world):
        lo = (units * r // world) * align
        hi = min(n_planes, (units * (r + 1) // world) * align)
        out.append((lo, hi))
    return out


def halo_window(lo: int, hi: int, n_planes: int) -> tuple:
    """Planes of the image a rank needs for seeding its slab [lo, hi)."""
    return max(0, lo - 2), min(n_planes, hi + 2)


class Comm:
    """The collectives the sharded run needs, over torch.distributed: sums
    and point-to-point copies of tensors on the device (NCCL), or through
    host copies (any other backend, e.g. gloo)."""

    def __init__(self, group=None):
        import torch.distributed as dist

        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.device_tensors = dist.get_backend(group) == "nccl"

    def _host(self, t):
        return t if (self.device_tensors or not t.is_cuda) else t.cpu()

    def allreduce_sum(self, t) -> None:
        h = self._host(t)
        self.dist.all_reduce(h, group=self.group)
        if h is not t:
            t.copy_(h)

    def send(self, t, dst: int) -> None:
        self.dist.send(self._host(t), dst, group=self.group)

    def recv(self, t, src: int) -> None:
        if self.device_tensors or not t.is_cuda:
            self.dist.recv(t, src, group=self.group)
            return
        h = t.new_empty(t.shape, device="cpu")
        self.dist.recv(h, src, group=self.group)
        t.copy_(h)

    def broadcast_int(self, v: int, src: int = 0, device=None) -> int:
        import torch

        dev = device if self.device_tensors else "cpu"
        t = torch.tensor([int(v)], dtype=torch.int64, device=dev)
        self.dist.broadcast(t, src, group=self.group)
        return int(t.item())


@dataclass
class ShardResult:
    labels: object       # this rank's slab of labels (device, (hi - lo) * plane int32)
    centres: object      # K x (C + n) float32, the same on every rank
    iterations: int
    residual: float
    num_labels: int


def run_sharded(ctx, params, image_halo, lo: int, hi: int, comm: Comm, bounds: list, device) -> ShardResult:
    """The whole method on one image shared by ``comm.world`` ranks (call on
    every rank).  ``ctx``: a context created with the WHOLE image's
    parameters ``params``; ``image_halo``: this rank's planes
    ``halo_window(lo, hi, N)`` of the image (device, flat); ``bounds``: every
    rank's slab, from ``slab_bounds``."""
    import torch

    NL = params.size[-1]
    plane = 1
    for s in params.size[:-1]:
        plane *= int(s)
    C = params.channels
    a, _ = halo_window(lo, hi, NL)
    if bounds[comm.rank] != (lo, hi):
        raise ValueError("this rank's slab differs from its entry in bounds")
    K, CW = ctx.K, ctx.centre_width
    centres = torch.empty(K * CW, dtype=torch.float32, device=device)
    ctx.shard_seed(image_halo, lo, hi, centres)
    comm.allreduce_sum(centres)
    image_slab = image_halo[(lo - a) * plane * C:(hi - a) * plane * C]
    labels = torch.empty((hi - lo) * plane, dtype=torch.int32, device=device)
    nu, nf = ctx.shard_sums_size()
    sums = torch.empty(nu + nf, dtype=torch.int64, device=device)
    thr = params.conv_threshold
    res = 0.0
    it = 0
    for it in range(1, params.max_iter + 1):
        ctx.shard_map(image_slab, labels, lo, hi, centres, sums)
        comm.allreduce_sum(sums[:nu])
        if nf:
            comm.allreduce_sum(sums[nu:].view(torch.float64))
        # the residual needs a host read-back: only for a threshold and the report
        want = thr > 0.0 or it == params.max_iter
        r = ctx.shard_finalize(sums, centres, centres, residual=want)
        if want:
            res = r
        if thr > 0.0 and res < thr:
            break
    num_labels = K
    if params.enforce_connectivity:
        if comm.rank == 0:
            ctx.conn_slabs_begin(centres)
            for r, (rlo, rhi) in enumerate(bounds):
                if r == 0:
                    ctx.conn_slabs_add(labels, rlo, rhi)
                else:
                    buf = torch.empty((rhi - rlo) * plane, dtype=torch.int32, device=device)
                    comm.recv(buf, r)
                    ctx.conn_slabs_add(buf, rlo, rhi)
            num_labels = ctx.conn_slabs_finish()
            for r, (rlo, rhi) in enumerate(bounds):
                if r == 0:
                    ctx.conn_slabs_relabel(labels, rlo, rhi)
                else:
                    buf = torch.empty((rhi - rlo) * plane, dtype=torch.int32, device=device)
                    ctx.conn_slabs_relabel(buf, rlo, rhi)
                    if buf.is_cuda:
                        torch.cuda.current_stream(buf.device).synchronize()
                    comm.send(buf, r)
        else:
            if labels.is_cuda:
                torch.cuda.current_stream(labels.device).synchronize()
            comm.send(labels, 0)
            comm.recv(labels, 0)
        num_labels = comm.broadcast_int(num_labels, 0, device)
    return ShardResult(labels, centres.view(K, CW), it, res, num_labels)
