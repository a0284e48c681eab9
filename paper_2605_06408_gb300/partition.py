"""One diagram's cells split over several processes, one per GPU.

The cells of Eq. 1 are independent of each other (Sec. 3), so a diagram
partitions by cells: every rank holds all sites and builds the whole LBVH
(a replica), then makes only the cells of its contiguous range of the
Morton-sorted order (``Context.set_partition``, vd_set_partition in the C
ABI). A rank's build returns full-size outputs in which the cells of the
other ranks have empty neighbour rows and volume and centroid 0.

The exchange steps:
  - forward: the outputs may stay sharded; ``gather`` makes the whole
    diagram on every rank (an all-gather of the neighbour rows, a sum of the
    volume and centroid arrays);
  - backward: each rank's adjoint covers its own cells and scatters into
    full-size gradient arrays; one all-reduce (sum) gives the gradient of
    the whole loss (``allreduce_gradients``).

Argument marshalling and collectives only: the cells come from libvd's
kernels. ``merge_parts`` is the host-free core of ``gather``: it takes every
part's rows and sums, as a single process holding all parts would.
"""
from __future__ import annotations

from typing import Optional, Sequence

import torch


def part_range(n: int, part: int, nparts: int) -> tuple[int, int]:
    """Sorted (Morton-order) indices [begin, end) of the cells of `part`."""
    return (n * part) // nparts, (n * (part + 1)) // nparts


def merge_parts(offsets: Sequence[torch.Tensor], neighbors: Sequence[torch.Tensor]):
    """The whole diagram's CSR (int32 offsets [n+1], int32 neighbours) from
    every part's CSR (same n; a cell's row is non-empty in at most one
    part): each row is copied to its place in the merged CSR."""
    n = offsets[0].shape[0] - 1
    dev = offsets[0].device
    counts = torch.zeros(n, dtype=torch.int64, device=dev)
    for off in offsets:
        counts += torch.diff(off.to(torch.int64))
    out_off = torch.zeros(n + 1, dtype=torch.int64, device=dev)
    out_off[1:] = torch.cumsum(counts, 0)
    out_nb = torch.empty(int(out_off[-1].item()), dtype=torch.int32, device=dev)
    rows = torch.arange(n, device=dev)
    for off, nb in zip(offsets, neighbors):
        off = off.to(torch.int64)
        cnt = torch.diff(off)
        m = int(off[-1].item())
        if m == 0:
            continue
        r = torch.repeat_interleave(rows, cnt)
        pos = torch.arange(m, device=dev) - off[r]
        out_nb[out_off[r] + pos] = nb[:m].to(torch.int32)
    return out_off.to(torch.int32), out_nb


def gather(offsets: torch.Tensor, neighbors: torch.Tensor, volume: torch.Tensor, centroid: torch.Tensor,
           group=None):
    """The whole diagram on every rank from each rank's part: returns
    (offsets, neighbors, volume, centroid). Collectives: one all-gather of
    the row sizes, one of the offsets, one of the (padded) neighbour arrays,
    and a sum of the volume and centroid arrays."""
    import torch.distributed as dist

    ws = dist.get_world_size(group)
    dev = offsets.device
    nnz = torch.tensor([int(offsets[-1].item())], dtype=torch.int64, device=dev)
    sizes = [torch.zeros_like(nnz) for _ in range(ws)]
    dist.all_gather(sizes, nnz, group=group)
    top = max(int(s.item()) for s in sizes)
    padded = torch.zeros(max(top, 1), dtype=torch.int32, device=dev)
    padded[: int(nnz.item())] = neighbors[: int(nnz.item())]
    all_nb = [torch.empty_like(padded) for _ in range(ws)]
    dist.all_gather(all_nb, padded, group=group)
    all_off = [torch.empty_like(offsets) for _ in range(ws)]
    dist.all_gather(all_off, offsets.contiguous(), group=group)
    vol = volume.clone()
    cen = centroid.clone()
    dist.all_reduce(vol, group=group)
    dist.all_reduce(cen, group=group)
    off, nb = merge_parts(all_off, all_nb)
    return off, nb, vol, cen


def allreduce_gradients(grad_sites: torch.Tensor, grad_weights: Optional[torch.Tensor] = None, group=None):
    """Sum every rank's partial gradients in place: each rank's adjoint
    covered only its own cells, whose faces also move neighbouring sites."""
    import torch.distributed as dist

    dist.all_reduce(grad_sites, group=group)
    if grad_weights is not None:
        dist.all_reduce(grad_weights, group=group)
    return grad_sites, grad_weights
