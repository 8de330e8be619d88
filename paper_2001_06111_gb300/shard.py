"""Single-graph counting shard over processes (one process per GPU).

Counting enumerates every priority-obeyed wedge from its start vertex, the
wedge's vertex of highest priority (Section IV-B), and Lemma 3 places every
butterfly in exactly one bloom, the one started at the butterfly's vertex of
highest priority.  So the start vertices can be cut into ranges that
processes count independently (``bt_count_support_part``: contiguous priority
ranks holding about equal numbers of wedges), and one sum reduction of the
per-edge arrays gives every process the supports.  Each process holds the
whole edge list; the only exchange is that reduction (over NCCL with CUDA
tensors, or any torch.distributed backend with host tensors).
"""
from __future__ import annotations

import numpy as np

from . import bitruss


def count_support_sharded(edges, nU: int, nL: int, handle=None, group=None, flags: int = 0,
                          count_part=None):
    """Supports of every edge (uint64, input order), counted as part
    ``rank`` of ``world_size`` wedge-balanced start-vertex ranges by each
    process of ``group`` and summed with one all-reduce.

    edges: numpy int32 (m, 2) -- every process passes the same graph.
    handle: a ``bitruss.Handle`` on this process's GPU.
    count_part: optional ``f(part, nparts) -> uint64[m]`` used instead of the
    library (so the reduction can be exercised without a GPU).
    Returns a numpy uint64 array on every process."""
    import torch
    import torch.distributed as dist

    rank = dist.get_rank(group)
    world = dist.get_world_size(group)
    on_gpu = dist.get_backend(group) == "nccl"
    if count_part is not None:
        part = torch.from_numpy(np.ascontiguousarray(count_part(rank, world), dtype=np.uint64).view(np.int64))
        if on_gpu:
            part = part.cuda()
    elif on_gpu:
        d_edges = torch.from_numpy(np.ascontiguousarray(edges, dtype=np.int32)).cuda()
        part = torch.empty(d_edges.shape[0], dtype=torch.int64, device=d_edges.device)
        bitruss.bt_count_support_part(handle, d_edges, nU, nL, rank, world, support_out=part, flags=flags)
    else:
        sup, _, _ = bitruss.bt_count_support_part(handle, edges, nU, nL, rank, world, flags=flags)
        part = torch.from_numpy(sup.view(np.int64))
    # supports are below 2^63: the signed sum is exact
    dist.all_reduce(part, op=dist.ReduceOp.SUM, group=group)
    return part.cpu().numpy().view(np.uint64)
