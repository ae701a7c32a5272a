"""Multi-GPU layout of the depth-map path (host side).

Reference views are independent units for initialisation, propagation and
refinement (the paper's pipeline loops over reference images), so they are
sharded over ranks with no data exchange.  The one exchange step is before
the geometric-consistency filter (Sec. III-D), which reads the depth maps of
the source views: every rank receives every view's plane map into its own
memory (one broadcast per view from its owner).  No kernel reads another
GPU's memory.
"""
from __future__ import annotations


def assign_views(pixel_counts, world):
    """Balanced partition of reference views over `world` ranks by pixel
    count (largest first onto the least-loaded rank).  Returns a list of
    view-index lists, one per rank."""
    load = [0] * world
    parts = [[] for _ in range(world)]
    for v in sorted(range(len(pixel_counts)), key=lambda i: (-pixel_counts[i], i)):
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(v)
        load[r] += pixel_counts[v]
    return [sorted(p) for p in parts]


def owner_of(assignment):
    return {v: r for r, views in enumerate(assignment) for v in views}


def exchange_plane_maps(maps, shapes, assignment, group=None, device=None):
    """maps: {view: tensor (H, W, 4)} for the views this rank owns.
    Returns {view: tensor} for all views (own tensors kept, others received
    by broadcast from their owner).  Received tensors are allocated on
    ``device`` when given, else on the device of this rank's own maps, else
    on the current CUDA device under NCCL and on the CPU otherwise (a rank
    may own no view).  ``assignment`` lists the views of each rank of
    ``group`` by group rank."""
    import torch
    import torch.distributed as dist
    rank = dist.get_rank(group)
    own = owner_of(assignment)
    if device is None:
        if maps:
            device = next(iter(maps.values())).device
        elif dist.get_backend(group) == "nccl":
            device = torch.device("cuda", torch.cuda.current_device())
        else:
            device = torch.device("cpu")
    out = {}
    for v in sorted(own):
        H, W = shapes[v]
        if own[v] == rank:
            t = maps[v].contiguous()
        else:
            t = torch.empty((H, W, 4), dtype=torch.float32, device=device)
        src = own[v] if group is None else dist.get_global_rank(group, own[v])
        dist.broadcast(t, src=src, group=group)
        out[v] = t
    return out
