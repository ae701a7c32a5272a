"""Multi-GPU layout of the depth-map path (host side).

Reference views are independent units for initialisation, propagation and
refinement (the paper's pipeline loops over reference images), so they are
sharded over ranks with no data exchange.  The one exchange step is before
the geometric-consistency filter (Sec. III-D), which reads the depth maps of
the source views: every rank receives every view's plane map into its own
memory (one broadcast per view from its owner).  No kernel reads another
GPU's memory.  filter_sharded runs the whole depth-map stage this way
through the library.
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


def filter_sharded(mvs, ctx, shapes, srcs_of, params, fparams, group=None, device=None):
    """Depth maps and geometric filter of all views of a context, sharded over
    the ranks of `group` (Algorithm 1's loop over reference images): this
    rank runs its share of the views (assign_views by pixel count) as one
    batched PatchMatch call, every rank receives every view's plane map (the
    one exchange), stores the maps of the other ranks' views in its context
    (mvs_set_depth_map) and filters its own views against their sources.
      mvs: the binding module; ctx: its Context over all views; shapes:
      (H, W) per view; srcs_of: the source views of each view.
    Returns ({view: keep mask (H, W) uint8 on `device`}, {view: plane map})
    for this rank's views.  The exchange runs on the device under NCCL and
    through host memory under gloo."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
    parts = assign_views([h * w for h, w in shapes], world)
    mine = parts[rank]
    planes = {v: torch.empty(tuple(shapes[v]) + (4,), dtype=torch.float32, device=dev) for v in mine}
    costs = {v: torch.empty(tuple(shapes[v]), dtype=torch.float32, device=dev) for v in mine}
    if mine:
        mvs.mvs_patchmatch_batch(ctx.h, mine, [list(srcs_of[v]) for v in mine], params, [planes[v] for v in mine],
                                 [costs[v] for v in mine])
    xdev = dev if dist.get_backend(group) == "nccl" else torch.device("cpu")
    torch.cuda.synchronize(dev)
    allm = exchange_plane_maps({v: planes[v].to(xdev) for v in mine}, shapes, parts, group=group, device=xdev)
    for v, m in allm.items():
        if v not in planes:
            mvs.mvs_set_depth_map(ctx.h, v, m.to(dev).contiguous())
    keeps = {}
    for v in mine:
        keeps[v] = torch.empty(tuple(shapes[v]), dtype=torch.uint8, device=dev)
        mvs.mvs_geo_filter(ctx.h, v, list(srcs_of[v]), fparams, keeps[v])
    return keeps, planes
