"""Strip sharding of one image: each rank (one GPU) labels a horizontal strip,
and the strips are joined at their seams by the boundary analysis of Sec. 3.2.

Rank r holds strip r (rows ``[y0_r, y0_r + H_r)``, in order).  The work per
rank is two library calls around one exchange:

1. ``ccl_strip_begin``: step 1 and the block merge of the strip, and its two
   edge rows (the key of the component of every pixel of its first and last
   row, as a raster position of the whole image);
2. ``all_gather`` of the edge rows (2 x W uint32 per rank) -- the only data
   the ranks exchange;
3. ``ccl_strip_resolve`` (host): the seam union, the same on every rank;
4. ``ccl_strip_finish``: the strip's roots take their keys of the whole image,
   and the write-out fills the strip's labels.

``label_strips_one_gpu`` runs the same steps for G strips on one GPU (the
gather is a stack of the edge rows).
"""
from __future__ import annotations

import numpy as np

from . import ccl

STRIP_ROWS = 64  # strips start on, and (but the last) span, whole 64-row block rows


def strip_bounds(H_total: int, strips: int) -> list[tuple[int, int]]:
    """(y0, H) of `strips` strips covering H_total rows: whole 64-row block
    rows, spread as evenly as they go; the last strip takes the ragged rest."""
    if strips < 1:
        raise ValueError("at least one strip")
    nblk = (H_total + STRIP_ROWS - 1) // STRIP_ROWS
    if strips > max(nblk, 1):
        raise ValueError(f"{strips} strips need at least {strips} block rows of {STRIP_ROWS} (have {nblk})")
    out, y = [], 0
    for g in range(strips):
        take = nblk // strips + (1 if g < nblk % strips else 0)
        h = min(take * STRIP_ROWS, H_total - y)
        out.append((y, h))
        y += h
    return out


def gather_edges(edges, group=None) -> np.ndarray:
    """All-gather of every rank's edge rows, in rank order: uint32 [ranks, 2, W]."""
    import torch
    import torch.distributed as dist

    if dist.get_backend(group) == "gloo":
        edges = edges.cpu()
    bufs = [torch.empty_like(edges) for _ in range(dist.get_world_size(group))]
    dist.all_gather(bufs, edges.contiguous(), group=group)
    return torch.stack(bufs).cpu().numpy().view(np.uint32)


def label_strip(img, y0: int, H_total: int, connectivity: int = 8, group=None, workspace=None, labels=None):
    """Labels of this rank's strip `img` (rows [y0, y0 + H) of the image), the
    labels of the whole image: 1 + the smallest position of each component
    over all strips.  Every rank of `group` calls it with its own strip, the
    ranks in strip order.  Runs on the current stream."""
    import torch

    H, W = img.shape
    if workspace is None:
        workspace = torch.empty(max(ccl.ccl_workspace_size(H, W, connectivity), 1), dtype=torch.uint8,
                                device=img.device)
    edges = ccl.ccl_strip_begin(img, y0, H_total, workspace, connectivity)
    pairs = ccl.ccl_strip_resolve(gather_edges(edges, group), connectivity)
    seam = torch.from_numpy(pairs.view(np.int32)).to(img.device) if len(pairs) else None
    return ccl.ccl_strip_finish(H, W, y0, H_total, seam, workspace, connectivity, labels)


def label_strips_one_gpu(img, strips: int, connectivity: int = 8, labels=None, workspaces=None):
    """The strip-sharded labelling of `img` as `strips` strips on its own GPU
    (current stream): begin per strip, gather, resolve, finish per strip."""
    import torch

    H_total, W = img.shape
    bounds = strip_bounds(H_total, strips)
    if labels is None:
        labels = torch.empty((H_total, W), dtype=torch.int32, device=img.device)
    if workspaces is None:
        workspaces = [torch.empty(max(ccl.ccl_workspace_size(h, W, connectivity), 1), dtype=torch.uint8,
                                  device=img.device) for _, h in bounds]
    edges = [ccl.ccl_strip_begin(img[y0:y0 + h], y0, H_total, ws, connectivity)
             for (y0, h), ws in zip(bounds, workspaces)]
    pairs = ccl.ccl_strip_resolve(torch.stack(edges).cpu().numpy(), connectivity)
    seam = torch.from_numpy(pairs.view(np.int32)).to(img.device) if len(pairs) else None
    for (y0, h), ws in zip(bounds, workspaces):
        ccl.ccl_strip_finish(h, W, y0, H_total, seam, ws, connectivity, labels[y0:y0 + h])
    return labels
