"""Multi-GPU partitioning of the event-rendering path.

The path shards without exchanging data while it runs: every frame is rendered
independently (the random numbers are keyed by pixel, sample and frame), and
both event generators keep per-pixel state only.  Two partitions are offered:

* frames: rank r renders and converts its own contiguous segment of the camera
  path (weak scaling; each rank carries its own event state, so segments are
  independent clips);
* bands: rank r owns a band of image rows for the whole clip.  The threshold
  generator and the point-wise (kernel 1) EvSNet need no halo; a stack of L
  3x3 convolutions needs L halo rows, which each rank recomputes from its own
  rendered rows (no exchange): bands are rendered with the halo included and
  the halo's events are dropped.

The one exchange step is the final gather of the event lists: an all_gather of
the per-rank counts, then an all_gather of the (padded) event arrays, with the
band offset added to y.  Rows are returned sorted by (t, y, x, p) so that the
sharded result is bitwise the unsharded one.

Training is data-parallel over clips: every rank computes the gradient of the
loss on its own clips and one all_reduce makes the mean over ranks.  The loss
(Eq. 7-11) is a mean over the batch's pixels, so with equal shards the mean of
the ranks' gradients is the whole batch's gradient.
"""
from __future__ import annotations

from typing import List, Tuple

import numpy as np


def frame_ranges(n_frames: int, world: int) -> List[Tuple[int, int]]:
    """Contiguous frame segments [a, b) per rank (sizes differ by at most one)."""
    base, extra = divmod(n_frames, world)
    out, a = [], 0
    for r in range(world):
        b = a + base + (1 if r < extra else 0)
        out.append((a, b))
        a = b
    return out


def row_bands(H: int, world: int, halo: int = 0) -> List[Tuple[int, int, int, int]]:
    """Per rank: (y0, y1) owned rows and (h0, h1) rows to compute (owned + halo)."""
    out = []
    for (y0, y1) in frame_ranges(H, world):
        out.append((y0, y1, max(0, y0 - halo), min(H, y1 + halo)))
    return out


def sort_events(ev: np.ndarray) -> np.ndarray:
    ev = np.asarray(ev, np.int32).reshape(-1, 4)
    if len(ev) == 0:
        return ev
    return ev[np.lexsort((ev[:, 3], ev[:, 0], ev[:, 1], ev[:, 2]))]


def gather_events(local: np.ndarray, y_offset: int = 0, group=None) -> np.ndarray:
    """All ranks' event lists (int32 [n, 4] = x, y, t, p), y shifted by each rank's
    band offset, concatenated and sorted; every rank receives the result."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    ev = np.asarray(local, np.int32).reshape(-1, 4).copy()
    ev[:, 1] += y_offset
    n = torch.tensor([len(ev)], dtype=torch.int64)
    counts = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(counts, n, group=group)
    m = int(max(c.item() for c in counts))
    buf = torch.zeros((max(m, 1), 4), dtype=torch.int32)
    buf[: len(ev)] = torch.from_numpy(ev)
    parts = [torch.zeros_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf, group=group)
    full = np.concatenate([p[: int(c.item())].numpy() for p, c in zip(parts, counts)])
    return sort_events(full)


def allreduce_mean(tensors, group=None):
    """Mean over ranks of each tensor, in place (one all_reduce for all of them:
    they are flattened into one buffer).  With the gloo backend the buffer goes
    through host memory."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    flat = torch.cat([t.reshape(-1) for t in tensors])
    buf = flat.cpu() if dist.get_backend(group) == "gloo" else flat
    dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
    buf = buf.to(flat.device) / world
    o = 0
    for t in tensors:
        n = t.numel()
        t.copy_(buf[o:o + n].reshape(t.shape))
        o += n
    return tensors
