"""Data exchange of the FMM partitioned over several GPUs (Sec. "Numerical solution": each
process owns a part of the octree and receives its locally essential tree from the others).

The plan (``kfmm_shard_plan``) and the locally essential trees (``kfmm_shard_let``) come from
the library; this module moves the data with torch.distributed collectives (NCCL between
GPUs, gloo in the CPU tests):
  - ghost sources: the points and densities of the leaves another rank's U and X lists need,
    one all-to-all (variable sizes);
  - shared boxes: upward densities of the coarse boxes that span several ranks, one
    all-reduce of every rank's partial sums;
  - ghost upward densities: those of boxes of another rank's V and W lists, one all-to-all.
Every rank derives every rank's locally essential tree from the same plan, so each knows what
to send without a request round.  Rows are in the tree's sorted source order (sources) or box
order (upward densities).
"""
from __future__ import annotations

import numpy as np

from . import TreeView, kfmm_shard_let, kfmm_shard_plan


class ShardExchange:
    def __init__(self, tv: TreeView, rank: int, world: int, box_cost=None, group=None):
        self.tv, self.rank, self.world, self.group = tv, rank, world, group
        self.owner, self.leaf_order, self.rank_cost = kfmm_shard_plan(tv, world, box_cost)
        self.lets = [kfmm_shard_let(tv, self.owner, q) for q in range(world)]
        self.src_range = tv.arrays["box_src"].reshape(-1, 2)
        self.shared = np.flatnonzero(self.owner == -1).astype(np.int32)

    # ------------------------------------------------------------------ helpers
    def owned_leaves(self, q=None):
        q = self.rank if q is None else q
        return self.leaf_order[self.owner[self.leaf_order] == q]

    def _rows(self, boxes):
        """Sorted-source rows of the given boxes, concatenated in box order."""
        if len(boxes) == 0:
            return np.zeros(0, np.int64)
        return np.concatenate([np.arange(self.src_range[b, 0], self.src_range[b, 1]) for b in boxes])

    def _a2a(self, send_parts, recv_counts, width, dtype):
        import torch
        import torch.distributed as dist
        send = np.concatenate([p.reshape(-1, width) for p in send_parts]) if send_parts else np.zeros((0, width))
        inp = torch.from_numpy(np.ascontiguousarray(send, dtype=dtype)).reshape(-1)
        out = torch.empty(int(sum(recv_counts)) * width, dtype=inp.dtype)
        dist.all_to_all_single(out, inp, output_split_sizes=[c * width for c in recv_counts],
                               input_split_sizes=[len(p) * width for p in send_parts], group=self.group)
        return out.numpy().reshape(-1, width)

    # ------------------------------------------------------------------ exchanges
    def gather_sources(self, values):
        """values [n_src, k]: rows of this rank's leaves valid.  Returns a copy in which the
        rows of its ghost source leaves hold the owners' values."""
        values = np.asarray(values)
        k = values.shape[1]
        send = []
        for q in range(self.world):
            boxes = [b for b in self.lets[q][0] if self.owner[b] == self.rank] if q != self.rank else []
            send.append(values[self._rows(boxes)])
        recv_boxes = [[b for b in self.lets[self.rank][0] if self.owner[b] == q] if q != self.rank else []
                      for q in range(self.world)]
        got = self._a2a(send, [len(self._rows(bx)) for bx in recv_boxes], k, values.dtype)
        out = values.copy()
        at = 0
        for bx in recv_boxes:
            rows = self._rows(bx)
            out[rows] = got[at:at + len(rows)]
            at += len(rows)
        return out

    def reduce_shared(self, partial):
        """partial [n_boxes, k]: this rank's part of every box's upward density (zero where it
        owns nothing below).  Returns a copy in which the shared boxes hold the sum over ranks."""
        import torch
        import torch.distributed as dist
        out = np.array(partial, copy=True)
        if len(self.shared):
            t = torch.from_numpy(np.ascontiguousarray(out[self.shared]))
            dist.all_reduce(t, group=self.group)
            out[self.shared] = t.numpy()
        return out

    def gather_up(self, values):
        """values [n_boxes, k]: rows of boxes this rank owns valid.  Returns a copy in which its
        ghost upward boxes hold the owners' values."""
        values = np.asarray(values)
        k = values.shape[1]
        send = []
        for q in range(self.world):
            boxes = [b for b in self.lets[q][1] if self.owner[b] == self.rank] if q != self.rank else []
            send.append(values[np.asarray(boxes, np.int64)])
        recv_boxes = [[b for b in self.lets[self.rank][1] if self.owner[b] == q] if q != self.rank else []
                      for q in range(self.world)]
        got = self._a2a(send, [len(bx) for bx in recv_boxes], k, values.dtype)
        out = values.copy()
        at = 0
        for bx in recv_boxes:
            out[np.asarray(bx, np.int64)] = got[at:at + len(bx)]
            at += len(bx)
        return out
