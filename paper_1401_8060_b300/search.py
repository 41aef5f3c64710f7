"""Host-side orchestration of a search over a template range (no scoring here).

Template g is fixed by (seed, g) alone, so a range of templates can be split in
any way -- over GPUs, over time, over interrupted runs -- and the pieces' k
loudest combined by taking the largest SNRs gives exactly the single run's k
loudest (Sec. V: runs "combined" by the largest SNR_tot, and intermediate data
files).  This module holds that bookkeeping:

  shard_range     contiguous share of [0, T) for rank r of W
  merge_hits      combine hit arrays: SNR descending, then index ascending
  ResumableSearch score [offset, offset + T) in chunks, saving (next index, k
                  loudest so far) after every chunk; a restarted search resumes
  distributed_topk each rank scores its share, one all-gather of k records
"""
from __future__ import annotations

import json
import os
import tempfile

import numpy as np

from ._lib import HIT_DTYPE


def shard_range(n_tracks: int, world: int, rank: int):
    """(offset, count) of rank's contiguous share of [0, n_tracks)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    base, rem = divmod(int(n_tracks), int(world))
    off = rank * base + min(rank, rem)
    return off, base + (1 if rank < rem else 0)


def merge_hits(parts, k: int):
    """The k first of the concatenated hit arrays, by SNR descending then index ascending."""
    parts = [np.asarray(p, dtype=HIT_DTYPE).reshape(-1) for p in parts if p is not None and len(p)]
    if not parts:
        return np.zeros(0, dtype=HIT_DTYPE)
    allh = np.concatenate(parts)
    order = np.lexsort((allh["index"], -allh["snr"]))
    return allh[order[:k]].copy()


class ResumableSearch:
    """Score templates offset .. offset + n_tracks - 1 in chunks, checkpointing.

    score_fn(offset, count, k) -> HIT_DTYPE array of that chunk's k loudest
    (e.g. ``lambda o, c, k: (ctx.set_tracks(c, seed, o, tau_max), ctx.score(m, k))[1]``).
    The checkpoint (JSON: identity of the search, next index, hits so far) is
    replaced atomically after each chunk, so an interrupted run resumes exactly
    where it stopped and ends with the uninterrupted run's result.
    """

    def __init__(self, path: str, identity: dict, n_tracks: int, k: int, offset: int = 0, chunk: int = 1 << 24):
        self.path, self.identity = path, dict(identity)
        self.n_tracks, self.k, self.offset, self.chunk = int(n_tracks), int(k), int(offset), int(chunk)
        self.next = self.offset
        self.hits = np.zeros(0, dtype=HIT_DTYPE)
        if os.path.exists(path):
            self._load()

    def _state(self):
        return {"identity": self.identity, "n_tracks": self.n_tracks, "k": self.k, "offset": self.offset,
                "next": self.next,
                "hits": [[float(h["snr"]), int(h["index"]), [int(v) for v in h["f"]], float(h["tau"])]
                         for h in self.hits]}

    def _load(self):
        with open(self.path) as fh:
            st = json.load(fh)
        if (st["identity"] != self.identity or st["n_tracks"] != self.n_tracks or st["k"] != self.k
                or st["offset"] != self.offset):
            raise ValueError(f"checkpoint {self.path} belongs to another search")
        self.next = int(st["next"])
        h = np.zeros(len(st["hits"]), dtype=HIT_DTYPE)
        for i, (snr, idx, f, tau) in enumerate(st["hits"]):
            h[i]["snr"], h[i]["index"], h[i]["f"], h[i]["tau"] = snr, idx, f, tau
        self.hits = h

    def _save(self):
        d = os.path.dirname(os.path.abspath(self.path))
        fd, tmp = tempfile.mkstemp(dir=d, prefix=".ckpt")
        with os.fdopen(fd, "w") as fh:
            json.dump(self._state(), fh)
        os.replace(tmp, self.path)

    @property
    def done(self) -> bool:
        return self.next >= self.offset + self.n_tracks

    def run(self, score_fn, max_chunks: int | None = None):
        """Score remaining chunks (all, or at most max_chunks); returns the k loudest so far."""
        n = 0
        while not self.done and (max_chunks is None or n < max_chunks):
            count = min(self.chunk, self.offset + self.n_tracks - self.next)
            part = score_fn(self.next, count, min(self.k, count))
            self.hits = merge_hits([self.hits, part], self.k)
            self.next += count
            self._save()
            n += 1
        return self.hits


def distributed_topk(score_fn, n_tracks: int, k: int, group=None):
    """Each rank of torch.distributed scores its share of [0, n_tracks) with
    score_fn(offset, count, k) and the ranks exchange k records each (one
    all-gather); every rank returns the merged k loudest."""
    import torch.distributed as dist
    world, rank = dist.get_world_size(group), dist.get_rank(group)
    off, cnt = shard_range(n_tracks, world, rank)
    mine = score_fn(off, cnt, min(k, cnt)) if cnt else np.zeros(0, dtype=HIT_DTYPE)
    gathered = [None] * world
    dist.all_gather_object(gathered, np.asarray(mine, dtype=HIT_DTYPE).tobytes(), group=group)
    return merge_hits([np.frombuffer(b, dtype=HIT_DTYPE) for b in gathered], k)
