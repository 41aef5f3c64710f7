"""Host-side search bookkeeping on CPU: range sharding, merging of k-records,
checkpoint/resume, and the multi-rank path over gloo (world size 2), including
a rank that fails before the exchange.  Scoring here is the FP64 oracle."""
import multiprocessing as mp
import socket

import numpy as np
import pytest

import oracle
from paper_1401_8060_b300 import HIT_DTYPE, search

from _dist_worker import oracle_scorer, run_rank


def _port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _full_topk(n_tracks, k):
    return oracle_scorer()(0, n_tracks, k)


@pytest.mark.parametrize("T,W", [(10, 3), (1000, 7), (5, 8), (2 ** 33 + 5, 4)])
def test_shard_range_partitions(T, W):
    parts = [search.shard_range(T, W, r) for r in range(W)]
    assert parts[0][0] == 0
    for (o1, c1), (o2, _) in zip(parts, parts[1:]):
        assert o1 + c1 == o2
    assert parts[-1][0] + parts[-1][1] == T
    assert max(c for _, c in parts) - min(c for _, c in parts) <= 1


def test_merge_matches_single_run():
    score = oracle_scorer()
    full = score(0, 3000, 20)
    parts = [score(o, c, 20) for o, c in [(0, 700), (700, 1500), (2200, 800)]]
    np.testing.assert_array_equal(search.merge_hits(parts, 20), full)


def test_checkpoint_resume_equals_uninterrupted(tmp_path):
    score = oracle_scorer()
    ident = {"map": "synthetic 40x60 seed 17", "seed": 3, "tau_max": 0.01}
    full = search.ResumableSearch(str(tmp_path / "a.json"), ident, 5000, 16, chunk=700).run(score)
    p = str(tmp_path / "b.json")
    s1 = search.ResumableSearch(p, ident, 5000, 16, chunk=700)
    s1.run(score, max_chunks=3)                    # interrupted after three chunks
    assert not s1.done and s1.next == 2100
    s2 = search.ResumableSearch(p, ident, 5000, 16, chunk=700)   # a new process would do this
    assert s2.next == 2100
    res = s2.run(score)
    assert s2.done
    np.testing.assert_array_equal(res, full)
    np.testing.assert_array_equal(full, _full_topk(5000, 16))
    with pytest.raises(ValueError):
        search.ResumableSearch(p, dict(ident, seed=4), 5000, 16, chunk=700)


def _spawn(world, n_tracks, k, fail_rank):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    procs = [ctx.Process(target=run_rank, args=(r, world, port, n_tracks, k, fail_rank, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
    return sorted(out)


def test_gloo_two_ranks_merge_exactly():
    out = _spawn(2, 4000, 12, fail_rank=-1)
    assert [o[1] for o in out] == ["ok", "ok"], out
    ref = _full_topk(4000, 12)
    for _, _, b in out:
        np.testing.assert_array_equal(np.frombuffer(b, dtype=HIT_DTYPE), ref)


def test_gloo_failed_rank_is_detected():
    out = _spawn(2, 2000, 4, fail_rank=1)
    assert out[1][1] == "error" and "fails before" in out[1][2]
    assert out[0][1] == "error"          # the surviving rank's exchange fails instead of hanging
