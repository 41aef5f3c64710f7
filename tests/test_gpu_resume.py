"""Checkpoint and resume of a search on the GPU.

Sec. V combines runs by their largest SNRs and keeps intermediate results; a
template is fixed by (seed, index) alone, so a range scored in chunks, with the
k loudest so far saved after every chunk, can stop anywhere and resume.  Here
search.ResumableSearch drives stk_set_tracks + stk_score over a range in uneven
chunks, is interrupted after three chunks, and resumes from its checkpoint file
in a new context (as a restarted process would): the result equals one
uninterrupted stk_score call over the whole range, bit for bit in indices, SNRs,
bins and delays.
"""
import json

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1401_8060_b300 as stk  # noqa: E402
from paper_1401_8060_b300 import search, synth  # noqa: E402

N_T, N_F, F_MIN, DF, TAU_MAX, SEED = 200, 1000, 40.0, 0.5, 0.010, 21


def _scorer(ctx, m):
    def score(offset, count, k):
        ctx.set_tracks(count, SEED, offset, TAU_MAX)
        return ctx.score(m, k)
    return score


def test_resumed_search_equals_one_call(tmp_path):
    from paper_1401_8060_b300 import build
    build.build()
    sig = synth.sigma_powerlaw(F_MIN + DF * np.arange(N_F))
    y = synth.noise_map(N_T, N_F, sig, 77)
    T, k, off, chunk = 2_000_003, 256, 1_000, 300_001
    ident = {"map": "noise 200x1000 seed 77", "seed": SEED, "tau_max": TAU_MAX}
    path = str(tmp_path / "search.json")

    ctx = stk.Context(0)
    m = ctx.load_map(torch.from_numpy(y).cuda(), torch.from_numpy(sig).cuda(), F_MIN, DF)
    ctx.set_tracks(T, SEED, off, TAU_MAX)
    whole = ctx.score(m, k)                                  # one uninterrupted call
    s1 = search.ResumableSearch(path, ident, T, k, offset=off, chunk=chunk)
    s1.run(_scorer(ctx, m), max_chunks=3)                    # interrupted after three chunks
    assert not s1.done and s1.next == off + 3 * chunk
    with open(path) as fh:
        assert json.load(fh)["next"] == off + 3 * chunk
    m.close()
    ctx.close()

    ctx2 = stk.Context(0)                                    # a restarted process: new context, new map
    m2 = ctx2.load_map(torch.from_numpy(y).cuda(), torch.from_numpy(sig).cuda(), F_MIN, DF)
    s2 = search.ResumableSearch(path, ident, T, k, offset=off, chunk=chunk)
    assert s2.next == off + 3 * chunk
    res = s2.run(_scorer(ctx2, m2))
    assert s2.done
    for field in ("snr", "index", "f", "tau"):
        np.testing.assert_array_equal(res[field], whole[field], err_msg=field)
    with pytest.raises(ValueError):                          # another search's checkpoint is refused
        search.ResumableSearch(path, dict(ident, seed=SEED + 1), T, k, offset=off, chunk=chunk)
    m2.close()
    ctx2.close()
