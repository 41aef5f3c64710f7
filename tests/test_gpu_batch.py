"""Batched scoring of many ragged maps in one persistent launch (stk_batch_*).

Every template's SNR uses the same per-pixel arithmetic as single-map scoring,
so each map's k loudest must equal what stk_score returns for that map alone
(bit for bit), and match the FP64 oracle within the parity tolerance.
"""
import time

import numpy as np
import pytest

from _parity import assert_topk_matches

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle  # noqa: E402
import paper_1401_8060_b300 as stk  # noqa: E402
from paper_1401_8060_b300 import _lib, synth  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    from paper_1401_8060_b300 import build
    build.build()
    c = stk.Context(0)
    yield c
    c.close()


def ragged(ctx, seed, n_maps, mode="freq", paper=False, fp16=False):
    rng = np.random.default_rng(seed)
    maps, hosts, nt, sd, of = [], [], [], [], []
    for i in range(n_maps):
        n_t = int(rng.integers(20, 91))
        n_f = int(rng.integers(40, 401))
        if mode == "pixel":
            sig = rng.uniform(0.5, 2.0, (n_t, n_f)).astype(np.float32)
        elif mode == "freq":
            sig = synth.sigma_powerlaw(40.0 + 0.5 * np.arange(n_f), float(rng.uniform(0.5, 2)))
        else:
            sig = np.full(n_f, 1.3, np.float32)
        y = synth.noise_map(n_t, n_f, sig, int(rng.integers(1 << 30)))
        maps.append(ctx.load_map(torch.from_numpy(y).cuda(), torch.from_numpy(sig).cuda(), 40.0, 0.5,
                                 paper_mode=paper, fp16=fp16))
        hosts.append((y, sig))
        nt.append(int(rng.integers(300, 30000)))
        sd.append(1000 + i)
        of.append(int(rng.integers(0, 1 << 40)))
    return maps, hosts, nt, sd, of


@pytest.mark.parametrize("mode,paper,fp16", [("freq", False, False), ("pixel", False, False),
                                             ("const", False, False), ("pixel", True, False),
                                             ("freq", False, True)])
def test_batch_equals_single_map_scoring(ctx, mode, paper, fp16):
    maps, _, nt, sd, of = ragged(ctx, 5, 11, mode, paper, fp16)
    k = 8
    b = stk.Batch(ctx, maps, nt, sd, of, 0.01)
    hits = b.score(k)
    for i, m in enumerate(maps):
        ctx.set_tracks(nt[i], sd[i], of[i], 0.01)
        ref = ctx.score(m, k)
        np.testing.assert_array_equal(hits[i], ref, err_msg=f"map {i}")
    b.close()


def test_batch_order_on_and_off_identical(ctx):
    """The batch scores each map's templates in coherent order by default (a
    bucket sort over all maps inside the captured graph); a batch created with
    index order returns the same hits bit for bit, also for many maps (fewer
    key bits per map) and ragged template counts."""
    maps, _, nt, sd, of = ragged(ctx, 15, 70, "freq")
    k = 5
    b1 = stk.Batch(ctx, maps, nt, sd, of, 0.01)
    h1 = b1.score(k)
    np.testing.assert_array_equal(b1.score(k), h1)
    ctx.set_option(_lib.STK_OPT_ORDER, 0)
    try:
        b0 = stk.Batch(ctx, maps, nt, sd, of, 0.01)
    finally:
        ctx.set_option(_lib.STK_OPT_ORDER, 1)
    np.testing.assert_array_equal(b0.score(k), h1)
    b0.close()
    b1.close()


def test_batch_map_without_exact_32bit_division(ctx):
    """An 885 x 2000 map has no exact 32-bit multiply-shift for its division by
    2 M^2 (the single-map path then uses the one-thread-per-template kernel);
    in a batch it takes the corrected division while the others keep theirs."""
    maps, hosts, nt, sd, of = ragged(ctx, 16, 3, "freq")
    sig = synth.sigma_powerlaw(40.0 + 0.5 * np.arange(2000), 1.0)
    y = synth.noise_map(885, 2000, sig, 17)
    maps.insert(1, ctx.load_map(torch.from_numpy(y).cuda(), torch.from_numpy(sig).cuda(), 40.0, 0.5))
    nt.insert(1, 3000)
    sd.insert(1, 77)
    of.insert(1, 5)
    k = 6
    b = stk.Batch(ctx, maps, nt, sd, of, 0.01)
    hits = b.score(k)
    for i, m in enumerate(maps):
        ctx.set_tracks(nt[i], sd[i], of[i], 0.01)
        np.testing.assert_array_equal(hits[i], ctx.score(m, k), err_msg=f"map {i}")
    om = oracle.OracleMap(y, sig, 40.0, 0.5, True)
    assert_topk_matches(hits[1], om.score_range(77, 5, 3000, 0.01), 5, k, what="885 x 2000 map")
    b.close()


def test_batch_vs_oracle(ctx):
    maps, hosts, nt, sd, of = ragged(ctx, 6, 5, "freq")
    k = 16
    b = stk.Batch(ctx, maps, nt, sd, of, 0.01)
    hits = b.score(k)
    for i in range(len(maps)):
        y, sig = hosts[i]
        om = oracle.OracleMap(y, sig, 40.0, 0.5, True)
        o = om.score_range(sd[i], of[i], nt[i], 0.01)
        assert_topk_matches(hits[i], o, of[i], k, what=f"batch map {i}")


def test_batch_graph_replay_k_change_and_tune(ctx):
    maps, _, nt, sd, of = ragged(ctx, 7, 9, "freq")
    b = stk.Batch(ctx, maps, nt, sd, of, 0.01)
    h8 = b.score(8)
    np.testing.assert_array_equal(b.score(8), h8)          # graph replay
    h3 = b.score(3)                                          # new graph for another k
    np.testing.assert_array_equal(h3, h8[:, :3])
    cfg = b.tune(8)
    assert cfg["threads"] in (512, 768, 1024) and 2 <= cfg["R"] <= 11 and cfg["nstage"] in (2, 3)
    assert cfg["R"] <= 5 or cfg["threads"] == 512
    np.testing.assert_array_equal(b.score(8), h8)          # any launch shape: same result
    out = torch.zeros(len(maps) * 8 * 40, dtype=torch.uint8, device="cuda")
    b.score(8, out=out)
    ctx.sync()
    np.testing.assert_array_equal(out.cpu().numpy().view(stk.HIT_DTYPE).reshape(len(maps), 8), h8)
    b.close()


def test_batch_cancel_before_and_during(ctx):
    maps, _, nt, sd, of = ragged(ctx, 8, 4, "freq")
    b = stk.Batch(ctx, maps, nt, sd, of, 0.01)
    ref = b.score(4)
    b.cancel(True)
    with pytest.raises(stk.StkError) as e:
        b.score(4)
    assert e.value.code == _lib.STK_ECANCELED
    b.cancel(False)
    np.testing.assert_array_equal(b.score(4), ref)           # usable again
    b.close()
    # a long batch (one 500 x 1600 map used 64 times, 2e6 templates each) stopped mid-run
    fm = synth.realistic_map(inject_signal=False)
    m = ctx.load_map(torch.from_numpy(fm.y).cuda(), torch.from_numpy(fm.sigma).cuda(), fm.f_min, fm.df)
    n = 64
    big = stk.Batch(ctx, [m] * n, [2_000_000] * n, list(range(n)), [0] * n, 0.01)
    out = torch.zeros(n * 4 * 40, dtype=torch.uint8, device="cuda")
    big.score(4, out=out)
    ctx.sync()
    t0 = time.perf_counter()
    big.score(4, out=out)
    ctx.sync()
    full = time.perf_counter() - t0
    big.score(4, out=out)
    time.sleep(full * 0.2)
    big.cancel(True)
    t1 = time.perf_counter()
    with pytest.raises(stk.StkError) as e:
        ctx.sync()
    assert e.value.code == _lib.STK_ECANCELED
    assert time.perf_counter() - t1 < full          # stopped well before a full run
    big.cancel(False)
    big.close()


def test_batch_rejects_mixed_maps(ctx):
    y = np.ones((10, 20), np.complex64)
    s = np.ones(20, np.float32)
    m1 = ctx.load_map(y, s, 40.0, 0.5)
    m2 = ctx.load_map(y, s, 40.0, 0.5, paper_mode=True)
    with pytest.raises(stk.StkError) as e:
        stk.Batch(ctx, [m1, m2], [100, 100], [1, 2], [0, 0], 0.01)
    assert e.value.code == _lib.STK_EINVAL
    b = stk.Batch(ctx, [m1], [100], [1], [0], 0.01)
    with pytest.raises(stk.StkError):
        b.score(_lib.STK_BATCH_MAX_K + 1)
    b.close()
