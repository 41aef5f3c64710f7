"""stk_score_noalloc: scoring for callers that cannot allocate device memory.

Callers whose device memory is owned by another allocator, or that cannot take
cudaFree's synchronisation in a hot loop, score through stk_score_noalloc,
whose scratch is a fixed device array inside the library.  This file checks,
through the C ABI, that two calls in a row return exactly the hits stk_score
returns (the SNR of a template does not depend on the order templates are
scored in, and the selection is exact), that the loudest agrees with the FP64
oracle, that the steady-state call allocates nothing, that the call waits for a
map update still packing on the context's stream when it runs on another
stream, that a timed-out wait or bad deferred map data marks every hit invalid
(with or without a status word), and that ranges beyond the fixed scratch are
refused.  It is collected last so a failure here never hides another test.
"""
import ctypes as C

import numpy as np
import pytest

from _parity import RTOL

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle  # noqa: E402
import paper_1401_8060_b300 as stk  # noqa: E402
from paper_1401_8060_b300 import _lib, synth  # noqa: E402

N_T, N_F, F_MIN, DF, TAU_MAX = 240, 900, 40.0, 0.5, 0.010


def _map_data(seed):
    sig = synth.sigma_powerlaw(F_MIN + DF * np.arange(N_F))
    return synth.noise_map(N_T, N_F, sig, seed), sig


def _noalloc(L, m, n, seed, off, k, out, status, stream):
    return L.stk_score_noalloc(m.handle, n, seed, off, TAU_MAX, k, C.c_void_p(out.data_ptr()),
                               C.c_void_p(status.data_ptr()) if status is not None else None,
                               C.c_void_p(stream.cuda_stream))


def _hits(out):
    return out.cpu().numpy().view(stk.HIT_DTYPE)


def _assert_same_hits(got, ref, what):
    for field in ("snr", "index", "f", "tau"):
        np.testing.assert_array_equal(got[field], ref[field], err_msg=f"{what}: {field}")
    assert np.all(got["reserved"] == 0), what


def _assert_invalid(got, what):
    assert np.all(np.isnan(got["snr"])), what
    assert np.all(got["index"] == np.iinfo(np.uint64).max), what


@pytest.fixture(scope="module")
def L():
    from paper_1401_8060_b300 import build
    build.build()
    return _lib.lib()


def test_noalloc_matches_stk_score_twice(L):
    ctx = stk.Context(0)
    y, sig = _map_data(99)
    m = ctx.load_map(torch.from_numpy(y).cuda(), torch.from_numpy(sig).cuda(), F_MIN, DF)
    om = oracle.OracleMap(y, sig, F_MIN, DF, True)
    k = 256
    stream = torch.cuda.current_stream()
    out = torch.zeros(k * 40, dtype=torch.uint8, device="cuda")
    status = torch.full((1,), -99, dtype=torch.int32, device="cuda")
    calls = [(600_000, 3, 0), (_lib.STK_NOALLOC_MAX_TRACKS, 8, 123_456)]   # (n_tracks, seed, offset)
    for i, (n, seed, off) in enumerate(calls):
        ctx.set_tracks(n, seed, off, TAU_MAX)
        ref = ctx.score(m, k)                        # the existing, allocating entry point
        out.fill_(0)
        status.fill_(-99)
        torch.cuda.synchronize()
        free_before, reserved_before = torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()
        rc = _noalloc(L, m, n, seed, off, k, out, status, stream)
        assert rc == _lib.STK_OK, L.stk_last_error(None).decode()
        torch.cuda.synchronize()
        if i == 1:   # the steady-state call: the array's address is resolved already
            assert torch.cuda.mem_get_info()[0] == free_before
            assert torch.cuda.memory_reserved() == reserved_before
        assert int(status.item()) == _lib.STK_OK
        got = _hits(out)
        _assert_same_hits(got, ref, f"call {i}")
        g = int(got["index"][0])                     # the loudest, against the FP64 oracle
        o = om.score_range(seed, g, 1, TAU_MAX)[0]
        assert abs(got["snr"][0] - o) <= RTOL * abs(o), (got["snr"][0], o)

    # beyond the fixed scratch: refused with a clear message, nothing launched
    rc = L.stk_score_noalloc(m.handle, _lib.STK_NOALLOC_MAX_TRACKS + 1, 1, 0, TAU_MAX, k,
                             C.c_void_p(out.data_ptr()), None, C.c_void_p(stream.cuda_stream))
    assert rc == _lib.STK_EINVAL
    assert b"limit" in L.stk_last_error(None)
    rc = L.stk_score_noalloc(m.handle, 1000, 1, 0, TAU_MAX, 1001, C.c_void_p(out.data_ptr()), None,
                             C.c_void_p(stream.cuda_stream))
    assert rc == _lib.STK_EINVAL
    m.close()
    ctx.close()


def test_noalloc_waits_for_a_map_update_on_the_context_stream(L):
    ctx_stream, other = torch.cuda.Stream(), torch.cuda.Stream()
    ctx = stk.Context(0, stream=ctx_stream)
    y0, sig = _map_data(5)
    y1, _ = _map_data(6)
    y0d, y1d, sd = (torch.from_numpy(a).cuda() for a in (y0, y1, sig))
    torch.cuda.synchronize()
    m = ctx.load_map(y0d, sd, F_MIN, DF)
    n, seed, k = 300_000, 11, 64
    out = torch.zeros(k * 40, dtype=torch.uint8, device="cuda")
    status = torch.full((1,), -99, dtype=torch.int32, device="cuda")
    ctx.set_tracks(n, seed, 0, TAU_MAX)
    ctx.update_map(m, y1d, sd)          # packs on the context's stream and returns at once
    rc = _noalloc(L, m, n, seed, 0, k, out, status, other)   # issued on the other stream right away
    assert rc == _lib.STK_OK, L.stk_last_error(None).decode()
    torch.cuda.synchronize()
    assert int(status.item()) == _lib.STK_OK
    ref = ctx.score(m, k)               # the updated map, on the context's stream
    _assert_same_hits(_hits(out), ref, "after stk_update_map")
    m.close()
    ctx.close()


def test_noalloc_marks_hits_invalid_on_timeout_and_bad_data(L):
    ctx = stk.Context(0)
    y, sig = _map_data(7)
    yd, sd = torch.from_numpy(y).cuda(), torch.from_numpy(sig).cuda()
    m = ctx.load_map(yd, sd, F_MIN, DF)
    n, seed, k = 200_000, 4, 32
    stream = torch.cuda.current_stream()
    out = torch.zeros(k * 40, dtype=torch.uint8, device="cuda")
    status = torch.full((1,), -99, dtype=torch.int32, device="cuda")
    ctx.set_tracks(n, seed, 0, TAU_MAX)
    ref = ctx.score(m, k)

    # a slab copy that never comes: the first CTA's bounded wait gives up after 50 ms
    ctx.set_option(_lib.STK_OPT_KERNEL, 2)
    ctx.set_option(_lib.STK_OPT_WAIT_MS, 50)
    ctx.set_option(_lib.STK_OPT_WITHHOLD_SLAB, 0)
    for with_status in (True, False):
        out.fill_(0)
        status.fill_(-99)
        rc = _noalloc(L, m, n, seed, 0, k, out, status if with_status else None, stream)
        assert rc == _lib.STK_OK, L.stk_last_error(None).decode()
        torch.cuda.synchronize()
        _assert_invalid(_hits(out), f"timeout, status word given: {with_status}")
        assert int(status.item()) == (_lib.STK_ETIMEOUT if with_status else -99)
    ctx.set_option(_lib.STK_OPT_WITHHOLD_SLAB, -1)
    assert _noalloc(L, m, n, seed, 0, k, out, status, stream) == _lib.STK_OK
    torch.cuda.synchronize()
    assert int(status.item()) == _lib.STK_OK
    _assert_same_hits(_hits(out), ref, "after the timeout")

    # bad data packed by a deferred stk_update_map: reported here, and by stk_sync
    bad = y.copy()
    bad[3, 17] = np.nan
    ctx.update_map(m, torch.from_numpy(bad).cuda(), sd)
    assert _noalloc(L, m, n, seed, 0, k, out, status, stream) == _lib.STK_OK
    torch.cuda.synchronize()
    assert int(status.item()) == _lib.STK_EINVAL
    _assert_invalid(_hits(out), "bad map data")
    with pytest.raises(stk.StkError):
        ctx.sync()                       # reads and clears the deferred error
    ctx.update_map(m, yd, sd)
    assert _noalloc(L, m, n, seed, 0, k, out, status, stream) == _lib.STK_OK
    torch.cuda.synchronize()
    assert int(status.item()) == _lib.STK_OK
    _assert_same_hits(_hits(out), ref, "after the good data again")
    m.close()
    ctx.close()
