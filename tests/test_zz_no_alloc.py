"""stk_score_noalloc: scoring for callers that cannot allocate device memory.

Callers whose device memory is owned by another allocator, or that cannot take
cudaFree's synchronisation in a hot loop, score through stk_score_noalloc,
whose scratch is a fixed device array inside the library.  This file checks,
through the C ABI, that two calls in a row give what stk_score gives (within
the tolerance the other parity tests use), that the steady-state call does not
change the device's free memory, and that ranges beyond the fixed scratch are
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

import paper_1401_8060_b300 as stk  # noqa: E402
from paper_1401_8060_b300 import _lib, synth  # noqa: E402


def _same_selection(got, ref, what):
    np.testing.assert_allclose(got["snr"], ref["snr"], rtol=RTOL, atol=0, err_msg=what)
    for i in np.nonzero(got["index"] != ref["index"])[0]:   # only near-ties may swap
        assert abs(got["snr"][i] - ref["snr"][i]) <= 2 * RTOL * abs(ref["snr"][i]), what
    assert np.all(got["reserved"] == 0)


def test_noalloc_matches_stk_score_twice():
    from paper_1401_8060_b300 import build
    build.build()
    L = _lib.lib()
    ctx = stk.Context(0)
    n_t, n_f = 240, 900
    sig = synth.sigma_powerlaw(40.0 + 0.5 * np.arange(n_f))
    y = synth.noise_map(n_t, n_f, sig, 99)
    m = ctx.load_map(torch.from_numpy(y).cuda(), torch.from_numpy(sig).cuda(), 40.0, 0.5)
    k = 256
    stream = torch.cuda.current_stream()
    out = torch.zeros(k * 40, dtype=torch.uint8, device="cuda")
    status = torch.full((1,), -99, dtype=torch.int32, device="cuda")
    calls = [(600_000, 3, 0), (_lib.STK_NOALLOC_MAX_TRACKS, 8, 123_456)]   # (n_tracks, seed, offset)
    free_before = free_after = None
    for i, (n, seed, off) in enumerate(calls):
        ctx.set_tracks(n, seed, off, 0.010)
        ref = ctx.score(m, k)                        # the existing, allocating entry point
        out.fill_(0)
        status.fill_(-99)
        torch.cuda.synchronize()
        if i == 1:
            free_before = torch.cuda.mem_get_info()[0]
        rc = L.stk_score_noalloc(m.handle, n, seed, off, 0.010, k, C.c_void_p(out.data_ptr()),
                                 C.c_void_p(status.data_ptr()), C.c_void_p(stream.cuda_stream))
        assert rc == _lib.STK_OK, L.stk_last_error(None).decode()
        torch.cuda.synchronize()
        if i == 1:
            free_after = torch.cuda.mem_get_info()[0]
        assert int(status.item()) == _lib.STK_OK
        got = out.cpu().numpy().view(stk.HIT_DTYPE)
        _same_selection(got, ref, f"call {i}")
    assert free_after == free_before   # nothing allocated by the steady-state call

    # beyond the fixed scratch: refused with a clear message, nothing launched
    rc = L.stk_score_noalloc(m.handle, _lib.STK_NOALLOC_MAX_TRACKS + 1, 1, 0, 0.01, k,
                             C.c_void_p(out.data_ptr()), None, C.c_void_p(stream.cuda_stream))
    assert rc == _lib.STK_EINVAL
    assert b"limit" in L.stk_last_error(None)
    rc = L.stk_score_noalloc(m.handle, 1000, 1, 0, 0.01, 1001, C.c_void_p(out.data_ptr()), None,
                             C.c_void_p(stream.cuda_stream))
    assert rc == _lib.STK_EINVAL
    m.close()
    ctx.close()
