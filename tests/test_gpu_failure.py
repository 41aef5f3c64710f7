"""Failure detection without a GPU fault: every in-kernel wait is bounded.

A test option makes the first CTA withhold one slab copy (a barrier nothing
completes).  The kernel's wait must give up after the configured limit, let the
copies it did issue land, report STK_ETIMEOUT, and leave the context usable:
the next call gives the same result as before the failure.
"""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1401_8060_b300 as stk  # noqa: E402
from paper_1401_8060_b300 import _lib, synth  # noqa: E402


def test_withheld_slab_times_out_and_context_survives():
    from paper_1401_8060_b300 import build
    build.build()
    ctx = stk.Context(0)
    n_t, n_f = 64, 300
    sig = synth.sigma_powerlaw(40.0 + 0.5 * np.arange(n_f))
    y = synth.noise_map(n_t, n_f, sig, 5)
    m = ctx.load_map(torch.from_numpy(y).cuda(), torch.from_numpy(sig).cuda(), 40.0, 0.5)
    ctx.set_tracks(400_000, 1, 0, 0.01)
    ctx.set_option(_lib.STK_OPT_KERNEL, 2)
    ctx.set_option(_lib.STK_OPT_SMEM_KB, 40)            # several slabs per batch
    ref = ctx.score(m, 8)
    assert ctx.last_plan()["kernel"] == 2
    ctx.set_option(_lib.STK_OPT_WAIT_MS, 50)
    ctx.set_option(_lib.STK_OPT_WITHHOLD_SLAB, 3)
    t0 = time.perf_counter()
    with pytest.raises(stk.StkError) as e:
        ctx.score(m, 8)
    elapsed = time.perf_counter() - t0
    assert e.value.code == _lib.STK_ETIMEOUT
    assert elapsed < 5.0                                 # bounded: two 50 ms waits, not a hang
    ctx.set_option(_lib.STK_OPT_WITHHOLD_SLAB, -1)
    ctx.set_option(_lib.STK_OPT_WAIT_MS, 0)
    np.testing.assert_array_equal(ctx.score(m, 8), ref)  # the context is still usable
    ctx.set_option(_lib.STK_OPT_KERNEL, 0)
    ctx.set_option(_lib.STK_OPT_SMEM_KB, 0)
    m.close()
    ctx.close()
