"""The bounds-checked debug build (libstk_debug.so, compiled with STK_DEBUG_BOUNDS).

With no memory checker available, the debug build stands in for one: every
pixel gather checks its column and its bin against the template's convex hull
of control bins within the map (Eq. 7's pixel set: the Bezier curve of Sec. III
lies inside that hull) and reports STK_EBOUNDS instead of reading outside; the
packed map and the context's scratch end in canary words, checked after every
call.  Here every scoring path (slab and one-thread kernels, explicit and
general templates, interpolation, refinement, polish, batches) runs on small
maps of each weighting and precision in a subprocess on the debug build: every
call succeeds (no out-of-range gather, no damaged canary), and the results equal
the release build's bit for bit (the checks change no arithmetic).
"""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

HERE = os.path.dirname(os.path.abspath(__file__))


def test_debug_build_clean_and_identical(tmp_path):
    from paper_1401_8060_b300 import build
    build.build()
    assert os.path.exists(build.DEBUG_LIB)
    out = str(tmp_path / "debug.npz")
    env = dict(os.environ, STK_LIBRARY=build.DEBUG_LIB)
    run = subprocess.run([sys.executable, os.path.join(HERE, "_debug_worker.py"), out], env=env,
                         capture_output=True, text=True, timeout=600)
    assert run.returncode == 0, run.stdout[-2000:] + run.stderr[-4000:]
    dbg = dict(np.load(out))
    assert int(dbg["build_flags"][0]) == 1
    sys.path.insert(0, HERE)
    import _debug_worker
    rel = _debug_worker.run_all()
    assert int(rel["build_flags"][0]) == 0
    assert set(dbg) == set(rel)
    for key in sorted(rel):
        if key != "build_flags":
            np.testing.assert_array_equal(dbg[key], rel[key], err_msg=key)
