"""CPU checks of the C-ABI boundary: the library builds, loads and exports
every entry point include/stk.h declares; no GPU compute is called."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "stk.h")


def header_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^STK_API\s+[\w\s\*]*?\b(stk_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def built():
    from paper_1401_8060_b300 import build
    return build.build()


def test_header_declares_calls():
    names = header_functions()
    for needed in ["stk_create", "stk_destroy", "stk_load_map", "stk_free_map", "stk_set_tracks", "stk_score",
                   "stk_score_all", "stk_track_params", "stk_score_explicit", "stk_last_error", "stk_sync"]:
        assert needed in names
    # plain C: no torch or C++ types in the signatures
    text = open(HEADER).read()
    assert "torch" not in text.lower().replace("pytorch", "") and "std::" not in text


def test_library_exports_every_header_symbol(built):
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s+(stk_\w+)", out))
    missing = [n for n in header_functions() if n not in exported]
    assert not missing, missing
    # and nothing else of ours leaks out
    assert exported == set(header_functions())


def test_binding_declares_every_symbol(built):
    from paper_1401_8060_b300 import _lib
    assert sorted(n for n, _, _ in _lib.SIGNATURES) == header_functions()
    L = _lib.lib()
    for n in header_functions():
        assert getattr(L, n) is not None
    assert L.stk_version() >= 100


def test_hit_layout_matches_header(built):
    from paper_1401_8060_b300 import HIT_DTYPE
    assert HIT_DTYPE.itemsize == 40
    assert [HIT_DTYPE.fields[k][1] for k in ("snr", "index", "f", "reserved", "tau")] == [0, 8, 16, 28, 32]


def test_null_arguments_rejected_without_gpu(built):
    from paper_1401_8060_b300 import _lib
    L = _lib.lib()
    assert L.stk_create(None, 0, None) == _lib.STK_EINVAL
    assert L.stk_set_tracks(None, 1, 0, 0, 0.0) == _lib.STK_EINVAL
    assert L.stk_score(None, None, 1, None, 0) == _lib.STK_EINVAL
    assert L.stk_sync(None) == _lib.STK_EINVAL
    assert L.stk_refine(None, None, None, None, 1, 1, 0.1, 0.1, 1.0, None) == _lib.STK_EINVAL
    assert L.stk_interp_forward(None, None, None, None, 1, None) == _lib.STK_EINVAL
    L.stk_destroy(None)
    L.stk_free_map(None)
    assert isinstance(L.stk_last_error(None), bytes)


def test_no_oracle_on_product_path():
    """The package never imports the oracle (the oracle is test infrastructure)."""
    pkg = os.path.join(ROOT, "paper_1401_8060_b300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle", text, flags=re.M), f
                assert "stk_oracle" not in text and "liboracle" not in text, f


C_PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "stk.h"

int main(void)
{
    /* the boundary is plain C: these calls need no GPU and must reject bad arguments */
    stk_hit h;
    if (sizeof(h) != 40) return 1;
    if (stk_create(NULL, 0, NULL) != STK_EINVAL) return 2;
    if (stk_set_tracks(NULL, 1, 0, 0, 0.0) != STK_EINVAL) return 3;
    if (stk_score(NULL, NULL, 1, NULL, 0) != STK_EINVAL) return 4;
    if (stk_sync(NULL) != STK_EINVAL) return 5;
    stk_destroy(NULL);
    stk_free_map(NULL);
    const char *msg = stk_last_error(NULL);
    if (msg == NULL) return 6;
    if (stk_version() < 100) return 7;
    printf("ok %d\n", stk_version());
    return 0;
}
"""


def test_header_compiles_as_c_and_links(built, tmp_path):
    """A C99 program (gcc, no C++) includes include/stk.h, links libstk.so and
    calls the argument checks of the ABI."""
    src = tmp_path / "use_stk.c"
    exe = tmp_path / "use_stk"
    src.write_text(C_PROGRAM)
    libdir = os.path.dirname(built)
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-L",
                    libdir, "-lstk", "-Wl,-rpath," + libdir, "-o", str(exe)], check=True)
    run = subprocess.run([str(exe)], capture_output=True, text=True)
    assert run.returncode == 0, (run.returncode, run.stdout, run.stderr)
    assert run.stdout.startswith("ok ")
