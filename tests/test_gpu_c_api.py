"""The C ABI used from plain C on the GPU: a C99 program (gcc, linked only
against libstk.so) creates a context, loads a map from host memory, scores a
template range and writes its k loudest; they must equal the Python binding's
hits for the same map and range bit for bit, and the oracle's."""
import os
import subprocess

import numpy as np
import pytest

from _parity import assert_topk_matches

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle  # noqa: E402
import paper_1401_8060_b300 as stk  # noqa: E402
from paper_1401_8060_b300 import synth  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

C_PROGRAM = r"""
#include <stdio.h>
#include <stdlib.h>
#include "stk.h"

/* usage: prog map.bin sigma.bin n_t n_f n_tracks seed k out.bin */
int main(int argc, char **argv)
{
    if (argc != 9) return 64;
    const int n_t = atoi(argv[3]), n_f = atoi(argv[4]), k = atoi(argv[7]);
    const unsigned long long T = strtoull(argv[5], NULL, 10), seed = strtoull(argv[6], NULL, 10);
    float *y = malloc(sizeof(float) * 2 * (size_t)n_t * n_f), *sigma = malloc(sizeof(float) * n_f);
    stk_hit *hits = malloc(sizeof(stk_hit) * k);
    FILE *f = fopen(argv[1], "rb");
    if (!f || fread(y, sizeof(float), 2 * (size_t)n_t * n_f, f) != 2 * (size_t)n_t * n_f) return 65;
    fclose(f);
    f = fopen(argv[2], "rb");
    if (!f || fread(sigma, sizeof(float), n_f, f) != (size_t)n_f) return 66;
    fclose(f);
    stk_ctx *ctx = NULL;
    stk_map *map = NULL;
    int rc = stk_create(&ctx, 0, NULL);
    if (rc) { fprintf(stderr, "create: %s\n", stk_last_error(NULL)); return 67; }
    rc = stk_load_map(ctx, y, sigma, n_t, n_f, 40.0, 0.5, STK_HOST_PTR | STK_SIGMA_PER_FREQ, &map);
    if (!rc) rc = stk_set_tracks(ctx, T, seed, 0, 0.01);
    if (!rc) rc = stk_score(ctx, map, k, hits, STK_OUT_HOST);
    if (rc) { fprintf(stderr, "stk: %d %s\n", rc, stk_last_error(ctx)); return 68; }
    f = fopen(argv[8], "wb");
    fwrite(hits, sizeof(stk_hit), k, f);
    fclose(f);
    stk_free_map(map);
    stk_destroy(ctx);
    free(y); free(sigma); free(hits);
    return 0;
}
"""


def test_c_program_scores_like_the_binding(tmp_path):
    from paper_1401_8060_b300 import build
    lib = build.build()
    src, exe = tmp_path / "score.c", tmp_path / "score"
    src.write_text(C_PROGRAM)
    libdir = os.path.dirname(lib)
    subprocess.run(["gcc", "-std=c99", "-O2", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                    "-L", libdir, "-lstk", "-Wl,-rpath," + libdir, "-o", str(exe)], check=True)
    n_t, n_f, T, seed, k = 60, 300, 200_000, 17, 64
    sig = synth.sigma_powerlaw(40.0 + 0.5 * np.arange(n_f), 1.2)
    y = synth.noise_map(n_t, n_f, sig, 71)
    (tmp_path / "y.bin").write_bytes(np.ascontiguousarray(y).tobytes())
    (tmp_path / "s.bin").write_bytes(np.ascontiguousarray(sig).tobytes())
    out = tmp_path / "hits.bin"
    run = subprocess.run([str(exe), str(tmp_path / "y.bin"), str(tmp_path / "s.bin"), str(n_t), str(n_f), str(T),
                          str(seed), str(k), str(out)], capture_output=True, text=True)
    assert run.returncode == 0, (run.returncode, run.stderr)
    c_hits = np.frombuffer(out.read_bytes(), dtype=stk.HIT_DTYPE)
    ctx = stk.Context(0)
    m = ctx.load_map(torch.from_numpy(y).cuda(), torch.from_numpy(sig).cuda(), 40.0, 0.5)
    ctx.set_tracks(T, seed, 0, 0.01)
    np.testing.assert_array_equal(c_hits, ctx.score(m, k))
    o = oracle.OracleMap(y, sig, 40.0, 0.5, True).score_range(seed, 0, T, 0.01)
    assert_topk_matches(c_hits, o, 0, k, what="C program")
    m.close()
    ctx.close()
