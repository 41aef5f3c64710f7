"""FP16 pixel storage (|y|/sigma in FP16, phase in Q0.16 turns, FP32 sums) vs the FP64 oracle.

Bound, from the storage alone: FP16 rounding of |y|/sigma is at most 2^-12
relative and the Q0.16 phase at most 2^-17 turns (4.8e-5 rad), so each pixel's
term moves by at most 2.9e-4 |z_j| and
    |SNR_fp16 - SNR_oracle| <= 3.5e-4 * sum_j |z_j| / norm + 1e-5 |SNR|.
The observed error (RMS and maximum, relative to that scale) is printed.
"""
import numpy as np
import pytest

from _parity import scale

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle  # noqa: E402
import paper_1401_8060_b300 as stk  # noqa: E402
from paper_1401_8060_b300 import _lib, synth  # noqa: E402

RTOL16 = 3.5e-4


@pytest.fixture(scope="module")
def ctx():
    from paper_1401_8060_b300 import build
    build.build()
    c = stk.Context(0)
    yield c
    c.close()


def _params(seed, off, n, n_f, tmax):
    f3, tau = zip(*[oracle.track_params(seed, off + i, n_f, tmax) for i in range(n)])
    return np.array(f3, np.uint32), np.array(tau)


def _check(g, o, ex, paper, n_t, what):
    sc = scale(ex, paper, n_t)
    err = np.abs(g - o)
    bound = RTOL16 * sc + 1e-5 * np.abs(o)
    assert np.all(err <= bound), f"{what}: max err/scale {np.max(err / sc):.3g}"
    return float(np.sqrt(np.mean((err / sc) ** 2))), float(np.max(err / sc))


@pytest.mark.parametrize("mode,paper", [("freq", False), ("pixel", False), ("const", False), ("pixel", True)])
@pytest.mark.parametrize("kernel", [1, 2])
def test_fp16_matches_oracle(ctx, mode, paper, kernel):
    n_t, n_f, T, seed, off, tmax = 53, 301, 15013, 7, 55, 0.01
    rng = np.random.default_rng(70)
    if mode == "pixel":
        sig = rng.uniform(0.4, 2.5, (n_t, n_f)).astype(np.float32)
    elif mode == "freq":
        sig = synth.sigma_powerlaw(40.0 + 0.5 * np.arange(n_f), 1.3)
    else:
        sig = np.full(n_f, 1.7, np.float32)
    y = synth.noise_map(n_t, n_f, sig, 71)
    m = ctx.load_map(torch.from_numpy(y).cuda(), torch.from_numpy(sig).cuda(), 40.0, 0.5, paper_mode=paper, fp16=True)
    om = oracle.OracleMap(y, sig, 40.0, 0.5, sig.ndim == 1, paper_mode=paper)
    ctx.set_option(_lib.STK_OPT_KERNEL, kernel)
    ctx.set_option(_lib.STK_OPT_SMEM_KB, 20)
    try:
        ctx.set_tracks(T, seed, off, tmax)
        g = ctx.score_all(m).cpu().numpy()
        assert ctx.last_plan()["kernel"] == kernel
    finally:
        ctx.set_option(_lib.STK_OPT_KERNEL, 0)
        ctx.set_option(_lib.STK_OPT_SMEM_KB, 0)
    f3, tau = _params(seed, off, T, n_f, tmax)
    o, ex = om.score_explicit(f3, tau, extras=True)
    rms, mx = _check(g, o, ex, paper, n_t, f"fp16 {mode} paper={paper} kernel={kernel}")
    print(f"fp16 {mode} paper={paper}: error / scale rms {rms:.2e} max {mx:.2e}")


def test_fp16_kernels_agree_bitwise(ctx):
    n_t, n_f, T = 70, 400, 12000
    sig = synth.sigma_powerlaw(40.0 + 0.5 * np.arange(n_f))
    y = synth.noise_map(n_t, n_f, sig, 72)
    m = ctx.load_map(torch.from_numpy(y).cuda(), torch.from_numpy(sig).cuda(), 40.0, 0.5, fp16=True)
    ctx.set_tracks(T, 2, 0, 0.01)
    res = []
    for kernel in (1, 2):
        ctx.set_option(_lib.STK_OPT_KERNEL, kernel)
        res.append(ctx.score_all(m).cpu().numpy())
    ctx.set_option(_lib.STK_OPT_KERNEL, 0)
    f3, tau = _params(2, 0, T, n_f, 0.01)
    res.append(ctx.score_explicit(m, torch.from_numpy(f3.astype(np.int32)), torch.from_numpy(tau)).cpu().numpy())
    np.testing.assert_array_equal(res[1], res[0])
    np.testing.assert_array_equal(res[2], res[0])


def test_fp16_realistic_topk_vs_fp32(ctx):
    """Realistic map, 10^6 templates: FP16 and FP32 storage select nearly the same
    loudest templates; every FP16 top-k SNR is within the bound of its FP64 value."""
    w = synth.WORKLOADS["realistic"]
    fm = synth.realistic_map()
    yt, st = torch.from_numpy(fm.y).cuda(), torch.from_numpy(fm.sigma).cuda()
    m32 = ctx.load_map(yt, st, fm.f_min, fm.df)
    m16 = ctx.load_map(yt, st, fm.f_min, fm.df, fp16=True)
    T, k = 1_000_000, 256
    ctx.set_tracks(T, w["seed"], 0, w["tau_max"])
    h32 = ctx.score(m32, k)
    h16 = ctx.score(m16, k)
    overlap = len(set(h32["index"].tolist()) & set(h16["index"].tolist())) / k
    assert overlap > 0.9, overlap
    om = oracle.OracleMap.from_ftmap(fm)
    o, ex = om.score_explicit(np.array([list(f) for f in h16["f"]], np.uint32), h16["tau"], extras=True)
    rms, mx = _check(h16["snr"], o, ex, False, fm.n_t, "fp16 realistic top-k")
    print(f"fp16 realistic top-{k}: overlap with FP32 {overlap:.3f}; error / scale rms {rms:.2e} max {mx:.2e}")


def test_fp16_range_rejected(ctx):
    y = np.full((4, 8), 1e5 + 0j, np.complex64)
    with pytest.raises(stk.StkError) as e:
        ctx.load_map(y, np.ones(8, np.float32), 40.0, 0.5, fp16=True)
    assert e.value.code == _lib.STK_EINVAL
