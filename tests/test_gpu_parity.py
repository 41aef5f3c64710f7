"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bit-exact: template parameters and pixel bins.  Floating point: the per-template
SNR bound of tests/_parity.py (1e-5 relative to the pixel-magnitude scale) and
plain relative 1e-5 on selected top-k values; winning indices equal unless the
oracle's own SNRs are closer than that.
"""
import numpy as np
import pytest

from _parity import RTOL, assert_snr_close, assert_topk_matches

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


def rand_map(seed, n_t, n_f, mode):
    """mode: 'pixel' (sigma per pixel), 'freq' (per frequency), 'const' (sigma = 1.7 everywhere)."""
    rng = np.random.default_rng(seed)
    if mode == "pixel":
        sig = rng.uniform(0.4, 2.5, (n_t, n_f)).astype(np.float32)
    elif mode == "freq":
        sig = synth.sigma_powerlaw(40.0 + 0.5 * np.arange(n_f), 1.3)
    else:
        sig = np.full(n_f, 1.7, np.float32)
    y = synth.noise_map(n_t, n_f, sig, int(rng.integers(1 << 30)))
    return y, sig


def load_both(ctx, y, sig, f_min, df, paper=False, host=False):
    per_freq = sig.ndim == 1
    if host:
        m = ctx.load_map(y, sig, f_min, df, paper_mode=paper)
    else:
        m = ctx.load_map(torch.from_numpy(y).cuda(), torch.from_numpy(sig).cuda(), f_min, df, paper_mode=paper)
    om = oracle.OracleMap(y, sig, f_min, df, per_freq, paper_mode=paper)
    return m, om


def oracle_params(seed, offset, n, n_f, tau_max):
    f3, tau = zip(*[oracle.track_params(seed, offset + i, n_f, tau_max) for i in range(n)])
    return np.array(f3, dtype=np.uint32), np.array(tau)


# ------------------------------------------------------------------ bit-exact pieces
@pytest.mark.parametrize("n_t,n_f", [(200, 100), (500, 1600), (1000, 2000), (1000, 2200), (2, 1), (3, 7)])
def test_track_params_and_bins_bit_exact(ctx, n_t, n_f):
    y = np.zeros((n_t, n_f), np.complex64)
    m = ctx.load_map(torch.from_numpy(y).cuda(), torch.ones(n_f, device="cuda"), 10.0, 1.0)
    ctx.set_tracks(1, seed=12345, offset=0, tau_max=0.01)
    for g in [0, 1, 7, 99991, 2 ** 33 + 5, 2 ** 64 - 1]:
        f, tau, bins = ctx.track_params(m, g)
        fo, tauo = oracle.track_params(12345, g, n_f, 0.01)
        assert f == fo and tau == tauo, (g, f, fo, tau, tauo)
        np.testing.assert_array_equal(bins, oracle.track_bins(fo, n_t))


@pytest.mark.parametrize("mode", ["pixel", "freq", "const"])
@pytest.mark.parametrize("paper", [False, True])
def test_explicit_bruteforce_tiny(ctx, mode, paper):
    """Every template (f0, f1, f2) on a 5 x 6 map, at several delays."""
    n_t, n_f = 5, 6
    y, sig = rand_map(3, n_t, n_f, mode)
    m, om = load_both(ctx, y, sig, 100.0, 1.0, paper)
    trip = np.array([(a, b, c) for a in range(n_f) for b in range(n_f) for c in range(n_f)], np.uint32)
    for tau in [-0.0099, -0.003, 0.0, 0.0021, 0.0099]:
        taus = np.full(len(trip), tau)
        g = ctx.score_explicit(m, torch.from_numpy(trip.astype(np.int32)), torch.from_numpy(taus)).cpu().numpy()
        o, ex = om.score_explicit(trip, taus, extras=True)
        assert_snr_close(g, o, ex, paper, n_t, what=f"explicit {mode} paper={paper} tau={tau}")
    ctx.sync()


# ------------------------------------------------------------------ full scoring, both kernels
@pytest.mark.parametrize("kernel", [1, 2])
@pytest.mark.parametrize("mode,paper", [("pixel", False), ("freq", False), ("const", False), ("pixel", True)])
def test_score_all_matches_oracle(ctx, kernel, mode, paper):
    """Sizes that span several template batches and time slabs with ragged tails."""
    n_t, n_f, T, seed, off, tmax = 37, 203, 20011, 5, 1000, 0.01
    y, sig = rand_map(10 + kernel, n_t, n_f, mode)
    m, om = load_both(ctx, y, sig, 40.0, 0.5, paper)
    ctx.set_option(_lib.STK_OPT_KERNEL, kernel)
    ctx.set_option(_lib.STK_OPT_SMEM_KB, 24)   # small budget: several slabs per map
    try:
        ctx.set_tracks(T, seed, off, tmax)
        g = ctx.score_all(m).cpu().numpy()
        plan = ctx.last_plan()
        assert plan["kernel"] == kernel
        if kernel == 2:
            assert plan["S"] < n_t and plan["nbatches"] > 1
    finally:
        ctx.set_option(_lib.STK_OPT_KERNEL, 0)
        ctx.set_option(_lib.STK_OPT_SMEM_KB, 0)
    ctx.sync()
    f3, tau = oracle_params(seed, off, T, n_f, tmax)
    o, ex = om.score_explicit(f3, tau, extras=True)
    np.testing.assert_array_equal(o, om.score_range(seed, off, T, tmax))
    assert_snr_close(g, o, ex, paper, n_t, what=f"score_all kernel={kernel} {mode}")


def test_wide_rasteriser_map(ctx):
    """A map whose Bezier numerators exceed 32 bits (1000 x 2200): the 64-bit path."""
    n_t, n_f, T = 1000, 2200, 3000
    y, sig = rand_map(23, n_t, n_f, "freq")
    m, om = load_both(ctx, y, sig, 40.0, 0.5)
    ctx.set_tracks(T, 6, 0, 0.01)
    g = ctx.score_all(m).cpu().numpy()
    assert ctx.last_plan()["kernel"] == 1
    f3, tau = oracle_params(6, 0, T, n_f, 0.01)
    o, ex = om.score_explicit(f3, tau, extras=True)
    assert_snr_close(g, o, ex, False, n_t, what="wide map")


def test_kernels_agree_bitwise(ctx):
    """Simple and slab kernels, and explicit scoring, run the same per-template
    arithmetic in the same order: identical doubles."""
    n_t, n_f, T = 61, 517, 9000
    y, sig = rand_map(21, n_t, n_f, "freq")
    m, _ = load_both(ctx, y, sig, 40.0, 0.5)
    ctx.set_tracks(T, 9, 0, 0.01)
    res = []
    for kernel, smem in [(1, 0), (2, 0), (2, 40), (2, 20)]:
        ctx.set_option(_lib.STK_OPT_KERNEL, kernel)
        ctx.set_option(_lib.STK_OPT_SMEM_KB, smem)
        res.append(ctx.score_all(m).cpu().numpy())
    ctx.set_option(_lib.STK_OPT_KERNEL, 0)
    ctx.set_option(_lib.STK_OPT_SMEM_KB, 0)
    f3, tau = oracle_params(9, 0, T, n_f, 0.01)
    res.append(ctx.score_explicit(m, torch.from_numpy(f3.astype(np.int32)), torch.from_numpy(tau)).cpu().numpy())
    for r in res[1:]:
        np.testing.assert_array_equal(r, res[0])


@pytest.mark.parametrize("n_t,n_f,T,prior", [(40, 1, 5000, False), (33, 2, 7001, False), (50, 7, 20000, True),
                                              (64, 128, 30000, False), (64, 129, 30001, True),
                                              (20, 8192, 100003, False), (500, 1600, 200000, False)])
def test_coherent_order_identical(ctx, n_t, n_f, T, prior):
    """The slab kernel scores templates in coherent (Z-order) order by default;
    every template's SNR is bit for bit the one of index order and of the
    one-thread-per-template kernel, and lands at its own index."""
    y, sig = rand_map(23, n_t, n_f, "freq")
    m, om = load_both(ctx, y, sig, 40.0, 0.5)
    if prior:
        ctx.set_tau_prior(np.linspace(-0.004, 0.009, 17))
    ctx.set_tracks(T, 5, 123, 0.01)
    res = {}
    try:
        for kernel, order in [(2, 1), (2, 0), (1, 1)]:
            ctx.set_option(_lib.STK_OPT_KERNEL, kernel)
            ctx.set_option(_lib.STK_OPT_ORDER, order)
            res[(kernel, order)] = ctx.score_all(m).cpu().numpy()
            assert ctx.last_plan()["order"] == (1 if kernel == 2 and order else 0)
    finally:
        ctx.set_option(_lib.STK_OPT_KERNEL, 0)
        ctx.set_option(_lib.STK_OPT_ORDER, 1)
        if prior:
            ctx.set_tau_prior(None)
    np.testing.assert_array_equal(res[(2, 1)], res[(2, 0)])
    np.testing.assert_array_equal(res[(2, 1)], res[(1, 1)])
    # and the values are the oracle's for a sample of indices
    idx = np.random.default_rng(3).choice(T, 200, replace=False)
    if prior:
        pr = [oracle.track_params_prior(5, 123 + int(i), n_f, np.linspace(-0.004, 0.009, 17)) for i in idx]
    else:
        pr = [oracle.track_params(5, 123 + int(i), n_f, 0.01) for i in idx]
    f3 = np.array([p[0] for p in pr], dtype=np.uint32)
    tau = np.array([p[1] for p in pr])
    o, ex = om.score_explicit(f3, tau, extras=True)
    assert_snr_close(res[(2, 1)][idx], o, ex, False, n_t, what="coherent order")


@pytest.mark.parametrize("n_f", [8191, 8192, 8193, 20000])
def test_phase_forms_at_the_narrow_limit(ctx, n_f):
    """Up to 8192 bins the per-pixel phase is a 32-bit turn exact at the centre
    bin; wider maps keep 64 bits (one-thread-per-template kernel).  Both stay
    within the parity bound at the extreme bins, where the narrow form's error
    is largest, with the largest delay."""
    n_t = 24
    y, sig = rand_map(24, n_t, n_f, "freq")
    m, om = load_both(ctx, y, sig, 40.0, 0.5)
    rng = np.random.default_rng(25)
    ends = np.array([0, n_f - 1], dtype=np.uint32)
    f3 = ends[rng.integers(0, 2, (400, 3))]
    f3[:200, 1] = rng.integers(0, n_f, 200)
    tau = rng.choice([-1.0, 1.0], 400) * (0.01 - rng.uniform(0, 1e-6, 400))
    got = ctx.score_explicit(m, torch.from_numpy(f3.astype(np.int32)), torch.from_numpy(tau)).cpu().numpy()
    o, ex = om.score_explicit(f3, tau, extras=True)
    assert_snr_close(got, o, ex, False, n_t, what=f"phase n_f={n_f}")
    ctx.set_tracks(20000, 6, 0, 0.01)
    ctx.set_option(_lib.STK_OPT_KERNEL, 2)
    try:
        a = ctx.score_all(m).cpu().numpy()
        assert ctx.last_plan()["kernel"] == (2 if n_f <= 8192 else 1)
    finally:
        ctx.set_option(_lib.STK_OPT_KERNEL, 0)
    ctx.set_option(_lib.STK_OPT_KERNEL, 1)
    try:
        b = ctx.score_all(m).cpu().numpy()
    finally:
        ctx.set_option(_lib.STK_OPT_KERNEL, 0)
    np.testing.assert_array_equal(a, b)
    f3, tau = oracle_params(6, 0, 300, n_f, 0.01)
    o, ex = om.score_explicit(f3, tau, extras=True)
    assert_snr_close(a[:300], o, ex, False, n_t, what=f"generated n_f={n_f}")


@pytest.mark.parametrize("fp16", [False, True])
def test_angles_beyond_pi(ctx, fp16):
    """A pixel's angle is the template's phase 2 pi T (|T| < 1/2 turn) plus the
    stored angle of z (|arg z| <= pi), summed in FP32 before the cosine, so the
    cosine sees |angle| up to 2 pi, outside the [-pi, pi] range of its documented
    error bound.  Constant-frequency templates whose phase and pixel angles both
    sit in the outer quarter turns put every angle in (pi, 2 pi) or (-2 pi, -pi);
    the SNRs stay within the parity bound of the FP64 oracle (libm cos), and the
    FP32 records well inside it."""
    n_t, n_f, f_min, df = 64, 64, 40.0, 0.5
    rng = np.random.default_rng(31)
    sig = synth.sigma_powerlaw(f_min + df * np.arange(n_f), 1.1)
    side = np.where(np.arange(n_f) < n_f // 2, 1.0, -1.0)          # sign of the angles per bin
    phi = side * rng.uniform(np.pi / 2, np.pi, (n_t, n_f))
    y = (sig * rng.rayleigh(1.0, (n_t, n_f)) * np.exp(1j * phi)).astype(np.complex64)
    m = ctx.load_map(torch.from_numpy(y).cuda(), torch.from_numpy(sig).cuda(), f_min, df, fp16=fp16)
    om = oracle.OracleMap(y, sig, f_min, df, True)
    n = 2000
    b = rng.integers(0, n_f, n).astype(np.uint32)
    f3 = np.repeat(b[:, None], 3, axis=1)
    turns = side[b] * rng.uniform(0.25, 0.5, n)                     # the template's phase at its bin
    tau = turns / (f_min + df * b.astype(np.float64))
    got = ctx.score_explicit(m, torch.from_numpy(f3.astype(np.int32)), torch.from_numpy(tau)).cpu().numpy()
    o, ex = om.score_explicit(f3, tau, extras=True)
    rtol = 3.5e-4 if fp16 else RTOL
    assert_snr_close(got, o, ex, False, n_t, rtol=rtol, what="angles beyond pi")
    if not fp16:
        err = np.max(np.abs(got - o) / (ex["absz"] / np.sqrt(ex["W"])))
        assert err <= 3e-6, err
    m.close()


@pytest.mark.parametrize("threads,max_r,stages", [(64, 1, 2), (96, 3, 3), (1024, 4, 4), (512, 2, 2), (992, 5, 2),
                                                  (512, 11, 2), (448, 12, 3), (160, 7, 4), (480, 6, 2)])
def test_launch_shapes_agree(ctx, threads, max_r, stages):
    n_t, n_f, T = 45, 300, 30001
    y, sig = rand_map(22, n_t, n_f, "pixel")
    m, _ = load_both(ctx, y, sig, 40.0, 0.5)
    ctx.set_tracks(T, 4, 17, 0.01)
    ctx.set_option(_lib.STK_OPT_KERNEL, 1)
    ref = ctx.score_all(m).cpu().numpy()
    ctx.set_option(_lib.STK_OPT_KERNEL, 2)
    ctx.set_option(_lib.STK_OPT_THREADS, threads)
    ctx.set_option(_lib.STK_OPT_MAX_R, max_r)
    ctx.set_option(_lib.STK_OPT_STAGES, stages)
    ctx.set_option(_lib.STK_OPT_SMEM_KB, 30)
    try:
        got = ctx.score_all(m).cpu().numpy()
        plan = ctx.last_plan()
        assert plan["kernel"] == 2 and plan["threads"] == threads and plan["R"] <= max_r
    finally:
        for o, v in [(_lib.STK_OPT_KERNEL, 0), (_lib.STK_OPT_THREADS, 0), (_lib.STK_OPT_MAX_R, 12),
                     (_lib.STK_OPT_STAGES, 2), (_lib.STK_OPT_SMEM_KB, 0)]:
            ctx.set_option(o, v)
    np.testing.assert_array_equal(got, ref)


# ------------------------------------------------------------------ top-k
def test_tiny_workload_topk(ctx):
    """The 200 x 100 workload: 10^4 templates, k = 16, against the full oracle."""
    w = synth.WORKLOADS["tiny"]
    fm = synth.tiny_map()
    m, om = load_both(ctx, fm.y, fm.sigma, fm.f_min, fm.df)
    ctx.set_tracks(w["n_tracks"], w["seed"], 0, w["tau_max"])
    hits = ctx.score(m, w["k"])
    o = om.score_range(w["seed"], 0, w["n_tracks"], w["tau_max"])
    assert_topk_matches(hits, o, 0, w["k"], what="tiny top-k")
    f3, tau = oracle_params(w["seed"], 0, w["n_tracks"], fm.n_f, w["tau_max"])
    for h in hits:  # parameters of each hit are the template's own
        i = int(h["index"])
        assert tuple(int(v) for v in h["f"]) == tuple(int(v) for v in f3[i]) and h["tau"] == tau[i]
    # all SNRs too
    g = ctx.score_all(m).cpu().numpy()
    _, ex = om.score_explicit(f3, tau, extras=True)
    assert_snr_close(g, o, ex, False, fm.n_t, what="tiny all")


@pytest.mark.parametrize("k", [1, 2, 100, 1024, 4096])
def test_topk_sizes_and_device_output(ctx, k):
    n_t, n_f, T = 50, 400, 50000
    y, sig = rand_map(31, n_t, n_f, "freq")
    m, om = load_both(ctx, y, sig, 40.0, 0.5)
    ctx.set_tracks(T, 77, 3, 0.01)
    out = torch.zeros(k * 40, dtype=torch.uint8, device="cuda")
    ctx.score(m, k, out=out)
    ctx.sync()
    hits = out.cpu().numpy().view(stk.HIT_DTYPE)
    o = om.score_range(77, 3, T, 0.01)
    assert_topk_matches(hits, o, 3, k, what=f"k={k}")
    host_hits = ctx.score(m, k)
    np.testing.assert_array_equal(host_hits, hits)


def test_exact_threshold_route(ctx):
    """k small against n / S (here 8 of 4e7): a sampled threshold would admit
    about q n / S ~ 2e4 candidates, so the selection takes its threshold from two
    exact histogram passes; the k loudest are the top of the GPU's own SNR array
    (descending SNR, then ascending index)."""
    n_t, n_f, T, k = 20, 200, 40_000_000, 8
    y, sig = rand_map(81, n_t, n_f, "freq")
    m, _ = load_both(ctx, y, sig, 40.0, 0.5)
    ctx.set_tracks(T, 21, 3, 0.01)
    hits = ctx.score(m, k)
    g = ctx.score_all(m)
    v, i = torch.sort(g, descending=True, stable=True)
    np.testing.assert_array_equal(hits["snr"], v[:k].cpu().numpy())
    np.testing.assert_array_equal(hits["index"], i[:k].cpu().numpy() + 3)
    del g, v, i
    m.close()


def test_split_ranges_merge_exactly(ctx):
    """Sec. V: runs over disjoint template ranges combine by taking the largest."""
    n_t, n_f, T, k = 80, 300, 40000, 64
    y, sig = rand_map(41, n_t, n_f, "pixel")
    m, _ = load_both(ctx, y, sig, 40.0, 0.5)
    ctx.set_tracks(T, 5, 0, 0.01)
    full = ctx.score(m, k)
    parts = []
    for lo, hi in [(0, 12345), (12345, 30000), (30000, T)]:
        ctx.set_tracks(hi - lo, 5, lo, 0.01)
        parts.append(ctx.score(m, k))
    allh = np.concatenate(parts)
    order = np.lexsort((allh["index"], -allh["snr"]))[:k]
    np.testing.assert_array_equal(allh[order], full)


@pytest.mark.parametrize("T,k", [(5000, 10), (20000, 4096), (100000, 100)])
def test_constant_map_ties_take_smallest_index(ctx, T, k):
    """Every template ties: the smallest indices win.  Every template becomes a
    candidate, and the three sizes take the three routes of the final exact
    select (candidates staged in shared memory; too many to stage, read from
    global memory; candidate-buffer overflow, the full SNR array)."""
    n_t, n_f = 20, 30
    y = np.full((n_t, n_f), 1 + 0j, np.complex64)
    m = ctx.load_map(torch.from_numpy(y).cuda(), torch.ones(n_f, device="cuda"), 0.0, 1.0)
    ctx.set_tracks(T, 1, 1000, 0.0)      # tau = 0: every template scores exactly sqrt(n_t)
    hits = ctx.score(m, k)
    np.testing.assert_array_equal(hits["index"], np.arange(1000, 1000 + k))
    assert np.all(hits["snr"] == hits["snr"][0])
    assert abs(hits["snr"][0] - np.sqrt(n_t)) <= 1e-6 * np.sqrt(n_t)


def test_selection_with_many_near_ties(ctx):
    """SNRs rounded to few values (many exact ties across the boundary) vs numpy's ordering."""
    n_t, n_f, T, k = 40, 50, 200000, 3000
    rng = np.random.default_rng(61)
    y = (np.round(rng.standard_normal((n_t, n_f)) * 2) / 2 + 0j).astype(np.complex64)
    m = ctx.load_map(torch.from_numpy(y).cuda(), torch.ones(n_f, device="cuda"), 0.0, 1.0)
    ctx.set_tracks(T, 3, 0, 0.0)
    allg = ctx.score_all(m).cpu().numpy()
    assert np.unique(allg).size < T // 10
    hits = ctx.score(m, k)
    order = np.lexsort((np.arange(T), -allg))[:k]
    np.testing.assert_array_equal(hits["index"], order)
    np.testing.assert_array_equal(hits["snr"], allg[order])


@pytest.mark.parametrize("sample", [1, 2, 64, 49152])
def test_selection_sample_sizes_identical(ctx, sample):
    """The candidate threshold comes from a sample of the SNRs (or, when the
    sample would admit too many candidates, from two exact histogram passes);
    the k loudest do not depend on the sample's size.  With 200 000 templates a
    sample of 1, 2 or 64 keys takes the exact threshold; with 3 000 it takes
    the sampled one at the first templates' own prefix, which may admit fewer
    than k (the final select then runs over every SNR)."""
    n_t, n_f = 50, 400
    y, sig = rand_map(71, n_t, n_f, "freq")
    m, _ = load_both(ctx, y, sig, 40.0, 0.5)
    cases = [(200000, 1024), (3000, 100)]  # more, and fewer, templates than the default sample
    refs = []
    for T, k in cases:
        ctx.set_tracks(T, 13, 5, 0.01)
        ref = ctx.score(m, k)
        allg = ctx.score_all(m).cpu().numpy()
        order = np.lexsort((np.arange(T), -allg))[:k]
        np.testing.assert_array_equal(ref["index"], order + 5)
        np.testing.assert_array_equal(ref["snr"], allg[order])
        refs.append(ref)
    ctx.set_option(_lib.STK_OPT_SELECT_SAMPLE, sample)
    try:
        for (T, k), ref in zip(cases, refs):
            ctx.set_tracks(T, 13, 5, 0.01)
            np.testing.assert_array_equal(ctx.score(m, k), ref)
    finally:
        ctx.set_option(_lib.STK_OPT_SELECT_SAMPLE, 0)
    m.close()


def test_selection_sample_option_range(ctx):
    for bad in (-1, 49153):
        with pytest.raises(stk.StkError):
            ctx.set_option(_lib.STK_OPT_SELECT_SAMPLE, bad)


# ------------------------------------------------------------------ closed forms through the GPU
def test_zero_noise_injection_snr(ctx):
    """Signal on template g's own pixels only, with its own delay: SNR = A sqrt(W)."""
    n_t, n_f = 120, 700
    sig = synth.sigma_powerlaw(40.0 + 0.5 * np.arange(n_f))
    y = np.zeros((n_t, n_f), np.complex64)
    m0 = ctx.load_map(torch.from_numpy(y).cuda(), torch.from_numpy(sig).cuda(), 40.0, 0.5)
    ctx.set_tracks(1, 8, 0, 0.01)
    f, tau, bins = ctx.track_params(m0, 4242)
    A = 3.0
    synth.inject(y, bins, A, tau, 40.0, 0.5)
    m = ctx.load_map(torch.from_numpy(y).cuda(), torch.from_numpy(sig).cuda(), 40.0, 0.5)
    W = float(np.sum(sig.astype(np.float64)[bins] ** -2.0))
    g = ctx.score_explicit(m, torch.tensor([list(f)], dtype=torch.int32), torch.tensor([tau])).cpu().numpy()[0]
    assert g == pytest.approx(A * np.sqrt(W), rel=RTOL)


def test_single_frequency_delay_ratio(ctx):
    """Eq. 3 on the GPU: R = cos(2 pi f dtau) for a constant-frequency signal."""
    n_t, n_f, c = 64, 1000, 440
    tau_s = 0.0012
    y = np.zeros((n_t, n_f), np.complex64)
    y[:, c] = np.complex64(np.exp(-2j * np.pi * c * tau_s))
    m = ctx.load_map(torch.from_numpy(y).cuda(), torch.ones(n_f, device="cuda"), 0.0, 1.0)
    dts = np.array([0.0, -0.004, -0.0005, 0.0001, 0.0007, 0.003])
    g = ctx.score_explicit(m, torch.tensor([[c, c, c]] * len(dts), dtype=torch.int32),
                           torch.from_numpy(tau_s + dts)).cpu().numpy()
    np.testing.assert_allclose(g / g[0], np.cos(2 * np.pi * c * dts), atol=3e-6)


# ------------------------------------------------------------------ host pointers, errors
def test_host_and_device_maps_identical(ctx):
    y, sig = rand_map(51, 33, 77, "pixel")
    mh, _ = load_both(ctx, y, sig, 40.0, 0.5, host=True)
    md, _ = load_both(ctx, y, sig, 40.0, 0.5, host=False)
    ctx.set_tracks(3000, 1, 0, 0.01)
    np.testing.assert_array_equal(ctx.score_all(mh).cpu().numpy(), ctx.score_all(md).cpu().numpy())


@pytest.mark.parametrize("fp16", [False, True])
@pytest.mark.parametrize("host", [False, True])
def test_update_map_equals_fresh_load(ctx, fp16, host):
    """stk_update_map re-packs into the map's buffers.  A constant-weight map is
    re-examined and equals a fresh load bit for bit whatever the new sigma; a
    per-frequency-weighted map keeps its weighting, so it equals a fresh load
    bit for bit when the new sigma also varies, and agrees within the parity
    bound (the oracle's) when the new sigma happens to be constant."""
    n_t, n_f = 64, 150
    dev = (lambda a: a) if host else (lambda a: torch.from_numpy(a).cuda())
    ctx.set_tracks(4000, 3, 0, 0.01)
    f3, tau = oracle_params(3, 0, 300, n_f, 0.01)
    for start in ["freq", "const"]:
        ya, sa = rand_map(61, n_t, n_f, start)
        m = ctx.load_map(dev(ya), dev(sa), 40.0, 0.5, fp16=fp16)
        cls = start                                  # the map's weighting
        for seed, mode in [(62, "const"), (63, "freq"), (64, "const")]:
            yb, sb = rand_map(seed, n_t, n_f, mode)
            ctx.update_map(m, dev(yb), dev(sb))
            if cls == "const":
                cls = mode                           # re-examined; a varying weight stays
            fresh = ctx.load_map(dev(yb), dev(sb), 40.0, 0.5, fp16=fp16)
            a, b = ctx.score_all(m).cpu().numpy(), ctx.score_all(fresh).cpu().numpy()
            fresh.close()
            om = oracle.OracleMap(yb, sb, 40.0, 0.5, True)
            o, ex = om.score_explicit(f3, tau, extras=True)
            if cls == mode:                          # the fresh load's weighting
                np.testing.assert_array_equal(a, b)
            if not fp16:
                assert_snr_close(a[:300], o, ex, False, n_t, what=f"update {start} -> {mode}")
            else:
                sc = ex["absz"] / np.sqrt(ex["W"])
                assert np.all(np.abs(a[:300] - o) <= 3.5e-4 * sc + 1e-5 * np.abs(o))
        if start == "freq":
            with pytest.raises(ValueError):        # a different shape is rejected before any copy
                ctx.update_map(m, dev(np.ones((n_t, n_f + 1), np.complex64)), dev(np.ones(n_f + 1, np.float32)))
        m.close()


def test_pipelined_updates_on_two_streams(ctx):
    """Two maps alternate: each step's data is copied in and packed on a copy
    stream while the other map scores on a compute stream (the end-to-end
    benchmark's pattern); every step's records equal a plain load-and-score."""
    n_t, n_f, T, k = 48, 200, 30000, 8
    ectx = stk.Context(0)                      # follows the current torch stream
    ectx.set_tracks(T, 4, 0, 0.01)
    datas = [rand_map(70 + i, n_t, n_f, "freq") for i in range(6)]
    pins = [(torch.from_numpy(y).pin_memory(), torch.from_numpy(s).pin_memory()) for y, s in datas]
    maps = [ectx.load_map(pins[0][0], pins[0][1], 40.0, 0.5) for _ in range(2)]
    copy_s, comp_s = torch.cuda.Stream(), torch.cuda.Stream()
    outs = [torch.zeros(k * 40, dtype=torch.uint8, device="cuda") for _ in range(len(datas))]
    scored = [None, None]
    for i, (yp, sp) in enumerate(pins):
        j = i % 2
        if scored[j] is not None:
            scored[j].synchronize()
        with torch.cuda.stream(copy_s):
            ectx.update_map(maps[j], yp, sp)
            copied = torch.cuda.Event()
            copied.record(copy_s)
        with torch.cuda.stream(comp_s):
            comp_s.wait_event(copied)
            ectx.score(maps[j], k, out=outs[i])
            scored[j] = torch.cuda.Event()
            scored[j].record(comp_s)
    torch.cuda.synchronize()
    ectx.sync()
    for i, (y, s) in enumerate(datas):
        m = ctx.load_map(y, s, 40.0, 0.5)
        ctx.set_tracks(T, 4, 0, 0.01)
        np.testing.assert_array_equal(outs[i].cpu().numpy().view(stk.HIT_DTYPE), ctx.score(m, k),
                                      err_msg=f"step {i}")
        m.close()
    ectx.close()


def test_update_map_invalid_data_reported(ctx):
    """A weighted map's update does not wait: bad data surfaces at the next
    host-output scoring call; a constant-weight map's update checks at once."""
    n_t, n_f = 40, 90
    y, sig = rand_map(65, n_t, n_f, "freq")
    m = ctx.load_map(y, sig, 40.0, 0.5)
    ctx.set_tracks(2000, 3, 0, 0.01)
    ref = ctx.score(m, 4)
    bad = y.copy()
    bad[7, 11] = np.nan
    ctx.update_map(m, bad, sig)                      # returns at once
    with pytest.raises(stk.StkError) as e:
        ctx.score(m, 4)
    assert e.value.code == _lib.STK_EINVAL
    ctx.update_map(m, y, sig)
    np.testing.assert_array_equal(ctx.score(m, 4), ref)
    m.close()
    yc, sc = rand_map(66, n_t, n_f, "const")
    mc = ctx.load_map(yc, sc, 40.0, 0.5)
    bad = yc.copy()
    bad[3, 4] = np.inf
    with pytest.raises(stk.StkError) as e:
        ctx.update_map(mc, bad, sc)
    assert e.value.code == _lib.STK_EINVAL
    mc.close()


def _notched_map(seed, n_t, n_f, mode):
    """A map with notched pixels (sigma = +inf, NaN data there): whole notched
    lines with per-frequency sigma, lines and scattered pixels with per-pixel sigma."""
    y, sig = rand_map(seed, n_t, n_f, mode)
    rng = np.random.default_rng(seed + 1)
    y, sig = y.copy(), sig.copy()
    lines = rng.choice(n_f, max(1, n_f // 12), replace=False)
    if sig.ndim == 1:
        sig[lines] = np.inf
        y[:, lines] = np.complex64(complex(np.nan, np.nan))
    else:
        notch = rng.random((n_t, n_f)) < 0.05
        notch[:, lines] = True
        sig[notch] = np.inf
        y[notch] = np.complex64(complex(np.nan, np.nan))
    return y, sig


@pytest.mark.parametrize("mode,paper,fp16", [("freq", False, False), ("pixel", False, False), ("pixel", True, False),
                                             ("freq", False, True)])
def test_notched_pixels(ctx, mode, paper, fp16):
    """Notched pixels (sigma = +inf) add nothing: both kernels, generated and
    general templates, against the oracle; a fully notched map scores 0."""
    n_t, n_f, T = 48, 240, 30000
    y, sig = _notched_map(70, n_t, n_f, mode)
    m = ctx.load_map(torch.from_numpy(y).cuda(), torch.from_numpy(sig).cuda(), 40.0, 0.5, paper_mode=paper,
                     fp16=fp16)
    om = oracle.OracleMap(y, sig, 40.0, 0.5, sig.ndim == 1, paper_mode=paper)
    rtol = 3.5e-4 if fp16 else RTOL
    ctx.set_tracks(T, 12, 3, 0.01)
    o, sc = om.score_range_scale(12, 3, T, 0.01)
    got = {}
    for kernel in (1, 2):
        ctx.set_option(_lib.STK_OPT_KERNEL, kernel)
        try:
            got[kernel] = ctx.score_all(m).cpu().numpy()
        finally:
            ctx.set_option(_lib.STK_OPT_KERNEL, 0)
        bad = np.abs(got[kernel] - o) > rtol * np.maximum(np.abs(o), sc)
        assert not bad.any(), (kernel, np.count_nonzero(bad))
    np.testing.assert_array_equal(got[1], got[2])
    ctx.set_template_shape(True, 6)
    try:
        ctx.set_tracks(5000, 13, 0, 0.01)
        g = ctx.score_all(m).cpu().numpy()
        og, sg = om.score_range_ext(13, 0, 5000, 0.01, general=True, t_min=6, with_scale=True)
        assert np.all(np.abs(g - og) <= rtol * np.maximum(np.abs(og), sg))
    finally:
        ctx.set_template_shape(False)
    m.close()
    allnotch = np.full_like(sig, np.inf)
    ma = ctx.load_map(torch.from_numpy(y).cuda(), torch.from_numpy(allnotch).cuda(), 40.0, 0.5, paper_mode=paper,
                      fp16=fp16)
    ctx.set_tracks(2000, 12, 0, 0.01)
    assert np.all(ctx.score_all(ma).cpu().numpy() == 0.0)
    ma.close()


@pytest.mark.parametrize("kernel", [0, 1, 2])
def test_single_template(ctx, kernel):
    """One template (the smallest range): both kernels, with and without the
    coherent order, give the oracle's SNR at its index."""
    y, sig = rand_map(67, 30, 50, "freq")
    m, om = load_both(ctx, y, sig, 40.0, 0.5)
    ctx.set_tracks(1, 3, 12345, 0.01)
    ctx.set_option(_lib.STK_OPT_KERNEL, kernel)
    try:
        h = ctx.score(m, 1)
        a = ctx.score_all(m).cpu().numpy()
    finally:
        ctx.set_option(_lib.STK_OPT_KERNEL, 0)
    f3, tau = oracle_params(3, 12345, 1, 50, 0.01)
    o, ex = om.score_explicit(f3, tau, extras=True)
    assert int(h["index"][0]) == 12345 and a.shape == (1,)
    assert_snr_close(a, o, ex, False, 30, what="single template")
    assert h["snr"][0] == a[0]


def test_invalid_inputs_rejected(ctx):
    L = _lib
    y = np.ones((10, 8), np.complex64)
    s = np.ones(8, np.float32)
    for bad_y, bad_s in [(y.copy(), np.zeros(8, np.float32)), (y.copy(), -s), (y.copy(), -s * np.inf),
                         (y.copy(), s * np.nan)]:
        with pytest.raises(stk.StkError) as e:
            ctx.load_map(bad_y, bad_s, 40.0, 0.5)
        assert e.value.code == L.STK_EINVAL
    ynan = y.copy()
    ynan[3, 4] = np.nan
    with pytest.raises(stk.StkError):
        ctx.load_map(ynan, s, 40.0, 0.5)
    with pytest.raises(stk.StkError):
        ctx.load_map(np.ones((1, 8), np.complex64), s, 40.0, 0.5)   # n_t < 2
    with pytest.raises(stk.StkError):
        ctx.load_map(y, s, 40.0, 0.0)                               # df <= 0
    m = ctx.load_map(y, s, 40.0, 0.5)
    with pytest.raises(stk.StkError):
        ctx.set_tracks(0, 1, 0, 0.01)
    with pytest.raises(stk.StkError):
        ctx.set_tracks(10, 1, 0, -1.0)
    ctx.set_tracks(10, 1, 0, 0.01)
    for k in [0, 11, 5000]:
        with pytest.raises(stk.StkError):
            ctx.score(m, k)
    # an explicit template outside the map is reported at the next sync
    ctx.score_explicit(m, torch.tensor([[1, 2, 8]], dtype=torch.int32), torch.tensor([0.0]))
    with pytest.raises(stk.StkError) as e:
        ctx.sync()
    assert e.value.code == L.STK_EINVAL
    ctx.sync()   # cleared


# ------------------------------------------------------------------ full-size workload, sampled
@pytest.mark.slow
def test_realistic_workload_sampled(ctx):
    """500 x 1600 map, 5 x 10^6 templates, k = 1024, in the benchmark's launch
    configuration; the oracle checks a sample of templates one by one, every
    selected template, and the selection against the GPU's own full SNR array."""
    w = synth.WORKLOADS["realistic"]
    fm = synth.realistic_map()
    m, om = load_both(ctx, fm.y, fm.sigma, fm.f_min, fm.df)
    ctx.set_tracks(w["n_tracks"], w["seed"], 0, w["tau_max"])
    hits = ctx.score(m, w["k"])
    plan = ctx.last_plan()
    assert plan["kernel"] == 2
    allg = ctx.score_all(m).cpu().numpy()
    # selection is exactly the top-k of the GPU's own SNRs
    order = np.lexsort((np.arange(allg.size), -allg))[:w["k"]]
    np.testing.assert_array_equal(hits["index"], order)
    np.testing.assert_array_equal(hits["snr"], allg[order])
    # sampled templates and every selected template against the oracle
    rng = np.random.default_rng(0)
    idx = np.unique(np.concatenate([rng.integers(0, w["n_tracks"], 20000), order]))
    f3 = np.zeros((idx.size, 3), np.uint32)
    tau = np.zeros(idx.size)
    for j, i in enumerate(idx):
        f, t = oracle.track_params(w["seed"], int(i), fm.n_f, w["tau_max"])
        f3[j], tau[j] = f, t
    o, ex = om.score_explicit(f3, tau, extras=True)
    assert_snr_close(allg[idx], o, ex, False, fm.n_t, what="realistic sample")
    sel = np.searchsorted(idx, order)
    np.testing.assert_allclose(hits["snr"], o[sel], rtol=RTOL)
