"""General templates (random start / middle / end times, six random numbers per
template) and the sky-patch delay prior, against the FP64 oracle: times, delays
and pixels bit-exact; SNRs within the parity tolerance; top-k against the
oracle's full run."""
import numpy as np
import pytest

from _parity import RTOL, assert_topk_matches

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle  # noqa: E402
import paper_1401_8060_b300 as stk  # noqa: E402
from paper_1401_8060_b300 import synth  # noqa: E402


@pytest.fixture
def ctx():
    from paper_1401_8060_b300 import build
    build.build()
    c = stk.Context(0)
    yield c
    c.close()


def _map(mode, n_t, n_f, seed):
    rng = np.random.default_rng(seed)
    if mode == "pixel":
        sig = rng.uniform(0.5, 2.0, (n_t, n_f)).astype(np.float32)
    elif mode == "freq":
        sig = synth.sigma_powerlaw(40.0 + 0.5 * np.arange(n_f), 1.2)
    else:
        sig = np.full(n_f, 1.5, np.float32)
    return synth.noise_map(n_t, n_f, sig, seed + 7), sig


def _scale(y, sig, t3, f3, paper):
    """sum |z_j| / norm over each template's oracle pixels (the rounding scale of the FP32 path)."""
    n_t, n_f = y.shape
    out = []
    for t, f in zip(t3, f3):
        b = oracle.track_bins_general(t, f, n_t, n_f)
        j = np.nonzero(b >= 0)[0]
        s = (sig[b[j]] if sig.ndim == 1 else sig[j, b[j]]).astype(np.float64)
        z = np.abs(y[j, b[j]].astype(np.complex128)) / (s if paper else s ** 2)
        out.append(z.sum() / (len(j) if paper else np.sqrt(np.sum(s ** -2.0))))
    return np.array(out)


def test_times_delays_and_pixels_bit_exact(ctx):
    n_t, n_f = 300, 700
    y = np.zeros((n_t, n_f), np.complex64)
    m = ctx.load_map(torch.from_numpy(y).cuda(), torch.ones(n_f, device="cuda"), 40.0, 0.5)
    q = np.sort(np.random.default_rng(1).uniform(-0.01, 0.004, 33))
    ctx.set_tracks(1, 77, 0, 0.01)
    ctx.set_template_shape(True, 40)
    ctx.set_tau_prior(q)
    for g in [0, 5, 999, 2 ** 35 + 3]:
        f, tau, bins = ctx.track_params(m, g)
        t = ctx.track_times(m, g)
        fo, tauo = oracle.track_params_prior(77, g, n_f, q)
        assert f == fo and tau == tauo
        assert t == oracle.track_times(77, g, n_t, 40)
        np.testing.assert_array_equal(bins, oracle.track_bins_general(t, f, n_t, n_f))
    ctx.set_tau_prior(None)
    ctx.set_template_shape(False)
    f, tau, _ = ctx.track_params(m, 5)
    assert (f, tau) == oracle.track_params(77, 5, n_f, 0.01)


@pytest.mark.parametrize("mode,paper,fp16", [("freq", False, False), ("pixel", False, False),
                                             ("const", False, False), ("pixel", True, False)])
def test_general_score_all_vs_oracle(ctx, mode, paper, fp16):
    n_t, n_f, T, seed, off, t_min = 90, 250, 6000, 3, 100, 12
    y, sig = _map(mode, n_t, n_f, 50)
    m = ctx.load_map(torch.from_numpy(y).cuda(), torch.from_numpy(sig).cuda(), 40.0, 0.5, paper_mode=paper,
                     fp16=fp16)
    om = oracle.OracleMap(y, sig, 40.0, 0.5, sig.ndim == 1, paper_mode=paper)
    ctx.set_template_shape(True, t_min)
    ctx.set_tracks(T, seed, off, 0.01)
    g = ctx.score_all(m).cpu().numpy()
    assert ctx.last_plan()["kernel"] == 3
    o = om.score_range_ext(seed, off, T, 0.01, general=True, t_min=t_min)
    t3 = [oracle.track_times(seed, off + i, n_t, t_min) for i in range(T)]
    f3 = [oracle.track_params(seed, off + i, n_f, 0.01)[0] for i in range(T)]
    sc = _scale(y, sig, t3, f3, paper)
    assert np.all(np.abs(g - o) <= RTOL * np.maximum(np.abs(o), sc)), np.max(np.abs(g - o) / sc)
    # explicit general scoring of the same templates agrees bit for bit with the generated ones
    tau = [oracle.track_params(seed, off + i, n_f, 0.01)[1] for i in range(T)]
    e = ctx.score_explicit_general(m, t3, f3, tau).cpu().numpy()
    np.testing.assert_array_equal(e, g)
    np.testing.assert_array_equal(om.score_explicit_general(t3, f3, tau), o)


def test_general_topk_with_prior_vs_oracle(ctx):
    n_t, n_f, T, k = 120, 400, 20000, 32
    y, sig = _map("freq", n_t, n_f, 51)
    m = ctx.load_map(torch.from_numpy(y).cuda(), torch.from_numpy(sig).cuda(), 40.0, 0.5)
    q = np.linspace(-0.002, 0.009, 17) ** 1   # a patch of delays away from zero
    ctx.set_template_shape(True, 30)
    ctx.set_tau_prior(q)
    ctx.set_tracks(T, 9, 0, 0.01)
    hits = ctx.score(m, k)
    om = oracle.OracleMap(y, sig, 40.0, 0.5, True)
    o = om.score_range_ext(9, 0, T, 0.01, general=True, t_min=30, quantiles=q)
    assert_topk_matches(hits, o, 0, k, what="general templates with a delay prior")
    assert np.all(hits["tau"] >= q[0]) and np.all(hits["tau"] <= q[-1])


@pytest.mark.parametrize("n_t,n_f,T,prior", [(300, 700, 40000, False), (120, 5, 50000, True),
                                              (12, 2000, 400000, False)])
def test_general_coherent_order_identical(ctx, n_t, n_f, T, prior):
    """Large general-template jobs run in coherent order (start and end column,
    then bins); every SNR equals index order bit for bit at its own index."""
    from paper_1401_8060_b300 import _lib
    y, sig = _map("freq", n_t, n_f, 31)
    m = ctx.load_map(torch.from_numpy(y).cuda(), torch.from_numpy(sig).cuda(), 40.0, 0.5)
    ctx.set_template_shape(True, 3)
    if prior:
        ctx.set_tau_prior(np.linspace(-0.006, 0.008, 9))
    ctx.set_tracks(T, 5, 77, 0.01)
    try:
        a = ctx.score_all(m).cpu().numpy()
        assert ctx.last_plan()["order"] == 1
        ctx.set_option(_lib.STK_OPT_ORDER, 0)
        b = ctx.score_all(m).cpu().numpy()
        assert ctx.last_plan()["order"] == 0
    finally:
        ctx.set_option(_lib.STK_OPT_ORDER, 1)
        ctx.set_template_shape(False)
        if prior:
            ctx.set_tau_prior(None)
    np.testing.assert_array_equal(a, b)
    m.close()


def test_general_rejects_large_maps(ctx):
    y = np.zeros((10, 9000), np.complex64)
    m = ctx.load_map(y, np.ones(9000, np.float32), 40.0, 0.5)
    ctx.set_template_shape(True, 2)
    ctx.set_tracks(10, 1, 0, 0.01)
    with pytest.raises(stk.StkError):
        ctx.score(m, 1)
    with pytest.raises(stk.StkError):
        ctx.set_tau_prior([0.001, -0.001])        # decreasing
    with pytest.raises(stk.StkError):
        ctx.set_template_shape(True, 0)
