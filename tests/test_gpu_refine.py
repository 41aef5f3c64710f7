"""Refinement of loud templates: the interpolated statistic of continuous
templates (forward and adjoint kernels) against the FP64 oracle, a
finite-difference check at step 1e-3 (bins, and units of tau_max) away from the
bin knots, autograd wiring, and end-to-end gradient ascent with the refined
templates rescored by the discrete statistic (GPU and oracle)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle  # noqa: E402
import paper_1401_8060_b300 as stk  # noqa: E402
from paper_1401_8060_b300 import synth  # noqa: E402

TAU_MAX = 0.01


@pytest.fixture(scope="module")
def ctx():
    from paper_1401_8060_b300 import build
    build.build()
    c = stk.Context(0)
    yield c
    c.close()


def _x(f, n_t):
    M = n_t - 1
    j = np.arange(n_t)
    return ((M - j) ** 2 * f[0] + 2 * (M - j) * j * f[1] + j ** 2 * f[2]) / M ** 2


def _away_from_knots(rng, n, n_t, n_f, margin):
    out = []
    while len(out) < n:
        f = rng.uniform(1, n_f - 2, 3).astype(np.float32).astype(np.float64)
        x = _x(f, n_t)
        if np.min(np.abs(x - np.round(x))) >= margin:
            out.append(f)
    return np.array(out)


def _map(mode, n_t, n_f, seed):
    rng = np.random.default_rng(seed)
    if mode == "pixel":
        sig = rng.uniform(0.5, 2.0, (n_t, n_f)).astype(np.float32)
    elif mode == "freq":
        sig = synth.sigma_powerlaw(40.0 + 0.5 * np.arange(n_f), 1.1)
    else:
        sig = np.full(n_f, 1.4, np.float32)
    return synth.noise_map(n_t, n_f, sig, seed + 1), sig


@pytest.mark.parametrize("mode,paper,fp16", [("freq", False, False), ("pixel", False, False), ("const", False, False),
                                             ("pixel", True, False), ("freq", False, True)])
def test_forward_and_adjoint_vs_oracle(ctx, mode, paper, fp16):
    n_t, n_f, n = 120, 300, 400
    y, sig = _map(mode, n_t, n_f, 80)
    m = ctx.load_map(torch.from_numpy(y).cuda(), torch.from_numpy(sig).cuda(), 40.0, 0.5, paper_mode=paper,
                     fp16=fp16)
    om = oracle.OracleMap(y, sig, 40.0, 0.5, sig.ndim == 1, paper_mode=paper)
    rng = np.random.default_rng(81)
    f3 = rng.uniform(0, n_f - 1, (n, 3)).astype(np.float32)
    tau = rng.uniform(-TAU_MAX, TAU_MAX, n).astype(np.float32)
    f3t, taut = torch.from_numpy(f3).cuda(), torch.from_numpy(tau).cuda()
    snr = ctx.interp_forward(m, f3t, taut).cpu().numpy()
    g = rng.standard_normal(n).astype(np.float32)
    gf, gt = ctx.interp_adjoint(m, f3t, taut, torch.from_numpy(g).cuda())
    gf, gt = gf.cpu().numpy(), gt.cpu().numpy()
    o, og = om.interp_score(f3.astype(np.float64), tau.astype(np.float64), grad=True)
    # scale of rounding: the discrete statistic's pixel-magnitude sum for the nearest template
    _, ex = om.score_explicit(np.clip(np.round(f3), 0, n_f - 1).astype(np.uint32), tau.astype(np.float64),
                              extras=True)
    sc = ex["absz"] / (n_t if paper else np.sqrt(ex["W"]))
    rt = 3.5e-4 if fp16 else 2e-5
    assert np.all(np.abs(snr - o) <= rt * sc + 1e-5 * np.abs(o)), np.max(np.abs(snr - o) / sc)
    # gradients: relative to each component's largest magnitude over the templates
    for q in range(4):
        got = gf[:, q] if q < 3 else gt
        ref = g * og[:, q]
        tol = (3e-3 if fp16 else 2e-4) * np.max(np.abs(ref)) + 1e-4 * np.abs(ref)
        assert np.all(np.abs(got - ref) <= tol), (q, np.max(np.abs(got - ref) / np.max(np.abs(ref))))


@pytest.mark.parametrize("threads", [32, 128])
def test_long_and_wide_maps_vs_oracle(ctx, threads):
    """Long maps (3000 columns: each thread's position and phase advance over up
    to 94 steps from starts formed in 128-bit fixed point) and a wide band (8000
    bins, steep curves) against the FP64 oracle, forward and adjoint."""
    from paper_1401_8060_b300 import _lib
    ctx.set_option(_lib.STK_OPT_INTERP_THREADS, threads)
    try:
        for n_t, n_f, n in ((3000, 60, 48), (40, 8000, 96)):
            y, sig = _map("freq", n_t, n_f, 60 + n_t)
            m = ctx.load_map(torch.from_numpy(y).cuda(), torch.from_numpy(sig).cuda(), 40.0, 0.5)
            om = oracle.OracleMap(y, sig, 40.0, 0.5, True)
            rng = np.random.default_rng(n_t)
            f3 = rng.uniform(0, n_f - 1, (n, 3)).astype(np.float32)
            tau = rng.uniform(-TAU_MAX, TAU_MAX, n).astype(np.float32)
            f3t, taut = torch.from_numpy(f3).cuda(), torch.from_numpy(tau).cuda()
            snr = ctx.interp_forward(m, f3t, taut).cpu().numpy()
            gf, gt = ctx.interp_adjoint(m, f3t, taut, torch.ones(n, device="cuda"))
            gf, gt = gf.cpu().numpy(), gt.cpu().numpy()
            o, og = om.interp_score(f3.astype(np.float64), tau.astype(np.float64), grad=True)
            _, ex = om.score_explicit(np.clip(np.round(f3), 0, n_f - 1).astype(np.uint32), tau.astype(np.float64),
                                      extras=True)
            sc = ex["absz"] / np.sqrt(ex["W"])
            assert np.all(np.abs(snr - o) <= 2e-5 * sc + 1e-5 * np.abs(o)), (n_t, np.max(np.abs(snr - o) / sc))
            for q in range(4):
                got = gf[:, q] if q < 3 else gt
                tol = 2e-4 * np.max(np.abs(og[:, q])) + 1e-4 * np.abs(og[:, q])
                assert np.all(np.abs(got - og[:, q]) <= tol), (n_t, q)
            m.close()
    finally:
        ctx.set_option(_lib.STK_OPT_INTERP_THREADS, 0)


def test_finite_differences_at_step_1e3(ctx):
    n_t, n_f, n = 200, 400, 64
    y, sig = _map("freq", n_t, n_f, 82)
    m = ctx.load_map(torch.from_numpy(y).cuda(), torch.from_numpy(sig).cuda(), 40.0, 0.5)
    rng = np.random.default_rng(83)
    f3 = _away_from_knots(rng, n, n_t, n_f, 2e-3)
    tau = rng.uniform(-0.8, 0.8, n) * TAU_MAX
    f3t = torch.tensor(f3, dtype=torch.float32, device="cuda")
    taut = torch.tensor(tau, dtype=torch.float32, device="cuda")
    gf, gt = ctx.interp_adjoint(m, f3t, taut, torch.ones(n, device="cuda"))
    grad = np.concatenate([gf.cpu().numpy(), gt.cpu().numpy()[:, None] * TAU_MAX], axis=1)  # tau in units of tau_max
    h = 1e-3
    fd = np.zeros((n, 4))
    for q in range(4):
        fp, fm, tp, tm = f3t.clone(), f3t.clone(), taut.clone(), taut.clone()
        if q < 3:
            fp[:, q] += h
            fm[:, q] -= h
        else:
            tp += h * TAU_MAX
            tm -= h * TAU_MAX
        fd[:, q] = (ctx.interp_forward(m, fp, tp) - ctx.interp_forward(m, fm, tm)).cpu().numpy() / (2 * h)
    # FP32 sums make the difference quotient noisy at ~1e-5 / 2e-3: compare with that slack
    err = np.abs(fd - grad)
    assert np.all(err <= 0.03 * np.abs(grad) + 0.02), np.max(err)
    # the FP64 oracle's gradient agrees with the adjoint too
    om = oracle.OracleMap(y, sig, 40.0, 0.5, True)
    _, og = om.interp_score(f3t.cpu().numpy().astype(np.float64), taut.cpu().numpy().astype(np.float64), grad=True)
    og[:, 3] *= TAU_MAX
    assert np.all(np.abs(og - grad) <= 2e-4 * np.max(np.abs(og), axis=0) + 1e-4 * np.abs(og))


def test_autograd_and_refinement(ctx):
    """Top templates of a noisy map with an injected chirp climb the interpolated
    statistic; their rounded versions are rescored by the discrete statistic and the
    oracle agrees with the GPU on those SNRs."""
    fm = synth.realistic_map(n_t=200, n_f=400)
    m = ctx.load_map(torch.from_numpy(fm.y).cuda(), torch.from_numpy(fm.sigma).cuda(), fm.f_min, fm.df)
    ctx.set_tracks(200_000, 2, 0, TAU_MAX)
    hits = ctx.score(m, 64)
    f3 = torch.tensor(np.array([list(h) for h in hits["f"]]), dtype=torch.float32, device="cuda")
    tau = torch.tensor(hits["tau"], dtype=torch.float32, device="cuda")
    # autograd gradient equals the adjoint kernel
    f_ = f3.clone().requires_grad_(True)
    t_ = tau.clone().requires_grad_(True)
    s = stk.interp_snr(ctx, m, f_, t_)
    s.sum().backward()
    gf, gt = ctx.interp_adjoint(m, f3, tau, torch.ones_like(tau))
    assert torch.equal(f_.grad, gf) and torch.equal(t_.grad, gt)
    # 50 ascent steps
    f_new, tau_new, hist = stk.refine(ctx, m, f3, tau, TAU_MAX, steps=50)
    gain = (hist[-1] - hist[0]).cpu().numpy()
    assert np.mean(gain) > 0 and np.mean(gain > -1e-3) > 0.9, gain
    assert float(f_new.min()) >= 0 and float(f_new.max()) <= fm.n_f - 1 and float(tau_new.abs().max()) <= TAU_MAX
    # discrete rescoring of the rounded refined templates: GPU vs the FP64 oracle
    f_int = torch.round(f_new).to(torch.int32)
    d = ctx.score_explicit(m, f_int, tau_new.to(torch.float64)).cpu().numpy()
    om = oracle.OracleMap.from_ftmap(fm)
    o = om.score_explicit(f_int.cpu().numpy().astype(np.uint32), tau_new.cpu().numpy().astype(np.float64))
    np.testing.assert_allclose(d, o, rtol=1e-5, atol=1e-5)
    print(f"refine: interpolated SNR {hist[0].mean():.3f} -> {hist[-1].mean():.3f}; "
          f"discrete before {hits['snr'].mean():.3f}, after rounding {d.mean():.3f}")


def _torch_adam_refine(ctx, m, f3, tau, tau_max, steps, lr_bins=0.25, lr_tau_frac=0.02):
    """The ascent written with torch.autograd and torch.optim.Adam over the same
    interpolated statistic: the comparison for the loop that runs on the device."""
    f = f3.detach().clone().requires_grad_(True)
    u = (tau.detach() / tau_max).clone().requires_grad_(True)
    opt = torch.optim.Adam([{"params": [f], "lr": lr_bins}, {"params": [u], "lr": lr_tau_frac}])
    hist = []
    for _ in range(steps):
        opt.zero_grad()
        snr = stk.interp_snr(ctx, m, f, u * tau_max)
        hist.append(snr.detach().clone())
        (-snr.sum()).backward()
        opt.step()
        with torch.no_grad():
            f.clamp_(0.0, float(m.n_f - 1))
            u.clamp_(-1.0, 1.0)
    hist.append(ctx.interp_forward(m, f.detach(), u.detach() * tau_max))
    return f.detach(), u.detach() * tau_max, torch.stack(hist)


def _loud_templates(ctx, n):
    fm = synth.realistic_map(n_t=200, n_f=400)
    m = ctx.load_map(torch.from_numpy(fm.y).cuda(), torch.from_numpy(fm.sigma).cuda(), fm.f_min, fm.df)
    ctx.set_tracks(200_000, 2, 0, TAU_MAX)
    hits = ctx.score(m, n)
    f3 = torch.tensor(np.array([list(h) for h in hits["f"]]), dtype=torch.float32, device="cuda")
    tau = torch.tensor(hits["tau"], dtype=torch.float32, device="cuda")
    return fm, m, f3, tau


def test_device_loop_matches_torch_adam(ctx):
    """The device loop against torch's Adam over autograd, 50 steps of 256 loud
    templates: the same ascent up to FP32 rounding order."""
    fm, m, f3, tau = _loud_templates(ctx, 256)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ctx.refine(m, f3, tau, TAU_MAX, steps=2)
    _torch_adam_refine(ctx, m, f3, tau, TAU_MAX, 2)
    torch.cuda.synchronize()
    ev[0].record()
    f_d, t_d, h_d = ctx.refine(m, f3, tau, TAU_MAX, steps=50)
    ev[1].record()
    ev[2].record()
    f_t, t_t, h_t = _torch_adam_refine(ctx, m, f3, tau, TAU_MAX, 50)
    ev[3].record()
    torch.cuda.synchronize()
    print(f"refine 50 steps x 256: device loop {ev[0].elapsed_time(ev[1]):.2f} ms, "
          f"torch Adam over autograd {ev[2].elapsed_time(ev[3]):.2f} ms")
    assert h_d.shape == h_t.shape == (51, 256)
    # the device loop starts from the given delays; the torch loop from (tau / tau_max) * tau_max
    assert torch.equal(h_d[0], ctx.interp_forward(m, f3, tau))
    assert torch.allclose(h_d[0], h_t[0], rtol=1e-5, atol=1e-5)
    d = (h_d - h_t).abs().cpu().numpy()
    scale = h_t.abs().cpu().numpy() + 1.0
    # Adam normalises each step, so rounding differences stay at the ulp level
    # except where a curve point sits within an ulp of a bin knot (a kink)
    assert np.quantile(d / scale, 0.99) < 1e-4, np.quantile(d / scale, 0.99)
    assert abs(float(h_d[-1].mean() - h_t[-1].mean())) < 1e-3 * float(h_t[-1].abs().mean())
    assert float((f_d - f_t).abs().max()) < 0.5 and float((t_d - t_t).abs().max()) <= 0.1 * TAU_MAX
    # the inputs are untouched; the last history row is the SNR at the returned templates
    assert torch.equal(h_d[-1], ctx.interp_forward(m, f_d, t_d))


def test_first_step_is_signed_learning_rate(ctx):
    """Adam's first step from zero moments is lr * g / (|g| + eps) per coordinate: a
    step of the learning rate along the sign of the oracle's FP64 gradient,
    then the projection."""
    n_t, n_f, n = 160, 300, 200
    y, sig = _map("freq", n_t, n_f, 84)
    m = ctx.load_map(torch.from_numpy(y).cuda(), torch.from_numpy(sig).cuda(), 40.0, 0.5)
    om = oracle.OracleMap(y, sig, 40.0, 0.5, True)
    rng = np.random.default_rng(85)
    f3 = _away_from_knots(rng, n, n_t, n_f, 2e-3).astype(np.float32)
    f3[:8, 0] = 0.0                                            # some start on the band edge
    tau = (rng.uniform(-1.0, 1.0, n) * TAU_MAX).astype(np.float32)
    tau[8:16] = TAU_MAX                                        # and some on the delay bound
    lr_f, lr_u = 0.3, 0.05
    f_new, t_new, h = ctx.refine(m, torch.from_numpy(f3).cuda(), torch.from_numpy(tau).cuda(), TAU_MAX, steps=1,
                                 lr_bins=lr_f, lr_tau_frac=lr_u)
    snr0, og = om.interp_score(f3.astype(np.float64), tau.astype(np.float64), grad=True)
    og[:, 3] *= TAU_MAX
    f_new, t_new = f_new.cpu().numpy(), t_new.cpu().numpy()
    exp_f = np.clip(f3 + lr_f * np.sign(og[:, :3]), 0, n_f - 1)
    exp_u = np.clip(tau / TAU_MAX + lr_u * np.sign(og[:, 3]), -1, 1)
    # where the gradient is too small to have a reliable sign in FP32 the step may go
    # either way; everywhere else it is the signed learning rate, to FP32 rounding
    sure = np.abs(og) > 1e-3 * np.max(np.abs(og), axis=0)
    assert np.mean(sure) > 0.95
    err_f = np.abs(f_new - exp_f)
    assert np.all(err_f[sure[:, :3]] <= 1e-4 * (1 + np.abs(exp_f[sure[:, :3]]))), np.max(err_f[sure[:, :3]])
    err_u = np.abs(t_new / TAU_MAX - exp_u)
    assert np.all(err_u[sure[:, 3]] <= 1e-5), np.max(err_u[sure[:, 3]])
    assert np.all(f_new >= 0) and np.all(f_new <= n_f - 1) and np.all(np.abs(t_new) <= TAU_MAX)
    # history rows: the oracle's SNR before the step, the forward kernel's after it
    sc = np.abs(snr0) + 1.0
    assert np.all(np.abs(h[0].cpu().numpy() - snr0) <= 2e-5 * sc * np.sqrt(n_t))
    assert torch.equal(h[1], ctx.interp_forward(m, torch.from_numpy(f_new).cuda(), torch.from_numpy(t_new).cuda()))


def test_refine_edge_cases(ctx):
    n_t, n_f = 64, 50
    y, sig = _map("const", n_t, n_f, 86)
    m = ctx.load_map(torch.from_numpy(y).cuda(), torch.from_numpy(sig).cuda(), 40.0, 0.5)
    rng = np.random.default_rng(87)
    f3 = torch.tensor(rng.uniform(0, n_f - 1, (33, 3)), dtype=torch.float32, device="cuda")
    tau = torch.tensor(rng.uniform(-TAU_MAX, TAU_MAX, 33), dtype=torch.float32, device="cuda")
    # zero steps: parameters unchanged, one history row
    f0, t0, h0 = ctx.refine(m, f3, tau, TAU_MAX, steps=0)
    assert torch.equal(f0, f3) and torch.equal(h0[0], ctx.interp_forward(m, f3, tau))
    # no templates
    fe, te, he = ctx.refine(m, f3[:0], tau[:0], TAU_MAX, steps=5)
    assert fe.numel() == 0 and he.shape == (6, 0)
    # no history requested
    f1, t1, h1 = ctx.refine(m, f3, tau, TAU_MAX, steps=3, history=False)
    f2, t2, h2 = ctx.refine(m, f3, tau, TAU_MAX, steps=3)
    assert h1 is None and torch.equal(f1, f2) and torch.equal(t1, t2)  # deterministic
    # zero learning rates leave the parameters where they are
    fz, tz, _ = ctx.refine(m, f3, tau, TAU_MAX, steps=4, lr_bins=0.0, lr_tau_frac=0.0)
    assert torch.equal(fz, f3) and torch.allclose(tz, tau, rtol=1e-6, atol=0)
    # control frequencies beyond 2^29 bins or non-finite, or a non-finite delay: NaN, the others unaffected
    fw, tw = f3[:4].clone(), tau[:4].clone()
    fw[0, 1], fw[1, 2], tw[2] = 2.0 ** 31, float("nan"), float("inf")
    sw = ctx.interp_forward(m, fw, tw)
    assert torch.isnan(sw[:3]).all() and torch.equal(sw[3], ctx.interp_forward(m, f3[3:4], tau[3:4])[0])
    for bad in ({"tau_max": 0.0}, {"tau_max": -1.0}, {"steps": -1}, {"lr_bins": -0.1}, {"lr_tau_frac": float("nan")}):
        kw = {"tau_max": TAU_MAX, "steps": 2}
        kw.update(bad)
        with pytest.raises(stk.StkError):
            ctx.refine(m, f3, tau, **kw)


@pytest.mark.parametrize("threads", [32, 64, 128])
def test_threads_per_template(ctx, threads):
    """Every template layout (one warp, two, four per template; a ragged last block)
    against the FP64 oracle, and the device ascent for each."""
    from paper_1401_8060_b300 import _lib
    n_t, n_f, n = 150, 260, 77
    y, sig = _map("pixel", n_t, n_f, 88)
    m = ctx.load_map(torch.from_numpy(y).cuda(), torch.from_numpy(sig).cuda(), 40.0, 0.5)
    om = oracle.OracleMap(y, sig, 40.0, 0.5, False)
    rng = np.random.default_rng(89)
    f3 = rng.uniform(0, n_f - 1, (n, 3)).astype(np.float32)
    tau = rng.uniform(-TAU_MAX, TAU_MAX, n).astype(np.float32)
    f3t, taut = torch.from_numpy(f3).cuda(), torch.from_numpy(tau).cuda()
    ctx.set_option(_lib.STK_OPT_INTERP_THREADS, threads)
    try:
        snr = ctx.interp_forward(m, f3t, taut).cpu().numpy()
        gf, gt = ctx.interp_adjoint(m, f3t, taut, torch.ones(n, device="cuda"))
        f_new, t_new, h = ctx.refine(m, f3t, taut, TAU_MAX, steps=5)
    finally:
        ctx.set_option(_lib.STK_OPT_INTERP_THREADS, 0)
    o, og = om.interp_score(f3.astype(np.float64), tau.astype(np.float64), grad=True)
    _, ex = om.score_explicit(np.clip(np.round(f3), 0, n_f - 1).astype(np.uint32), tau.astype(np.float64),
                              extras=True)
    sc = ex["absz"] / np.sqrt(ex["W"])
    assert np.all(np.abs(snr - o) <= 2e-5 * sc + 1e-5 * np.abs(o))
    got = np.concatenate([gf.cpu().numpy(), gt.cpu().numpy()[:, None]], axis=1)
    assert np.all(np.abs(got - og) <= 2e-4 * np.max(np.abs(og), axis=0) + 1e-4 * np.abs(og))
    # the ascent: history row 0 is the forward statistic, the last row the SNR at the result
    assert np.allclose(h[0].cpu().numpy(), snr, rtol=0, atol=1e-5 * (1 + np.max(np.abs(snr))))
    o5 = om.interp_score(f_new.cpu().numpy().astype(np.float64), t_new.cpu().numpy().astype(np.float64))
    assert np.all(np.abs(h[-1].cpu().numpy() - o5) <= 2e-5 * sc * 2 + 1e-5 * np.abs(o5))
    assert float((h[-1] - h[0]).mean()) > 0


def test_threads_option_range(ctx):
    from paper_1401_8060_b300 import _lib
    for bad in (1, 16, 96, 256, -32):
        with pytest.raises(stk.StkError):
            ctx.set_option(_lib.STK_OPT_INTERP_THREADS, bad)


@pytest.mark.parametrize("mode,fp16", [("freq", False), ("pixel", False), ("const", False), ("freq", True)])
def test_polish_never_loses_and_matches_oracle(ctx, mode, fp16):
    """The discrete follow-up (stk_polish) of the loudest templates: every kept
    template's SNR is the scorer's own (bit-identical to stk_score_explicit), at
    least the start's, and within the parity bound of the FP64 oracle, whose
    rescoring also finds no template below its start beyond that bound.  With
    the refined continuous templates as alternatives, most templates gain."""
    n_t, n_f, T, k = 160, 400, 60_000, 192
    y, sig = _map(mode, n_t, n_f, 90)
    m = ctx.load_map(torch.from_numpy(y).cuda(), torch.from_numpy(sig).cuda(), 40.0, 0.5, fp16=fp16)
    om = oracle.OracleMap(y, sig, 40.0, 0.5, sig.ndim == 1)
    ctx.set_tracks(T, 5, 0, TAU_MAX)
    hits = ctx.score(m, k)
    f_start = np.array([list(v) for v in hits["f"]], dtype=np.int64)
    t_start = hits["tau"].copy()
    f_ref = torch.tensor(f_start, dtype=torch.float32, device="cuda")
    t_ref = torch.tensor(t_start, dtype=torch.float32, device="cuda")
    f_ref, t_ref, _ = ctx.refine(m, f_ref, t_ref, TAU_MAX, steps=30)
    f_out, t_out, snr, which = ctx.polish(m, f_start, t_start, TAU_MAX, alt_f3=f_ref, alt_tau=t_ref, moves=6)
    f_out, t_out, snr, which = (x.cpu().numpy() for x in (f_out, t_out, snr, which))
    assert np.all((which >= 0) & (which <= 2))
    assert np.all((f_out >= 0) & (f_out < n_f)) and np.all(np.abs(t_out) <= TAU_MAX)
    assert np.all(snr >= hits["snr"]), np.min(snr - hits["snr"])            # never below the start
    again = ctx.score_explicit(m, torch.from_numpy(f_out.astype(np.int32)), torch.from_numpy(t_out)).cpu().numpy()
    np.testing.assert_array_equal(again.astype(np.float32), snr.astype(np.float32))   # the scorer's own SNR
    o, ex = om.score_explicit(f_out.astype(np.uint32), t_out, extras=True)
    sc = ex["absz"] / np.sqrt(ex["W"])
    rt = 3.5e-4 if fp16 else 1e-5
    assert np.all(np.abs(snr - o) <= rt * np.maximum(np.abs(o), sc)), np.max(np.abs(snr - o) / sc)
    o0, ex0 = om.score_explicit(f_start.astype(np.uint32), t_start, extras=True)
    sc0 = ex0["absz"] / np.sqrt(ex0["W"])
    assert np.all(o >= o0 - 2 * rt * np.maximum(sc, sc0)), np.min(o - o0)   # the oracle agrees
    gain = snr - hits["snr"]
    assert np.mean(gain > 0) > 0.8 and np.mean(gain) > 0, (np.mean(gain > 0), np.mean(gain))
    # delay only, no alternative: still never below the start
    f1, t1, s1, w1 = ctx.polish(m, f_start, t_start, TAU_MAX, moves=0)
    s1, f1 = s1.cpu().numpy(), f1.cpu().numpy()
    assert np.all(s1 >= hits["snr"]) and np.array_equal(f1, f_start)
    m.close()


def test_polish_non_finite_alternatives(ctx):
    """A NaN alternative bin counts as bin 0 and a NaN alternative delay as the
    start's delay: the polish still returns templates inside the map and the delay
    range, never below the start, and the same as with those bins given as 0."""
    n_t, n_f, T, k = 120, 300, 20_000, 64
    y, sig = _map("freq", n_t, n_f, 41)
    m = ctx.load_map(torch.from_numpy(y).cuda(), torch.from_numpy(sig).cuda(), 40.0, 0.5)
    ctx.set_tracks(T, 9, 0, TAU_MAX)
    hits = ctx.score(m, k)
    f_start = np.array([list(v) for v in hits["f"]], dtype=np.int64)
    t_start = hits["tau"].copy()
    alt_f = f_start.astype(np.float32) + 0.4
    alt_t = t_start.astype(np.float32)
    alt_f[::3, 1] = np.nan
    alt_t[1::3] = np.nan
    f1, t1, s1, w1 = (x.cpu().numpy() for x in ctx.polish(m, f_start, t_start, TAU_MAX, alt_f3=alt_f,
                                                            alt_tau=alt_t, moves=4))
    assert np.all((f1 >= 0) & (f1 < n_f)) and np.all(np.abs(t1) <= TAU_MAX)
    assert np.all(s1 >= hits["snr"]), np.min(s1 - hits["snr"])
    # the NaN bins replaced by 0 as documented
    exp_f = np.where(np.isnan(alt_f), 0.0, alt_f).astype(np.float32)
    f2, t2, s2, w2 = (x.cpu().numpy() for x in ctx.polish(m, f_start, t_start, TAU_MAX, alt_f3=exp_f,
                                                            alt_tau=alt_t, moves=4))
    for a, b in ((f1, f2), (t1, t2), (s1, s2), (w1, w2)):
        np.testing.assert_array_equal(a, b)
    m.close()


def test_polish_invalid_inputs(ctx):
    y, sig = _map("freq", 40, 64, 3)
    m = ctx.load_map(torch.from_numpy(y).cuda(), torch.from_numpy(sig).cuda(), 40.0, 0.5)
    f = np.zeros((4, 3), np.int64)
    t = np.zeros(4)
    for kw in ({"tau_max": 0.0}, {"tau_max": TAU_MAX, "moves": -1}, {"tau_max": TAU_MAX, "moves": 2000}):
        with pytest.raises(stk.StkError):
            ctx.polish(m, f, t, **kw)
    m.close()
