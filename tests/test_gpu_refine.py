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
