"""Pins of the FP64 oracle against things other than itself.

Each test ties one part of the oracle to the paper or to mathematics that is
independent of the oracle's own code: a library routine (numpy's Philox), the
parametric Bezier curve evaluated in exact rational arithmetic, closed forms
(Eq. 3), the paper's printed worked numbers (tests/golden), invariants
(linearity, time reversal, sign), brute-force enumeration on tiny maps, and
noise statistics.  A dropped term, swapped index or wrong sign anywhere in the
oracle fails at least one of these.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")


# ---------------------------------------------------------------- helpers
def bezier_bins_exact(f, n_t):
    """Sec. III curve (t, f)(xi) = (1-xi)^2 P0 + 2(1-xi)xi P1 + xi^2 P2, with
    P0 = (0, f0), P1 = (M/2, f1), P2 = (M, f2), evaluated exactly at xi = j/M;
    the pixel is the nearest bin (halves up)."""
    M = n_t - 1
    P = [(Fraction(0), Fraction(f[0])), (Fraction(M, 2), Fraction(f[1])), (Fraction(M), Fraction(f[2]))]
    out = []
    for j in range(n_t):
        xi = Fraction(j, M)
        b0, b1, b2 = (1 - xi) ** 2, 2 * (1 - xi) * xi, xi ** 2
        t = b0 * P[0][0] + b1 * P[1][0] + b2 * P[2][0]
        fr = b0 * P[0][1] + b1 * P[1][1] + b2 * P[2][1]
        assert t == j  # control times pinned so column j sits at xi = j / M
        out.append(math.floor(fr + Fraction(1, 2)))
    return np.array(out, dtype=np.int32)


def brute_snr(y, sigma_full, f_min, df, bins, tau, paper_mode=False):
    """Eq. 7 written with complex exponentials (numpy, complex128)."""
    j = np.arange(len(bins))
    yv = y[j, bins].astype(np.complex128)
    s = sigma_full[j, bins].astype(np.float64)
    fr = f_min + bins * df
    rot = np.exp(2j * np.pi * fr * tau)
    if paper_mode:
        return float(np.sum((rot * (yv / s)).real) / len(bins))
    return float(np.sum((rot * yv / s ** 2).real) / np.sqrt(np.sum(s ** -2.0)))


# ---------------------------------------------------------------- Philox
@pytest.mark.parametrize("ctr,key", [
    ((0, 0, 0, 0), (0, 0)),
    ((1, 0, 0, 0), (5, 7)),
    ((12345678901234, 0, 0, 0), (2, 0)),
    ((0, 6, 99, 2 ** 63), (123456789, 2 ** 64 - 5)),   # carry from word 0 in numpy's increment
    ((2 ** 64 - 1, 2 ** 64 - 1, 2 ** 64 - 1, 2 ** 64 - 1), (2 ** 64 - 1, 2 ** 64 - 1)),
])
def test_philox_matches_numpy(orc, ctr, key):
    # numpy's Philox adds one to the 256-bit counter before each block.
    c = (ctr[0] + (ctr[1] << 64) + (ctr[2] << 128) + (ctr[3] << 192) - 1) % 2 ** 256
    prev = [(c >> (64 * i)) & (2 ** 64 - 1) for i in range(4)]
    ref = np.random.Philox(key=np.array(key, dtype=np.uint64),
                          counter=np.array(prev, dtype=np.uint64)).random_raw(4)
    assert orc.philox4x64_10(ctr, key) == [int(v) for v in ref]


# ---------------------------------------------------------------- template draws
def test_track_params_definition(orc):
    n_f, tau_max, seed = 1600, 0.010, 2
    for g in [0, 1, 2, 1000, 2 ** 40 + 3]:
        prev = [g - 1, 0, 0, 0] if g else [2 ** 64 - 1] * 4   # numpy steps the counter first
        u = np.random.Philox(key=np.array([seed, 0], dtype=np.uint64),
                             counter=np.array(prev, dtype=np.uint64)).random_raw(4)
        u = [int(v) for v in u]
        f, tau = orc.track_params(seed, g, n_f, tau_max)
        for k in range(3):   # f_k is the integer with f 2^64 <= u n_f < (f + 1) 2^64
            assert f[k] * 2 ** 64 <= u[k] * n_f < (f[k] + 1) * 2 ** 64
        unit = Fraction(2 * (u[3] >> 12) + 1, 2 ** 52) - 1
        assert -1 < unit < 1
        assert tau == float(Fraction(tau_max) * unit)   # one correctly rounded product


def test_track_params_uniform(orc):
    n_f, seed, n = 7, 3, 70_000
    counts = np.zeros((3, n_f))
    taus = np.zeros(n)
    for g in range(n):
        f, tau = orc.track_params(seed, g, n_f, 1.0)
        for k in range(3):
            counts[k, f[k]] += 1
        taus[g] = tau
    exp = n / n_f
    chi2 = ((counts - exp) ** 2 / exp).sum(axis=1)
    assert np.all(chi2 < 30.0)           # 6 dof: p < 1e-4 beyond 30
    assert abs(taus.mean()) < 0.02 and abs(taus.var() - 1 / 3) < 0.01
    assert taus.min() > -1 and taus.max() < 1


# ---------------------------------------------------------------- rasterisation
@pytest.mark.parametrize("n_t", [2, 3, 5, 17])
def test_rasterise_exhaustive_tiny(orc, n_t):
    n_f = 8
    for f0 in range(n_f):
        for f1 in range(n_f):
            for f2 in range(n_f):
                b = orc.track_bins((f0, f1, f2), n_t)
                np.testing.assert_array_equal(b, bezier_bins_exact((f0, f1, f2), n_t))


def test_rasterise_random_large(orc):
    rng = np.random.default_rng(0)
    for n_t, n_f in [(500, 1600), (200, 100), (1000, 2000), (101, 151)]:
        for _ in range(20):
            f = tuple(int(v) for v in rng.integers(0, n_f, 3))
            np.testing.assert_array_equal(orc.track_bins(f, n_t), bezier_bins_exact(f, n_t))


def test_rasterise_invariants(orc):
    rng = np.random.default_rng(1)
    for _ in range(200):
        n_t = int(rng.integers(2, 300))
        n_f = int(rng.integers(1, 3000))
        f = [int(v) for v in rng.integers(0, n_f, 3)]
        b = orc.track_bins(f, n_t)
        assert b[0] == f[0] and b[-1] == f[2]                    # endpoints
        assert b.min() >= min(f) and b.max() <= max(f)           # convex hull
        rev = orc.track_bins((f[2], f[1], f[0]), n_t)            # time reversal
        np.testing.assert_array_equal(rev[::-1], b)
    c = 37
    np.testing.assert_array_equal(orc.track_bins((c, c, c), 64), np.full(64, c))
    # f1 midway between f0 and f2: the curve is the straight line, rounded halves up
    n_t = 41
    b = orc.track_bins((10, 30, 50), n_t)
    M = n_t - 1
    line = [math.floor(Fraction(10) + Fraction(40 * j, M) + Fraction(1, 2)) for j in range(n_t)]
    np.testing.assert_array_equal(b, line)


# ---------------------------------------------------------------- statistic
def _tiny_map(seed, n_t, n_f, per_pixel_sigma=True):
    rng = np.random.default_rng(seed)
    y = (rng.standard_normal((n_t, n_f)) + 1j * rng.standard_normal((n_t, n_f))).astype(np.complex64)
    sig = rng.uniform(0.5, 2.0, (n_t, n_f) if per_pixel_sigma else n_f).astype(np.float32)
    return y, sig


@pytest.mark.parametrize("paper_mode", [False, True])
def test_brute_force_enumeration(orc, paper_mode):
    """Every template (f0, f1, f2) on a 5 x 6 map at several delays vs a direct
    complex-exponential evaluation of Eq. 7 over exactly rasterised pixels."""
    n_t, n_f, f_min, df = 5, 6, 100.0, 1.0
    y, sig = _tiny_map(4, n_t, n_f)
    om = orc.OracleMap(y, sig, f_min, df, sigma_per_freq=False, paper_mode=paper_mode)
    trip = np.array([(a, b, c) for a in range(n_f) for b in range(n_f) for c in range(n_f)], dtype=np.uint32)
    for tau in [-0.0093, -0.001, 0.0, 0.0025, 0.00999]:
        got = om.score_explicit(trip, np.full(len(trip), tau))
        ref = [brute_snr(y, sig, f_min, df, bezier_bins_exact(t, n_t), tau, paper_mode) for t in trip]
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)


def brute_snr_notched(y, sigma_full, f_min, df, bins, tau, paper_mode=False):
    """Eq. 7 over the template's pixels that are not notched (sigma = +inf):
    those add nothing to S or W; the paper form keeps N = the pixel count; no
    un-notched pixel at all (weighted form) gives 0."""
    j = np.arange(len(bins))
    s = sigma_full[j, bins].astype(np.float64)
    keep = np.isfinite(s)
    yv = y[j, bins].astype(np.complex128)[keep]
    s, fr = s[keep], f_min + bins[keep] * df
    rot = np.exp(2j * np.pi * fr * tau)
    if paper_mode:
        return float(np.sum((rot * (yv / s)).real) / len(bins))
    W = np.sum(s ** -2.0)
    return float(np.sum((rot * yv / s ** 2).real) / np.sqrt(W)) if W > 0 else 0.0


@pytest.mark.parametrize("paper_mode", [False, True])
def test_notched_pixels_brute_force(orc, paper_mode):
    """Fig. 1's notched (black) lines: pixels with sigma = +inf, whatever y holds
    there (NaN here), add nothing; every template of a 5 x 6 map at several
    delays against the direct evaluation over the remaining pixels."""
    n_t, n_f, f_min, df = 5, 6, 100.0, 1.0
    y, sig = _tiny_map(8, n_t, n_f)
    rng = np.random.default_rng(9)
    notch = rng.random((n_t, n_f)) < 0.3
    notch[:, 2] = True                              # a whole notched line
    sig = sig.copy()
    sig[notch] = np.inf
    y = y.copy()
    y[notch] = np.complex64(complex(np.nan, np.nan))
    om = orc.OracleMap(y, sig, f_min, df, sigma_per_freq=False, paper_mode=paper_mode)
    trip = np.array([(a, b, c) for a in range(n_f) for b in range(n_f) for c in range(n_f)], dtype=np.uint32)
    for tau in [-0.0071, 0.0, 0.0043]:
        got = om.score_explicit(trip, np.full(len(trip), tau))
        ref = [brute_snr_notched(y, sig, f_min, df, bezier_bins_exact(t, n_t), tau, paper_mode) for t in trip]
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)
    assert om.score_explicit(np.array([(2, 2, 2)]), np.array([0.001]))[0] == 0.0   # all its pixels notched


def test_notched_injection_closed_form(orc):
    """Zero-noise injection on a template that crosses a notched band: the SNR
    at the injected delay is A sqrt(sum of sigma^-2 over its un-notched pixels)."""
    n_t, n_f, f_min, df = 64, 200, 40.0, 0.5
    sig = (1.0 + np.linspace(0, 3, n_f) ** 2).astype(np.float32)
    sig[90:110] = np.inf                             # a notched band the template crosses
    f = (17, 180, 60)
    b = bezier_bins_exact(f, n_t)
    assert np.any((b >= 90) & (b < 110)) and np.any((b < 90) | (b >= 110))
    A, tau_s = 2.5, -0.0061
    y = np.zeros((n_t, n_f), np.complex64)
    y[np.arange(n_t), b] = (A * np.exp(-2j * np.pi * (f_min + b * df) * tau_s)).astype(np.complex64)
    om = orc.OracleMap(y, sig, f_min, df, True)
    s = sig.astype(np.float64)[b]
    W = float(np.sum(s[np.isfinite(s)] ** -2.0))
    got = om.score_explicit(np.array([f]), np.array([tau_s]))[0]
    assert got == pytest.approx(A * math.sqrt(W), rel=1e-6)
    everywhere = orc.OracleMap(y, np.full(n_f, np.inf, np.float32), f_min, df, True)
    assert everywhere.score_explicit(np.array([f]), np.array([tau_s]))[0] == 0.0   # no data at all


def test_eq5_special_case_real_map(orc):
    """tau = 0 on a real-valued map reduces Eq. 7 to Eq. 5: the plain mean of rho over the pixels."""
    n_t, n_f = 30, 40
    rng = np.random.default_rng(5)
    rho = rng.standard_normal((n_t, n_f)).astype(np.float32)
    y = rho.astype(np.complex64)
    om = orc.OracleMap(y, np.ones(n_f, np.float32), 50.0, 1.0, True, paper_mode=True)
    for f in [(3, 30, 10), (0, 39, 39), (20, 20, 20)]:
        got = om.score_explicit(np.array([f]), np.array([0.0]))[0]
        b = bezier_bins_exact(f, n_t)
        assert got == pytest.approx(float(np.mean(rho[np.arange(n_t), b].astype(np.float64))), rel=1e-13)


def test_zero_noise_injection_closed_form(orc):
    """Signal only on the template's own pixels, arriving with delay tau_s:
    SNR(tau_s) = A sqrt(sum sigma^-2) exactly (weighted form)."""
    n_t, n_f, f_min, df = 64, 200, 40.0, 0.5
    sig = (1.0 + np.linspace(0, 3, n_f) ** 2).astype(np.float32)
    f = (17, 180, 60)
    b = bezier_bins_exact(f, n_t)
    A, tau_s = 2.5, -0.0061
    y = np.zeros((n_t, n_f), np.complex64)
    fr = f_min + b * df
    y[np.arange(n_t), b] = (A * np.exp(-2j * np.pi * fr * tau_s)).astype(np.complex64)
    om = orc.OracleMap(y, sig, f_min, df, True)
    W = float(np.sum(sig.astype(np.float64)[b] ** -2.0))
    yv = y[np.arange(n_t), b].astype(np.complex128)  # the stored (float32-rounded) signal
    exact_store = float(np.sum((yv * np.exp(2j * np.pi * fr * tau_s)).real * sig.astype(np.float64)[b] ** -2.0)) / math.sqrt(W)
    got = om.score_explicit(np.array([f]), np.array([tau_s]))[0]
    assert got == pytest.approx(exact_store, rel=1e-12)
    assert got == pytest.approx(A * math.sqrt(W), rel=1e-6)      # float32 storage of y only
    # a template outside the signal's convex hull [17, 180] sees none of it
    assert om.score_explicit(np.array([(195, 195, 195)]), np.array([tau_s]))[0] == 0.0


def test_eq3_single_frequency_ratio(orc):
    """Eq. 3: a constant-frequency signal scored with delay error dtau keeps cos(2 pi f dtau) of its SNR."""
    n_t, n_f, f_min, df = 50, 1001, 0.0, 1.0
    c = 440
    y = np.zeros((n_t, n_f), np.complex64)
    tau_s = 0.0012
    y[:, c] = np.complex64(np.exp(-2j * np.pi * (f_min + c * df) * tau_s))
    om = orc.OracleMap(y, np.ones(n_f, np.float32), f_min, df, True)
    s0 = om.score_explicit(np.array([(c, c, c)]), np.array([tau_s]))[0]
    for dt in [-0.004, -0.0005, 0.0001, 0.0007, 0.003]:
        s = om.score_explicit(np.array([(c, c, c)]), np.array([tau_s + dt]))[0]
        assert s / s0 == pytest.approx(math.cos(2 * math.pi * (f_min + c * df) * dt), abs=1e-6)


def test_paper_worked_numbers(orc):
    """The paper's printed tolerances and stripe width, reproduced through the oracle."""
    g = json.load(open(GOLDEN))
    R = g["timing_tolerance"]["R"]
    for case in g["timing_tolerance"]["cases"]:
        f_hz, dtau = case["f_hz"], case["dtau_s"]
        n_t, n_f = 20, 3
        y = np.zeros((n_t, n_f), np.complex64)
        y[:, 1] = 1.0                              # delay 0 signal at bin 1 = f_hz
        om = orc.OracleMap(y, np.ones(n_f, np.float32), f_hz - 1.0, 1.0, True)
        s0 = om.score_explicit(np.array([(1, 1, 1)]), np.array([0.0]))[0]
        s = om.score_explicit(np.array([(1, 1, 1)]), np.array([dtau]))[0]
        # the printed delays are the R >= 90% bound rounded to two figures
        assert s / s0 == pytest.approx(R, abs=2e-3)
        bound = math.acos(R) / (2 * math.pi * f_hz)
        assert bound == pytest.approx(dtau, rel=0.01)
    st = g["minimum_stripe"]
    n_t, n_f = 10, 2
    y = np.zeros((n_t, n_f), np.complex64)
    y[:, 1] = 1.0
    om = orc.OracleMap(y, np.ones(n_f, np.float32), st["df_min_hz"] - 1.0, 1.0, True)
    # at f = 1/(4 dtau_max) the cross-power has rotated a quarter turn: it vanishes
    assert abs(om.score_explicit(np.array([(1, 1, 1)]), np.array([st["dtau_max_s"]]))[0]) < 1e-12
    # and just below / above the stripe edge it has the sign the paper describes
    om2 = orc.OracleMap(y, np.ones(n_f, np.float32), st["df_min_hz"] - 2.0, 1.0, True)
    assert om2.score_explicit(np.array([(1, 1, 1)]), np.array([st["dtau_max_s"]]))[0] > 0
    om3 = orc.OracleMap(y, np.ones(n_f, np.float32), st["df_min_hz"], 1.0, True)
    assert om3.score_explicit(np.array([(1, 1, 1)]), np.array([st["dtau_max_s"]]))[0] < 0


def test_linearity_sign_and_time_reversal(orc):
    n_t, n_f = 40, 64
    y1, sig = _tiny_map(6, n_t, n_f)
    y2, _ = _tiny_map(7, n_t, n_f)
    rng = np.random.default_rng(8)
    f3 = rng.integers(0, n_f, (50, 3)).astype(np.uint32)
    tau = rng.uniform(-0.01, 0.01, 50)
    m1 = orc.OracleMap(y1, sig, 80.0, 0.5, False)
    m2 = orc.OracleMap(y2, sig, 80.0, 0.5, False)
    m12 = orc.OracleMap((y1.astype(np.complex128) + y2).astype(np.complex64), sig, 80.0, 0.5, False)
    mneg = orc.OracleMap(-y1, sig, 80.0, 0.5, False)
    s1, s2, s12 = m1.score_explicit(f3, tau), m2.score_explicit(f3, tau), m12.score_explicit(f3, tau)
    np.testing.assert_allclose(s12, s1 + s2, atol=1e-5)          # y1+y2 rounded to float32
    np.testing.assert_allclose(mneg.score_explicit(f3, tau), -s1, rtol=0, atol=0)
    # reversing time and swapping f0 <-> f2 visits the same pixels in the opposite order
    mrev = orc.OracleMap(y1[::-1].copy(), sig[::-1].copy(), 80.0, 0.5, False)
    np.testing.assert_allclose(mrev.score_explicit(f3[:, ::-1].copy(), tau), s1, rtol=1e-12, atol=1e-12)
    # the per-frequency sigma row equals the same sigma broadcast per pixel
    srow = sig[0]
    ma = orc.OracleMap(y1, srow, 80.0, 0.5, True)
    mb = orc.OracleMap(y1, np.ascontiguousarray(np.broadcast_to(srow, (n_t, n_f))), 80.0, 0.5, False)
    np.testing.assert_array_equal(ma.score_explicit(f3, tau), mb.score_explicit(f3, tau))


def test_noise_only_unit_variance(orc):
    """Weighted form: under Gaussian noise with Re, Im ~ N(0, sigma^2) each, any
    fixed template's SNR has mean 0 and variance 1 (it is a sum of independent
    sigma^-1-scaled unit normals divided by sqrt(sum sigma^-2))."""
    n_t, n_f, n = 50, 30, 2000
    rng = np.random.default_rng(10)
    s = np.zeros(n)
    for r in range(n):   # one map realisation per sample: samples independent
        sig = rng.uniform(0.3, 3.0, (n_t, n_f)).astype(np.float32)
        y = ((rng.standard_normal((n_t, n_f)) + 1j * rng.standard_normal((n_t, n_f))) * sig).astype(np.complex64)
        om = orc.OracleMap(y, sig, 100.0, 1.0, False)
        s[r] = om.score_explicit(rng.integers(0, n_f, (1, 3)), rng.uniform(-0.01, 0.01, 1))[0]
    assert abs(s.mean()) < 0.1 and abs(s.var() - 1.0) < 0.15   # 4.5 and 4.7 standard errors


# ---------------------------------------------------------------- range driver and selection
def test_score_range_matches_explicit(orc):
    n_t, n_f = 60, 90
    y, sig = _tiny_map(11, n_t, n_f, per_pixel_sigma=False)
    om = orc.OracleMap(y, sig, 100.0, 1.0, True)
    seed, off, T, tmax = 77, 1000, 500, 0.01
    a = om.score_range(seed, off, T, tmax, nthreads=1)
    b = om.score_range(seed, off, T, tmax, nthreads=7)
    np.testing.assert_array_equal(a, b)
    f3, tau = zip(*[orc.track_params(seed, off + i, n_f, tmax) for i in range(T)])
    np.testing.assert_array_equal(a, om.score_explicit(np.array(f3), np.array(tau)))


def test_topk_order_and_split(orc):
    rng = np.random.default_rng(12)
    snr = np.round(rng.standard_normal(5000), 2)   # many exact ties
    v, i = orc.topk(snr, 100, 64)
    order = np.lexsort((np.arange(5000), -snr))[:64]
    np.testing.assert_array_equal(i, order + 100)
    np.testing.assert_array_equal(v, snr[order])
    # Sec. V: runs over disjoint index ranges combine by taking the largest
    a = 1234
    v1, i1 = orc.topk(snr[:a], 100, 64)
    v2, i2 = orc.topk(snr[a:], 100 + a, 64)
    vv = np.concatenate([v1, v2]); ii = np.concatenate([i1, i2])
    o = np.lexsort((ii, -vv))[:64]
    np.testing.assert_array_equal(ii[o], i)
    # all ties: the smallest indices win
    v, i = orc.topk(np.zeros(300), 7, 10)
    np.testing.assert_array_equal(i, np.arange(7, 17))


# ---------------------------------------------------------------- interpolated statistic (refinement)
def _bezier_x(f, n_t):
    M = n_t - 1
    j = np.arange(n_t)
    return ((M - j) ** 2 * f[0] + 2 * (M - j) * j * f[1] + j ** 2 * f[2]) / M ** 2


def test_interp_reduces_to_discrete_at_integer_bins(orc):
    n_t, n_f = 40, 60
    y, sig = _tiny_map(30, n_t, n_f)
    for paper in (False, True):
        om = orc.OracleMap(y, sig, 70.0, 0.5, False, paper_mode=paper)
        for c in (0, 7, 31, 59):
            for tau in (-0.006, 0.0, 0.0041):
                d = om.score_explicit(np.array([(c, c, c)]), np.array([tau]))[0]
                s = om.interp_score(np.array([(c, c, c)], float), np.array([tau]))[0]
                assert s == pytest.approx(d, rel=1e-12, abs=1e-12)


def test_interp_exact_on_maps_linear_in_frequency(orc):
    """z(j, k) = A_j + B_j k: linear interpolation is exact, so the statistic is
    the plain sum over the continuous curve."""
    n_t, n_f, f_min, df = 30, 80, 50.0, 0.5
    rng = np.random.default_rng(31)
    A = rng.standard_normal(n_t) + 1j * rng.standard_normal(n_t)
    B = (rng.standard_normal(n_t) + 1j * rng.standard_normal(n_t)) * 0.05
    k = np.arange(n_f)
    y = (A[:, None] + B[:, None] * k[None, :]).astype(np.complex64)
    om = orc.OracleMap(y, np.ones(n_f, np.float32), f_min, df, True)
    yd = y.astype(np.complex128)
    for _ in range(20):
        f = rng.uniform(1, n_f - 2, 3)
        tau = rng.uniform(-0.01, 0.01)
        x = _bezier_x(f, n_t)
        kk = np.minimum(np.floor(x).astype(int), n_f - 2)
        a = x - kk
        z = (1 - a) * yd[np.arange(n_t), kk] + a * yd[np.arange(n_t), kk + 1]
        S = np.sum((np.exp(2j * np.pi * (f_min + x * df) * tau) * z).real)
        assert om.interp_score(f[None], np.array([tau]))[0] == pytest.approx(S / np.sqrt(n_t), rel=1e-9)


def test_interp_constant_frequency_closed_form(orc):
    """A map constant along frequency: any real constant template c sees
    sum_j Re[exp(2 pi i (f_min + c df) tau) z_j] (continuous Eq. 3 phase)."""
    n_t, n_f, f_min, df = 25, 40, 100.0, 1.0
    rng = np.random.default_rng(32)
    zj = (rng.standard_normal(n_t) + 1j * rng.standard_normal(n_t)).astype(np.complex64)
    y = np.repeat(zj[:, None], n_f, axis=1)
    om = orc.OracleMap(y, np.full(n_f, 2.0, np.float32), f_min, df, True)
    for c in (3.25, 17.5, 38.9):
        for tau in (-0.0031, 0.0077):
            S = np.sum((np.exp(2j * np.pi * (f_min + c * df) * tau) * zj.astype(np.complex128) / 4.0).real)
            W = n_t / 4.0
            got = om.interp_score(np.array([(c, c, c)]), np.array([tau]))[0]
            assert got == pytest.approx(S / np.sqrt(W), rel=1e-10)


@pytest.mark.parametrize("paper", [False, True])
def test_interp_gradient_matches_finite_differences(orc, paper):
    n_t, n_f = 50, 120
    y, sig = _tiny_map(33, n_t, n_f)
    om = orc.OracleMap(y, sig, 40.0, 0.5, False, paper_mode=paper)
    rng = np.random.default_rng(34)
    checked = 0
    while checked < 25:
        f = rng.uniform(2, n_f - 3, 3)
        tau = rng.uniform(-0.01, 0.01)
        x = _bezier_x(f, n_t)
        if np.min(np.abs(x - np.round(x))) < 1e-3:      # stay off the bin knots
            continue
        _, g = om.interp_score(f[None], np.array([tau]), grad=True)
        hf, ht = 1e-6, 1e-10
        fd = []
        for q in range(3):
            e = np.zeros(3)
            e[q] = hf
            fd.append((om.interp_score((f + e)[None], np.array([tau]))[0] -
                       om.interp_score((f - e)[None], np.array([tau]))[0]) / (2 * hf))
        fd.append((om.interp_score(f[None], np.array([tau + ht]))[0] -
                   om.interp_score(f[None], np.array([tau - ht]))[0]) / (2 * ht))
        np.testing.assert_allclose(g[0], fd, rtol=2e-5, atol=2e-5 * np.max(np.abs(fd)))
        checked += 1


# ---------------------------------------------------------------- general templates (six random numbers)
from decimal import Decimal, getcontext  # noqa: E402


def general_bins_decimal(t, f, n_t):
    """Independent rasteriser: solve t(xi) = j with 60-digit decimals, take the
    nearest bin of f(xi_j) (halves up).  Columns where f(xi_j) is within 1e-40
    of a half-integer are decided exactly with fractions when Delta is a square,
    else reported as None (undecided here)."""
    getcontext().prec = 60
    t0, t1, t2 = (Decimal(v) for v in t)
    f0, f1, f2 = (Decimal(v) for v in f)
    a, b = t0 - 2 * t1 + t2, 2 * (t1 - t0)
    out = []
    for j in range(n_t):
        if j < t[0] or j > t[2]:
            out.append(-1)
            continue
        if j == t[0]:
            out.append(int(f[0]))
            continue
        dj = Decimal(j) - t0
        delta = b * b + 4 * a * dj
        xi = 2 * dj / (delta.sqrt() + b)
        fx = (1 - xi) ** 2 * f0 + 2 * (1 - xi) * xi * f1 + xi ** 2 * f2
        k = int((fx + Decimal("0.5")).to_integral_value(rounding="ROUND_FLOOR"))
        frac = fx + Decimal("0.5") - k
        if frac < Decimal("1e-40") or frac > 1 - Decimal("1e-40"):
            di = int(b * b + 4 * a * dj)
            r = math.isqrt(di)
            if r * r != di:
                out.append(None)
                continue
            xr = Fraction(2 * (j - t[0]), r + int(b))
            fr = (1 - xr) ** 2 * f[0] + 2 * (1 - xr) * xr * f[1] + xr ** 2 * f[2]
            k = math.floor(fr + Fraction(1, 2))
        out.append(k)
    return out


def _same_except_undecided(got, ref):
    for g, r in zip(got, ref):
        if r is not None:
            assert g == r, (list(got), ref)


def test_general_times_definition(orc):
    n_t, t_min, seed = 200, 30, 5
    M = n_t - 1
    for g in [0, 1, 17, 123456, 2 ** 50 + 1]:
        prev = [g - 1, 1, 0, 0] if g else [2 ** 64 - 1, 0, 0, 0]       # numpy steps the counter first
        v = [int(x) for x in np.random.Philox(key=np.array([seed, 0], dtype=np.uint64),
                                              counter=np.array(prev, dtype=np.uint64)).random_raw(4)]
        t = orc.track_times(seed, g, n_t, t_min)
        d = t[2] - t[0]
        assert (d - t_min) * 2 ** 64 <= v[0] * (M - t_min + 1) < (d - t_min + 1) * 2 ** 64
        assert t[0] * 2 ** 64 <= v[1] * (M - d + 1) < (t[0] + 1) * 2 ** 64
        assert (t[1] - t[0]) * 2 ** 64 <= v[2] * (d + 1) < (t[1] - t[0] + 1) * 2 ** 64
        assert 0 <= t[0] <= t[1] <= t[2] <= M and d >= t_min


@pytest.mark.parametrize("n_t", [3, 5, 9])
def test_general_rasteriser_exhaustive_tiny(orc, n_t):
    n_f = 6
    for t0 in range(n_t):
        for t2 in range(t0 + 1, n_t):
            for t1 in range(t0, t2 + 1):
                for f in [(0, 5, 2), (3, 3, 3), (5, 0, 5), (1, 4, 0), (2, 2, 5)]:
                    got = orc.track_bins_general((t0, t1, t2), f, n_t, n_f)
                    _same_except_undecided(got, general_bins_decimal((t0, t1, t2), f, n_t))


def test_general_rasteriser_random_and_invariants(orc):
    rng = np.random.default_rng(40)
    for _ in range(60):
        n_t = int(rng.integers(3, 400))
        n_f = int(rng.integers(2, 3000))
        t0, t2 = sorted(int(v) for v in rng.choice(n_t, 2, replace=False))
        t1 = int(rng.integers(t0, t2 + 1))
        f = [int(v) for v in rng.integers(0, n_f, 3)]
        b = orc.track_bins_general((t0, t1, t2), f, n_t, n_f)
        _same_except_undecided(b, general_bins_decimal((t0, t1, t2), f, n_t))
        assert b[t0] == f[0] and b[t2] == f[2]
        span = b[t0:t2 + 1]
        assert span.min() >= min(f) and span.max() <= max(f) and np.all(b[:t0] == -1) and np.all(b[t2 + 1:] == -1)
        M = n_t - 1   # time reversal: the same curve traversed backwards
        rb = orc.track_bins_general((M - t2, M - t1, M - t0), f[::-1], n_t, n_f)
        np.testing.assert_array_equal(rb[::-1], b)
    # middle time at the midpoint: the pinned rasteriser
    for n_t in (5, 21, 201):
        M = n_t - 1
        for f in [(3, 90, 40), (0, 0, 77), (99, 1, 50)]:
            np.testing.assert_array_equal(orc.track_bins_general((0, M // 2, M), f, n_t, 100), orc.track_bins(f, n_t))


def test_general_score_bruteforce(orc):
    n_t, n_f = 30, 40
    y, sig = _tiny_map(41, n_t, n_f)
    rng = np.random.default_rng(42)
    for paper in (False, True):
        om = orc.OracleMap(y, sig, 60.0, 0.5, False, paper_mode=paper)
        t3, f3, taus, ref = [], [], [], []
        for _ in range(40):
            t0, t2 = sorted(int(v) for v in rng.choice(n_t, 2, replace=False))
            t1 = int(rng.integers(t0, t2 + 1))
            f = [int(v) for v in rng.integers(0, n_f, 3)]
            tau = float(rng.uniform(-0.01, 0.01))
            bins = orc.track_bins_general((t0, t1, t2), f, n_t, n_f)
            j = np.nonzero(bins >= 0)[0]
            yv = y[j, bins[j]].astype(np.complex128)
            s = sig[j, bins[j]].astype(np.float64)
            rot = np.exp(2j * np.pi * (60.0 + bins[j] * 0.5) * tau)
            ref.append(np.sum((rot * yv / s).real) / len(j) if paper else
                       np.sum((rot * yv / s ** 2).real) / np.sqrt(np.sum(s ** -2.0)))
            t3.append((t0, t1, t2)); f3.append(f); taus.append(tau)
        np.testing.assert_allclose(om.score_explicit_general(t3, f3, taus), ref, rtol=1e-12, atol=1e-12)


def test_delay_prior_quantiles(orc):
    """Delays drawn through a quantile table follow its piecewise-linear CDF (KS),
    and a two-point table from -tau_max to tau_max is the uniform prior."""
    from scipy import stats
    q = np.array([-0.004, -0.0035, -0.001, 0.0, 0.0005, 0.0042])
    taus = np.array([orc.track_params_prior(7, g, 100, q)[1] for g in range(20000)])
    assert taus.min() >= q[0] and taus.max() <= q[-1]
    probs = np.linspace(0, 1, q.size)
    cdf = lambda x: np.interp(x, q, probs)   # noqa: E731
    assert stats.kstest(taus, cdf).pvalue > 1e-4
    uni = np.array([orc.track_params_prior(7, g, 100, [-0.01, 0.01])[1] for g in range(200)])
    ref = np.array([orc.track_params(7, g, 100, 0.01)[1] for g in range(200)])
    np.testing.assert_allclose(uni, ref, rtol=0, atol=1e-17)
    # bins do not depend on the prior
    assert orc.track_params_prior(7, 5, 100, q)[0] == orc.track_params(7, 5, 100, 0.01)[0]
