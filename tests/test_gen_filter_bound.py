"""The error bound behind the general-template filter, checked on the host.

The GPU decides a pixel of a general template from an FP32 estimate of f(xi_j)
when it lies farther than a margin (twice a derived bound) from a rounding
boundary, and runs the exact integer test otherwise.  This test reproduces the
estimate's FP32 arithmetic exactly in numpy (IEEE float32 sqrt, add and divide;
each FMA as an exact float64 sum rounded once to float32, exact here because
every operand is short) and compares it with f(xi_j) in 64-bit-mantissa
precision over random curves and columns: the error must stay below the bound
(half the margin, less its absolute floor)."""
import numpy as np

U = 2.0 ** -24


def bound(f0, f1, f2):
    G = 2 * (f1 - f0)
    F = f0 - 2 * f1 + f2
    gmax = np.maximum(np.abs(G), np.abs(G + 2 * F)).astype(np.float64)
    fmax = np.maximum(f0, np.maximum(f1, f2)).astype(np.float64)
    return 2.4e-7 * (gmax + 1) + 1.8e-7 * (fmax + 1) + 6e-8


def fma32(a, b, c):
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(np.float32)


def test_estimate_error_within_bound():
    rng = np.random.default_rng(2024)
    n = 400_000
    n_t, n_f = 4096, 8192
    t = np.sort(rng.integers(0, n_t, (n, 3)), axis=1)
    ok = t[:, 0] < t[:, 2]
    t = t[ok]
    f = rng.integers(0, n_f, (len(t), 3))
    t0, t1, t2 = t[:, 0], t[:, 1], t[:, 2]
    j = t0 + 1 + (rng.random(len(t)) * (t2 - t0)).astype(np.int64)   # j in (t0, t2]
    A = t0 - 2 * t1 + t2
    B = 2 * (t1 - t0)
    F = f[:, 0] - 2 * f[:, 1] + f[:, 2]
    G = 2 * (f[:, 1] - f[:, 0])
    du = j - t0
    Dl = B * B + 4 * A * du                       # exact; 0 only at xi = 1 with t1 = t2 (then B > 0)
    assert Dl.min() >= 0 and Dl.max() < 2 ** 27 and np.all((Dl > 0) | (B > 0))
    # the kernel's FP32 estimate
    s = np.sqrt(Dl.astype(np.float32))
    xi = (2 * du).astype(np.float32) / (s + B.astype(np.float32))
    inner = fma32(F.astype(np.float32), xi, G.astype(np.float32))
    fx = fma32(xi, inner, f[:, 0].astype(np.float32))
    h = fx + np.float32(0.5)
    # f(xi_j) + 1/2 in extended precision
    L = np.longdouble
    xl = (2 * du).astype(L) / (np.sqrt(Dl.astype(L)) + B.astype(L))
    exact = f[:, 0].astype(L) + xl * (G.astype(L) + F.astype(L) * xl) + L(0.5)
    err = np.abs(h.astype(L) - exact).astype(np.float64)
    b = bound(f[:, 0], f[:, 1], f[:, 2])
    ratio = err / b
    assert ratio.max() < 1.0, ratio.max()
    # the bound is not vacuous: the estimate errs by a sizeable part of it somewhere
    assert ratio.max() > 0.05
