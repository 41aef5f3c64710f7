"""Helpers for comparing the CUDA path with the FP64 oracle.

Tolerance: SNRs within 1e-5 relative of the FP64 oracle in FP32.  Relative error
is ill-conditioned for SNRs near zero, so each template is held to
    |SNR_gpu - SNR_oracle| <= RTOL * max(|SNR_oracle|, sum_j |z_j| / norm)
where norm is sqrt(sum_j w_j) (weighted) or N (paper form): the FP32 pixel
storage, the fixed-point phase and the FP32 sum all err in proportion to the
pixel magnitudes |z_j|, not to the (possibly cancelling) SNR.  Selected
top-k values are also held to plain relative 1e-5.
"""
import numpy as np

RTOL = 1e-5


def scale(extras, paper_mode, n_t):
    norm = n_t if paper_mode else np.sqrt(extras["W"])
    return extras["absz"] / norm


def assert_snr_close(gpu, orc_snr, extras, paper_mode, n_t, rtol=RTOL, what=""):
    gpu = np.asarray(gpu, dtype=np.float64)
    bound = rtol * np.maximum(np.abs(orc_snr), scale(extras, paper_mode, n_t))
    err = np.abs(gpu - orc_snr)
    bad = np.nonzero(err > bound)[0]
    if bad.size:
        i = bad[0]
        raise AssertionError(f"{what}: {bad.size}/{gpu.size} SNRs out of tolerance; first i={i} "
                             f"gpu={gpu[i]!r} oracle={orc_snr[i]!r} err={err[i]:.3g} bound={bound[i]:.3g}")
    return float(np.max(err / np.maximum(bound / rtol, 1e-300))) if gpu.size else 0.0


def assert_topk_matches(hits, orc_all, offset, k, rtol=RTOL, what=""):
    """Top-k of the GPU vs the oracle's full SNR array (template g at orc_all[g - offset]).

    Values: relative rtol against the oracle's k largest.  Indices: equal to the
    oracle's, or else the template the GPU ranked i-th has an oracle SNR within
    2 rtol of the oracle's i-th value (a near-tie the FP32 path cannot order)."""
    import oracle
    orc_vals, orc_idx = oracle.topk(orc_all, offset, k)
    g_vals = np.asarray(hits["snr"], dtype=np.float64)
    g_idx = np.asarray(hits["index"], dtype=np.int64)
    assert len(set(g_idx.tolist())) == k, f"{what}: duplicate indices"
    np.testing.assert_allclose(g_vals, orc_vals, rtol=rtol, atol=0, err_msg=what)
    assert np.all(np.diff(g_vals) <= 0), f"{what}: not sorted"
    for i in range(k):
        if g_idx[i] == orc_idx[i]:
            continue
        true_v = orc_all[g_idx[i] - offset]
        assert abs(true_v - orc_vals[i]) <= 2 * rtol * abs(orc_vals[i]), \
            f"{what}: rank {i}: gpu index {g_idx[i]} (oracle SNR {true_v!r}) vs oracle index {orc_idx[i]} ({orc_vals[i]!r})"
    return int(np.count_nonzero(g_idx != orc_idx))
