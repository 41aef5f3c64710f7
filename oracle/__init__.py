"""FP64 CPU oracle for the all-sky seedless-clustering scorer (test infrastructure).

Only the tests, the package's ``smoke()`` check and the benchmark's CPU-baseline
leg may import this package.  It is independent of the CUDA library: the
arithmetic lives in ``stk_oracle.c`` (plain binary64 C), and this module only
marshals numpy arrays through ctypes.  Each function names the part of the
paper it follows (Sec. III templates and Eq. 7 statistic; Sec. V combination of
runs by a maximum).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    """Load (building first if needed) liboracle.so."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        u64p = C.POINTER(C.c_uint64)
        u32p = C.POINTER(C.c_uint32)
        i32p = C.POINTER(C.c_int32)
        dp = C.POINTER(C.c_double)
        fp = C.POINTER(C.c_float)
        L.orc_philox4x64_10.argtypes = [u64p, u64p, u64p]
        L.orc_track_params.argtypes = [C.c_uint64, C.c_uint64, C.c_int, C.c_double, u32p, dp]
        L.orc_track_bins.argtypes = [u32p, C.c_int, i32p]
        L.orc_map_create.argtypes = [fp, fp, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                                     C.c_int]
        L.orc_map_create.restype = C.c_void_p
        L.orc_map_free.argtypes = [C.c_void_p]
        L.orc_score_explicit.argtypes = [C.c_void_p, u32p, dp, C.c_uint64, dp, dp, dp, dp, dp]
        L.orc_score_range.argtypes = [C.c_void_p, C.c_uint64, C.c_uint64, C.c_uint64, C.c_double,
                                      C.c_int, dp]
        L.orc_score_range.restype = C.c_int
        L.orc_score_range_scale.argtypes = [C.c_void_p, C.c_uint64, C.c_uint64, C.c_uint64, C.c_double,
                                            C.c_int, dp, dp]
        L.orc_score_range_scale.restype = C.c_int
        L.orc_interp_explicit.argtypes = [C.c_void_p, dp, dp, C.c_uint64, dp, dp]
        L.orc_track_times.argtypes = [C.c_uint64, C.c_uint64, C.c_int, C.c_int, u32p]
        L.orc_track_params_prior.argtypes = [C.c_uint64, C.c_uint64, C.c_int, dp, C.c_int, u32p, dp]
        L.orc_track_bins_general.argtypes = [u32p, u32p, C.c_int, C.c_int, i32p]
        L.orc_score_explicit_general.argtypes = [C.c_void_p, u32p, u32p, dp, C.c_uint64, dp]
        L.orc_score_range_ext.argtypes = [C.c_void_p, C.c_uint64, C.c_uint64, C.c_uint64, C.c_double, C.c_int,
                                          C.c_int, dp, C.c_int, C.c_int, dp]
        L.orc_score_range_ext.restype = C.c_int
        L.orc_score_range_ext_scale.argtypes = L.orc_score_range_ext.argtypes + [dp]
        L.orc_score_range_ext_scale.restype = C.c_int
        L.orc_topk.argtypes = [dp, C.c_uint64, C.c_uint64, C.c_int, dp, u64p]
        L.orc_topk.restype = C.c_int
        _lib = L
    return _lib


def _ptr(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def philox4x64_10(counter, key):
    """Philox4x64-10 block (Salmon et al., SC'11) for a 4-word counter and 2-word key."""
    ctr = np.asarray(counter, dtype=np.uint64).reshape(4).copy()
    k = np.asarray(key, dtype=np.uint64).reshape(2).copy()
    out = np.zeros(4, dtype=np.uint64)
    lib().orc_philox4x64_10(_ptr(ctr, C.c_uint64), _ptr(k, C.c_uint64), _ptr(out, C.c_uint64))
    return [int(v) for v in out]


def track_params(seed: int, g: int, n_f: int, tau_max: float):
    """Template g's control bins (f0, f1, f2) and delay tau (Sec. III)."""
    f = np.zeros(3, dtype=np.uint32)
    tau = C.c_double()
    lib().orc_track_params(seed, g, n_f, tau_max, _ptr(f, C.c_uint32), C.byref(tau))
    return tuple(int(v) for v in f), float(tau.value)


def track_bins(f, n_t: int) -> np.ndarray:
    """The template's pixel (frequency bin) in each of the n_t columns (Sec. III Bezier)."""
    fa = np.asarray(f, dtype=np.uint32).reshape(3).copy()
    out = np.zeros(n_t, dtype=np.int32)
    lib().orc_track_bins(_ptr(fa, C.c_uint32), n_t, _ptr(out, C.c_int32))
    return out


def track_times(seed: int, g: int, n_t: int, t_min: int):
    """Control times (t0, t1, t2) of general template g (Sec. III, six random numbers)."""
    t = np.zeros(3, dtype=np.uint32)
    lib().orc_track_times(seed, g, n_t, t_min, _ptr(t, C.c_uint32))
    return tuple(int(v) for v in t)


def track_params_prior(seed: int, g: int, n_f: int, quantiles):
    """Control bins and a delay drawn from a quantile table (Sec. VI sky-patch prior)."""
    q = np.ascontiguousarray(quantiles, dtype=np.float64)
    f = np.zeros(3, dtype=np.uint32)
    tau = C.c_double()
    lib().orc_track_params_prior(seed, g, n_f, _ptr(q, C.c_double), q.size, _ptr(f, C.c_uint32), C.byref(tau))
    return tuple(int(v) for v in f), float(tau.value)


def track_bins_general(t, f, n_t: int, n_f: int) -> np.ndarray:
    """Pixels of a general template: the nearest bin in each column t0..t2, -1 elsewhere."""
    ta = np.asarray(t, dtype=np.uint32).reshape(3).copy()
    fa = np.asarray(f, dtype=np.uint32).reshape(3).copy()
    out = np.zeros(n_t, dtype=np.int32)
    lib().orc_track_bins_general(_ptr(ta, C.c_uint32), _ptr(fa, C.c_uint32), n_t, n_f, _ptr(out, C.c_int32))
    return out


class OracleMap:
    """The map as the statistic reads it, held in binary64 by the C oracle."""

    def __init__(self, y, sigma, f_min: float, df: float, sigma_per_freq: bool,
                 paper_mode: bool = False):
        y = np.ascontiguousarray(y, dtype=np.complex64)
        s = np.ascontiguousarray(sigma, dtype=np.float32)
        n_t, n_f = y.shape
        if sigma_per_freq:
            assert s.shape == (n_f,)
        else:
            assert s.shape == (n_t, n_f)
        yf = y.view(np.float32)
        self.n_t, self.n_f = n_t, n_f
        self.f_min, self.df = float(f_min), float(df)
        self.paper_mode = bool(paper_mode)
        self._h = lib().orc_map_create(_ptr(yf, C.c_float), _ptr(s, C.c_float), int(sigma_per_freq),
                                       n_t, n_f, self.f_min, self.df, int(paper_mode))
        if not self._h:
            raise MemoryError("oracle map allocation failed")

    @classmethod
    def from_ftmap(cls, fm, paper_mode: bool = False):
        return cls(fm.y, fm.sigma, fm.f_min, fm.df, fm.sigma_per_freq, paper_mode)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_map_free(h)
            self._h = None

    def score_explicit(self, f3, tau, extras: bool = False):
        """Eq. 7 for explicit templates: f3 [n][3] bins, tau [n] seconds."""
        f3 = np.ascontiguousarray(f3, dtype=np.uint32).reshape(-1, 3)
        tau = np.ascontiguousarray(tau, dtype=np.float64).reshape(-1)
        n = f3.shape[0]
        assert tau.shape[0] == n
        snr = np.zeros(n)
        S = np.zeros(n); W = np.zeros(n); A = np.zeros(n); Z = np.zeros(n)
        lib().orc_score_explicit(self._h, _ptr(f3, C.c_uint32), _ptr(tau, C.c_double), n,
                                 _ptr(snr, C.c_double), _ptr(S, C.c_double), _ptr(W, C.c_double),
                                 _ptr(A, C.c_double), _ptr(Z, C.c_double))
        if extras:
            return snr, dict(S=S, W=W, absterm=A, absz=Z)
        return snr

    def interp_score(self, f3, tau, grad: bool = False):
        """Interpolated statistic of continuous templates (real f0, f1, f2 in bins;
        tau in s) and optionally its analytic gradient d SNR / d (f0, f1, f2, tau)."""
        f3 = np.ascontiguousarray(f3, dtype=np.float64).reshape(-1, 3)
        tau = np.ascontiguousarray(tau, dtype=np.float64).reshape(-1)
        n = f3.shape[0]
        snr = np.zeros(n)
        g = np.zeros((n, 4))
        lib().orc_interp_explicit(self._h, _ptr(f3, C.c_double), _ptr(tau, C.c_double), n, _ptr(snr, C.c_double),
                                  _ptr(g, C.c_double))
        return (snr, g) if grad else snr

    def score_explicit_general(self, t3, f3, tau):
        """Eq. 7 for explicit general templates (t3, f3 [n][3]; tau [n])."""
        t3 = np.ascontiguousarray(t3, dtype=np.uint32).reshape(-1, 3)
        f3 = np.ascontiguousarray(f3, dtype=np.uint32).reshape(-1, 3)
        tau = np.ascontiguousarray(tau, dtype=np.float64).reshape(-1)
        out = np.zeros(tau.size)
        lib().orc_score_explicit_general(self._h, _ptr(t3, C.c_uint32), _ptr(f3, C.c_uint32), _ptr(tau, C.c_double),
                                         tau.size, _ptr(out, C.c_double))
        return out

    def score_range_ext(self, seed: int, offset: int, n_tracks: int, tau_max: float, general: bool = False,
                        t_min: int = 1, quantiles=None, nthreads: int | None = None, with_scale: bool = False):
        """score_range with general templates and/or a delay prior; with_scale also
        returns each template's comparison scale sum_j |z_j| / norm."""
        if nthreads is None:
            nthreads = os.cpu_count() or 1
        q = np.ascontiguousarray(quantiles if quantiles is not None else np.zeros(1), dtype=np.float64)
        nq = int(q.size) if quantiles is not None else 0
        out = np.zeros(n_tracks)
        if with_scale:
            sc = np.zeros(n_tracks)
            rc = lib().orc_score_range_ext_scale(self._h, seed, offset, n_tracks, tau_max, int(general), int(t_min),
                                                 _ptr(q, C.c_double), nq, int(nthreads), _ptr(out, C.c_double),
                                                 _ptr(sc, C.c_double))
        else:
            rc = lib().orc_score_range_ext(self._h, seed, offset, n_tracks, tau_max, int(general), int(t_min),
                                           _ptr(q, C.c_double), nq, int(nthreads), _ptr(out, C.c_double))
        if rc != 0:
            raise RuntimeError("oracle score_range_ext failed (%d)" % rc)
        return (out, sc) if with_scale else out

    def score_range_scale(self, seed: int, offset: int, n_tracks: int, tau_max: float,
                          nthreads: int | None = None):
        """score_range, plus each template's comparison scale sum_j |z_j| / norm."""
        if nthreads is None:
            nthreads = os.cpu_count() or 1
        out = np.zeros(n_tracks)
        sc = np.zeros(n_tracks)
        rc = lib().orc_score_range_scale(self._h, seed, offset, n_tracks, tau_max, int(nthreads),
                                         _ptr(out, C.c_double), _ptr(sc, C.c_double))
        if rc != 0:
            raise RuntimeError("oracle score_range_scale failed (%d)" % rc)
        return out, sc

    def score_range(self, seed: int, offset: int, n_tracks: int, tau_max: float,
                    nthreads: int | None = None) -> np.ndarray:
        """SNR of templates offset .. offset+n_tracks-1 (Sec. III draws, Eq. 7)."""
        if nthreads is None:
            nthreads = os.cpu_count() or 1
        out = np.zeros(n_tracks)
        rc = lib().orc_score_range(self._h, seed, offset, n_tracks, tau_max, int(nthreads),
                                   _ptr(out, C.c_double))
        if rc != 0:
            raise RuntimeError("oracle score_range failed (%d)" % rc)
        return out


def topk(snr, offset: int, k: int):
    """K loudest templates: SNR descending, then index ascending (Sec. III; Sec. V)."""
    snr = np.ascontiguousarray(snr, dtype=np.float64)
    vals = np.zeros(k)
    idx = np.zeros(k, dtype=np.uint64)
    rc = lib().orc_topk(_ptr(snr, C.c_double), snr.shape[0], offset, k, _ptr(vals, C.c_double),
                        _ptr(idx, C.c_uint64))
    if rc != 0:
        raise ValueError("oracle topk: bad k (%d)" % rc)
    return vals, idx.astype(np.int64)
