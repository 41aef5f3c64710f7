"""B300 scorer for all-sky seedless clustering (Thrane & Coughlin).

A thin Python binding over libstk.so.  Every step of scoring (template draws,
rasterisation, phase rotation, sums, normalisation, top-k) runs in the
library's CUDA kernels; this module only marshals arguments.  PyTorch supplies
device memory and the CUDA stream.

    ctx = Context()                                 # device 0, torch's current stream
    m = ctx.load_map(y, sigma, f_min=40.0, df=0.5)   # y complex64 [n_t][n_f]; sigma [n_f] or [n_t][n_f]
    ctx.set_tracks(5_000_000, seed=2, offset=0, tau_max=0.010)
    hits = ctx.score(m, k=16)                       # numpy structured array, loudest first
"""
from __future__ import annotations

import ctypes as C
import weakref

import numpy as np

from . import _lib as L
from ._lib import HIT_DTYPE, STK_MAX_K  # noqa: F401

__all__ = ["Context", "Map", "Batch", "StkError", "HIT_DTYPE", "STK_MAX_K", "lib"]

lib = L.lib


class StkError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"stk error {code}: {msg}")
        self.code = code


def _torch():
    import torch
    return torch


def _is_tensor(x):
    try:
        import torch
    except ImportError:  # pragma: no cover
        return False
    return isinstance(x, torch.Tensor)


class Map:
    """A packed ft-map owned by the library (freed on close / garbage collection)."""

    def __init__(self, ctx, handle, n_t, n_f, flags):
        self._ctx, self._h, self.n_t, self.n_f, self.flags = ctx, handle, n_t, n_f, flags
        ctx._children.add(self)

    @property
    def handle(self):
        if not self._h:
            raise ValueError("map has been freed")
        return self._h

    def close(self):
        if self._h:
            lib().stk_free_map(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Context:
    """A scoring context on one CUDA device (calls stk_create)."""

    def __init__(self, device: int = 0, stream=None):
        torch = _torch()
        self.device = int(device)
        h = C.c_void_p()
        self._stream = stream
        rc = lib().stk_create(C.byref(h), self.device, C.c_void_p(self._stream_ptr()))
        if rc != 0:
            raise StkError(rc, lib().stk_last_error(None).decode())
        self._h = h
        self._torch = torch
        self._children = weakref.WeakSet()   # maps and batches: freed before the context

    # ---- plumbing
    def _stream_ptr(self):
        torch = _torch()
        s = self._stream if self._stream is not None else torch.cuda.current_stream(self.device)
        return int(s.cuda_stream)

    def _check(self, rc):
        if rc != 0:
            raise StkError(rc, lib().stk_last_error(self._h).decode())

    def _bind_stream(self):
        self._check(lib().stk_set_stream(self._h, C.c_void_p(self._stream_ptr())))

    def close(self):
        if getattr(self, "_h", None):
            for child in sorted(list(self._children), key=lambda c: 0 if isinstance(c, Batch) else 1):
                child.close()           # batches first, then maps
            lib().stk_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- calls
    def load_map(self, y, sigma, f_min: float, df: float, paper_mode: bool = False, fp16: bool = False) -> Map:
        """stk_load_map.  y: complex64 [n_t][n_f] (CUDA tensor, or host numpy/tensor);
        sigma: float32 [n_f] (per frequency) or [n_t][n_f]; fp16: 4-byte pixel storage."""
        self._bind_stream()
        host = not (_is_tensor(y) and y.is_cuda)
        if host:
            ya = y.numpy() if _is_tensor(y) else y
            sa = sigma.numpy() if _is_tensor(sigma) else sigma
            ya = np.ascontiguousarray(ya, dtype=np.complex64)
            sa = np.ascontiguousarray(sa, dtype=np.float32)
            yp, sp = ya.ctypes.data, sa.ctypes.data
            keep = (ya, sa)
        else:
            torch = self._torch
            if y.dtype != torch.complex64 or sigma.dtype != torch.float32:
                raise TypeError("y must be complex64 and sigma float32")
            if not sigma.is_cuda:
                raise TypeError("y and sigma must both be CUDA tensors or both host arrays")
            y = y.contiguous()
            sigma = sigma.contiguous()
            yp, sp = y.data_ptr(), sigma.data_ptr()
            keep = (y, sigma)
        n_t, n_f = keep[0].shape
        per_freq = tuple(keep[1].shape) == (n_f,)
        if not per_freq and tuple(keep[1].shape) != (n_t, n_f):
            raise ValueError(f"sigma shape {tuple(keep[1].shape)} is neither ({n_f},) nor ({n_t}, {n_f})")
        flags = (L.STK_HOST_PTR if host else 0) | (L.STK_SIGMA_PER_FREQ if per_freq else 0) | \
            (L.STK_NORM_PAPER if paper_mode else 0) | (L.STK_FP16 if fp16 else 0)
        h = C.c_void_p()
        self._check(lib().stk_load_map(self._h, C.c_void_p(yp), C.c_void_p(sp), int(n_t), int(n_f),
                                       float(f_min), float(df), flags, C.byref(h)))
        del keep
        return Map(self, h, int(n_t), int(n_f), flags)

    def update_map(self, m: Map, y, sigma):
        """stk_update_map: new data of the same shape into an existing map (no allocation)."""
        self._bind_stream()
        host = not (_is_tensor(y) and y.is_cuda)
        if host:
            ya = np.ascontiguousarray(y.numpy() if _is_tensor(y) else y, dtype=np.complex64)
            sa = np.ascontiguousarray(sigma.numpy() if _is_tensor(sigma) else sigma, dtype=np.float32)
            yp, sp, keep = ya.ctypes.data, sa.ctypes.data, (ya, sa)
        else:
            y, sigma = y.contiguous(), sigma.contiguous()
            yp, sp, keep = y.data_ptr(), sigma.data_ptr(), (y, sigma)
        if tuple(keep[0].shape) != (m.n_t, m.n_f):
            raise ValueError("y shape differs from the map's")
        flags = (m.flags & ~L.STK_HOST_PTR) | (L.STK_HOST_PTR if host else 0)
        self._check(lib().stk_update_map(self._h, m.handle, C.c_void_p(yp), C.c_void_p(sp), flags))
        del keep

    def set_tracks(self, n_tracks: int, seed: int, offset: int = 0, tau_max: float = 0.010):
        """stk_set_tracks: templates offset .. offset+n_tracks-1 drawn with `seed`."""
        self._check(lib().stk_set_tracks(self._h, int(n_tracks), int(seed), int(offset), float(tau_max)))
        self.n_tracks = int(n_tracks)

    def score(self, m: Map, k: int, out=None):
        """stk_score.  Returns a numpy HIT_DTYPE array (host, waits) or, when `out`
        is a CUDA uint8 tensor of k*40 bytes, fills it asynchronously and returns it."""
        self._bind_stream()
        if out is None:
            res = np.zeros(k, dtype=HIT_DTYPE)
            self._check(lib().stk_score(self._h, m.handle, int(k), C.c_void_p(res.ctypes.data), L.STK_OUT_HOST))
            return res
        if out.numel() * out.element_size() < 40 * k or not out.is_cuda:
            raise ValueError("out must be a CUDA tensor of at least 40*k bytes")
        self._check(lib().stk_score(self._h, m.handle, int(k), C.c_void_p(out.data_ptr()), 0))
        return out

    def score_all(self, m: Map, out=None):
        """stk_score_all: SNR of every template (float64 CUDA tensor)."""
        torch = self._torch
        self._bind_stream()
        if out is None:
            out = torch.empty(self.n_tracks, dtype=torch.float64, device=f"cuda:{self.device}")
        if out.dtype != torch.float64 or not out.is_cuda or out.numel() < self.n_tracks:
            raise ValueError("out must be a CUDA float64 tensor of n_tracks elements")
        self._check(lib().stk_score_all(self._h, m.handle, C.c_void_p(out.data_ptr())))
        return out

    def track_params(self, m: Map, g: int, bins: bool = True):
        """stk_track_params: ((f0, f1, f2), tau, bins[n_t] or None) of template g."""
        self._bind_stream()
        f = np.zeros(3, dtype=np.uint32)
        tau = C.c_double()
        b = np.zeros(m.n_t, dtype=np.int32) if bins else None
        self._check(lib().stk_track_params(self._h, m.handle, int(g), C.c_void_p(f.ctypes.data), C.byref(tau),
                                           C.c_void_p(b.ctypes.data) if bins else None))
        return tuple(int(v) for v in f), float(tau.value), b

    def score_explicit(self, m: Map, f3, tau, out=None):
        """stk_score_explicit on CUDA tensors f3 [n][3] (int32/uint32 bins) and tau [n] (float64)."""
        torch = self._torch
        self._bind_stream()
        dev = f"cuda:{self.device}"
        f3 = torch.as_tensor(f3).to(device=dev).contiguous()
        if f3.dtype not in (torch.int32, torch.uint32):
            f3 = f3.to(torch.int32)
        tau = torch.as_tensor(tau, dtype=torch.float64).to(device=dev).contiguous()
        n = tau.numel()
        if f3.numel() != 3 * n:
            raise ValueError("f3 must have shape [n][3]")
        if out is None:
            out = torch.empty(n, dtype=torch.float64, device=dev)
        self._check(lib().stk_score_explicit(self._h, m.handle, C.c_void_p(f3.data_ptr()),
                                             C.c_void_p(tau.data_ptr()), n, C.c_void_p(out.data_ptr())))
        return out

    def set_template_shape(self, general: bool, t_min: int = 1):
        """stk_set_template_shape: random start / middle / end times (duration >= t_min columns)."""
        self._check(lib().stk_set_template_shape(self._h, 1 if general else 0, int(t_min)))

    def set_tau_prior(self, quantiles=None):
        """stk_set_tau_prior: delay quantiles (s) at probabilities i/(n-1); None: uniform."""
        if quantiles is None:
            self._check(lib().stk_set_tau_prior(self._h, None, 0))
            return
        q = np.ascontiguousarray(quantiles, dtype=np.float64)
        self._check(lib().stk_set_tau_prior(self._h, C.c_void_p(q.ctypes.data), int(q.size)))

    def track_times(self, m: Map, g: int):
        """stk_track_times: control times (t0, t1, t2) of template g."""
        t = np.zeros(3, dtype=np.uint32)
        self._check(lib().stk_track_times(self._h, m.handle, int(g), C.c_void_p(t.ctypes.data)))
        return tuple(int(v) for v in t)

    def score_explicit_general(self, m: Map, t3, f3, tau, out=None):
        """stk_score_explicit_general on [n][3] times, [n][3] bins and [n] delays."""
        torch = self._torch
        self._bind_stream()
        dev = f"cuda:{self.device}"
        t3 = torch.as_tensor(t3).to(device=dev, dtype=torch.int32).contiguous()
        f3 = torch.as_tensor(f3).to(device=dev, dtype=torch.int32).contiguous()
        tau = torch.as_tensor(tau, dtype=torch.float64).to(device=dev).contiguous()
        n = tau.numel()
        if out is None:
            out = torch.empty(n, dtype=torch.float64, device=dev)
        self._check(lib().stk_score_explicit_general(self._h, m.handle, C.c_void_p(t3.data_ptr()),
                                                     C.c_void_p(f3.data_ptr()), C.c_void_p(tau.data_ptr()), n,
                                                     C.c_void_p(out.data_ptr())))
        return out

    def interp_forward(self, m: Map, f3, tau):
        """stk_interp_forward: SNR of continuous templates (f3 float32 [n][3] bins, tau float32 [n] s)."""
        torch = self._torch
        self._bind_stream()
        f3 = f3.detach().to(torch.float32).contiguous()
        tau = tau.detach().to(torch.float32).contiguous()
        out = torch.empty(tau.numel(), dtype=torch.float32, device=tau.device)
        self._check(lib().stk_interp_forward(self._h, m.handle, C.c_void_p(f3.data_ptr()), C.c_void_p(tau.data_ptr()),
                                             tau.numel(), C.c_void_p(out.data_ptr())))
        return out

    def interp_adjoint(self, m: Map, f3, tau, g):
        """stk_interp_adjoint: (g * dSNR/df3, g * dSNR/dtau)."""
        torch = self._torch
        self._bind_stream()
        f3 = f3.detach().to(torch.float32).contiguous()
        tau = tau.detach().to(torch.float32).contiguous()
        g = g.detach().to(torch.float32).contiguous()
        gf = torch.empty_like(f3)
        gt = torch.empty_like(tau)
        self._check(lib().stk_interp_adjoint(self._h, m.handle, C.c_void_p(f3.data_ptr()), C.c_void_p(tau.data_ptr()),
                                             C.c_void_p(g.data_ptr()), tau.numel(), C.c_void_p(gf.data_ptr()),
                                             C.c_void_p(gt.data_ptr())))
        return gf, gt

    def refine(self, m: Map, f3, tau, tau_max: float, steps: int = 50, lr_bins: float = 0.25,
               lr_tau_frac: float = 0.02, history: bool = True):
        """stk_refine: `steps` Adam steps of gradient ascent on the device.  Returns new
        tensors (f3, tau, snr_history [steps + 1][n] or None); the inputs are not modified."""
        torch = self._torch
        self._bind_stream()
        f = f3.detach().to(torch.float32).contiguous().clone()
        t = tau.detach().to(torch.float32).contiguous().clone()
        n = t.numel()
        h = torch.empty((steps + 1, n), dtype=torch.float32, device=t.device) if history else None
        self._check(lib().stk_refine(self._h, m.handle, C.c_void_p(f.data_ptr()), C.c_void_p(t.data_ptr()), n,
                                     int(steps), float(lr_bins), float(lr_tau_frac), float(tau_max),
                                     C.c_void_p(h.data_ptr() if h is not None else 0)))
        return f, t, h

    def polish(self, m: Map, f3, tau, tau_max: float, alt_f3=None, alt_tau=None, moves: int = 8):
        """stk_polish: discrete follow-up of templates f3 (int [n][3] bins) and tau
        (float64 [n] s), with optional continuous alternatives alt_f3 (float32 [n][3])
        and alt_tau (float32 [n]).  Returns (f3 uint32-valued int64 tensor, tau float64,
        snr float64, which int32), all on the device."""
        torch = self._torch
        self._bind_stream()
        f = torch.as_tensor(f3, device="cuda").to(torch.int32).contiguous().clone()   # same bits as uint32
        t = torch.as_tensor(tau, device="cuda").to(torch.float64).contiguous().clone()
        n = t.numel()
        if f.shape != (n, 3):
            raise ValueError("f3 must be [n][3]")
        a_f = a_t = None
        if (alt_f3 is None) != (alt_tau is None):
            raise ValueError("alt_f3 and alt_tau go together")
        if alt_f3 is not None:
            a_f = torch.as_tensor(alt_f3, device="cuda").to(torch.float32).contiguous()
            a_t = torch.as_tensor(alt_tau, device="cuda").to(torch.float32).contiguous()
            if a_f.shape != (n, 3) or a_t.numel() != n:
                raise ValueError("alternatives must match f3 and tau")
        snr = torch.empty(n, dtype=torch.float64, device="cuda")
        which = torch.empty(n, dtype=torch.int32, device="cuda")
        self._check(lib().stk_polish(self._h, m.handle, C.c_void_p(f.data_ptr()), C.c_void_p(t.data_ptr()),
                                     C.c_void_p(a_f.data_ptr() if a_f is not None else 0),
                                     C.c_void_p(a_t.data_ptr() if a_t is not None else 0), n, float(tau_max),
                                     int(moves), C.c_void_p(snr.data_ptr()), C.c_void_p(which.data_ptr())))
        return f.to(torch.int64), t, snr, which

    def sync(self):
        """stk_sync: wait and raise the first deferred kernel error."""
        self._check(lib().stk_sync(self._h))

    def set_option(self, option: int, value: int):
        self._check(lib().stk_set_option(self._h, int(option), int(value)))

    def last_plan(self) -> dict:
        a = (C.c_int64 * 9)()
        self._check(lib().stk_last_plan(self._h, a))
        keys = ["kernel", "R", "threads", "grid", "S", "nstage", "nbatches", "smem", "order"]
        return dict(zip(keys, [int(v) for v in a]))

    def set_profiling(self, on: bool):
        self._check(lib().stk_set_profiling(self._h, 1 if on else 0))

    def last_timings(self) -> dict:
        a = (C.c_double * 4)()
        self._check(lib().stk_last_timings(self._h, a))
        return dict(score_ms=a[0], select_ms=a[1], launches=int(a[2]), order_ms=a[3])


class Batch:
    """Many maps scored in one persistent launch (stk_batch_create / stk_batch_score).

    maps: list of Map (all loaded on ctx, same statistic, precision and weighting);
    n_tracks, seeds, offsets: one per map; tau_max: seconds.
    """

    def __init__(self, ctx: Context, maps, n_tracks, seeds, offsets=None, tau_max: float = 0.010):
        n = len(maps)
        self._ctx = ctx
        self._maps = list(maps)           # keep them alive
        self.n_maps = n
        hs = (C.c_void_p * n)(*[m.handle for m in maps])
        nt = np.ascontiguousarray(n_tracks, dtype=np.uint64)
        sd = np.ascontiguousarray(seeds, dtype=np.uint64)
        of = np.ascontiguousarray(offsets if offsets is not None else np.zeros(n), dtype=np.uint64)
        if not (nt.size == sd.size == of.size == n):
            raise ValueError("n_tracks, seeds and offsets need one entry per map")
        h = C.c_void_p()
        ctx._bind_stream()
        ctx._check(lib().stk_batch_create(ctx._h, hs, n, C.c_void_p(nt.ctypes.data), C.c_void_p(sd.ctypes.data),
                                          C.c_void_p(of.ctypes.data), float(tau_max), C.byref(h)))
        self._h = h
        ctx._children.add(self)

    def score(self, k: int, out=None):
        """Each map's k loudest: numpy HIT_DTYPE [n_maps][k] (waits), or fills a CUDA
        uint8 tensor of n_maps*k*40 bytes asynchronously."""
        self._ctx._bind_stream()
        if out is None:
            res = np.zeros(self.n_maps * k, dtype=HIT_DTYPE)
            self._ctx._check(lib().stk_batch_score(self._h, int(k), C.c_void_p(res.ctypes.data), L.STK_OUT_HOST))
            return res.reshape(self.n_maps, k)
        if not out.is_cuda or out.numel() * out.element_size() < 40 * k * self.n_maps:
            raise ValueError("out must be a CUDA tensor of at least n_maps*k*40 bytes")
        self._ctx._check(lib().stk_batch_score(self._h, int(k), C.c_void_p(out.data_ptr()), 0))
        return out

    def cancel(self, on: bool = True):
        self._ctx._check(lib().stk_batch_cancel(self._h, 1 if on else 0))

    def tune(self, k: int) -> dict:
        self._ctx._bind_stream()
        a = (C.c_int64 * 4)()
        self._ctx._check(lib().stk_batch_tune(self._h, int(k), a))
        return dict(threads=int(a[0]), R=int(a[1]), nstage=int(a[2]), sample_ms=a[3] / 1e6)

    def close(self):
        if getattr(self, "_h", None):
            lib().stk_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _autograd_function():
    import torch

    class InterpSNR(torch.autograd.Function):
        """SNR of continuous templates with the library's forward and adjoint kernels."""

        @staticmethod
        def forward(fctx, f3, tau, stk_ctx, m):
            fctx.save_for_backward(f3, tau)
            fctx.stk = (stk_ctx, m)
            return stk_ctx.interp_forward(m, f3, tau)

        @staticmethod
        def backward(fctx, g):
            f3, tau = fctx.saved_tensors
            stk_ctx, m = fctx.stk
            gf, gt = stk_ctx.interp_adjoint(m, f3, tau, g)
            return gf, gt, None, None

    return InterpSNR


def interp_snr(ctx: Context, m: Map, f3, tau):
    """Differentiable SNR of continuous templates (torch.autograd)."""
    return _autograd_function().apply(f3, tau, ctx, m)


def refine(ctx: Context, m: Map, f3, tau, tau_max: float, steps: int = 50, lr_bins: float = 0.25,
           lr_tau_frac: float = 0.02):
    """Gradient ascent of the interpolated SNR over (f0, f1, f2, tau) of each template
    (Adam; f in bins, tau in units of tau_max), projected onto f in [0, n_f - 1] and
    |tau| <= tau_max, every step on the device (stk_refine).  Returns (f3, tau,
    snr_history [steps + 1][n]) as tensors."""
    return ctx.refine(m, f3, tau, tau_max, steps, lr_bins, lr_tau_frac)
