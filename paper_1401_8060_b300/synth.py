"""Seeded synthetic ft-maps shaped like the paper's searches.

This module is the one place where inputs are made; both the CUDA path (through
the tests and the benchmark) and the FP64 oracle receive the arrays it returns.
It holds none of the scoring arithmetic: no template generator, no track
rasteriser, no phase rotation, no sums.  An injected signal is a quadratic
chirp whose frequency path is given here by its own continuous formula, or is
placed on an explicit list of pixels handed in by the caller.

The paper's data (recoloured LIGO noise, the FA/ADI waveforms; Sec. IV) are not
available, so these maps stand in for them with the paper's shapes: maps of a
few hundred time segments by a few hundred to a few thousand frequency bins
(Sec. IV; Table III's 151 x 500 map), complex cross-power pixels (Eq. 6) whose
real and imaginary parts are independent Gaussians with a per-pixel standard
deviation sigma (Appendix A).

Map layout: ``y`` is complex64 ``[n_t][n_f]`` (time-major, frequency fastest),
``sigma`` is float32, either ``[n_t][n_f]`` or a per-frequency ``[n_f]`` row.
Frequency of bin k is ``f_min + k * df``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "FtMap",
    "sigma_powerlaw",
    "noise_map",
    "chirp_path",
    "inject",
    "tiny_map",
    "realistic_map",
    "batched_maps",
    "WORKLOADS",
]


@dataclass
class FtMap:
    """One synthetic ft-map plus the recipe that made it."""

    y: np.ndarray            # complex64 [n_t][n_f]
    sigma: np.ndarray        # float32 [n_t][n_f] or [n_f]
    f_min: float             # Hz, frequency of bin 0
    df: float                # Hz, bin width
    sigma_per_freq: bool     # sigma has shape [n_f]
    injections: list = field(default_factory=list)  # dicts describing injected chirps

    @property
    def n_t(self) -> int:
        return int(self.y.shape[0])

    @property
    def n_f(self) -> int:
        return int(self.y.shape[1])

    def sigma_full(self) -> np.ndarray:
        """sigma broadcast to [n_t][n_f] (float32)."""
        if self.sigma_per_freq:
            return np.ascontiguousarray(np.broadcast_to(self.sigma[None, :], self.y.shape))
        return self.sigma


def sigma_powerlaw(f_hz: np.ndarray, sigma0: float = 1.0) -> np.ndarray:
    """Smooth power-law-plus-floor noise shape: sigma0 * sqrt(1 + (f/100 Hz)^-4)."""
    f = np.asarray(f_hz, dtype=np.float64)
    return (sigma0 * np.sqrt(1.0 + (f / 100.0) ** -4)).astype(np.float32)


def noise_map(n_t: int, n_f: int, sigma: np.ndarray, seed: int) -> np.ndarray:
    """Complex Gaussian noise: Re and Im each N(0, sigma^2), independent per pixel."""
    rng = np.random.default_rng(seed)
    s = np.asarray(sigma, dtype=np.float64)
    if s.ndim == 1:
        s = s[None, :]
    re = rng.standard_normal((n_t, n_f))
    im = rng.standard_normal((n_t, n_f))
    return ((re + 1j * im) * s).astype(np.complex64)


def chirp_path(n_t: int, n_f: int, p0: float, p1: float, p2: float) -> np.ndarray:
    """Frequency bin per time column of a quadratic chirp used as an injected signal.

    The chirp's frequency (in bins) runs along a quadratic Bezier curve through
    p0 at the first column, with p1 as middle control value, to p2 at the last
    column; its value at each column is rounded to the nearest bin.  Evaluated
    in float64 from the continuous curve; returns int32 [n_t].
    """
    x = np.linspace(0.0, 1.0, n_t)
    f = (1 - x) ** 2 * p0 + 2 * (1 - x) * x * p1 + x ** 2 * p2
    return np.clip(np.floor(f + 0.5), 0, n_f - 1).astype(np.int32)


def inject(y: np.ndarray, bins: np.ndarray, amplitude, tau_s: float, f_min: float,
           df: float) -> None:
    """Add a cross-power signal that arrived with delay tau_s, in place.

    Column j gets ``amplitude[j] * exp(-2 pi i f tau_s)`` at bin ``bins[j]``
    (f the bin's frequency).  A scorer that rotates by exp(+2 pi i f tau) sees
    it real and positive at tau = tau_s.  ``amplitude`` is a scalar or [n_t].
    """
    n_t = y.shape[0]
    j = np.arange(n_t)
    b = np.asarray(bins, dtype=np.int64)
    f = f_min + b * df
    amp = np.broadcast_to(np.asarray(amplitude, dtype=np.float64), (n_t,))
    sig = amp * np.exp(-2j * np.pi * f * tau_s)
    y[j, b] = (y[j, b].astype(np.complex128) + sig).astype(np.complex64)


# Workloads: a tiny 200 x 100 map and the realistic 500 x 1600 map (the bands and
# resolutions of the paper's searches).
WORKLOADS = {
    "tiny": dict(n_t=200, n_f=100, f_min=100.0, df=1.0, n_tracks=10_000, seed=1,
                 tau_max=0.010, k=16, noise_seed=11),
    "realistic": dict(n_t=500, n_f=1600, f_min=40.0, df=0.5, n_tracks=5_000_000, seed=2,
                      tau_max=0.010, k=1024, noise_seed=12),
}


def tiny_map(inject_signal: bool = True) -> FtMap:
    """200 x 100 map (1 Hz bins from 100 Hz), sigma = 1, one injected track of per-pixel SNR 1."""
    w = WORKLOADS["tiny"]
    n_t, n_f = w["n_t"], w["n_f"]
    sigma = np.ones(n_f, dtype=np.float32)
    y = noise_map(n_t, n_f, sigma, w["noise_seed"])
    fm = FtMap(y=y, sigma=sigma, f_min=w["f_min"], df=w["df"], sigma_per_freq=True)
    if inject_signal:
        bins = chirp_path(n_t, n_f, 20, 70, 45)
        inject(y, bins, 1.0, 0.0037, fm.f_min, fm.df)
        fm.injections.append(dict(p=(20, 70, 45), tau_s=0.0037, amplitude=1.0))
    return fm


def realistic_map(inject_signal: bool = True, n_t: int | None = None,
                  n_f: int | None = None) -> FtMap:
    """500 x 1600 map (0.5 Hz bins from 40 Hz) with per-frequency power-law sigma.

    One injected chirp (bins 200 -> 500 -> 1300, tau_s = -6.1 ms) with a constant
    amplitude chosen so that its noise-free weighted SNR is 20.
    """
    w = WORKLOADS["realistic"]
    n_t = n_t or w["n_t"]
    n_f = n_f or w["n_f"]
    f_min, df = w["f_min"], w["df"]
    sigma = sigma_powerlaw(f_min + df * np.arange(n_f))
    y = noise_map(n_t, n_f, sigma, w["noise_seed"])
    fm = FtMap(y=y, sigma=sigma, f_min=f_min, df=df, sigma_per_freq=True)
    if inject_signal:
        p = (200 * n_f / 1600, 500 * n_f / 1600, 1300 * n_f / 1600)
        bins = chirp_path(n_t, n_f, *p)
        wsum = float(np.sum(sigma.astype(np.float64)[bins] ** -2))
        amp = 20.0 / np.sqrt(wsum)
        inject(y, bins, amp, -0.0061, f_min, df)
        fm.injections.append(dict(p=p, tau_s=-0.0061, amplitude=amp, snr=20.0))
    return fm


def batched_maps(n_maps: int = 256, seed: int = 13, f_min: float = 40.0, df: float = 0.5,
                 n_t_range=(100, 1000), n_f_range=(200, 2000), inject_frac: float = 0.1):
    """Ragged list of maps: n_t ~ U{100..1000}, n_f ~ U{200..2000}, sigma0 ~ U(0.5, 2).

    About ``inject_frac`` of the maps carry one chirp with random control values,
    tau_s ~ U(-10 ms, 10 ms) and weighted SNR ~ U(10, 30).
    """
    rng = np.random.default_rng(seed)
    maps = []
    n_inj = int(round(inject_frac * n_maps))
    inj_ids = set(rng.choice(n_maps, size=n_inj, replace=False).tolist()) if n_inj else set()
    for i in range(n_maps):
        n_t = int(rng.integers(n_t_range[0], n_t_range[1] + 1))
        n_f = int(rng.integers(n_f_range[0], n_f_range[1] + 1))
        s0 = float(rng.uniform(0.5, 2.0))
        sigma = sigma_powerlaw(f_min + df * np.arange(n_f), s0)
        y = noise_map(n_t, n_f, sigma, int(rng.integers(0, 2**31)))
        fm = FtMap(y=y, sigma=sigma, f_min=f_min, df=df, sigma_per_freq=True)
        if i in inj_ids:
            p = tuple(float(v) for v in rng.uniform(0, n_f - 1, size=3))
            tau_s = float(rng.uniform(-0.010, 0.010))
            snr = float(rng.uniform(10, 30))
            bins = chirp_path(n_t, n_f, *p)
            wsum = float(np.sum(sigma.astype(np.float64)[bins] ** -2))
            amp = snr / np.sqrt(wsum)
            inject(y, bins, amp, tau_s, f_min, df)
            fm.injections.append(dict(p=p, tau_s=tau_s, amplitude=amp, snr=snr))
        maps.append(fm)
    return maps
