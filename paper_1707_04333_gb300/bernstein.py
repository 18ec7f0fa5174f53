"""Dispersion diagnostic of the Bernstein-mode study (Sec. III.C).

The field is sampled along a line of the domain at every time step (the
library's field probes) and Fourier-transformed in space and time; the (k, omega)
power shows the Bernstein branches between the harmonics of the cyclotron
frequency.  `band_centroids` reduces a spectrum to one frequency per harmonic
band (the power-weighted mean over a k range), the figure compared between the
FP32 and FP64 paths.  Host-side analysis of probe data; no part of the step.
"""
from __future__ import annotations

import numpy as np


def spectrum(samples, dx: float, dt: float):
    """Power of samples[t, j] (uniform line spacing dx, one row per step dt) in (k, omega).

    The mean is removed and a Hann window applied in both directions; the 2-D FFT power is folded
    onto k >= 0, omega >= 0 (a wave and its mirror images add up).  Returns (k [rad/m],
    omega [rad/s], P[k, omega])."""
    a = np.asarray(samples, np.float64)
    a = a - a.mean()
    nt, nx = a.shape
    win = np.hanning(nt)[:, None] * np.hanning(nx)[None, :]
    S = np.abs(np.fft.fft2(a * win)) ** 2
    it = np.abs(np.fft.fftfreq(nt) * nt).round().astype(np.int64)
    ix = np.abs(np.fft.fftfreq(nx) * nx).round().astype(np.int64)
    P = np.zeros((nx // 2 + 1, nt // 2 + 1))
    np.add.at(P, (ix[None, :].repeat(nt, 0), it[:, None].repeat(nx, 1)), S)
    k = 2.0 * np.pi * np.arange(nx // 2 + 1) / (nx * dx)
    omega = 2.0 * np.pi * np.arange(nt // 2 + 1) / (nt * dt)
    return k, omega, P


def band_centroids(k, omega, P, wc: float, harmonics=(1, 2, 3), k_range=None):
    """Power-weighted mean frequency in each band [(n - 1/2) wc, (n + 1/2) wc), n in `harmonics`,
    of the spectrum summed over k in k_range = (k_lo, k_hi) (all k > 0 when None)."""
    k = np.asarray(k)
    lo, hi = (k[1], k[-1]) if k_range is None else k_range
    sel = (k >= lo) & (k <= hi)
    p = P[sel].sum(axis=0)
    out = []
    for n in harmonics:
        m = (omega >= (n - 0.5) * wc) & (omega < (n + 0.5) * wc)
        w = p[m]
        out.append(float((omega[m] * w).sum() / w.sum()) if w.sum() > 0 else float("nan"))
    return np.array(out)
