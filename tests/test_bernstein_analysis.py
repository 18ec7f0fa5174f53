"""Pins of the (k, omega) analysis used for the Bernstein-mode comparison (CPU only): known waves
land on their own bins and band centroids recover their frequencies."""
import numpy as np

from paper_1707_04333_gb300 import bernstein


def _grid(nt=512, nx=64, dt=1e-3, dx=0.01):
    t = np.arange(nt)[:, None] * dt
    x = np.arange(nx)[None, :] * dx
    return t, x, dt, dx, nt, nx


def test_travelling_and_standing_waves_land_on_their_bins():
    t, x, dt, dx, nt, nx = _grid()
    mk, mw = 5, 37                                   # on-bin wavenumber and frequency indices
    k0 = 2 * np.pi * mk / (nx * dx)
    w0 = 2 * np.pi * mw / (nt * dt)
    for f in (np.cos(k0 * x - w0 * t), np.cos(k0 * x + w0 * t), np.cos(k0 * x) * np.cos(w0 * t)):
        k, om, P = bernstein.spectrum(f, dx, dt)
        i, j = np.unravel_index(np.argmax(P), P.shape)
        assert (i, j) == (mk, mw)
        np.testing.assert_allclose(k[i], k0, rtol=1e-12)
        np.testing.assert_allclose(om[j], w0, rtol=1e-12)


def test_band_centroids_recover_tone_frequencies():
    """A sum of on-bin tones, one per harmonic band: the Hann leakage is symmetric about each tone,
    so each band's power-weighted mean frequency is the tone's frequency."""
    t, x, dt, dx, nt, nx = _grid(nt=2048)
    dw = 2 * np.pi / (nt * dt)
    wc = 100 * dw
    tones = [1.2 * wc, 1.9 * wc, 3.1 * wc]
    tones = [round(w / dw) * dw for w in tones]
    ks = [2 * np.pi * m / (nx * dx) for m in (3, 7, 11)]
    f = sum(a * np.cos(kk * x - w * t) for a, kk, w in zip((1.0, 0.5, 2.0), ks, tones))
    k, om, P = bernstein.spectrum(f, dx, dt)
    c = bernstein.band_centroids(k, om, P, wc, harmonics=(1, 2, 3))
    np.testing.assert_allclose(c, tones, rtol=1e-9)


def test_white_noise_centroid_is_band_centre():
    """Flat (white) spectra put each band's centroid at its centre n wc, within sampling noise."""
    rng = np.random.default_rng(0)
    nt, nx, dt, dx = 4096, 64, 1e-3, 0.01
    f = rng.normal(size=(nt, nx))
    k, om, P = bernstein.spectrum(f, dx, dt)
    wc = 2 * np.pi * 200 / (nt * dt)
    c = bernstein.band_centroids(k, om, P, wc, harmonics=(1, 2, 3))
    np.testing.assert_allclose(c / wc, [1.0, 2.0, 3.0], atol=0.02)
