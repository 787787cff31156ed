"""Spectral peak picking (test helper; stands in for a neural pitch tracker).

Hann window, zero padding and a parabolic fit of the log-magnitude around
the largest bin inside a search band.
"""

from __future__ import annotations

import numpy as np


def peak_frequency(y: np.ndarray, fs: float, f_lo: float, f_hi: float, pad: int = 16) -> float:
    y = np.asarray(y, dtype=np.float64)
    y = y - y.mean()
    w = np.hanning(len(y))
    nfft = int(2 ** np.ceil(np.log2(len(y) * pad)))
    spec = np.abs(np.fft.rfft(y * w, nfft))
    freqs = np.fft.rfftfreq(nfft, 1.0 / fs)
    band = np.where((freqs >= f_lo) & (freqs <= f_hi))[0]
    i = band[np.argmax(spec[band])]
    a, b, c = np.log(spec[i - 1] + 1e-300), np.log(spec[i] + 1e-300), np.log(spec[i + 1] + 1e-300)
    off = 0.5 * (a - c) / (a - 2 * b + c)
    return float(freqs[i] + off * (freqs[1] - freqs[0]))
