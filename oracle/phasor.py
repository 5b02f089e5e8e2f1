"""FP64 CPU oracle of phasor extraction from sampled signals.

TEST INFRASTRUCTURE ONLY (same rule as oracle/theta.py).

The paper's time-domain post-processing (Sec. 4.6) takes the Fourier transform of
the sampled responses and reads the phasor of each excitation tone.  With samples
y_k at t_k = t0 + k dt, k = 0..T-1, the phasor of tone f is the single-frequency
discrete Fourier coefficient  X(f) = (2/T) sum_k y_k exp(-j 2 pi f t_k).
For a record holding an integer number of periods of every tone this is the
complex amplitude W of y(t) = Im(W exp(j 2 pi f t)) times -j.
"""
from __future__ import annotations

import numpy as np


def phasors(y, t0: float, dt: float, freqs) -> np.ndarray:
    """y: (P, T) samples -> (F, P) complex phasors."""
    y = np.asarray(y, np.float64)
    T = y.shape[1]
    t = t0 + dt * np.arange(T, dtype=np.float64)
    f = np.asarray(freqs, np.float64)
    E = np.exp(-2j * np.pi * f[:, None] * t[None, :])      # (F, T)
    return (2.0 / T) * (E @ y.T)
