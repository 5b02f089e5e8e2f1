"""Pins of the multi-sine generator and of the phasor oracle."""
import os

import numpy as np

from oracle import phasor as ph
from workloads import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "multisine_envelope.txt")


def _golden():
    out = {}
    for ln in open(GOLDEN):
        if ln.strip() and not ln.startswith("#"):
            k, v, tol = ln.split()
            out[k] = (float(v), float(tol))
    return out


def test_multisine_envelope_matches_the_printed_figure():
    """Over one period of the 1 Hz fundamental the 30-tone current peaks near +48 A and
    dips near -43 A (Sec. 4.3, excitation figure)."""
    g = _golden()
    y = synth.multisine(400000, 2.5e-6)          # 1 s at 400 kS/s
    assert abs(y.max() - g["max_A"][0]) <= g["max_A"][1], y.max()
    assert abs(y.min() - g["min_A"][0]) <= g["min_A"][1], y.min()


def test_phasor_of_pure_tones_over_integer_periods():
    """y = sum_j Im(W_j exp(j w_j t)) over integer periods: each phasor is -j W_j
    (orthogonality of the DFT basis)."""
    T, dt = 1000, 1e-4                      # 0.1 s record: 10 Hz bins
    f = np.array([30.0, 120.0, 1990.0])
    W = np.array([1.5 * np.exp(0.3j), 0.2 * np.exp(-2.0j), 3.0 * np.exp(1.1j)])
    t = dt * np.arange(T)
    y = np.imag(W[:, None] * np.exp(2j * np.pi * f[:, None] * t[None, :])).sum(axis=0)[None, :]
    X = ph.phasors(y, 0.0, dt, f)[:, 0]
    assert np.allclose(X, -1j * W, rtol=0, atol=1e-12)


def test_multisine_phasors_recover_tone_amplitudes():
    """The generator's tones come back at 4 A with phases phi_k - pi/2 (sin = Im e^{j.})."""
    T, dt = 200000, 5e-6                    # exactly 1 s
    y = synth.multisine(T - 1, dt)[None, :]
    X = ph.phasors(y, 0.0, dt, synth.MULTISINE_HZ)[:, 0]
    k = np.arange(1, 31)
    expect = -1j * 4.0 * np.exp(-1j * np.pi * k * (k - 1) / 30)
    assert np.allclose(X, expect, atol=1e-9)
