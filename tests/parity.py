"""Per-output comparisons for the FP64 parity tests.

The FP64 bar is a relative error per output trace (one probe's time series) and per
snapshot (one current vector), not one norm over the whole output array: a wrong
low-amplitude pickup trace must not hide under the large ones.
"""
import numpy as np


def _per_slice(a, b, axis):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if a.shape != b.shape:
        raise AssertionError(f"shape {a.shape} != {b.shape}")
    if a.ndim == 1:
        a, b = a[None, :], b[None, :]
        axis = -1
    a = np.moveaxis(a, axis, -1).reshape(-1, a.shape[axis])
    b = np.moveaxis(b, axis, -1).reshape(-1, b.shape[axis])
    num = np.linalg.norm(a - b, axis=1)
    den = np.linalg.norm(b, axis=1)
    # an identically zero reference slice is compared against the largest slice
    scale = den.max() if den.size and den.max() > 0 else 1.0
    den = np.where(den > 0, den, scale)
    return num / den


def rel_traces(a, b):
    """Max over probe traces (slices along the last axis, time) of ||a - b|| / ||b||."""
    e = _per_slice(a, b, -1)
    return float(e.max()) if e.size else 0.0


def rel_snaps(a, b):
    """Max over snapshots (slices along the first axis, the n currents) of ||a - b|| / ||b||.

    Snapshot arrays are (n, nsnap) or (ntraj, n, nsnap); every (trajectory, snapshot)
    current vector is one slice."""
    a = np.asarray(a)
    b = np.asarray(b)
    axis = 0 if a.ndim <= 2 else a.ndim - 2
    e = _per_slice(a, b, axis)
    return float(e.max()) if e.size else 0.0


def rel_vec(a, b):
    """||a - b|| / ||b|| for one vector (a gradient, a solution)."""
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / (nb if nb > 0 else 1.0))


def rel_probes_functional(a, b, C, snaps):
    """Max over probes p of max_k |a_pk - b_pk| / (||C_p|| max_j ||I_j||): each probe
    value's error against what a relative error of the current would produce through
    that probe row (I_j: the reference snapshots, columns of `snaps`)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    Inorm = float(np.linalg.norm(np.asarray(snaps), axis=0).max())
    cn = np.linalg.norm(np.asarray(C), axis=1)
    err = np.abs(a - b).max(axis=1)
    return float((err / (cn * Inorm)).max())
