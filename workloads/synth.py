"""Seeded synthetic inputs for the eddy-current theta-method.

This module only *draws and tabulates* inputs: element positions and
directions, the inductance kernel L, the resistance matrix R, the electrode
operator E, coil mutuals M, probe rows C and source waveforms.  It holds none
of the integration method's arithmetic, and both the FP64 oracle and the CUDA
path read the very same arrays it produces.

Physical stand-in (the paper's FEM tube mesh is not available): a 40 x 20 x 2 mm
plate split into a regular grid of cells.  Each cell carries one current
unknown I_j flowing along an in-plane unit direction d_j.

* L_ij = mu0/(4 pi) (d_i . d_j) exp(-|x_i - x_j| / 2 mm) / (1 mm) + 1e-9 delta_ij  [H]
  (symmetric positive definite: a Schur product of two PSD kernels plus a
  positive diagonal; Sec. 3.1 requires L SPD).
* R = diag(rho_e g) + 1e-4 Ohm x (6-neighbour grid-graph Laplacian), with
  log10(rho_e) ~ U[-8, -7] Ohm m and g = 1e3 1/m  (SPD, Sec. 3.1).
* Coil / probe mutuals: mu0/(4 pi) exp(-|x_j - x_c| / 5 mm) / (1 mm)  [H]
  (Eq. induced_voltages_0: V = -M di/dt).
* Electrode operator (Eq. definition_E, one electrode dropped): a single row,
  E_j = -(d_j . x_hat) on the cells of the x-min face, 0 elsewhere; the x-max
  face is the dropped electrode.

Random draws use numpy ``default_rng(seed)`` in a fixed order: directions
phi ~ U[0, 2 pi) first, then log10 rho ~ U[-8, -7].
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

MU0_4PI = 1e-7            # mu0 / (4 pi)  [H/m]
PLATE_MM = (40.0, 20.0, 2.0)
L_RANGE_MM = 2.0          # inductance kernel range
M_RANGE_MM = 5.0          # coil / probe kernel range
L_REG = 1e-9              # diagonal regularisation of L [H]
G_FACTOR = 1e3            # rho -> R_ee [1/m]
LAP_OHM = 1e-4            # weight of the grid-graph Laplacian [Ohm]

# Named grids (nx, ny, nz) of the plate for the workload sizes.
GRIDS = {
    512: (16, 8, 4),
    4096: (32, 16, 8),
    8192: (32, 32, 8),
    16384: (64, 32, 8),
    65536: (64, 64, 16),
}


def grid_for(n: int) -> tuple[int, int, int]:
    """Grid whose first ``n`` cells (x fastest, then y, then z) hold the unknowns."""
    if n in GRIDS:
        return GRIDS[n]
    nz = 2 if n >= 8 else 1
    ny = max(1, math.ceil(math.sqrt(n / (2.0 * nz))))
    nx = 2 * ny
    while nx * ny * nz < n:
        ny += 1
        nx = 2 * ny
    return nx, ny, nz


@dataclass
class Geometry:
    n: int
    grid: tuple[int, int, int]
    pos_mm: np.ndarray        # (n, 3) cell centres [mm]
    ijk: np.ndarray           # (n, 3) integer grid coordinates
    phi: np.ndarray           # (n,) in-plane direction angle
    rho: np.ndarray           # (n,) resistivity [Ohm m]

    @property
    def dirs(self) -> np.ndarray:
        return np.stack([np.cos(self.phi), np.sin(self.phi), np.zeros_like(self.phi)], axis=1)


def geometry(n: int, seed: int = 0) -> Geometry:
    nx, ny, nz = grid_for(n)
    idx = np.arange(n)
    i = idx % nx
    j = (idx // nx) % ny
    k = idx // (nx * ny)
    h = (PLATE_MM[0] / nx, PLATE_MM[1] / ny, PLATE_MM[2] / nz)
    pos = np.stack([(i + 0.5) * h[0], (j + 0.5) * h[1], (k + 0.5) * h[2]], axis=1)
    rng = np.random.default_rng(seed)
    phi = rng.uniform(0.0, 2.0 * np.pi, size=n)
    rho = 10.0 ** rng.uniform(-8.0, -7.0, size=n)
    return Geometry(n, (nx, ny, nz), pos, np.stack([i, j, k], axis=1), phi, rho)


def _fill_L_rows(g: Geometry, out: np.ndarray, r0: int, r1: int) -> None:
    d = g.dirs
    p = g.pos_mm
    diff = p[r0:r1, None, :] - p[None, :, :]
    dist = np.sqrt(np.einsum("abk,abk->ab", diff, diff))
    dd = d[r0:r1] @ d.T
    blk = (MU0_4PI / 1e-3) * dd * np.exp(-dist / L_RANGE_MM)
    rows = np.arange(r0, r1)
    blk[rows - r0, rows] += L_REG
    out[r0:r1] = blk


def inductance(g: Geometry, out: np.ndarray | None = None, threads: int | None = None,
               rows_per_task: int = 256) -> np.ndarray:
    """Dense symmetric L (n x n, FP64).  Symmetric, so row- and column-major agree."""
    n = g.n
    if out is None:
        out = np.empty((n, n), dtype=np.float64)
    tasks = [(r, min(n, r + rows_per_task)) for r in range(0, n, rows_per_task)]
    threads = threads or min(32, os.cpu_count() or 1)
    if threads <= 1 or len(tasks) == 1:
        for r0, r1 in tasks:
            _fill_L_rows(g, out, r0, r1)
    else:
        with ThreadPoolExecutor(threads) as ex:
            list(ex.map(lambda t: _fill_L_rows(g, out, *t), tasks))
    return out


def laplacian_edges(g: Geometry) -> np.ndarray:
    """Pairs (a, b), a < b, of 6-neighbour cells that are both among the n unknowns."""
    nx, ny, nz = g.grid
    n = g.n
    idx = np.arange(n)
    edges = []
    for step, ax_len, coord in ((1, nx, g.ijk[:, 0]), (nx, ny, g.ijk[:, 1]), (nx * ny, nz, g.ijk[:, 2])):
        a = idx[(coord + 1 < ax_len) & (idx + step < n)]
        edges.append(np.stack([a, a + step], axis=1))
    return np.concatenate(edges, axis=0)


def resistance(g: Geometry, out: np.ndarray | None = None) -> np.ndarray:
    """Dense R = diag(rho g) + LAP_OHM * graph Laplacian (n x n, FP64)."""
    n = g.n
    if out is None:
        out = np.zeros((n, n), dtype=np.float64)
    else:
        out[...] = 0.0
    e = laplacian_edges(g)
    deg = np.bincount(e.ravel(), minlength=n).astype(np.float64)
    out[np.arange(n), np.arange(n)] = g.rho * G_FACTOR + LAP_OHM * deg
    out[e[:, 0], e[:, 1]] = -LAP_OHM
    out[e[:, 1], e[:, 0]] = -LAP_OHM
    return out


def mutual(g: Geometry, points_mm: np.ndarray) -> np.ndarray:
    """(n x q) mutuals between the cells and q points (coil centres or pickups)."""
    diff = g.pos_mm[:, None, :] - np.asarray(points_mm, dtype=np.float64)[None, :, :]
    dist = np.sqrt(np.einsum("abk,abk->ab", diff, diff))
    return (MU0_4PI / 1e-3) * np.exp(-dist / M_RANGE_MM)


def pickup_grid(nx: int, ny: int, z_mm: float = 5.0) -> np.ndarray:
    xs = (np.arange(nx) + 0.5) * PLATE_MM[0] / nx
    ys = (np.arange(ny) + 0.5) * PLATE_MM[1] / ny
    X, Y = np.meshgrid(xs, ys, indexing="xy")
    return np.stack([X.ravel(), Y.ravel(), np.full(X.size, z_mm)], axis=1)


def electrode_rows(g: Geometry) -> np.ndarray:
    """(1 x n) reduced incidence: x-min face kept, x-max face dropped."""
    e = np.zeros((1, g.n), dtype=np.float64)
    face = g.ijk[:, 0] == 0
    e[0, face] = -np.cos(g.phi[face])
    return e


# Tone frequencies [Hz] of the multi-sine excitation of the paper's NdT experiment
# (Sec. 4.3): 30 tones from 1 Hz to 10 kHz, amplitude 4 A each.
MULTISINE_HZ = (1.0, 50.0, 100.0, 150.0, 250.0, 300.0, 400.0, 600.0, 700.0, 800.0, 900.0,
                1000.0, 1500.0, 2000.0, 2500.0, 3000.0, 3500.0, 4000.0, 4500.0, 5000.0, 5500.0,
                6000.0, 6500.0, 7000.0, 7500.0, 8000.0, 8500.0, 9000.0, 9500.0, 10000.0)
MULTISINE_AMP = 4.0


def multisine(T: int, dt: float, t0: float = 0.0, freqs=MULTISINE_HZ,
              amp: float = MULTISINE_AMP) -> np.ndarray:
    """i(t) = sum_k amp sin(2 pi f_k t + phi_k), phi_k = -pi k (k-1) / N_s (k = 1..N_s),
    sampled at t_j = t0 + j dt, j = 0..T."""
    t = t0 + np.arange(T + 1, dtype=np.float64) * dt
    ns = len(freqs)
    out = np.zeros(T + 1)
    for k, f in enumerate(freqs, start=1):
        out += amp * np.sin(2.0 * np.pi * f * t - np.pi * k * (k - 1) / ns)
    return out


def sine(T: int, dt: float, f_hz: float, amp: float = 1.0, phase: float = 0.0) -> np.ndarray:
    t = np.arange(T + 1, dtype=np.float64) * dt
    return amp * np.sin(2.0 * np.pi * f_hz * t + phase)


def step_current(T: int, amp: float = 1.0) -> np.ndarray:
    s = np.full(T + 1, amp, dtype=np.float64)
    s[0] = 0.0
    return s


@dataclass
class Problem:
    """One seeded workload: matrices, sources and run parameters."""
    name: str
    L: np.ndarray
    R: np.ndarray
    E: np.ndarray            # (m, n), m = Ne - 1 (may be 0)
    M: np.ndarray            # (n, S) coil mutuals
    MD: np.ndarray           # (n, m) electrode-source mutuals
    C: np.ndarray            # (P, n) probe rows
    src: np.ndarray          # (S, T+1) coil currents i_0 at t_k = k dt
    iD: np.ndarray           # (m, T+1) electrode currents
    theta: float
    dt: float
    T: int
    snap_stride: int
    geom: Geometry | None = None
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.L.shape[0]


def config1(T: int = 2000, seed: int = 0, n: int = 512) -> Problem:
    """N=512 plate, one coil at (20,10,5) mm, sin 10 kHz, dt = 1 us, probe = coil self-pickup."""
    g = geometry(n, seed)
    M = mutual(g, np.array([[20.0, 10.0, 5.0]]))
    dt = 1e-6
    return Problem("n512_coil", inductance(g), resistance(g), np.zeros((0, n)), M,
                   np.zeros((n, 0)), M.T.copy(), sine(T, dt, 1e4)[None, :], np.zeros((0, T + 1)),
                   0.5, dt, T, 0, g)


def config2(T: int = 20000, seed: int = 0, n: int = 8192, snap_stride: int = 100) -> Problem:
    """N=8192 plate, 2 electrodes with a 1 A step, 16 pickups at z = 5 mm, dt = 0.5 us."""
    g = geometry(n, seed)
    C = mutual(g, pickup_grid(4, 4)).T.copy()
    dt = 0.5e-6
    return Problem("n8192_electrodes", inductance(g), resistance(g), electrode_rows(g),
                   np.zeros((n, 0)), np.zeros((n, 1)), C, np.zeros((0, T + 1)),
                   step_current(T)[None, :], 0.5, dt, T, snap_stride, g)


def config4(T: int = 100000, seed: int = 0, n: int = 65536, snap_stride: int = 1000,
            L_out: np.ndarray | None = None, R_out: np.ndarray | None = None) -> Problem:
    """N=65536 plate, one coil (sin 10 kHz), 4 pickups, dt = 0.1 us, no electrodes."""
    g = geometry(n, seed)
    M = mutual(g, np.array([[20.0, 10.0, 5.0]]))
    C = mutual(g, pickup_grid(2, 2)).T.copy()
    dt = 1e-7
    return Problem("n65536_coil", inductance(g, L_out), resistance(g, R_out), np.zeros((0, n)), M,
                   np.zeros((n, 0)), C, sine(T, dt, 1e4)[None, :], np.zeros((0, T + 1)),
                   0.5, dt, T, snap_stride, g)


def small(n: int, T: int, seed: int = 0, electrodes: bool = True, coil: bool = True,
          probes: int = 4, dt: float = 1e-6, theta: float = 0.5, snap_stride: int = 0,
          f_hz: float = 1e4) -> Problem:
    """Small mixed case: optional electrode step and coil, a few pickups."""
    g = geometry(n, seed)
    E = electrode_rows(g) if electrodes else np.zeros((0, n))
    M = mutual(g, np.array([[20.0, 10.0, 5.0]])) if coil else np.zeros((n, 0))
    px = max(1, int(math.isqrt(probes)))
    pts = pickup_grid(px, max(1, probes // px))
    C = mutual(g, pts).T.copy()
    MD = 0.25 * mutual(g, np.array([[0.0, 10.0, 3.0]])) if electrodes else np.zeros((n, 0))
    src = sine(T, dt, f_hz)[None, :] if coil else np.zeros((0, T + 1))
    iD = step_current(T)[None, :] if electrodes else np.zeros((0, T + 1))
    return Problem(f"n{n}_small", inductance(g), resistance(g), E, M, MD, C, src, iD,
                   theta, dt, T, snap_stride, g)


def coil_scan(n: int, T: int, n_side: int = 16, seed: int = 0, dt: float = 1e-6,
              f_hz: float = 1e4, probes: int = 0) -> Problem:
    """Independent excitations: n_side x n_side coils at z = 5 mm over the plate (one
    right-hand side each), every coil driven by sin(2 pi f t); probes: each coil's own
    pickup (C = M^T) unless ``probes`` > 0 pickups on a grid are requested."""
    g = geometry(n, seed)
    M = mutual(g, pickup_grid(n_side, n_side))
    if probes:
        px = max(1, int(math.isqrt(probes)))
        C = mutual(g, pickup_grid(px, max(1, probes // px), z_mm=4.0)).T.copy()
    else:
        C = M.T.copy()
    S = M.shape[1]
    src = np.repeat(sine(T, dt, f_hz)[None, :], S, axis=0)
    return Problem(f"n{n}_coilscan{S}", inductance(g), resistance(g), np.zeros((0, n)), M,
                   np.zeros((n, 0)), C, src, np.zeros((0, T + 1)), 0.5, dt, T, 0, g)
