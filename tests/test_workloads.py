"""The synthetic input recipe: the generator builds exactly the arrays the recipe states
(grid, cell centres, draw order, kernels, electrode row, waveforms), reproducibly."""
import numpy as np
import pytest

from workloads import synth


@pytest.mark.parametrize("n,grid", [(512, (16, 8, 4)), (8192, (32, 32, 8)), (65536, (64, 64, 16))])
def test_named_grids_and_cell_centres(n, grid):
    g = synth.geometry(n, seed=0)
    assert g.grid == grid and g.pos_mm.shape == (n, 3)
    h = np.array(synth.PLATE_MM) / np.array(grid)
    assert np.allclose(g.pos_mm.min(axis=0), 0.5 * h) and np.allclose(g.pos_mm.max(axis=0),
                                                                       np.array(synth.PLATE_MM) - 0.5 * h)
    assert np.array_equal(g.ijk[1], [1, 0, 0]) and np.array_equal(g.ijk[grid[0]], [0, 1, 0])


def test_draw_order_and_ranges():
    g = synth.geometry(300, seed=7)
    rng = np.random.default_rng(7)
    assert np.array_equal(g.phi, rng.uniform(0.0, 2.0 * np.pi, size=300))
    assert np.array_equal(g.rho, 10.0 ** rng.uniform(-8.0, -7.0, size=300))
    assert np.all((g.rho >= 1e-8) & (g.rho <= 1e-7))
    g2 = synth.geometry(300, seed=7)
    assert np.array_equal(g.phi, g2.phi) and np.array_equal(g.rho, g2.rho)


def test_inductance_and_resistance_follow_the_recipe():
    g = synth.geometry(200, seed=3)
    L = synth.inductance(g)
    R = synth.resistance(g)
    i, j = 5, 77
    dist = np.linalg.norm(g.pos_mm[i] - g.pos_mm[j])
    expect = 1e-7 * (g.dirs[i] @ g.dirs[j]) * np.exp(-dist / 2.0) / 1e-3
    assert np.isclose(L[i, j], expect, rtol=1e-14)
    assert np.isclose(L[i, i], 1e-7 / 1e-3 + 1e-9, rtol=1e-14)
    assert np.array_equal(L, L.T)
    deg = -(R - np.diag(np.diag(R))).sum(axis=1) / 1e-4
    assert np.allclose(np.diag(R), g.rho * 1e3 + 1e-4 * deg)
    assert set(np.unique(R[R < 0])) == {-1e-4}


def test_electrode_row_on_the_x_min_face():
    g = synth.geometry(512, seed=0)
    E = synth.electrode_rows(g)
    assert E.shape == (1, 512)
    face = g.ijk[:, 0] == 0
    assert np.allclose(E[0, face], -g.dirs[face, 0])
    assert np.all(E[0, ~face] == 0.0)


def test_waveforms():
    T, dt = 1000, 1e-6
    s = synth.sine(T, dt, 1e4)
    assert s.shape == (T + 1,) and s[0] == 0.0
    assert np.isclose(s[25], np.sin(2 * np.pi * 1e4 * 25 * dt))
    st = synth.step_current(T)
    assert st[0] == 0.0 and np.all(st[1:] == 1.0)
    assert len(synth.MULTISINE_HZ) == 30 and synth.MULTISINE_AMP == 4


def test_coil_scan_pairs_each_coil_with_its_own_pickup():
    p = synth.coil_scan(256, T=4, n_side=3)
    assert p.M.shape == (256, 9) and p.C.shape == (9, 256) and np.array_equal(p.C, p.M.T)
    assert p.src.shape == (9, 5) and np.allclose(p.src, p.src[0])
