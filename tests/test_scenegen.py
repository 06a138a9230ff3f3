"""Input generators: the on-demand cell records equal what the grid fill stores (the oracle's tabled
render of the 1024^3 precision workload relies on it)."""

import numpy as np

import scenegen


def test_cell_records_equal_grid_fill_tiny():
    w = scenegen.tiny()
    _, uvw = scenegen.fill_position_grid(w.scene, w.k)
    cells = np.unique(np.random.default_rng(3).integers(0, w.k ** 3, 4000))
    assert np.array_equal(scenegen.cell_records(w.scene, w.k, cells), uvw.reshape(-1, 3 * w.D)[cells])


def test_cell_records_equal_grid_fill_k1024_slab():
    w = scenegen.precision()
    k, z0, nz = w.k, 517, 2
    sig, uvw = scenegen.fill_position_grid(w.scene, k, z0, nz)
    rng = np.random.default_rng(4)
    local = np.unique(rng.integers(0, nz * k * k, 3000))
    cells = local + z0 * k * k
    assert np.array_equal(scenegen.cell_records(w.scene, k, cells), uvw.reshape(-1, 3 * w.D)[local])
    # the slab contains occupied cells, so the sigma plane is not trivially empty
    assert (sig > 0).any()


def test_precision_workload_shape():
    w = scenegen.precision()
    assert (w.k, w.l, w.D, w.W, w.H, w.n_samples, w.n_cams) == (1024, 768, 8, 800, 800, 192, 16)
