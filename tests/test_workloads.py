"""The seeded synthetic workloads have the sizes of the workloads they stand
for (mesh 64 x 4 bar with 1024 particles; 200 x 40 x 100 column with 512,000
particles and 832,341 nodes; 256 batched 2D columns; 800 x 200 x 200 slope with
about 64M particles) and are reproducible from their seeds."""
import numpy as np

from paper_1909_13380_gb300 import workloads as W


def test_bar_counts():
    wl = W.elastic_bar()
    assert wl.n == 1024 and wl.num_nodes == 65 * 5
    assert np.isclose(wl.vol.sum() * 1000.0, 2560.0)
    # all particles strictly inside the mesh, 4 per cell
    cells = np.floor(wl.pos / wl.h).astype(int)
    _, counts = np.unique(cells[:, 0] + 64 * cells[:, 1], return_counts=True)
    assert len(counts) == 256 and np.all(counts == 4)


def test_column3d_counts():
    wl = W.column3d()
    assert wl.n == 512_000 and wl.num_nodes == 832_341
    assert wl.pos.max() < 0.2 and wl.pos.min() > 0.0


def test_columns2d_batch_reproducible():
    a = W.columns2d_batch(count=256)
    b = W.columns2d_batch(count=256)
    assert len(a) == 256
    n = np.array([w.n for w in a])
    assert np.array_equal(n, [w.n for w in b])
    assert n.min() >= 4000 and n.max() <= 70000
    assert 4e6 < n.sum() < 8e6


def test_slope_section_and_cohesion():
    wl = W.slope3d(ncells=(800, 2, 200))
    per_slice = wl.meta["filled_cells"] // 2
    assert abs(per_slice - 40_000) <= 400          # 100 m2 section / 0.05^2
    assert wl.n == 8 * wl.meta["filled_cells"]
    coh = wl.coh[::8]
    assert abs(coh.mean() / 10e3 - 1) < 0.02 and abs(coh.std() / coh.mean() - 0.3) < 0.02
    # full size: 200 slices of the same section -> about 64M particles
    assert abs(8 * 200 * per_slice - 64.0e6) < 0.7e6
