"""Host-side helpers of bench.py that prepare inputs (no GPU)."""
import os
import sys

import numpy as np
import pytest

import synthetic as S

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_tile_links_repeats_the_small_lattice():
    """The RHMC start repeats a small lattice's links along every direction: every link of the
    large lattice is the small lattice's link at the coordinates taken modulo the small extents,
    so the gauge action (periodic links) is the small one times the number of copies."""
    import bench
    from oracle import gauge as og
    small, reps = (4, 2, 4, 6), 2
    u = S.gauge_links(small, "expih", 7)
    big = bench.tile_links(torch.from_numpy(u), small, reps).numpy()
    dims = tuple(reps * n for n in small)
    assert big.shape == (4, int(np.prod(dims)), 3, 3)
    rng = np.random.default_rng(1)
    for _ in range(50):
        x = [int(rng.integers(n)) for n in dims]
        i = x[0] + dims[0] * (x[1] + dims[1] * (x[2] + dims[2] * x[3]))
        j = (x[0] % small[0]) + small[0] * ((x[1] % small[1]) + small[1] * ((x[2] % small[2]) + small[2] * (x[3] % small[3])))
        assert np.array_equal(big[:, i], u[:, j])
    s_small = og.action(small, u, 5.6)
    s_big = og.action(dims, big, 5.6)
    assert abs(s_big / reps ** 4 - s_small) <= 1e-12 * abs(s_small)
