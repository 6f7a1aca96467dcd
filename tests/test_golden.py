"""Stored expected values (tests/golden/) re-derived from the oracle, and the
data-structure sizes the paper prints (no GPU)."""
import json
import os

import numpy as np

import oracle
import synthetic as S

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_mscg_scalar_log_reproduces():
    ref = np.loadtxt(os.path.join(GOLDEN, "mscg_4x4x4x4_scalars.txt"))
    cfg = S.CONFIGS["small_4x4x4x4"]
    u = S.gauge_links(cfg["dims"], cfg["links"], 1000 + cfg["k"])
    b = S.gaussian_field(cfg["dims"], 2000 + cfg["k"])
    res = oracle.mscg(cfg["dims"], u, cfg["mass"], cfg["shifts"](), b, tol=cfg["tol"], log_rows=ref.shape[0])
    np.testing.assert_allclose(res["scalar_log"], ref, rtol=1e-12)


def test_paper_sizes_file_is_consistent():
    """The printed sizes agree with each other: 3 double complex per site is
    48 B; a packet of one colour component over n0 n1 n2 / 2 sites is
    8 n0 n1 n2 B; a 2-thick gauge halo of 4 compressed links per site is 768 B."""
    sizes = json.load(open(os.path.join(GOLDEN, "paper_sizes.json")))
    assert sizes["fermion_bytes_per_site_fp64"]["value"] == 3 * 16
    assert sizes["gauge_halo_bytes_per_surface_site_compressed"]["value"] == 2 * 4 * 12 * 8
    n0, n1, n2 = 32, 32, 32
    assert sizes["dirac_halo_packet_bytes_per_n0n1n2"]["value"] * n0 * n1 * n2 == 16 * (n0 * n1 * n2 // 2)
