"""Writes the stored expected values under tests/golden/ by calling only the
FP64 oracle (oracle/) on seeded synthetic inputs (synthetic/).

    python tests/golden/make_golden.py

mscg_4x4x4x4_scalars.txt: the first 25 rows (alpha_k, beta_k, zeta_i^{k+1}) of
the multi-shift CG recurrences on the 4^4 workload (Haar links seed 1001,
Gaussian source seed 2001, m = 0.1, 8 shifts log-spaced 1e-4..1).
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import synthetic as S  # noqa: E402


def main():
    cfg = S.CONFIGS["small_4x4x4x4"]
    dims = cfg["dims"]
    u = S.gauge_links(dims, cfg["links"], 1000 + cfg["k"])
    b = S.gaussian_field(dims, 2000 + cfg["k"])
    res = oracle.mscg(dims, u, cfg["mass"], cfg["shifts"](), b, tol=cfg["tol"], log_rows=25)
    hdr = ("multi-shift CG recurrences, 4^4 Haar links (seed 1001), source seed 2001, m=0.1, "
           "8 shifts logspace(1e-4,1); columns: alpha_k beta_k zeta_0..zeta_7 (Sec. 2, Eq. shift_eo); "
           f"written by tests/golden/make_golden.py from the FP64 oracle; total iterations {res['iters']}")
    np.savetxt(os.path.join(HERE, "mscg_4x4x4x4_scalars.txt"), res["scalar_log"], fmt="%.17e", header=hdr)


if __name__ == "__main__":
    main()
