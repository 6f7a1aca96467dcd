"""Writes rhmc_rational_m0.3.json: Remez approximations (paper_1801_01473_gb300.rational, mpmath)
of x^(+1/8) (pseudofermion heatbath) and x^(-1/4) (action and force) on [0.05, 16.5], which holds
the spectrum of m^2 - D_eo D_oe at m = 0.3 on any SU(3) links (m^2 <= lambda <= m^2 + 16).  The
table serves machines without mpmath (the RHMC tests and the trajectory benchmark).

    python paper_1801_01473_gb300/data/make_rational.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))  # the repository root

from paper_1801_01473_gb300.rational import remez  # noqa: E402


def main():
    out = {}
    for name, power in (("heatbath", 0.125), ("action", -0.25)):
        r = remez(power, 10, 0.05, 16.5)
        out[name] = {"power": r.power, "lo": r.lo, "hi": r.hi, "alpha0": r.alpha0, "residues": r.residues,
                     "poles": r.poles, "max_rel_error": r.max_rel_error}
    with open(os.path.join(HERE, "rhmc_rational_m0.3.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
