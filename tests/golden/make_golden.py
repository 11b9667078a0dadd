"""Write tests/golden/cell32.json: the oracle's result for the single-cell case.

Calls only ``oracle/`` and the seeded input generator. Case: 32 species /
200 reactions (seed 1032), n_H = 1e4 cm^-3, T = 20 K, A_V = 5, G0 = 1,
zeta = 1.3e-17 s^-1, integrated 0 -> 1e6 yr at rtol 1e-4, atol 1e-20.

Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import bdf  # noqa: E402
from paper_2511_10558_gb300 import synth  # noqa: E402


def main():
    net = synth.make_network(32, 200)
    x0 = synth.initial_abundances(net)
    phi = synth.one_cell()[0]
    res = bdf.solve_cell(net, phi, x0, 0.0, 1e6 * synth.YEAR, 1e-4, 1e-20)
    out = dict(case="32 species / 200 reactions, seed 1032, one cell, 1e6 yr, rtol 1e-4, atol 1e-20",
               phi=list(map(float, phi)), t_end=1e6 * synth.YEAR, status=res.status,
               stats=res.stats, names=net.names, x=[float(v) for v in res.x])
    with open(os.path.join(ROOT, "tests", "golden", "cell32.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
