"""The oracle still reproduces its stored single-cell result (regression pin)."""
import json
import os

import numpy as np

from oracle import bdf
from paper_2511_10558_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def test_cell32_golden(net32):
    g = json.load(open(os.path.join(HERE, "golden", "cell32.json")))
    assert g["names"] == net32.names
    res = bdf.solve_cell(net32, np.array(g["phi"]), synth.initial_abundances(net32), 0.0,
                         g["t_end"], 1e-4, 1e-20)
    assert res.status == g["status"]
    assert res.stats == g["stats"]
    np.testing.assert_allclose(res.x, g["x"], rtol=1e-12, atol=1e-30)
