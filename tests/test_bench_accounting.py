"""The benchmark's flop accounting, the numerator of every ALU roofline (no GPU).

Per unit, as the roofline states it: one LU = F_LU of the symbolic fill; one
Newton iteration = one triangular-solve pair = 2 nnz(L+U); one right-hand side
= 2 R_two + R_one (rates) + n_nu (gather); one Jacobian = 2 R_two + 2 n_nu;
one refinement sweep = 2 nnz(J) in FP64 (residual) + 2 nnz(L+U) in FP32
(correction solve). The mixed path counts the LU and every solve pair in FP32
and the rest in FP64. Checked on a hand-built network whose counts are
written out, with counters chosen so that each term has its own magnitude.
"""
import numpy as np
import pytest

import bench
from paper_2511_10558_gb300 import synth
from tests.nets import tiny

TB, CR, PH = synth.TWO_BODY, synth.COSMIC_RAY, synth.PHOTO


def _net():
    # 4 species; reactions: A+B->C+D (two-body), A+A->B (two-body),
    # C->D (CR), D->A+B (photo)
    return tiny(4, [(TB, (0, 1), (2, 3), 1.0, 0.0, 0.0),
                    (TB, (0, 0), (1,), 1.0, 0.0, 0.0),
                    (CR, (2,), (3,), 1.0, 0.0, 0.0),
                    (PH, (3,), (0, 1), 1.0, 0.0, 0.0)])


def test_network_counts_by_hand():
    # two-body reactions: 2; one-body: 2; stoichiometric entries (reactant and
    # product slots): (2+2) + (2+1) + (1+1) + (1+2) = 12
    assert bench.network_counts(_net()) == (2, 2, 12)


def _stats():
    # two cells, counters of distinct magnitudes so that a swapped term shows
    return {"lu_factors": np.array([3, 4]), "newton_iters": np.array([10, 20]),
            "rhs_evals": np.array([100, 300]), "jac_evals": np.array([1000, 2000]),
            "refine_sweeps": np.array([5, 7])}


INFO = {"lu_flops": 1.0e6, "nnz_lu": 1000, "nnz_jac": 50}


def test_algorithmic_flops_terms():
    fl = bench.algorithmic_flops(INFO, _stats(), 2, 2, 12)
    assert fl["lu"] == 7 * 1.0e6
    assert fl["solve"] == 30 * 2 * 1000
    assert fl["rhs"] == 400 * (2 * 2 + 2 + 12)
    assert fl["jac"] == 3000 * (2 * 2 + 2 * 12)
    assert fl["refine_fp64"] == 12 * 2 * 50
    assert fl["refine_fp32"] == 12 * 2 * 1000


def test_mixed_flops_split():
    f32, f64 = bench.mixed_flops(INFO, _stats(), 2, 2, 12)
    # FP32: the LUs, the solve pair of every Newton iteration and of every sweep
    assert f32 == 7 * 1.0e6 + 30 * 2 * 1000 + 12 * 2 * 1000
    # FP64: rates and gathers, Jacobians, the residual of every sweep
    assert f64 == 400 * 18 + 3000 * 28 + 12 * 2 * 50


@pytest.mark.parametrize("S,R", [(32, 200), (150, 1500)])
def test_network_counts_synthetic(S, R):
    net = synth.make_network(S, R)
    r_two, r_one, n_nu = bench.network_counts(net)
    assert r_two + r_one == R
    assert r_two == sum(1 for j in range(R) if net.rtype[j] == TB)
    assert n_nu == sum(int(s >= 0) for j in range(R) for s in list(net.reac[j]) + list(net.prod[j]))
