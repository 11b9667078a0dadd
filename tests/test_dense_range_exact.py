"""Pin of the FP64 LU's dense-range reading (no GPU).

The CUDA path factors pivots k >= kd over the full index ranges k+1..S-1
instead of the symbolic L(:,k) / U(k,:) lists, with kd chosen by a cost
model. That is exact: an entry outside the symbolic fill of I - cJ is never
written by an earlier pivot, so it holds an exact zero, and every extra
a_ik u_kj term is zero. Restated in numpy on the 150-species synthetic
network's pattern with random values: the Crout factorisation with pattern
lists for k < kd and full ranges for k >= kd equals, bit for bit, the one with
pattern lists throughout, for every kd.
"""
import numpy as np
import pytest

from oracle import chem
from paper_2511_10558_gb300 import synth


def pattern_and_fill(net):
    S = net.n_species
    P = np.eye(S, dtype=bool)
    for j in range(net.n_reactions):
        species = [s for s in list(net.reac[j]) + list(net.prod[j]) if s >= 0]
        for l in [s for s in net.reac[j] if s >= 0]:
            for i in species:
                P[i, l] = True
    F = P.copy()
    for k in range(S):
        rows = np.flatnonzero(F[k + 1:, k]) + k + 1
        cols = np.flatnonzero(F[k, k + 1:]) + k + 1
        F[np.ix_(rows, cols)] = True
    return P, F


def crout(A, F, kd):
    """U rows scaled by 1/pivot as they are finished, rank-1 updates; pattern lists
    for k < kd, full ranges for k >= kd."""
    M = A.copy()
    S = M.shape[0]
    for k in range(S):
        inv = 1.0 / M[k, k]
        if k < kd:
            rows = np.flatnonzero(F[k + 1:, k]) + k + 1
            cols = np.flatnonzero(F[k, k + 1:]) + k + 1
        else:
            rows = cols = np.arange(k + 1, S)
        M[k, cols] *= inv
        for i in rows:
            M[i, cols] -= M[i, k] * M[k, cols]
    return M


@pytest.mark.parametrize("seed", [0, 1])
def test_dense_range_is_exact(seed):
    net = synth.make_network(150, 1500)
    P, F = pattern_and_fill(net)
    S = net.n_species
    rng = np.random.default_rng(seed)
    A = np.where(P, rng.normal(0.0, 1.0, (S, S)), 0.0)
    A[np.diag_indices(S)] = 5.0 + np.abs(A).sum(axis=1)
    ref = crout(A, F, S)          # pattern lists throughout
    for kd in (0, 23, 37, 100):
        np.testing.assert_array_equal(crout(A, F, kd), ref)
    # and the result is a factorisation: L D U = A
    L = np.tril(ref, -1) + np.eye(S)
    D = np.diag(np.diag(ref))
    U = np.triu(ref, 1) + np.eye(S)
    Lu = L.copy()
    Lu[np.tril_indices(S, -1)] = (ref / np.diag(ref)[None, :])[np.tril_indices(S, -1)]
    np.testing.assert_allclose(Lu @ D @ U, A, rtol=1e-12, atol=1e-12 * np.abs(A).max())
