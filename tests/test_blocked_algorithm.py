"""The mixed path's blocked LU and block triangular solves, restated in numpy
(no GPU).

The FP32 factorisation in the CUDA path (lu_blocked / solve_blocked) keeps its
factors in an unusual layout: panels of 32 columns; after a panel, L11^{-1}
(strict lower part, unit diagonal implied) is stored over L11 and U12 =
L11^{-1} A12 over A12; after the last panel each upper diagonal block holds
U_bb^{-1} (strict upper part) with the reciprocal pivots kept apart; the block
solves then apply those inverses. This restatement, in float64, must solve
M x = b for sizes with one partial block, exact multiples of 32 and ragged
tails. It pins the layout conventions (which block an inverse belongs to, how
a partial last block is aligned) independently of the GPU; the GPU parity
tests check the CUDA code itself against the oracle.
"""
import numpy as np
import pytest
import scipy.linalg

NB = 32


def lu_blocked(A):
    M = np.array(A, dtype=float)
    S = M.shape[0]
    invd = np.zeros(S)
    for kb in range(0, S, NB):
        nb = min(NB, S - kb)
        ke = kb + nb
        # panel: columns kb..ke-1 of rows kb..S-1, right-looking inside the panel
        for c in range(nb):
            k = kb + c
            invd[k] = 1.0 / M[k, k]
            M[k + 1:, k] *= invd[k]
            M[k + 1:, k + 1:ke] -= np.outer(M[k + 1:, k], M[k, k + 1:ke])
        L11 = np.tril(M[kb:ke, kb:ke], -1) + np.eye(nb)
        L11inv = scipy.linalg.solve_triangular(L11, np.eye(nb), lower=True, unit_diagonal=True)
        M[kb:ke, ke:] = L11inv @ M[kb:ke, ke:]                              # U12
        M[kb:ke, kb:ke] = np.triu(M[kb:ke, kb:ke]) + np.tril(L11inv, -1)   # L11^{-1} over L11
        M[ke:, ke:] -= M[ke:, kb:ke] @ M[kb:ke, ke:]                        # A22 -= L21 U12
    for kb in range(0, S, NB):
        ke = min(S, kb + NB)
        U = np.triu(M[kb:ke, kb:ke])
        Uinv = scipy.linalg.solve_triangular(U, np.eye(ke - kb), lower=False)
        np.testing.assert_allclose(np.diag(Uinv), invd[kb:ke], rtol=1e-14)
        M[kb:ke, kb:ke] = np.tril(M[kb:ke, kb:ke], -1) + np.triu(Uinv, 1)
    return M, invd


def solve_blocked(M, invd, b):
    v = np.array(b, dtype=float)
    S = v.size
    for kb in range(0, S, NB):
        ke = min(S, kb + NB)
        v[kb:ke] = (np.tril(M[kb:ke, kb:ke], -1) + np.eye(ke - kb)) @ v[kb:ke]
        v[ke:] -= M[ke:, kb:ke] @ v[kb:ke]
    for kb in reversed(range(0, S, NB)):
        ke = min(S, kb + NB)
        v[kb:ke] = (np.triu(M[kb:ke, kb:ke], 1) + np.diag(invd[kb:ke])) @ v[kb:ke]
        v[:kb] -= M[:kb, kb:ke] @ v[kb:ke]
    return v


@pytest.mark.parametrize("S", [1, 5, 31, 32, 33, 64, 95, 150, 257])
def test_blocked_factor_solves(S):
    rng = np.random.default_rng(S)
    # I - cJ-like: unit-dominant diagonal, mixed-sign off-diagonal entries
    A = np.eye(S) * (1.0 + rng.uniform(0.0, 5.0, S)) + rng.normal(0.0, 0.3 / np.sqrt(S), (S, S))
    b = rng.normal(size=S)
    M, invd = lu_blocked(A)
    x = solve_blocked(M, invd, b)
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-9, atol=1e-12)


def test_bottom_aligned_partial_block_is_caught():
    # a plausible slip: reading the partial last block as the bottom NB rows
    # (overlapping the previous block) in the block solves; the restated solve
    # above would then fail, so the parametrised test distinguishes the two
    S = 45
    rng = np.random.default_rng(1)
    A = np.eye(S) * 3.0 + rng.normal(0.0, 0.2, (S, S))
    b = rng.normal(size=S)
    M, invd = lu_blocked(A)
    starts = [0, S - NB]
    v = np.array(b)
    for kb in starts:
        ke = kb + NB
        v[kb:ke] = (np.tril(M[kb:ke, kb:ke], -1) + np.eye(NB)) @ v[kb:ke]
        v[ke:] -= M[ke:, kb:ke] @ v[kb:ke]
    for kb in reversed(starts):
        ke = kb + NB
        v[kb:ke] = (np.triu(M[kb:ke, kb:ke], 1) + np.diag(invd[kb:ke])) @ v[kb:ke]
        v[:kb] -= M[:kb, kb:ke] @ v[kb:ke]
    assert not np.allclose(v, np.linalg.solve(A, b), rtol=1e-6)
    np.testing.assert_allclose(solve_blocked(M, invd, b), np.linalg.solve(A, b), rtol=1e-9)
