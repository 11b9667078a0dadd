"""The reorganised schedules of the LU and solves, restated in numpy (no GPU).

Three restructurings of the CUDA path change when an operation runs but not
what it computes; each is restated here with the same loop bounds and
operation order as the kernel, and checked against the plain form:

* FP64 LU, dense range: two pivots per barrier (dense_rank_rows). Every later
  row forms its L entry of column k+1 first, then takes -a u_k and -b u_{k+1};
  warp 0 finishes the next two U rows. The schedule performs each element's
  operations in the same order as single pivots do, so the factors must agree
  bit for bit. That includes the single-pivot steps before the 128-column
  limit and the one-pivot step that enters the pairs.
* FP64 triangular solves, look-ahead (forward_crout / backward_crout): block
  b-1 reaches the rows beyond block b+1 while block b's chain runs, and block
  b reaches block b+1 through per-warp partial sums. The schedule must solve
  the system (to rounding) for every size, ragged or not.
* FP64 blocked LU for networks in global memory, sparse leading panels: the
  trailing update of a leading panel is taken from each pivot's structural U
  list, restricted to the columns after the panel, and skips zero
  multipliers. On the 500-species synthetic network's fill pattern it must
  equal the dense update bit for bit, i.e. the lists cover every non-zero of
  the panel's U12 and L21.
"""
import numpy as np
import pytest
import scipy.linalg

from paper_2511_10558_gb300 import synth
from tests.test_dense_range_exact import crout, pattern_and_fill

NB = 32
PAIR_COLS = 128  # the pair step's column limit in the kernel


def _finish_row(M, p, prev=None):
    """Warp 0's finish of row p: pivot `prev` (a finished row above, applied to
    columns > prev) if given, then the reciprocal pivot and the scaling of U(p, :)."""
    if prev is not None:
        a = M[p, prev]
        M[p, prev + 1:] = M[p, prev + 1:] - a * M[prev, prev + 1:]
    inv = 1.0 / M[p, p]
    M[p, p + 1:] = M[p, p + 1:] * inv


def _rank_step(M, k, R):
    """Pivots k..k+R-1 (finished U rows, scaled) applied to every row i >= k+R:
    for R = 2 the L entry of column k+1 first, then -a u_k and -b u_{k+1}, each
    column in that order; warp 0 then finishes rows k+R and k+R+1."""
    S = M.shape[0]
    c0 = k + R
    for i in range(c0, S):
        a = M[i, k]
        if R == 2:
            b = M[i, k + 1] - a * M[k, k + 1]
            M[i, k + 1] = b
        x = M[i, c0:] - a * M[k, c0:]
        if R == 2:
            x = x - b * M[k + 1, c0:]
        M[i, c0:] = x
    _finish_row(M, c0)
    if c0 + 1 < S:
        _finish_row(M, c0 + 1, prev=c0)


def crout_pairs(A, F, kd):
    """The kernel's schedule: single pivots (pattern lists below kd, full ranges
    above) up to kp, the first dense pivot with at most PAIR_COLS columns after
    it; then pivot kp alone, finishing rows kp+1 and kp+2; then pairs."""
    M = A.copy()
    S = M.shape[0]
    kp = max(kd, S - 1 - PAIR_COLS)
    pairs = S - kp >= 3
    k_single = kp if pairs else S
    for k in range(k_single):
        inv = 1.0 / M[k, k]
        if k < kd:
            rows = np.flatnonzero(F[k + 1:, k]) + k + 1
            cols = np.flatnonzero(F[k, k + 1:]) + k + 1
        else:
            rows = cols = np.arange(k + 1, S)
        M[k, cols] *= inv
        for i in rows:
            M[i, cols] -= M[i, k] * M[k, cols]
    if pairs:
        M[kp, kp + 1:] *= 1.0 / M[kp, kp]   # U row kp finished by the single steps
        _rank_step(M, kp, 1)
        k = kp + 1
        while k + 2 < S:
            _rank_step(M, k, 2)
            k += 2
    return M


def _dense_case(S, seed):
    rng = np.random.default_rng(seed)
    A = rng.normal(0.0, 1.0, (S, S))
    A[np.diag_indices(S)] = 5.0 + np.abs(A).sum(axis=1)
    return A, np.ones((S, S), dtype=bool)


@pytest.mark.parametrize("S", [3, 4, 5, 6, 33, 64, 129, 130, 131, 200, 256])
def test_paired_pivots_dense_bitwise(S):
    # kd = 0: every pivot dense; S > 129 has single dense steps before the pairs
    A, F = _dense_case(S, S)
    np.testing.assert_array_equal(crout_pairs(A, F, 0), crout(A, F, 0))


@pytest.mark.parametrize("kd", [0, 23, 37, 146, 147, 148, 150])
def test_paired_pivots_network_bitwise(kd):
    # the 150-species network's pattern, kd from all-dense to no dense range
    # (S - kd < 3: no pairs at all)
    net = synth.make_network(150, 1500)
    P, F = pattern_and_fill(net)
    S = net.n_species
    rng = np.random.default_rng(kd)
    A = np.where(P, rng.normal(0.0, 1.0, (S, S)), 0.0)
    A[np.diag_indices(S)] = 5.0 + np.abs(A).sum(axis=1)
    np.testing.assert_array_equal(crout_pairs(A, F, kd), crout(A, F, kd))


def _forward_lookahead(L, v):
    """forward_crout's schedule on a unit lower L: per block b, warp 0's chain on
    block b (its right-hand side less the partial sums of block b-1), the other
    warps' block b-1 on the rows below block b+1, then warps 0..3 (8 columns
    each) block b on block b+1's rows into partial sums."""
    S = len(v)
    v = v.copy()
    nblk = (S + 31) // 32
    part = np.zeros((4, 32))
    for b in range(nblk):
        kb = 32 * b
        nb = min(32, S - kb)
        if b > 0:
            v[kb + 32:] -= L[kb + 32:, kb - 32:kb] @ v[kb - 32:kb]
        val = v[kb:kb + nb].copy()
        if b > 0:
            val -= part.sum(axis=0)[:nb]
        for c in range(nb):
            val[c + 1:] -= L[kb + c + 1:kb + nb, kb + c] * val[c]
        v[kb:kb + nb] = val
        if b + 1 < nblk:
            part[:] = 0.0
            rows = np.arange(kb + 32, min(kb + 64, S))
            for w in range(4):
                cw = slice(kb + 8 * w, kb + 8 * w + 8)
                part[w, :len(rows)] = L[rows, cw] @ v[cw]
    return v


def _backward_lookahead(U, v):
    """backward_crout's schedule on a unit upper U, blocks from the bottom (the
    bottom block may be partial): block b+1 reaches the rows above block b
    while block b's chain runs; block b reaches block b-1 through partial sums."""
    S = len(v)
    v = v.copy()
    nblk = (S + 31) // 32
    part = np.zeros((4, 32))
    for b in range(nblk - 1, -1, -1):
        kb = 32 * b
        nb = min(32, S - kb)
        if b + 1 < nblk and b > 0:
            kn = kb + 32
            nc = min(32, S - kn)
            v[:kb] -= U[:kb, kn:kn + nc] @ v[kn:kn + nc]
        val = v[kb:kb + nb].copy()
        if b + 1 < nblk:
            val -= part.sum(axis=0)[:nb]
        for c in range(nb - 1, -1, -1):
            val[:c] -= U[kb:kb + c, kb + c] * val[c]
        v[kb:kb + nb] = val
        if b > 0:
            part[:] = 0.0
            rows = np.arange(kb - 32, kb)
            for w in range(4):
                c1 = min(kb + 8 * w + 8, kb + nb)
                if kb + 8 * w < c1:
                    part[w] = U[rows, kb + 8 * w:c1] @ v[kb + 8 * w:c1]
    return v


@pytest.mark.parametrize("S", [1, 5, 31, 32, 33, 63, 64, 65, 96, 100, 150, 200, 255, 256])
def test_lookahead_solves(S):
    rng = np.random.default_rng(S)
    A = rng.normal(0.0, 0.1, (S, S))
    L = np.tril(A, -1) + np.eye(S)
    U = np.triu(A, 1) + np.eye(S)
    v = rng.normal(0.0, 1.0, S)
    want_f = scipy.linalg.solve_triangular(L, v, lower=True, unit_diagonal=True)
    want_b = scipy.linalg.solve_triangular(U, v, lower=False, unit_diagonal=True)
    np.testing.assert_allclose(_forward_lookahead(L, v), want_f, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(_backward_lookahead(U, v), want_b, rtol=1e-12, atol=1e-12)


def _panel(M, kb):
    """The blocked LU's panel (columns kb..kb+31 of the rows below, then U12 =
    L11^{-1} A12), as in the kernel's panel_factor and panel_u12."""
    ke = kb + NB
    for c in range(NB):
        k = kb + c
        M[k + 1:, k] /= M[k, k]
        M[k + 1:, k + 1:ke] -= np.outer(M[k + 1:, k], M[k, k + 1:ke])
    L11 = np.tril(M[kb:ke, kb:ke], -1) + np.eye(NB)
    M[kb:ke, ke:] = scipy.linalg.solve_triangular(L11, M[kb:ke, ke:], lower=True, unit_diagonal=True)


def test_sparse_leading_panels_listed_update_is_exact():
    from paper_2511_10558_gb300 import carbox
    net = synth.make_network(500, 6000)
    N = carbox.Network.from_synth(net)
    perm, F, _kd = N.symbolic()
    N.close()
    P_user, _ = pattern_and_fill(net)
    P = P_user[np.ix_(perm, perm)]          # the library's (internal) order
    S = P.shape[0]
    rng = np.random.default_rng(7)
    A = np.where(P, rng.normal(0.0, 1.0, (S, S)), 0.0)
    A[np.diag_indices(S)] = 5.0 + np.abs(A).sum(axis=1)
    dense, listed = A.copy(), A.copy()
    touched = 0
    for kb in (0, NB):                      # the 500-species network's two sparse panels
        ke = kb + NB
        _panel(dense, kb)
        _panel(listed, kb)
        np.testing.assert_array_equal(dense, listed)
        for k in range(kb, ke):
            dense[ke:, ke:] -= np.outer(dense[ke:, k], dense[k, ke:])
            rows = np.flatnonzero(listed[ke:, k] != 0.0) + ke
            cols = np.flatnonzero(F[k, ke:]) + ke
            listed[np.ix_(rows, cols)] -= np.outer(listed[rows, k], listed[k, cols])
            touched += len(rows) * len(cols)
        np.testing.assert_array_equal(dense, listed)
    # and the lists do skip most of the dense work on these panels
    assert touched < 0.25 * sum((S - kb - NB) ** 2 * NB for kb in (0, NB))
