"""The C-ABI library builds, loads and exports every symbol of include/*.h (no GPU)."""
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2511_10558_gb300 import build
    build.build()
    from paper_2511_10558_gb300 import carbox
    return carbox


def declared_symbols():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"^\s*(?:int|double|const char\*)\s+(cbx_\w+)\s*\(", txt, re.M))
    return names


def test_exports_every_declared_symbol(lib):
    names = declared_symbols()
    assert {"cbx_network_create", "cbx_solve", "cbx_solve_host", "cbx_last_error", "cbx_peak_fma"} <= names
    out = subprocess.run(["nm", "-D", "--defined-only", lib._LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (cbx_\w+)", out))
    assert names <= exported, names - exported
    for n in names:
        assert hasattr(lib.lib, n)


def test_host_compiler_figures(lib):
    from paper_2511_10558_gb300 import synth
    N = lib.Network.from_synth(synth.make_network(150, 1500))
    info = N.info()
    assert info["S"] == 150 and info["R"] == 1500
    assert info["nnz_jac"] <= info["nnz_lu"] <= 150 * 150
    assert 0 < info["lu_flops"] <= info["lu_flops_dense"] * 1.0001 + 150 * 150


def _jacobian_pattern(net):
    # J(i, l) != 0 when l is a reactant of a reaction whose net stoichiometry
    # changes species i, plus the diagonal of I - cJ (user order)
    S = net.n_species
    pat = np.eye(S, dtype=bool)
    for j in range(net.n_reactions):
        nu = {}
        for a in net.reac[j]:
            if a >= 0:
                nu[a] = nu.get(a, 0) - 1
        for p in net.prod[j]:
            if p >= 0:
                nu[p] = nu.get(p, 0) + 1
        for l in (a for a in net.reac[j] if a >= 0):
            for i, v in nu.items():
                if v != 0:
                    pat[i, l] = True
    return pat


def _eliminate(F):
    """Plain boolean Gaussian elimination with diagonal pivots, in order."""
    F = F.copy()
    S = F.shape[0]
    flops = 0.0
    for k in range(S):
        rows = np.flatnonzero(F[k + 1:, k]) + k + 1
        cols = np.flatnonzero(F[k, k + 1:]) + k + 1
        F[np.ix_(rows, cols)] = True
        flops += len(rows) + 2.0 * len(rows) * len(cols)
    return F, flops


@pytest.mark.parametrize("S,R", [(32, 200), (150, 1500), (500, 6000)])
def test_host_compiler_fill_matches_dense_elimination(lib, S, R):
    # bit-exact: the library's L + U pattern in its own order equals a plain
    # boolean elimination of pattern(J + I) permuted to that order, and its
    # flop count and nnz follow from that pattern
    from paper_2511_10558_gb300 import synth
    net = synth.make_network(S, R)
    N = lib.Network.from_synth(net)
    info = N.info()
    perm, fill, kdense = N.symbolic()
    assert sorted(perm) == list(range(S))
    pat = _jacobian_pattern(net)
    assert info["nnz_jac"] == pat.sum()
    want, flops = _eliminate(pat[np.ix_(perm, perm)])
    np.testing.assert_array_equal(fill, want)
    assert info["nnz_lu"] == want.sum()
    assert info["lu_flops"] == flops
    assert 0 <= kdense <= S


def test_host_compiler_order_is_minimum_degree(lib):
    # property of the order: each eliminated node had the smallest degree (ties:
    # smallest index) in the elimination graph of pattern(J + J^T) at its turn
    from paper_2511_10558_gb300 import synth
    net = synth.make_network(32, 200)
    N = lib.Network.from_synth(net)
    perm, _, _ = N.symbolic()
    pat = _jacobian_pattern(net)
    adj = (pat | pat.T) & ~np.eye(net.n_species, dtype=bool)
    alive = np.ones(net.n_species, bool)
    for v in perm:
        deg = np.where(alive, (adj & alive[None, :]).sum(axis=1), np.iinfo(np.int64).max)
        assert deg[v] == deg.min() and v == int(np.flatnonzero(deg == deg.min())[0])
        nb = np.flatnonzero(adj[v] & alive)
        alive[v] = False
        adj[np.ix_(nb, nb)] = True
        adj[nb, nb] = False


def test_create_rejects_bad_input(lib):
    import ctypes as C
    sp = (lib.cbx_species * 2)()
    rx = (lib.cbx_reaction * 1)()
    rx[0].type = lib.CBX_TWO_BODY
    rx[0].reac[:] = [0, 5]          # out of range
    rx[0].prod[:] = [1, -1, -1, -1]
    h = C.c_void_p()
    assert lib.lib.cbx_network_create(sp, 2, rx, 1, C.byref(h)) == lib.CBX_E_ARG
    assert b"out of range" in lib.lib.cbx_last_error() or b"do not fit" in lib.lib.cbx_last_error()
    rx[0].reac[:] = [0, 1]
    rx[0].prod[:] = [-1, -1, -1, -1]  # no product
    assert lib.lib.cbx_network_create(sp, 2, rx, 1, C.byref(h)) == lib.CBX_E_ARG
    rx[0].type = 9
    assert lib.lib.cbx_network_create(sp, 2, rx, 1, C.byref(h)) == lib.CBX_E_ARG


def test_set_albedo_checks(lib):
    import ctypes as C
    from paper_2511_10558_gb300 import synth
    N = lib.Network.from_synth(synth.make_network(32, 200, cr_photo_frac=0.5))
    assert lib.lib.cbx_network_set_albedo(N.handle, C.c_double(0.3)) == lib.CBX_OK
    for bad in (1.0, -0.1, float("nan"), 2.0):
        assert lib.lib.cbx_network_set_albedo(N.handle, C.c_double(bad)) == lib.CBX_E_ARG
    assert lib.lib.cbx_network_set_albedo(None, C.c_double(0.3)) == lib.CBX_E_ARG


def test_esdirk_tableau_of_the_library(lib):
    # the library derives the ESDIRK tableau on its own (C++); it must satisfy
    # the order conditions and match the oracle's independent derivation
    from oracle import esdirk
    A, c, gamma = lib.esdirk_tableau()
    b, bh = A[4], A[3]
    Ac = A @ c
    for v, want in ((b.sum(), 1), (b @ c, 1 / 2), (b @ c ** 2, 1 / 3), (b @ Ac, 1 / 6), (b @ c ** 3, 1 / 4),
                    (b @ (c * Ac), 1 / 8), (b @ (A @ c ** 2), 1 / 12), (b @ (A @ Ac), 1 / 24),
                    (bh.sum(), 1), (bh @ c, 1 / 2), (bh @ c ** 2, 1 / 3), (bh @ Ac, 1 / 6)):
        assert abs(v - want) < 1e-14
    assert gamma == pytest.approx(0.5728160625, abs=1e-9)
    np.testing.assert_allclose(A, esdirk.A_TAB, rtol=0, atol=1e-14)
    np.testing.assert_allclose(c, esdirk.C_TAB, rtol=0, atol=1e-14)
