"""Pins for the oracle's starting step and simplified-Newton corrector (no GPU).

initial_step (Hairer, Norsett & Wanner I, Sec. II.4):
  * against scipy's own implementation of the same published procedure
    (``scipy.integrate._ivp.common.select_initial_step``, a library routine
    used as a checker) on the 32- and 150-species networks;
  * against a value derived by hand for a linear network A -> B, where the
    Euler difference f(y0 + h0 f0) - f0 = h0 K^2 y0 is exact, so d2 = |K^2 y0|;
  * a planted wrong exponent (order 2 in place of 1, i.e. 1/3 in place of
    1/2) must fail that hand-derived value.

newton_corrector (Hairer & Wanner II, Sec. IV.8): for a scalar corrector
G(d) = a d + b with a frozen derivative m, every increment is known in closed
form: the error contracts by exactly theta = |1 - a/m| per increment and the
increment norms are n_k = (a/m) theta^(k-1) |d*| / scale. The tests pick
(a, m) so that the published rules give a known outcome at a known increment
and compare the oracle's outcome, increment count and result with it; a
linear system with the exact matrix must converge to the direct solution.
"""
import numpy as np
import pytest
import scipy.linalg

from oracle import bdf, chem
from paper_2511_10558_gb300 import synth
from tests.nets import tiny

YR = synth.YEAR


def _scipy_h0(f, t0, y0, f0, t_end, rtol, atol):
    common = pytest.importorskip("scipy.integrate._ivp.common")
    try:
        return common.select_initial_step(f, t0, y0, t_end, np.inf, f0, 1.0, 1, rtol, atol)
    except TypeError:
        pytest.skip("scipy's select_initial_step has another signature here")


@pytest.mark.parametrize("S,R", [(32, 200), (150, 1500)])
@pytest.mark.parametrize("rtol,atol", [(1e-4, 1e-20), (1e-8, 1e-26)])
def test_initial_step_matches_library(S, R, rtol, atol):
    net = synth.make_network(S, R)
    x0 = synth.initial_abundances(net)
    nu = chem.stoichiometry(net)
    for phi in synth.cells(3, seed=5):
        kap = chem.effective_coefficients(net, phi)
        f = lambda t, y: chem.rhs(net, kap, y, nu)  # noqa: E731
        f0 = f(0.0, x0)
        t_end = 1e6 * YR
        mine = bdf.initial_step(f, 0.0, x0, f0, t_end, rtol, atol)
        lib = _scipy_h0(f, 0.0, x0, f0, t_end, rtol, atol)
        assert mine == pytest.approx(lib, rel=1e-12)


def _decay_case(alpha=1e11):
    # A -> B (cosmic-ray form), x0 = (a, b): f = K x with K = [[-k, 0], [k, 0]]
    net = tiny(2, [(synth.COSMIC_RAY, (0,), (1,), alpha, 0.0, 0.0)])
    phi = [1e4, 20.0, 0.0, 1.0, 1.3e-17]
    k = alpha * 1.3e-17
    kap = chem.effective_coefficients(net, phi)
    f = lambda t, y: chem.rhs(net, kap, y)  # noqa: E731
    return net, k, f


def _hand_h0(k, y0, rtol, atol, t_end, p=1):
    # derived by hand for f = K y, K = [[-k, 0], [k, 0]]:
    #   f0 = (-k a, k a); K^2 y0 = (k^2 a, -k^2 a) (the Euler step is exact
    #   for the difference of f), so d2 = |K^2 y0| with the same weights
    a, b = y0
    s = atol + rtol * np.abs(y0)
    rms = lambda v: float(np.sqrt(np.mean((np.asarray(v) / s) ** 2)))  # noqa: E731
    d0, d1 = rms([a, b]), rms([-k * a, k * a])
    h0 = 1e-6 if min(d0, d1) < 1e-5 else 0.01 * d0 / d1
    d2 = rms([k * k * a, -k * k * a])
    h1 = (0.01 / max(d1, d2)) ** (1.0 / (p + 1))
    return min(100 * h0, h1, t_end), h0, h1


@pytest.mark.parametrize("alpha,a,b,binding", [(1e11, 2e-4, 5e-5, "h1"), (1e11, 1e-3, 1e-4, "h1"),
                                                (1e11, 1e-3, 1e-20, "100 h0"), (50.0, 2e-4, 5e-5, "100 h0")])
def test_initial_step_hand_derived(alpha, a, b, binding):
    # (the last case has d1 < 1e-5, where step (b) takes h0 = 1e-6)
    net, k, f = _decay_case(alpha)
    y0 = np.array([a, b])
    rtol, atol, t_end = 1e-4, 1e-20, 1e13
    got = bdf.initial_step(f, 0.0, y0, f(0.0, y0), t_end, rtol, atol)
    want, h0, h1 = _hand_h0(k, y0, rtol, atol, t_end)
    assert got == pytest.approx(want, rel=1e-12)
    assert (h1 < 100 * h0) == (binding == "h1") and min(h1, 100 * h0) < t_end


def test_initial_step_planted_exponent_is_caught():
    net, k, f = _decay_case(1e11)
    y0 = np.array([2e-4, 5e-5])
    rtol, atol, t_end = 1e-4, 1e-20, 1e13
    want = _hand_h0(k, y0, rtol, atol, t_end)[0]
    planted = bdf.initial_step(f, 0.0, y0, f(0.0, y0), t_end, rtol, atol, order=2)
    assert abs(planted / want - 1) > 1e-3


def _scalar_newton(a, m, b, tol, scale=1.0, maxiter=bdf.NEWTON_MAXITER):
    # G(d) = d - c f(y_p + d) + psi with f(y) = -k y, so G(d) = a d + b with
    # a = 1 + c k and b = c k y_p + psi; frozen "matrix" m (its 1x1 LU)
    c = 1.0
    k = a - 1.0
    y_p = 0.0
    psi = b
    lu = scipy.linalg.lu_factor(np.array([[m]]))
    fun = lambda t, y: -k * y  # noqa: E731
    return bdf.newton_corrector(fun, 0.0, np.array([y_p]), c, np.array([psi]), lu, np.array([scale]), tol,
                                maxiter)


def test_newton_exact_matrix_solves_linear_corrector():
    # exact frozen matrix on a linear problem: d_1 is the solution, the second
    # increment is zero up to rounding, so it converges at increment 2
    rng = np.random.default_rng(3)
    S = 6
    K = -np.diag(rng.uniform(1, 5, S)) + 0.3 * rng.uniform(0, 1, (S, S))
    c = 0.7
    y_p = rng.uniform(0.5, 1.0, S)
    psi = rng.normal(size=S) * 0.1
    lu = scipy.linalg.lu_factor(np.eye(S) - c * K)
    conv, n, y, d = bdf.newton_corrector(lambda t, y: K @ y, 0.0, y_p, c, psi, lu, np.ones(S), 1e-8)
    want = np.linalg.solve(np.eye(S) - c * K, c * K @ y_p - psi)
    assert conv and n == 2
    np.testing.assert_allclose(d, want, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(y, y_p + want, rtol=1e-12, atol=1e-14)


def test_newton_converges_where_the_tail_bound_says():
    # theta = 1 - a/m = 0.1; n_k = 0.9 * 0.1^(k-1) |d*|, |d*| = b/a
    a, m, b = 0.9, 1.0, 0.9
    dstar = -b / a
    tol = 0.005
    # k = 2: theta/(1-theta) n_2 = (1/9) 0.09 = 0.01 >= tol -> continue;
    # k = 3: (1/9) 0.009 = 0.001 < tol -> converged at increment 3
    conv, n, y, d = _scalar_newton(a, m, b, tol)
    assert conv and n == 3
    assert abs(d[0] - dstar) <= 0.1 ** 3 * abs(dstar) * (1 + 1e-12)


def test_newton_abandoned_by_the_tail_rule():
    # theta = 0.5, |d*| = 1: n_1 = 0.5, n_2 = 0.25; after increment 2 the
    # expected bound after the last permitted increment is
    # theta^(4-2+1)/(1-theta) n_2 = 0.0625 > tol = 0.05 -> abandoned at k = 2,
    # before increment 2 is applied (d = d_1 = 0.5 d*)
    a, m, b = 1.0, 2.0, 1.0
    conv, n, y, d = _scalar_newton(a, m, b, tol=0.05)
    assert not conv and n == 2
    assert d[0] == pytest.approx(-0.5, rel=1e-15)
    # with tol just above that bound it continues, and converges once
    # theta/(1-theta) n_k < tol: n_3 = 0.125 -> 0.125 >= 0.07, n_4 = 0.0625 < 0.07
    conv, n, y, d = _scalar_newton(a, m, b, tol=0.07)
    assert conv and n == 4


def test_newton_stops_without_contraction():
    # theta = |1 - a/m| = 1.5 >= 1: abandoned at the second increment
    a, m, b = 2.5, 1.0, 1.0
    conv, n, y, d = _scalar_newton(a, m, b, tol=1e-3)
    assert not conv and n == 2
    assert d[0] == pytest.approx(-b / m, rel=1e-15)  # only the first increment was applied


def test_newton_nonfinite_rhs_abandons():
    lu = scipy.linalg.lu_factor(np.eye(2))
    conv, n, y, d = bdf.newton_corrector(lambda t, y: np.array([np.nan, 0.0]), 0.0, np.ones(2), 1.0,
                                         np.zeros(2), lu, np.ones(2), 1e-3)
    assert not conv and n == 1
    np.testing.assert_array_equal(d, 0.0)
