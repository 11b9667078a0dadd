"""Pins for the oracle's ESDIRK integrator of Kvaerno's family (no GPU).

* The tableau: every order condition of Butcher's trees up to order 4 for the
  solution and up to order 3 for the embedded solution (including the trees
  the derivation does not impose directly), stage order 2, the published
  diagonal value gamma = 0.5728160625 of Kvaerno's order-4 method (BIT 44,
  2004), and the stability function R(z) = det(I - zA + z 1 b^T) / det(I - zA)
  evaluated in 50-digit arithmetic: R(-inf) = 0 and |R| <= 1 on the imaginary
  axis and in the left half-plane.
* Observed orders with fixed steps on a linear system against its matrix
  exponential: 4 for the solution, 3 for the embedded one; a planted change of
  one coefficient is caught.
* Closed forms (A -> B, A + B -> C, A + A -> C), conservation on synthetic
  networks, scipy's Radau IIA at tight tolerance, and agreement with the BDF
  oracle within the methods' global errors.
"""
import mpmath
import numpy as np
import pytest
import scipy.integrate
import scipy.linalg

from oracle import bdf, chem, esdirk
from paper_2511_10558_gb300 import synth
from tests.nets import tiny

YR = synth.YEAR
A, c, gamma = esdirk.A_TAB, esdirk.C_TAB, esdirk.GAMMA
b, bh = A[4], A[3]


def test_order_conditions():
    Ac, Ac2 = A @ c, A @ c ** 2
    AAc = A @ Ac
    conds = {  # Butcher trees up to order 4: sum over the weights equals 1 / tree factorial
        "1": (b.sum(), 1), "c": (b @ c, 1 / 2), "c2": (b @ c ** 2, 1 / 3), "Ac": (b @ Ac, 1 / 6),
        "c3": (b @ c ** 3, 1 / 4), "cAc": (b @ (c * Ac), 1 / 8), "Ac2": (b @ Ac2, 1 / 12), "AAc": (b @ AAc, 1 / 24)}
    for name, (v, want) in conds.items():
        assert v == pytest.approx(want, abs=1e-14), name
    for name, (v, want) in {"1": (bh.sum(), 1), "c": (bh @ c, 1 / 2), "c2": (bh @ c ** 2, 1 / 3),
                            "Ac": (bh @ Ac, 1 / 6)}.items():
        assert v == pytest.approx(want, abs=1e-14), name
    # the embedded solution is only order 3
    assert abs(bh @ c ** 3 - 1 / 4) > 1e-3
    # stage order 2 and the structure of the family
    np.testing.assert_allclose(A.sum(axis=1), c, atol=1e-15)
    np.testing.assert_allclose(Ac[1:], c[1:] ** 2 / 2, atol=1e-15)
    assert np.all(A[0] == 0) and c[3] == c[4] == 1.0 and c[1] == pytest.approx(2 * gamma)
    np.testing.assert_array_equal(np.diag(A)[1:], gamma)
    assert np.all(np.triu(A, 1) == 0)


def test_gamma_is_kvaernos():
    assert gamma == pytest.approx(0.5728160625, abs=1e-9)


def _R(z, Am=A):
    mpmath.mp.dps = 50
    s = Am.shape[0]
    M = mpmath.matrix(s, s)
    N = mpmath.matrix(s, s)
    for i in range(s):
        for j in range(s):
            M[i, j] = (1 if i == j else 0) - z * mpmath.mpf(float(Am[i, j]))
            N[i, j] = M[i, j] + z * mpmath.mpf(float(Am[-1, j]))
    return mpmath.det(N) / mpmath.det(M)


def test_stability_function():
    assert abs(_R(mpmath.mpf("-1e40"))) < 1e-12          # L-stable
    for y in np.logspace(-3, 6, 40):
        assert abs(_R(mpmath.mpc(0, y))) <= 1 + 1e-12      # A-stable on the axis
    for x in -np.logspace(-2, 4, 12):
        for y in np.concatenate([[0.0], np.logspace(-2, 4, 12)]):
            assert abs(_R(mpmath.mpc(x, y))) <= 1 + 1e-12
    # the embedded method is A-stable too (not L-stable)
    for y in np.logspace(-3, 6, 20):
        assert abs(_R(mpmath.mpc(0, y), A[:4, :4])) <= 1 + 1e-12
    # the oracle's closed form for R(-inf) agrees
    assert abs(esdirk.stability_at_infinity(A)) < 1e-14


def _linear_problem():
    K = np.array([[-2.0, 1.0, 0.0], [1.0, -3.0, 0.5], [0.2, 0.4, -1.0]])
    y0 = np.array([1.0, 0.5, -0.3])
    return K, y0


def _fixed_errors(tab=None):
    K, y0 = _linear_problem()
    T = 2.0
    exact = scipy.linalg.expm(K * T) @ y0
    out = []
    for n in (16, 32, 64):  # powers of two: the steps sum to T exactly
        res = esdirk.integrate(lambda t, y: K @ y, lambda t, y: K, 0.0, y0, T, 1e-12, 1e-14,
                               fixed_h=T / n, tableau=tab)
        assert res.stats["steps"] == n
        out.append((np.max(np.abs(res.x - exact)), n))
    return out, K, y0, exact


def _observed_orders(errs):
    return [np.log2(e1 / e2) for (e1, _), (e2, _) in zip(errs, errs[1:])]


def test_observed_order_four():
    errs, *_ = _fixed_errors()
    for p in _observed_orders(errs):
        assert 3.8 < p < 4.3, p


def test_embedded_order_three():
    # the embedded solution after one step of size h has local error O(h^4)
    K, y0 = _linear_problem()
    loc = []
    for h in (2.0 ** -4, 2.0 ** -5, 2.0 ** -6):
        res = esdirk.integrate(lambda t, y: K @ y, lambda t, y: K, 0.0, y0, h, 1e-12, 1e-14, fixed_h=h)
        exact = scipy.linalg.expm(K * h) @ y0
        loc.append((np.max(np.abs(res.stats["embedded"] - exact)), np.max(np.abs(res.x - exact))))
    for (e1, m1), (e2, m2) in zip(loc, loc[1:]):
        assert 3.7 < np.log2(e1 / e2) < 4.3      # local order p_hat + 1 = 4
        assert 4.6 < np.log2(m1 / m2) < 5.4      # local order p + 1 = 5


def test_planted_coefficient_is_caught():
    bad = A.copy()
    bad[4, 2] += 1e-3
    bad[4, 0] -= 1e-3  # keep the row sum (consistency) so only the higher conditions break
    errs, *_ = _fixed_errors((bad, c, gamma))
    assert min(_observed_orders(errs)) < 3.0


def _solve(net, phi, x0, t_end, rtol=1e-10, atol=1e-30):
    res = esdirk.solve_cell(net, phi, np.asarray(x0, float), 0.0, t_end, rtol, atol)
    assert res.status == esdirk.OK and res.t == t_end
    return res.x


@pytest.mark.parametrize("rt", [synth.COSMIC_RAY, synth.PHOTO, synth.CR_PHOTO])
def test_first_order_decay(rt):
    alpha = {synth.COSMIC_RAY: 50.0, synth.PHOTO: 1e-10, synth.CR_PHOTO: 1.2}[rt]
    net = tiny(2, [(rt, (0,), (1,), alpha, 0.0, 1500.0 if rt == synth.CR_PHOTO else 1.5)])
    net.albedo = 0.5
    phi = [1e4, 20.0, 0.5, 1.0, 1.3e-17]
    k = chem.rate_coefficients(net, phi)[0]
    t = 4.0 / k
    a, b0 = 1e-3, 1e-20
    x = _solve(net, phi, [a, b0], t)
    np.testing.assert_allclose(x, [a * np.exp(-k * t), b0 + a * (1 - np.exp(-k * t))], rtol=2e-7)


def test_second_order_closed_forms():
    net = tiny(3, [(synth.TWO_BODY, (0, 1), (2,), 1e-10, 0.5, 20.0)])
    phi = [1e3, 50.0, 0.0, 1.0, 0.0]
    kap = chem.effective_coefficients(net, phi)[0]
    a, bb = 3e-4, 1e-4
    dlt = a - bb
    t = 5.0 / (dlt * kap)
    x = _solve(net, phi, [a, bb, 0.0], t)
    xa = dlt * a / (a - bb * np.exp(-dlt * kap * t))
    np.testing.assert_allclose(x, [xa, xa - dlt, a - xa], rtol=2e-7)
    net = tiny(2, [(synth.TWO_BODY, (0, 0), (1,), 2e-10, 0.0, 0.0)])
    phi = [1e4, 300.0, 0.0, 1.0, 0.0]
    kap = chem.effective_coefficients(net, phi)[0]
    t = 50.0 / (kap * 1e-3)
    x = _solve(net, phi, [1e-3, 0.0], t)
    xa = 1.0 / (1.0 / 1e-3 + 2 * kap * t)
    np.testing.assert_allclose(x, [xa, (1e-3 - xa) / 2], rtol=2e-7)


@pytest.mark.parametrize("S,R", [(32, 200), (150, 1500)])
def test_conservation_synthetic(S, R):
    net = synth.make_network(S, R)
    x0 = synth.initial_abundances(net)
    E0, Q0 = chem.element_totals(net, x0)
    phi = synth.cells(1, seed=2)[0]
    res = esdirk.solve_cell(net, phi, x0, 0.0, 1e6 * YR, 1e-4, 1e-20)
    assert res.status == esdirk.OK
    E1, Q1 = chem.element_totals(net, res.x)
    assert np.all(np.abs(E1 - E0) <= 1e-10 * E0)
    assert abs(Q1 - Q0) <= 1e-10 * (np.abs(net.charge) @ x0)


def test_against_library_radau(net32):
    x0 = synth.initial_abundances(net32)
    phi = synth.one_cell()[0]
    kap = chem.effective_coefficients(net32, phi)
    nu = chem.stoichiometry(net32)
    t = 1e4 * YR
    lib = scipy.integrate.solve_ivp(lambda t, y: chem.rhs(net32, kap, y, nu), (0, t), x0, method="Radau",
                                    jac=lambda t, y: chem.jacobian(net32, kap, y, nu), rtol=1e-11, atol=1e-30)
    assert lib.success
    x = esdirk.solve_cell(net32, phi, x0, 0.0, t, 1e-9, 1e-28).x
    big = lib.y[:, -1] > 1e-12
    np.testing.assert_allclose(x[big], lib.y[big, -1], rtol=3e-6)


def test_self_convergence_and_agreement_with_bdf(net32):
    x0 = synth.initial_abundances(net32)
    phi = synth.one_cell()[0]
    t = 1e5 * YR
    ref = bdf.solve_cell(net32, phi, x0, 0.0, t, 1e-12, 1e-30).x
    big = ref > 1e-12
    errs = []
    for rtol in [1e-4, 1e-6]:
        x = esdirk.solve_cell(net32, phi, x0, 0.0, t, rtol, 1e-20 * rtol / 1e-4).x
        errs.append(np.max(np.abs(x[big] / ref[big] - 1)))
    assert errs[1] < errs[0] / 10
    for e, rtol in zip(errs, [1e-4, 1e-6]):
        assert e < 1e3 * rtol
    # cross-method: at rtol 1e-4 both methods are within their global errors of the reference
    xb = bdf.solve_cell(net32, phi, x0, 0.0, t, 1e-4, 1e-20).x
    xe = esdirk.solve_cell(net32, phi, x0, 0.0, t, 1e-4, 1e-20).x
    assert np.max(np.abs(xb[big] / ref[big] - 1)) < 1e-1 and np.max(np.abs(xe[big] / ref[big] - 1)) < 1e-1
