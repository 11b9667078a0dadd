"""Pins for the oracle's BDF integrator (no GPU).

Each pin comes from outside the oracle: polynomial interpolation (numpy
polyfit) for the step-size rescale, exactness of order-q BDF on degree-q
polynomials, closed-form solutions of one-reaction networks, the matrix
exponential (scipy) for linear networks, element/charge conservation,
self-convergence under tightened tolerances, and an independent library
integrator (scipy's Radau IIA) at tight tolerance.
"""
import math

import numpy as np
import pytest
import scipy.integrate
import scipy.linalg

from oracle import bdf, chem
from paper_2511_10558_gb300 import synth
from tests.nets import tiny

YR = synth.YEAR


@pytest.mark.parametrize("q", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("rho", [0.2, 0.5, 2.0, 10.0])
def test_rescale_matches_interpolation(q, rho):
    rng = np.random.default_rng(q)
    coef = rng.normal(size=q + 1)
    h = 0.7
    ts = -h * np.arange(q + 1)
    ys = np.polyval(coef, ts)
    D = np.zeros((bdf.MAX_ORDER + 3, 1))
    # backward differences of the samples
    for k in range(q + 1):
        D[k, 0] = sum((-1) ** i * math.comb(k, i) * ys[i] for i in range(k + 1))
    bdf.rescale_differences(D, q, rho)
    ys_new = np.polyval(coef, -rho * h * np.arange(q + 1))
    want = [sum((-1) ** i * math.comb(k, i) * ys_new[i] for i in range(k + 1)) for k in range(q + 1)]
    np.testing.assert_allclose(D[:q + 1, 0], want, rtol=1e-10, atol=1e-10)


@pytest.mark.parametrize("q", [1, 2, 3, 4, 5])
def test_bdf_exact_on_polynomials(q):
    # order-q BDF reproduces degree-q polynomials: predictor exact (d = 0) and
    # gamma_q * psi = sum_j gamma_j nabla^j y_n equals h y'(t_{n+1})
    rng = np.random.default_rng(10 + q)
    coef = rng.normal(size=q + 1)
    h = 0.3
    ts = -h * np.arange(q + 1)
    ys = np.polyval(coef, ts)
    D = np.array([sum((-1) ** i * math.comb(k, i) * ys[i] for i in range(k + 1)) for k in range(q + 1)])
    assert D.sum() == pytest.approx(np.polyval(coef, h), rel=1e-12, abs=1e-12)
    psi_times_gamma = sum(bdf.GAMMA[j] * D[j] for j in range(1, q + 1))
    assert psi_times_gamma == pytest.approx(h * np.polyval(np.polyder(coef), h), rel=1e-10, abs=1e-12)
    assert bdf.GAMMA[q] == pytest.approx(sum(1.0 / j for j in range(1, q + 1)))


def _solve(net, phi, x0, t_end, rtol=1e-10, atol=1e-30):
    res = bdf.solve_cell(net, phi, np.asarray(x0, float), 0.0, t_end, rtol, atol)
    assert res.status == bdf.OK
    assert res.t == t_end
    return res.x


@pytest.mark.parametrize("rt", [synth.COSMIC_RAY, synth.PHOTO, synth.CR_PHOTO])
def test_first_order_decay(rt):
    # A -> B: x_A = a exp(-k t), x_B = b0 + a (1 - exp(-k t))
    alpha = {synth.COSMIC_RAY: 50.0, synth.PHOTO: 1e-10, synth.CR_PHOTO: 1.2}[rt]
    net = tiny(2, [(rt, (0,), (1,), alpha, 0.4 if rt == synth.CR_PHOTO else 0, 1500.0 if rt == synth.CR_PHOTO else 1.5)])
    net.albedo = 0.5
    phi = [1e4, 20.0, 0.5, 1.0, 1.3e-17]
    k = chem.rate_coefficients(net, phi)[0]
    t = 4.0 / k
    a, b0 = 1e-3, 1e-20
    x = _solve(net, phi, [a, b0], t)
    np.testing.assert_allclose(x, [a * np.exp(-k * t), b0 + a * (1 - np.exp(-k * t))], rtol=2e-7)


def test_second_order_distinct():
    # A + B -> C: x_A = D a / (a - b exp(-D kappa t)), D = a - b
    net = tiny(3, [(synth.TWO_BODY, (0, 1), (2,), 1e-10, 0.5, 20.0)])
    phi = [1e3, 50.0, 0.0, 1.0, 0.0]
    kap = chem.effective_coefficients(net, phi)[0]
    a, b = 3e-4, 1e-4
    dlt = a - b
    t = 5.0 / (dlt * kap)
    x = _solve(net, phi, [a, b, 0.0], t)
    xa = dlt * a / (a - b * np.exp(-dlt * kap * t))
    np.testing.assert_allclose(x, [xa, xa - dlt, a - xa], rtol=2e-7)


def test_second_order_identical():
    # A + A -> C: 1/x_A = 1/a + 2 kappa t (A consumed twice per event)
    net = tiny(2, [(synth.TWO_BODY, (0, 0), (1,), 2e-10, 0.0, 0.0)])
    phi = [1e4, 300.0, 0.0, 1.0, 0.0]
    kap = chem.effective_coefficients(net, phi)[0]
    a = 1e-3
    t = 50.0 / (kap * a)
    x = _solve(net, phi, [a, 0.0], t)
    xa = 1.0 / (1.0 / a + 2 * kap * t)
    np.testing.assert_allclose(x, [xa, (a - xa) / 2], rtol=2e-7)


def test_reversible_equilibrium():
    # A <-> B: x_B / x_A -> k_f / k_b, total conserved
    net = tiny(2, [(synth.COSMIC_RAY, (0,), (1,), 300.0, 0, 0), (synth.COSMIC_RAY, (1,), (0,), 100.0, 0, 0)])
    phi = [1e4, 20.0, 0.0, 1.0, 1.3e-17]
    k = chem.rate_coefficients(net, phi)
    t = 40.0 / (k[0] + k[1])
    x = _solve(net, phi, [1e-3, 0.0], t)
    assert x[1] / x[0] == pytest.approx(3.0, rel=1e-7)
    assert x.sum() == pytest.approx(1e-3, rel=1e-12)


def test_linear_network_matches_expm():
    # random first-order (cosmic-ray / photo) network: x(t) = exp(K t) x(0)
    rng = np.random.default_rng(21)
    S = 24
    rx = []
    for _ in range(80):
        a = int(rng.integers(S))
        p = [int(v) for v in rng.choice(S, size=int(rng.integers(1, 3)), replace=False) if v != a]
        if not p:
            continue
        if rng.random() < 0.5:
            rx.append((synth.COSMIC_RAY, (a,), tuple(p), rng.uniform(1, 1e3), 0, 0))
        else:
            rx.append((synth.PHOTO, (a,), tuple(p), 10 ** rng.uniform(-11, -9), 0, rng.uniform(1, 3)))
    net = tiny(S, rx)
    phi = [1e4, 20.0, 1.0, 1.0, 1.3e-17]
    K = chem.jacobian(net, chem.effective_coefficients(net, phi), np.zeros(S))
    x0 = 10.0 ** rng.uniform(-8, -3, S)
    t = 1e5 * YR
    want = scipy.linalg.expm(K * t) @ x0
    x = _solve(net, phi, x0, t)
    big = want > 1e-12 * want.max()
    np.testing.assert_allclose(x[big], want[big], rtol=1e-7)


@pytest.mark.parametrize("S,R,n", [(32, 200, 1), (150, 1500, 2)])
def test_conservation_synthetic(S, R, n):
    net = synth.make_network(S, R)
    x0 = synth.initial_abundances(net)
    E0, Q0 = chem.element_totals(net, x0)
    qscale = np.abs(net.charge) @ x0
    cells = synth.one_cell() if n == 1 else synth.cells(n)
    for phi in cells:
        res = bdf.solve_cell(net, phi, x0, 0.0, 1e6 * YR, 1e-4, 1e-20)
        assert res.status == bdf.OK
        E1, Q1 = chem.element_totals(net, res.x)
        assert np.all(np.abs(E1 - E0) <= 1e-10 * E0)
        assert abs(Q1 - Q0) <= 1e-10 * qscale


def test_self_convergence(net32):
    x0 = synth.initial_abundances(net32)
    phi = synth.one_cell()[0]
    t = 1e5 * YR
    ref = bdf.solve_cell(net32, phi, x0, 0.0, t, 1e-12, 1e-30).x
    big = ref > 1e-12
    errs = []
    for rtol in [1e-4, 1e-6, 1e-8, 1e-10]:
        x = bdf.solve_cell(net32, phi, x0, 0.0, t, rtol, 1e-20 * rtol / 1e-4).x
        errs.append(np.max(np.abs(x[big] / ref[big] - 1)))
    # error falls with rtol: at least 10x per 100x tightening, and stays within 1000 rtol
    for e1, e2 in zip(errs, errs[1:]):
        assert e2 < e1 / 10
    for e, rtol in zip(errs, [1e-4, 1e-6, 1e-8, 1e-10]):
        assert e < 1e3 * rtol


def test_against_library_radau(net32):
    # an independent method (Radau IIA, order 5) from scipy at tight tolerance
    x0 = synth.initial_abundances(net32)
    phi = synth.one_cell()[0]
    kap = chem.effective_coefficients(net32, phi)
    nu = chem.stoichiometry(net32)
    t = 1e5 * YR
    lib = scipy.integrate.solve_ivp(lambda t, y: chem.rhs(net32, kap, y, nu), (0, t), x0, method="Radau",
                                    jac=lambda t, y: chem.jacobian(net32, kap, y, nu),
                                    rtol=1e-11, atol=1e-30)
    assert lib.success
    x = bdf.solve_cell(net32, phi, x0, 0.0, t, 1e-11, 1e-30).x
    big = lib.y[:, -1] > 1e-12
    np.testing.assert_allclose(x[big], lib.y[big, -1], rtol=1e-6)


def test_planted_mistake_is_caught(monkeypatch):
    # a wrong BDF coefficient (gamma_2) must break the closed-form pin
    net = tiny(3, [(synth.TWO_BODY, (0, 1), (2,), 1e-10, 0.5, 20.0)])
    phi = [1e3, 50.0, 0.0, 1.0, 0.0]
    kap = chem.effective_coefficients(net, phi)[0]
    a, b = 3e-4, 1e-4
    t = 5.0 / ((a - b) * kap)
    xa = (a - b) * a / (a - b * np.exp(-(a - b) * kap * t))
    bad = bdf.GAMMA.copy()
    bad[2] = 1.4
    monkeypatch.setattr(bdf, "GAMMA", bad)
    x = bdf.solve_cell(net, phi, np.array([a, b, 0.0]), 0.0, t, 1e-10, 1e-30).x
    assert abs(x[0] / xa - 1) > 1e-6
