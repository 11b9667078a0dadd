"""Pins for the oracle's discrete adjoint (no GPU).

* A -> B: d x_B / d ln k = a k t exp(-k t) (closed form), within the
  integrator's accuracy at tight tolerance; zero n_H and T gradients.
* A + B -> C: derivatives of the closed form x_A(t) w.r.t. ln kappa, taken by
  complex-step differentiation of that closed form; the n_H gradient equals the
  ln alpha gradient and the T gradient is (beta/T + gamma/T^2) times it.
* A -> B by a photo reaction: d x_B / d ln G0 and d x_B / dA_V from the
  closed form (environment gradients).
* A synthetic 32-species cell: the adjoint of the replayed (frozen
  step/order, exact corrector) map against central finite differences of the
  same map, step 1e-6 in ln alpha, ln n_H, ln zeta, ln G0, A_V and 1e-6 T in T.
"""
import numpy as np
import pytest

from oracle import adjoint as adj
from oracle import bdf, chem
from paper_2511_10558_gb300 import synth
from tests.nets import tiny


def test_first_order_decay_sensitivity():
    net = tiny(2, [(synth.COSMIC_RAY, (0,), (1,), 50.0, 0, 0)])
    phi = [1e4, 20.0, 0.5, 1.0, 1.3e-17]
    k = chem.rate_coefficients(net, phi)[0]
    t = 2.0 / k
    a = 1e-3
    res = bdf.solve_cell(net, phi, np.array([a, 1e-20]), 0.0, t, 1e-10, 1e-30, record=True)
    g_la, g_nH, g_T = adj.adjoint(net, phi, [a, 1e-20], res.program, np.array([0.0, 1.0]))
    assert g_la[0] == pytest.approx(a * k * t * np.exp(-k * t), rel=1e-6)
    assert g_nH == 0.0 and g_T == 0.0
    # k = alpha zeta: the zeta sensitivity is the same closed form; no photo terms
    g_z, g_g0, g_av = adj.environment_gradients(net, g_la)
    assert g_z == pytest.approx(a * k * t * np.exp(-k * t), rel=1e-6)
    assert g_g0 == 0.0 and g_av == 0.0


def test_photo_decay_environment_sensitivity():
    # A -> B by a photo reaction, k = alpha G0 exp(-gamma A_V): x_B = a (1 - exp(-k t)),
    # d x_B / d ln G0 = a k t exp(-k t), d x_B / dA_V = -gamma a k t exp(-k t)
    gam = 2.0
    net = tiny(2, [(synth.PHOTO, (0,), (1,), 1e-9, 0, gam)])
    phi = [1e4, 20.0, 1.5, 3.0, 1.3e-17]
    k = chem.rate_coefficients(net, phi)[0]
    assert k == pytest.approx(1e-9 * 3.0 * np.exp(-gam * 1.5), rel=1e-15)
    t = 1.5 / k
    a = 1e-3
    res = bdf.solve_cell(net, phi, np.array([a, 1e-20]), 0.0, t, 1e-10, 1e-30, record=True)
    g_la, _, _ = adj.adjoint(net, phi, [a, 1e-20], res.program, np.array([0.0, 1.0]))
    g_z, g_g0, g_av = adj.environment_gradients(net, g_la)
    exact = a * k * t * np.exp(-k * t)
    assert g_z == 0.0
    assert g_g0 == pytest.approx(exact, rel=1e-6)
    assert g_av == pytest.approx(-gam * exact, rel=1e-6)


def test_cr_photo_decay_sensitivity():
    # A -> B by secondary photons induced by cosmic rays (App. B.1),
    # k = alpha (T/300)^beta E/(1 - omega) zeta: x_B = a (1 - exp(-k t)), so
    # d x_B / d ln k = a k t exp(-k t) = d x_B / d ln zeta, d x_B / dT = (beta/T) that,
    # and no n_H, G0 or A_V dependence
    beta, T = 0.7, 40.0
    net = tiny(2, [(synth.CR_PHOTO, (0,), (1,), 1.3, beta, 3000.0)])
    net.albedo = 0.5
    phi = [1e4, T, 2.0, 1.0, 1.3e-17]
    k = chem.rate_coefficients(net, phi)[0]
    assert k == pytest.approx(1.3 * (T / 300) ** beta * 3000 / 0.5 * 1.3e-17, rel=1e-14)
    t = 2.0 / k
    a = 1e-3
    res = bdf.solve_cell(net, phi, np.array([a, 1e-20]), 0.0, t, 1e-10, 1e-30, record=True)
    g_la, g_nH, g_T = adj.adjoint(net, phi, [a, 1e-20], res.program, np.array([0.0, 1.0]))
    exact = a * k * t * np.exp(-k * t)
    assert g_la[0] == pytest.approx(exact, rel=1e-6)
    assert g_nH == 0.0
    assert g_T == pytest.approx(beta / T * exact, rel=1e-6)
    g_z, g_g0, g_av = adj.environment_gradients(net, g_la)
    assert g_z == pytest.approx(exact, rel=1e-6)
    assert g_g0 == 0.0 and g_av == 0.0


def test_second_order_sensitivity():
    net = tiny(3, [(synth.TWO_BODY, (0, 1), (2,), 1e-10, 0.5, 20.0)])
    phi = [1e3, 50.0, 0.0, 1.0, 0.0]
    kap = chem.effective_coefficients(net, phi)[0]
    a, b = 3e-4, 1e-4
    dlt = a - b
    t = 3.0 / (dlt * kap)

    def xa(lnk):  # closed form, complex-step differentiable
        kk = np.exp(lnk)
        return dlt * a / (a - b * np.exp(-dlt * kk * t))

    h = 1e-20
    dxa = (xa(np.log(kap) + 1j * h)).imag / h
    res = bdf.solve_cell(net, phi, np.array([a, b, 0.0]), 0.0, t, 1e-10, 1e-30, record=True)
    g_la, g_nH, g_T = adj.adjoint(net, phi, [a, b, 0.0], res.program, np.array([1.0, 0.0, 0.0]))
    assert g_la[0] == pytest.approx(dxa, rel=1e-5)
    assert g_nH == pytest.approx(g_la[0], rel=1e-12)
    assert g_T == pytest.approx(g_la[0] * (0.5 / 50.0 + 20.0 / 50.0 ** 2), rel=1e-12)


def _setup_cell(net, seed=11):
    phi = synth.one_cell()[0]
    x0 = synth.initial_abundances(net)
    t_end = 1e5 * synth.YEAR
    res = bdf.solve_cell(net, phi, x0, 0.0, t_end, 1e-4, 1e-20, record=True)
    rng = np.random.default_rng(seed)
    cand = np.flatnonzero(res.x > 1e-12)
    targets = np.sort(rng.choice(cand, size=min(10, len(cand)), replace=False))
    y_t = np.log10(res.x[targets]) + rng.uniform(-0.5, 0.5, len(targets))
    return phi, x0, res, targets, y_t


def test_adjoint_matches_frozen_finite_differences(net32):
    phi, x0, res, targets, y_t = _setup_cell(net32)
    x_rep, prog = adj.replay(net32, phi, x0, res.program)
    L0, cot = adj.log10_loss(x_rep, targets, y_t)
    g_la, g_nH, g_T = adj.adjoint(net32, phi, x0, prog, cot)
    eps = 1e-6

    def loss(net=net32, p=phi):
        x, _ = adj.replay(net, p, x0, res.program)
        return adj.log10_loss(x, targets, y_t)[0]

    order = np.argsort(-np.abs(g_la))
    for j in list(order[:4]) + [int(order[len(order) // 3])]:
        a_p = net32.alpha.copy()
        a_m = net32.alpha.copy()
        a_p[j] *= np.exp(eps)
        a_m[j] *= np.exp(-eps)
        fd = (loss(adj.with_alpha(net32, a_p)) - loss(adj.with_alpha(net32, a_m))) / (2 * eps)
        assert fd == pytest.approx(g_la[j], rel=1e-3, abs=1e-8 * max(1.0, abs(g_la).max())), j
    p_p, p_m = phi.copy(), phi.copy()
    p_p[0] *= np.exp(eps)
    p_m[0] *= np.exp(-eps)
    assert (loss(p=p_p) - loss(p=p_m)) / (2 * eps) == pytest.approx(g_nH, rel=1e-3)
    p_p, p_m = phi.copy(), phi.copy()
    p_p[1] += eps * phi[1]
    p_m[1] -= eps * phi[1]
    assert (loss(p=p_p) - loss(p=p_m)) / (2 * eps * phi[1]) == pytest.approx(g_T, rel=1e-3)
    # environment: ln zeta (phi[4]), ln G0 (phi[3]), A_V (phi[2])
    g_z, g_g0, g_av = adj.environment_gradients(net32, g_la)
    for col, g_env in ((4, g_z), (3, g_g0)):
        p_p, p_m = phi.copy(), phi.copy()
        p_p[col] *= np.exp(eps)
        p_m[col] *= np.exp(-eps)
        assert (loss(p=p_p) - loss(p=p_m)) / (2 * eps) == pytest.approx(g_env, rel=1e-3), col
    p_p, p_m = phi.copy(), phi.copy()
    p_p[2] += eps
    p_m[2] -= eps
    assert (loss(p=p_p) - loss(p=p_m)) / (2 * eps) == pytest.approx(g_av, rel=1e-3)


def test_adjoint_of_adaptive_run_close_to_replayed(net32):
    # the adaptive run's Newton stops at its tolerance; its adjoint agrees with
    # the exact-corrector one to far better than the 1e-3 gradient gate
    phi, x0, res, targets, y_t = _setup_cell(net32)
    x_rep, prog = adj.replay(net32, phi, x0, res.program)
    _, cot = adj.log10_loss(res.x, targets, y_t)
    g1 = adj.adjoint(net32, phi, x0, res.program, cot)
    _, cot2 = adj.log10_loss(x_rep, targets, y_t)
    g2 = adj.adjoint(net32, phi, x0, prog, cot2)
    big = np.abs(g2[0]) > 1e-6 * np.abs(g2[0]).max()
    np.testing.assert_allclose(g1[0][big], g2[0][big], rtol=1e-3)
    assert g1[1] == pytest.approx(g2[1], rel=1e-3)
    assert g1[2] == pytest.approx(g2[2], rel=1e-3)
