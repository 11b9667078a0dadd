"""Pins for the oracle's adjoint through a time-dependent environment (no GPU).

* A -> B by cosmic rays with zeta(t) linear in time: with K = integral of
  k(t) = alpha zeta(t) over [0, t1], x_B(t1) = a (1 - exp(-K)), so
  d x_B / d ln alpha = d x_B / d ln(common zeta factor) = a K exp(-K).
* A -> B by secondary photons induced by cosmic rays (App. B.1) with T(t)
  linear in time: k(t) = alpha (T(t)/300)^beta E/(1 - omega) zeta, so the
  derivative with respect to a common shift of the track's T is
  a exp(-K) * integral of k(t) beta / T(t) dt, the integral by scipy quadrature.
* A synthetic 32-species cell on a collapse track: the adjoint of the replayed
  (frozen program, exact corrector) map against central finite differences of
  that map in ln alpha, in ln of a common n_H factor and in a common T shift.
"""
import numpy as np
import pytest
import scipy.integrate

from oracle import adjoint as adj
from oracle import bdf, chem
from paper_2511_10558_gb300 import synth
from tests.nets import tiny

YR = synth.YEAR


def _track(t1, **ends):
    # two knots at 0 and t1; ends maps a field to its (start, end) values
    base = {"n_H": (1e4, 1e4), "T": (20.0, 20.0), "A_V": (2.0, 2.0), "G0": (1.0, 1.0), "zeta": (1.3e-17, 1.3e-17)}
    base.update(ends)
    tr = np.zeros((2, 6))
    tr[:, 0] = [0.0, t1]
    for i, f in enumerate(("n_H", "T", "A_V", "G0", "zeta")):
        tr[:, 1 + i] = base[f]
    return tr


def test_linear_zeta_track_sensitivity():
    alpha = 80.0
    net = tiny(2, [(synth.COSMIC_RAY, (0,), (1,), alpha, 0, 0)])
    z0, z1 = 1.3e-17, 6.0e-17
    t1 = 1.5 / (alpha * 0.5 * (z0 + z1)) * 1.0
    tr = _track(t1, zeta=(z0, z1))
    a = 1e-3
    res = bdf.solve_cell_track(net, tr, np.array([a, 1e-20]), 0.0, t1, 1e-10, 1e-30, record=True)
    g_la, g_nH, g_T = adj.adjoint(net, None, [a, 1e-20], res.program, np.array([0.0, 1.0]), track=tr)
    K = alpha * 0.5 * (z0 + z1) * t1
    exact = a * K * np.exp(-K)
    assert g_la[0] == pytest.approx(exact, rel=1e-6)
    assert g_nH == 0.0 and g_T == 0.0
    assert adj.environment_gradients(net, g_la)[0] == pytest.approx(exact, rel=1e-6)
    # the constant-environment adjoint of the same program is wrong here
    g_const = adj.adjoint(net, tr[0, 1:], [a, 1e-20], res.program, np.array([0.0, 1.0]))[0][0]
    assert abs(g_const / exact - 1) > 1e-2


def test_cr_photo_temperature_track_sensitivity():
    alpha, beta, E = 1.1, 0.8, 2500.0
    net = tiny(2, [(synth.CR_PHOTO, (0,), (1,), alpha, beta, E)])
    net.albedo = 0.5
    T0, T1 = 20.0, 140.0
    probe = chem.rate_coefficients(net, [1e4, 60.0, 0.0, 1.0, 1.3e-17])[0]
    t1 = 1.2 / probe
    tr = _track(t1, T=(T0, T1))

    def k(t):
        return chem.rate_coefficients(net, bdf.track_params(tr, t))[0]

    def T(t):
        return T0 + (T1 - T0) * t / t1

    K = scipy.integrate.quad(k, 0.0, t1, epsabs=0, epsrel=1e-13)[0]
    dK_dT = scipy.integrate.quad(lambda t: k(t) * beta / T(t), 0.0, t1, epsabs=0, epsrel=1e-13)[0]
    a = 1e-3
    res = bdf.solve_cell_track(net, tr, np.array([a, 1e-20]), 0.0, t1, 1e-10, 1e-30, record=True)
    g_la, g_nH, g_T = adj.adjoint(net, None, [a, 1e-20], res.program, np.array([0.0, 1.0]), track=tr)
    assert res.x[1] == pytest.approx(a * (1 - np.exp(-K)), rel=1e-7)
    assert g_la[0] == pytest.approx(a * K * np.exp(-K), rel=1e-6)
    assert g_T == pytest.approx(a * np.exp(-K) * dK_dT, rel=1e-6)
    assert g_nH == 0.0


def test_track_adjoint_matches_frozen_finite_differences(net32):
    t_end = 1e5 * YR
    phi = synth.cells(1, seed=9)
    tr = synth.tracks(phi, t_end)[0]
    x0 = synth.initial_abundances(net32)
    res = bdf.solve_cell_track(net32, tr, x0, 0.0, t_end, 1e-4, 1e-20, record=True)
    prog = res.program
    rng = np.random.default_rng(4)
    tg = np.sort(rng.choice(np.flatnonzero(res.x > 1e-12), 8, replace=False))
    yt = np.log10(res.x[tg]) + rng.uniform(-0.5, 0.5, len(tg))
    x_rep, prog_rep = adj.replay(net32, None, x0, prog, track=tr)
    _, cot = adj.log10_loss(x_rep, tg, yt)
    g_la, g_nH, g_T = adj.adjoint(net32, None, x0, prog_rep, cot, track=tr)
    eps = 1e-6

    def loss(net=net32, track=tr):
        x, _ = adj.replay(net, None, x0, prog, track=track)
        return adj.log10_loss(x, tg, yt)[0]

    for j in np.argsort(-np.abs(g_la))[:3]:
        ap, am = net32.alpha.copy(), net32.alpha.copy()
        ap[j] *= np.exp(eps)
        am[j] *= np.exp(-eps)
        fd = (loss(adj.with_alpha(net32, ap)) - loss(adj.with_alpha(net32, am))) / (2 * eps)
        assert fd == pytest.approx(g_la[j], rel=1e-4), j
    tp, tm = tr.copy(), tr.copy()
    tp[:, 1] *= np.exp(eps)
    tm[:, 1] *= np.exp(-eps)
    assert (loss(track=tp) - loss(track=tm)) / (2 * eps) == pytest.approx(g_nH, rel=1e-4)
    d = eps * tr[0, 2]
    tp, tm = tr.copy(), tr.copy()
    tp[:, 2] += d
    tm[:, 2] -= d
    assert (loss(track=tp) - loss(track=tm)) / (2 * d) == pytest.approx(g_T, rel=1e-4)
