"""Pins for the oracle's rates, right-hand side and Jacobian (no GPU).

Rates are checked against the Sec. 2 / App. B.1 formulas evaluated with
40-digit decimal arithmetic (an independent evaluation, not a re-call of
numpy); the right-hand side against conservation (element and charge balance
makes e^T f = 0 exactly) and hand-derived one-reaction cases; the Jacobian
against central finite differences, which are exact for the quadratic
mass-action terms up to rounding.
"""
import decimal

import numpy as np
import pytest

from oracle import chem
from paper_2511_10558_gb300 import synth
from tests.nets import tiny

decimal.getcontext().prec = 40
D = decimal.Decimal


def _rate_decimal(rt, a, b, g, phi, omega=0.0):
    n_H, T, A_V, G0, zeta = (D(repr(float(v))) for v in phi)
    a, b, g = D(repr(float(a))), D(repr(float(b))), D(repr(float(g)))
    if rt == synth.TWO_BODY:
        return a * ((b * (T / D(300)).ln()).exp()) * (-(g / T)).exp()
    if rt == synth.COSMIC_RAY:
        return a * zeta
    if rt == synth.CR_PHOTO:
        # App. B.1: alpha (T/300)^beta E / (1 - omega) zeta, E in the gamma field
        return a * ((b * (T / D(300)).ln()).exp()) * g / (D(1) - D(repr(float(omega)))) * zeta
    return a * G0 * (-(g * A_V)).exp()


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_rates_against_decimal(net150, seed):
    phi = synth.cells(1, seed=seed)[0]
    k = chem.rate_coefficients(net150, phi)
    for j in range(0, net150.n_reactions, 7):
        ref = _rate_decimal(net150.rtype[j], net150.alpha[j], net150.beta[j], net150.gamma[j], phi)
        if ref == 0:
            assert k[j] == 0
            continue
        assert abs(D(repr(float(k[j]))) / ref - 1) < D("1e-14"), j
    kap = chem.effective_coefficients(net150, phi)
    tb = net150.rtype == synth.TWO_BODY
    np.testing.assert_array_equal(kap[tb], k[tb] * phi[0])
    np.testing.assert_array_equal(kap[~tb], k[~tb])


@pytest.mark.parametrize("seed", [0, 1])
def test_cr_photo_rates_against_decimal(seed):
    net = synth.make_network(150, 1500, cr_photo_frac=0.4)
    assert (net.rtype == synth.CR_PHOTO).sum() > 50 and net.albedo == 0.5
    phi = synth.cells(1, seed=seed)[0]
    k = chem.rate_coefficients(net, phi)
    for j in np.flatnonzero(net.rtype == synth.CR_PHOTO):
        ref = _rate_decimal(synth.CR_PHOTO, net.alpha[j], net.beta[j], net.gamma[j], phi, net.albedo)
        assert abs(D(repr(float(k[j]))) / ref - 1) < D("1e-14"), j
    # one reactant: no n_H factor in the effective coefficient
    kap = chem.effective_coefficients(net, phi)
    crp = net.rtype == synth.CR_PHOTO
    np.testing.assert_array_equal(kap[crp], k[crp])


def test_cr_photo_special_values():
    # T = 300 K: (T/300)^beta = 1, so k = alpha E / (1 - omega) zeta; omega = 0 gives alpha E zeta
    net = tiny(2, [(synth.CR_PHOTO, (0,), (1,), 1.5, 0.8, 2000.0)])
    net.albedo = 0.6
    k = chem.rate_coefficients(net, [1e4, 300.0, 7.0, 3.0, 2e-17])[0]
    assert k == pytest.approx(1.5 * 2000.0 / 0.4 * 2e-17, rel=1e-15)
    net.albedo = 0.0
    assert chem.rate_coefficients(net, [1e4, 300.0, 0.0, 0.0, 2e-17])[0] == pytest.approx(1.5 * 2000 * 2e-17,
                                                                                         rel=1e-15)
    # no dependence on A_V or G0; T enters as (T/300)^beta
    k2 = chem.rate_coefficients(net, [1e2, 75.0, 0.0, 9.0, 2e-17])[0]
    assert k2 == pytest.approx(1.5 * 0.25 ** 0.8 * 2000 * 2e-17, rel=1e-14)


def test_rate_special_values():
    # T = 300 K makes (T/300)^beta = 1; gamma = 0 removes the exponential
    net = tiny(3, [(synth.TWO_BODY, (0, 1), (2,), 2e-10, 0.7, 0.0),
                   (synth.TWO_BODY, (0, 1), (2,), 2e-10, -0.3, 150.0),
                   (synth.COSMIC_RAY, (0,), (1,), 300.0, 0, 0),
                   (synth.PHOTO, (0,), (1,), 1e-10, 0, 2.0)])
    k = chem.rate_coefficients(net, [1e4, 300.0, 0.0, 1.0, 1.3e-17])
    assert k[0] == 2e-10
    assert k[1] == pytest.approx(2e-10 * np.exp(-0.5), rel=1e-15)
    assert k[2] == pytest.approx(300.0 * 1.3e-17, rel=1e-15)
    assert k[3] == 1e-10  # A_V = 0, G0 = 1


def test_rhs_one_reaction_cases():
    # A + B -> C + D and A + A -> C: signs, multiplicities and n_H scaling
    net = tiny(4, [(synth.TWO_BODY, (0, 1), (2, 3), 1e-9, 0.0, 0.0)])
    x = np.array([0.3, 0.2, 0.1, 0.05])
    f = chem.rhs(net, chem.effective_coefficients(net, [1e3, 300, 0, 1, 0]), x)
    r = 1e-9 * 1e3 * 0.3 * 0.2
    np.testing.assert_allclose(f, [-r, -r, r, r], rtol=1e-15)
    net = tiny(2, [(synth.TWO_BODY, (0, 0), (1,), 1e-9, 0.0, 0.0)])
    f = chem.rhs(net, chem.effective_coefficients(net, [1e3, 300, 0, 1, 0]), np.array([0.3, 0.0]))
    r = 1e-9 * 1e3 * 0.3 * 0.3
    np.testing.assert_allclose(f, [-2 * r, r], rtol=1e-15)
    J = chem.jacobian(net, chem.effective_coefficients(net, [1e3, 300, 0, 1, 0]), np.array([0.3, 0.0]))
    np.testing.assert_allclose(J, [[-4e-6 * 0.3, 0], [2e-6 * 0.3, 0]], rtol=1e-15)


@pytest.mark.parametrize("which", ["net32", "net150"])
def test_rhs_conserves_elements_and_charge(which, request):
    net = request.getfixturevalue(which)
    rng = np.random.default_rng(3)
    nu = chem.stoichiometry(net)
    E = np.vstack([net.composition.T, net.charge]).astype(float)
    assert np.all(E @ nu == 0)
    for phi in synth.cells(4):
        kap = chem.effective_coefficients(net, phi)
        x = 10.0 ** rng.uniform(-12, -1, net.n_species)
        f = chem.rhs(net, kap, x, nu)
        terms = np.abs(nu) @ np.abs(chem.reaction_rates(net, kap, x))
        assert np.all(np.abs(E @ f) <= 1e-13 * (np.abs(E) @ terms))
        J = chem.jacobian(net, kap, x, nu)
        assert np.all(np.abs(E @ J) <= 1e-13 * (np.abs(E) @ np.abs(J)) + 1e-300)


@pytest.mark.parametrize("which", ["net32", "net150"])
def test_jacobian_against_central_differences(which, request):
    net = request.getfixturevalue(which)
    rng = np.random.default_rng(5)
    nu = chem.stoichiometry(net)
    phi = synth.cells(1)[0]
    kap = chem.effective_coefficients(net, phi)
    x = 10.0 ** rng.uniform(-8, -1, net.n_species)
    J = chem.jacobian(net, kap, x, nu)
    Jfd = np.empty_like(J)
    for l in range(net.n_species):
        h = 1e-6 * x[l]
        xp = x.copy()
        xm = x.copy()
        xp[l] += h
        xm[l] -= h
        Jfd[:, l] = (chem.rhs(net, kap, xp, nu) - chem.rhs(net, kap, xm, nu)) / (2 * h)
    # central differences are exact for the quadratic terms; what is left is the
    # rounding of f (sum of |nu_ij r_j| terms) divided by the step
    absJ = np.abs(nu) @ np.abs(chem.rate_jacobian(net, kap, x))
    terms = np.abs(nu) @ np.abs(chem.reaction_rates(net, kap, x))
    bound = 1e-9 * absJ + 8 * np.finfo(float).eps * terms[:, None] / (1e-6 * x[None, :])
    assert np.all(np.abs(Jfd - J) <= bound)
    # and the check has teeth: a Jacobian with one dropped term fails it
    bad = J.copy()
    i, l = np.unravel_index(np.argmax(np.abs(J) - bound), J.shape)
    bad[i, l] = 0.0
    assert not np.all(np.abs(Jfd - bad) <= bound)


def test_invariant_totals(net32):
    x = synth.initial_abundances(net32)
    E, Q = chem.element_totals(net32, x)
    np.testing.assert_allclose(E, [1.0 + 1e-20 * 0, 0.1, 1e-4, 7.5e-5, 3e-4], rtol=1e-10)
    assert abs(Q) < 1e-18
