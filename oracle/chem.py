"""Rates, right-hand side and Jacobian of the mass-action network, in FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

State: x_i = n_i / n_H (abundance per hydrogen nucleus). The paper writes the
ODE for number densities n_i in cm^-3 (Sec. 2). With n_H constant (one
zero-dimensional cell), dividing that ODE by n_H gives the same dynamics in x
when every two-body coefficient is multiplied by n_H:

    dx_i/dt = sum_j nu_ij r_j,   r_j = kappa_j x_a x_b  (two-body, kappa_j = k_j n_H)
                                 r_j = k_j x_a          (one reactant)

with nu = products - reactants (the incidence / stoichiometry matrix, Sec. 4).
A reaction A + A consumes A twice and its rate is kappa x_A^2 (no 1/2 factor).
"""
from __future__ import annotations

import numpy as np

TWO_BODY, COSMIC_RAY, PHOTO, CR_PHOTO = 0, 1, 2, 3


def rate_coefficients(net, phi):
    """k_j for one cell phi = (n_H, T, A_V, G0, zeta).

    Two-body, Sec. 2 (Kooij-Arrhenius):  k = alpha (T/300)^beta exp(-gamma/T)
    Cosmic-ray ionisation, Sec. 2:       k = alpha zeta
    Photo-reaction, App. B.1:            k = alpha F_UV exp(-gamma A_V)
    (the extinction factor written "k" in App. B.1 is the reaction's gamma; F_UV is G0).
    Secondary photons induced by cosmic rays, App. B.1:
                                         k = alpha (T/300)^beta E / (1 - omega) zeta
    (E, the cosmic-ray efficiency of the reaction, is its gamma; omega is the
    dust grain albedo of the network, ``net.albedo``).
    """
    n_H, T, A_V, G0, zeta = (float(v) for v in phi)
    omega = float(getattr(net, "albedo", 0.0))
    k = np.zeros(net.n_reactions)
    for j in range(net.n_reactions):
        a, b, g = net.alpha[j], net.beta[j], net.gamma[j]
        if net.rtype[j] == TWO_BODY:
            k[j] = a * (T / 300.0) ** b * np.exp(-g / T)
        elif net.rtype[j] == COSMIC_RAY:
            k[j] = a * zeta
        elif net.rtype[j] == PHOTO:
            k[j] = a * G0 * np.exp(-g * A_V)
        elif net.rtype[j] == CR_PHOTO:
            k[j] = a * (T / 300.0) ** b * g / (1.0 - omega) * zeta
        else:
            raise ValueError(f"unknown reaction type {net.rtype[j]}")
    return k


def effective_coefficients(net, phi):
    """kappa_j: k_j, times n_H for two-body reactions (x = n / n_H)."""
    k = rate_coefficients(net, phi)
    return np.where(net.rtype == TWO_BODY, k * float(phi[0]), k)


def stoichiometry(net):
    """nu [S, R] = (product multiplicity) - (reactant multiplicity)."""
    nu = np.zeros((net.n_species, net.n_reactions))
    for j in range(net.n_reactions):
        for a in net.reac[j]:
            if a >= 0:
                nu[a, j] -= 1.0
        for p in net.prod[j]:
            if p >= 0:
                nu[p, j] += 1.0
    return nu


def reaction_rates(net, kappa, x):
    """r_j = kappa_j * product of the reactants' abundances."""
    r = np.array(kappa, dtype=float)
    for j in range(net.n_reactions):
        for a in net.reac[j]:
            if a >= 0:
                r[j] *= x[a]
    return r


def rhs(net, kappa, x, nu=None):
    """dx/dt = nu r(x)  (Sec. 2 ODE, divided by n_H)."""
    if nu is None:
        nu = stoichiometry(net)
    return nu @ reaction_rates(net, kappa, x)


def rate_jacobian(net, kappa, x):
    """dr_j/dx_l [R, S] from the product rule on r_j = kappa_j x_a (x_b)."""
    dr = np.zeros((net.n_reactions, net.n_species))
    for j in range(net.n_reactions):
        a, b = net.reac[j]
        if b < 0:
            dr[j, a] += kappa[j]
        else:
            dr[j, a] += kappa[j] * x[b]
            dr[j, b] += kappa[j] * x[a]
    return dr


def jacobian(net, kappa, x, nu=None):
    """Analytic J = d(dx/dt)/dx = nu dr/dx  [S, S]."""
    if nu is None:
        nu = stoichiometry(net)
    return nu @ rate_jacobian(net, kappa, x)


def element_totals(net, x):
    """E_e = sum_i comp_ie x_i for e in (H, He, C, N, O); Q = sum_i q_i x_i."""
    return net.composition.T.astype(float) @ x, float(net.charge.astype(float) @ x)
