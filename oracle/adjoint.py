"""Discrete adjoint of the oracle's BDF map, and an exact-corrector replay (TEST INFRASTRUCTURE ONLY).

The paper's aim is a differentiable model, giving sensitivities of model
outputs to physical and chemical inputs (Sec. 3; abstract); here the
derivatives are those of the discrete BDF map of ``oracle/bdf.py`` with its
step/order program frozen and each corrector equation solved exactly:

    init     D[0] = y0, D[1] = h0 f(y0; p)
    rescale  D[1..q] <- T(rho) D[1..q]
    step     y_p = sum_{j<=q} D[j], psi = sum_{j=1..q} (gamma_j/gamma_q) D[j],
             d solves d - c f(y_p + d; p) + psi = 0 (c = h/gamma_q),
             D'[i] = sum_{k=i..q} D[k] + d (i <= q), D'[q+1] = d, D'[q+2] = d - D[q+1]

Reverse sweep for a cotangent Lam' on the difference array:
    lam_d = sum_{i=0..q+2} Lam'[i]
    mu    = (I - c J(y))^{-T} lam_d,  y = y_p + d the step's result
    Lam[k] = sum_{i<=k} Lam'[i] + (mu - lam_d) - [k>=1] (gamma_k/gamma_q) mu   (k <= q)
    Lam[q+1] = -Lam'[q+2], Lam[q+2] = 0, higher rows unchanged
    dL/dp += c (nu^T mu)_j r_j(y) dlnk_j/dp   (per reaction j)
rescale reverses with T^T; init adds h0 (nu^T Lam[1])_j r_j(y0) dlnk_j/dp.
Parameters: ln alpha_j (dlnk_j = 1), ln n_H (two-body reactions, dlnk = 1) and
T (two-body, dlnk/dT = beta_j/T + gamma_j/T^2; cosmic-ray-induced photo,
dlnk/dT = beta_j/T).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from . import bdf, chem


def _log_k_derivatives(net, phi):
    """(d ln k_j / d ln n_H, d ln k_j / dT): two-body coefficients carry n_H
    (x = n / n_H) and (T/300)^beta exp(-gamma/T); the cosmic-ray-induced photo
    form carries (T/300)^beta."""
    T = float(phi[1])
    tb = (net.rtype == chem.TWO_BODY).astype(float)
    crp = (net.rtype == chem.CR_PHOTO).astype(float)
    return tb, tb * (net.beta / T + net.gamma / T ** 2) + crp * net.beta / T


def _environment(phi, track, t):
    """The cell's environment at time t: phi, or the track's phi(t)."""
    return phi if track is None else bdf.track_params(track, t)


def adjoint(net, phi, x0, program, cot_x, track=None, t0=0.0):
    """Gradients of <cot_x, x(t_end)> w.r.t. (ln alpha [R], ln n_H, T) for one cell.

    With a track (phi is then unused), every step's coefficients are those of
    phi(t_new) and the initial difference's those of phi(t0), as in the
    forward solve; ln n_H and T are then a common factor on the track's n_H
    and a common shift of its T."""
    nu = chem.stoichiometry(net)

    def coefficients(t):
        p = _environment(phi, track, t)
        return (chem.effective_coefficients(net, p),) + _log_k_derivatives(net, p)

    kappa, dlnH, dT = coefficients(t0)
    S = len(x0)
    Lam = np.zeros((bdf.MAX_ORDER + 3, S))
    Lam[0] = cot_x
    g_la = np.zeros(net.n_reactions)
    g_nH = 0.0
    g_T = 0.0

    def accumulate(scale, w, y):
        nonlocal g_la, g_nH, g_T
        contrib = scale * w * chem.reaction_rates(net, kappa, y)
        g_la = g_la + contrib
        g_nH += float(contrib @ dlnH)
        g_T += float(contrib @ dT)

    for op in reversed(program):
        if op[0] == "step":
            _, q, h, t_new, y = op
            if track is not None:
                kappa, dlnH, dT = coefficients(t_new)
            c = h / bdf.GAMMA[q]
            lam_d = Lam[:q + 3].sum(axis=0)
            new = Lam.copy()
            for k in range(q + 1):
                new[k] = Lam[:k + 1].sum(axis=0)
            new[q + 1] = -Lam[q + 2]
            new[q + 2] = 0.0
            M = np.eye(S) - c * chem.jacobian(net, kappa, y, nu)
            mu = scipy.linalg.solve(M.T, lam_d)
            for k in range(q + 1):
                new[k] += mu - lam_d
            for k in range(1, q + 1):
                new[k] -= bdf.GAMMA[k] / bdf.GAMMA[q] * mu
            accumulate(c, nu.T @ mu, y)
            Lam = new
        elif op[0] == "rescale":
            _, q, rho = op
            Lam[1:q + 1] = bdf.rescale_matrix(q, rho).T @ Lam[1:q + 1]
        elif op[0] == "init":
            if track is not None:
                kappa, dlnH, dT = coefficients(t0)
            accumulate(op[1], nu.T @ Lam[1], np.asarray(x0, float))
    return g_la, g_nH, g_T


def environment_gradients(net, g_lnk):
    """(dL/d ln zeta, dL/d ln G0, dL/dA_V) of one cell from its per-reaction
    gradients dL/d ln k_j, which equal dL/d ln alpha_j because k_j is
    proportional to alpha_j. Cosmic-ray coefficients are alpha_j zeta (Sec. 2),
    and so are those of secondary photons induced by cosmic rays (App. B.1,
    times (T/300)^beta E / (1 - omega)); photo coefficients are
    alpha_j G0 exp(-gamma_j A_V) (App. B.1): so d ln k_j / d ln zeta = 1 (both
    cosmic-ray forms), d ln k_j / d ln G0 = 1 and d ln k_j / dA_V = -gamma_j
    (photo), and zero otherwise."""
    g = np.asarray(g_lnk, dtype=float)
    cr = (net.rtype == chem.COSMIC_RAY) | (net.rtype == chem.CR_PHOTO)
    ph = net.rtype == chem.PHOTO
    return float(g[cr].sum()), float(g[ph].sum()), float(-(net.gamma[ph] * g[ph]).sum())


def replay(net, phi, x0, program, newton_tol=1e-13, max_iter=60, track=None, t0=0.0):
    """Re-run a recorded program with each corrector solved to convergence.

    Full Newton (fresh Jacobian every iteration) until the max-norm of the
    update relative to |y| + 1e-30 is below newton_tol. Returns x(t_end) and
    the program with the replayed step results (for ``adjoint``). With a
    track, each step uses the coefficients of phi(t_new) (its recorded time)
    and the initial difference those of phi(t0).
    """
    kappa = chem.effective_coefficients(net, _environment(phi, track, t0))
    nu = chem.stoichiometry(net)
    y0 = np.asarray(x0, float)
    S = len(y0)
    D = np.zeros((bdf.MAX_ORDER + 3, S))
    out = []
    for op in program:
        if op[0] == "init":
            D[0] = y0
            D[1] = op[1] * chem.rhs(net, kappa, y0, nu)
            out.append(op)
        elif op[0] == "rescale":
            _, q, rho = op
            D[1:q + 1] = bdf.rescale_matrix(q, rho) @ D[1:q + 1]
            out.append(op)
        else:
            _, q, h, t_new, _y = op
            if track is not None:
                kappa = chem.effective_coefficients(net, bdf.track_params(track, t_new))
            c = h / bdf.GAMMA[q]
            y_p = D[:q + 1].sum(axis=0)
            psi = (bdf.GAMMA[1:q + 1] @ D[1:q + 1]) / bdf.GAMMA[q]
            d = np.zeros(S)
            for _ in range(max_iter):
                y = y_p + d
                G = d - c * chem.rhs(net, kappa, y, nu) + psi
                M = np.eye(S) - c * chem.jacobian(net, kappa, y, nu)
                delta = np.linalg.solve(M, -G)
                d = d + delta
                if np.max(np.abs(delta) / (np.abs(y_p + d) + 1e-30)) < newton_tol:
                    break
            y = y_p + d
            D[q + 2] = d - D[q + 1]
            D[q + 1] = d
            for i in range(q, -1, -1):
                D[i] += D[i + 1]
            out.append(("step", q, h, t_new, y.copy()))
    return D[0].copy(), out


def with_alpha(net, alpha):
    """A copy of the network with other alpha values (for finite differences)."""
    import copy
    n2 = copy.copy(net)
    n2.alpha = np.asarray(alpha, float)
    return n2


def log10_loss(x, targets, y_target):
    """L = sum_i (log10 x_i - y_i)^2 over the target species, and dL/dx."""
    lx = np.log10(x[targets])
    L = float(np.sum((lx - y_target) ** 2))
    g = np.zeros_like(x)
    g[targets] = 2.0 * (lx - y_target) / (x[targets] * np.log(10.0))
    return L, g
