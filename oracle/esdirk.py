"""ESDIRK integrator of Kvaerno's family for one cell, plain FP64 (TEST INFRASTRUCTURE ONLY).

The paper integrates its networks with Kvaerno's fifth-order stiff method, an
ESDIRK (explicit first stage, singly diagonally implicit Runge-Kutta) from
Kvaerno, "Singly diagonally implicit Runge-Kutta methods with an explicit
first stage", BIT 44 (2004), through Diffrax with custom tolerances (Sec. 4).
The paper prints no coefficients. This module takes the defining structure of
that family and derives the member of order 4 with an embedded order-3
solution (five stages) from it:

  * explicit first stage (c_1 = 0, a_1j = 0) and one diagonal value gamma;
  * stage order 2: sum_j a_ij = c_i and sum_j a_ij c_j = c_i^2 / 2 (i >= 2),
    so c_2 = 2 gamma;
  * the embedded solution is stage 4 and the solution is stage 5, both with
    c = 1 (each is stiffly accurate): row 4 has order 3, row 5 order 4;
  * L-stability of the solution: R(infinity) = 0.

Rows 2-5 then follow from linear conditions once (gamma, c_3) are known; c_3
solves the one order-4 condition that is not a moment condition,
sum_i b_i (A c^2)_i = 1/12, and gamma the L-stability condition. (Kvaerno
gives gamma = 0.5728160625 for this method; the derivation reproduces it.)

One step of size h from (t_n, y_n), f_1 = f(t_n, y_n):
    for i = 2..5:  Y_i = y_n + h sum_{j<i} a_ij f_j + h gamma f(t_n + c_i h, Y_i),
                   f_i = f(t_n + c_i h, Y_i)
    y_{n+1} = Y_5, embedded Y_4, error estimate e = Y_5 - Y_4.
Each implicit stage is solved by simplified Newton with the matrix
I - h gamma J (one LU serves all four stages), started from the previous
stage value, with the stopping rules of ``bdf.newton_corrector``.
Because y_{n+1} = Y_5 is a stage value at t_n + h, f_5 is the next step's f_1.

Controller (the BDF module's conventions where they apply):
    norms        weighted RMS with weights 1/(atol + rtol |y|): |y_n| for the
                 Newton test, |y_{n+1}| for the error test
    error test   err = |e| <= 1
    step size    h_new = h min(10, max(0.2, 0.9 err^(-1/4))) after an accepted
                 step, h max(0.2, 0.9 err^(-1/4)) after a rejected one
                 (1/4 = 1/(embedded order + 1))
    Newton       at most 4 increments per stage; failure with a Jacobian that
                 is not current -> new J at (t_n, y_n) and retry, else h / 2
    Jacobian     at (t0, y0), and again only after a Newton failure with a
                 Jacobian that is not current (it is current from its
                 evaluation until the next accepted step)
    LU           of I - h gamma J whenever h or J changed
    initial h    Hairer, Norsett & Wanner I, Sec. II.4, with p = 3
    last step    shortened to end at t_end; max_steps attempts -> MAX_STEPS;
                 h < 10 ulp(t) -> H_UNDERFLOW; negative values not clipped
"""
from __future__ import annotations

import numpy as np
import scipy.linalg
from scipy.optimize import brentq

from . import bdf, chem

STAGES = 5
ORDER, EMBEDDED_ORDER = 4, 3
OK, MAX_STEPS, H_UNDERFLOW = bdf.OK, bdf.MAX_STEPS, bdf.H_UNDERFLOW


def _rows(gamma, c3):
    """A [5, 5] and c [5] for given (gamma, c_3) from the linear conditions."""
    c = np.array([0.0, 2.0 * gamma, c3, 1.0, 1.0])
    A = np.zeros((STAGES, STAGES))
    A[1, 0] = A[1, 1] = gamma
    # stage 3: a_31 + a_32 + gamma = c_3, a_32 c_2 + gamma c_3 = c_3^2 / 2
    A[2, 2] = gamma
    A[2, 1] = (0.5 * c3 * c3 - gamma * c3) / c[1]
    A[2, 0] = c3 - gamma - A[2, 1]
    # stage 4 (embedded, order 3): sum a_4j c_j^k = 1/(k+1), k = 0, 1, 2 (a_44 = gamma)
    V = np.vander(c[:3], 3, increasing=True).T
    A[3, :3] = np.linalg.solve(V, [1.0 - gamma, 0.5 - gamma, 1.0 / 3.0 - gamma])
    A[3, 3] = gamma
    # stage 5 (solution, order 4): sum b_j c_j^k = 1/(k+1), k = 0..3 (b_5 = gamma)
    V = np.vander(c[:4], 4, increasing=True).T
    A[4, :4] = np.linalg.solve(V, [1.0 - gamma, 0.5 - gamma, 1.0 / 3.0 - gamma, 0.25 - gamma])
    A[4, 4] = gamma
    return A, c


def _tree_bac2(gamma, c3):
    A, c = _rows(gamma, c3)
    return A[4] @ (A @ c ** 2) - 1.0 / 12.0


def _c3(gamma):
    return brentq(lambda x: _tree_bac2(gamma, x), 0.4, 0.8, xtol=1e-16, rtol=1e-15)


def stability_at_infinity(A):
    """R(z) of the stiffly accurate method as z -> -infinity. Stages 2..s
    satisfy (I - z A~) Y~ = 1 + z a y0 (A~ the implicit block, a its first
    column), so Y~ -> -A~^{-1} a y0, and R(infinity) is the last component."""
    return -np.linalg.solve(A[1:, 1:], A[1:, 0])[-1]


def tableau():
    """(A [5, 5], c [5], gamma): the derived ESDIRK 4(3) of Kvaerno's family."""
    gamma = brentq(lambda g: stability_at_infinity(_rows(g, _c3(g))[0]), 0.56, 0.59, xtol=1e-16, rtol=1e-15)
    A, c = _rows(gamma, _c3(gamma))
    return A, c, gamma


A_TAB, C_TAB, GAMMA = tableau()


def integrate(fun, jac, t0, y0, t_end, rtol, atol, max_steps=100000, tableau=None, fixed_h=None):
    """Integrate y' = fun(t, y) from t0 to t_end (see the module docstring).

    tableau: (A, c, gamma) to use instead of the derived one (tests plant
    mistakes through it). fixed_h: take steps of exactly that size with no
    error control (order checks); the error estimate is then still reported.
    Returns a bdf.Result (program = None) whose stats also hold the last
    step's embedded solution under "embedded".
    """
    A, c, gamma = tableau if tableau is not None else (A_TAB, C_TAB, GAMMA)
    S = y0.size
    stats = dict(steps=0, attempts=0, error_fails=0, newton_fails=0, rhs=0, jac=0, lu=0, newton_iters=0)

    def f(t, y):
        stats["rhs"] += 1
        return fun(t, y)

    tol_n = bdf.newton_tolerance(rtol)
    t = float(t0)
    y = np.array(y0, dtype=float)
    f1 = f(t, y)
    h = fixed_h if fixed_h is not None else bdf.initial_step(f, t, y, f1, t_end, rtol, atol, order=EMBEDDED_ORDER)
    J = jac(t, y)
    stats["jac"] += 1
    jac_current = True
    lu, lu_h = None, None
    status = OK
    embedded = y.copy()
    while t < t_end:
        accepted = False
        while not accepted:
            if stats["attempts"] >= max_steps:
                status = MAX_STEPS
                break
            stats["attempts"] += 1
            if h < 10.0 * (np.nextafter(t, np.inf) - t):
                status = H_UNDERFLOW
                break
            if t + h > t_end:
                h = t_end - t
            scale = atol + rtol * np.abs(y)
            F = np.zeros((STAGES, S))
            Y = np.zeros((STAGES, S))
            F[0] = f1
            Y[0] = y
            failed = False
            while True:
                if lu is None or lu_h != h:
                    lu = scipy.linalg.lu_factor(np.eye(S) - h * gamma * J)
                    lu_h = h
                    stats["lu"] += 1
                failed = False
                for i in range(1, STAGES):
                    ti = t + c[i] * h
                    known = y + h * (A[i, :i] @ F[:i])
                    ok, n_it, Yi = _stage_newton(f, ti, known, Y[i - 1], h * gamma, lu, scale, tol_n)
                    stats["newton_iters"] += n_it
                    if not ok:
                        failed = True
                        break
                    Y[i] = Yi
                    F[i] = f(ti, Yi)
                if not failed or jac_current:
                    break
                J = jac(t, y)
                stats["jac"] += 1
                jac_current = True
                lu = None
            if failed:
                stats["newton_fails"] += 1
                h *= 0.5
                continue
            err = bdf.wrms(Y[4] - Y[3], atol + rtol * np.abs(Y[4]))
            if fixed_h is None and err > 1.0:
                stats["error_fails"] += 1
                h *= max(0.2, 0.9 * err ** (-1.0 / (EMBEDDED_ORDER + 1)))
                continue
            accepted = True
        if not accepted:
            break
        stats["steps"] += 1
        t = t + h
        y = Y[4].copy()
        embedded = Y[3].copy()
        f1 = F[4]
        jac_current = False
        if fixed_h is None:
            factor = 10.0 if err == 0.0 else 0.9 * err ** (-1.0 / (EMBEDDED_ORDER + 1))
            h *= min(10.0, max(0.2, factor))
    stats["embedded"] = embedded
    return bdf.Result(y, status, t, stats, None)


def _stage_newton(f, ti, known, guess, hg, lu, scale, tol):
    """Solve Y = known + hg f(ti, Y) by simplified Newton from `guess`: the
    corrector of ``bdf.newton_corrector`` with c = hg and psi = y_p - known,
    y_p = guess, so that G(d) = d - hg f(y_p + d) + (y_p - known)."""
    ok, n_it, Yi, _d = bdf.newton_corrector(f, ti, guess, hg, guess - known, lu, scale, tol)
    return ok, n_it, Yi


def solve_cell(net, phi, x0, t0, t_end, rtol, atol, max_steps=100000):
    """Integrate one cell of the network from x0 at t0 to t_end (seconds)."""
    kappa = chem.effective_coefficients(net, phi)
    nu = chem.stoichiometry(net)
    return integrate(lambda t, y: chem.rhs(net, kappa, y, nu),
                     lambda t, y: chem.jacobian(net, kappa, y, nu),
                     t0, np.asarray(x0, dtype=float), t_end, rtol, atol, max_steps)


def solve_cell_track(net, track, x0, t0, t_end, rtol, atol, max_steps=100000):
    """Integrate one cell whose environment follows `track` (see
    bdf.solve_cell_track): the coefficients are those of phi(t) at every time
    at which the method evaluates f or J."""
    nu = chem.stoichiometry(net)
    last = {}

    def kappa(t):
        if last.get("t") != t:
            last["t"] = t
            last["k"] = chem.effective_coefficients(net, bdf.track_params(track, t))
        return last["k"]

    return integrate(lambda t, y: chem.rhs(net, kappa(t), y, nu),
                     lambda t, y: chem.jacobian(net, kappa(t), y, nu),
                     t0, np.asarray(x0, dtype=float), t_end, rtol, atol, max_steps)
