"""Variable-order BDF integrator for one cell, plain FP64 (TEST INFRASTRUCTURE ONLY).

The paper names the backward differentiation formulae as the field's stiff
integrator (Sec. 1; Byrne & Hindmarsh 1975, GEAR, DLSODES, SUNDIALS) and gives
no variant of its own (its solver is an ESDIRK method, Sec. 4). The variant
written out here is the quasi-constant step-size BDF in backward-difference
form of Shampine & Reichelt, "The MATLAB ODE Suite" (SIAM J. Sci. Comput. 18,
1997), with the NDF parameter kappa = 0 (plain BDF), orders 1..5.

Notation (one cell, S species):
    D[j] = backward difference nabla^j y_n on the current equal spacing h,
           j = 0..q+2 (D[0] = y_n).
    gamma_q = sum_{j=1..q} 1/j.
    BDF of order q:  sum_{j=1..q} (1/j) nabla^j y_{n+1} = h f(t_{n+1}, y_{n+1}).

One step, order q, size h:
    predictor  y0  = sum_{j=0..q} D[j]
    psi            = (1/gamma_q) sum_{j=1..q} gamma_j D[j]
    corrector  d - c f(t_{n+1}, y0 + d) + psi = 0,   c = h / gamma_q
               (this is the BDF equation rewritten with d = y_{n+1} - y0)
    Newton     (I - c J) dy = c f(y) - psi - d ;  y += dy ; d += dy
    error      err = || d / (q + 1) ||   (leading BDF error constant 1/(q+1))
    accept     D[q+2] = d - D[q+1]; D[q+1] = d; D[i] += D[i+1] for i = q..0

Constants and policies (the CUDA path restates the same values on its own):
    norms        weighted RMS with weights 1/(atol + rtol |y_i|): the Newton
                 test uses |y| of the predictor, the error test |y| of the result
    Newton       simplified Newton, at most 4 increments, with the stopping
                 rules of Hairer & Wanner II, Sec. IV.8 (contraction factor
                 from successive increment norms, geometric-tail error bound;
                 see newton_corrector), tolerance
                 tol_N = max(10 eps / rtol, min(0.03, sqrt(rtol))): a small
                 fraction of the error test's unit scale, never below the
                 rounding level of the weighted norm
    Jacobian     evaluated at (t0, y0), and again at the predictor when Newton
                 fails with a Jacobian that is not current (it is current only
                 between its evaluation and the next accepted step)
    LU           of M = I - c J, refactored whenever h or J changed since the
                 last factorisation; dense LU with partial pivoting (LAPACK getrf)
    Newton fail  with a current Jacobian: h <- h/2
    error fail   h <- h * max(0.2, 0.9 err^(-1/(q+1)))
    step/order   after q+1 accepted steps at the same h: error estimates at
                 orders q-1 (||D[q]/q||), q, q+1 (||D[q+2]/(q+2)||); the order
                 with the largest factor err_k^(-1/(k+1)) is taken, and
                 h <- h * min(10, 0.9 * that factor)
    h change     the differences D[1..q] are mapped to the new spacing by the
                 matrix of the interpolating polynomial (rescale_differences)
    last step    a step that would pass t_end is shortened to end at t_end
    initial h    Hairer, Norsett & Wanner, Solving ODEs I, Sec. II.4 (order 1)
    limits       max_steps step attempts -> MAX_STEPS; h < 10 ulp(t) ->
                 H_UNDERFLOW. Negative abundances are not clipped.
"""
from __future__ import annotations

import math
import numpy as np
import scipy.linalg

from . import chem

MAX_ORDER = 5
NEWTON_MAXITER = 4
SAFETY = 0.9
MIN_FACTOR = 0.2
MAX_FACTOR = 10.0

OK, MAX_STEPS, H_UNDERFLOW = 0, 1, 2

# gamma_q = sum_{j=1..q} 1/j, q = 0..MAX_ORDER+1
GAMMA = np.array([sum(1.0 / j for j in range(1, q + 1)) for q in range(MAX_ORDER + 2)])
# leading error constant of BDF order q
ERROR_CONST = np.array([1.0 / (q + 1) for q in range(MAX_ORDER + 2)])


def newton_tolerance(rtol):
    eps = np.finfo(float).eps
    return max(10.0 * eps / rtol, min(0.03, math.sqrt(rtol)))


def wrms(v, scale):
    """Weighted root-mean-square norm sqrt(mean((v_i / scale_i)^2))."""
    return float(np.sqrt(np.mean((v / scale) ** 2)))


def initial_step(f, t0, y0, f0, t_end, rtol, atol, order=1):
    """Starting step of Hairer, Norsett & Wanner, Solving ODEs I, Sec. II.4
    ("Starting step size"), for a method of order p = `order` (the BDF starts
    at order 1). Norms are weighted RMS with scale atol + rtol |y0|:
      (a) d0 = |y0|, d1 = |f0|;
      (b) a first guess h0 = 0.01 d0 / d1 (1e-6 when d0 or d1 < 1e-5);
      (c) one explicit Euler step y1 = y0 + h0 f0, and f1 = f(t0 + h0, y1);
      (d) d2 = |f1 - f0| / h0, an estimate of the second derivative;
      (e) h1 from 0.01 = h1^(p+1) max(d1, d2), i.e.
          h1 = (0.01 / max(d1, d2))^(1/(p+1)), or max(1e-6, 1e-3 h0) when
          max(d1, d2) <= 1e-15;
      (f) h = min(100 h0, h1), here also capped at t_end - t0.
    """
    scale = atol + rtol * np.abs(y0)
    d0 = wrms(y0, scale)
    d1 = wrms(f0, scale)
    h0 = 1e-6 if (d0 < 1e-5 or d1 < 1e-5) else 0.01 * d0 / d1
    y1 = y0 + h0 * f0
    f1 = f(t0 + h0, y1)
    d2 = wrms(f1 - f0, scale) / h0
    dmax = max(d1, d2)
    h1 = max(1e-6, h0 * 1e-3) if dmax <= 1e-15 else (0.01 / dmax) ** (1.0 / (order + 1))
    return min(100.0 * h0, h1, t_end - t0)


def _growth(err, p):
    """err^(-1/p), with a zero error giving an unbounded factor."""
    return math.inf if err == 0.0 else err ** (-1.0 / p)


def _newton_binomial(s, j):
    """s (s+1) ... (s+j-1) / j!  (weight of nabla^j in Newton's backward form)."""
    v = 1.0
    for m in range(j):
        v *= (s + m) / (m + 1)
    return v


def rescale_matrix(q, rho):
    """T[k-1, j-1], k, j = 1..q: the map of rescale_differences below."""
    T = np.zeros((q, q))
    for k in range(1, q + 1):
        for j in range(1, q + 1):
            T[k - 1, j - 1] = sum(((-1) ** i) * math.comb(k, i) * _newton_binomial(-i * rho, j)
                                  for i in range(k + 1))
    return T


def rescale_differences(D, q, rho):
    """Replace D[1..q] (spacing h) by the differences of the same polynomial on spacing rho*h.

    P(s) = sum_j D[j] C(s+j-1, j) interpolates y_{n-i} at s = -i. The new k-th
    difference is sum_i (-1)^i C(k, i) P(-i rho), i = 0..k. The D[0] term of that
    sum carries the weight sum_i (-1)^i C(k, i) = 0 for k >= 1, so
        D'[k] = sum_{j=1..q} T[k, j] D[j],
        T[k, j] = sum_{i=0..k} (-1)^i C(k, i) C(-i rho + j - 1, j),
    and D[0] = y_n is unchanged. Applying T to the differences alone (rather
    than evaluating P and re-differencing) keeps y_n out of the arithmetic: the
    conserved sums e^T D[j], j >= 1, then stay at rounding level.
    """
    D[1:q + 1] = rescale_matrix(q, rho) @ D[1:q + 1]


def newton_corrector(fun, t_new, y_pred, c, psi, lu, scale, tol, maxiter=NEWTON_MAXITER):
    """Solve the corrector equation G(d) = d - c f(t_new, y_pred + d) + psi = 0
    by simplified Newton: the matrix I - c J stays frozen (its LU is `lu`).

    Iteration m = 1, 2, ..., maxiter computes the increment
        Delta_m = (I - c J)^{-1} (-G(d_{m-1})),   d_0 = 0,
    and its weighted RMS norm n_m. The stopping rules are those of Hairer &
    Wanner, Solving ODEs II, Sec. IV.8 (simplified Newton for implicit
    methods), which assume the iterates contract linearly:

      * from m = 2 on, the contraction factor is estimated as
        theta = n_m / n_{m-1} (increment m = 1 gives no estimate);
      * with a factor theta < 1 the distance of d_m = d_{m-1} + Delta_m to
        the solution is at most the geometric tail theta / (1 - theta) n_m:
        d_m is accepted when that bound is below `tol` (or n_m is exactly 0);
      * the iteration is abandoned, before Delta_m is applied, when
        theta >= 1 (no contraction), or when the bound expected after the
        last permitted increment, theta^(maxiter - m + 1) / (1 - theta) n_m
        (maxiter - m further contractions of the tail), still exceeds `tol`;
      * a non-finite right-hand side also abandons the iteration.

    The iterate y = y_pred + d is carried as its own running sum (each
    increment added to y and to d), so y is never re-formed from y_pred + d.

    Returns (converged, increments computed, y, d).
    """
    d = np.zeros_like(y_pred)
    y = np.array(y_pred, dtype=float)
    n_prev = None  # norm of the previous increment
    for m in range(1, maxiter + 1):
        f = fun(t_new, y)
        if not np.all(np.isfinite(f)):
            return False, m, y, d
        delta = scipy.linalg.lu_solve(lu, c * f - psi - d)
        n_m = wrms(delta, scale)
        theta = None if n_prev is None else n_m / n_prev
        if theta is not None:
            hopeless = theta >= 1.0 or theta ** (maxiter - m + 1) / (1.0 - theta) * n_m > tol
            if hopeless:
                return False, m, y, d
        y = y + delta
        d = d + delta
        if n_m == 0.0 or (theta is not None and theta / (1.0 - theta) * n_m < tol):
            return True, m, y, d
        n_prev = n_m
    return False, maxiter, y, d


class Result:
    def __init__(self, x, status, t, stats, program):
        self.x = x
        self.status = status
        self.t = t
        self.stats = stats
        self.program = program


def integrate(fun, jac, t0, y0, t_end, rtol, atol, max_steps=100000, record=False):
    """Integrate y' = fun(t, y) from t0 to t_end with the BDF described above.

    Returns a Result with y(t_end), the status, counters, and (record=True) the
    program of difference-array operations that an exact replay needs:
    ("init", h0), ("rescale", q, rho) and ("step", q, h, t_new, y_new) in order.
    """
    S = y0.size
    stats = dict(steps=0, attempts=0, error_fails=0, newton_fails=0, rhs=0, jac=0, lu=0,
                 newton_iters=0)

    def f(t, y):
        stats["rhs"] += 1
        return fun(t, y)

    tol_n = newton_tolerance(rtol)
    t = float(t0)
    y = np.array(y0, dtype=float)
    f0 = f(t, y)
    h = initial_step(f, t, y, f0, t_end, rtol, atol)
    D = np.zeros((MAX_ORDER + 3, S))
    D[0] = y
    D[1] = h * f0
    q = 1
    n_equal = 0
    J = jac(t, y)
    stats["jac"] += 1
    jac_current = True
    lu = None
    program = [("init", h)] if record else None
    status = OK

    def change_h(factor, new_q):
        nonlocal h, lu, n_equal
        rescale_differences(D, new_q, factor)
        if record:
            program.append(("rescale", new_q, factor))
        h *= factor
        n_equal = 0
        lu = None

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
            t_new = t + h
            if t_new > t_end:
                t_new = t_end
                change_h((t_end - t) / h, q)
                h = t_end - t
            y_pred = D[:q + 1].sum(axis=0)
            scale = atol + rtol * np.abs(y_pred)
            psi = (GAMMA[1:q + 1] @ D[1:q + 1]) / GAMMA[q]
            c = h / GAMMA[q]
            while True:
                if lu is None:
                    lu = scipy.linalg.lu_factor(np.eye(S) - c * J)
                    stats["lu"] += 1
                converged, n_it, y_new, d = newton_corrector(f, t_new, y_pred, c, psi, lu,
                                                             scale, tol_n)
                stats["newton_iters"] += n_it
                if converged or jac_current:
                    break
                J = jac(t_new, y_pred)
                stats["jac"] += 1
                jac_current = True
                lu = None
            if not converged:
                stats["newton_fails"] += 1
                change_h(0.5, q)
                continue
            scale = atol + rtol * np.abs(y_new)
            err = wrms(ERROR_CONST[q] * d, scale)
            if err > 1.0:
                stats["error_fails"] += 1
                change_h(max(MIN_FACTOR, SAFETY * err ** (-1.0 / (q + 1))), q)
                continue
            accepted = True
        if not accepted:
            break
        # accepted step: update the differences to the new point
        stats["steps"] += 1
        if record:
            program.append(("step", q, h, t_new, y_new.copy()))
        t = t_new
        jac_current = False
        n_equal += 1
        D[q + 2] = d - D[q + 1]
        D[q + 1] = d
        for i in range(q, -1, -1):
            D[i] += D[i + 1]
        if n_equal < q + 1:
            continue
        # step size and order selection
        err_m = wrms(ERROR_CONST[q - 1] * D[q], scale) if q > 1 else np.inf
        err_p = wrms(ERROR_CONST[q + 1] * D[q + 2], scale) if q < MAX_ORDER else np.inf
        factors = np.array([_growth(err_m, q), _growth(err, q + 1), _growth(err_p, q + 2)])
        best = int(np.argmax(factors))
        q += best - 1
        change_h(min(MAX_FACTOR, SAFETY * factors[best]), q)
    return Result(D[0].copy(), status, t, stats, program)


def solve_cell(net, phi, x0, t0, t_end, rtol, atol, max_steps=100000, record=False):
    """Integrate one cell of the network from x0 at t0 to t_end (seconds)."""
    kappa = chem.effective_coefficients(net, phi)
    nu = chem.stoichiometry(net)
    return integrate(lambda t, y: chem.rhs(net, kappa, y, nu),
                     lambda t, y: chem.jacobian(net, kappa, y, nu),
                     t0, np.asarray(x0, dtype=float), t_end, rtol, atol, max_steps, record)


def track_params(track, t):
    """phi(t) = (n_H, T, A_V, G0, zeta) of one cell from its knots [K, 6]
    (t_k, n_H, T, A_V, G0, zeta): linear between knots, the end values
    outside [t_0, t_{K-1}] (the environment phi of the generalised system
    dn/dt = f(n, k(phi), phi) of Sec. 2, here a function of time)."""
    track = np.asarray(track, dtype=float)
    K = track.shape[0]
    k = 0
    while k + 1 < K and track[k + 1, 0] <= t:
        k += 1
    A = track[k]
    if k + 1 >= K or t <= A[0]:
        return A[1:].copy()
    B = track[k + 1]
    w = (t - A[0]) / (B[0] - A[0])
    return A[1:] + w * (B[1:] - A[1:])


def solve_cell_track(net, track, x0, t0, t_end, rtol, atol, max_steps=100000, record=False):
    """Integrate one cell whose environment follows `track`: the rate
    coefficients are those of phi(t) at every time the method evaluates f or J.
    x is per n_H, so a changing n_H enters only the two-body coefficients."""
    nu = chem.stoichiometry(net)
    last = {}

    def kappa(t):
        if last.get("t") != t:
            last["t"] = t
            last["k"] = chem.effective_coefficients(net, track_params(track, t))
        return last["k"]

    return integrate(lambda t, y: chem.rhs(net, kappa(t), y, nu),
                     lambda t, y: chem.jacobian(net, kappa(t), y, nu),
                     t0, np.asarray(x0, dtype=float), t_end, rtol, atol, max_steps, record)
