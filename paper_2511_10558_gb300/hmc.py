"""Gradient-based sampling of reaction-rate uncertainty with Hamiltonian Monte Carlo.

The paper's aim is sensitivity analysis of astrochemical models to their
reaction rates (Sec. 3), and its appendix samples the rates of a whole network
with MCMC (App. A). Here the parameters are theta = ln alpha [R] and the
posterior (a reading; the paper gives no likelihood) is Gaussian in log10
abundances with a Gaussian prior around the network's own values:

    U(theta) = sum_{c,i} (log10 x_ci(theta) - y_ci)^2 / (2 sigma^2)
             + sum_j (theta_j - theta0_j)^2 / (2 s_j^2),

x_ci the abundance of target species i of cell c at t_end. grad U comes from
one recorded forward solve with alpha = exp(theta) passed for that call only
(cbx_solve_with_alpha: the network is not modified) and the discrete adjoint
(cbx_grad: dL/d ln alpha summed over cells) -- the derivative of the discrete
map with its step program frozen. Sampling: leapfrog integration of
H = U + |p|^2 / 2 with unit mass, step eps, L steps, then Metropolis acceptance
of the endpoint (Duane, Kennedy, Pendleton & Roweth 1987; Neal 2011).
"""
from __future__ import annotations

import numpy as np


def leapfrog(theta, p, g, U_and_grad, eps, L):
    """L leapfrog steps from (theta, p) with grad U(theta) = g; returns the end
    state (theta, p, U, g)."""
    theta = np.array(theta, dtype=float)
    p = np.array(p, dtype=float) - 0.5 * eps * g
    U = None
    for step in range(L):
        theta = theta + eps * p
        U, g = U_and_grad(theta)
        if step + 1 < L:
            p = p - eps * g
    p = p - 0.5 * eps * g
    return theta, p, U, g


def hmc_step(theta, U0, g0, U_and_grad, eps, L, rng):
    """One HMC transition from theta (with U0 = U(theta), g0 = grad U(theta)).
    Returns (theta', U', g', accepted, dH)."""
    p0 = rng.standard_normal(np.shape(theta))
    th, p, U1, g1 = leapfrog(theta, p0, g0, U_and_grad, eps, L)
    dH = (U1 + 0.5 * float(p @ p)) - (U0 + 0.5 * float(p0 @ p0))
    if np.isfinite(dH) and np.log(rng.uniform()) < -dH:
        return th, U1, g1, True, dH
    return np.array(theta, dtype=float), U0, g0, False, dH


class RatePosterior:
    """U(theta) and grad U for theta = ln alpha of `net` (a carbox.Network) given
    observed log10 abundances y [C, n] of species `targets` [C, n] at t_end for
    cells phi [C, 5] (torch CUDA, float64) from x0 [S, C]. Cells that do not end
    CBX_CELL_OK make U infinite (the transition is rejected)."""

    def __init__(self, net, phi, x0, t_end, targets, y_obs, sigma, prior_sd, theta0, opt=None, max_steps=4000):
        from . import carbox
        self.carbox = carbox
        self.net, self.phi, self.x0, self.t_end = net, phi, x0, float(t_end)
        self.targets = np.asarray(targets, dtype=np.int64)
        self.y = np.asarray(y_obs, dtype=float)
        self.sigma = float(sigma)
        self.prior_sd = np.broadcast_to(np.asarray(prior_sd, dtype=float), (net.R,)).copy()
        self.theta0 = np.asarray(theta0, dtype=float)
        self.opt = opt if opt is not None else carbox.options()
        self.tape = carbox.Tape(net, phi.shape[0], max_steps)

    def __call__(self, theta):
        import torch
        cb = self.carbox
        theta = np.asarray(theta, dtype=float)
        alpha = torch.tensor(np.exp(theta), dtype=torch.float64, device=self.phi.device)
        x, st = cb.solve_with_alpha(self.net, alpha, self.phi, self.x0, 0.0, self.t_end, self.opt, tape=self.tape)
        xh = x.cpu().numpy()
        if not bool((st == 0).all().item()):
            return np.inf, np.zeros_like(theta)
        C = xh.shape[1]
        cols = np.arange(C)[:, None]
        xt = xh[self.targets, cols]                      # [C, n]
        r = np.log10(xt) - self.y
        cot = np.zeros_like(xh)
        np.add.at(cot, (self.targets, np.broadcast_to(cols, self.targets.shape)),
                  r / (self.sigma ** 2 * xt * np.log(10.0)))
        ga, _, _ = cb.grad(self.tape, torch.tensor(cot, device=self.phi.device).contiguous(), C)
        d = theta - self.theta0
        U = float(np.sum(r ** 2)) / (2.0 * self.sigma ** 2) + float(np.sum(d ** 2 / (2.0 * self.prior_sd ** 2)))
        g = ga.cpu().numpy() + d / self.prior_sd ** 2
        return U, g
