"""HMC over ln alpha driven by the CUDA solver and its discrete adjoint (GPU).

* The posterior gradient of hmc.RatePosterior (one recorded solve + cbx_grad,
  plus the prior) agrees within 1e-3 with the oracle's adjoint of the same
  recorded step programs (replayed exactly) plus the prior.
* Two HMC transitions run end to end from the prior mean.
"""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import adjoint as adj  # noqa: E402
from paper_2511_10558_gb300 import build as _build  # noqa: E402

_build.build()
from paper_2511_10558_gb300 import carbox, hmc, synth  # noqa: E402

YR = synth.YEAR


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def program_of(tape, cell):
    prog = []
    for kind, q, v in tape.program(cell):
        prog.append(("init", v) if kind == 0 else ("rescale", q, v) if kind == 1 else ("step", q, v, 0.0, None))
    return prog


def test_rate_posterior_gradient_and_transitions(dev, net32):
    N = carbox.Network.from_synth(net32)
    R = net32.n_reactions
    theta0 = np.log(net32.alpha)
    phi = np.array([[1e4, 20.0, 5.0, 1.0, synth.ZETA0], [3e3, 50.0, 2.0, 1.0, synth.ZETA0]])
    C = phi.shape[0]
    x0 = np.repeat(synth.initial_abundances(net32)[:, None], C, axis=1)
    t_end = 1e5 * YR
    phi_d = torch.tensor(phi, device=dev).contiguous()
    x0_d = torch.tensor(x0, device=dev).contiguous()
    # synthetic observations: abundances under perturbed rates
    rng = np.random.default_rng(5)
    theta_true = theta0 + 0.2 * rng.standard_normal(R)
    N.set_alpha(np.exp(theta_true))
    xt, st, _ = carbox.solve(N, phi_d, x0_d, 0.0, t_end)
    xt = xt.cpu().numpy()
    assert np.all(st.cpu().numpy() == 0)
    targets = np.array([np.sort(rng.choice(np.flatnonzero(xt[:, c] > 1e-10), 5, replace=False)) for c in range(C)])
    y = np.log10(xt[targets, np.arange(C)[:, None]])
    sigma, prior_sd = 0.1, 0.5
    post = hmc.RatePosterior(N, phi_d, x0_d, t_end, targets, y, sigma, prior_sd, theta0)
    U0, g0 = post(theta0)
    assert np.isfinite(U0) and np.all(np.isfinite(g0))
    # oracle: adjoint of the recorded programs at theta0, plus the prior (zero at theta0)
    net_a = adj.with_alpha(net32, np.exp(theta0))
    g_ref = np.zeros(R)
    U_ref = 0.0
    for c in range(C):
        x_rep, prog_rep = adj.replay(net_a, phi[c], x0[:, c], program_of(post.tape, c))
        r = np.log10(x_rep[targets[c]]) - y[c]
        U_ref += float(np.sum(r ** 2)) / (2 * sigma ** 2)
        cot = np.zeros_like(x_rep)
        cot[targets[c]] = r / (sigma ** 2 * x_rep[targets[c]] * np.log(10.0))
        g_ref += adj.adjoint(net_a, phi[c], x0[:, c], prog_rep, cot)[0]
    assert U0 == pytest.approx(U_ref, rel=1e-3)
    big = np.abs(g_ref) > 1e-6 * np.abs(g_ref).max()
    np.testing.assert_allclose(g0[big], g_ref[big], rtol=1e-3)
    # two transitions
    th, U, g = theta0.copy(), U0, g0
    rng2 = np.random.default_rng(9)
    t = time.perf_counter()
    for _ in range(2):
        th, U, g, acc, dH = hmc.hmc_step(th, U, g, post, 2e-3, 3, rng2)
        assert np.isfinite(U) and np.all(np.isfinite(g)) and np.isfinite(dH)
        print(f"accepted {acc}, dH {dH:.3e}, U {U:.4f}")
    print(f"{(time.perf_counter() - t) / 2:.3f} s per transition (3 leapfrog steps, {C} cells, {R} rates)")
