"""GPU adjoint (cbx_grad) vs the oracle's adjoint and vs finite differences (GPU).

* For single cells, the GPU gradients of L = sum over 10 seeded targets of
  (log10 x_i(t_f) - y_i)^2 w.r.t. ln alpha [R], ln n_H and T agree within
  1e-3 relative with the oracle's discrete adjoint of the same program (the
  GPU's step/order sequence read back from the tape and replayed exactly).
* Against the oracle's adjoint of its own solve (its own step sequence, which
  can differ from the GPU's by a step where a decision is at its threshold)
  they agree to the accuracy of the discretisation (5e-2 relative here).
* Central finite differences (step 1e-6) of the exact-corrector replay of the
  GPU's recorded program (read back from the tape) agree with the GPU gradient
  within 1e-3 relative.
* The torch.autograd.Function gives the same gradients through backward().
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import adjoint as adj  # noqa: E402
from oracle import bdf  # noqa: E402
from paper_2511_10558_gb300 import build as _build  # noqa: E402

_build.build()
from paper_2511_10558_gb300 import carbox, synth  # noqa: E402

YR = synth.YEAR


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def targets_for(x, seed):
    rng = np.random.default_rng(seed)
    cand = np.flatnonzero(x > 1e-12)
    t = np.sort(rng.choice(cand, size=min(10, len(cand)), replace=False))
    return t, np.log10(x[t]) + rng.uniform(-0.5, 0.5, len(t))


def gpu_grad(N, phi, x0, t_end, targets, y_t, dev, prec=carbox.CBX_FP64):
    Cn = phi.shape[0]
    phi_d = torch.tensor(phi, device=dev).contiguous()
    x0_d = torch.tensor(x0, device=dev).contiguous()
    tape = carbox.Tape(N, Cn, 4000)
    x, st = carbox.solve_record(N, tape, phi_d, x0_d, 0.0, t_end, carbox.options(precision=prec))
    xh = x.cpu().numpy()
    cot = np.zeros_like(xh)
    for c in range(Cn):
        cot[:, c] = adj.log10_loss(xh[:, c], targets[c], y_t[c])[1]
    ga, gn, gt = carbox.grad(tape, torch.tensor(cot, device=dev).contiguous(), Cn)
    torch.cuda.synchronize()
    return tape, xh, st.cpu().numpy(), ga.cpu().numpy(), gn.cpu().numpy(), gt.cpu().numpy()


def program_of(tape, cell):
    prog = []
    for kind, q, v in tape.program(cell):
        prog.append(("init", v) if kind == 0 else ("rescale", q, v) if kind == 1 else ("step", q, v, 0.0, None))
    return prog


def close(a, b, rel=1e-3):
    big = np.abs(b) > 1e-6 * np.abs(b).max()
    assert np.all(np.abs(a[big] - b[big]) <= rel * np.abs(b[big])), np.max(np.abs(a[big] / b[big] - 1))


@pytest.mark.parametrize("S,R", [(32, 200), (150, 1500)])
def test_grad_matches_oracle_adjoint(dev, S, R):
    net = synth.make_network(S, R)
    N = carbox.Network.from_synth(net)
    phi = synth.one_cell() if S == 32 else synth.cells(2, seed=4)
    Cn = phi.shape[0]
    x0 = np.repeat(synth.initial_abundances(net)[:, None], Cn, axis=1)
    t_end = 1e5 * YR
    refs, tg, yt = [], [], []
    for c in range(Cn):
        r = bdf.solve_cell(net, phi[c], x0[:, c], 0.0, t_end, 1e-4, 1e-20, record=True)
        t_, y_ = targets_for(r.x, 11 + c)
        refs.append(r)
        tg.append(t_)
        yt.append(y_)
    tape, xh, st, ga, gn, gt = gpu_grad(N, phi, x0, t_end, tg, yt, dev)
    assert np.all(st == carbox.CBX_CELL_OK)
    ga_same = np.zeros(R)
    ga_own = np.zeros(R)
    for c in range(Cn):
        # oracle adjoint of the GPU's own program (exact replay)
        prog = program_of(tape, c)
        x_rep, prog_rep = adj.replay(net, phi[c], x0[:, c], prog)
        _, cot = adj.log10_loss(x_rep, tg[c], yt[c])
        g = adj.adjoint(net, phi[c], x0[:, c], prog_rep, cot)
        ga_same += g[0]
        assert gn[c] == pytest.approx(g[1], rel=1e-3)
        assert gt[c] == pytest.approx(g[2], rel=1e-3)
        # oracle adjoint of its own solve
        _, cot = adj.log10_loss(refs[c].x, tg[c], yt[c])
        g2 = adj.adjoint(net, phi[c], x0[:, c], refs[c].program, cot)
        ga_own += g2[0]
        assert gn[c] == pytest.approx(g2[1], rel=5e-2)
        print(f"cell {c}: steps gpu {sum(1 for op in prog if op[0] == 'step')} oracle "
              f"{refs[c].stats['steps']}; d ln nH rel diff same-program {abs(gn[c] / g[1] - 1):.2e}, "
              f"own-solve {abs(gn[c] / g2[1] - 1):.2e}")
    close(ga, ga_same)
    close(ga, ga_own, rel=5e-2)


def test_grad_matches_finite_differences_of_gpu_program(dev, net32):
    phi = synth.one_cell()
    x0 = synth.initial_abundances(net32)[:, None]
    t_end = 1e5 * YR
    r = bdf.solve_cell(net32, phi[0], x0[:, 0], 0.0, t_end, 1e-4, 1e-20)
    tg, yt = targets_for(r.x, 11)
    N = carbox.Network.from_synth(net32)
    tape, xh, st, ga, gn, gt = gpu_grad(N, phi, x0, t_end, [tg], [yt], dev)
    prog = program_of(tape, 0)
    eps = 1e-6

    def loss(net=net32, p=phi[0]):
        x, _ = adj.replay(net, p, x0[:, 0], prog)
        return adj.log10_loss(x, tg, yt)[0]

    order = np.argsort(-np.abs(ga))
    for j in order[:4]:
        ap, am = net32.alpha.copy(), net32.alpha.copy()
        ap[j] *= np.exp(eps)
        am[j] *= np.exp(-eps)
        fd = (loss(adj.with_alpha(net32, ap)) - loss(adj.with_alpha(net32, am))) / (2 * eps)
        assert fd == pytest.approx(ga[j], rel=1e-3), j
    pp, pm = phi[0].copy(), phi[0].copy()
    pp[0] *= np.exp(eps)
    pm[0] *= np.exp(-eps)
    assert (loss(p=pp) - loss(p=pm)) / (2 * eps) == pytest.approx(gn[0], rel=1e-3)
    pp, pm = phi[0].copy(), phi[0].copy()
    pp[1] += eps * phi[0, 1]
    pm[1] -= eps * phi[0, 1]
    assert (loss(p=pp) - loss(p=pm)) / (2 * eps * phi[0, 1]) == pytest.approx(gt[0], rel=1e-3)


def test_autograd_function(dev, net32):
    N = carbox.Network.from_synth(net32)
    Cn = 3
    phi = synth.cells(Cn, seed=5)
    x0 = torch.tensor(np.repeat(synth.initial_abundances(net32)[:, None], Cn, axis=1), device=dev).contiguous()
    la = torch.tensor(np.log(net32.alpha), device=dev, requires_grad=True)
    lnH = torch.tensor(np.log(phi[:, 0]), device=dev, requires_grad=True)
    T = torch.tensor(phi[:, 1], device=dev, requires_grad=True)
    rest = torch.tensor(phi[:, 2:], device=dev).contiguous()
    t_end = 1e5 * YR
    lx = carbox.cell_solve(la, lnH, T, N, x0, rest, t_end)
    tgt = [2, 3, 6]
    loss = ((lx[tgt] + 5.0) ** 2).sum()
    loss.backward()
    # same gradients straight from the C ABI
    cot = torch.zeros_like(lx)
    cot[tgt] = 2 * (lx[tgt].detach() + 5.0)
    x = torch.pow(10.0, lx.detach())
    cotx = (cot / (x * np.log(10.0))).contiguous()
    tape = carbox.Tape(N, Cn, 4000)
    phi_d = torch.tensor(phi, device=dev).contiguous()
    phi_d[:, 0] = torch.exp(lnH.detach())
    carbox.solve_record(N, tape, phi_d, x0, 0.0, t_end)
    ga, gn, gt = carbox.grad(tape, cotx, Cn)
    # the Function solves with n_H = exp(ln n_H) and alpha = exp(ln alpha), one
    # ulp from the inputs above: the gradients agree to ~1e-9, not bitwise
    torch.testing.assert_close(la.grad, ga, rtol=1e-6, atol=1e-12)
    torch.testing.assert_close(lnH.grad, gn, rtol=1e-6, atol=1e-12)
    torch.testing.assert_close(T.grad, gt, rtol=1e-6, atol=1e-12)


def test_cell_solve_leaves_the_network_alone(dev, net32):
    # the autograd Function passes alpha for its call only: a plain solve on the
    # same Network afterwards returns the original result, and the Function's
    # result equals a solve of a separate network that holds those alpha values
    N = carbox.Network.from_synth(net32)
    Cn = 3
    phi = synth.cells(Cn, seed=5)
    phi_d = torch.tensor(phi, device=dev).contiguous()
    x0 = torch.tensor(np.repeat(synth.initial_abundances(net32)[:, None], Cn, axis=1), device=dev).contiguous()
    t_end = 1e5 * YR
    base, _, _ = carbox.solve(N, phi_d, x0, 0.0, t_end)
    base = base.cpu().numpy()
    la = torch.tensor(np.log(net32.alpha) + np.linspace(-0.4, 0.4, net32.n_reactions), device=dev,
                      requires_grad=True)
    lnH = torch.tensor(np.log(phi[:, 0]), device=dev)
    lx = carbox.cell_solve(la, lnH, torch.tensor(phi[:, 1], device=dev), N, x0,
                           torch.tensor(phi[:, 2:], device=dev).contiguous(), t_end)
    after, _, _ = carbox.solve(N, phi_d, x0, 0.0, t_end)
    np.testing.assert_array_equal(after.cpu().numpy(), base)
    other = adj.with_alpha(net32, torch.exp(la.detach()).cpu().numpy())
    N2 = carbox.Network.from_synth(other)
    phi2 = phi_d.clone()
    phi2[:, 0] = torch.exp(lnH)
    x2, _, _ = carbox.solve(N2, phi2.contiguous(), x0, 0.0, t_end)
    np.testing.assert_array_equal(torch.log10(x2).cpu().numpy(), lx.detach().cpu().numpy())
    assert np.max(np.abs(lx.detach().cpu().numpy() - np.log10(base))) > 1e-3  # the other alpha mattered


def test_environment_gradients(dev, net32):
    # cbx_grad_env: d/d ln zeta, d/d ln G0, d/dA_V of the GPU program against
    # (a) the oracle's adjoint of the same program mapped by
    # environment_gradients and (b) central differences of its exact replay
    phi = synth.one_cell()
    x0 = synth.initial_abundances(net32)[:, None]
    t_end = 1e5 * YR
    r = bdf.solve_cell(net32, phi[0], x0[:, 0], 0.0, t_end, 1e-4, 1e-20)
    tg, yt = targets_for(r.x, 11)
    N = carbox.Network.from_synth(net32)
    phi_d = torch.tensor(phi, device=dev).contiguous()
    x0_d = torch.tensor(x0, device=dev).contiguous()
    tape = carbox.Tape(N, 1, 4000)
    x, st = carbox.solve_record(N, tape, phi_d, x0_d, 0.0, t_end, carbox.options())
    xh = x.cpu().numpy()
    cot = adj.log10_loss(xh[:, 0], tg, yt)[1][:, None]
    out = carbox.grad_env(tape, torch.tensor(cot, device=dev).contiguous(), 1)
    torch.cuda.synchronize()
    ga, gn, gt, gz, gg, gav = [o.cpu().numpy() for o in out]
    # the plain entry point gives the same first three outputs
    ga2, gn2, gt2 = carbox.grad(tape, torch.tensor(cot, device=dev).contiguous(), 1)
    np.testing.assert_array_equal(ga, ga2.cpu().numpy())
    assert gn[0] == gn2.cpu().numpy()[0] and gt[0] == gt2.cpu().numpy()[0]
    prog = program_of(tape, 0)
    x_rep, prog_rep = adj.replay(net32, phi[0], x0[:, 0], prog)
    _, cot_rep = adj.log10_loss(x_rep, tg, yt)
    g_ref = adj.adjoint(net32, phi[0], x0[:, 0], prog_rep, cot_rep)
    z_ref, g0_ref, av_ref = adj.environment_gradients(net32, g_ref[0])
    assert gz[0] == pytest.approx(z_ref, rel=1e-3)
    assert gg[0] == pytest.approx(g0_ref, rel=1e-3)
    assert gav[0] == pytest.approx(av_ref, rel=1e-3)
    eps = 1e-6

    def loss(p):
        xr, _ = adj.replay(net32, p, x0[:, 0], prog)
        return adj.log10_loss(xr, tg, yt)[0]

    for col, g_env in ((4, gz[0]), (3, gg[0])):
        pp, pm = phi[0].copy(), phi[0].copy()
        pp[col] *= np.exp(eps)
        pm[col] *= np.exp(-eps)
        assert (loss(pp) - loss(pm)) / (2 * eps) == pytest.approx(g_env, rel=1e-3), col
    pp, pm = phi[0].copy(), phi[0].copy()
    pp[2] += eps
    pm[2] -= eps
    assert (loss(pp) - loss(pm)) / (2 * eps) == pytest.approx(gav[0], rel=1e-3)
