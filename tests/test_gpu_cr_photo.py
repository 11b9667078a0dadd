"""Networks with the cosmic-ray-induced photo form of App. B.1 (GPU).

k = alpha (T/300)^beta E/(1 - omega) zeta for CBX_CR_PHOTO reactions (E in the
gamma field, omega the network's albedo). The GPU solve is compared with the
oracle element by element (twin parity, 1e-4 relative above 1e-12 per n_H)
with element and charge conservation at 1e-10 on every cell, in FP64 and
mixed precision; the adjoint's gradients with respect to ln alpha, T and
ln zeta (which now also enter through the CR-photo terms) are compared with
the oracle's adjoint of the same recorded program.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import adjoint as adj  # noqa: E402
from oracle import bdf, chem  # noqa: E402
from paper_2511_10558_gb300 import build as _build  # noqa: E402

_build.build()
from paper_2511_10558_gb300 import carbox, synth  # noqa: E402

YR = synth.YEAR
TOL, FLOOR = 1e-4, 1e-12


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


@pytest.mark.parametrize("prec", [carbox.CBX_FP64, carbox.CBX_MIXED])
def test_cr_photo_twin_parity(dev, prec):
    net = synth.make_network(150, 1500, cr_photo_frac=0.3)
    assert (net.rtype == synth.CR_PHOTO).sum() > 50
    N = carbox.Network.from_synth(net)
    Cn = 8
    phi = synth.cells(Cn, seed=21)
    x0 = np.repeat(synth.initial_abundances(net)[:, None], Cn, axis=1)
    t_end = 1e6 * YR
    x, st, _ = carbox.solve(N, torch.tensor(phi, device=dev), torch.tensor(x0, device=dev).contiguous(), 0.0, t_end,
                            carbox.options(precision=prec))
    torch.cuda.synchronize()
    x, st = x.cpu().numpy(), st.cpu().numpy()
    assert np.all(st == carbox.CBX_CELL_OK)
    qs = np.abs(net.charge) @ x0[:, 0]
    E0, Q0 = chem.element_totals(net, x0[:, 0])
    for c in range(Cn):
        E1, Q1 = chem.element_totals(net, x[:, c])
        assert np.all(np.abs(E1 - E0) <= 1e-10 * E0) and abs(Q1 - Q0) <= 1e-10 * qs
    for c in (0, 3, Cn - 1):
        ref = bdf.solve_cell(net, phi[c], x0[:, c], 0.0, t_end, 1e-4, 1e-20).x
        big = ref > FLOOR
        rel = np.max(np.abs(x[big, c] / ref[big] - 1))
        assert rel <= TOL, (c, rel)


def test_cr_photo_gradients_match_oracle_adjoint(dev):
    net = synth.make_network(32, 200, cr_photo_frac=0.5)
    assert (net.rtype == synth.CR_PHOTO).sum() >= 10
    # give the CR-photo reactions a temperature dependence that matters
    crp = np.flatnonzero(net.rtype == synth.CR_PHOTO)
    net.beta[crp] = np.linspace(0.3, 1.0, len(crp))
    N = carbox.Network.from_synth(net)
    phi = np.array([[1e4, 60.0, 5.0, 1.0, 1.3e-16]])
    x0 = synth.initial_abundances(net)[:, None]
    t_end = 1e5 * YR
    tape = carbox.Tape(N, 1, 4000)
    x, st = carbox.solve_record(N, tape, torch.tensor(phi, device=dev), torch.tensor(x0, device=dev).contiguous(),
                                0.0, t_end, carbox.options())
    xh = x.cpu().numpy()[:, 0]
    assert int(st.cpu()[0]) == carbox.CBX_CELL_OK
    rng = np.random.default_rng(5)
    tg = np.sort(rng.choice(np.flatnonzero(xh > 1e-12), 10, replace=False))
    yt = np.log10(xh[tg]) + rng.uniform(-0.5, 0.5, 10)
    cot = adj.log10_loss(xh, tg, yt)[1][:, None]
    ga, gn, gt, gz, gg, gav = [o.cpu().numpy() for o in
                               carbox.grad_env(tape, torch.tensor(cot, device=dev).contiguous(), 1)]
    prog = []
    for kind, q, v in tape.program(0):
        prog.append(("init", v) if kind == 0 else ("rescale", q, v) if kind == 1 else ("step", q, v, 0.0, None))
    x_rep, prog_rep = adj.replay(net, phi[0], x0[:, 0], prog)
    _, cot_rep = adj.log10_loss(x_rep, tg, yt)
    g_la, g_nH, g_T = adj.adjoint(net, phi[0], x0[:, 0], prog_rep, cot_rep)
    z_ref, g0_ref, av_ref = adj.environment_gradients(net, g_la)
    big = np.abs(g_la) > 1e-6 * np.abs(g_la).max()
    assert np.all(np.abs(ga[big] - g_la[big]) <= 1e-3 * np.abs(g_la[big]))
    assert np.abs(g_la[crp]).max() > 1e-6 * np.abs(g_la).max()  # the CR-photo terms take part
    assert gt[0] == pytest.approx(g_T, rel=1e-3)
    assert gn[0] == pytest.approx(g_nH, rel=1e-3)
    assert gz[0] == pytest.approx(z_ref, rel=1e-3)
    # the T gradient includes the CR-photo terms beta_j/T dL/d ln k_j
    tb = net.rtype == synth.TWO_BODY
    g_T_tb = float(g_la[tb] @ (net.beta[tb] / phi[0, 1] + net.gamma[tb] / phi[0, 1] ** 2))
    g_T_crp = float(g_la[crp] @ (net.beta[crp] / phi[0, 1]))
    assert g_T == pytest.approx(g_T_tb + g_T_crp, rel=1e-9)
    assert abs(g_T_crp) > 1e-3 * abs(g_T)
