"""Time-dependent environment phi(t) (cbx_solve_track) vs the oracle (GPU).

* A constant track gives bitwise the constant-phi GPU solve.
* A collapse-and-warming track: abundances within 1e-4 of the oracle's
  solve_cell_track, or (on another step program) as accurate as the oracle
  against an rtol-1e-8 reference; conservation on every cell.
* A cell with knot times out of order ends BAD_INPUT without touching others;
  K < 1 is an argument error.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import bdf, chem  # noqa: E402
from paper_2511_10558_gb300 import build as _build  # noqa: E402
from tests import parity  # noqa: E402

_build.build()
from paper_2511_10558_gb300 import carbox, synth  # noqa: E402

YR = synth.YEAR


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def run_track(N, tr, x0, t_end, dev):
    x, st, _ = carbox.solve_track(N, torch.tensor(tr, device=dev).contiguous(),
                                  torch.tensor(x0, device=dev).contiguous(), 0.0, t_end)
    torch.cuda.synchronize()
    return x.cpu().numpy(), st.cpu().numpy()


def test_constant_track_is_constant_phi(dev, net150):
    C = 16
    phi = synth.cells(C)
    x0 = np.repeat(synth.initial_abundances(net150)[:, None], C, axis=1)
    t_end = 1e5 * YR
    N = carbox.Network.from_synth(net150)
    xr, sr, _ = carbox.solve(N, torch.tensor(phi, device=dev), torch.tensor(x0, device=dev).contiguous(), 0.0, t_end)
    tr = np.concatenate([np.zeros((C, 1, 1)), phi[:, None, :]], axis=2)  # K = 1
    x, st = run_track(N, tr, x0, t_end, dev)
    np.testing.assert_array_equal(x, xr.cpu().numpy())
    np.testing.assert_array_equal(st, sr.cpu().numpy())


def test_collapse_track_matches_oracle(dev, net150):
    C = 40
    t_end = 1e6 * YR
    phi = synth.cells(C)
    tr = synth.tracks(phi, t_end)
    x0 = np.repeat(synth.initial_abundances(net150)[:, None], C, axis=1)
    N = carbox.Network.from_synth(net150)
    x, st = run_track(N, tr, x0, t_end, dev)
    assert np.all(st == carbox.CBX_CELL_OK)
    for c in range(C):
        E0, Q0 = chem.element_totals(net150, x0[:, c])
        E1, Q1 = chem.element_totals(net150, x[:, c])
        assert np.all(np.abs(E1 - E0) <= 1e-10 * E0)
    # the track changes the answer (it is not ignored)
    xc, _, _ = carbox.solve(N, torch.tensor(phi, device=dev), torch.tensor(x0, device=dev).contiguous(), 0.0, t_end)
    assert np.max(np.abs(xc.cpu().numpy()[:, 0] / x[:, 0] - 1)) > 1e-2
    # the gate of tests/parity.py (twin parity, else the converged gate, no floor)
    sel = [0, 3, 7, C - 1]
    ref = parity.oracle_cells(net150, None, x0[:, sel], t_end, tracks=tr[sel])
    rep = parity.gate(x[:, sel], ref, net150, None, x0[:, sel], t_end, tracks=tr[sel])
    print(rep)


def test_bad_track_and_arguments(dev, net32):
    phi = np.repeat(synth.one_cell(), 3, axis=0)
    t_end = 1e4 * YR
    tr = synth.tracks(phi, t_end)
    tr[1, 2, 0] = tr[1, 1, 0]  # knot times not increasing in cell 1
    x0 = np.repeat(synth.initial_abundances(net32)[:, None], 3, axis=1)
    N = carbox.Network.from_synth(net32)
    x, st = run_track(N, tr, x0, t_end, dev)
    assert st[1] == carbox.CBX_CELL_BAD_INPUT and st[0] == carbox.CBX_CELL_OK and st[2] == carbox.CBX_CELL_OK
    np.testing.assert_array_equal(x[:, 1], x0[:, 1])
    np.testing.assert_array_equal(x[:, 0], x[:, 2])
    with pytest.raises(RuntimeError):
        carbox.solve_track(N, torch.zeros((3, 0, 6), dtype=torch.float64, device=dev),
                           torch.tensor(x0, device=dev).contiguous(), 0.0, t_end)


def test_track_gradients_match_oracle_adjoint(dev, net32):
    # gradients through phi(t): the reverse sweep re-evaluates the coefficients
    # at every recorded step time; compared with the oracle's adjoint of the
    # same program (step times read back from the tape) and with central
    # differences of its exact replay (common n_H factor, common T shift)
    from oracle import adjoint as adj
    t_end = 1e5 * YR
    C = 2
    phi = synth.cells(C, seed=9)
    tr = synth.tracks(phi, t_end)
    x0 = np.repeat(synth.initial_abundances(net32)[:, None], C, axis=1)
    N = carbox.Network.from_synth(net32)
    tr_d = torch.tensor(tr, device=dev).contiguous()
    x0_d = torch.tensor(x0, device=dev).contiguous()
    tape = carbox.Tape(N, C, 4000)
    x, st = carbox.solve_track_record(N, tape, tr_d, x0_d, 0.0, t_end)
    xp, _, _ = carbox.solve_track(N, tr_d, x0_d, 0.0, t_end)
    np.testing.assert_array_equal(x.cpu().numpy(), xp.cpu().numpy())  # recording does not change the solve
    xh = x.cpu().numpy()
    assert np.all(st.cpu().numpy() == carbox.CBX_CELL_OK)
    rng = np.random.default_rng(4)
    tgs, yts, cot = [], [], np.zeros_like(xh)
    for c in range(C):
        tg = np.sort(rng.choice(np.flatnonzero(xh[:, c] > 1e-12), 8, replace=False))
        yt = np.log10(xh[tg, c]) + rng.uniform(-0.5, 0.5, len(tg))
        tgs.append(tg)
        yts.append(yt)
        cot[:, c] = adj.log10_loss(xh[:, c], tg, yt)[1]
    ga, gn, gt, gz, gg, gav = [o.cpu().numpy() for o in
                               carbox.grad_env(tape, torch.tensor(cot, device=dev).contiguous(), C)]
    ga_ref = np.zeros(net32.n_reactions)
    for c in range(C):
        ts = tape.step_times(c)
        prog, k = [], 0
        for kind, q, v in tape.program(c):
            if kind == 2:
                prog.append(("step", q, v, ts[k], None))
                k += 1
            else:
                prog.append(("init", v) if kind == 0 else ("rescale", q, v))
        assert k == len(ts) and ts[-1] == t_end
        x_rep, prog_rep = adj.replay(net32, None, x0[:, c], prog, track=tr[c])
        _, cot_rep = adj.log10_loss(x_rep, tgs[c], yts[c])
        g_la, g_nH, g_T = adj.adjoint(net32, None, x0[:, c], prog_rep, cot_rep, track=tr[c])
        ga_ref += g_la
        assert gn[c] == pytest.approx(g_nH, rel=1e-3)
        assert gt[c] == pytest.approx(g_T, rel=1e-3)
        z, g0, av = adj.environment_gradients(net32, g_la)
        assert gz[c] == pytest.approx(z, rel=1e-3) and gg[c] == pytest.approx(g0, rel=1e-3)
        assert gav[c] == pytest.approx(av, rel=1e-3)
        if c == 0:
            eps = 1e-6

            def loss(track):
                xr, _ = adj.replay(net32, None, x0[:, 0], prog, track=track)
                return adj.log10_loss(xr, tgs[0], yts[0])[0]

            tp, tm = tr[0].copy(), tr[0].copy()
            tp[:, 1] *= np.exp(eps)
            tm[:, 1] *= np.exp(-eps)
            assert (loss(tp) - loss(tm)) / (2 * eps) == pytest.approx(gn[0], rel=1e-3)
            d = eps * tr[0, 0, 2]
            tp, tm = tr[0].copy(), tr[0].copy()
            tp[:, 2] += d
            tm[:, 2] -= d
            assert (loss(tp) - loss(tm)) / (2 * d) == pytest.approx(gt[0], rel=1e-3)
    big = np.abs(ga_ref) > 1e-6 * np.abs(ga_ref).max()
    assert np.all(np.abs(ga[big] - ga_ref[big]) <= 1e-3 * np.abs(ga_ref[big]))
