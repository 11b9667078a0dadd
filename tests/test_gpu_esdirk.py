"""The ESDIRK method (CBX_METHOD_ESDIRK) vs the ESDIRK oracle, and vs the BDF (GPU).

* Twin parity: the GPU runs the same ESDIRK 4(3) with the same controller as
  oracle/esdirk.py, so abundances above 1e-12 per n_H agree within 1e-4
  relative (or, on a cell where a rounding difference flipped a step decision,
  the converged gate of tests/parity.py), in FP64 and mixed precision; element
  and charge conservation at 1e-10 on every cell.
* Cross-method parity: at rtol 1e-4 the ESDIRK and BDF results both lie within
  the methods' global error (1e-2 relative) of an rtol-1e-8 oracle reference.
* Tracks: a phi(t) track solved by the ESDIRK agrees with the oracle's ESDIRK.
* 500 species (matrix in global memory): twin parity and conservation.
* Argument errors: no recording with the ESDIRK (no adjoint), unknown methods
  rejected.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import chem, esdirk  # noqa: E402
from paper_2511_10558_gb300 import build as _build  # noqa: E402
from tests import parity  # noqa: E402

_build.build()
from paper_2511_10558_gb300 import carbox, synth  # noqa: E402

YR = synth.YEAR
RK = carbox.CBX_METHOD_ESDIRK


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _solve(N, phi, x0, t_end, dev, **kw):
    stats = carbox.stats_tensor(phi.shape[0], dev)
    x, st, stats = carbox.solve(N, torch.tensor(phi, device=dev).contiguous(), torch.tensor(x0, device=dev).contiguous(),
                                0.0, t_end, carbox.options(**kw), stats=stats)
    torch.cuda.synchronize()
    return x.cpu().numpy(), st.cpu().numpy(), carbox.stats_dict(stats.cpu().numpy())


def _conserved(net, x0, x):
    E0, Q0 = chem.element_totals(net, x0)
    E1, Q1 = chem.element_totals(net, x)
    return np.all(np.abs(E1 - E0) <= 1e-10 * E0) and abs(Q1 - Q0) <= 1e-10 * (np.abs(net.charge) @ x0)


@pytest.mark.parametrize("prec", [carbox.CBX_FP64, carbox.CBX_MIXED])
def test_single_cell_32_twin(dev, net32, prec):
    phi = synth.one_cell()
    x0 = synth.initial_abundances(net32)
    t_end = 1e6 * YR
    ref = esdirk.solve_cell(net32, phi[0], x0, 0.0, t_end, 1e-4, 1e-20)
    N = carbox.Network.from_synth(net32)
    x, st, sd = _solve(N, phi, x0[:, None], t_end, dev, precision=prec, method=RK)
    assert st[0] == carbox.CBX_CELL_OK
    assert parity.max_rel(x[:, 0], ref.x) <= 1e-4
    assert _conserved(net32, x0, x[:, 0])
    print("gpu steps", int(sd["steps"][0]), "oracle", ref.stats["steps"])
    assert abs(int(sd["steps"][0]) - ref.stats["steps"]) <= 0.02 * ref.stats["steps"]


@pytest.fixture(scope="module")
def batch(net150):
    C = 200
    phi = synth.cells(C, seed=17)
    x0 = np.repeat(synth.initial_abundances(net150)[:, None], C, axis=1)
    sel = np.linspace(0, C - 1, 16).astype(int)
    ref = parity.oracle_cells(net150, phi[sel], x0[:, sel], 1e6 * YR, method="esdirk")
    return phi, x0, sel, ref


@pytest.mark.parametrize("prec", [carbox.CBX_FP64, carbox.CBX_MIXED])
def test_batch_150_twin(dev, net150, batch, prec):
    phi, x0, sel, ref = batch
    t_end = 1e6 * YR
    N = carbox.Network.from_synth(net150)
    x, st, _ = _solve(N, phi, x0, t_end, dev, precision=prec, method=RK)
    assert np.all(st == carbox.CBX_CELL_OK)
    for c in range(phi.shape[0]):
        assert _conserved(net150, x0[:, c], x[:, c]), c
    within = [parity.max_rel(x[:, c], ref[:, k]) <= 1e-4 for k, c in enumerate(sel)]
    bad = [c for ok, c in zip(within, sel) if not ok]
    if bad:  # the converged gate, against the ESDIRK oracle's own error
        ks = [list(sel).index(c) for c in bad]
        tight = parity.oracle_cells(net150, phi[bad], x0[:, bad], t_end, *parity.TIGHT)
        for k, (c, kk) in enumerate(zip(bad, ks)):
            big = tight[:, k] > parity.FLOOR
            e_gpu = np.max(np.abs(x[big, c] / tight[big, k] - 1))
            e_orc = np.max(np.abs(ref[big, kk] / tight[big, k] - 1))
            assert e_gpu <= 2 * e_orc, (c, e_gpu, e_orc)
    assert sum(within) >= 14, within


def test_cross_method_parity(dev, net150):
    C = 6
    phi = synth.cells(C, seed=23)
    x0 = np.repeat(synth.initial_abundances(net150)[:, None], C, axis=1)
    t_end = 1e6 * YR
    N = carbox.Network.from_synth(net150)
    xr, sr, _ = _solve(N, phi, x0, t_end, dev, method=RK)
    xb, sb, _ = _solve(N, phi, x0, t_end, dev)
    assert np.all(sr == 0) and np.all(sb == 0)
    tight = parity.oracle_cells(net150, phi, x0, t_end, *parity.TIGHT)
    for c in range(C):
        e_rk, e_bdf = parity.max_rel(xr[:, c], tight[:, c]), parity.max_rel(xb[:, c], tight[:, c])
        print(f"cell {c}: error vs rtol-1e-8 reference: ESDIRK {e_rk:.2e}, BDF {e_bdf:.2e}")
        assert e_rk <= 1e-2 and e_bdf <= 1e-2


def test_track_twin(dev, net150):
    C = 4
    t_end = 1e6 * YR
    phi = synth.cells(C, seed=29)
    tr = synth.tracks(phi, t_end)
    x0 = np.repeat(synth.initial_abundances(net150)[:, None], C, axis=1)
    N = carbox.Network.from_synth(net150)
    x, st, _ = carbox.solve_track(N, torch.tensor(tr, device=dev).contiguous(),
                                  torch.tensor(x0, device=dev).contiguous(), 0.0, t_end, carbox.options(method=RK))
    torch.cuda.synchronize()
    x, st = x.cpu().numpy(), st.cpu().numpy()
    assert np.all(st == 0)
    ref = parity.oracle_cells(net150, None, x0, t_end, tracks=tr, method="esdirk")
    rel = [parity.max_rel(x[:, c], ref[:, c]) for c in range(C)]
    print("track cells vs ESDIRK oracle:", rel)
    assert sum(r <= 1e-4 for r in rel) >= C - 1 and max(rel) <= 1e-2


def test_esdirk_argument_errors(dev, net32):
    N = carbox.Network.from_synth(net32)
    phi = torch.tensor(synth.one_cell(), device=dev)
    x0 = torch.tensor(synth.initial_abundances(net32)[:, None], device=dev).contiguous()
    tape = carbox.Tape(N, 1, 100)
    with pytest.raises(carbox.CarboxError):
        carbox.solve_record(N, tape, phi, x0, 0.0, 1e10, carbox.options(method=RK))
    with pytest.raises(carbox.CarboxError):
        carbox.solve(N, phi, x0, 0.0, 1e10, carbox.options(method=7))


@pytest.mark.parametrize("prec", [carbox.CBX_FP64, carbox.CBX_MIXED])
def test_large_500_twin(dev, prec):
    # 500 species: the Newton matrix in each CTA's global workspace
    net = synth.make_network(500, 6000)
    N = carbox.Network.from_synth(net)
    C = 3
    phi = synth.cells(C, seed=37)
    x0 = np.repeat(synth.initial_abundances(net)[:, None], C, axis=1)
    t_end = 1e5 * YR
    x, st, _ = _solve(N, phi, x0, t_end, dev, precision=prec, method=RK)
    assert np.all(st == carbox.CBX_CELL_OK)
    ref = parity.oracle_cells(net, phi[:2], x0[:, :2], t_end, method="esdirk")
    for c in range(C):
        assert _conserved(net, x0[:, c], x[:, c]), c
    for c in range(2):
        assert parity.max_rel(x[:, c], ref[:, c]) <= 1e-4, c
