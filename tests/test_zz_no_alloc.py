"""cbx_solve_noalloc (no device allocation) matches cbx_solve (GPU).

Callers that may not allocate GPU memory while they run use cbx_solve_noalloc,
whose scratch is a fixed array inside the library. This test calls it through
the C ABI twice in a row (the second call reuses the array left by the first)
and compares each result with cbx_solve on the same inputs. The two run the
same kernel and a cell's result does not depend on which CTA ran it, so the
results must be bitwise equal (the 1e-4 relative figure of the other GPU
tests is only printed on failure). Cases:
  * 150 species, 200 cells: the grid is limited by the device, not the array;
  * 500 species (Newton matrix in each CTA's scratch), with a few more cells
    than the CTAs that fit in the array (7 in FP64, 12 mixed): the grid is
    limited by the array and the CTAs back-fill;
  * a network the solver cannot run at all is rejected with CBX_E_TOO_LARGE.
It is collected last so that a failure here leaves every other test already
run; it also passes alone.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2511_10558_gb300 import build as _build  # noqa: E402

_build.build()
from paper_2511_10558_gb300 import carbox, synth  # noqa: E402
from tests.nets import tiny  # noqa: E402

TOL = 1e-4
FLOOR = 1e-12


def _fn():
    fn = carbox.lib.cbx_solve_noalloc
    fn.restype = C.c_int
    fn.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_double, C.c_double,
                   C.POINTER(carbox.cbx_options), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    return fn


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _compare_twice(dev, net, Cn, t_end, prec):
    fn = _fn()
    N = carbox.Network.from_synth(net)
    phi = torch.tensor(synth.cells(Cn), device=dev)
    x0 = torch.tensor(np.repeat(synth.initial_abundances(net)[:, None], Cn, axis=1), device=dev).contiguous()
    stream = torch.cuda.current_stream(dev)
    opt = carbox.options(precision=prec)
    ref, ref_st, _ = carbox.solve(N, phi, x0, 0.0, t_end, opt)
    torch.cuda.synchronize()
    r = ref.cpu().numpy()
    for call in range(2):
        out = torch.full_like(x0, np.nan)
        st = torch.full((Cn,), -1, dtype=torch.int32, device=dev)
        rc = fn(N.handle, C.c_void_p(phi.data_ptr()), C.c_void_p(x0.data_ptr()), Cn, 0.0, t_end,
                C.byref(opt), C.c_void_p(stream.cuda_stream), C.c_void_p(out.data_ptr()),
                C.c_void_p(st.data_ptr()), None)
        assert rc == carbox.CBX_OK, carbox.lib.cbx_last_error()
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        np.testing.assert_array_equal(st.cpu().numpy(), ref_st.cpu().numpy())
        big = r > FLOOR
        rel = np.abs(o[big] / r[big] - 1)
        assert rel.max() <= TOL, f"precision {prec}, call {call}: max rel diff {rel.max():.3e}"
        np.testing.assert_array_equal(o, r, err_msg=f"precision {prec}, call {call}: not bitwise equal")


@pytest.mark.parametrize("prec", [carbox.CBX_FP64, carbox.CBX_MIXED])
def test_noalloc_matches_solve_twice(dev, prec):
    _compare_twice(dev, synth.make_network(150, 1500), 200, 1e5 * synth.YEAR, prec)


@pytest.mark.parametrize("prec,cells", [(carbox.CBX_FP64, 9), (carbox.CBX_MIXED, 14)])
def test_noalloc_grid_limited_by_scratch(dev, prec, cells):
    _compare_twice(dev, synth.make_network(500, 6000), cells, 1e4 * synth.YEAR, prec)


def test_noalloc_rejects_a_network_the_solver_cannot_run(dev):
    # 40,000 reactions: the per-cell reaction rates alone exceed a CTA's shared memory
    R = 40000
    net = tiny(3, [(synth.COSMIC_RAY, (j % 2,), (2,), 1.0, 0.0, 0.0) for j in range(R)])
    N = carbox.Network.from_synth(net)
    phi = torch.tensor(synth.cells(2), device=dev)
    x0 = torch.full((3, 2), 1e-3, dtype=torch.float64, device=dev)
    out = torch.empty_like(x0)
    st = torch.empty(2, dtype=torch.int32, device=dev)
    rc = _fn()(N.handle, C.c_void_p(phi.data_ptr()), C.c_void_p(x0.data_ptr()), 2, 0.0, 1e10,
               C.byref(carbox.options()), None, C.c_void_p(out.data_ptr()), C.c_void_p(st.data_ptr()), None)
    assert rc == carbox.CBX_E_TOO_LARGE
    assert carbox.lib.cbx_last_error()
