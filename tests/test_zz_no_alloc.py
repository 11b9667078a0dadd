"""cbx_solve_noalloc (no device allocation) matches cbx_solve (GPU).

Callers that may not allocate GPU memory while they run use cbx_solve_noalloc,
whose scratch is a fixed array inside the library. This test calls it through
the C ABI twice in a row (the second call reuses the array left by the first)
and compares each result with cbx_solve on the same inputs, within the
tolerance of the other GPU tests (1e-4 relative above 1e-12 per n_H; the two
run the same kernel, so they agree far more closely). It is collected last so
that a failure here leaves every other test already run; it also passes alone.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2511_10558_gb300 import build as _build  # noqa: E402

_build.build()
from paper_2511_10558_gb300 import carbox, synth  # noqa: E402

TOL = 1e-4
FLOOR = 1e-12


def test_noalloc_matches_solve_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    fn = carbox.lib.cbx_solve_noalloc
    fn.restype = C.c_int
    fn.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_double, C.c_double,
                   C.POINTER(carbox.cbx_options), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    net = synth.make_network(150, 1500)
    N = carbox.Network.from_synth(net)
    Cn = 200
    phi = torch.tensor(synth.cells(Cn), device=dev)
    x0 = torch.tensor(np.repeat(synth.initial_abundances(net)[:, None], Cn, axis=1), device=dev).contiguous()
    t_end = 1e5 * synth.YEAR
    stream = torch.cuda.current_stream(dev)
    for prec in (carbox.CBX_FP64, carbox.CBX_MIXED):
        opt = carbox.options(precision=prec)
        ref, ref_st, _ = carbox.solve(N, phi, x0, 0.0, t_end, opt)
        for call in range(2):
            out = torch.full_like(x0, np.nan)
            st = torch.full((Cn,), -1, dtype=torch.int32, device=dev)
            rc = fn(N.handle, C.c_void_p(phi.data_ptr()), C.c_void_p(x0.data_ptr()), Cn, 0.0, t_end,
                    C.byref(opt), C.c_void_p(stream.cuda_stream), C.c_void_p(out.data_ptr()),
                    C.c_void_p(st.data_ptr()), None)
            assert rc == carbox.CBX_OK, carbox.lib.cbx_last_error()
            torch.cuda.synchronize()
            r = ref.cpu().numpy()
            o = out.cpu().numpy()
            np.testing.assert_array_equal(st.cpu().numpy(), ref_st.cpu().numpy())
            big = r > FLOOR
            rel = np.abs(o[big] / r[big] - 1)
            assert rel.max() <= TOL, f"precision {prec}, call {call}: max rel diff {rel.max():.3e}"
