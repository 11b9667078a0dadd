"""Continuous-batching server (GPU).

* Requests of the 32-, 150- and 500-species networks with different cell
  counts and time spans are submitted together while a long request runs; each
  result is the same (bitwise, hence within any tolerance) as the same request
  solved alone, and as a direct cbx_solve.
* With a memory budget that fits one request at a time, every request still
  completes, the peak reservation stays within the budget and only one request
  runs at a time; with a large budget several run concurrently.
* Queued requests of the same network (different cell counts and time spans)
  are merged into one launch, and each result is bitwise the result of that
  request solved alone.
* The default budget is derived from the free device memory; destroying a
  server with queued requests and a thread blocked waiting on one of them
  fails those requests and returns.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2511_10558_gb300 import build as _build  # noqa: E402

_build.build()
from paper_2511_10558_gb300 import carbox, synth  # noqa: E402

YR = synth.YEAR


@pytest.fixture(scope="module")
def nets():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    out = {}
    for S, R in [(32, 200), (150, 1500), (500, 6000)]:
        net = synth.make_network(S, R)
        out[S] = (net, carbox.Network.from_synth(net))
    return out


def make_requests(nets):
    rng = np.random.default_rng(13)
    reqs = []
    for k, (S, C, yrs) in enumerate([(150, 300, 1e6), (32, 7, 1e4), (500, 3, 1e3), (150, 40, 1e5),
                                     (32, 200, 1e7), (500, 1, 1e4), (150, 1, 1e3)]):
        net, _ = nets[S]
        phi = synth.cells(C, seed=100 + k)
        x0 = np.repeat(synth.initial_abundances(net)[:, None], C, axis=1)
        reqs.append((S, phi, x0, yrs * YR))
    return reqs


def test_same_alone_and_in_the_mix(nets):
    opt = carbox.options(precision=carbox.CBX_MIXED)
    reqs = make_requests(nets)
    srv = carbox.Server(mem_budget=16 << 30, n_streams=8, max_ctas=64)
    ids = [srv.submit(nets[S][1], phi, x0, 0.0, t, opt) for S, phi, x0, t in reqs]
    mixed = [srv.wait(i) for i in ids]
    stats = srv.stats()
    assert stats["peak_running"] >= 2, stats
    for (S, phi, x0, t), (x, st, _) in zip(reqs, mixed):
        srv2 = carbox.Server(mem_budget=16 << 30, n_streams=1, max_ctas=0)
        x1, st1, _ = srv2.wait(srv2.submit(nets[S][1], phi, x0, 0.0, t, opt))
        srv2.close()
        np.testing.assert_array_equal(st, st1)
        np.testing.assert_array_equal(x, x1)
        xd, sd = carbox.solve_host(nets[S][1], phi, x0, 0.0, t, opt)[:2]
        np.testing.assert_array_equal(x, xd)
        assert np.all(st == carbox.CBX_CELL_OK)
    srv.close()


def test_memory_admission(nets):
    opt = carbox.options(precision=carbox.CBX_MIXED)
    net, N = nets[150]
    phi = synth.cells(64, seed=9)
    x0 = np.repeat(synth.initial_abundances(net)[:, None], 64, axis=1)
    # size the budget to one request
    srv = carbox.Server(mem_budget=1 << 40, n_streams=4, max_ctas=32)
    big = srv.submit(N, phi, x0, 0.0, 1e4 * YR, opt)
    srv.wait(big)
    srv.close()
    one = 64 * (40 + 2 * 150 * 8 + 8 + 4) + 64 * 80 * 1024 + 8192  # upper bound of one request's reservation
    srv = carbox.Server(mem_budget=one, n_streams=4, max_ctas=32)
    ids = [srv.submit(N, phi, x0, 0.0, 1e4 * YR, opt) for _ in range(5)]
    outs = [srv.wait(i) for i in ids]
    st = srv.stats()
    assert st["peak_bytes"] <= one and st["peak_running"] == 1, st
    for x, s_, _ in outs[1:]:
        np.testing.assert_array_equal(x, outs[0][0])
    srv.close()
    with pytest.raises(carbox.CarboxError):
        tiny = carbox.Server(mem_budget=1024, n_streams=1, max_ctas=0)
        tiny.submit(N, phi, x0, 0.0, 1e4 * YR, opt)


def test_merged_requests_same_as_alone(nets):
    # one stream: while the first request runs, the others queue and are merged
    opt = carbox.options(precision=carbox.CBX_MIXED)
    net, N = nets[150]
    srv = carbox.Server(mem_budget=0, n_streams=1, max_ctas=76)
    first = srv.submit(N, synth.cells(152, seed=40), np.repeat(synth.initial_abundances(net)[:, None], 152, axis=1),
                       0.0, 1e6 * YR, opt)
    reqs = []
    for k, (C, yrs) in enumerate([(5, 1e3), (40, 1e5), (1, 1e4), (17, 1e6), (60, 3e4)]):
        phi = synth.cells(C, seed=50 + k)
        x0 = np.repeat(synth.initial_abundances(net)[:, None], C, axis=1)
        reqs.append((phi, x0, yrs * YR, srv.submit(N, phi, x0, 0.0, yrs * YR, opt)))
    srv.wait(first)
    outs = [srv.wait(rid) for *_, rid in reqs]
    info = srv.info()
    srv.close()
    assert info["merged_requests"] >= 3 and info["launches"] <= 3, info
    for (phi, x0, t, _), (x, st, _) in zip(reqs, outs):
        xd, sd = carbox.solve_host(N, phi, x0, 0.0, t, opt)[:2]
        np.testing.assert_array_equal(st, sd)
        np.testing.assert_array_equal(x, xd)
        assert np.all(st == carbox.CBX_CELL_OK)


def test_budget_and_destroy_with_waiters(nets):
    import threading
    free, _ = torch.cuda.mem_get_info()
    srv = carbox.Server(mem_budget=0, n_streams=1, max_ctas=76)
    assert 0 < srv.info()["budget"] <= free
    capped = carbox.Server(mem_budget=1 << 30, n_streams=1, max_ctas=76)
    assert capped.info()["budget"] == 1 << 30
    capped.close()
    net, N = nets[500]  # a long launch (~1 s): the later requests are still queued at destroy
    opt = carbox.options(precision=carbox.CBX_MIXED)
    x0 = np.repeat(synth.initial_abundances(net)[:, None], 152, axis=1)
    running = srv.submit(N, synth.cells(152, seed=41), x0, 0.0, 1e6 * YR, opt)
    queued = [srv.submit(nets[32][1], synth.cells(3, seed=42 + k),
                         np.repeat(synth.initial_abundances(nets[32][0])[:, None], 3, axis=1), 0.0,
                         (1e3 + k) * YR, carbox.options()) for k in range(2)]
    result = {}

    def waiter():
        try:
            srv.wait(queued[0])
            result["ok"] = True
        except carbox.CarboxError as e:
            result["error"] = e.code

    th = threading.Thread(target=waiter)
    th.start()
    import time
    time.sleep(0.2)
    state, _ = srv.poll(queued[1])
    assert state in (0, 1)
    srv.close()  # fails what is still queued, waits for the running launch and the waiter
    th.join(timeout=60)
    assert not th.is_alive()
    assert result.get("error") == carbox.CBX_E_ARG or result.get("ok"), result
    del running
