"""Pins for the oracle's time-dependent environment phi(t) (no GPU).

* track_params: knots reproduced exactly, linear in between, end values
  outside the knot range.
* A constant track gives exactly the constant-phi solve.
* A -> B by cosmic rays with zeta(t) linear in time: x_A(t1) =
  a exp(-alpha (zeta_a + zeta_b) t1 / 2) (closed form of dx/dt = -alpha zeta(t) x).
* x is per n_H: an n_H track leaves a network without two-body reactions
  exactly unchanged.
"""
import numpy as np
import pytest

from oracle import bdf
from paper_2511_10558_gb300 import synth
from tests.nets import tiny


def test_track_interpolation():
    tr = np.array([[10.0, 1e3, 20.0, 1.0, 1.0, 1e-17],
                   [20.0, 1e5, 40.0, 3.0, 2.0, 3e-17]])
    np.testing.assert_array_equal(bdf.track_params(tr, 10.0), tr[0, 1:])
    np.testing.assert_array_equal(bdf.track_params(tr, 20.0), tr[1, 1:])
    np.testing.assert_array_equal(bdf.track_params(tr, 0.0), tr[0, 1:])
    np.testing.assert_array_equal(bdf.track_params(tr, 99.0), tr[1, 1:])
    np.testing.assert_allclose(bdf.track_params(tr, 15.0), 0.5 * (tr[0, 1:] + tr[1, 1:]), rtol=1e-15)


def test_constant_track_equals_constant_phi(net32):
    phi = synth.one_cell()[0]
    x0 = synth.initial_abundances(net32)
    t_end = 1e5 * synth.YEAR
    ref = bdf.solve_cell(net32, phi, x0, 0.0, t_end, 1e-4, 1e-20)
    for tr in (np.concatenate([[0.0], phi])[None, :],
               np.array([np.concatenate([[0.0], phi]), np.concatenate([[t_end], phi])])):
        res = bdf.solve_cell_track(net32, tr, x0, 0.0, t_end, 1e-4, 1e-20)
        np.testing.assert_array_equal(res.x, ref.x)
        assert res.stats == ref.stats


def test_linear_zeta_decay_closed_form():
    alpha = 50.0
    net = tiny(2, [(synth.COSMIC_RAY, (0,), (1,), alpha, 0, 0)])
    za, zb = 1e-17, 5e-17
    t1 = 4.0 / (alpha * 0.5 * (za + zb))
    tr = np.array([[0.0, 1e4, 20.0, 0.5, 1.0, za], [t1, 1e4, 20.0, 0.5, 1.0, zb]])
    a = 1e-3
    res = bdf.solve_cell_track(net, tr, np.array([a, 1e-20]), 0.0, t1, 1e-10, 1e-30)
    assert res.x[0] == pytest.approx(a * np.exp(-alpha * (za + zb) * t1 / 2), rel=1e-7)
    # the constant-phi solve at either end value is far off: the track is used
    const = bdf.solve_cell(net, tr[0, 1:], np.array([a, 1e-20]), 0.0, t1, 1e-10, 1e-30)
    assert abs(const.x[0] / res.x[0] - 1) > 0.5


def test_density_track_leaves_one_body_network_unchanged():
    net = tiny(3, [(synth.COSMIC_RAY, (0,), (1,), 50.0, 0, 0), (synth.PHOTO, (1,), (2,), 1e-10, 0, 1.5)])
    x0 = np.array([1e-3, 1e-20, 1e-20])
    t1 = 1e11
    phi = np.array([1e3, 20.0, 0.5, 1.0, 1.3e-17])
    tr = np.array([np.concatenate([[0.0], phi]), np.concatenate([[t1], phi])])
    tr[1, 1] = 1e6  # n_H x 1000 over the interval
    ref = bdf.solve_cell(net, phi, x0, 0.0, t1, 1e-8, 1e-30)
    res = bdf.solve_cell_track(net, tr, x0, 0.0, t1, 1e-8, 1e-30)
    np.testing.assert_array_equal(res.x, ref.x)
