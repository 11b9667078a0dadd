"""The seeded generator draws balanced, covered, reproducible networks."""
import numpy as np
import pytest

from paper_2511_10558_gb300 import synth


@pytest.mark.parametrize("S,R", [(32, 200), (150, 1500)])
def test_balanced_and_covered(S, R):
    net = synth.make_network(S, R)
    assert net.n_species == S and net.n_reactions == R
    key = np.hstack([net.composition, net.charge[:, None]])
    sigs = set()
    for j in range(R):
        rc = [a for a in net.reac[j] if a >= 0]
        pr = [p for p in net.prod[j] if p >= 0]
        assert 1 <= len(rc) <= 2 and 1 <= len(pr) <= 4
        assert (net.rtype[j] == synth.TWO_BODY) == (len(rc) == 2)
        np.testing.assert_array_equal(key[rc].sum(0), key[pr].sum(0))
        assert sorted(rc) != sorted(pr)
        sig = (int(net.rtype[j]), tuple(sorted(rc)), tuple(sorted(pr)))
        assert sig not in sigs
        sigs.add(sig)
    reactant = np.zeros(S, bool)
    product = np.zeros(S, bool)
    for j in range(R):
        reactant[[a for a in net.reac[j] if a >= 0]] = True
        product[[p for p in net.prod[j] if p >= 0]] = True
    assert reactant.all() and product.all()
    counts = np.bincount(net.rtype, minlength=3)
    assert counts[0] == round(0.7 * R) and counts[1] == round(0.15 * R)
    # species are unique (composition, charge) pairs and the electron is species 0
    assert len({tuple(k) for k in key}) == S
    assert net.names[0] == "e-" and net.charge[0] == -1 and key[0, :5].sum() == 0


def test_parameter_ranges(net150):
    tb = net150.rtype == synth.TWO_BODY
    cr = net150.rtype == synth.COSMIC_RAY
    ph = net150.rtype == synth.PHOTO
    assert np.all((net150.alpha[tb] >= 1e-12) & (net150.alpha[tb] <= 1e-9))
    assert np.all(np.abs(net150.beta[tb]) <= 1)
    assert np.all((net150.gamma[tb] >= 0) & (net150.gamma[tb] <= 500))
    assert 0.35 < np.mean(net150.gamma[tb] == 0) < 0.65
    assert np.all((net150.alpha[cr] >= 1) & (net150.alpha[cr] <= 1e3))
    assert np.all((net150.alpha[ph] >= 1e-11) & (net150.alpha[ph] <= 1e-9))
    assert np.all((net150.gamma[ph] >= 1) & (net150.gamma[ph] <= 3))


def test_reproducible():
    a = synth.make_network(32, 200)
    b = synth.make_network(32, 200)
    np.testing.assert_array_equal(a.reac, b.reac)
    np.testing.assert_array_equal(a.alpha, b.alpha)
    c = synth.cells(64)
    assert np.all((c[:, 0] >= 1e2) & (c[:, 0] <= 1e6))
    assert np.all((c[:, 1] >= 10) & (c[:, 1] <= 300))
    assert np.all((c[:, 2] >= 0) & (c[:, 2] <= 20))
    np.testing.assert_array_equal(c, synth.cells(64))


def test_initial_abundances(net32):
    x = synth.initial_abundances(net32)
    assert x[net32.index("H2")] == 0.5 and x[net32.index("e-")] == x[net32.index("C+")]
    assert np.sum(x == 1e-20) == net32.n_species - 6


def test_tracks_recipe():
    phi = synth.cells(5)
    t_end = 1e6 * synth.YEAR
    tr = synth.tracks(phi, t_end)
    assert tr.shape == (5, 4, 6)
    assert np.all(np.diff(tr[:, :, 0], axis=1) > 0) and tr[0, -1, 0] == t_end
    np.testing.assert_allclose(tr[:, 0, 1:], phi)                       # starts at the cell's phi
    np.testing.assert_allclose(tr[:, -1, 1], 10.0 * phi[:, 0])           # n_H x10
    np.testing.assert_allclose(tr[:, -1, 2], 1.5 * phi[:, 1])            # T x1.5
    np.testing.assert_allclose(tr[:, -1, 3], phi[:, 2] + 5.0)            # A_V + 5 mag
    np.testing.assert_array_equal(tr[:, :, 4:], np.repeat(phi[:, None, 3:], 4, axis=1))


def test_cr_photo_share_leaves_the_rest_unchanged():
    base = synth.make_network(150, 1500)
    net = synth.make_network(150, 1500, cr_photo_frac=0.3)
    crp = net.rtype == synth.CR_PHOTO
    assert crp.sum() == round(0.3 * (base.rtype == synth.COSMIC_RAY).sum())
    assert np.all(base.rtype[crp] == synth.COSMIC_RAY)
    np.testing.assert_array_equal(net.reac, base.reac)
    np.testing.assert_array_equal(net.prod, base.prod)
    for f in ("alpha", "beta", "gamma"):
        np.testing.assert_array_equal(getattr(net, f)[~crp], getattr(base, f)[~crp])
    assert np.all((net.alpha[crp] >= 0.5) & (net.alpha[crp] <= 2.0))
    assert np.all((net.gamma[crp] >= 100) & (net.gamma[crp] <= 5000))
    assert np.all((net.beta[crp] >= 0) & (net.beta[crp] <= 1))
    assert net.albedo == 0.5 and base.albedo == 0.0
