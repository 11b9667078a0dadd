"""Hand-built tiny networks for closed-form tests."""
import numpy as np

from paper_2511_10558_gb300 import synth


def tiny(n_species, reactions, names=None):
    """reactions: list of (type, (reactants), (products), alpha, beta, gamma)."""
    R = len(reactions)
    reac = -np.ones((R, 2), dtype=np.int32)
    prod = -np.ones((R, 4), dtype=np.int32)
    rtype = np.zeros(R, dtype=np.int32)
    a = np.zeros(R)
    b = np.zeros(R)
    g = np.zeros(R)
    for j, (rt, rc, pr, al, be, ga) in enumerate(reactions):
        rtype[j] = rt
        reac[j, :len(rc)] = rc
        prod[j, :len(pr)] = pr
        a[j], b[j], g[j] = al, be, ga
    names = names or [f"X{i}" for i in range(n_species)]
    comp = np.zeros((n_species, 5), dtype=np.int32)
    charge = np.zeros(n_species, dtype=np.int32)
    return synth.Network(names, comp, charge, rtype, reac, prod, a, b, g)
