"""Seeded synthetic inputs: reaction networks, cell parameters, initial abundances.

This module only draws inputs. It holds none of the method's arithmetic (no rate
coefficient, right-hand side, Jacobian or integrator step), and it is the one
module that both the CPU oracle's tests and the CUDA path's callers share.

The paper's own networks (App. B.1: an atomic network of 31-34 species and 380
reactions; App. B.2: a molecular network of 161 species and 2227 reactions)
come from the UMIST / UCLCHEM databases, which are not available. The networks
drawn here stand in for them: element- and charge-balanced, built from the same
three rate classes the method uses (two-body Kooij-Arrhenius, Sec. 2;
cosmic-ray ionisation, Sec. 2; photo-reactions, App. B.1), with sizes 32/200,
150/1500 and 500/6000 species/reactions.

Recipe (all draws from ``numpy.random.Generator(PCG64(seed))``):

* Species. Always e-, H, H+, H2, H2+, H3+, He, He+, C, C+, N, N+, O, O+.
  The rest are unique (composition, charge) pairs with H 0-4, C 0-3, N 0-2,
  O 0-2 atoms (no He), at least two atoms, and charge 0 / +1 / -1 with
  probability 0.60 / 0.35 / 0.05. Composition order is (H, He, C, N, O).
* Reactions. A reaction is balanced when the summed composition and the summed
  charge of its reactants equal those of its products. Classes: 70 % two-body
  A + B -> C (+ D); 15 % cosmic-ray X -> X+ + e- or X -> C + D; 15 % photo
  with the same product forms. No duplicates; the product set never equals
  the reactant set. First every species gets one destruction channel (it is a
  reactant) and one formation channel (it is a product), then each class is
  filled with random balanced candidates.
* Parameters. Two-body: alpha log-uniform [1e-12, 1e-9] cm^3 s^-1,
  beta U[-1, 1], gamma = 0 with probability 0.5 else U[0, 500] K.
  Cosmic-ray: alpha U[1, 1e3]. Photo: alpha log-uniform [1e-11, 1e-9] s^-1,
  gamma U[1, 3]. beta = gamma = 0 where unused.
* Optional (``cr_photo_frac``): a share of the cosmic-ray reactions becomes
  the cosmic-ray-induced photo form of App. B.1 (see make_network).
* Cells. One cell: n_H = 1e4 cm^-3, T = 20 K, A_V = 5, G0 = 1,
  zeta = 1.3e-17 s^-1 (the galactic value zeta_0 of Sec. 4). Batches:
  n_H log-uniform [1e2, 1e6], T U[10, 300] K, A_V U[0, 20], G0 = 1,
  zeta = 1.3e-17.
* Initial abundances per n_H: H2 0.5, He 0.1, C+ 1e-4, O 3e-4, N 7.5e-5,
  e- = C+, every other species 1e-20.
"""
from __future__ import annotations

import dataclasses
import numpy as np

# Reaction classes (the integer codes are part of the C ABI, see include/carbox.h).
TWO_BODY = 0
COSMIC_RAY = 1
PHOTO = 2
CR_PHOTO = 3   # secondary photons induced by cosmic rays (App. B.1)

ELEMENTS = ("H", "He", "C", "N", "O")
ZETA0 = 1.3e-17          # s^-1, galactic cosmic-ray ionisation rate (Sec. 4)
YEAR = 3.15576e7          # s, Julian year

_FIXED = [
    ("e-", (0, 0, 0, 0, 0), -1),
    ("H", (1, 0, 0, 0, 0), 0),
    ("H+", (1, 0, 0, 0, 0), 1),
    ("H2", (2, 0, 0, 0, 0), 0),
    ("H2+", (2, 0, 0, 0, 0), 1),
    ("H3+", (3, 0, 0, 0, 0), 1),
    ("He", (0, 1, 0, 0, 0), 0),
    ("He+", (0, 1, 0, 0, 0), 1),
    ("C", (0, 0, 1, 0, 0), 0),
    ("C+", (0, 0, 1, 0, 0), 1),
    ("N", (0, 0, 0, 1, 0), 0),
    ("N+", (0, 0, 0, 1, 0), 1),
    ("O", (0, 0, 0, 0, 1), 0),
    ("O+", (0, 0, 0, 0, 1), 1),
]


@dataclasses.dataclass
class Network:
    """A species list and a reaction list, as plain arrays.

    composition: int32 [S, 5]; charge: int32 [S]
    rtype: int32 [R]; reac: int32 [R, 2] (-1 = absent); prod: int32 [R, 4]
    (-1 = absent); alpha, beta, gamma: float64 [R].
    """
    names: list
    composition: np.ndarray
    charge: np.ndarray
    rtype: np.ndarray
    reac: np.ndarray
    prod: np.ndarray
    alpha: np.ndarray
    beta: np.ndarray
    gamma: np.ndarray
    albedo: float = 0.0   # dust grain albedo omega of the CR-photo form (App. B.1)

    @property
    def n_species(self) -> int:
        return len(self.names)

    @property
    def n_reactions(self) -> int:
        return len(self.rtype)

    def index(self, name: str) -> int:
        return self.names.index(name)


def _formula(comp, charge) -> str:
    s = "".join(f"{el}{'' if n == 1 else n}" for el, n in zip(ELEMENTS, comp) if n > 0)
    return s + {0: "", 1: "+", -1: "-"}[charge]


def _key(comp, charge):
    return tuple(int(c) for c in comp) + (int(charge),)


def _add_keys(a, b):
    return tuple(x + y for x, y in zip(a, b))


def _sub_keys(a, b):
    return tuple(x - y for x, y in zip(a, b))


def make_network(n_species: int, n_reactions: int, seed: int | None = None,
                 cr_photo_frac: float = 0.0) -> Network:
    """Draw a balanced synthetic network of the given size (seed default 1000 + S).

    cr_photo_frac > 0 turns that fraction of the cosmic-ray reactions into
    reactions by secondary photons induced by cosmic rays (App. B.1), drawn
    from a separate stream so that the rest of the network is unchanged:
    alpha U[0.5, 2], beta = 0 with probability 0.5 else U[0, 1], efficiency
    E (the gamma field) U[100, 5000], and a grain albedo omega = 0.5.
    """
    net = _draw_network(n_species, n_reactions, seed)
    if cr_photo_frac > 0.0:
        rng = np.random.default_rng((1000 + n_species if seed is None else seed) + 77)
        cr = np.flatnonzero(net.rtype == COSMIC_RAY)
        pick = np.sort(rng.choice(cr, size=int(round(cr_photo_frac * len(cr))), replace=False))
        for j in pick:
            net.rtype[j] = CR_PHOTO
            net.alpha[j] = rng.uniform(0.5, 2.0)
            net.beta[j] = 0.0 if rng.random() < 0.5 else rng.uniform(0.0, 1.0)
            net.gamma[j] = rng.uniform(100.0, 5000.0)
        net.albedo = 0.5
    return net


def _draw_network(n_species: int, n_reactions: int, seed: int | None) -> Network:
    if seed is None:
        seed = 1000 + n_species
    if n_species < len(_FIXED):
        raise ValueError(f"need at least {len(_FIXED)} species")
    rng = np.random.default_rng(seed)

    # ---- species: grown by fragments, so every species has a balanced
    # route to two species already present (keeps the chemistry connected)
    species = list(_FIXED)
    keys = [_key(c, q) for _, c, q in species]
    seen = set(keys)
    pair_by_key = {}

    def add_pairs(i):
        for a in range(i + 1):
            pair_by_key.setdefault(_add_keys(keys[a], keys[i]), []).append((a, i))

    for i in range(len(keys)):
        add_pairs(i)
    cand = []
    for h in range(5):
        for c in range(4):
            for n in range(3):
                for o in range(3):
                    if h + c + n + o >= 2:
                        cand.append((h, 0, c, n, o))
    guard = 0
    while len(species) < n_species:
        guard += 1
        if guard > 200000:
            raise ValueError("too many species for the composition space")
        comp = cand[rng.integers(len(cand))]
        u = rng.random()
        q = 0 if u < 0.60 else (1 if u < 0.95 else -1)
        k = _key(comp, q)
        if k in seen or k not in pair_by_key:
            continue
        seen.add(k)
        species.append((_formula(comp, q), comp, q))
        keys.append(k)
        add_pairs(len(keys) - 1)
    S = n_species
    names = [sp[0] for sp in species]
    by_key = {}
    for i, k in enumerate(keys):
        by_key.setdefault(k, []).append(i)

    def products_of(key):
        """All product sets (1 or 2 species) with the given summed key."""
        out = [(c,) for c in by_key.get(key, [])]
        out += list(pair_by_key.get(key, []))
        return out

    reactions = []          # (type, reactants tuple, products tuple)
    signature = set()

    def add(rt, reac, prod):
        reac = tuple(sorted(reac))
        prod = tuple(sorted(prod))
        if reac == prod:
            return False
        sig = (rt, reac, prod)
        if sig in signature:
            return False
        signature.add(sig)
        reactions.append(sig)
        return True

    n_two = int(round(0.70 * n_reactions))
    n_cr = int(round(0.15 * n_reactions))
    n_ph = n_reactions - n_two - n_cr
    electron = 0

    def count(rt):
        return sum(1 for r in reactions if r[0] == rt)

    def random_unimolecular(x, rt):
        if x == electron:
            return False
        opts = products_of(keys[x])
        opts = [p for p in opts if p != (x,)]
        if not opts:
            return False
        return add(rt, (x,), opts[rng.integers(len(opts))])

    def random_two_body_with(a):
        for _ in range(200):
            b = int(rng.integers(S))
            opts = [p for p in products_of(_add_keys(keys[a], keys[b]))
                    if tuple(sorted(p)) != tuple(sorted((a, b)))]
            if opts and add(TWO_BODY, (a, b), opts[rng.integers(len(opts))]):
                return True
        return False

    def destruction_options(s):
        opts = []
        if s != electron:
            for p in products_of(keys[s]):
                if p != (s,):
                    opts.append(((s,), p))
        for b in range(S):
            for p in products_of(_add_keys(keys[s], keys[b])):
                if tuple(sorted(p)) != tuple(sorted((s, b))):
                    opts.append(((s, b), p))
        return opts

    def formation_options(s):
        opts = []
        for d in range(-1, S):
            need = keys[s] if d < 0 else _add_keys(keys[s], keys[d])
            prod = (s,) if d < 0 else (s, d)
            for pr in pair_by_key.get(need, []):
                if tuple(sorted(pr)) != tuple(sorted(prod)):
                    opts.append((pr, prod))
            for x in by_key.get(need, []):
                if x != electron and (x,) != prod:
                    opts.append(((x,), prod))
        return opts

    def add_option(opts):
        while opts:
            i = int(rng.integers(len(opts)))
            reac, prod = opts.pop(i)
            if len(reac) == 2:
                rt = TWO_BODY
            else:
                rt = COSMIC_RAY if rng.random() < 0.5 else PHOTO
            if add(rt, reac, prod):
                return True
        return False

    # coverage: one destruction and one formation channel per species
    for s in range(S):
        if not any(s in r[1] for r in reactions):
            if not add_option(destruction_options(s)):
                raise RuntimeError(f"no destruction channel for {names[s]}")
        if not any(s in r[2] for r in reactions):
            if not add_option(formation_options(s)):
                raise RuntimeError(f"no formation channel for {names[s]}")
    if count(TWO_BODY) > n_two or count(COSMIC_RAY) > n_cr or count(PHOTO) > n_ph:
        raise RuntimeError("network too small for its coverage reactions")
    # fill each class
    guard = 0
    while count(COSMIC_RAY) < n_cr or count(PHOTO) < n_ph:
        guard += 1
        if guard > 100000:
            raise RuntimeError("cannot draw enough unimolecular reactions")
        x = int(rng.integers(S))
        if count(COSMIC_RAY) < n_cr:
            random_unimolecular(x, COSMIC_RAY)
        else:
            random_unimolecular(x, PHOTO)
    guard = 0
    while count(TWO_BODY) < n_two:
        guard += 1
        if guard > 100000:
            raise RuntimeError("cannot draw enough two-body reactions")
        random_two_body_with(int(rng.integers(S)))

    # stable order: by class, then in draw order
    reactions.sort(key=lambda r: r[0])
    R = len(reactions)
    rtype = np.array([r[0] for r in reactions], dtype=np.int32)
    reac = -np.ones((R, 2), dtype=np.int32)
    prod = -np.ones((R, 4), dtype=np.int32)
    for j, (_, rc, pr) in enumerate(reactions):
        reac[j, :len(rc)] = rc
        prod[j, :len(pr)] = pr
    alpha = np.zeros(R)
    beta = np.zeros(R)
    gamma = np.zeros(R)
    for j in range(R):
        if rtype[j] == TWO_BODY:
            alpha[j] = 10.0 ** rng.uniform(-12.0, -9.0)
            beta[j] = rng.uniform(-1.0, 1.0)
            gamma[j] = 0.0 if rng.random() < 0.5 else rng.uniform(0.0, 500.0)
        elif rtype[j] == COSMIC_RAY:
            alpha[j] = rng.uniform(1.0, 1e3)
        else:
            alpha[j] = 10.0 ** rng.uniform(-11.0, -9.0)
            gamma[j] = rng.uniform(1.0, 3.0)
    comp = np.array([s[1] for s in species], dtype=np.int32)
    charge = np.array([s[2] for s in species], dtype=np.int32)
    return Network(names, comp, charge, rtype, reac, prod, alpha, beta, gamma)


# Cell parameter record, in the C ABI's field order: n_H, T, A_V, G0, zeta.
PARAM_FIELDS = ("n_H", "T", "A_V", "G0", "zeta")


def one_cell() -> np.ndarray:
    """The single reference cell: n_H = 1e4, T = 20 K, A_V = 5, G0 = 1, zeta_0."""
    return np.array([[1e4, 20.0, 5.0, 1.0, ZETA0]])


def cells(n_cells: int, seed: int = 7) -> np.ndarray:
    """A seeded batch of cells, float64 [C, 5] in PARAM_FIELDS order."""
    rng = np.random.default_rng(seed)
    out = np.empty((n_cells, 5))
    out[:, 0] = 10.0 ** rng.uniform(2.0, 6.0, n_cells)
    out[:, 1] = rng.uniform(10.0, 300.0, n_cells)
    out[:, 2] = rng.uniform(0.0, 20.0, n_cells)
    out[:, 3] = 1.0
    out[:, 4] = ZETA0
    return out


def initial_abundances(net: Network) -> np.ndarray:
    """x0 per n_H, float64 [S]."""
    x = np.full(net.n_species, 1e-20)
    x[net.index("H2")] = 0.5
    x[net.index("He")] = 0.1
    x[net.index("C+")] = 1e-4
    x[net.index("O")] = 3e-4
    x[net.index("N")] = 7.5e-5
    x[net.index("e-")] = 1e-4
    return x


def tracks(phi: np.ndarray, t_end: float, n_knots: int = 4) -> np.ndarray:
    """Environment tracks [C, K, 6] (t, n_H, T, A_V, G0, zeta) for the cells phi [C, 5]:
    a collapse with warming over [0, t_end] -- n_H rising tenfold, T by half again,
    A_V by 5 mag -- at K knots equally spaced in time (G0 and zeta held). The knot
    values follow s = (k / (K-1)) on a geometric path for n_H, linear for T and A_V."""
    phi = np.asarray(phi, dtype=float)
    C = phi.shape[0]
    out = np.empty((C, n_knots, 6))
    for k in range(n_knots):
        s = k / (n_knots - 1) if n_knots > 1 else 0.0
        out[:, k, 0] = s * t_end
        out[:, k, 1] = phi[:, 0] * 10.0 ** s
        out[:, k, 2] = phi[:, 1] * (1.0 + 0.5 * s)
        out[:, k, 3] = phi[:, 2] + 5.0 * s
        out[:, k, 4] = phi[:, 3]
        out[:, k, 5] = phi[:, 4]
    return out
