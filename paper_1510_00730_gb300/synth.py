"""Seeded synthetic workloads for the multideterminant hot path.

This module only draws inputs: a one-nucleus "atom" with a contracted
Cartesian-Gaussian basis, a random orthonormal AO->MO matrix, a selected-CI-like
expansion over bit-string determinants, and walker positions. It holds none of
the method's arithmetic (no determinants, no orbital evaluation), so both the
CUDA path and the FP64 oracle can take their inputs from it.

Recipe (stand-in for the chlorine CIPSI wavefunctions of Sec. 4, which are not
available):

* nucleus at the origin with charge Z;
* shells of angular momentum l=0..3, three primitives each, exponents
  log-uniform over [alpha_min, alpha_max], contraction weights U(0.2, 1)
  multiplied by the primitive normalisation of the x^l component;
* MO coefficients: Q of the QR factorisation of a Gaussian K x M matrix;
* spin determinants: the aufbau determinant plus distinct excitations of degree
  1..k_max from it; degree shares follow the excitation histogram of the
  10^6-determinant expansion (Table 4) renormalised to the allowed degrees;
  holes uniform over occupied orbitals, particles geometric (p=0.1) over the
  virtual orbitals; the number of unique determinants per spin follows
  0.9 * N_det^0.6 (the fitted exponent of Sec. 4);
* products (i, j) drawn without replacement with weight 1/((i+1)(j+1)), every
  unique spin determinant used at least once, (0, 0) first;
* coefficients: power law |c_r| = r^-1.5 in rank r (or log-normal magnitudes
  sorted descending), random signs;
* walkers: electron radii Exp(scale 1 bohr), isotropic directions.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Degree histograms of the 10^6-determinant wavefunction (Table 4), degrees 0..8.
_TABLE4_UP = [1, 90, 1603, 7811, 8581, 2090, 77, 0, 0]
_TABLE4_DN = [1, 88, 1520, 6507, 5071, 579, 0, 0, 0]


@dataclass
class Workload:
    name: str
    n_up: int
    n_dn: int
    Z: np.ndarray             # [n_nuc] nuclear charges
    nuc_xyz: np.ndarray       # [n_nuc, 3]
    shell_l: np.ndarray       # [n_shell] int32
    shell_center: np.ndarray  # [n_shell] int32
    shell_nprim: np.ndarray   # [n_shell] int32
    alpha: np.ndarray         # [sum nprim] primitive exponents
    coef: np.ndarray          # [sum nprim] contraction coefficients (normalisation included)
    mo_coef: np.ndarray       # [n_ao, n_mo] (C order; column m = MO m)
    det_up: np.ndarray        # [n_det, n_int] uint64, bit (m) set <=> MO m+1 occupied
    det_dn: np.ndarray        # [n_det, n_int] uint64
    ci_coef: np.ndarray       # [n_det] float64
    R: np.ndarray             # [n_walk, n_up + n_dn, 3] float64
    meta: dict = field(default_factory=dict)

    @property
    def n_elec(self) -> int:
        return self.n_up + self.n_dn

    @property
    def n_ao(self) -> int:
        return int(sum((l + 1) * (l + 2) // 2 for l in self.shell_l))

    @property
    def n_mo(self) -> int:
        return int(self.mo_coef.shape[1])

    @property
    def n_int(self) -> int:
        return int(self.det_up.shape[1])

    @property
    def n_det(self) -> int:
        return int(self.ci_coef.shape[0])

    @property
    def n_walk(self) -> int:
        return int(self.R.shape[0])


def _dfact(n: int) -> int:
    r = 1
    while n > 1:
        r *= n
        n -= 2
    return r


def make_basis(rng, shells_per_l, alpha_min, alpha_max, nprim=3):
    """Contracted Cartesian Gaussian shells on nucleus 0."""
    shell_l, nprims, alphas, coefs = [], [], [], []
    for l, count in enumerate(shells_per_l):
        for _ in range(count):
            a = np.sort(np.exp(rng.uniform(math.log(alpha_min), math.log(alpha_max), nprim)))
            d = rng.uniform(0.2, 1.0, nprim)
            norm = (2 * a / math.pi) ** 0.75 * (4 * a) ** (l / 2) / math.sqrt(_dfact(2 * l - 1))
            shell_l.append(l)
            nprims.append(nprim)
            alphas.extend(a.tolist())
            coefs.extend((d * norm).tolist())
    n = len(shell_l)
    return (np.array(shell_l, np.int32), np.zeros(n, np.int32), np.array(nprims, np.int32),
            np.array(alphas, np.float64), np.array(coefs, np.float64))


def random_orthonormal(rng, k, m):
    q, r = np.linalg.qr(rng.standard_normal((k, m)))
    return np.ascontiguousarray(q * np.sign(np.diag(r))[None, :])


def occ_to_bits(occ, n_int):
    """Occupied MO indices (0-based) -> n_int 64-bit words (bit m%64 of word m//64)."""
    words = [0] * n_int
    for m in occ:
        words[m // 64] |= 1 << (m % 64)
    return words


def _degree_shares(table, k_max):
    w = np.array(table[1:k_max + 1], np.float64)
    return w / w.sum()


def make_spin_dets(rng, n_elec, n_mo, n_unique, k_max, table):
    """Aufbau determinant followed by (n_unique - 1) distinct excitations of it.

    Returns a list of sorted occupied-orbital tuples in generation order, which
    is also the importance rank used to pair determinants."""
    ref = tuple(range(n_elec))
    virt = np.arange(n_elec, n_mo)
    shares = _degree_shares(table, k_max)
    seen = {ref}
    out = [ref]
    # geometric preference for low virtual orbitals
    pv = 0.1 * (0.9 ** np.arange(len(virt)))
    pv /= pv.sum()
    attempts = 0
    while len(out) < n_unique:
        attempts += 1
        if attempts > 200 * n_unique + 10000:
            raise RuntimeError("could not draw enough distinct determinants")
        k = int(rng.choice(np.arange(1, k_max + 1), p=shares))
        k = min(k, n_elec, len(virt))
        holes = rng.choice(n_elec, size=k, replace=False)
        parts = rng.choice(virt, size=k, replace=False, p=pv)
        occ = tuple(sorted(set(ref) - set(holes.tolist()) | set(parts.tolist())))
        if occ in seen:
            continue
        seen.add(occ)
        out.append(occ)
    # importance order: lower excitation degree first, generation order otherwise
    deg = [len(set(o) - set(ref)) for o in out]
    order = sorted(range(len(out)), key=lambda i: (deg[i], i))
    return [out[i] for i in order]


def pick_products(rng, n_a, n_b, n_det):
    """Distinct (i, j) pairs with weight 1/((i+1)(j+1)), each row and column
    used at least once, returned in importance order ((0, 0) first)."""
    if n_det > n_a * n_b:
        raise ValueError("more products than cells")
    if n_det < max(n_a, n_b):
        raise ValueError("too few products to use every spin determinant")
    ii = np.arange(n_a, dtype=np.float64)[:, None] + 1.0
    jj = np.arange(n_b, dtype=np.float64)[None, :] + 1.0
    key = rng.exponential(1.0, size=(n_a, n_b)) * ii * jj   # Efraimidis-Spirakis keys
    key[0, 0] = -1.0
    forced = np.zeros((n_a, n_b), bool)
    forced[np.arange(n_a), np.argmin(key, axis=1)] = True
    forced[np.argmin(key, axis=0), np.arange(n_b)] = True
    forced[0, 0] = True
    n_forced = int(forced.sum())
    flat = key.ravel()
    free = np.flatnonzero(~forced.ravel())
    n_rest = n_det - n_forced
    if n_rest < 0:
        raise ValueError("n_det below the coverage minimum")
    if n_rest > 0:
        part = np.argpartition(flat[free], n_rest - 1)[:n_rest]
        chosen = np.concatenate([np.flatnonzero(forced.ravel()), free[part]])
    else:
        chosen = np.flatnonzero(forced.ravel())
    chosen = chosen[np.argsort(flat[chosen], kind="stable")]
    return chosen // n_b, chosen % n_b


def make_walkers(rng, n_walk, n_elec, scale=1.0):
    r = rng.exponential(scale, size=(n_walk, n_elec))
    v = rng.standard_normal((n_walk, n_elec, 3))
    v /= np.linalg.norm(v, axis=-1, keepdims=True)
    return np.ascontiguousarray(v * r[..., None])


def make_workload(name, seed, n_up, n_dn, Z, shells_per_l, alpha_range, n_mo,
                  n_det, k_max, n_walk, coef_law="power", n_unique=None):
    rng = np.random.default_rng(seed)
    shell_l, shell_center, shell_nprim, alpha, coef = make_basis(rng, shells_per_l, *alpha_range)
    n_ao = int(sum((l + 1) * (l + 2) // 2 for l in shell_l))
    if n_mo > n_ao:
        raise ValueError("n_mo > n_ao")
    mo = random_orthonormal(rng, n_ao, n_mo)
    n_int = (n_mo + 63) // 64
    if n_unique is None:
        n_unique = (max(1, int(round(0.9 * n_det ** 0.6))),) * 2
    nu_up = min(n_unique[0], n_det)
    nu_dn = min(n_unique[1], n_det)
    ups = make_spin_dets(rng, n_up, n_mo, nu_up, k_max, _TABLE4_UP)
    dns = make_spin_dets(rng, n_dn, n_mo, nu_dn, k_max, _TABLE4_DN)
    pi, pj = pick_products(rng, len(ups), len(dns), n_det)
    if coef_law == "power":
        mag = np.arange(1, n_det + 1, dtype=np.float64) ** -1.5
    elif coef_law == "lognormal":
        mag = np.sort(np.exp(rng.normal(-4.0, 1.5, n_det)))[::-1].copy()
        mag[0] = max(mag[0], 1.0)
    else:
        raise ValueError(coef_law)
    sgn = np.where(rng.random(n_det) < 0.5, -1.0, 1.0)
    sgn[0] = 1.0
    c = mag * sgn
    up_bits = np.array([occ_to_bits(o, n_int) for o in ups], dtype=np.uint64)
    dn_bits = np.array([occ_to_bits(o, n_int) for o in dns], dtype=np.uint64)
    # present products in a shuffled order: the library must not rely on input order
    perm = rng.permutation(n_det)
    det_up = np.ascontiguousarray(up_bits[pi][perm])
    det_dn = np.ascontiguousarray(dn_bits[pj][perm])
    ci = np.ascontiguousarray(c[perm])
    R = make_walkers(rng, n_walk, n_up + n_dn)
    return Workload(name=name, n_up=n_up, n_dn=n_dn,
                    Z=np.array([float(Z)]), nuc_xyz=np.zeros((1, 3)),
                    shell_l=shell_l, shell_center=shell_center, shell_nprim=shell_nprim,
                    alpha=alpha, coef=coef, mo_coef=mo,
                    det_up=det_up, det_dn=det_dn, ci_coef=ci, R=R,
                    meta=dict(seed=seed, n_unique=(len(ups), len(dns)), k_max=k_max))


# Named workloads. Seeds are 151000730 + index.
def oxygen_like_1k(n_walk=64, seed=151000731):
    """8 electrons (4 up, 4 down), Z=8, 40 AOs (10 s, 8 p, 1 d), 20 MOs,
    1,000 determinants over ~57 unique determinants per spin, degrees 1..3,
    log-normal coefficients; 64 walkers."""
    return make_workload("oxygen_like_1k", seed, 4, 4, 8, (10, 8, 1), (0.05, 5000.0), 20,
                         1000, 3, n_walk, coef_law="lognormal")


def chlorine_like_100k(n_walk=4096, seed=151000732):
    """17 electrons (9 up, 8 down), Z=17, 110 AOs (12 s, 10 p, 8 d, 2 f), 80 MOs,
    10^5 determinants over ~900 unique determinants per spin, degrees 1..4; 4,096 walkers."""
    return make_workload("chlorine_like_100k", seed, 9, 8, 17, (12, 10, 8, 2), (0.03, 1.0e5), 80,
                         100_000, 4, n_walk)


def chlorine_like_750k(n_walk=8192, seed=151000733):
    """Same chlorine-like system with 750,000 determinants over ~3,000 unique
    determinants per spin; 8,192 walkers."""
    return make_workload("chlorine_like_750k", seed, 9, 8, 17, (12, 10, 8, 2), (0.03, 1.0e5), 80,
                         750_000, 4, n_walk)


def tiny(n_up=2, n_dn=2, n_mo=5, n_det=None, n_walk=4, seed=7, k_max=2, shells=(3, 2, 0)):
    """Small system for brute-force checks."""
    n_ao = sum(c * (l + 1) * (l + 2) // 2 for l, c in enumerate(shells))
    assert n_mo <= n_ao
    from math import comb
    nu = (comb(n_mo, n_up), comb(n_mo, n_dn))
    if n_det is None:
        n_det = nu[0] * nu[1]
    return make_workload("tiny", seed, n_up, n_dn, max(n_up + n_dn, 1), shells, (0.1, 10.0), n_mo,
                         n_det, k_max, n_walk, coef_law="lognormal", n_unique=nu)


def _shell_counts(rng, n_ao):
    """s/p/d/f shell counts whose Cartesian AOs add up to n_ao exactly."""
    while True:
        n_f = int(rng.integers(0, 1 + n_ao // 60))
        n_d = int(rng.integers(1, 1 + n_ao // 15))
        n_p = int(rng.integers(1, 1 + n_ao // 8))
        n_s = n_ao - 10 * n_f - 6 * n_d - 3 * n_p
        if n_s >= 2:
            return (n_s, n_p, n_d, n_f)


def batched_uneven(n_exp=64, seed=151000734, walkers=(256, 4096), n_det_range=(1e3, 1e6),
                   elec_range=(8, 34), ao_range=(40, 160)):
    """Independent expansions of uneven size: N_elec uniform in [8, 34] split as
    evenly as possible between the spins (up >= down), AOs uniform in [40, 160],
    N_MO = max(round(0.73 N_AO), N_up + 4), N_det log-uniform in [1e3, 1e6],
    walkers uniform in [256, 4096], degrees up to 4."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_exp):
        ne = int(rng.integers(elec_range[0], elec_range[1] + 1))
        n_up, n_dn = (ne + 1) // 2, ne // 2
        n_ao = int(rng.integers(ao_range[0], ao_range[1] + 1))
        n_mo = min(n_ao, 255, max(int(round(0.73 * n_ao)), n_up + 4))
        n_det = int(round(math.exp(rng.uniform(math.log(n_det_range[0]), math.log(n_det_range[1])))))
        n_walk = int(rng.integers(walkers[0], walkers[1] + 1))
        wl = make_workload("uneven_%02d" % i, seed * 100 + i, n_up, n_dn, ne, _shell_counts(rng, n_ao),
                           (0.03, 1.0e5), n_mo, n_det, 4, n_walk)
        out.append(wl)
    return out


def subset_products(wl, mask):
    """The same system with only the products selected by the boolean mask (e.g.
    a truncation's keep mask); walkers and orbitals are shared."""
    import dataclasses
    mask = np.asarray(mask, dtype=bool)
    return dataclasses.replace(wl, name=wl.name + "_subset", det_up=wl.det_up[mask], det_dn=wl.det_dn[mask],
                               ci_coef=wl.ci_coef[mask], meta=dict(wl.meta, subset_of=wl.name))


WORKLOADS = {
    "oxygen_like_1k": oxygen_like_1k,
    "chlorine_like_100k": chlorine_like_100k,
    "chlorine_like_750k": chlorine_like_750k,
}
