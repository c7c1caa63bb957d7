"""Seeded synthetic inputs shaped like the workloads of arXiv 2303.13632.

This module draws random numbers and lays out shell tables and quartet lists.
It contains none of the integral, Rys or compression arithmetic, so both the CUDA
path and the CPU oracle may use it.

Recipes (the seed of workload k is 2303_13632 + k):
  * one class, primitive:  centres uniform in [-3, 3]^3 bohr, exponents log-uniform in
    [0.1, 10], unit coefficients, contraction degree 1;
  * class sweep: the same distributions, quartets of each class drawn from a pool of
    shells per angular momentum, round(2^26 / n_ERIQ) quartets per class;
  * lattice (Sec. IV-A): 32 sites on a 4 x 4 x 2 cubic lattice with 1 Angstrom spacing,
    one primitive s, p, d and f shell per site with exponent 1.5, all site quartets.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

SEED_BASE = 2303_13632
BOHR_PER_ANGSTROM = 1.8897261246257702


@dataclass
class ShellSet:
    centers: np.ndarray  # [n, 3] float64, bohr
    L: np.ndarray        # [n] int32
    nprim: np.ndarray    # [n] int32
    pofs: np.ndarray     # [n] int64, offset of the shell's first primitive
    exps: np.ndarray     # [total prims] float64
    coefs: np.ndarray    # [total prims] float64

    @property
    def n(self) -> int:
        return len(self.L)


def make_shellset(centers, L, exps_list, coefs_list) -> ShellSet:
    nprim = np.array([len(e) for e in exps_list], dtype=np.int32)
    pofs = np.zeros(len(nprim), dtype=np.int64)
    if len(nprim) > 1:
        pofs[1:] = np.cumsum(nprim)[:-1]
    exps = np.concatenate([np.asarray(e, dtype=np.float64) for e in exps_list]) if len(nprim) else np.zeros(0)
    coefs = np.concatenate([np.asarray(c, dtype=np.float64) for c in coefs_list]) if len(nprim) else np.zeros(0)
    return ShellSet(np.ascontiguousarray(centers, dtype=np.float64).reshape(-1, 3),
                    np.asarray(L, dtype=np.int32), nprim, pofs, exps, coefs)


def rng_for(k: int) -> np.random.Generator:
    return np.random.default_rng(SEED_BASE + k)


def class_id(La: int, Lb: int, Lc: int, Ld: int) -> int:
    """Class id: ((La*4 + Lb)*4 + Lc)*4 + Ld (0..255) when every L <= 3, else
    256 + ((La*5 + Lb)*5 + Lc)*5 + Ld (classes with a g shell)."""
    if max(La, Lb, Lc, Ld) <= 3:
        return ((La * 4 + Lb) * 4 + Lc) * 4 + Ld
    return 256 + ((La * 5 + Lb) * 5 + Lc) * 5 + Ld


def class_of_id(c: int):
    if c < 256:
        return (c >> 6) & 3, (c >> 4) & 3, (c >> 2) & 3, c & 3
    r = c - 256
    return r // 125, (r // 25) % 5, (r // 5) % 5, r % 5


def g_class_ids():
    """Ids of the 369 classes with a g shell, ascending."""
    return [class_id(a, b, c, d) for a in range(5) for b in range(5) for c in range(5) for d in range(5)
            if 4 in (a, b, c, d)]


def shell_size(L: int) -> int:
    return (L + 1) * (L + 2) // 2


def quartet_size(La, Lb, Lc, Ld) -> int:
    return shell_size(La) * shell_size(Lb) * shell_size(Lc) * shell_size(Ld)


def random_primitive_pool(rng, n_per_L: int, Ls=(0, 1, 2, 3), box: float = 3.0,
                          alpha_lo: float = 0.1, alpha_hi: float = 10.0, nprim: int = 1,
                          coef_range=None) -> ShellSet:
    """n_per_L shells for each L in Ls; ids of angular momentum Ls[i] are
    [i*n_per_L, (i+1)*n_per_L).  Centres uniform in [-box, box]^3, exponents log-uniform."""
    n = n_per_L * len(Ls)
    centers = rng.uniform(-box, box, size=(n, 3))
    L = np.repeat(np.asarray(Ls, dtype=np.int32), n_per_L)
    exps = np.exp(rng.uniform(np.log(alpha_lo), np.log(alpha_hi), size=(n, nprim)))
    if coef_range is None:
        coefs = np.ones((n, nprim))
    else:
        coefs = rng.uniform(coef_range[0], coef_range[1], size=(n, nprim))
    return make_shellset(centers, L, list(exps), list(coefs))


def random_class_quartets(rng, cls, n_quartets: int, n_per_L: int, Ls=(0, 1, 2, 3)) -> np.ndarray:
    """n_quartets rows of shell ids of class cls = (La, Lb, Lc, Ld) drawn from a pool
    built by random_primitive_pool with the same n_per_L and Ls."""
    q = np.empty((n_quartets, 4), dtype=np.int32)
    for x, Lx in enumerate(cls):
        base = list(Ls).index(Lx) * n_per_L
        q[:, x] = base + rng.integers(0, n_per_L, size=n_quartets)
    return q


def one_class_workload(cls=(1, 1, 1, 1), n_quartets: int = 10_000, seed_k: int = 1):
    """Primitive quartets of one class, four fresh shells per quartet
    (centres U[-3,3]^3 bohr, exponents log-U[0.1,10], unit coefficients)."""
    rng = rng_for(seed_k)
    n = 4 * n_quartets
    centers = rng.uniform(-3.0, 3.0, size=(n, 3))
    L = np.tile(np.asarray(cls, dtype=np.int32), n_quartets)
    exps = np.exp(rng.uniform(np.log(0.1), np.log(10.0), size=n))
    shells = make_shellset(centers, L, list(exps.reshape(-1, 1)), list(np.ones((n, 1))))
    quartets = np.arange(n, dtype=np.int32).reshape(n_quartets, 4)
    return shells, quartets


def sweep_quartet_count(cls, target_eris: int = 1 << 26) -> int:
    return max(1, int(round(target_eris / quartet_size(*cls))))


SWEEP_POOL_PER_L = 4096


def sweep_pool(seed_k: int = 2) -> ShellSet:
    """Shell pool of the 256-class sweep: SWEEP_POOL_PER_L primitive shells per L."""
    return random_primitive_pool(rng_for(seed_k), SWEEP_POOL_PER_L)


def sweep_quartets_device(torch, counts, device, seed_k: int = 2, n_per_L: int = SWEEP_POOL_PER_L):
    """Class-major int32 quartet table [sum(counts), 4] of the sweep, drawn on the device with
    a seeded torch generator (class c gets counts[c] rows of shell ids of its four angular
    momenta from the pool of sweep_pool); returns (table, first row of each class)."""
    n_total = sum(counts[c] for c in range(256))
    q = torch.empty((n_total, 4), dtype=torch.int32, device=device)
    gen = torch.Generator(device=device)
    gen.manual_seed(SEED_BASE + seed_k)
    first = {}
    pos = 0
    for c in range(256):
        cls = class_of_id(c)
        n = counts[c]
        first[c] = pos
        for x in range(4):
            q[pos:pos + n, x] = (torch.randint(0, n_per_L, (n,), generator=gen, device=device,
                                               dtype=torch.int32) + cls[x] * n_per_L)
        pos += n
    return q, first


def lattice_sites() -> np.ndarray:
    """32 sites of the 4 x 4 x 2 cubic lattice of Sec. IV-A, spacing 1 Angstrom, in bohr."""
    g = np.array([(i, j, k) for i in range(4) for j in range(4) for k in range(2)], dtype=np.float64)
    return g * BOHR_PER_ANGSTROM


def lattice_shells(alpha: float = 1.5) -> ShellSet:
    """One primitive s, p, d, f shell per site (ids: site*4 + L), exponent 1.5, coefficient 1."""
    sites = lattice_sites()
    centers = np.repeat(sites, 4, axis=0)
    L = np.tile(np.arange(4, dtype=np.int32), len(sites))
    n = len(L)
    return make_shellset(centers, L, [[alpha]] * n, [[1.0]] * n)


def lattice_class_quartets(cls, sites: np.ndarray | None = None) -> np.ndarray:
    """All site quartets (32^4) of class cls over lattice_shells() ids."""
    ns = 32 if sites is None else len(sites)
    s = np.arange(ns, dtype=np.int32)
    a, b, c, d = np.meshgrid(s, s, s, s, indexing="ij")
    q = np.stack([a.ravel() * 4 + cls[0], b.ravel() * 4 + cls[1],
                  c.ravel() * 4 + cls[2], d.ravel() * 4 + cls[3]], axis=1)
    return q.astype(np.int32)


def random_contracted_pool(rng, n_per_L: int, K: int, Ls=(1, 2), box: float = 3.0) -> ShellSet:
    """Contracted shells of degree K: even-tempered exponents alpha0 * 3^k with alpha0
    log-uniform so the largest stays below 50, coefficients U[0.1, 1]."""
    n = n_per_L * len(Ls)
    centers = rng.uniform(-box, box, size=(n, 3))
    L = np.repeat(np.asarray(Ls, dtype=np.int32), n_per_L)
    hi = 50.0 / 3.0 ** (K - 1)
    a0 = np.exp(rng.uniform(np.log(0.05), np.log(max(hi, 0.051)), size=n))
    exps = a0[:, None] * 3.0 ** np.arange(K)[None, :]
    coefs = rng.uniform(0.1, 1.0, size=(n, K))
    return make_shellset(centers, L, list(exps), list(coefs))


def molecule_basis(n_atoms: int = 200, box: float = 20.0, min_sep: float = 1.8, seed_k: int = 4,
                   shells_per_atom=(0, 0, 1, 1, 2, 3), kmax: int = 6) -> ShellSet:
    """Atoms at random positions in a cubic box with a minimum separation; every atom carries
    the shells `shells_per_atom` (s, s, p, p, d, f), each contracted over K ~ U{1..kmax}
    even-tempered primitives alpha0 * 3^k with alpha0 log-uniform in [0.05, 50 / 3^(K-1)]
    (so exponents span 0.05..50) and coefficients U[0.1, 1]."""
    rng = rng_for(seed_k)
    atoms = []
    while len(atoms) < n_atoms:
        p = rng.uniform(0.0, box, size=3)
        if all(np.linalg.norm(p - a) >= min_sep for a in atoms):
            atoms.append(p)
    centers, L, exps, coefs = [], [], [], []
    for a in atoms:
        for l in shells_per_atom:
            K = int(rng.integers(1, kmax + 1))
            hi = 50.0 / 3.0 ** (K - 1)
            a0 = np.exp(rng.uniform(np.log(0.05), np.log(hi)))
            centers.append(a)
            L.append(l)
            exps.append(a0 * 3.0 ** np.arange(K))
            coefs.append(rng.uniform(0.1, 1.0, size=K))
    return make_shellset(np.array(centers), L, exps, coefs)
