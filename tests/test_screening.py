"""Host logic of the batched workload: Schwarz screening and 8-fold unique quartets, checked
against brute-force enumeration with exact Schwarz factors from the oracle."""
import itertools

import numpy as np

import oracle
from paper_2303_13632_gb300 import screening as S, workloads as W


def schwarz_factors(shells, pairs):
    q = np.stack([pairs[:, 0], pairs[:, 1], pairs[:, 0], pairs[:, 1]], axis=1)
    vals, offs = oracle.eri_batch(shells, q)
    return np.array([np.sqrt(np.max(np.abs(vals[offs[i]:offs[i + 1]]))) for i in range(len(q))])


def test_unique_pairs_cover_every_unordered_pair_once():
    sh = W.molecule_basis(n_atoms=3, box=6.0, shells_per_atom=(0, 1, 2), kmax=2, seed_k=9)
    pairs = S.unique_pairs(sh)
    n = sh.n
    assert len(pairs) == n * (n + 1) // 2
    keys = {tuple(sorted(p)) for p in pairs.tolist()}
    assert len(keys) == len(pairs)
    L = np.asarray(sh.L)
    assert np.all(L[pairs[:, 0]] >= L[pairs[:, 1]])


def test_counts_match_brute_force():
    sh = W.molecule_basis(n_atoms=4, box=8.0, shells_per_atom=(0, 1, 2), kmax=2, seed_k=10)
    pairs = S.unique_pairs(sh)
    qf = schwarz_factors(sh, pairs)
    tau = 1e-6
    sq = S.ScreenedQuartets(sh, pairs, qf, tau)
    got = sq.class_counts()
    pc = S.pair_class(sh, pairs)
    size = S.pair_size(pc)
    expect = {}
    for a, b in itertools.combinations_with_replacement(range(len(pairs)), 2):
        if qf[a] * qf[b] < tau:
            continue
        bra, ket = (a, b) if size[a] >= size[b] else (b, a)
        cls = int(pc[bra]) * 16 + int(pc[ket])
        expect[cls] = expect.get(cls, 0) + 1
    assert {k: v for k, v in got.items() if v} == expect


def test_sample_is_screened_canonical_and_unique():
    sh = W.molecule_basis(n_atoms=4, box=8.0, shells_per_atom=(0, 1, 2), kmax=2, seed_k=11)
    pairs = S.unique_pairs(sh)
    qf = schwarz_factors(sh, pairs)
    sq = S.ScreenedQuartets(sh, pairs, qf, 1e-6)
    q = sq.sample(np.random.default_rng(0), eri_budget=10**9)
    assert len(q) == sum(sq.class_counts().values())
    L = np.asarray(sh.L)
    n = [W.shell_size(int(L[q[:, x]][i])) for x in range(4) for i in range(1)]
    assert n
    assert np.all(L[q[:, 0]] >= L[q[:, 1]]) and np.all(L[q[:, 2]] >= L[q[:, 3]])
    sizes_bra = (L[q[:, 0]] + 1) * (L[q[:, 0]] + 2) * (L[q[:, 1]] + 1) * (L[q[:, 1]] + 2)
    sizes_ket = (L[q[:, 2]] + 1) * (L[q[:, 2]] + 2) * (L[q[:, 3]] + 1) * (L[q[:, 3]] + 2)
    assert np.all(sizes_bra >= sizes_ket)
    keys = {frozenset([tuple(sorted(r[:2])), tuple(sorted(r[2:]))]) for r in q.tolist()}
    assert len(keys) == len(q)
