"""Quartet lists built by eri_plan_create on the device: the 8-fold unique quartets (Sec. II-B)
and Schwarz screening, against brute-force enumeration with Schwarz factors from the oracle.

Brute force: every unordered pair of unordered shell pairs {P, R} is kept when
Q_P Q_R >= tau, Q_P = sqrt(max |(ij|ij)|) from the oracle's FP64 ERIs.  Thresholds are moved
away from every product Q_P Q_R by at least 1e-8 relative, so FP64 rounding of the library's
own diagonal ERIs cannot decide a borderline quartet differently.
"""
import itertools

import numpy as np
import pytest
import torch

import oracle
from paper_2303_13632_gb300 import api, workloads as W

pytestmark = pytest.mark.gpu


def small_basis(seed=10, n_atoms=4):
    return W.molecule_basis(n_atoms=n_atoms, box=8.0, shells_per_atom=(0, 1, 2), kmax=2, seed_k=seed)


def pair_list(n):
    return [(i, j) for i in range(n) for j in range(i + 1)]


def oracle_q(shells):
    pairs = np.array(pair_list(shells.n), dtype=np.int32)
    q = np.stack([pairs[:, 0], pairs[:, 1], pairs[:, 0], pairs[:, 1]], axis=1)
    vals, offs = oracle.eri_batch(shells, q)
    return pairs, np.array([np.sqrt(np.max(np.abs(vals[offs[i]:offs[i + 1]]))) for i in range(len(q))])


def safe_tau(Q, tau):
    """A threshold near tau that no product Q_P Q_R approaches within 1e-8 relative."""
    prods = np.sort(np.outer(Q, Q).ravel())
    for k in range(200):
        t = tau * (1.0 + 0.0137 * k)
        i = np.searchsorted(prods, t)
        near = [prods[j] for j in (i - 1, i) if 0 <= j < len(prods)]
        if all(abs(p - t) > 1e-8 * t for p in near):
            return t
    raise AssertionError("no safe threshold")


def brute_force(pairs, Q, tau):
    keep = set()
    for P, R in itertools.combinations_with_replacement(range(len(pairs)), 2):
        if Q[P] * Q[R] >= tau:
            keep.add(frozenset([tuple(sorted(pairs[P])), tuple(sorted(pairs[R]))]))
    return keep


def plan_keys(plan):
    """The plan's quartets and their 8-fold symmetry classes (unordered pairs of unordered pairs)."""
    q = api.eri_plan_quartets(plan)
    keys = [frozenset([tuple(sorted((int(r[0]), int(r[1])))), tuple(sorted((int(r[2]), int(r[3]))))])
            for r in q]
    return q, keys


@pytest.mark.parametrize("tau", [0.0, 1e-6, 3e-3])
def test_unique8_matches_brute_force(tau):
    sh = small_basis()
    pairs, Q = oracle_q(sh)
    npairs = len(pairs)
    t = safe_tau(Q, tau) if tau > 0 else 0.0
    plan = api.eri_plan_create(sh, None, mode="unique8", schwarz_threshold=t)
    q, keys = plan_keys(plan)
    expect = brute_force([tuple(p) for p in pairs], Q, t) if t > 0 else \
        {frozenset([tuple(sorted(P)), tuple(sorted(R))]) for P, R in
         itertools.combinations_with_replacement([tuple(p) for p in pairs], 2)}
    assert len(keys) == len(set(keys))       # no symmetry class twice
    assert set(keys) == expect               # exactly the brute-force set
    cand, kept = api.eri_plan_screening(plan)
    assert cand == npairs * (npairs + 1) // 2 and kept == len(expect) == api.eri_plan_num_quartets(plan)
    assert np.all(q[:, 0] >= q[:, 1]) and np.all(q[:, 2] >= q[:, 3])
    # the quartet order is a permutation of the enumeration positions
    order = api.eri_plan_quartet_order(plan)
    assert sorted(order.tolist()) == list(range(len(q)))


def test_unique8_expands_to_every_ordered_quartet_and_values_match():
    """Without screening the unique quartets of an s, p, d, f pool expand (8-fold) to every
    ordered quartet once, and the plan's FP64 ERIs of them match the oracle."""
    rng = np.random.default_rng(3)
    pool = W.random_primitive_pool(rng, 1, Ls=(0, 1, 2, 3), box=2.0)
    plan = api.eri_plan_create(pool, None, mode="unique8")
    q = api.eri_plan_quartets(plan)
    vals, offs = oracle.eri_batch(pool, q)
    eq, _, _ = oracle.expand_unique8(pool, q, vals, offs)
    assert sorted(map(tuple, eq.tolist())) == sorted(itertools.product(range(pool.n), repeat=4))
    nb, _ = api.eri_output_bytes(plan, 0)
    out = torch.empty(nb // 8, dtype=torch.float64, device="cuda")
    api.eri_compute(plan, out)
    api.eri_sync(plan)
    got = out.cpu().numpy()
    err = np.abs(got - vals)
    assert np.all((err <= 1e-12) | (err <= 1e-10 * np.abs(vals)))


def test_shards_partition_the_enumeration():
    sh = small_basis(seed=12)
    pairs, Q = oracle_q(sh)
    t = safe_tau(Q, 1e-5)
    full = api.eri_plan_create(sh, None, mode="unique8", schwarz_threshold=t)
    _, full_keys = plan_keys(full)
    n = len(full_keys)
    seen = []
    for k in range(5):
        p = api.eri_plan_create(sh, None, mode="unique8", schwarz_threshold=t, shard=(k, 5))
        _, keys = plan_keys(p)
        assert len(keys) in (n // 5, n // 5 + 1)
        assert api.eri_plan_screening(p)[1] == n
        seen += keys
    assert len(seen) == n and set(seen) == set(full_keys)


@pytest.mark.parametrize("shard", [(0, 1 << 62), (3, 1 << 62), ((1 << 63) - 2, (1 << 63) - 1)])
def test_extreme_shard_counts(shard):
    """A shard count far beyond the enumeration keeps at most the one quartet at shard_index."""
    sh = small_basis(seed=16)
    full = api.eri_plan_create(sh, None, mode="unique8", schwarz_threshold=1e-6)
    q_full = api.eri_plan_quartets(full)
    order = api.eri_plan_quartet_order(full)
    by_pos = {int(p): tuple(r) for p, r in zip(order, q_full.tolist())}
    p = api.eri_plan_create(sh, None, mode="unique8", schwarz_threshold=1e-6, shard=shard)
    q = api.eri_plan_quartets(p)
    if shard[0] < len(q_full):
        assert len(q) == 1 and tuple(q[0]) == by_pos[shard[0]]
    else:
        assert len(q) == 0
    assert api.eri_plan_screening(p)[1] == len(q_full)


def test_screened_explicit_list_keeps_caller_indices():
    """A caller's list (ordered quartets, any orientation, repeats) filtered by the threshold:
    the kept ones are exactly those with Q_ij Q_kl >= tau, in the caller's order within a class,
    and eri_plan_quartet_order returns indices into the unscreened list."""
    sh = small_basis(seed=13)
    pairs, Q = oracle_q(sh)
    qidx = {tuple(sorted(p)): i for i, p in enumerate(map(tuple, pairs))}
    t = safe_tau(Q, 1e-4)
    rng = np.random.default_rng(14)
    q = rng.integers(0, sh.n, size=(3000, 4)).astype(np.int32)
    want = np.array([Q[qidx[tuple(sorted(r[:2]))]] * Q[qidx[tuple(sorted(r[2:]))]] >= t for r in q.tolist()])
    assert 0 < want.sum() < len(q)
    plan = api.eri_plan_create(sh, q, schwarz_threshold=t)
    assert api.eri_plan_screening(plan) == (len(q), int(want.sum()))
    order = api.eri_plan_quartet_order(plan)
    assert sorted(order.tolist()) == np.nonzero(want)[0].tolist()
    np.testing.assert_array_equal(api.eri_plan_quartets(plan), q[order])


def test_schwarz_bound_holds_for_kept_and_dropped():
    """Cauchy-Schwarz: every ERI of a quartet is at most Q_ij Q_kl, so a dropped quartet's ERIs
    are all below tau; checked on the oracle values of a sample of the unscreened list."""
    sh = small_basis(seed=15)
    pairs, Q = oracle_q(sh)
    qidx = {tuple(sorted(p)): i for i, p in enumerate(map(tuple, pairs))}
    full = api.eri_plan_create(sh, None, mode="unique8")
    q = api.eri_plan_quartets(full)
    vals, offs = oracle.eri_batch(sh, q)
    for i, r in enumerate(q.tolist()):
        bound = Q[qidx[tuple(sorted(r[:2]))]] * Q[qidx[tuple(sorted(r[2:]))]]
        assert np.max(np.abs(vals[offs[i]:offs[i + 1]])) <= bound * (1 + 1e-12) + 1e-300


def test_invalid_screening_options():
    sh = small_basis()
    with pytest.raises(api.EriError):
        api.eri_plan_create(sh, None, mode="unique8", schwarz_threshold=-1.0)
    with pytest.raises(api.EriError):
        api.eri_plan_create(sh, None, mode="unique8", shard=(3, 3))
    with pytest.raises(api.EriError):
        api.eri_plan_create(sh, np.zeros((1, 4), dtype=np.int32), shard=(0, 2))
