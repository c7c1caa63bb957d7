"""Pins of the oracle's gradients of E = sum G_abcd (ab|cd) with respect to shell centres
and primitive exponents: central finite differences of the (separately pinned) ERIs, and
the translational sum rule."""
import numpy as np
import pytest

import oracle
from paper_2303_13632_gb300 import workloads as W


def energy(shells, quartets, G, offsets):
    vals, offs = oracle.eri_batch(shells, quartets)
    assert np.array_equal(offs, offsets)
    return float(np.dot(vals, G))


def setup(cls_list, K, seed):
    rng = np.random.default_rng(seed)
    pool = W.random_contracted_pool(rng, 3, K=K, Ls=(0, 1, 2, 3))
    qs = np.concatenate([W.random_class_quartets(rng, c, 2, 3, Ls=(0, 1, 2, 3)) for c in cls_list])
    sizes = oracle.quartet_sizes(pool, qs)
    offsets = np.zeros(len(qs) + 1, dtype=np.int64)
    np.cumsum(sizes, out=offsets[1:])
    G = rng.standard_normal(int(offsets[-1]))
    return pool, qs, G, offsets


@pytest.mark.parametrize("cls", [(1, 1, 1, 1), (2, 1, 0, 2), (2, 2, 1, 1)])
def test_centre_gradient_vs_finite_differences(cls):
    pool, qs, G, offs = setup([cls], K=2, seed=21)
    dR, _ = oracle.eri_grad_batch(pool, qs, G, offs)
    h = 1e-4
    used = np.unique(qs)
    for s in used[:6]:
        for xi in range(3):
            p = W.ShellSet(pool.centers.copy(), pool.L, pool.nprim, pool.pofs, pool.exps, pool.coefs)
            m = W.ShellSet(pool.centers.copy(), pool.L, pool.nprim, pool.pofs, pool.exps, pool.coefs)
            p.centers[s, xi] += h
            m.centers[s, xi] -= h
            fd = (energy(p, qs, G, offs) - energy(m, qs, G, offs)) / (2 * h)
            assert abs(fd - dR[s, xi]) <= 1e-7 * max(1.0, abs(fd)), (s, xi, fd, dR[s, xi])


@pytest.mark.parametrize("cls", [(1, 1, 1, 1), (2, 0, 1, 2)])
def test_exponent_gradient_vs_finite_differences(cls):
    pool, qs, G, offs = setup([cls], K=2, seed=22)
    _, da = oracle.eri_grad_batch(pool, qs, G, offs)
    used = np.unique(qs)
    for s in used[:4]:
        for k in range(int(pool.nprim[s])):
            j = int(pool.pofs[s]) + k
            h = 1e-5 * pool.exps[j]
            ep, em = pool.exps.copy(), pool.exps.copy()
            ep[j] += h
            em[j] -= h
            p = W.ShellSet(pool.centers, pool.L, pool.nprim, pool.pofs, ep, pool.coefs)
            m = W.ShellSet(pool.centers, pool.L, pool.nprim, pool.pofs, em, pool.coefs)
            fd = (energy(p, qs, G, offs) - energy(m, qs, G, offs)) / (2 * h)
            assert abs(fd - da[j]) <= 2e-7 * max(1.0, abs(fd)), (s, k, fd, da[j])


def test_translational_sum_rule():
    """Moving all four centres together leaves every ERI unchanged: sum of dE/dR_x = 0."""
    pool, qs, G, offs = setup([(1, 1, 1, 1), (3, 2, 1, 0), (2, 2, 2, 2)], K=2, seed=23)
    dR, _ = oracle.eri_grad_batch(pool, qs, G, offs)
    scale = np.max(np.abs(dR))
    assert np.all(np.abs(dR.sum(axis=0)) <= 1e-12 * max(1.0, scale))
