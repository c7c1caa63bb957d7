"""Pins of the oracle's Coulomb/exchange digestion of ERI blocks (the use of the ERIs and their
compressed copies that Sec. I and Sec. II-D motivate): a closed form, brute force over the full
ERI tensor of a tiny basis, the 8-fold symmetry expansion, and the compression bound carried
through the contraction."""
import itertools
import math

import numpy as np

import oracle
from paper_2303_13632_gb300 import workloads as W


def tiny_basis(seed=3):
    """One shell each of s, p, d (1 + 3 + 6 = 10 functions), contracted (K = 2)."""
    rng = np.random.default_rng(seed)
    centers = rng.uniform(-1.5, 1.5, size=(3, 3))
    exps = [list(np.exp(rng.uniform(np.log(0.3), np.log(3.0), size=2))) for _ in range(3)]
    coefs = [list(rng.uniform(0.3, 1.0, size=2)) for _ in range(3)]
    return W.make_shellset(centers, [0, 1, 2], exps, coefs)


def all_ordered(n):
    return np.array(list(itertools.product(range(n), repeat=4)), dtype=np.int32)


def full_tensor(shells):
    """(mu nu|lam sig) over the whole basis, assembled block by block from eri_batch."""
    q = all_ordered(shells.n)
    vals, offs = oracle.eri_batch(shells, q)
    bf = oracle.basis_offsets(shells)
    nbf = int(bf[-1])
    T = np.zeros((nbf,) * 4)
    for i, row in enumerate(q):
        shape = tuple(oracle.ncart(int(shells.L[s])) for s in row)
        sl = tuple(slice(bf[s], bf[s] + n) for s, n in zip(row, shape))
        T[sl] = vals[offs[i]:offs[i + 1]].reshape(shape)
    return T, q, vals, offs


def random_density(rng, n, symmetric=True):
    D = rng.standard_normal((n, n))
    return (D + D.T) / 2 if symmetric else D


def test_single_s_function_closed_form():
    """One normalised s function with exponent alpha: (ss|ss) = 2 sqrt(alpha/pi) (same-centre
    closed form), so J = K = 2 sqrt(alpha/pi) D."""
    for alpha in (0.5, 1.0, 3.7):
        sh = W.make_shellset(np.zeros((1, 3)), [0], [[alpha]], [[1.0]])
        vals, offs = oracle.eri_batch(sh, np.zeros((1, 4), dtype=np.int32))
        J, K = oracle.digest_jk(sh, np.zeros((1, 4), dtype=np.int32), vals, offs, np.array([[0.7]]))
        ref = 2.0 * math.sqrt(alpha / math.pi) * 0.7
        assert abs(J[0, 0] - ref) <= 1e-14 and abs(K[0, 0] - ref) <= 1e-14


def test_brute_force_over_the_full_tensor():
    """J and K of every ordered quartet equal the contractions of the assembled 4-index tensor:
    J = sum_ls T[m,n,l,s] D[l,s], K = sum_ns T[m,n,l,s] D[n,s] (non-symmetric D, so a swapped
    index would show)."""
    sh = tiny_basis()
    T, q, vals, offs = full_tensor(sh)
    D = random_density(np.random.default_rng(1), T.shape[0], symmetric=False)
    J, K = oracle.digest_jk(sh, q, vals, offs, D)
    np.testing.assert_allclose(J, np.einsum("mnls,ls->mn", T, D), rtol=0, atol=1e-13)
    np.testing.assert_allclose(K, np.einsum("mnls,ns->ml", T, D), rtol=0, atol=1e-13)


def test_symmetric_density_gives_symmetric_j_and_k():
    sh = tiny_basis(4)
    q = all_ordered(sh.n)
    vals, offs = oracle.eri_batch(sh, q)
    D = random_density(np.random.default_rng(2), int(oracle.basis_offsets(sh)[-1]))
    J, K = oracle.digest_jk(sh, q, vals, offs, D)
    np.testing.assert_allclose(J, J.T, atol=1e-13)
    np.testing.assert_allclose(K, K.T, atol=1e-13)


def test_unique_quartets_expand_to_every_ordered_quartet():
    """The unique quartets (a >= b, c >= d, pair ab >= pair cd) of the 8-fold symmetry (Sec. II-B)
    expand to each ordered quartet exactly once, with blocks equal to the directly computed
    ones, so digesting the expansion equals digesting every ordered quartet."""
    rng = np.random.default_rng(5)
    pool = W.random_primitive_pool(rng, 1, Ls=(0, 1, 2, 3))  # s, p, d, f shells
    n = pool.n
    pairs = [(a, b) for a in range(n) for b in range(a + 1)]
    uq = np.array([(a, b, c, d) for i, (a, b) in enumerate(pairs) for (c, d) in pairs[:i + 1]],
                  dtype=np.int32)
    vals, offs = oracle.eri_batch(pool, uq)
    eq, ev, eo = oracle.expand_unique8(pool, uq, vals, offs)
    full = all_ordered(n)
    assert sorted(map(tuple, eq.tolist())) == sorted(map(tuple, full.tolist()))
    fv, fo = oracle.eri_batch(pool, eq)
    np.testing.assert_allclose(ev, fv, rtol=0, atol=1e-13 * max(1.0, np.max(np.abs(fv))))
    D = random_density(rng, int(oracle.basis_offsets(pool)[-1]))
    J1, K1 = oracle.digest_jk(pool, eq, ev, eo, D)
    fv2, fo2 = oracle.eri_batch(pool, full)
    J2, K2 = oracle.digest_jk(pool, full, fv2, fo2, D)
    np.testing.assert_allclose(J1, J2, atol=1e-12)
    np.testing.assert_allclose(K1, K2, atol=1e-12)


def test_linearity_in_the_density():
    sh = tiny_basis(6)
    q = all_ordered(sh.n)
    vals, offs = oracle.eri_batch(sh, q)
    rng = np.random.default_rng(7)
    nbf = int(oracle.basis_offsets(sh)[-1])
    D1, D2 = random_density(rng, nbf), random_density(rng, nbf, symmetric=False)
    J1, K1 = oracle.digest_jk(sh, q, vals, offs, D1)
    J2, K2 = oracle.digest_jk(sh, q, vals, offs, D2)
    J3, K3 = oracle.digest_jk(sh, q, vals, offs, D1 - 2.5 * D2)
    np.testing.assert_allclose(J3, J1 - 2.5 * J2, atol=1e-12)
    np.testing.assert_allclose(K3, K1 - 2.5 * K2, atol=1e-12)


def test_compression_bound_carries_through_the_contraction():
    """With the ERIs replaced by their 16-bit decompressed copies (Eqs. 9-11), each element of J
    moves by at most sum over its quartets of (eps_q / 2) sum |D[l,s]| (the ANINT bound,
    |x - q eps| <= eps / 2, times the contraction's absolute weights); same for K."""
    sh = tiny_basis(8)
    q = all_ordered(sh.n)
    vals, offs = oracle.eri_batch(sh, q)
    codes, eps = oracle.compress_batch(vals, offs, 16)
    dec = np.concatenate([oracle.decompress_quartet(codes[offs[i]:offs[i + 1]], eps[i])
                          for i in range(len(q))])
    D = random_density(np.random.default_rng(9), int(oracle.basis_offsets(sh)[-1]))
    J, K = oracle.digest_jk(sh, q, vals, offs, D)
    Jc, Kc = oracle.digest_jk(sh, q, dec, offs, D)
    # the bound: digest |error| <= eps/2 element-wise, i.e. digest a block of eps_q/2 against |D|
    half = np.concatenate([np.full(offs[i + 1] - offs[i], eps[i] / 2.0) for i in range(len(q))])
    bJ, bK = oracle.digest_jk(sh, q, half * (1 + 1e-7), offs, np.abs(D))
    assert np.all(np.abs(Jc - J) <= bJ + 1e-15)
    assert np.all(np.abs(Kc - K) <= bK + 1e-15)
    assert np.max(np.abs(Jc - J)) > 0  # the compression did change something
