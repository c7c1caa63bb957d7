"""Pins of the oracle's ERIs (Eq. 1 of arXiv 2303.13632) against facts that do not
come from the oracle's own recursions: textbook closed forms, an independent second
evaluator, and the symmetries and inequalities every ERI satisfies (Sec. II-B)."""
import itertools
import math

import numpy as np
import pytest

import oracle
from oracle.classes import all_classes
from paper_2303_13632_gb300 import workloads as W


def shells_from(centers, Ls, exps, coefs=None):
    coefs = coefs if coefs is not None else [[1.0] * len(e) for e in exps]
    return W.make_shellset(np.asarray(centers, dtype=float), Ls, exps, coefs)


# ---------------------------------------------------------------- normalisation

@pytest.mark.parametrize("L", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("alpha", [0.3, 1.5, 7.0])
def test_norm_axis_aligned_unit(L, alpha):
    """Sec. II-A: N makes the axis-aligned component x^L exp(-alpha r^2) normalised.
    int x^{2L} e^{-2 alpha x^2} dx * (pi / (2 alpha)) over y, z by numerical quadrature."""
    from scipy.integrate import quad

    ix, _ = quad(lambda x: x ** (2 * L) * math.exp(-2 * alpha * x * x), -np.inf, np.inf,
                 epsabs=0, epsrel=2e-14)
    n2 = oracle.norm(alpha, L) ** 2 * ix * math.pi / (2 * alpha)
    assert abs(n2 - 1.0) < 1e-12


# ---------------------------------------------------------------- closed forms

@pytest.mark.parametrize("alpha", [0.2, 1.0, 1.5, 9.0])
def test_ssss_same_centre(alpha):
    """Four identical normalised s Gaussians on one centre: 2 sqrt(alpha / pi)."""
    sh = shells_from(np.zeros((4, 3)), [0, 0, 0, 0], [[alpha]] * 4)
    v = oracle.eri_quartet(sh, [0, 1, 2, 3])[0, 0, 0, 0]
    assert abs(v - 2 * math.sqrt(alpha / math.pi)) < 1e-15


def test_ssss_golden_unit_exponent(golden):
    rows = golden("ssss_closed_form.txt")
    for alpha, R, expected in ((float(a), float(r), float(e)) for a, r, e in rows):
        sh = shells_from([[0, 0, 0], [0, 0, 0], [0, 0, R], [0, 0, R]], [0] * 4, [[alpha]] * 4)
        assert abs(oracle.eri_quartet(sh, [0, 1, 2, 3])[0, 0, 0, 0] - expected) < 1e-15


@pytest.mark.parametrize("alpha,gamma,R", [(0.5, 0.5, 1.3), (1.5, 0.2, 2.7), (3.0, 8.0, 0.4), (0.1, 4.0, 6.0)])
def test_ssss_two_gaussian_charges(alpha, gamma, R):
    """(s_A s_A | s_C s_C) is the Coulomb energy of two unit spherical Gaussian charges
    with exponents 2 alpha and 2 gamma: erf(sqrt(mu) R) / R, mu = 4 alpha gamma / (2 alpha + 2 gamma)."""
    sh = shells_from([[0, 0, 0], [0, 0, 0], [0, 0, R], [0, 0, R]], [0] * 4,
                     [[alpha], [alpha], [gamma], [gamma]])
    mu = (2 * alpha) * (2 * gamma) / (2 * alpha + 2 * gamma)
    v = oracle.eri_quartet(sh, [0, 1, 2, 3])[0, 0, 0, 0]
    assert abs(v - math.erf(math.sqrt(mu) * R) / R) < 2e-15


def test_far_separation_point_charges():
    """Well separated charge distributions interact like point charges S_ab S_cd / R."""
    R = 60.0
    sh = shells_from([[0, 0, 0], [0, 0, 0], [0, 0, R], [0, 0, R]], [0] * 4, [[1.0]] * 4)
    assert abs(oracle.eri_quartet(sh, [0, 1, 2, 3])[0, 0, 0, 0] - 1.0 / R) < 1e-15


def test_component_order_on_axis():
    """Components are ordered xx, xy, xz, yy, yz, zz (a_x descending, then a_y): with all
    centres on the x axis every component odd in y or z vanishes."""
    sh = shells_from([[0.0, 0, 0], [0.7, 0, 0], [-1.1, 0, 0], [1.9, 0, 0]], [3, 2, 1, 0],
                     [[0.8], [1.3], [0.6], [2.0]])
    v = oracle.eri_quartet(sh, [0, 1, 2, 3])
    comps = {L: oracle.cart_components(L) for L in range(4)}
    assert comps[2] == [(2, 0, 0), (1, 1, 0), (1, 0, 1), (0, 2, 0), (0, 1, 1), (0, 0, 2)]
    for ia, ib, ic in itertools.product(range(10), range(6), range(3)):
        tot = np.add(np.add(comps[3][ia], comps[2][ib]), comps[1][ic])
        odd = tot[1] % 2 == 1 or tot[2] % 2 == 1
        if odd:
            assert v[ia, ib, ic, 0] == 0.0 or abs(v[ia, ib, ic, 0]) < 1e-16
        if tuple(tot) == (6, 0, 0):
            assert abs(v[ia, ib, ic, 0]) > 1e-6


# ---------------------------------------------------------------- two evaluators

@pytest.mark.parametrize("cls", all_classes())
def test_os_matches_mcmurchie_davidson_all_classes(cls):
    rng = np.random.default_rng(1000 + W.class_id(*cls))
    pool = W.random_primitive_pool(rng, 4)
    q = W.random_class_quartets(rng, cls, 2, 4)
    a, _ = oracle.eri_batch(pool, q, "os")
    b, _ = oracle.eri_batch(pool, q, "md")
    # the Head-Gordon-Pople transfer loses up to ~2 digits for separated centres
    scale = max(1.0, np.max(np.abs(a)))
    assert np.max(np.abs(a - b)) <= 2e-12 * scale


G_CLASSES = [c for c in all_classes(4) if 4 in c]


def test_os_matches_mcmurchie_davidson_g_classes():
    """The 369 classes with a g shell (L = 4), one quartet each: the two evaluators agree."""
    assert len(G_CLASSES) == 369
    rng = np.random.default_rng(2000)
    Ls = (0, 1, 2, 3, 4)
    pool = W.random_primitive_pool(rng, 3, Ls=Ls)
    for cls in G_CLASSES:
        q = W.random_class_quartets(rng, cls, 1, 3, Ls=Ls)
        a, _ = oracle.eri_batch(pool, q, "os")
        b, _ = oracle.eri_batch(pool, q, "md")
        assert np.max(np.abs(a - b)) <= 2e-12 * max(1.0, np.max(np.abs(a))), cls


def test_os_matches_md_contracted():
    rng = np.random.default_rng(7)
    pool = W.random_contracted_pool(rng, 3, K=3, Ls=(0, 1, 2, 3))
    for cls in [(1, 1, 1, 1), (2, 1, 2, 0), (3, 2, 1, 3), (2, 2, 2, 2)]:
        q = W.random_class_quartets(rng, cls, 2, 3, Ls=(0, 1, 2, 3))
        a, _ = oracle.eri_batch(pool, q, "os")
        b, _ = oracle.eri_batch(pool, q, "md")
        assert np.max(np.abs(a - b)) <= 2e-12 * max(1.0, np.max(np.abs(a)))


# ---------------------------------------------------------------- invariants

def random_quartet_shells(rng, cls, K=1):
    centers = rng.uniform(-2.0, 2.0, size=(4, 3))
    exps = [list(np.exp(rng.uniform(np.log(0.2), np.log(5.0), size=K))) for _ in range(4)]
    coefs = [list(rng.uniform(0.3, 1.0, size=K)) for _ in range(4)]
    return shells_from(centers, list(cls), exps, coefs)


@pytest.mark.parametrize("cls", [(1, 0, 2, 1), (3, 1, 2, 2), (2, 2, 3, 0), (3, 3, 1, 1), (4, 2, 1, 3),
                                 (4, 4, 2, 0)])
@pytest.mark.parametrize("method", ["md", "os"])
def test_eightfold_symmetry(cls, method):
    """Sec. II-B: [ab|cd] = [ba|cd] = [ab|dc] = [cd|ab] = ... (8 variants)."""
    rng = np.random.default_rng(11)
    sh = random_quartet_shells(rng, cls, K=2)
    v = oracle.eri_quartet(sh, [0, 1, 2, 3], method)
    perms = {
        (1, 0, 2, 3): (1, 0, 2, 3), (0, 1, 3, 2): (0, 1, 3, 2), (1, 0, 3, 2): (1, 0, 3, 2),
        (2, 3, 0, 1): (2, 3, 0, 1), (3, 2, 0, 1): (3, 2, 0, 1), (2, 3, 1, 0): (2, 3, 1, 0),
        (3, 2, 1, 0): (3, 2, 1, 0),
    }
    for order, axes in perms.items():
        w = oracle.eri_quartet(sh, list(order), method)
        np.testing.assert_allclose(np.transpose(v, axes), w, rtol=0, atol=1e-13)


@pytest.mark.parametrize("cls", [(1, 1, 1, 1), (3, 2, 2, 1), (0, 3, 3, 0), (4, 1, 0, 4)])
@pytest.mark.parametrize("method,tol", [("md", 1e-15), ("os", 1e-12)])
def test_translation_invariance(cls, method, tol):
    rng = np.random.default_rng(12)
    sh = random_quartet_shells(rng, cls)
    v = oracle.eri_quartet(sh, [0, 1, 2, 3], method)
    sh2 = W.ShellSet(sh.centers + np.array([3.1, -7.2, 0.45]), sh.L, sh.nprim, sh.pofs, sh.exps, sh.coefs)
    w = oracle.eri_quartet(sh2, [0, 1, 2, 3], method)
    np.testing.assert_allclose(v, w, rtol=0, atol=tol * max(1, np.max(np.abs(v))))


def monomial_rotation(L, R):
    """M[a, b]: (R x)^a = sum_b M[a, b] x^b for the Cartesian monomials of degree L."""
    comps = oracle.cart_components(L)
    index = {c: i for i, c in enumerate(comps)}
    M = np.zeros((len(comps), len(comps)))
    for ia, a in enumerate(comps):
        # expand prod_i (sum_j R_ij x_j)^{a_i} as a polynomial dict {(e0,e1,e2): coef}
        poly = {(0, 0, 0): 1.0}
        for i in range(3):
            for _ in range(a[i]):
                new = {}
                for e, c in poly.items():
                    for j in range(3):
                        e2 = list(e)
                        e2[j] += 1
                        new[tuple(e2)] = new.get(tuple(e2), 0.0) + c * R[i, j]
                poly = new
        for e, c in poly.items():
            M[ia, index[e]] += c
    return M


@pytest.mark.parametrize("cls", [(1, 0, 0, 0), (1, 1, 1, 1), (2, 1, 3, 0), (3, 3, 2, 2), (2, 2, 2, 2), (4, 0, 0, 0),
                                 (4, 3, 1, 2), (4, 4, 4, 4)])
def test_rotational_invariance(cls):
    """Rotating every centre by R about the origin maps each Cartesian shell by the monomial
    transform of R (one normalisation per shell), so (ab|cd)_rot = M_a M_b M_c M_d (ab|cd)."""
    rng = np.random.default_rng(13)
    sh = random_quartet_shells(rng, cls)
    v = oracle.eri_quartet(sh, [0, 1, 2, 3])
    from scipy.spatial.transform import Rotation

    R = Rotation.from_euler("zyx", [0.7, -1.1, 2.3]).as_matrix()
    sh2 = W.ShellSet(sh.centers @ R.T, sh.L, sh.nprim, sh.pofs, sh.exps, sh.coefs)
    w = oracle.eri_quartet(sh2, [0, 1, 2, 3])
    M = [monomial_rotation(L, R) for L in cls]
    pred = np.einsum("ai,bj,ck,dl,ijkl->abcd", M[0], M[1], M[2], M[3], v)
    np.testing.assert_allclose(w, pred, rtol=0, atol=1e-13 * max(1, np.max(np.abs(v))))


@pytest.mark.parametrize("cls", [(1, 1, 1, 1), (2, 1, 2, 1), (3, 0, 2, 2), (3, 3, 3, 3), (4, 2, 4, 1)])
def test_schwarz_inequality(cls):
    """|(ab|cd)| <= sqrt((ab|ab)(cd|cd)) for every component."""
    rng = np.random.default_rng(14)
    sh = random_quartet_shells(rng, cls, K=2)
    v = oracle.eri_quartet(sh, [0, 1, 2, 3])
    ab = oracle.eri_quartet(sh, [0, 1, 0, 1])
    cd = oracle.eri_quartet(sh, [2, 3, 2, 3])
    na, nb, nc, nd = v.shape
    dab = np.array([[ab[i, j, i, j] for j in range(nb)] for i in range(na)])
    dcd = np.array([[cd[k, l, k, l] for l in range(nd)] for k in range(nc)])
    assert np.all(dab >= 0) and np.all(dcd >= 0)
    bound = np.sqrt(np.einsum("ij,kl->ijkl", dab, dcd))
    assert np.all(np.abs(v) <= bound * (1 + 1e-12) + 1e-300)


def test_contraction_linearity():
    """A contracted quartet equals the coefficient-weighted sum of its primitive quartets."""
    rng = np.random.default_rng(15)
    cls = (2, 1, 1, 2)
    sh = random_quartet_shells(rng, cls, K=2)
    v = oracle.eri_quartet(sh, [0, 1, 2, 3])
    total = np.zeros_like(v)
    for idx in itertools.product(range(2), repeat=4):
        exps = [[sh.exps[sh.pofs[x] + idx[x]]] for x in range(4)]
        coefs = [[sh.coefs[sh.pofs[x] + idx[x]]] for x in range(4)]
        p = shells_from(sh.centers, list(cls), exps, coefs)
        total += oracle.eri_quartet(p, [0, 1, 2, 3])
    np.testing.assert_allclose(v, total, rtol=0, atol=1e-14)


# ---------------------------------------------------------------- the paper's Rys route

@pytest.mark.parametrize("n", range(1, 8))
def test_rys_roots_reproduce_boys_moments(n):
    """Sec. II-C: the n roots x = t^2 and weights integrate x^k exactly against the Rys weight,
    sum w x^k = F_k(T) for k < 2n (F_k from the oracle's pinned Boys function); 0 < x < 1,
    w > 0.  T spans the small-T series, the erf branch and the far tail."""
    for T in [0.0, 1e-8, 0.5, 3.0, 17.0, 39.9, 40.1, 100.0, 169.0, 170.0, 1e3, 1e5, 1e7]:
        x, w = oracle.rys_roots(n, T)
        F = oracle.boys(2 * n - 1, T)
        mom = np.array([np.sum(w * x ** k) for k in range(2 * n)])
        np.testing.assert_allclose(mom, F, rtol=1e-13, atol=0, err_msg=f"n={n} T={T}")
        assert np.all((x > 0) & (x < 1)) and np.all(w > 0)


def test_rys_one_root_closed_form():
    """n = 1: w = F_0(T) and x = F_1(T) / F_0(T); at T = 0 that is w = 1, x = 1/3 (to the
    rounding of the 256-node sums, a few 1e-15)."""
    x, w = oracle.rys_roots(1, 0.0)
    assert abs(w[0] - 1.0) < 1e-14 and abs(x[0] - 1.0 / 3.0) < 1e-14
    for T in [0.3, 5.0, 60.0]:
        x, w = oracle.rys_roots(1, T)
        F = oracle.boys(1, T)
        assert abs(w[0] - F[0]) <= 1e-14 * F[0] and abs(x[0] - F[1] / F[0]) <= 1e-14 * x[0]


@pytest.mark.parametrize("n", [1, 3, 5, 7])
def test_rys_large_T_gauss_hermite_limit(n):
    """For large T the weight exp(-T t^2) on (0, 1) is the half-line Gaussian up to exp(-T):
    t_mu sqrt(T) are the positive nodes u of the 2n-point Gauss-Hermite rule and
    w_mu = W(u) / sqrt(T) (numpy's hermgauss, an independent routine)."""
    T = 400.0
    u, W_ = np.polynomial.hermite.hermgauss(2 * n)
    pos = u > 0
    x, w = oracle.rys_roots(n, T)
    np.testing.assert_allclose(x, np.sort(u[pos] ** 2 / T), rtol=1e-11)
    np.testing.assert_allclose(w, W_[pos][np.argsort(u[pos])] / math.sqrt(T), rtol=1e-11)


@pytest.mark.parametrize("cls", all_classes())
def test_paper_rys_route_matches_md_all_classes(cls):
    """The paper's scheme written out (roots and weights, B and C of Eq. 6 as read, the weight
    counted once, Eq. 7 transfer, Eq. 8 quadrature) reproduces the McMurchie-Davidson ERIs on
    every class: a check of those readings by a route that shares only the Boys function.
    (A sign flipped in C00' moves results by 1e-10 to 1e-4 of the largest ERI.)"""
    rng = np.random.default_rng(1000 + W.class_id(*cls))
    pool = W.random_primitive_pool(rng, 4)
    q = W.random_class_quartets(rng, cls, 2, 4)
    a, _ = oracle.eri_batch(pool, q, "rys")
    b, _ = oracle.eri_batch(pool, q, "md")
    assert np.max(np.abs(a - b)) <= 1e-13 * max(1.0, np.max(np.abs(b)))


def test_paper_rys_route_matches_md_contracted():
    rng = np.random.default_rng(8)
    pool = W.random_contracted_pool(rng, 3, K=3, Ls=(0, 1, 2, 3))
    for cls in [(1, 1, 1, 1), (2, 1, 2, 0), (3, 2, 1, 3), (3, 3, 3, 3)]:
        q = W.random_class_quartets(rng, cls, 2, 3, Ls=(0, 1, 2, 3))
        a, _ = oracle.eri_batch(pool, q, "rys")
        b, _ = oracle.eri_batch(pool, q, "md")
        assert np.max(np.abs(a - b)) <= 1e-13 * max(1.0, np.max(np.abs(b)))
