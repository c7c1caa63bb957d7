"""The algorithmic work per quartet (the numerator of every roofline figure) against the
paper's own counts, and the canonical-class mapping it uses."""
import itertools

import pytest

from oracle.classes import n_eriq
from paper_2303_13632_gb300 import perfmodel as P


def _paper_count(cls):
    """n_FLOPQ as the paper counts it (Sec. III-A): the Rys roots are prepared on the host there,
    so the on-device root term 60 n_Rys of the model is left out."""
    f64, rr = P.flops_per_quartet(cls)
    La, Lb, Lc, Ld = P.canonical(cls)
    n = (La + Lb + Lc + Ld) // 2 + 1
    return f64 - 60 * n + rr


def test_matches_the_papers_operation_counts():
    # Sec. III-A: total n_FLOPQ grows from 80 for [ss|ss] to 2.5e5 for [ff|ff]
    assert _paper_count((0, 0, 0, 0)) == pytest.approx(80, rel=0.2)
    assert _paper_count((3, 3, 3, 3)) == pytest.approx(2.5e5, rel=0.05)


def test_quadrature_dominates_large_classes_and_setup_small_ones():
    # Sec. III-A: setup dominates a few small classes, quadrature the large ones
    f64, rr = P.flops_per_quartet((0, 0, 0, 0))
    assert f64 > rr
    La, Lb, Lc, Ld = 3, 3, 3, 3
    quad = 3 * 7 * n_eriq(La, Lb, Lc, Ld)
    assert quad > 0.8 * P.flops_per_quartet((La, Lb, Lc, Ld))[1]


def test_canonical_classes():
    canon = {P.canonical(c) for c in itertools.product(range(4), repeat=4)}
    assert len(canon) == 55
    for c in itertools.product(range(4), repeat=4):
        k = P.canonical(c)
        assert n_eriq(*k) == n_eriq(*c)
        assert sorted(k[:2]) in (sorted(c[:2]), sorted(c[2:]))
        assert k[0] >= k[1] and k[2] >= k[3]
        assert P.ncart(k[0]) * P.ncart(k[1]) >= P.ncart(k[2]) * P.ncart(k[3])


def test_mixed_split_keeps_the_total():
    """The mixed path moves two thirds of the root evaluation to the recurrence type, and the B,
    C arrays where it forms them in two-float FP32; the total count per quartet is the same as
    the plain path's."""
    for cls in [(0, 0, 0, 0), (1, 0, 0, 0), (2, 0, 2, 0), (1, 0, 1, 0), (1, 1, 1, 1), (3, 2, 1, 0),
                (3, 3, 3, 3)]:
        a, b = P.flops_per_quartet(cls, "fp64"), P.flops_per_quartet(cls, "mixed")
        n = sum(cls) // 2 + 1
        moved = 40 * n + (20 * n if P.two_float_setup(cls) else 0)
        assert sum(a) == sum(b) and a[0] - b[0] == moved


def test_two_float_setup_classes():
    """Inline-setup classes with one root keep the FP64 B, C; split-path classes use two-float."""
    assert not P.two_float_setup((0, 0, 0, 0)) and not P.two_float_setup((1, 0, 0, 0))
    assert not P.two_float_setup((2, 0, 2, 0)) and not P.two_float_setup((0, 0, 1, 2))
    assert P.two_float_setup((1, 0, 1, 0)) and P.two_float_setup((3, 0, 1, 0))
    assert P.two_float_setup((2, 1, 1, 0)) and P.two_float_setup((3, 3, 3, 3))


def test_roofline_time_is_the_larger_bound():
    cls, n = (1, 1, 1, 1), 1000
    t = P.roofline_seconds(cls, n, "mixed", 16, 7000.0)
    f64, rr = P.flops_per_quartet(cls, "mixed")
    t_alu = n * (f64 / (P.PEAK_FP64_TFLOPS * 1e12) + rr / (P.PEAK_FP32_TFLOPS * 1e12))
    t_mem = n * P.bytes_per_quartet(cls, 16) / 7000e9
    assert t == pytest.approx(max(t_alu, t_mem))
    assert P.roofline_seconds(cls, n, "fp64", 16, 7000.0) > t


def test_gpu_model_fits_the_committed_class_table():
    import os

    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "profiles",
                        "sweep256_per_class.md")
    table = P.read_class_table(path)
    assert len(table) == 256
    measured = {c: n_eriq(*c) / (g * 1e9) for c, (n, g) in table.items()}
    p, q = P.fit_gpu_model(measured)
    assert q["r2_log"] > 0.95
    assert q["median_abs_log_err"] < 0.2
    # the fitted rates stay below the nominal peaks
    assert p["R64"] < P.PEAK_FP64_TFLOPS * 1e12 and p["R32"] < P.PEAK_FP32_TFLOPS * 1e12


def test_adjoint_count():
    """The adjoint's count: [ss|ss] by hand (extended class [dd|dd] for the recurrences, two roots),
    the contraction term growing as n_ERIQ, and the mixed split keeping the total."""
    f64, rr = P.adjoint_flops_per_quartet((0, 0, 0, 0))
    n = 2  # floor(2 / 2) + 1 roots for the ranges L + 2 of [ss|ss]
    vrr = 5 * 3 * n * (5 * 5 - 1)
    hrr = 2 * 3 * n * (sum(4 - j + 1 for j in range(1, 3)) * 5 + 3 * 3 * sum(4 - l + 1 for l in range(1, 3)))
    assert f64 == 40 + 20 * n + 60 * n + 20
    assert rr == vrr + hrr + 9 * n * 1 + 90 * n * 1
    a, b = P.adjoint_flops_per_quartet((2, 2, 2, 2), "fp64"), P.adjoint_flops_per_quartet((2, 2, 2, 2), "mixed")
    assert sum(a) == sum(b) and a[0] - b[0] == 40 * 6
    # the contraction (9 n n_ERIQ) is the largest term of the large classes
    n = (12 + 2) // 2 + 1
    assert 9 * n * 10000 > 0.5 * P.adjoint_flops_per_quartet((3, 3, 3, 3))[1]
