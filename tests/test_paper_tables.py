"""Class bookkeeping pinned to the numbers printed in arXiv 2303.13632.

Sec. II-B: 256 generic and 55 canonical classes (Eq. 3).
Table III: trip counts after the general optimisation (Sec. III-C).
Table V: n_ERIQ, n_GQ, n_CS and the model of Eq. 12.
"""
import pytest

from oracle import classes as C


def test_class_counts():
    cls = C.all_classes()
    assert len(cls) == 256
    assert sum(C.is_canonical(*c) for c in cls) == 55


def test_table3_trip_counts(golden):
    for name, nrr, ngq, ncs in golden("paper_table3_trip_counts.txt"):
        c = C.parse_class(name)
        assert C.n_rr(*c) == int(nrr), name
        assert C.n_gq(*c) == int(ngq), name
        assert C.n_cs(*c, bits=16) == int(ncs), name


def test_intermediate_buffer_sizes():
    """Sec. III-C: I(i,j,k,l,mu,xi) holds 3 values for [ss|ss] and 5376 for [ff|ff]."""
    def size(La, Lb, Lc, Ld):
        return 3 * C.n_rys(La, Lb, Lc, Ld) * (La + 1) * (Lb + 1) * (Lc + 1) * (Ld + 1)

    assert size(0, 0, 0, 0) == 3
    assert size(3, 3, 3, 3) == 5376


def test_table5_counts_and_model(golden):
    for row in golden("paper_table5_permutations.txt"):
        name, fmax, neri, nrr, ngq, ncs, gmodel, _gmeas, canon = row
        c = C.parse_class(name)
        assert C.n_eriq(*c) == int(neri)
        assert C.n_gq(*c) == int(ngq)
        assert C.n_cs(*c, bits=16) == int(ncs)
        assert C.is_canonical(*c) == bool(int(canon))
        # Eq. 12 with the printed trip counts reproduces the printed model GERIS
        g = C.geris_model(float(fmax) * 1e6, int(neri), int(nrr), int(ngq), int(ncs))
        assert abs(g - float(gmodel)) < 0.006, (name, g, gmodel)
        # the general-optimisation n_RR of Sec. III-C is an upper bound of the printed one
        # wherever further unrolling (Table IV) applied, except [fd|fd]/[df|fd], whose printed
        # 72 is not reproduced by the rule (reading recorded in the design notes)
        if name not in ("[fd|fd]", "[df|fd]"):
            assert int(nrr) <= C.n_rr(*c)


@pytest.mark.parametrize("L,n", [(0, 1), (1, 3), (2, 6), (3, 10)])
def test_shell_sizes(L, n):
    assert C.n_g(L) == n
