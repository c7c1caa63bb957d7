"""The adjoint's contraction table (csrc/eri_bwd_table.h), built by the host compiler for every
canonical class and checked against the definitions it encodes: per axis, every output appears
exactly once; the outputs of group w = (i0, i1, i2, i3) are those whose four centres have those
components along the axis; the two offsets of an entry point at the output's components along
the other two axes in the layout of the extended 2-D integrals ([a][c][b][d], index ranges
L + 2, (b, d) blocks padded to an odd length)."""
import itertools
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2303_13632_gb300 import perfmodel as P

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                      "paper_2303_13632_gb300", "csrc", "eri_bwd_table.h")
CANON = sorted({P.canonical(c) for c in itertools.product(range(4), repeat=4)})


def cartesian(L):
    """Components (x, y, z) of a shell in output order: x from L down, then y from L - x down."""
    return [(lx, ly, L - lx - ly) for lx in range(L, -1, -1) for ly in range(L - lx, -1, -1)]


@pytest.fixture(scope="module")
def tables(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("bwdtab")
    body = ["#include <cstdio>", f'#include "{HEADER}"', "template <int A, int B, int C, int D> void dump() {",
            "    static const auto t = eri::make_bwd_tab<A, B, C, D>();",
            "    using T = eri::BwdTab<A, B, C, D>;",
            '    std::printf("class %d %d %d %d %d %d\\n", A, B, C, D, T::N, T::WN);',
            '    for (int w = 0; w <= T::WN; ++w) std::printf("%d\\n", (int)t.start[w]);',
            '    for (int i = 0; i < 3 * T::N; ++i) std::printf("%llu\\n", t.e[i]);', "}", "int main() {"]
    body += [f"    dump<{a}, {b}, {c}, {dd}>();" for a, b, c, dd in CANON] + ["}"]
    src, exe = d / "dump.cpp", d / "dump"
    src.write_text("\n".join(body) + "\n")
    subprocess.run([cxx, "-std=c++17", "-O1", str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    res, i = {}, 0
    while i < len(out) and out[i]:
        _, a, b, c, dd, n, wn = out[i].split()
        a, b, c, dd, n, wn = map(int, (a, b, c, dd, n, wn))
        start = np.array(out[i + 1:i + 2 + wn], dtype=np.int64)
        e = np.array(out[i + 2 + wn:i + 2 + wn + 3 * n], dtype=np.uint64)
        res[(a, b, c, dd)] = (n, wn, start, e)
        i += 2 + wn + 3 * n
    return res


def test_every_canonical_class_is_tabulated(tables):
    assert sorted(tables) == CANON and len(CANON) == 55


@pytest.mark.parametrize("cls", CANON, ids=lambda c: "".join("spdf"[x] for x in c))
def test_table_encodes_the_grouped_contraction(tables, cls):
    A, B, C, D = cls
    n, wn, start, e = tables[cls]
    Ls = (A, B, C, D)
    comps = [cartesian(L) for L in Ls]
    nb, nc, nd = len(comps[1]), len(comps[2]), len(comps[3])
    assert n == len(comps[0]) * nb * nc * nd and wn == (A + 1) * (B + 1) * (C + 1) * (D + 1)
    lc1, ld1 = C + 3, D + 3  # extended ranges L + 2 of the c and d indices
    jl = (B + 3) * (D + 3)
    jlp = jl if jl % 2 else jl + 1
    assert start[0] == 0 and start[-1] == n and np.all(np.diff(start) >= 0)
    for x in range(3):
        y, z = (x + 1) % 3, (x + 2) % 3
        seen = np.zeros(n, dtype=np.int64)
        for w in range(wn):
            i3, i2, i1, i0 = w % (D + 1), (w // (D + 1)) % (C + 1), (w // ((D + 1) * (C + 1))) % (B + 1), \
                w // ((D + 1) * (C + 1) * (B + 1))
            ws = (i0, i1, i2, i3)
            assert start[w + 1] - start[w] == np.prod([L - i + 1 for L, i in zip(Ls, ws)])
            for v in e[x * n + start[w]:x * n + start[w + 1]]:
                v = int(v)
                g, yo, zo = v & 0xFFFF, (v >> 16) & 0xFFFF, v >> 32
                seen[g] += 1
                ia, ib, ic, idd = g // (nb * nc * nd), (g // (nc * nd)) % nb, (g // nd) % nc, g % nd
                ca, cb, cc, cd = comps[0][ia], comps[1][ib], comps[2][ic], comps[3][idd]
                assert (ca[x], cb[x], cc[x], cd[x]) == ws
                assert yo == (ca[y] * lc1 + cc[y]) * jlp + cb[y] * ld1 + cd[y]
                assert zo == (ca[z] * lc1 + cc[z]) * jlp + cb[z] * ld1 + cd[z]
        assert np.all(seen == 1), (cls, x)
