"""CPU oracle for the ERI hot path of arXiv 2303.13632 (FP64, plain and slow).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product library never
imports this package and this package never imports the product library; the two
share only the seeded input generators, which hold none of the method's arithmetic.

The C source ``eri_oracle.c`` evaluates Eq. 1 (the ERI definition) through two
independent exact-in-principle routes named in Sec. II-C (Obara-Saika/Head-Gordon-
Pople and McMurchie-Davidson), the Boys function, the compression of Sec. II-D
(Eqs. 9-11) and the centre/exponent gradients.  This module compiles it with gcc
on first use and wraps it with ctypes.
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess
import threading

import numpy as np

from . import classes  # noqa: F401  (paper trip-count model, Sec. III-C/III-D)

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "eri_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_lock = threading.Lock()
_lib = None


def build() -> str:
    """Compiles the oracle shared library (cached by source hash); returns its path."""
    with open(_SRC, "rb") as f:
        digest = hashlib.sha1(f.read()).hexdigest()[:12]
    os.makedirs(_BUILD, exist_ok=True)
    so = os.path.join(_BUILD, f"liberi_oracle_{digest}.so")
    if not os.path.exists(so):
        tmp = so + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, so)
    return so


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        d = ctypes.c_double
        i32 = ctypes.c_int32
        i64 = ctypes.c_int64
        p = ctypes.c_void_p
        lib.orc_norm.restype = d
        lib.orc_norm.argtypes = [d, ctypes.c_int]
        lib.orc_boys.restype = None
        lib.orc_boys.argtypes = [ctypes.c_int, d, p]
        lib.orc_eri_batch.restype = ctypes.c_int
        lib.orc_eri_batch.argtypes = [p, p, p, p, p, p, p, i64, p, p, ctypes.c_int, ctypes.c_int]
        lib.orc_eri_grad_batch.restype = ctypes.c_int
        lib.orc_eri_grad_batch.argtypes = [p, p, p, p, p, p, p, i64, p, p, p, p]
        lib.orc_compress_quartet.restype = None
        lib.orc_compress_quartet.argtypes = [p, i64, ctypes.c_int, p, p]
        lib.orc_decompress_quartet.restype = None
        lib.orc_decompress_quartet.argtypes = [p, i64, ctypes.c_float, p]
        lib.orc_pack_bits.restype = None
        lib.orc_pack_bits.argtypes = [p, i64, ctypes.c_int, p]
        lib.orc_unpack_bits.restype = None
        lib.orc_unpack_bits.argtypes = [p, i64, ctypes.c_int, p]
        lib.orc_rys_roots.restype = ctypes.c_int
        lib.orc_rys_roots.argtypes = [ctypes.c_int, d, p, p]
        lib.orc_digest_jk.restype = None
        lib.orc_digest_jk.argtypes = [p, p, p, i64, p, p, i64, p, p, p]
        lib.orc_pack_paper512.restype = None
        lib.orc_pack_paper512.argtypes = [p, i64, i64, ctypes.c_int, p]
        lib.orc_unpack_paper512.restype = None
        lib.orc_unpack_paper512.argtypes = [p, i64, i64, ctypes.c_int, p]
        lib.orc_max_threads.restype = ctypes.c_int
        lib.orc_max_threads.argtypes = []
        lib.orc_ncart.restype = ctypes.c_int
        lib.orc_ncart.argtypes = [ctypes.c_int]
        _ = i32
        _lib = lib
        return lib


def _ptr(a: np.ndarray) -> ctypes.c_void_p:
    return ctypes.c_void_p(a.ctypes.data)


def ncart(L: int) -> int:
    """Shell size n_g = (L+1)(L+2)/2 (Sec. II-A)."""
    return (L + 1) * (L + 2) // 2


def cart_components(L: int) -> list[tuple[int, int, int]]:
    """Cartesian components of a shell: a_x from L down to 0, then a_y from L-a_x down to 0."""
    return [(ax, ay, L - ax - ay) for ax in range(L, -1, -1) for ay in range(L - ax, -1, -1)]


def norm(alpha: float, L: int) -> float:
    """Axis-aligned normalisation N(alpha, L) of Sec. II-A."""
    return _load().orc_norm(float(alpha), int(L))


def boys(mmax: int, T: float) -> np.ndarray:
    """F_m(T) for m = 0..mmax."""
    out = np.zeros(mmax + 1)
    _load().orc_boys(int(mmax), float(T), _ptr(out))
    return out


class _Table:
    """Contiguous views of a shell set (centres, L, nprim, prim offsets, exps, coefs)."""

    def __init__(self, shells):
        self.centers = np.ascontiguousarray(shells.centers, dtype=np.float64)
        self.L = np.ascontiguousarray(shells.L, dtype=np.int32)
        self.nprim = np.ascontiguousarray(shells.nprim, dtype=np.int32)
        self.pofs = np.ascontiguousarray(shells.pofs, dtype=np.int64)
        self.exps = np.ascontiguousarray(shells.exps, dtype=np.float64)
        self.coefs = np.ascontiguousarray(shells.coefs, dtype=np.float64)

    def args(self):
        return [_ptr(self.centers), _ptr(self.L), _ptr(self.nprim), _ptr(self.pofs),
                _ptr(self.exps), _ptr(self.coefs)]


def quartet_sizes(shells, quartets: np.ndarray) -> np.ndarray:
    L = np.asarray(shells.L)
    q = np.asarray(quartets)
    n = [(L[q[:, x]] + 1) * (L[q[:, x]] + 2) // 2 for x in range(4)]
    return (n[0] * n[1] * n[2] * n[3]).astype(np.int64)


def eri_batch(shells, quartets: np.ndarray, method: str = "md", nthreads: int = 0):
    """ERIs of each shell quartet (rows of ``quartets``: four shell ids).

    Returns (values, offsets): quartet q occupies values[offsets[q] : offsets[q+1]],
    row major over the four shells' Cartesian components (a slowest, d fastest).
    method "md" = McMurchie-Davidson (the reference for parity: it works only with
    centre differences and, checked against an extended-precision build of this same
    source, keeps about 1e-15 relative accuracy), "os" = Obara-Saika + Head-Gordon-Pople
    (the independent cross-check; its horizontal transfer loses up to two digits for
    well-separated centres), "rys" = the paper's Rys route of Sec. II-C written out (a check
    of the readings of Eqs. 6-8, not a reference).
    """
    lib = _load()
    t = _Table(shells)
    q = np.ascontiguousarray(quartets, dtype=np.int32).reshape(-1, 4)
    sizes = quartet_sizes(t, q)
    offsets = np.zeros(len(q) + 1, dtype=np.int64)
    np.cumsum(sizes, out=offsets[1:])
    out = np.zeros(int(offsets[-1]))
    rc = lib.orc_eri_batch(*t.args(), _ptr(q), len(q), _ptr(offsets), _ptr(out),
                           {"os": 0, "md": 1, "rys": 2}[method], int(nthreads))
    if rc != 0:
        raise ValueError("oracle rejected a quartet")
    return out, offsets


def eri_quartet(shells, quartet, method: str = "md") -> np.ndarray:
    """One shell quartet as a 4-D array [na, nb, nc, nd]."""
    vals, _ = eri_batch(shells, np.asarray(quartet).reshape(1, 4), method)
    L = np.asarray(shells.L)
    return vals.reshape([ncart(int(L[s])) for s in quartet])


def eri_grad_batch(shells, quartets: np.ndarray, G: np.ndarray, offsets: np.ndarray):
    """Gradient of E = sum_q sum_abcd G_q,abcd (ab|cd)_q.

    Returns (dR [n_shells, 3], dalpha [total primitives])."""
    lib = _load()
    t = _Table(shells)
    q = np.ascontiguousarray(quartets, dtype=np.int32).reshape(-1, 4)
    G = np.ascontiguousarray(G, dtype=np.float64)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    dR = np.zeros((len(t.L), 3))
    dalpha = np.zeros(len(t.exps))
    lib.orc_eri_grad_batch(*t.args(), _ptr(q), len(q), _ptr(offsets), _ptr(G), _ptr(dR),
                           _ptr(dalpha))
    return dR, dalpha


def compress_quartet(x: np.ndarray, bits: int):
    """Eqs. 9-10: returns (q int32 array, eps float32)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    q = np.zeros(len(x), dtype=np.int32)
    eps = np.zeros(1, dtype=np.float32)
    _load().orc_compress_quartet(_ptr(x), len(x), int(bits), _ptr(q), _ptr(eps))
    return q, np.float32(eps[0])


def compress_batch(values: np.ndarray, offsets: np.ndarray, bits: int):
    """Per-quartet compression of a batch laid out like eri_batch's output."""
    q = np.zeros(len(values), dtype=np.int32)
    eps = np.zeros(len(offsets) - 1, dtype=np.float32)
    for i in range(len(offsets) - 1):
        a, b = int(offsets[i]), int(offsets[i + 1])
        q[a:b], eps[i] = compress_quartet(values[a:b], bits)
    return q, eps


def decompress_quartet(q: np.ndarray, eps: float) -> np.ndarray:
    """Eq. 11."""
    q = np.ascontiguousarray(q, dtype=np.int32)
    out = np.zeros(len(q))
    _load().orc_decompress_quartet(_ptr(q), len(q), ctypes.c_float(eps), _ptr(out))
    return out


def pack_bits(q: np.ndarray, bits: int) -> np.ndarray:
    """LSB-first little-endian bitstream of n-bit fields (uint32 words)."""
    q = np.ascontiguousarray(q, dtype=np.int32)
    words = np.zeros((len(q) * bits + 31) // 32, dtype=np.uint32)
    _load().orc_pack_bits(_ptr(q), len(q), int(bits), _ptr(words))
    return words


def unpack_bits(words: np.ndarray, count: int, bits: int) -> np.ndarray:
    words = np.ascontiguousarray(words, dtype=np.uint32)
    q = np.zeros(count, dtype=np.int32)
    _load().orc_unpack_bits(_ptr(words), int(count), int(bits), _ptr(q))
    return q


def rys_roots(n: int, T: float):
    """Rys roots x = t^2 and weights (ascending roots) with sum w x^k = F_k(T), k < 2n."""
    x = np.zeros(n)
    w = np.zeros(n)
    if _load().orc_rys_roots(int(n), float(T), _ptr(x), _ptr(w)) != 0:
        raise ValueError("n out of range")
    return x, w


def basis_offsets(shells) -> np.ndarray:
    """First basis function of every shell (shells in order, ncart(L) functions each)."""
    n = np.array([ncart(int(l)) for l in shells.L], dtype=np.int64)
    off = np.zeros(len(n) + 1, dtype=np.int64)
    np.cumsum(n, out=off[1:])
    return off


def digest_jk(shells, quartets: np.ndarray, values: np.ndarray, offsets: np.ndarray, D: np.ndarray):
    """Coulomb J[mu,nu] = sum (mu nu|lam sig) D[lam,sig] and exchange K[mu,lam] =
    sum (mu nu|lam sig) D[nu,sig] over the listed quartets, each counted once as listed;
    values/offsets as eri_batch returns them.  Returns (J, K)."""
    t = _Table(shells)
    bf = basis_offsets(shells)
    nbf = int(bf[-1])
    q = np.ascontiguousarray(quartets, dtype=np.int32).reshape(-1, 4)
    x = np.ascontiguousarray(values, dtype=np.float64)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    D = np.ascontiguousarray(D, dtype=np.float64)
    assert D.shape == (nbf, nbf) and len(off) >= len(q)
    J = np.zeros((nbf, nbf))
    K = np.zeros((nbf, nbf))
    _load().orc_digest_jk(_ptr(x), _ptr(off), _ptr(q), len(q), _ptr(t.L), _ptr(bf), nbf,
                          _ptr(D), _ptr(J), _ptr(K))
    return J, K


# The eight index permutations of (ab|cd) under which a real ERI is invariant (Sec. II-B):
# position i of the permuted quartet holds position PERM8[k][i] of the original.
PERM8 = ((0, 1, 2, 3), (1, 0, 2, 3), (0, 1, 3, 2), (1, 0, 3, 2),
         (2, 3, 0, 1), (3, 2, 0, 1), (2, 3, 1, 0), (3, 2, 1, 0))


def expand_unique8(shells, quartets: np.ndarray, values: np.ndarray, offsets: np.ndarray):
    """Every distinct ordered quartet reachable from the listed ones by the 8-fold symmetry,
    each once, with its ERI block (the listed block with its axes permuted alike).  Applied to
    the unique quartets (a >= b, c >= d, pair ab >= pair cd) it yields every ordered quartet
    once.  Returns (quartets, values, offsets) in the layout of eri_batch."""
    q = np.asarray(quartets).reshape(-1, 4)
    L = np.asarray(shells.L)
    seen = set()
    out_q, blocks = [], []
    for i, row in enumerate(q):
        shape = tuple(ncart(int(L[s])) for s in row)
        block = np.asarray(values[offsets[i]:offsets[i + 1]]).reshape(shape)
        for perm in PERM8:
            t = tuple(int(row[k]) for k in perm)
            if t in seen:
                continue
            seen.add(t)
            out_q.append(t)
            blocks.append(np.transpose(block, perm).ravel())
    off = np.zeros(len(blocks) + 1, dtype=np.int64)
    np.cumsum([len(b) for b in blocks], out=off[1:])
    vals = np.concatenate(blocks) if blocks else np.zeros(0)
    return np.array(out_q, dtype=np.int32).reshape(-1, 4), vals, off


def paper512_chunks(n_eri: int, bits: int) -> int:
    """n_CS = ceil(n_ERIQ / floor(512/n)) 512-bit chunks per quartet (Sec. III-C)."""
    f = 512 // bits
    return (n_eri + f - 1) // f


def pack_paper512(q: np.ndarray, n_quartets: int, n_eri: int, bits: int) -> np.ndarray:
    """The paper's per-quartet 512-bit output chunks (Sec. III-C), as uint32 words."""
    q = np.ascontiguousarray(q, dtype=np.int32)
    assert len(q) == n_quartets * n_eri
    words = np.zeros(n_quartets * paper512_chunks(n_eri, bits) * 16, dtype=np.uint32)
    _load().orc_pack_paper512(_ptr(q), int(n_quartets), int(n_eri), int(bits), _ptr(words))
    return words


def unpack_paper512(words: np.ndarray, n_quartets: int, n_eri: int, bits: int) -> np.ndarray:
    words = np.ascontiguousarray(words, dtype=np.uint32)
    assert len(words) >= n_quartets * paper512_chunks(n_eri, bits) * 16
    q = np.zeros(n_quartets * n_eri, dtype=np.int32)
    _load().orc_unpack_paper512(_ptr(words), int(n_quartets), int(n_eri), int(bits), _ptr(q))
    return q


def max_threads() -> int:
    return int(_load().orc_max_threads())
