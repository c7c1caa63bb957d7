"""Pins of the oracle's compression (arXiv 2303.13632 Sec. II-D, Eqs. 9-11) and of the
bitstream layout used for n-bit integers."""
import numpy as np
import pytest

import oracle
from paper_2303_13632_gb300 import workloads as W


def test_worked_example(golden):
    for row in golden("compression_worked_example.txt"):
        sep = row.index(";")
        bits, eps = int(row[0]), float(row[1])
        x = np.array([float(v) for v in row[2:sep]])
        expected = np.array([int(v) for v in row[sep + 1:]])
        q, e = oracle.compress_quartet(x, bits)
        assert e == np.float32(eps)
        np.testing.assert_array_equal(q, expected)
        xt = oracle.decompress_quartet(q, e)
        assert np.all(np.abs(x - xt) <= eps / 2)


@pytest.mark.parametrize("bits", [2, 3, 8, 12, 16, 20, 23, 24])
def test_bound_and_full_range(bits):
    """|x - q eps| <= eps / 2 (the ANINT rounding error) and max |q| = 2^{n-1} - 1."""
    rng = np.random.default_rng(bits)
    M = 2 ** (bits - 1) - 1
    for _ in range(50):
        n = int(rng.integers(1, 400))
        x = rng.standard_normal(n) * 10.0 ** rng.uniform(-8, 1)
        q, e = oracle.compress_quartet(x, bits)
        assert np.max(np.abs(q)) == M
        xt = oracle.decompress_quartet(q, e)
        # eps is stored as FP32; q is taken against the stored eps, so the bound is exact
        # up to the FP64 rounding of x / eps and q * eps.
        assert np.all(np.abs(x - xt) <= float(e) / 2 * (1 + 1e-12))


def test_subnormal_scale():
    """A quartet whose eps = b_max / M is below the smallest normal FP32 number keeps the
    ANINT rounding of Eq. 10 against the stored (subnormal) eps; codes stay within +-M."""
    x = np.array([3e-40, -1e-40, 2e-41])
    q, e = oracle.compress_quartet(x, 16)
    assert 0 < e < np.finfo(np.float32).tiny
    assert np.max(np.abs(q)) <= 2 ** 15 - 1


def test_zero_quartet():
    q, e = oracle.compress_quartet(np.zeros(7), 16)
    assert e == 0.0 and np.all(q == 0)


@pytest.mark.parametrize("bits", [8, 16, 32])
def test_pack_byte_aligned_matches_plain_arrays(bits):
    """For n = 8/16/32 the LSB-first little-endian stream is the plain int array."""
    rng = np.random.default_rng(3)
    M = 2 ** (bits - 1) - 1
    q = rng.integers(-M, M + 1, size=257).astype(np.int32)
    words = oracle.pack_bits(q, bits)
    plain = q.astype({8: np.int8, 16: np.int16, 32: np.int32}[bits]).tobytes()
    assert words.tobytes()[: len(plain)] == plain


def test_pack_12bit_hand_example():
    """Fields 0x123, -1 (0xFFF), 0x7FF, -2048 (0x800) in a 12-bit stream."""
    q = np.array([0x123, -1, 0x7FF, -2048], dtype=np.int32)
    words = oracle.pack_bits(q, 12)
    bits = 0
    for i, v in enumerate([0x123, 0xFFF, 0x7FF, 0x800]):
        bits |= v << (12 * i)
    expected = np.array([(bits >> (32 * k)) & 0xFFFFFFFF for k in range(2)], dtype=np.uint32)
    np.testing.assert_array_equal(words, expected)
    np.testing.assert_array_equal(oracle.unpack_bits(words, 4, 12), q)


@pytest.mark.parametrize("bits", [2, 5, 12, 20, 27])
def test_pack_roundtrip(bits):
    rng = np.random.default_rng(bits + 100)
    M = 2 ** (bits - 1) - 1
    q = rng.integers(-M, M + 1, size=1000).astype(np.int32)
    np.testing.assert_array_equal(oracle.unpack_bits(oracle.pack_bits(q, bits), len(q), bits), q)


def test_paper_accuracy_magnitudes_on_lattice_sample():
    """Sec. IV-D: after decompression the maximum absolute error is about 1e-7..1e-5 Ha at
    16 bit and 1e-5..1e-4 Ha at 12 bit (except [ss|ss]) on the lattice benchmark.  Soft check
    on a subsample of the lattice: the error never exceeds eps/2 and lands in those decades.
    [ss|ss] is the paper's exception: its single ERI equals b_max and is coded exactly as
    +-M, so only the FP32 rounding of eps remains."""
    sh = W.lattice_shells()
    rng = np.random.default_rng(5)
    for cls in [(0, 0, 0, 0), (1, 1, 1, 1), (2, 1, 2, 1), (3, 3, 2, 2)]:
        allq = W.lattice_class_quartets(cls)
        # quartets on few sites carry the largest b_max; include them
        near = allq[(allq[:, 0] // 4 == allq[:, 1] // 4) & (allq[:, 2] // 4 == allq[:, 3] // 4)]
        pick = np.concatenate([near[rng.choice(len(near), 40, replace=False)],
                               allq[rng.choice(len(allq), 40, replace=False)]])
        vals, offs = oracle.eri_batch(sh, pick)
        for bits, lo, hi in ((16, 1e-8, 3e-5), (12, 1e-6, 5e-4)):
            q, eps = oracle.compress_batch(vals, offs, bits)
            err = 0.0
            for i in range(len(pick)):
                a, b = offs[i], offs[i + 1]
                e = np.max(np.abs(vals[a:b] - oracle.decompress_quartet(q[a:b], eps[i])))
                assert e <= eps[i] / 2 * (1 + 1e-12)
                err = max(err, e)
            if cls == (0, 0, 0, 0):
                assert err <= 1e-6 * np.max(np.abs(vals))
            else:
                assert lo <= err <= hi, (cls, bits, err)


# --- the paper's 512-bit output chunks (Sec. III-C, compress-store loops) -------------------

def test_paper512_hand_built_12bit():
    """12-bit fields, worked by hand: F = floor(512/12) = 42 fields (504 bits) per chunk.
    Codes 1, -1, 2047, -2047 fill bits 0-47: word 0 = 0x001 | 0xFFF << 12 | 0xFF << 24, word 1
    = 0x7 | 0x801 << 4.  Field 42 opens the second chunk at bit 0; bits 504-511 of the first
    chunk stay zero."""
    q = np.zeros(43, dtype=np.int32)
    q[:4] = [1, -1, 2047, -2047]
    q[41] = -1   # last field of chunk 0: bits 492-503 -> word 15 bits 12-23
    q[42] = 5
    w = oracle.pack_paper512(q, 1, 43, 12)
    assert len(w) == 32  # n_CS = 2 chunks of 16 words
    assert w[0] == 0xFFFFF001
    assert w[1] == 0x00008017
    assert w[15] == 0x00FFF000  # bits 24-31 of the last word (chunk bits 504-511) are padding
    assert w[16] == 5 and not np.any(w[17:])
    assert not np.any(w[2:15])


@pytest.mark.parametrize("bits", [8, 16, 32])
def test_paper512_byte_widths_are_padded_arrays(bits):
    """For 8-, 16- and 32-bit codes a chunk is a plain little-endian array of 64, 32 or 16
    integers, the last chunk of each quartet zero-padded."""
    rng = np.random.default_rng(bits)
    M = 2 ** (bits - 1) - 1
    dt = {8: np.int8, 16: np.int16, 32: np.int32}[bits]
    per = 512 // bits
    for n_eri in (1, per - 1, per, per + 1, 1000):
        nq = 3
        q = rng.integers(-M, M + 1, size=nq * n_eri).astype(np.int32)
        w = oracle.pack_paper512(q, nq, n_eri, bits)
        ncs = -(-n_eri // per)
        arr = w.view(dt).reshape(nq, ncs * per)
        np.testing.assert_array_equal(arr[:, :n_eri], q.reshape(nq, n_eri))
        assert not np.any(arr[:, n_eri:])


def test_paper512_chunk_count_matches_paper_tables():
    """Chunks per quartet at 16 bit equal the n_CS the paper tabulates (classes.n_cs is pinned
    to Tables III and V), for all 256 classes."""
    from oracle import classes as C
    for c in C.all_classes():
        n_eri = C.n_eriq(*c)
        w = oracle.pack_paper512(np.zeros(2 * n_eri, dtype=np.int32), 2, n_eri, 16)
        assert len(w) == 2 * 16 * C.n_cs(*c, bits=16)
        assert oracle.paper512_chunks(n_eri, 16) == C.n_cs(*c, bits=16)


@pytest.mark.parametrize("bits", [2, 4, 8, 16])
def test_paper512_equals_dense_stream_when_chunks_are_full(bits):
    """When n divides 512 and n_eri is a multiple of 512/n no chunk is padded, so the chunked
    layout is the dense LSB-first stream of the same codes."""
    rng = np.random.default_rng(100 + bits)
    M = 2 ** (bits - 1) - 1
    n_eri = 3 * (512 // bits)
    q = rng.integers(-M, M + 1, size=5 * n_eri).astype(np.int32)
    np.testing.assert_array_equal(oracle.pack_paper512(q, 5, n_eri, bits),
                                  oracle.pack_bits(q, bits))


@pytest.mark.parametrize("bits", [2, 3, 5, 7, 12, 13, 20, 23, 24])
def test_paper512_round_trip_and_padding(bits):
    """unpack(pack(q)) = q, and every bit past a chunk's last field is zero."""
    rng = np.random.default_rng(200 + bits)
    M = 2 ** (bits - 1) - 1
    per = 512 // bits
    for n_eri in (1, 10, per, per + 1, 2 * per + 3, 1000):
        nq = 4
        q = rng.integers(-M, M + 1, size=nq * n_eri).astype(np.int32)
        w = oracle.pack_paper512(q, nq, n_eri, bits)
        np.testing.assert_array_equal(oracle.unpack_paper512(w, nq, n_eri, bits), q)
        ncs = -(-n_eri // per)
        chunks = w.reshape(nq * ncs, 16)
        for ch in range(nq * ncs):
            used = min(per, n_eri - (ch % ncs) * per) * bits
            bitsarr = np.unpackbits(chunks[ch].view(np.uint8), bitorder="little")
            assert not np.any(bitsarr[used:]), (bits, n_eri, ch)
