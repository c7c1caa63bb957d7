"""Decompression fused with Coulomb/exchange digestion on the GPU (eri_digest_jk) against the
oracle's digestion (orc_digest_jk, pinned in test_oracle_jk.py by brute force over the full
ERI tensor) of the same decompressed codes, and against the oracle's own FP64 ERIs within the
compression bound carried through the contraction.

Tolerances: the GPU forms each quartet's sums of codes x D in FP32 (sums of at most 100 terms)
and accumulates in FP64, so against the oracle's digestion of the same decompressed values
each element of J and K agrees within 1e-5 of its absolute weight digest(|x~|, |D|) (100 terms
at 2^-24 each, plus the FP32 rounding of D).  Against the exact ERIs the difference is also
bounded by digest(eps/2, |D|) (Eq. 10's ANINT bound, as pinned on the oracle side).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2303_13632_gb300 import api, workloads as W

pytestmark = pytest.mark.gpu


def unique_quartets(n):
    """(a >= b, c >= d, pair ab >= pair cd) over n shells: the 8-fold unique set (Sec. II-B)."""
    pairs = [(a, b) for a in range(n) for b in range(a + 1)]
    return np.array([(a, b, c, d) for i, (a, b) in enumerate(pairs) for (c, d) in pairs[:i + 1]],
                    dtype=np.int32)


def gpu_codes(plan, bits, n, precision_calibrate=False):
    """Compressed output on the device plus its decoded codes and eps in the caller's order."""
    stream = torch.cuda.current_stream()
    nb, sb = api.eri_output_bytes(plan, bits)
    packed = torch.full((max(1, nb // 4),), -1, dtype=torch.int32, device="cuda")
    scales = torch.full((max(1, sb // 4),), -1.0, dtype=torch.float32, device="cuda")
    api.eri_compute_compressed(plan, bits, packed, scales, stream)
    api.eri_sync(plan, stream)
    words = packed.cpu().numpy().view(np.uint32)
    eps_sorted = scales.cpu().numpy()
    order = api.eri_plan_quartet_order(plan)
    codes, eps = [None] * n, np.zeros(n, dtype=np.float32)
    for cls in range(256):
        nq, neri, first, _ = api.eri_plan_class_info(plan, cls)
        if nq == 0:
            continue
        off, seg = api.eri_packed_class_offset(plan, bits, cls)
        vals = oracle.unpack_bits(words[off // 4:(off + seg) // 4], nq * neri, bits)
        for i in range(nq):
            codes[order[first + i]] = vals[i * neri:(i + 1) * neri]
            eps[order[first + i]] = eps_sorted[first + i]
    return packed, scales, codes, eps


def gpu_digest(plan, bits, packed, scales, D, unique8, accumulate_into=None):
    nbf = api.eri_plan_num_basis_functions(plan)
    Dd = torch.tensor(D, dtype=torch.float64, device="cuda")
    if accumulate_into is None:
        J = torch.full((nbf, nbf), float("nan"), dtype=torch.float64, device="cuda")
        K = torch.full((nbf, nbf), float("nan"), dtype=torch.float64, device="cuda")
    else:
        J, K = accumulate_into
    api.eri_digest_jk(plan, bits, packed, scales, Dd, J, K, unique8=unique8,
                      accumulate=accumulate_into is not None)
    api.eri_sync(plan)
    return J, K


def oracle_digest(shells, q, blocks, D, unique8):
    offs = np.zeros(len(q) + 1, dtype=np.int64)
    np.cumsum([len(b) for b in blocks], out=offs[1:])
    vals = np.concatenate(blocks)
    if unique8:
        q, vals, offs = oracle.expand_unique8(shells, q, vals, offs)
    return oracle.digest_jk(shells, q, vals, offs, D)


def check_case(shells, q, bits, precision, unique8, seed):
    rng = np.random.default_rng(seed)
    nbf = int(oracle.basis_offsets(shells)[-1])
    D = rng.standard_normal((nbf, nbf))  # not symmetric: a transposed index would show
    plan = api.eri_plan_create(shells, q, precision=precision)
    assert api.eri_plan_num_basis_functions(plan) == nbf
    packed, scales, codes, eps = gpu_codes(plan, bits, len(q))
    J, K = gpu_digest(plan, bits, packed, scales, D, unique8)
    Jg, Kg = J.cpu().numpy(), K.cpu().numpy()
    # the same decompressed values (Eq. 11) through the oracle
    dec = [codes[i].astype(np.float64) * float(eps[i]) for i in range(len(q))]
    Jr, Kr = oracle_digest(shells, q, dec, D, unique8)
    bJ, bK = oracle_digest(shells, q, [np.abs(d) for d in dec], np.abs(D), unique8)
    assert np.all(np.abs(Jg - Jr) <= 1e-5 * bJ + 1e-300), float(np.max(np.abs(Jg - Jr) - 1e-5 * bJ))
    assert np.all(np.abs(Kg - Kr) <= 1e-5 * bK + 1e-300), float(np.max(np.abs(Kg - Kr) - 1e-5 * bK))
    return plan, packed, scales, D, (Jg, Kg), dec, eps


@pytest.mark.parametrize("bits,precision", [(16, "fp64"), (12, "mixed"), (8, "fp64")])
def test_unique8_all_quartets_small_basis(bits, precision):
    """Every unique quartet of two shells per L (s, s, p, p, d, d, f, f): quartets with repeated
    shells and pairs exercise the removal of coinciding permutations."""
    rng = np.random.default_rng(bits)
    pool = W.random_primitive_pool(rng, 2, Ls=(0, 1, 2, 3), box=2.0)
    q = unique_quartets(pool.n)
    q = q[rng.permutation(len(q))]
    check_case(pool, q, bits, precision, True, seed=bits + 1)


def test_unique8_equals_full_tensor_contraction():
    """On a contracted s, p, d basis the 8-fold digestion of the unique quartets equals the
    oracle's digestion of every ordered quartet of the same decompressed ERIs (to the GPU's FP32
    tolerance), i.e. J and K of the full tensor."""
    rng = np.random.default_rng(21)
    pool = W.random_contracted_pool(rng, 2, K=2, Ls=(0, 1, 2))
    uq = unique_quartets(pool.n)
    plan, packed, scales, D, (Jg, Kg), dec, eps = check_case(pool, uq, 16, "fp64", True, seed=22)
    offs = np.zeros(len(uq) + 1, dtype=np.int64)
    np.cumsum([len(b) for b in dec], out=offs[1:])
    eq, ev, eo = oracle.expand_unique8(pool, uq, np.concatenate(dec), offs)
    assert len(eq) == pool.n ** 4
    Jf, Kf = oracle.digest_jk(pool, eq, ev, eo, D)
    scale = np.max(np.abs(Jf)) + np.max(np.abs(Kf))
    assert np.max(np.abs(Jg - Jf)) <= 1e-6 * scale
    assert np.max(np.abs(Kg - Kf)) <= 1e-6 * scale


def test_against_exact_eris_within_the_compression_bound():
    """GPU ERIs -> 16-bit codes -> GPU digestion against the oracle's FP64 ERIs digested in
    FP64: within digest(eps/2, |D|) plus the FP32 sums' tolerance."""
    rng = np.random.default_rng(31)
    pool = W.random_contracted_pool(rng, 2, K=3, Ls=(0, 1, 2, 3))
    q = unique_quartets(pool.n)
    plan, packed, scales, D, (Jg, Kg), dec, eps = check_case(pool, q, 16, "fp64", True, seed=32)
    vals, offs = oracle.eri_batch(pool, q)
    exact = [vals[offs[i]:offs[i + 1]] for i in range(len(q))]
    Je, Ke = oracle_digest(pool, q, exact, D, True)
    half = [np.full(len(e), float(eps[i]) / 2 * (1 + 1e-6)) for i, e in enumerate(exact)]
    hJ, hK = oracle_digest(pool, q, half, np.abs(D), True)
    aJ, aK = oracle_digest(pool, q, [np.abs(e) for e in exact], np.abs(D), True)
    assert np.all(np.abs(Jg - Je) <= hJ + 1e-5 * aJ + 1e-300)
    assert np.all(np.abs(Kg - Ke) <= hK + 1e-5 * aK + 1e-300)
    assert np.max(np.abs(Jg - Je)) > 0


def test_as_listed_and_accumulate():
    """Without ERI_DIGEST_UNIQUE8 each quartet counts once as listed (ordered quartets drawn at
    random, repeats allowed); ERI_DIGEST_ACCUMULATE adds to the previous J and K."""
    rng = np.random.default_rng(41)
    pool = W.random_primitive_pool(rng, 6, Ls=(0, 1, 2, 3))
    q = rng.integers(0, pool.n, size=(900, 4)).astype(np.int32)
    plan, packed, scales, D, (Jg, Kg), _, _ = check_case(pool, q, 16, "mixed", False, seed=42)
    J = torch.tensor(Jg, device="cuda")
    K = torch.tensor(Kg, device="cuda")
    gpu_digest(plan, 16, packed, scales, D, False, accumulate_into=(J, K))
    np.testing.assert_allclose(J.cpu().numpy(), 2 * Jg, rtol=1e-12, atol=1e-300)
    np.testing.assert_allclose(K.cpu().numpy(), 2 * Kg, rtol=1e-12, atol=1e-300)


@pytest.mark.parametrize("shard", [None, 3])
def test_symmetric_density_mode(shard):
    """ERI_DIGEST_SYMMETRIC (one sum and one atomic per item, then J = (J + J^T) / 2) equals the
    general digestion for a symmetric D, and the oracle's digestion of the same values: on all
    unique quartets and on a subset of them (every third), whose 8-fold images are still closed
    under the index swaps."""
    unique8 = True
    rng = np.random.default_rng(61)
    pool = W.random_contracted_pool(rng, 2, K=2, Ls=(0, 1, 2, 3))
    q = unique_quartets(pool.n)
    if shard:
        q = q[::shard]
    nbf = int(oracle.basis_offsets(pool)[-1])
    D = rng.standard_normal((nbf, nbf))
    D = D + D.T
    plan = api.eri_plan_create(pool, q, precision="mixed")
    packed, scales, codes, eps = gpu_codes(plan, 16, len(q))
    Dd = torch.tensor(D, device="cuda")
    out = {}
    for sym in (False, True):
        J = torch.full((nbf, nbf), float("nan"), dtype=torch.float64, device="cuda")
        K = torch.full_like(J, float("nan"))
        api.eri_digest_jk(plan, 16, packed, scales, Dd, J, K, unique8=unique8, symmetric=sym)
        api.eri_sync(plan)
        out[sym] = (J.cpu().numpy(), K.cpu().numpy())
    dec = [codes[i].astype(np.float64) * float(eps[i]) for i in range(len(q))]
    Jr, Kr = oracle_digest(pool, q, dec, D, unique8)
    bJ, bK = oracle_digest(pool, q, [np.abs(d) for d in dec], np.abs(D), unique8)
    for sym in (False, True):
        Jg, Kg = out[sym]
        assert np.all(np.abs(Jg - Jr) <= 1e-5 * bJ + 1e-300), sym
        assert np.all(np.abs(Kg - Kr) <= 1e-5 * bK + 1e-300), sym
    # J and K of 8-fold closed quartet sets are symmetric for a symmetric D
    np.testing.assert_array_equal(out[True][0], out[True][0].T)
    np.testing.assert_array_equal(out[True][1], out[True][1].T)


def test_digest_rejects_bad_arguments():
    rng = np.random.default_rng(51)
    pool = W.random_primitive_pool(rng, 1, Ls=(0, 1))
    plan = api.eri_plan_create(pool, unique_quartets(pool.n))
    nbf = api.eri_plan_num_basis_functions(plan)
    nb, sb = api.eri_output_bytes(plan, 16)
    packed = torch.zeros(nb // 4, dtype=torch.int32, device="cuda")
    scales = torch.zeros(sb // 4, dtype=torch.float32, device="cuda")
    D = torch.zeros((nbf, nbf), dtype=torch.float64, device="cuda")
    J, K = torch.empty_like(D), torch.empty_like(D)
    for bits in (1, 25):
        with pytest.raises(api.EriError):
            api.eri_digest_jk(plan, bits, packed, scales, D, J, K)
    with pytest.raises(api.EriError):
        api.eri_digest_jk(plan, 16, packed, scales, None, J, K)
    with pytest.raises(api.EriError):  # the symmetric mode needs the 8-fold expansion
        api.eri_digest_jk(plan, 16, packed, scales, D, J, K, unique8=False, symmetric=True)
