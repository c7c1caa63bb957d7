"""Long contractions and the batched persistent form against the oracle.

* Shells contracted over K = 4, 5 and 6 primitives on every centre (up to 6^4 = 1296 primitive
  quartets per contracted quartet): FP64 ERIs within 1e-12 Ha / 1e-10 relative, FP64-path
  16-bit codes within +-1 of the oracle's quantisation; the mixed path (FP32 recurrences,
  Kahan-compensated primitive sums) below one 16-bit quantisation step of the oracle once the
  per-class calibration (sample covering every quartet) has moved the classes whose FP32
  error exceeds half a step to FP64, and its uncalibrated FP32 error below the bound stated for
  long contractions.
* A sample of the batched workload (atoms with s, s, p, p, d, f shells, contraction degree
  1..6, unique quartets after Schwarz screening) through eri_autotune and the graph-replayed
  eri_compute_compressed_batched, element by element against the oracle (not only against
  the per-class launches).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2303_13632_gb300 import api, workloads as W

pytestmark = pytest.mark.gpu

# canonical and generic classes from [ss|ss] to [ff|ff]; (count of quartets per K)
CLASSES = [((0, 0, 0, 0), 40), ((1, 0, 1, 0), 40), ((1, 1, 1, 1), 24), ((2, 1, 0, 1), 24),
           ((2, 2, 2, 2), 4), ((3, 2, 1, 1), 4), ((3, 3, 0, 0), 8), ((3, 0, 3, 0), 6),
           ((3, 3, 2, 2), 1), ((0, 1, 3, 2), 4), ((1, 2, 2, 3), 2), ((3, 3, 3, 3), 1)]
# FP32 error of the mixed path relative to the quartet's b_max, uncalibrated, for contraction
# degree up to 6 on every shell.  Measured on the 55 canonical classes (2048 quartets per class
# up to 100 ERIs, 256 above, every shell of degree K): worst 8.0e-7 at K = 1, 4.4e-7, 5.0e-7,
# 4.7e-7, 3.3e-7 and 2.8e-7 at K = 6 -- the Kahan-compensated sum adds nothing visible to the
# per-primitive FP32 rounding.  The bound is the one the primitive sweep is held to; one 16-bit
# quantisation step is 1 / 32767 = 3.05e-5.
MIXED_LONG_BOUND = 4e-6


def fp64_ok(gpu, ref):
    err = np.abs(gpu - ref)
    return (err <= 1e-12) | ((np.abs(ref) > 1e-8) & (err <= 1e-10 * np.abs(ref)))


def contracted_workload(K):
    rng = np.random.default_rng(400 + K)
    pool = W.random_contracted_pool(rng, 8, K=K, Ls=(0, 1, 2, 3))
    q = np.concatenate([W.random_class_quartets(rng, c, n, 8) for c, n in CLASSES])
    return pool, q[rng.permutation(len(q))]


def caller_order(plan, host, sizes):
    """Per-quartet arrays of a class-sorted FP64 output, in the caller's order."""
    order = api.eri_plan_quartet_order(plan)
    out = [None] * len(order)
    pos = 0
    for i, qi in enumerate(order):
        out[qi] = host[pos:pos + sizes[qi]]
        pos += sizes[qi]
    return out


def codes_caller_order(plan, bits, packed, scales, n):
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
    return codes, eps


def fp64_output(plan, n_total):
    stream = torch.cuda.current_stream()
    out = torch.empty(max(1, n_total), dtype=torch.float64, device="cuda")
    api.eri_compute(plan, out, stream)
    api.eri_sync(plan, stream)
    return out.cpu().numpy()


def compressed(plan, bits, batched=False):
    stream = torch.cuda.current_stream()
    nb, sb = api.eri_output_bytes(plan, bits)
    packed = torch.full((max(1, nb // 4),), -1, dtype=torch.int32, device="cuda")
    scales = torch.full((max(1, sb // 4),), -1.0, dtype=torch.float32, device="cuda")
    if batched:
        api.eri_autotune(plan, bits, packed, scales, None, stream)
        packed.fill_(-1)
        scales.fill_(-1.0)
        api.eri_compute_compressed_batched(plan, bits, packed, scales, stream)
        api.eri_compute_compressed_batched(plan, bits, packed, scales, stream)  # graph replay
    else:
        api.eri_compute_compressed(plan, bits, packed, scales, stream)
    api.eri_sync(plan, stream)
    return packed, scales


@pytest.fixture(scope="module", params=[4, 5, 6])
def long_case(request):
    K = request.param
    pool, q = contracted_workload(K)
    vals, offs = oracle.eri_batch(pool, q)
    ref = [vals[offs[i]:offs[i + 1]] for i in range(len(q))]
    return K, pool, q, ref


def test_long_contraction_fp64(long_case):
    K, pool, q, ref = long_case
    sizes = oracle.quartet_sizes(pool, q)
    plan = api.eri_plan_create(pool, q, precision="fp64")
    got = caller_order(plan, fp64_output(plan, int(sizes.sum())), sizes)
    for i in range(len(q)):
        assert np.all(fp64_ok(got[i], ref[i])), (K, i)
    packed, scales = compressed(plan, 16)
    codes, eps = codes_caller_order(plan, 16, packed, scales, len(q))
    for i in range(len(q)):
        rq, reps = oracle.compress_quartet(ref[i], 16)
        assert np.max(np.abs(codes[i].astype(np.int64) - rq)) <= 1, (K, i)
        assert abs(float(eps[i]) - float(reps)) <= 1.2e-7 * float(reps) + 1e-300, (K, i)


def test_long_contraction_mixed(long_case):
    """Uncalibrated FP32 error below the stated long-contraction bound; calibrated 16-bit output
    (every quartet in the calibration sample) within one quantisation step of the oracle."""
    K, pool, q, ref = long_case
    sizes = oracle.quartet_sizes(pool, q)
    plan = api.eri_plan_create(pool, q, precision="mixed")
    got = caller_order(plan, fp64_output(plan, int(sizes.sum())), sizes)
    worst = 0.0
    for i in range(len(q)):
        bmax = float(np.max(np.abs(ref[i])))
        if bmax > 1e-30:
            worst = max(worst, float(np.max(np.abs(got[i] - ref[i]))) / bmax)
    assert worst <= MIXED_LONG_BOUND, (K, worst)
    api.eri_plan_calibrate_precision(plan, 16, sample=1 << 20, max_err_steps=0.5)
    packed, scales = compressed(plan, 16)
    codes, eps = codes_caller_order(plan, 16, packed, scales, len(q))
    for i in range(len(q)):
        xt = codes[i].astype(np.float64) * float(eps[i])
        assert np.all(np.abs(xt - ref[i]) <= float(eps[i]) * (1.0 + 1e-5) + 1e-30), (K, i)
        assert np.max(np.abs(codes[i])) == 32767 or float(eps[i]) < np.finfo(np.float32).tiny


@pytest.fixture(scope="module")
def molecule_sample():
    """Unique Schwarz-screened quartets (ERI_UNIQUE8 at 1e-10, enumerated by the library) of a
    40-atom system with the batched workload's density and shell mix (s, s, p, p, d, f per atom,
    K ~ U{1..6}): an even 1-in-s shard of the enumeration, from which quartets the oracle
    finishes in seconds are drawn, plus quartets whose four shells are all contracted over 4..6
    primitives."""
    basis = W.molecule_basis(n_atoms=40, box=20.0 * (40 / 200) ** (1 / 3), seed_k=41)
    tau = 1e-10
    probe = api.eri_plan_create(basis, None, mode="unique8", schwarz_threshold=tau, shard=(0, 1 << 62))
    _, kept = api.eri_plan_screening(probe)
    probe.destroy()
    shard = api.eri_plan_create(basis, None, mode="unique8", schwarz_threshold=tau,
                                shard=(0, max(1, kept // 20000)))
    rows = api.eri_plan_quartets(shard)
    shard.destroy()
    rng = np.random.default_rng(42)
    nprim = np.asarray(basis.nprim)
    cost = np.prod([nprim[rows[:, x]] for x in range(4)], axis=0) * oracle.quartet_sizes(basis, rows)
    kmin = np.min([nprim[rows[:, x]] for x in range(4)], axis=0)
    cheap = np.nonzero(cost <= 150000)[0]
    long_ = np.nonzero((kmin >= 4) & (cost <= 600000))[0]
    pick = np.union1d(rng.choice(cheap, size=min(400, len(cheap)), replace=False),
                      rng.choice(long_, size=min(12, len(long_)), replace=False))
    q = rows[pick]
    vals, offs = oracle.eri_batch(basis, q)
    return basis, q, [vals[offs[i]:offs[i + 1]] for i in range(len(q))]


def test_molecule_sample_shape(molecule_sample):
    basis, q, _ = molecule_sample
    nprim = np.asarray(basis.nprim)
    kmin = np.min([nprim[q[:, x]] for x in range(4)], axis=0)
    assert np.any(kmin >= 4) and len(q) > 100
    L = np.asarray(basis.L)
    classes = {W.class_id(*[int(L[s]) for s in row]) for row in q}
    assert len(classes) >= 12


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batched_matches_oracle(molecule_sample, precision):
    basis, q, ref = molecule_sample
    plan = api.eri_plan_create(basis, q, precision=precision)
    if precision == "mixed":
        api.eri_plan_calibrate_precision(plan, 16, sample=1 << 20, max_err_steps=0.5)
    packed, scales = compressed(plan, 16, batched=True)
    codes, eps = codes_caller_order(plan, 16, packed, scales, len(q))
    for i in range(len(q)):
        if precision == "fp64":
            rq, reps = oracle.compress_quartet(ref[i], 16)
            assert np.max(np.abs(codes[i].astype(np.int64) - rq)) <= 1, i
            assert abs(float(eps[i]) - float(reps)) <= 1.2e-7 * float(reps) + 1e-300, i
        else:
            xt = codes[i].astype(np.float64) * float(eps[i])
            assert np.all(np.abs(xt - ref[i]) <= float(eps[i]) * (1.0 + 1e-5) + 1e-30), i


def test_molecule_fp64_values(molecule_sample):
    basis, q, ref = molecule_sample
    sizes = oracle.quartet_sizes(basis, q)
    plan = api.eri_plan_create(basis, q, precision="fp64")
    got = caller_order(plan, fp64_output(plan, int(sizes.sum())), sizes)
    for i in range(len(q)):
        assert np.all(fp64_ok(got[i], ref[i])), i
