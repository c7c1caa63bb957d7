"""The single-launch work-queue form (eri_compute_compressed_queue) against the oracle.

One persistent launch serves every class of a plan; its codes are checked element by element:
* all 256 classes of s..f (primitive shells, shuffled) and, in the same plan, classes with a g
  shell: FP64 codes within +-1 of the oracle's quantisation and eps equal up to one FP32 step;
  mixed precision within one quantisation step of the oracle after decompression;
* a sample of the batched workload (device-enumerated, screened unique quartets of a 40-atom
  system with the s, s, p, p, d, f mix, contraction degree up to 6) in both precisions;
* against the per-class launches (codes within +-1, eps within one FP32 step) and across two
  calls (the output is zeroed by the call).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2303_13632_gb300 import _lib, api, workloads as W

pytestmark = pytest.mark.gpu


def queue_codes(plan, q, bits, queue=True):
    nb, sb = api.eri_output_bytes(plan, bits)
    packed = torch.full((max(1, nb // 4),), -1, dtype=torch.int32, device="cuda")
    scales = torch.full((max(1, sb // 4),), -1.0, dtype=torch.float32, device="cuda")
    if queue:
        api.eri_compute_compressed_queue(plan, bits, packed, scales)
    else:
        api.eri_compute_compressed(plan, bits, packed, scales)
    api.eri_sync(plan)
    words = packed.cpu().numpy().view(np.uint32)
    eps_sorted = scales.cpu().numpy()
    order = api.eri_plan_quartet_order(plan)
    codes, eps = [None] * len(q), np.zeros(len(q), dtype=np.float32)
    for cls in range(_lib.ERI_NUM_CLASS_IDS):
        if W.class_id(*W.class_of_id(cls)) != cls:
            continue
        nq, neri, first, _ = api.eri_plan_class_info(plan, cls)
        if nq == 0:
            continue
        off, seg = api.eri_packed_class_offset(plan, bits, cls)
        seg_words = words[off // 4:(off + seg) // 4]
        vals = oracle.unpack_bits(seg_words, nq * neri, bits)
        tail = nq * neri * bits
        assert np.all(seg_words[(tail + 31) // 32:] == 0), cls
        for i in range(nq):
            codes[order[first + i]] = vals[i * neri:(i + 1) * neri]
            eps[order[first + i]] = eps_sorted[first + i]
    return codes, eps


@pytest.fixture(scope="module")
def sf_g_workload():
    # one pool with s..g shells: every class of s..f plus classes with a g shell
    rng = np.random.default_rng(94)
    Ls = (0, 1, 2, 3, 4)
    pool = W.random_primitive_pool(rng, 8, Ls=Ls)
    classes = [W.class_of_id(c) for c in range(256)] + [(4, 0, 0, 0), (4, 2, 1, 3), (0, 4, 4, 1), (4, 4, 2, 2)]
    q = np.concatenate([W.random_class_quartets(rng, c, 4 if W.quartet_size(*c) > 1000 else 12, 8, Ls=Ls)
                        for c in classes])
    q = q[rng.permutation(len(q))]
    vals, offs = oracle.eri_batch(pool, q)
    return pool, q, [vals[offs[i]:offs[i + 1]] for i in range(len(q))]


@pytest.mark.parametrize("bits", [16, 12])
def test_queue_fp64_codes(sf_g_workload, bits):
    pool, q, ref = sf_g_workload
    plan = api.eri_plan_create(pool, q, precision="fp64")
    codes, eps = queue_codes(plan, q, bits)
    for i in range(len(q)):
        rq, reps = oracle.compress_quartet(ref[i], bits)
        assert np.max(np.abs(codes[i].astype(np.int64) - rq)) <= 1, i
        assert abs(float(eps[i]) - float(reps)) <= 1.2e-7 * float(reps) + 1e-300, i


def test_queue_mixed_within_one_step(sf_g_workload):
    pool, q, ref = sf_g_workload
    plan = api.eri_plan_create(pool, q, precision="mixed")
    codes, eps = queue_codes(plan, q, 16)
    for i in range(len(q)):
        x = codes[i].astype(np.float64) * float(eps[i])
        assert np.all(np.abs(x - ref[i]) <= float(eps[i]) * (1 + 1e-5) + 1e-30), i


def test_queue_against_per_class_launches_and_repeat(sf_g_workload):
    pool, q, _ = sf_g_workload
    plan = api.eri_plan_create(pool, q, precision="fp64")
    a_codes, a_eps = queue_codes(plan, q, 16, queue=False)
    b_codes, b_eps = queue_codes(plan, q, 16)
    c_codes, c_eps = queue_codes(plan, q, 16)
    for i in range(len(q)):
        assert np.max(np.abs(a_codes[i].astype(np.int64) - b_codes[i])) <= 1, i
        assert abs(float(a_eps[i]) - float(b_eps[i])) <= 1.2e-7 * float(a_eps[i]) + 1e-300, i
        np.testing.assert_array_equal(b_codes[i], c_codes[i])
    np.testing.assert_array_equal(b_eps, c_eps)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_queue_contracted_molecule_sample(precision):
    basis = W.molecule_basis(n_atoms=40, box=20.0 * (40 / 200) ** (1 / 3), seed_k=41)
    tau = 1e-10
    probe = api.eri_plan_create(basis, None, mode="unique8", schwarz_threshold=tau, shard=(0, 1 << 62))
    _, kept = api.eri_plan_screening(probe)
    probe.destroy()
    shard = api.eri_plan_create(basis, None, mode="unique8", schwarz_threshold=tau, shard=(0, max(1, kept // 20000)))
    rows = api.eri_plan_quartets(shard)
    shard.destroy()
    rng = np.random.default_rng(43)
    nprim = np.asarray(basis.nprim)
    cost = np.prod([nprim[rows[:, x]] for x in range(4)], axis=0) * oracle.quartet_sizes(basis, rows)
    kmin = np.min([nprim[rows[:, x]] for x in range(4)], axis=0)
    cheap = np.nonzero(cost <= 150000)[0]
    long_ = np.nonzero((kmin >= 4) & (cost <= 600000))[0]
    pick = np.union1d(rng.choice(cheap, size=min(300, len(cheap)), replace=False),
                      rng.choice(long_, size=min(10, len(long_)), replace=False))
    q = rows[pick]
    vals, offs = oracle.eri_batch(basis, q)
    plan = api.eri_plan_create(basis, q, precision=precision)
    codes, eps = queue_codes(plan, q, 16)
    for i in range(len(q)):
        ref = vals[offs[i]:offs[i + 1]]
        if precision == "fp64":
            rq, reps = oracle.compress_quartet(ref, 16)
            assert np.max(np.abs(codes[i].astype(np.int64) - rq)) <= 1, i
        else:
            x = codes[i].astype(np.float64) * float(eps[i])
            assert np.all(np.abs(x - ref) <= float(eps[i]) * (1 + 1e-5) + 1e-30), i


def test_queue_empty_plan_and_arguments():
    rng = np.random.default_rng(95)
    pool = W.random_primitive_pool(rng, 2)
    plan = api.eri_plan_create(pool, np.zeros((0, 4), dtype=np.int32))
    api.eri_compute_compressed_queue(plan, 16, None, None)
    plan = api.eri_plan_create(pool, np.array([[0, 1, 2, 3]], dtype=np.int32))
    nb, sb = api.eri_output_bytes(plan, 16)
    packed = torch.zeros(nb // 4, dtype=torch.int32, device="cuda")
    scales = torch.zeros(sb // 4, dtype=torch.float32, device="cuda")
    with pytest.raises(api.EriError):
        api.eri_compute_compressed_queue(plan, 25, packed, scales)
    with pytest.raises(api.EriError):
        api.eri_compute_compressed_queue(plan, 16, None, scales)
