"""Classes with a g shell (L = 4): the run-time-L kernel of the library against the oracle.

* FP64 ERIs of all 369 classes with a g shell (the oracle's McMurchie-Davidson values, pinned
  against its Obara-Saika route and invariants in test_oracle_eri.py) within 1e-12 Ha or 1e-10
  relative, primitive and contracted shells, with and without the pair table;
* 16-bit codes of the FP64 path within +-1 of the oracle's quantisation and eps equal up to one
  FP32 step, for 12, 16 and 20 bits;
* the mixed path (FP32 recurrences, FP64 sums over primitives) below MIXED_G_BOUND of each
  quartet's b_max, and after calibration within one quantisation step of the oracle;
* the compressed output of many [gg|gg] quartets, which the library computes in several
  chunks of its scratch buffer, against the plan's own FP64 output (every quartet: codes within
  half a step, eps from b_max, zero padding);
* the batched form with g and non-g classes in one plan equal to the per-class launches;
* Schwarz screening with the 8-fold unique enumeration on a basis with g shells against brute
  force with the oracle's Schwarz factors;
* the entry points that do not serve g shells return ERI_E_UNSUPPORTED.
"""
import itertools

import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import gpu_compressed, gpu_fp64
from paper_2303_13632_gb300 import _lib, api, workloads as W

pytestmark = pytest.mark.gpu

LS = (0, 1, 2, 3, 4)
G_CLASSES = [c for c in itertools.product(LS, repeat=4) if 4 in c]
# FP32 error of the mixed run-time-L kernel relative to the quartet's b_max (B and C rounded to
# FP32 once, four-index recursion and quadrature in FP32).  One 16-bit quantisation step is
# 1 / 32767 = 3.05e-5.
MIXED_G_BOUND = 1e-5


def fp64_ok(gpu, ref):
    err = np.abs(gpu - ref)
    return (err <= 1e-12) | ((np.abs(ref) > 1e-8) & (err <= 1e-10 * np.abs(ref)))


def per_class_count(cls):
    n = W.quartet_size(*cls)
    return 3 if n <= 2000 else (2 if n <= 20000 else 1)


@pytest.fixture(scope="module")
def g_workload():
    rng = np.random.default_rng(444)
    pool = W.random_primitive_pool(rng, 4, Ls=LS)
    q = np.concatenate([W.random_class_quartets(rng, c, per_class_count(c), 4, Ls=LS) for c in G_CLASSES])
    q = q[rng.permutation(len(q))]
    vals, offs = oracle.eri_batch(pool, q)
    ref = [vals[offs[i]:offs[i + 1]] for i in range(len(q))]
    return pool, q, ref


@pytest.mark.parametrize("pair_table", [True, False])
def test_fp64_all_g_classes(g_workload, pair_table):
    pool, q, ref = g_workload
    got, plan = gpu_fp64(pool, q, "fp64", pair_table=pair_table)
    bad = {}
    for i in range(len(q)):
        if not np.all(fp64_ok(got[i], ref[i])):
            cls = tuple(int(pool.L[s]) for s in q[i])
            bad[cls] = float(np.max(np.abs(got[i] - ref[i])))
    assert not bad, bad
    counts = {c: api.eri_plan_class_info(plan, W.class_id(*c))[0] for c in G_CLASSES}
    assert all(v > 0 for v in counts.values())


@pytest.mark.parametrize("bits", [12, 16, 20])
def test_fp64_codes_g_classes(g_workload, bits):
    pool, q, ref = g_workload
    codes, eps, _ = gpu_compressed(pool, q, bits, "fp64")
    for i in range(len(q)):
        rq, reps = oracle.compress_quartet(ref[i], bits)
        assert np.max(np.abs(codes[i].astype(np.int64) - rq)) <= 1, i
        assert abs(float(eps[i]) - float(reps)) <= 1.2e-7 * float(reps) + 1e-300, i


def test_mixed_g_classes(g_workload):
    pool, q, ref = g_workload
    got, _ = gpu_fp64(pool, q, "mixed")
    worst = {}
    for i in range(len(q)):
        bmax = float(np.max(np.abs(ref[i])))
        if bmax > 1e-30:
            cls = tuple(int(pool.L[s]) for s in q[i])
            worst[cls] = max(worst.get(cls, 0.0), float(np.max(np.abs(got[i] - ref[i]))) / bmax)
    print("worst mixed error / b_max:", max(worst.values()), max(worst, key=worst.get))
    assert max(worst.values()) <= MIXED_G_BOUND, sorted(worst.items(), key=lambda kv: -kv[1])[:5]


def test_mixed_g_calibrated_16bit(g_workload):
    pool, q, ref = g_workload
    plan = api.eri_plan_create(pool, q, precision="mixed")
    api.eri_plan_calibrate_precision(plan, 16, sample=1 << 20, max_err_steps=0.5)
    nb, sb = api.eri_output_bytes(plan, 16)
    packed = torch.full((max(1, nb // 4),), -1, dtype=torch.int32, device="cuda")
    scales = torch.full((max(1, sb // 4),), -1.0, dtype=torch.float32, device="cuda")
    api.eri_compute_compressed(plan, 16, packed, scales)
    api.eri_sync(plan)
    words = packed.cpu().numpy().view(np.uint32)
    eps_sorted = scales.cpu().numpy()
    order = api.eri_plan_quartet_order(plan)
    for c in G_CLASSES:
        cls = W.class_id(*c)
        nq, neri, first, _ = api.eri_plan_class_info(plan, cls)
        off, seg = api.eri_packed_class_offset(plan, 16, cls)
        vals = oracle.unpack_bits(words[off // 4:(off + seg) // 4], nq * neri, 16)
        for k in range(nq):
            i = order[first + k]
            e = float(eps_sorted[first + k])
            x = vals[k * neri:(k + 1) * neri].astype(np.float64) * e
            assert np.all(np.abs(x - ref[i]) <= e * (1.0 + 1e-5) + 1e-30), (c, k)


def test_contracted_g_classes():
    rng = np.random.default_rng(445)
    pool = W.random_contracted_pool(rng, 3, K=2, Ls=LS)
    classes = [(4, 0, 0, 0), (4, 1, 2, 0), (3, 4, 1, 1), (2, 2, 4, 4), (4, 4, 1, 0), (0, 4, 3, 3)]
    q = np.concatenate([W.random_class_quartets(rng, c, 2, 3, Ls=LS) for c in classes])
    vals, offs = oracle.eri_batch(pool, q)
    got, _ = gpu_fp64(pool, q, "fp64")
    for i in range(len(q)):
        assert np.all(fp64_ok(got[i], vals[offs[i]:offs[i + 1]])), i
    got, _ = gpu_fp64(pool, q, "mixed")
    for i in range(len(q)):
        ref = vals[offs[i]:offs[i + 1]]
        bmax = float(np.max(np.abs(ref)))
        assert np.max(np.abs(got[i] - ref)) <= MIXED_G_BOUND * bmax + 1e-30, i


def test_many_gggg_quartets_in_chunks():
    """1700 [gg|gg] quartets: more than one chunk of the scratch buffer (1536 quartets of 50625
    FP64 values each); every quartet's codes against the plan's own FP64 values (half a step
    plus the FP32 rounding of eps), eps against b_max, the padding zero; a sample against the
    oracle."""
    rng = np.random.default_rng(446)
    pool = W.random_primitive_pool(rng, 6, Ls=(4,), box=2.0)
    q = rng.integers(0, 6, size=(1700, 4)).astype(np.int32)
    plan = api.eri_plan_create(pool, q)
    nbf, _ = api.eri_output_bytes(plan, 0)
    out = torch.empty(nbf // 8, dtype=torch.float64, device="cuda")
    api.eri_compute(plan, out)
    nb, sb = api.eri_output_bytes(plan, 16)
    packed = torch.full((nb // 4,), -1, dtype=torch.int32, device="cuda")
    scales = torch.full((sb // 4,), -1.0, dtype=torch.float32, device="cuda")
    api.eri_compute_compressed(plan, 16, packed, scales)
    api.eri_sync(plan)
    x = out.cpu().numpy().reshape(1700, 50625)
    eps = scales.cpu().numpy()
    words = packed.cpu().numpy().view(np.uint32)
    codes = oracle.unpack_bits(words, 1700 * 50625, 16).reshape(1700, 50625)
    bmax = np.max(np.abs(x), axis=1)
    np.testing.assert_array_equal(eps, (bmax / 32767.0).astype(np.float32))
    err = np.abs(codes * eps[:, None].astype(np.float64) - x)
    assert np.all(err <= eps[:, None] * 0.5 * (1 + 1e-6) + 1e-300)
    tail = 1700 * 50625 * 16
    assert np.all(words[(tail + 31) // 32:] == 0)
    order = api.eri_plan_quartet_order(plan)
    pick = [0, 1535, 1536, 1699]
    vals, offs = oracle.eri_batch(pool, q[order[pick]])
    for k, i in enumerate(pick):
        assert np.all(fp64_ok(x[i], vals[offs[k]:offs[k + 1]])), i


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batched_with_g_equals_per_class(precision):
    rng = np.random.default_rng(447)
    pool = W.random_primitive_pool(rng, 4, Ls=LS)
    classes = [(1, 1, 0, 0), (3, 2, 1, 0), (4, 0, 0, 0), (4, 2, 1, 1), (2, 4, 4, 0), (4, 4, 4, 4)]
    q = np.concatenate([W.random_class_quartets(rng, c, 40, 4, Ls=LS) for c in classes])
    plan = api.eri_plan_create(pool, q, precision=precision)
    outs = []
    for batched in (False, True):
        nb, sb = api.eri_output_bytes(plan, 16)
        packed = torch.full((nb // 4,), -1, dtype=torch.int32, device="cuda")
        scales = torch.full((sb // 4,), -1.0, dtype=torch.float32, device="cuda")
        if batched:
            api.eri_autotune(plan, 16, packed, scales, None)
            api.eri_compute_compressed_batched(plan, 16, packed, scales)
        else:
            api.eri_compute_compressed(plan, 16, packed, scales)
        api.eri_sync(plan)
        outs.append((packed.cpu().numpy(), scales.cpu().numpy()))
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    np.testing.assert_array_equal(outs[0][1], outs[1][1])


def test_screening_with_g_shells():
    sh = W.molecule_basis(n_atoms=3, box=6.0, shells_per_atom=(0, 2, 4), kmax=2, seed_k=20)
    n = sh.n
    pairs = np.array([(i, j) for i in range(n) for j in range(i + 1)], dtype=np.int32)
    qd = np.stack([pairs[:, 0], pairs[:, 1], pairs[:, 0], pairs[:, 1]], axis=1)
    vals, offs = oracle.eri_batch(sh, qd)
    Q = np.array([np.sqrt(np.max(np.abs(vals[offs[i]:offs[i + 1]]))) for i in range(len(qd))])
    prods = np.sort(np.outer(Q, Q).ravel())
    tau = 1e-6
    while np.min(np.abs(prods - tau)) <= 1e-8 * tau:
        tau *= 1.0137
    expect = {frozenset([tuple(sorted(pairs[P])), tuple(sorted(pairs[R]))])
              for P, R in itertools.combinations_with_replacement(range(len(pairs)), 2) if Q[P] * Q[R] >= tau}
    plan = api.eri_plan_create(sh, None, mode="unique8", schwarz_threshold=tau)
    got = api.eri_plan_quartets(plan)
    keys = [frozenset([tuple(sorted((int(r[0]), int(r[1])))), tuple(sorted((int(r[2]), int(r[3]))))]) for r in got]
    assert len(keys) == len(set(keys)) and set(keys) == expect
    assert any(4 in (int(sh.L[s]) for s in r) for r in got)


def test_unsupported_entry_points_for_g():
    rng = np.random.default_rng(448)
    pool = W.random_primitive_pool(rng, 2, Ls=LS)
    q = W.random_class_quartets(rng, (4, 1, 0, 0), 3, 2, Ls=LS)
    plan = api.eri_plan_create(pool, q)
    nbf = api.eri_plan_num_basis_functions(plan)
    G = torch.zeros(3 * 45, dtype=torch.float64, device="cuda")
    dR = torch.zeros((pool.n, 3), dtype=torch.float64, device="cuda")
    da = torch.zeros(len(pool.exps), dtype=torch.float64, device="cuda")
    with pytest.raises(api.EriError) as e:
        api.eri_backward(plan, G, dR, da)
    assert e.value.status == _lib.ERI_E_UNSUPPORTED
    nb, sb = api.eri_output_bytes(plan, 16)
    packed = torch.zeros(nb // 4, dtype=torch.int32, device="cuda")
    scales = torch.zeros(sb // 4, dtype=torch.float32, device="cuda")
    D = torch.zeros((nbf, nbf), dtype=torch.float64, device="cuda")
    J, K = torch.zeros_like(D), torch.zeros_like(D)
    with pytest.raises(api.EriError) as e:
        api.eri_digest_jk(plan, 16, packed, scales, D, J, K)
    assert e.value.status == _lib.ERI_E_UNSUPPORTED
    cls = W.class_id(4, 1, 0, 0)
    z = lambda n, dt: torch.zeros(n, dtype=dt, device="cuda")
    dev = (z(pool.n, torch.float64), z(pool.n, torch.float64), z(pool.n, torch.float64),
           z(pool.n, torch.int32), z(pool.n, torch.int32), z(len(pool.exps), torch.float64),
           z(len(pool.exps), torch.float64))
    with pytest.raises(api.EriError) as e:
        api.eri_compute_class_noalloc(cls, "fp64", *dev, z((3, 4), torch.int32), z(3 * 45, torch.float64),
                                      z(1, torch.int32))
    assert e.value.status == _lib.ERI_E_UNSUPPORTED


def test_engine_quartet_arrays():
    """The libint-style Engine: per-quartet arrays (n_a, n_b, n_c, n_d) in the caller's order,
    classes with and without a g shell, against the oracle's quartets."""
    rng = np.random.default_rng(449)
    pool = W.random_primitive_pool(rng, 3, Ls=LS)
    classes = [(0, 0, 0, 0), (2, 1, 3, 0), (4, 0, 1, 2), (1, 4, 4, 0), (3, 3, 3, 3)]
    q = np.concatenate([W.random_class_quartets(rng, c, 2, 3, Ls=LS) for c in classes])
    q = q[rng.permutation(len(q))]
    got = api.Engine(pool).compute(q)
    for i, row in enumerate(q):
        ref = oracle.eri_quartet(pool, [int(x) for x in row])
        assert got[i].shape == ref.shape, i
        assert np.all(fp64_ok(got[i].ravel(), ref.ravel())), i
