"""GPU parity of the CUDA path (through the C ABI) against the CPU oracle.

Tolerances (from the benchmark spec of the target):
  * FP64 ERIs: |gpu - oracle| <= 1e-12 Ha, or <= 1e-10 relative where |ERI| > 1e-8;
  * compressed integers: within +-1 of the oracle's quantisation of its own values, eps
    equal to the oracle's up to one FP32 rounding step;
  * mixed precision (FP32 recurrences): error per quartet below the 16-bit quantisation
    step eps_16 / 2 = b_max / 65534 (the precision study reports the actual values); ERIs
    below the FP32 normal range (quartets with b_max < 1e-30 Ha) may flush to zero, so an
    absolute floor of 1e-30 Ha applies.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle.classes import all_classes
from paper_2303_13632_gb300 import api, workloads as W
from gpu_helpers import gpu_compressed, gpu_fp64

pytestmark = pytest.mark.gpu


def fp64_ok(gpu, ref):
    err = np.abs(gpu - ref)
    ok = (err <= 1e-12) | ((np.abs(ref) > 1e-8) & (err <= 1e-10 * np.abs(ref)))
    return ok


def mixed_workload(seed=7, per_class=None, K=1, coef_range=None):
    """All 256 classes from one shell pool, quartets shuffled so the plan's class sort and
    the stable order within a class are exercised."""
    rng = np.random.default_rng(seed)
    if K == 1:
        pool = W.random_primitive_pool(rng, 24, coef_range=coef_range)
    else:
        pool = W.random_contracted_pool(rng, 12, K=K, Ls=(0, 1, 2, 3))
    qs = []
    for cls in all_classes():
        neri = W.quartet_size(*cls)
        n = per_class(neri) if per_class else max(3, min(300, 60000 // neri))
        qs.append(W.random_class_quartets(rng, cls, n, 24 if K == 1 else 12))
    q = np.concatenate(qs)
    q = q[rng.permutation(len(q))]
    return pool, q


@pytest.fixture(scope="module")
def workload():
    return mixed_workload()


@pytest.fixture(scope="module")
def oracle_values(workload):
    pool, q = workload
    vals, offs = oracle.eri_batch(pool, q)
    return [vals[offs[i]:offs[i + 1]] for i in range(len(q))]


def test_integer_pipe_conversions_match_ieee():
    """The setup stages' binary64 -> binary32 rounding (integer arithmetic) against numpy's
    IEEE casts: random magnitudes across the binary32 range, exact ties at the 29th bit, the
    largest finite values, subnormal results, zeros, infinities and NaN."""
    rng = np.random.default_rng(5)
    x = rng.standard_normal(200000) * np.exp(rng.uniform(-95.0, 95.0, 200000))
    base = rng.integers(0, 2**52, 20000, dtype=np.uint64) & ~np.uint64((1 << 29) - 1)
    expo = rng.integers(897, 1150, 20000, dtype=np.uint64) << np.uint64(52)
    ties = (expo | base | np.uint64(1 << 28)).view(np.float64)  # exactly halfway
    near = (expo | base | np.uint64((1 << 28) - 1)).view(np.float64)
    special = np.array([0.0, -0.0, 1.0, -1.0, 3.4028234663852886e38, 3.4028235677973366e38,
                        3.5e38, 1e300, -1e300, 1.1754943508222875e-38, 1.1754942e-38, 1e-40,
                        1.4e-45, 7e-46, 1e-50, 5e-324, np.inf, -np.inf, np.nan])
    h = np.concatenate([x, ties, -ties, near, special])
    d = torch.as_tensor(h, device="cuda")
    f = torch.empty(len(h), dtype=torch.float32, device="cuda")
    back = torch.empty(len(h), dtype=torch.float64, device="cuda")
    api.eri_convert_device(d, f, back)
    torch.cuda.synchronize()
    with np.errstate(over="ignore"):
        ref = h.astype(np.float32)
    got = f.cpu().numpy()
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32)) or \
        np.array_equal(np.isnan(got), np.isnan(ref)) and \
        np.array_equal(got[~np.isnan(ref)].view(np.uint32), ref[~np.isnan(ref)].view(np.uint32))
    bk = back.cpu().numpy()
    ok = ~np.isnan(ref)
    assert np.array_equal(bk[ok].view(np.uint64), ref[ok].astype(np.float64).view(np.uint64))
    assert np.all(np.isnan(bk[~ok]))


def test_boys_device_matches_oracle():
    Ts = np.concatenate([[0.0, 1e-12, 1e-6, 0.05, 0.0999, 0.1, 0.15, 35.94, 35.96, 36.0, 49.94,
                          49.96, 49.999, 50.0, 50.0001, 1e3, 1e6],
                         np.random.default_rng(1).uniform(0, 60, 400)])
    T = torch.tensor(Ts, dtype=torch.float64, device="cuda")
    F = torch.empty(len(Ts) * 17, dtype=torch.float64, device="cuda")
    api.eri_boys_device(16, T, F)
    torch.cuda.synchronize()
    F = F.cpu().numpy().reshape(-1, 17)
    for i, t in enumerate(Ts):
        ref = oracle.boys(16, float(t))
        np.testing.assert_allclose(F[i], ref, rtol=5e-14, atol=0, err_msg=f"T={t}")


@pytest.mark.parametrize("n", range(1, 10))
def test_rys_roots_reproduce_boys_moments(n):
    """Sec. II-C: the order-n rule integrates x^k against the Rys weight exactly for
    k < 2n, i.e. sum_mu w_mu x_mu^k = F_k(T)."""
    rng = np.random.default_rng(n)
    Ts = np.concatenate([[0.0, 1e-9, 0.5, 1.0, 29.999, 30.0], rng.uniform(0, 100, 300),
                         np.arange(0, 95, 1.0) + 0.999999, [150.0, 1e4]])
    T = torch.tensor(Ts, dtype=torch.float64, device="cuda")
    x = torch.empty(len(Ts) * n, dtype=torch.float64, device="cuda")
    w = torch.empty_like(x)
    api.eri_rys_device(n, T, x, w)
    torch.cuda.synchronize()
    x = x.cpu().numpy().reshape(-1, n)
    w = w.cpu().numpy().reshape(-1, n)
    assert np.all(x > 0) and np.all(x < 1) and np.all(w > 0)
    assert np.all(np.diff(x, axis=1) > 0)
    for i, t in enumerate(Ts):
        F = oracle.boys(2 * n - 1, float(t))
        mom = np.array([np.sum(w[i] * x[i] ** k) for k in range(2 * n)])
        np.testing.assert_allclose(mom, F, rtol=2e-13, atol=0, err_msg=f"T={t}")


@pytest.mark.parametrize("n", range(1, 10))
def test_rys_mixed_setup_evaluation(n):
    """The root/weight evaluation of the mixed-precision setup (FP32 tails, Newton-refined
    reciprocals) agrees with the FP64 evaluation to 1e-8 relative across both branches (the
    polynomial pieces and the Gauss-Hermite limit) and every unit interval of T; its values
    are rounded to FP32 (6e-8) afterwards."""
    rng = np.random.default_rng(100 + n)
    Ts = np.concatenate([[0.0, 1e-9, 0.05, 0.5, 1.0, 29.999, 30.0, 49.99, 50.0, 50.01],
                         rng.uniform(0, 100, 2000), np.arange(0, 95, 1.0) + 0.999999,
                         np.arange(0, 95, 1.0) + 1e-7, [150.0, 1e4, 1e6]])
    T = torch.tensor(Ts, dtype=torch.float64, device="cuda")
    x64, w64 = torch.empty(len(Ts) * n, dtype=torch.float64, device="cuda"), torch.empty(len(Ts) * n, dtype=torch.float64, device="cuda")
    xm, wm = torch.empty_like(x64), torch.empty_like(w64)
    api.eri_rys_device(n, T, x64, w64)
    api.eri_rys_device_mixed(n, T, xm, wm)
    torch.cuda.synchronize()
    for a, b in ((xm, x64), (wm, w64)):
        a, b = a.cpu().numpy(), b.cpu().numpy()
        rel = np.abs(a - b) / np.abs(b)
        assert np.max(rel) < 1e-8, (n, float(np.max(rel)), float(Ts[np.argmax(rel) // n]))


def test_fp64_all_classes(workload, oracle_values):
    pool, q = workload
    per, _ = gpu_fp64(pool, q, "fp64")
    bad = {}
    for i in range(len(q)):
        ok = fp64_ok(per[i], oracle_values[i])
        if not np.all(ok):
            cls = W.class_id(*[int(pool.L[s]) for s in q[i]])
            e = np.max(np.abs(per[i] - oracle_values[i]))
            bad[cls] = max(bad.get(cls, 0.0), e)
    assert not bad, f"classes out of tolerance (class id -> max abs err): {bad}"


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_without_pair_table(workload, oracle_values, precision):
    """Plans built with ERI_NO_PAIR_TABLE compute the pair quantities per quartet: same
    tolerances against the oracle, and agreement with the pair-table plan to rounding."""
    pool, q = workload
    per, _ = gpu_fp64(pool, q, precision, pair_table=False)
    ref_pairs, _ = gpu_fp64(pool, q, precision)
    for i in range(len(q)):
        ref = oracle_values[i]
        bmax = np.max(np.abs(ref))
        if precision == "fp64":
            assert np.all(fp64_ok(per[i], ref)), i
            assert np.max(np.abs(per[i] - ref_pairs[i])) <= 1e-13 * bmax + 1e-300, i
        else:
            assert np.max(np.abs(per[i] - ref)) <= bmax / 65534.0 + 1e-30, i


def test_compressed_16bit_all_classes(workload, oracle_values):
    pool, q = workload
    codes, eps, _ = gpu_compressed(pool, q, 16, "fp64")
    M = 2 ** 15 - 1
    for i in range(len(q)):
        ref = oracle_values[i]
        rq, reps = oracle.compress_quartet(ref, 16)
        assert abs(float(eps[i]) - float(reps)) <= 1.2e-7 * float(reps) + 1e-300, i
        assert np.max(np.abs(codes[i].astype(np.int64) - rq)) <= 1, i
        # eps is stored in FP32 (Sec. III-C): when b_max / M falls below the smallest normal
        # float the stored eps is subnormal and the code range is no longer exactly +-M
        if reps >= np.finfo(np.float32).tiny:
            assert np.max(np.abs(codes[i])) == M
            xt = codes[i].astype(np.float64) * float(eps[i])
            assert np.all(np.abs(xt - ref) <= float(eps[i]) * (0.5 + 1e-6) + 1e-12)


def test_compressed_to_host_equals_device_output(workload):
    """eri_compute_compressed_to_host delivers the same bytes as eri_compute_compressed followed
    by copies, for a byte width and an odd width (word-split class segments)."""
    pool, q = workload
    plan = api.eri_plan_create(pool, q, precision="mixed")
    s = torch.cuda.current_stream()
    for bits in (16, 13):
        nb, sb = api.eri_output_bytes(plan, bits)
        packed = torch.full((nb // 4,), -1, dtype=torch.int32, device="cuda")
        scales = torch.full((sb // 4,), -1.0, dtype=torch.float32, device="cuda")
        api.eri_compute_compressed(plan, bits, packed, scales, s)
        api.eri_sync(plan, s)
        ref_p, ref_s = packed.cpu().numpy(), scales.cpu().numpy()
        packed.fill_(-1)
        scales.fill_(-1.0)
        hp = torch.full((nb // 4,), 7, dtype=torch.int32, pin_memory=True)
        hs = torch.full((sb // 4,), 7.0, dtype=torch.float32, pin_memory=True)
        api.eri_compute_compressed_to_host(plan, bits, packed, scales, hp, hs, s)
        api.eri_sync(plan, s)
        np.testing.assert_array_equal(hp.numpy(), ref_p)
        np.testing.assert_array_equal(hs.numpy(), ref_s)


@pytest.mark.parametrize("bits", [2, 8, 12, 20, 24])
def test_compressed_other_widths(bits):
    """Packed n-bit streams for odd widths, tile edges that split 32-bit words, and the
    zero padding after each class segment."""
    sel = [(0, 0, 0, 0), (1, 0, 0, 0), (1, 1, 1, 0), (2, 1, 0, 0), (1, 1, 1, 1), (2, 2, 1, 1),
           (3, 1, 2, 0), (3, 3, 2, 2), (0, 1, 3, 2)]
    rng = np.random.default_rng(bits)
    pool = W.random_primitive_pool(rng, 16)
    q = np.concatenate([W.random_class_quartets(rng, c, 131 if W.quartet_size(*c) < 200 else 7, 16)
                        for c in sel])
    q = q[rng.permutation(len(q))]
    vals, offs = oracle.eri_batch(pool, q)
    codes, eps, _ = gpu_compressed(pool, q, bits, "fp64")
    for i in range(len(q)):
        ref = vals[offs[i]:offs[i + 1]]
        rq, reps = oracle.compress_quartet(ref, bits)
        assert np.max(np.abs(codes[i].astype(np.int64) - rq)) <= 1, (i, bits)
        assert abs(float(eps[i]) - float(reps)) <= 1.2e-7 * float(reps) + 1e-300


def test_mixed_precision_all_classes(workload, oracle_values):
    pool, q = workload
    per, _ = gpu_fp64(pool, q, "mixed")
    worst = 0.0
    for i in range(len(q)):
        ref = oracle_values[i]
        bmax = np.max(np.abs(ref))
        err = np.max(np.abs(per[i] - ref))
        assert err <= bmax / 65534.0 + 1e-30, (i, err, bmax)
        if bmax > 1e-30:
            worst = max(worst, err / bmax)
    # FP32 error relative to b_max: measured at most 1.8e-6 over 9.8 M sampled sweep quartets
    # (the VRR + HRR form reached 1.9e-5 on the f classes before the four-index recursion)
    assert worst < 4e-6


def test_mixed_compressed_16bit(workload, oracle_values):
    pool, q = workload
    codes, eps, _ = gpu_compressed(pool, q, 16, "mixed")
    for i in range(len(q)):
        ref = oracle_values[i]
        xt = codes[i].astype(np.float64) * float(eps[i])
        # quantisation (eps/2) plus the FP32 arithmetic error (below eps/2 by the test above)
        assert np.all(np.abs(xt - ref) <= float(eps[i]) + 1e-12 + 1e-30), i


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("pair_table", [True, False])
def test_contracted_shells(precision, pair_table):
    """Contraction over primitives (K = 3): sum of primitive quartets, Kahan-compensated in
    mixed precision; with and without the primitive-pair table."""
    pool, q = mixed_workload(seed=11, per_class=lambda n: 2 if n > 1000 else 5, K=3)
    vals, offs = oracle.eri_batch(pool, q)
    per, _ = gpu_fp64(pool, q, precision, pair_table=pair_table)
    for i in range(len(q)):
        ref = vals[offs[i]:offs[i + 1]]
        if precision == "fp64":
            assert np.all(fp64_ok(per[i], ref)), i
        else:
            assert np.max(np.abs(per[i] - ref)) <= np.max(np.abs(ref)) / 65534.0 + 1e-30, i


def test_degenerate_geometries():
    """Coincident centres (A = B, C = D, all four), far-separated pairs (large T, the
    Gauss-Hermite regime), tiny and large exponents."""
    centers = np.array([[0, 0, 0], [0, 0, 0], [0, 0, 0], [0, 0, 0],
                        [0.1, -0.2, 0.3], [40.0, 0, 0], [0, 35.0, 0], [0.0, 0, 0]])
    Ls = [0, 1, 2, 3, 3, 2, 1, 3]
    exps = [[1.0], [0.7], [1.3], [0.9], [0.03], [12.0], [8.0], [60.0]]
    sh = W.make_shellset(centers, Ls, exps, [[1.0]] * 8)
    q = np.array([[0, 1, 2, 3], [3, 3, 3, 3], [2, 2, 1, 1], [4, 0, 5, 6], [7, 7, 5, 5],
                  [4, 4, 4, 4], [5, 6, 5, 6], [3, 2, 7, 1]], dtype=np.int32)
    vals, offs = oracle.eri_batch(sh, q)
    per, _ = gpu_fp64(sh, q, "fp64")
    for i in range(len(q)):
        assert np.all(fp64_ok(per[i], vals[offs[i]:offs[i + 1]])), i


def test_empty_plan_and_single_quartet():
    sh = W.make_shellset(np.zeros((4, 3)), [1, 1, 1, 1], [[1.0]] * 4, [[1.0]] * 4)
    plan = api.eri_plan_create(sh, np.zeros((0, 4), dtype=np.int32))
    assert api.eri_plan_num_quartets(plan) == 0
    assert api.eri_output_bytes(plan, 16) == (0, 0)
    per, _ = gpu_fp64(sh, np.array([[0, 1, 2, 3]], dtype=np.int32))
    ref = oracle.eri_quartet(sh, [0, 1, 2, 3]).ravel()
    assert np.all(fp64_ok(per[0], ref))


def test_invalid_arguments_are_rejected():
    sh = W.make_shellset(np.zeros((2, 3)), [1, 0], [[1.0]] * 2, [[1.0]] * 2)
    with pytest.raises(api.EriError) as e:
        api.eri_plan_create(sh, np.array([[0, 1, 0, 2]], dtype=np.int32))
    assert e.value.status == 1
    bad = W.make_shellset(np.zeros((1, 3)), [1], [[-1.0]], [[1.0]])
    with pytest.raises(api.EriError):
        api.eri_plan_create(bad, np.array([[0, 0, 0, 0]], dtype=np.int32))
    plan = api.eri_plan_create(sh, np.array([[0, 1, 0, 1]], dtype=np.int32))
    out = torch.empty(1024, dtype=torch.int32, device="cuda")
    sc = torch.empty(4, dtype=torch.float32, device="cuda")
    for bits in (1, 25, 32):
        with pytest.raises(api.EriError):
            api.eri_compute_compressed(plan, bits, out, sc)
