"""Parity at the benchmark's full sizes, in the launch configuration the benchmark times.

* One class [pp|pp]: 10,000 primitive quartets (centres U[-3,3]^3, exponents log-U[0.1,10],
  unit coefficients), every quartet against the oracle, FP64 and 16-bit.
* The 256-class sweep: round(2^26 / n_ERIQ) quartets per class drawn on the device.  Per
  class, on the whole output: the 16-bit codes of the FP64 path decompress to within half a
  step of the FP64 output, every quartet with a normal eps has max |q| = M, the mixed path's
  codes stay within half a step plus its FP32 error; and a sample of quartets per class
  against the oracle element by element (FP64 tolerance, codes within +-1 of the oracle's
  quantisation of its own values).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2303_13632_gb300 import api, workloads as W

pytestmark = pytest.mark.gpu

FLT_MIN = float(np.finfo(np.float32).tiny)


def fp64_ok(gpu, ref):
    err = np.abs(gpu - ref)
    return (err <= 1e-12) | ((np.abs(ref) > 1e-8) & (err <= 1e-10 * np.abs(ref)))


def test_one_class_pp_pp_10k_quartets():
    shells, q = W.one_class_workload((1, 1, 1, 1), 10_000, seed_k=1)
    ref, offs = oracle.eri_batch(shells, q)
    ref = ref.reshape(len(q), 81)
    for precision in ("fp64", "mixed"):
        plan = api.eri_plan_create(shells, q, precision=precision)
        out = torch.empty(len(q) * 81, dtype=torch.float64, device="cuda")
        s = torch.cuda.current_stream()
        api.eri_compute(plan, out, s)
        nb, sb = api.eri_output_bytes(plan, 16)
        packed = torch.empty(nb // 2, dtype=torch.int16, device="cuda")
        scales = torch.empty(sb // 4, dtype=torch.float32, device="cuda")
        api.eri_compute_compressed(plan, 16, packed, scales, s)
        api.eri_sync(plan, s)
        order = api.eri_plan_quartet_order(plan)  # one class: sorted position -> caller index
        got = out.cpu().numpy().reshape(len(q), 81)[np.argsort(order)]
        codes = packed.cpu().numpy()[:len(q) * 81].reshape(len(q), 81)[np.argsort(order)]
        eps = scales.cpu().numpy()[np.argsort(order)]
        bmax = np.max(np.abs(ref), axis=1)
        if precision == "fp64":
            assert np.all(fp64_ok(got, ref))
            for i in range(len(q)):
                rq, reps = oracle.compress_quartet(ref[i], 16)
                assert np.max(np.abs(codes[i].astype(np.int64) - rq)) <= 1, i
                assert abs(float(eps[i]) - float(reps)) <= 1.2e-7 * float(reps) + 1e-300
        else:
            assert np.all(np.abs(got - ref) <= bmax[:, None] / 65534.0 + 1e-30)
            xt = codes.astype(np.float64) * eps[:, None].astype(np.float64)
            assert np.all(np.abs(xt - ref) <= eps[:, None].astype(np.float64) + 1e-30)


@pytest.fixture(scope="module")
def sweep():
    counts = {c: W.sweep_quartet_count(W.class_of_id(c)) for c in range(256)}
    pool = W.sweep_pool()
    q, first = W.sweep_quartets_device(torch, counts, torch.device("cuda"))
    torch.cuda.synchronize()
    return pool, q, first, counts


def _class_check(pool, qc, cls, rng):
    """Full-output checks of one class plan and a sampled oracle comparison."""
    s = torch.cuda.current_stream()
    plan = api.eri_plan_create(pool, qc, precision="fp64")
    nq, neri, _, _ = api.eri_plan_class_info(plan, cls)
    assert nq == qc.shape[0]
    out = torch.empty(nq * neri, dtype=torch.float64, device="cuda")
    api.eri_compute(plan, out, s)
    nb, sb = api.eri_output_bytes(plan, 16)
    packed = torch.empty(nb // 2, dtype=torch.int16, device="cuda")
    scales = torch.empty(sb // 4, dtype=torch.float32, device="cuda")
    api.eri_compute_compressed(plan, 16, packed, scales, s)
    x = out.view(nq, neri)
    bmax = x.abs().amax(dim=1)
    codes = packed[:nq * neri].view(nq, neri)
    eps = scales[:nq].double()
    # FP64 path, whole output: |q eps - x| <= eps / 2 (codes from x * (1 / eps) in FP64); a
    # quartet whose b_max is below M * FLT_MIN (3.8e-34 Ha) has a subnormal FP32 eps, hence
    # the absolute floor
    dec = codes.double() * eps[:, None]
    assert bool(((dec - x).abs() <= eps[:, None] * (0.5 + 1e-6) + 1e-30).all()), cls
    normal = eps >= FLT_MIN
    assert bool((codes.abs().amax(dim=1)[normal] == 32767).all()), cls
    assert int(packed[nq * neri:].abs().sum().item()) == 0  # zero padding to the segment end
    # mixed path, whole output: half a step plus its FP32 error (measured at most 1.8e-6 b_max
    # over sampled sweep quartets; 1e-5 b_max allowed), FP32 flush below 1e-30 Ha
    api.eri_plan_set_precision(plan, "mixed")
    api.eri_compute_compressed(plan, 16, packed, scales, s)
    eps_m = scales[:nq].double()
    dec_m = codes.double() * eps_m[:, None]
    bound = eps_m[:, None] * (0.5 + 1e-3) + 1e-5 * bmax[:, None] + 1e-30
    assert bool(((dec_m - x).abs() <= bound).all()), cls
    # sampled quartets against the oracle (positions in the class-sorted order)
    order = api.eri_plan_quartet_order(plan)
    n_s = min(nq, max(4, min(2048, 20000 // neri)))
    pos = np.sort(rng.choice(nq, size=n_s, replace=False))
    qs = qc[torch.as_tensor(order[pos], device="cuda", dtype=torch.int64)].cpu().numpy()
    ref, offs = oracle.eri_batch(pool, qs)
    ref = ref.reshape(n_s, neri)
    got = x[torch.as_tensor(pos, device="cuda")].cpu().numpy()
    assert np.all(fp64_ok(got, ref)), cls
    api.eri_plan_set_precision(plan, "fp64")
    api.eri_compute_compressed(plan, 16, packed, scales, s)
    c_h = codes[torch.as_tensor(pos, device="cuda")].cpu().numpy().astype(np.int64)
    for i in range(n_s):
        rq, _ = oracle.compress_quartet(ref[i], 16)
        assert np.max(np.abs(c_h[i] - rq)) <= 1, (cls, i)
    plan.destroy()


@pytest.mark.parametrize("group", range(8))
def test_sweep_full_size(sweep, group):
    pool, q, first, counts = sweep
    rng = np.random.default_rng(1000 + group)
    for cls in range(group * 32, (group + 1) * 32):
        qc = q[first[cls]:first[cls] + counts[cls]]
        _class_check(pool, qc, cls, rng)
