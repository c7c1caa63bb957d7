"""Per-class precision: the override of one class, and the calibration that keeps the FP32
recurrences only for the classes whose measured error stays below a given fraction of the
quantisation step of the chosen bitwidth."""
import numpy as np
import pytest
import torch

import oracle
from paper_2303_13632_gb300 import api
from test_gpu_parity import mixed_workload

pytestmark = pytest.mark.gpu


def fp64_out(plan):
    nbytes, _ = api.eri_output_bytes(plan, 0)
    out = torch.empty(max(1, nbytes // 8), dtype=torch.float64, device="cuda")
    s = torch.cuda.current_stream()
    api.eri_compute(plan, out, s)
    api.eri_sync(plan, s)
    return out.cpu().numpy()


def test_class_override_switches_only_that_class():
    pool, q = mixed_workload(seed=81)
    mixed = api.eri_plan_create(pool, q, precision="mixed")
    ref_mixed = fp64_out(mixed)
    ref_fp64 = fp64_out(api.eri_plan_create(pool, q, precision="fp64"))
    cls = 0b01010101  # [pp|pp]
    api.eri_plan_set_class_precision(mixed, cls, "fp64")
    assert api.eri_plan_class_precision(mixed, cls)[0] == "fp64"
    assert api.eri_plan_class_precision(mixed, 0)[0] == "mixed"
    got = fp64_out(mixed)
    nq, neri, _, off = api.eri_plan_class_info(mixed, cls)
    sl = slice(off, off + nq * neri)
    np.testing.assert_array_equal(got[sl], ref_fp64[sl])
    rest = np.ones(len(got), dtype=bool)
    rest[sl] = False
    np.testing.assert_array_equal(got[rest], ref_mixed[rest])
    api.eri_plan_set_class_precision(mixed, cls, None)
    np.testing.assert_array_equal(fp64_out(mixed), ref_mixed)


@pytest.mark.parametrize("bits,K,steps", [(20, 1, 0.25), (16, 1, 0.25), (20, 2, 0.25), (16, 1, 0.5)])
def test_calibration_keeps_error_below_quantisation(bits, K, steps):
    pool, q = mixed_workload(seed=90 + bits + K, K=K,
                             per_class=(lambda n: 3 if n > 1000 else 9) if K > 1 else None)
    plan = api.eri_plan_create(pool, q, precision="mixed")
    api.eri_plan_calibrate_precision(plan, bits, sample=1 << 20, max_err_steps=steps)  # every quartet
    thr = steps / (2 ** (bits - 1) - 1)
    n_fp64 = 0
    for c in range(256):
        if api.eri_plan_class_info(plan, c)[0] == 0:
            continue
        prec, err = api.eri_plan_class_precision(plan, c)
        assert err >= 0.0
        assert (prec == "mixed") == (err < thr), (c, prec, err, thr)
        n_fp64 += prec == "fp64"
    # the compressed output of the calibrated plan against the oracle: quantisation (eps / 2),
    # the FP32 product x * (1 / eps) (2^-23 relative on codes up to 2^{bits-1}: at most 1/16
    # of a step at 20 bits) and the measured arithmetic error (below `steps` eps), with FP32
    # flush below 1e-30 Ha
    vals, offs = oracle.eri_batch(pool, q)
    nb, sb = api.eri_output_bytes(plan, bits)
    packed = torch.empty(max(1, nb // 4), dtype=torch.int32, device="cuda")
    scales = torch.empty(max(1, sb // 4), dtype=torch.float32, device="cuda")
    s = torch.cuda.current_stream()
    api.eri_compute_compressed(plan, bits, packed, scales, s)
    api.eri_sync(plan, s)
    words = packed.cpu().numpy().view(np.uint32)
    eps_sorted = scales.cpu().numpy()
    order = api.eri_plan_quartet_order(plan)
    for c in range(256):
        nq, neri, first, _ = api.eri_plan_class_info(plan, c)
        if nq == 0:
            continue
        off, seg = api.eri_packed_class_offset(plan, bits, c)
        codes = oracle.unpack_bits(words[off // 4:(off + seg) // 4], nq * neri, bits)
        for i in range(nq):
            qi = order[first + i]
            ref = vals[offs[qi]:offs[qi + 1]]
            eps = float(eps_sorted[first + i])
            xt = codes[i * neri:(i + 1) * neri].astype(np.float64) * eps
            assert np.max(np.abs(xt - ref)) <= (0.57 + steps) * eps + 1e-30, (c, i)
    assert n_fp64 < 256


def test_calibration_rejects_bad_arguments():
    pool, q = mixed_workload(seed=99, per_class=lambda n: 1)
    plan = api.eri_plan_create(pool, q, precision="mixed")
    for bits, sample, steps in [(1, 16, 0.5), (25, 16, 0.5), (16, 0, 0.5), (16, 16, 0.0), (16, 16, 1.5)]:
        with pytest.raises(RuntimeError):
            api.eri_plan_calibrate_precision(plan, bits, sample=sample, max_err_steps=steps)
    with pytest.raises(RuntimeError):
        api.eri_plan_set_class_precision(plan, 256, "fp64")
