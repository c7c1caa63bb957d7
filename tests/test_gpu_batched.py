"""Batched form (persistent work-queue kernels in one CUDA graph) against the per-class
launches, and the autotuner's cache file."""
import os

import numpy as np
import pytest
import torch

from paper_2303_13632_gb300 import api, workloads as W
from test_gpu_parity import mixed_workload

pytestmark = pytest.mark.gpu


def run(plan, bits, batched):
    nb, sb = api.eri_output_bytes(plan, bits)
    packed = torch.full((nb // 4,), -1, dtype=torch.int32, device="cuda")
    scales = torch.full((sb // 4,), -1.0, dtype=torch.float32, device="cuda")
    s = torch.cuda.current_stream()
    if batched:
        api.eri_compute_compressed_batched(plan, bits, packed, scales, s)
        api.eri_compute_compressed_batched(plan, bits, packed, scales, s)  # graph replay
    else:
        api.eri_compute_compressed(plan, bits, packed, scales, s)
    api.eri_sync(plan, s)
    return packed.cpu().numpy(), scales.cpu().numpy()


@pytest.mark.parametrize("precision,K,bits", [("mixed", 1, 16), ("fp64", 1, 12), ("mixed", 3, 16),
                                              ("fp64", 2, 20)])
def test_batched_equals_per_class(precision, K, bits):
    pool, q = mixed_workload(seed=61 + K, K=K,
                             per_class=(lambda n: 3 if n > 1000 else 9) if K > 1 else None)
    plan = api.eri_plan_create(pool, q, precision=precision)
    a = run(plan, bits, False)
    b = run(plan, bits, True)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])


def test_autotune_cache(tmp_path):
    pool, q = mixed_workload(seed=71)
    plan = api.eri_plan_create(pool, q, precision="mixed")
    nb, sb = api.eri_output_bytes(plan, 16)
    packed = torch.empty(nb // 4, dtype=torch.int32, device="cuda")
    scales = torch.empty(sb // 4, dtype=torch.float32, device="cuda")
    cache = str(tmp_path / "tune.txt")
    api.eri_autotune(plan, 16, packed, scales, cache)
    lines = open(cache).read().split("\n")
    lines = [l for l in lines if l]
    assert len(lines) == 55  # one choice per canonical class present in the plan
    api.eri_autotune(plan, 16, packed, scales, cache)  # everything known: nothing appended
    assert len([l for l in open(cache).read().split("\n") if l]) == 55
    # the tuned launch may use the other kernel family of a class, whose FP32 rounding differs:
    # codes within +-1, scales within the mixed path's relative error
    ref = run(plan, 16, False)
    got = run(plan, 16, True)
    a = ref[0].view(np.int16).astype(np.int64)
    b = got[0].view(np.int16).astype(np.int64)
    assert np.max(np.abs(a - b)) <= 1
    np.testing.assert_allclose(got[1], ref[1], rtol=2e-5, atol=0)
