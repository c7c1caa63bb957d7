"""Device-side error reporting with ordinary inputs (no GPU fault is involved): finite shells
whose contraction coefficients push the ERIs past the floating-point range latch ERI_E_NUMERIC,
which eri_sync returns once and then clears; injected allocation failures at every allocation of
eri_plan_create return ERI_E_NOMEM, release what was allocated, and leave the library usable."""
import numpy as np
import pytest
import torch

from paper_2303_13632_gb300 import _lib, api, workloads as W

pytestmark = pytest.mark.gpu


def overflowing_shells(coef):
    rng = np.random.default_rng(3)
    centers = rng.uniform(-1, 1, size=(8, 3))
    L = [0, 1, 2, 3, 0, 1, 2, 3]
    return W.make_shellset(centers, L, [[0.8]] * 8, [[coef]] * 8)


@pytest.mark.parametrize("precision,coef", [("fp64", 1e100), ("mixed", 1e12)])
def test_non_finite_results_latch_numeric(precision, coef):
    sh = overflowing_shells(coef)
    q = np.array([[0, 0, 0, 0], [1, 2, 1, 0], [3, 3, 2, 2], [5, 6, 7, 4]], dtype=np.int32)
    plan = api.eri_plan_create(sh, q, precision=precision)
    nb, _ = api.eri_output_bytes(plan, 0)
    out = torch.empty(nb // 8, dtype=torch.float64, device="cuda")
    api.eri_compute(plan, out)
    with pytest.raises(api.EriError) as e:
        api.eri_sync(plan)
    assert e.value.status == _lib.ERI_E_NUMERIC
    api.eri_sync(plan)  # latch cleared
    nb, sb = api.eri_output_bytes(plan, 16)
    packed = torch.empty(nb // 4, dtype=torch.int32, device="cuda")
    scales = torch.empty(sb // 4, dtype=torch.float32, device="cuda")
    api.eri_compute_compressed(plan, 16, packed, scales)
    with pytest.raises(api.EriError) as e:
        api.eri_sync(plan)
    assert e.value.status == _lib.ERI_E_NUMERIC
    # ordinary coefficients: no latch
    plan2 = api.eri_plan_create(overflowing_shells(1.0), q, precision=precision)
    api.eri_compute(plan2, out)
    api.eri_sync(plan2)


@pytest.mark.parametrize("screen", [False, True])
def test_injected_allocation_failures(monkeypatch, screen):
    rng = np.random.default_rng(4)
    pool = W.random_primitive_pool(rng, 6)
    q = rng.integers(0, pool.n, size=(500, 4)).astype(np.int32)
    kw = dict(schwarz_threshold=1e-9) if screen else {}
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    failures = 0
    for k in range(1, 60):
        monkeypatch.setenv("ERI_INJECT_NOMEM", str(k))
        try:
            p = api.eri_plan_create(pool, q, **kw)
        except api.EriError as e:
            assert e.status == _lib.ERI_E_NOMEM, (k, e.status)
            failures += 1
            continue
        p.destroy()  # k beyond the call's allocations: the plan was built
        break
    else:
        raise AssertionError("allocation count did not end")
    assert failures >= 10
    monkeypatch.delenv("ERI_INJECT_NOMEM")
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) < 64 << 20  # nothing of size leaked
    plan = api.eri_plan_create(pool, q, **kw)
    assert api.eri_plan_num_quartets(plan) > 0
