"""The entry point for callers that cannot let the library allocate device memory
(eri_compute_class_noalloc), called through the C ABI and compared with the plan-based
entry point on the same quartets, twice in a row (the second call finds the first call's
setup records in the shared device array)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2303_13632_gb300 import _lib, api, workloads as W

pytestmark = pytest.mark.gpu

# a thread-per-quartet class, classes of the split setup/recurrence path, generic orderings
CLASSES = [(1, 0, 0, 0), (1, 1, 1, 1), (2, 2, 1, 0), (0, 1, 3, 2), (3, 3, 3, 3), (2, 1, 2, 1)]


def device_inputs(pool):
    cn = np.array([c * oracle.norm(a, int(pool.L[s]))
                   for s in range(pool.n) for a, c in zip(pool.exps[pool.pofs[s]:pool.pofs[s] + pool.nprim[s]],
                                                          pool.coefs[pool.pofs[s]:pool.pofs[s] + pool.nprim[s]])])
    t = lambda a, dt: torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    return (t(pool.centers[:, 0], torch.float64), t(pool.centers[:, 1], torch.float64),
            t(pool.centers[:, 2], torch.float64), t(pool.pofs, torch.int32), t(pool.nprim, torch.int32),
            t(pool.exps, torch.float64), t(cn, torch.float64))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_noalloc_matches_plan_path(precision):
    rng = np.random.default_rng(77)
    pool = W.random_primitive_pool(rng, 32)
    dev = device_inputs(pool)
    stream = torch.cuda.current_stream()
    for cls in CLASSES:
        neri = W.quartet_size(*cls)
        n = 1000 if neri <= 100 else 37
        q = W.random_class_quartets(rng, cls, n, 32)
        plan = api.eri_plan_create(pool, q, precision=precision)
        ref = torch.empty(n * neri, dtype=torch.float64, device="cuda")
        api.eri_compute(plan, ref, stream)
        api.eri_sync(plan, stream)
        qd = torch.tensor(q, dtype=torch.int32, device="cuda")
        for call in range(2):
            out = torch.full((n * neri,), float("nan"), dtype=torch.float64, device="cuda")
            err = torch.zeros(1, dtype=torch.int32, device="cuda")
            api.eri_compute_class_noalloc(W.class_id(*cls), precision, *dev, qd, out, err, stream)
            torch.cuda.synchronize()
            assert int(err.item()) == 0
            a, b = out.cpu().numpy(), ref.cpu().numpy()
            tol = 1e-12 + 1e-10 * np.abs(b) if precision == "fp64" else 1e-30 + np.abs(b).max() / 65534.0
            assert np.all(np.abs(a - b) <= tol), (cls, call, float(np.max(np.abs(a - b))))


def test_noalloc_rejects_oversized_batches():
    rng = np.random.default_rng(78)
    pool = W.random_primitive_pool(rng, 4)
    dev = device_inputs(pool)
    n = _lib.ERI_NOALLOC_MAX_QUARTETS + 1
    q = torch.zeros((n, 4), dtype=torch.int32, device="cuda")
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(api.EriError) as e:
        api.eri_compute_class_noalloc(0, "fp64", *dev, q, out, err)
    assert e.value.status == _lib.ERI_E_INVALID
