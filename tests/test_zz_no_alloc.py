"""The entry point for callers that cannot let the library allocate device memory
(eri_compute_class_noalloc), called through the C ABI and compared with the plan-based
entry point on the same quartets.

Both run the same class launchers on the same inputs when the plan is built without the
primitive-pair table (ERI_NO_PAIR_TABLE), so the outputs must agree bit for bit once the
coefficient-times-norm values handed to the no-allocation call are computed exactly as the
plan computes them.  Each class is called twice in a row with different quartet lists, the
second one shorter: stale setup records left in the shared device array by the first call
would show up in the second call's output.  One call fills the array to its stated maximum.
"""
import math

import numpy as np
import pytest
import torch

from paper_2303_13632_gb300 import _lib, api, workloads as W

pytestmark = pytest.mark.gpu

# a thread-per-quartet class, classes of the split setup/recurrence path, generic orderings
CLASSES = [(1, 0, 0, 0), (1, 1, 1, 1), (2, 2, 1, 0), (0, 1, 3, 2), (3, 3, 3, 3), (2, 1, 2, 1)]


def shell_norm(alpha: float, L: int) -> float:
    """N(alpha, L) of the axis-aligned normalisation, with the same operations in the same
    order as the library's plan (so the products below round identically)."""
    df = 1.0
    for k in range(2 * L - 1, 1, -2):
        df *= k
    return math.pow(2.0 * alpha / 3.14159265358979323846, 0.75) * math.pow(4.0 * alpha, 0.5 * L) / math.sqrt(df)


def device_inputs(pool):
    cn = []
    for s in range(pool.n):
        for k in range(int(pool.pofs[s]), int(pool.pofs[s]) + int(pool.nprim[s])):
            cn.append(float(pool.coefs[k]) * shell_norm(float(pool.exps[k]), int(pool.L[s])))
    t = lambda a, dt: torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    return (t(pool.centers[:, 0], torch.float64), t(pool.centers[:, 1], torch.float64),
            t(pool.centers[:, 2], torch.float64), t(pool.pofs, torch.int32), t(pool.nprim, torch.int32),
            t(pool.exps, torch.float64), t(np.array(cn), torch.float64))


def plan_output(pool, q, precision):
    """ERIs of one class's quartets through the plan API without the pair table (one class: the
    plan's stable class sort keeps the caller's order)."""
    stream = torch.cuda.current_stream()
    plan = api.eri_plan_create(pool, q, precision=precision, pair_table=False)
    neri = W.quartet_size(*[int(pool.L[s]) for s in q[0]])
    ref = torch.empty(len(q) * neri, dtype=torch.float64, device="cuda")
    api.eri_compute(plan, ref, stream)
    api.eri_sync(plan, stream)
    plan.destroy()
    return ref.cpu().numpy()


def noalloc_output(cls, precision, dev, q):
    stream = torch.cuda.current_stream()
    neri = W.quartet_size(*cls)
    qd = torch.tensor(q, dtype=torch.int32, device="cuda")
    out = torch.full((len(q) * neri,), float("nan"), dtype=torch.float64, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    api.eri_compute_class_noalloc(W.class_id(*cls), precision, *dev, qd, out, err, stream)
    torch.cuda.synchronize()
    return out.cpu().numpy(), int(err.item())


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_noalloc_matches_plan_path(precision):
    rng = np.random.default_rng(77)
    pool = W.random_primitive_pool(rng, 32)
    dev = device_inputs(pool)
    for cls in CLASSES:
        neri = W.quartet_size(*cls)
        n_first = 1000 if neri <= 100 else 37
        # second call: other quartets, fewer of them
        for call, n in enumerate((n_first, n_first // 3 + 1)):
            q = W.random_class_quartets(rng, cls, n, 32)
            ref = plan_output(pool, q, precision)
            got, err = noalloc_output(cls, precision, dev, q)
            assert err == 0
            np.testing.assert_array_equal(got, ref, err_msg=f"{cls} call {call}")


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_noalloc_at_the_maximum_size(precision):
    """[pp|pp] runs on the split setup/recurrence path, so a full batch writes setup records up
    to the last slot of the static array; a short call afterwards must not see them."""
    rng = np.random.default_rng(79)
    pool = W.random_primitive_pool(rng, 64)
    dev = device_inputs(pool)
    cls = (1, 1, 1, 1)
    for n in (_lib.ERI_NOALLOC_MAX_QUARTETS, 517):
        q = W.random_class_quartets(rng, cls, n, 64)
        got, err = noalloc_output(cls, precision, dev, q)
        assert err == 0
        np.testing.assert_array_equal(got, plan_output(pool, q, precision), err_msg=str(n))


def test_noalloc_flags_contracted_shells():
    """A shell with two primitives is outside this entry point's contract: bit 2 of the error
    word is set (the values of the affected quartets are undefined and not inspected)."""
    rng = np.random.default_rng(80)
    pool = W.random_primitive_pool(rng, 8)
    exps = [pool.exps[pool.pofs[s]:pool.pofs[s] + 1] for s in range(pool.n)]
    coefs = [pool.coefs[pool.pofs[s]:pool.pofs[s] + 1] for s in range(pool.n)]
    exps[9] = np.array([0.8, 2.4])  # a p shell (ids 8..15) contracted over two primitives
    coefs[9] = np.array([0.6, 0.4])
    pool2 = W.make_shellset(pool.centers, pool.L, exps, coefs)
    dev = device_inputs(pool2)
    q = np.array([[8, 10, 11, 12], [9, 10, 11, 12], [12, 13, 14, 15]], dtype=np.int32)
    _, err = noalloc_output((1, 1, 1, 1), "fp64", dev, q)
    assert err & 4
    _, err = noalloc_output((1, 1, 1, 1), "fp64", dev, q[[0, 2]])
    assert err == 0


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
