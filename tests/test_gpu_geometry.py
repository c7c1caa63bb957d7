"""A plan moved to new shell geometry (eri_plan_update_shells) against a plan built at that
geometry (same kernels on the same values: bit for bit, with and without the primitive-pair
table, FP64 and compressed mixed outputs), against the oracle, and the differentiable
geometry loop (EriGeometry): a gradient taken after the shared plan has moved on still belongs
to its own forward pass."""
import numpy as np
import pytest
import torch

import oracle
from paper_2303_13632_gb300 import api, workloads as W
from paper_2303_13632_gb300.autograd import EriGeometry
from test_gpu_backward import SD_CLASSES, gpu_grad, to_sorted, workload

pytestmark = pytest.mark.gpu

CLASSES = [(0, 0, 0, 0), (1, 0, 0, 0), (1, 1, 1, 1), (2, 1, 0, 0), (2, 2, 1, 1), (3, 1, 2, 0), (3, 3, 2, 2)]


def moved(pool, rng, step=0.3):
    """The same basis layout at another geometry: centres shifted, exponents and coefficients
    scaled."""
    return W.ShellSet(pool.centers + step * rng.standard_normal(pool.centers.shape), pool.L, pool.nprim,
                      pool.pofs, pool.exps * np.exp(0.2 * rng.standard_normal(len(pool.exps))),
                      pool.coefs * (1.0 + 0.1 * rng.standard_normal(len(pool.coefs))))


def outputs(plan, bits=16):
    s = torch.cuda.current_stream()
    nb, _ = api.eri_output_bytes(plan, 0)
    out = torch.empty(nb // 8, dtype=torch.float64, device="cuda")
    api.eri_compute(plan, out, s)
    pb, sb = api.eri_output_bytes(plan, bits)
    packed = torch.empty(max(1, pb // 4), dtype=torch.int32, device="cuda")
    scales = torch.empty(max(1, sb // 4), dtype=torch.float32, device="cuda")
    api.eri_compute_compressed(plan, bits, packed, scales, s)
    api.eri_sync(plan, s)
    return out.cpu().numpy(), packed.cpu().numpy(), scales.cpu().numpy()


def class_mix(seed, K):
    rng = np.random.default_rng(seed)
    pool = W.random_contracted_pool(rng, 8, K=K, Ls=(0, 1, 2, 3))
    q = np.concatenate([W.random_class_quartets(rng, c, 40, 8, Ls=(0, 1, 2, 3)) for c in CLASSES])
    return rng, pool, q[rng.permutation(len(q))]


@pytest.mark.parametrize("pair_table", [True, False])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_updated_plan_equals_new_plan(pair_table, precision):
    rng, pool, q = class_mix(11, K=2)
    pool2 = moved(pool, rng)
    plan = api.eri_plan_create(pool, q, precision=precision, pair_table=pair_table)
    outputs(plan)  # work at the first geometry, then move
    api.eri_plan_update_shells(plan, pool2)
    got = outputs(plan)
    fresh = api.eri_plan_create(pool2, q, precision=precision, pair_table=pair_table)
    want = outputs(fresh)
    for g, w in zip(got, want):
        np.testing.assert_array_equal(g, w)
    # and the moved plan against the oracle at the new geometry (FP64 path)
    if precision == "fp64":
        ref, offs = oracle.eri_batch(pool2, q)
        order = api.eri_plan_quartet_order(plan)
        ref_sorted = np.concatenate([ref[offs[i]:offs[i + 1]] for i in order])
        np.testing.assert_allclose(got[0], ref_sorted, rtol=1e-10, atol=1e-12)
    plan.destroy()
    fresh.destroy()


def test_update_rejects_a_changed_layout_and_keeps_the_plan():
    rng, pool, q = class_mix(12, K=1)
    plan = api.eri_plan_create(pool, q)
    before = outputs(plan)[0]
    bad_L = W.ShellSet(pool.centers, np.where(pool.L == 0, 1, pool.L).astype(np.int32), pool.nprim,
                       pool.pofs, pool.exps, pool.coefs)
    bad_exp = W.ShellSet(pool.centers, pool.L, pool.nprim, pool.pofs, -pool.exps, pool.coefs)
    bad_centre = W.ShellSet(np.full_like(pool.centers, np.inf), pool.L, pool.nprim, pool.pofs, pool.exps,
                            pool.coefs)
    fewer = W.ShellSet(pool.centers[:-1], pool.L[:-1], pool.nprim[:-1], pool.pofs[:-1], pool.exps, pool.coefs)
    for sh in (bad_L, bad_exp, bad_centre, fewer):
        with pytest.raises(api.EriError) as e:
            api.eri_plan_update_shells(plan, sh)
        assert e.value.status == 1
    np.testing.assert_array_equal(outputs(plan)[0], before)
    plan.destroy()


def test_geometry_loop_gradients():
    """EriGeometry over two geometries: both forward passes first, then both backward passes;
    each gradient equals the direct adjoint of a plan built at its own geometry."""
    pool, q, G, offs = workload(61, 2, 3)
    rng = np.random.default_rng(62)
    pool2 = W.ShellSet(pool.centers + 0.2 * rng.standard_normal(pool.centers.shape), pool.L, pool.nprim,
                       pool.pofs, pool.exps, pool.coefs)
    geo = EriGeometry(pool, q)
    ref_plan = api.eri_plan_create(pool, q)
    Gs = torch.tensor(to_sorted(ref_plan, q, G, offs, pool), device="cuda")
    grads = []
    energies = []
    for p in (pool, pool2):
        c = torch.tensor(p.centers, dtype=torch.float64, requires_grad=True)
        e = torch.tensor(p.exps, dtype=torch.float64, requires_grad=True)
        energies.append(((geo(c, e) * Gs).sum(), c, e))
    for E, c, e in energies:
        E.backward()
        grads.append((c.grad.numpy(), e.grad.numpy()))
    for p, (dR, da) in zip((pool, pool2), grads):
        rR, ra = gpu_grad(p, q, G, offs)
        np.testing.assert_allclose(dR, rR, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(da, ra, rtol=1e-12, atol=1e-14)
    assert not np.allclose(grads[0][0], grads[1][0])  # the two geometries differ
    np.testing.assert_array_equal(geo.order(), api.eri_plan_quartet_order(ref_plan))
    geo.destroy()
