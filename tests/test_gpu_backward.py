"""GPU adjoint (eri_backward) against the oracle's shifted-L gradients and against central
finite differences of the GPU forward pass."""
import numpy as np
import pytest
import torch

import oracle
from paper_2303_13632_gb300 import api, perfmodel as P, workloads as W

pytestmark = pytest.mark.gpu

SD_CLASSES = [(1, 1, 1, 1), (2, 1, 1, 1), (2, 2, 1, 1), (2, 1, 2, 1), (2, 2, 2, 1), (2, 2, 2, 2),
              (1, 2, 1, 2), (0, 1, 2, 2), (1, 0, 0, 1), (0, 0, 0, 0), (2, 0, 1, 0)]


def workload(seed, K, per_class):
    rng = np.random.default_rng(seed)
    pool = W.random_contracted_pool(rng, 6, K=K, Ls=(0, 1, 2))
    q = np.concatenate([W.random_class_quartets(rng, c, per_class, 6, Ls=(0, 1, 2)) for c in SD_CLASSES])
    q = q[rng.permutation(len(q))]
    sizes = oracle.quartet_sizes(pool, q)
    offs = np.zeros(len(q) + 1, dtype=np.int64)
    np.cumsum(sizes, out=offs[1:])
    G = rng.standard_normal(int(offs[-1]))
    return pool, q, G, offs


def to_sorted(plan, q, G, offs, pool):
    """G (caller's quartet order) -> eri_compute layout (class-sorted)."""
    order = api.eri_plan_quartet_order(plan)
    return np.concatenate([G[offs[i]:offs[i + 1]] for i in order])


def gpu_grad(pool, q, G, offs, precision="fp64"):
    plan = api.eri_plan_create(pool, q, precision=precision)
    Gs = torch.tensor(to_sorted(plan, q, G, offs, pool), device="cuda")
    dR = torch.empty((pool.n, 3), dtype=torch.float64, device="cuda")
    da = torch.empty(len(pool.exps), dtype=torch.float64, device="cuda")
    api.eri_backward(plan, Gs, dR, da)
    api.eri_sync(plan)
    return dR.cpu().numpy(), da.cpu().numpy()


@pytest.mark.parametrize("K", [1, 3])
def test_backward_matches_oracle(K):
    pool, q, G, offs = workload(31 + K, K, 6 if K == 3 else 20)
    dR, da = gpu_grad(pool, q, G, offs)
    rR, ra = oracle.eri_grad_batch(pool, q, G, offs)
    np.testing.assert_allclose(dR, rR, rtol=1e-9, atol=1e-11 * max(1.0, np.abs(rR).max()))
    np.testing.assert_allclose(da, ra, rtol=1e-9, atol=1e-11 * max(1.0, np.abs(ra).max()))
    # translational sum rule (no term of the kernel uses it)
    assert np.all(np.abs(dR.sum(axis=0)) <= 1e-10 * max(1.0, np.abs(dR).max()))


def gpu_energy(pool, q, G, offs):
    plan = api.eri_plan_create(pool, q, precision="fp64")
    nb, _ = api.eri_output_bytes(plan, 0)
    out = torch.empty(nb // 8, dtype=torch.float64, device="cuda")
    api.eri_compute(plan, out)
    api.eri_sync(plan)
    return float(np.dot(out.cpu().numpy(), to_sorted(plan, q, G, offs, pool)))


def test_backward_matches_finite_differences_of_forward():
    pool, q, G, offs = workload(41, 2, 3)
    dR, da = gpu_grad(pool, q, G, offs)
    h = 1e-4
    for s in np.unique(q)[:5]:
        for x in range(3):
            cp, cm = pool.centers.copy(), pool.centers.copy()
            cp[s, x] += h
            cm[s, x] -= h
            ep = gpu_energy(W.ShellSet(cp, pool.L, pool.nprim, pool.pofs, pool.exps, pool.coefs), q, G, offs)
            em = gpu_energy(W.ShellSet(cm, pool.L, pool.nprim, pool.pofs, pool.exps, pool.coefs), q, G, offs)
            fd = (ep - em) / (2 * h)
            assert abs(fd - dR[s, x]) <= 1e-6 * max(1.0, abs(fd)), (s, x, fd, dR[s, x])
    for j in range(0, len(pool.exps), 7):
        h = 1e-5 * pool.exps[j]
        ep_, em_ = pool.exps.copy(), pool.exps.copy()
        ep_[j] += h
        em_[j] -= h
        ep = gpu_energy(W.ShellSet(pool.centers, pool.L, pool.nprim, pool.pofs, ep_, pool.coefs), q, G, offs)
        em = gpu_energy(W.ShellSet(pool.centers, pool.L, pool.nprim, pool.pofs, em_, pool.coefs), q, G, offs)
        fd = (ep - em) / (2 * h)
        assert abs(fd - da[j]) <= 1e-6 * max(1.0, abs(fd)), (j, fd, da[j])


# The mixed adjoint (FP32 recurrences on the extended ranges, FP32 per-thread sums, FP64
# geometry and accumulation) against the oracle derivative, relative to the largest gradient
# component.
MIXED_GRAD_TOL = 2e-5


@pytest.mark.parametrize("K", [1, 3])
def test_mixed_backward_matches_oracle(K):
    pool, q, G, offs = workload(31 + K, K, 6 if K == 3 else 20)
    dR, da = gpu_grad(pool, q, G, offs, "mixed")
    rR, ra = oracle.eri_grad_batch(pool, q, G, offs)
    assert np.max(np.abs(dR - rR)) <= MIXED_GRAD_TOL * np.abs(rR).max()
    assert np.max(np.abs(da - ra)) <= MIXED_GRAD_TOL * np.abs(ra).max()


def test_mixed_backward_with_f_shells():
    """The mixed adjoint serves f shells (extended ranges up to L = 5 fit in shared memory in
    FP32): s, p, d, f classes against the oracle derivative."""
    rng = np.random.default_rng(71)
    pool = W.random_contracted_pool(rng, 4, K=2, Ls=(0, 1, 2, 3))
    cls = [(3, 0, 0, 0), (3, 1, 2, 0), (3, 3, 1, 1), (2, 3, 3, 2), (0, 3, 1, 3), (3, 3, 3, 3)]
    q = np.concatenate([W.random_class_quartets(rng, c, 2, 4, Ls=(0, 1, 2, 3)) for c in cls])
    sizes = oracle.quartet_sizes(pool, q)
    offs = np.zeros(len(q) + 1, dtype=np.int64)
    np.cumsum(sizes, out=offs[1:])
    G = rng.standard_normal(int(offs[-1]))
    dR, da = gpu_grad(pool, q, G, offs, "mixed")
    rR, ra = oracle.eri_grad_batch(pool, q, G, offs)
    assert np.max(np.abs(dR - rR)) <= MIXED_GRAD_TOL * np.abs(rR).max()
    assert np.max(np.abs(da - ra)) <= MIXED_GRAD_TOL * np.abs(ra).max()


def test_mixed_backward_every_class():
    """Every canonical class (s to f, primitive shells, three quartets each) through the mixed
    adjoint against the oracle derivative."""
    rng = np.random.default_rng(5)
    pool = W.random_primitive_pool(rng, 6)
    canon = sorted({P.canonical((a, b, c, d)) for a in range(4) for b in range(4) for c in range(4)
                    for d in range(4)})
    assert len(canon) == 55
    for cls in canon:
        q = W.random_class_quartets(rng, cls, 3, 6)
        sizes = oracle.quartet_sizes(pool, q)
        offs = np.zeros(len(q) + 1, dtype=np.int64)
        np.cumsum(sizes, out=offs[1:])
        G = rng.standard_normal(int(offs[-1]))
        rR, ra = oracle.eri_grad_batch(pool, q, G, offs)
        dR, da = gpu_grad(pool, q, G, offs, "mixed")
        assert np.max(np.abs(dR - rR)) <= MIXED_GRAD_TOL * np.abs(rR).max(), cls
        assert np.max(np.abs(da - ra)) <= MIXED_GRAD_TOL * np.abs(ra).max(), cls


def test_backward_rejects_f_shells():
    """The FP64 adjoint does not serve f shells (the mixed one does)."""
    sh = W.make_shellset(np.zeros((4, 3)), [3, 1, 1, 1], [[1.0]] * 4, [[1.0]] * 4)
    plan = api.eri_plan_create(sh, np.array([[0, 1, 2, 3]], dtype=np.int32))
    G = torch.zeros(90, dtype=torch.float64, device="cuda")
    dR = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    da = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(api.EriError) as e:
        api.eri_backward(plan, G, dR, da)
    assert e.value.status == 2


def test_autograd_function():
    """E = sum(G * eri(centers, exps)) differentiated by torch equals the direct adjoint."""
    from paper_2303_13632_gb300.autograd import eri

    pool, q, G, offs = workload(51, 2, 4)
    plan = api.eri_plan_create(pool, q, precision="fp64")
    Gs = torch.tensor(to_sorted(plan, q, G, offs, pool), device="cuda")
    centers = torch.tensor(pool.centers, dtype=torch.float64, requires_grad=True)
    exps = torch.tensor(pool.exps, dtype=torch.float64, requires_grad=True)
    E = (eri(centers, exps, pool, q) * Gs).sum()
    E.backward()
    dR, da = gpu_grad(pool, q, G, offs)
    np.testing.assert_allclose(centers.grad.numpy(), dR, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(exps.grad.numpy(), da, rtol=1e-12, atol=1e-14)
