"""Guard bands around every output buffer of the C ABI's compute calls.

Each output is a slice in the middle of a larger buffer whose margins hold a byte pattern; after
the call and eri_sync the margins must be unchanged, so no kernel or copy writes past the sizes
that eri_output_bytes, eri_paper512_class_offset and the documented shapes give.  Small plans
with every class of s..f shells and some with a g shell, one to five quartets per class (ragged
tiles everywhere), FP64 and mixed, odd and byte-sized bit widths.
"""
import numpy as np
import pytest
import torch

from paper_2303_13632_gb300 import _lib, api, workloads as W

pytestmark = pytest.mark.gpu

GUARD = 4096  # bytes on each side; keeps the slice 256-byte aligned
PATTERN = 0x5A


class Guarded:
    """`view`: nbytes (rounded up to whole elements) of dtype inside a pattern-filled buffer."""

    def __init__(self, nbytes, dtype, device="cuda"):
        item = torch.empty(0, dtype=dtype).element_size()
        n = max(1, -(-int(nbytes) // item))
        if device == "cuda":
            self.raw = torch.full((2 * GUARD + n * item,), PATTERN, dtype=torch.uint8, device="cuda")
        else:
            self.raw = torch.full((2 * GUARD + n * item,), PATTERN, dtype=torch.uint8).pin_memory()
        self.view = self.raw[GUARD:GUARD + n * item].view(dtype)

    def intact(self):
        r = self.raw.cpu().numpy()
        return bool((r[:GUARD] == PATTERN).all() and (r[-GUARD:] == PATTERN).all())


def ragged_plan_inputs(seed, g_classes=()):
    rng = np.random.default_rng(seed)
    Ls = (0, 1, 2, 3, 4) if g_classes else (0, 1, 2, 3)
    pool = W.random_primitive_pool(rng, 6, Ls=Ls)
    classes = [W.class_of_id(c) for c in range(256)] + list(g_classes)
    q = np.concatenate([W.random_class_quartets(rng, c, 1 + i % 5, 6, Ls=Ls) for i, c in enumerate(classes)])
    return pool, q[rng.permutation(len(q))]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_forward_outputs_stay_in_their_buffers(precision):
    pool, q = ragged_plan_inputs(3, g_classes=[(4, 0, 0, 0), (2, 1, 4, 3), (4, 4, 1, 1)])
    s = torch.cuda.current_stream()
    plan = api.eri_plan_create(pool, q, precision=precision)
    nb, _ = api.eri_output_bytes(plan, 0)
    out = Guarded(nb, torch.float64)
    api.eri_compute(plan, out.view, s)
    api.eri_sync(plan, s)
    assert out.intact(), "eri_compute"
    for bits in (7, 12, 16):
        pb, sb = api.eri_output_bytes(plan, bits)
        for name, fn in (("eri_compute_compressed", api.eri_compute_compressed),
                         ("eri_compute_compressed_queue", api.eri_compute_compressed_queue),
                         ("eri_compute_compressed_batched", api.eri_compute_compressed_batched)):
            packed, scales = Guarded(pb, torch.int32), Guarded(sb, torch.float32)
            fn(plan, bits, packed.view, scales.view, s)
            api.eri_sync(plan, s)
            assert packed.intact() and scales.intact(), (name, bits)
        # the paper's 512-bit chunks of the last compressed output
        total, _ = api.eri_paper512_class_offset(plan, bits, _lib.ERI_NUM_CLASS_IDS)
        chunks = Guarded(total, torch.int32)
        api.eri_pack_paper512(plan, bits, packed.view, chunks.view, s)
        api.eri_sync(plan, s)
        assert chunks.intact(), ("eri_pack_paper512", bits)
    # streamed to pinned host memory
    pb, sb = api.eri_output_bytes(plan, 16)
    d_packed, d_scales = Guarded(pb, torch.int32), Guarded(sb, torch.float32)
    h_packed = Guarded(pb, torch.int32, device="cpu")
    h_scales = Guarded(sb, torch.float32, device="cpu")
    api.eri_compute_compressed_to_host(plan, 16, d_packed.view, d_scales.view, h_packed.view, h_scales.view, s)
    api.eri_sync(plan, s)
    torch.cuda.synchronize()
    assert d_packed.intact() and d_scales.intact() and h_packed.intact() and h_scales.intact()
    plan.destroy()


def test_adjoint_and_digestion_outputs_stay_in_their_buffers():
    rng = np.random.default_rng(4)
    pool = W.random_contracted_pool(rng, 4, K=2, Ls=(0, 1, 2))
    classes = [(a, b, c, d) for a in range(3) for b in range(3) for c in range(3) for d in range(3)]
    q = np.concatenate([W.random_class_quartets(rng, c, 1 + i % 3, 4, Ls=(0, 1, 2)) for i, c in enumerate(classes)])
    s = torch.cuda.current_stream()
    for precision in ("fp64", "mixed"):
        plan = api.eri_plan_create(pool, q, precision=precision)
        nb, _ = api.eri_output_bytes(plan, 0)
        G = torch.tensor(rng.standard_normal(nb // 8), device="cuda")
        dR = Guarded(8 * 3 * pool.n, torch.float64)
        da = Guarded(8 * len(pool.exps), torch.float64)
        api.eri_backward(plan, G, dR.view, da.view, s)
        api.eri_sync(plan, s)
        assert dR.intact() and da.intact(), ("eri_backward", precision)
        pb, sb = api.eri_output_bytes(plan, 16)
        packed = torch.empty(pb // 4, dtype=torch.int32, device="cuda")
        scales = torch.empty(max(1, sb // 4), dtype=torch.float32, device="cuda")
        api.eri_compute_compressed(plan, 16, packed, scales, s)
        n_bf = api.eri_plan_num_basis_functions(plan)
        D = torch.tensor(rng.standard_normal((n_bf, n_bf)), device="cuda")
        J, K = Guarded(8 * n_bf * n_bf, torch.float64), Guarded(8 * n_bf * n_bf, torch.float64)
        api.eri_digest_jk(plan, 16, packed, scales, D, J.view, K.view, stream=s)
        api.eri_sync(plan, s)
        assert J.intact() and K.intact(), ("eri_digest_jk", precision)
        plan.destroy()
