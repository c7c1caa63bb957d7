"""The paper's 512-bit output chunks (Sec. III-C, compress-store loops) on the GPU: the re-layout
kernel against the oracle's chunk packing on seeded codes (bit-exact), and the plan-level call
on the compressed output of all 256 classes."""
import numpy as np
import pytest
import torch

import oracle
from paper_2303_13632_gb300 import _lib, api
from test_gpu_parity import mixed_workload

pytestmark = pytest.mark.gpu


def relayout(codes, nq, n_eri, bits):
    dense = oracle.pack_bits(codes, bits)
    d_in = torch.tensor(dense.view(np.int32), device="cuda")
    nwords = nq * oracle.paper512_chunks(n_eri, bits) * 16
    d_out = torch.full((max(1, nwords),), -1, dtype=torch.int32, device="cuda")  # garbage fill
    s = torch.cuda.current_stream()
    api.eri_pack_paper512_stream(d_in, nq, n_eri, bits, d_out, s)
    torch.cuda.synchronize()
    return d_out.cpu().numpy().view(np.uint32)[:nwords]


@pytest.mark.parametrize("bits", [2, 3, 7, 8, 12, 13, 16, 20, 24])
def test_stream_relayout_bit_exact(bits):
    rng = np.random.default_rng(500 + bits)
    M = 2 ** (bits - 1) - 1
    per = 512 // bits
    # one field, a chunk minus/plus one, the class sizes of [pp|pp], [dd|dd], [ff|ff]
    for n_eri in (1, 10, per - 1, per, per + 1, 81, 1296, 10000):
        nq = max(2, min(700, 200000 // n_eri))
        q = rng.integers(-M, M + 1, size=nq * n_eri).astype(np.int32)
        got = relayout(q, nq, n_eri, bits)
        np.testing.assert_array_equal(got, oracle.pack_paper512(q, nq, n_eri, bits),
                                      err_msg=f"bits={bits} n_eri={n_eri}")


def test_stream_relayout_grid_stride_and_empty():
    """More output words than the grid has threads (grid-stride loop), and zero quartets."""
    rng = np.random.default_rng(9)
    q = rng.integers(-32767, 32768, size=20000 * 100).astype(np.int32)
    got = relayout(q, 20000, 100, 16)  # 1.28 M words
    np.testing.assert_array_equal(got, oracle.pack_paper512(q, 20000, 100, 16))
    d = torch.zeros(4, dtype=torch.int32, device="cuda")
    api.eri_pack_paper512_stream(d, 0, 10, 16, d, torch.cuda.current_stream())


@pytest.mark.parametrize("bits", [12, 16])
def test_plan_relayout_matches_dense_output(bits):
    """eri_compute_compressed -> eri_pack_paper512 on all 256 classes: every class segment, read
    as chunks, holds the same codes as the dense segment, padding zero, sizes n_CS * 64."""
    pool, quartets = mixed_workload(seed=91, per_class=lambda n: 5 if n > 1000 else 17)
    plan = api.eri_plan_create(pool, quartets, precision="mixed")
    nb, sb = api.eri_output_bytes(plan, bits)
    packed = torch.full((nb // 4,), -1, dtype=torch.int32, device="cuda")
    scales = torch.empty(sb // 4, dtype=torch.float32, device="cuda")
    s = torch.cuda.current_stream()
    api.eri_compute_compressed(plan, bits, packed, scales, s)
    total, _ = api.eri_paper512_class_offset(plan, bits, _lib.ERI_NUM_CLASS_IDS)
    chunks = torch.full((total // 4,), -1, dtype=torch.int32, device="cuda")
    api.eri_pack_paper512(plan, bits, packed, chunks, s)
    api.eri_sync(plan, s)
    dense = packed.cpu().numpy().view(np.uint32)
    cw = chunks.cpu().numpy().view(np.uint32)
    expect_off = 0
    for cls in range(256):
        nq, neri, _, _ = api.eri_plan_class_info(plan, cls)
        off, seg = api.eri_paper512_class_offset(plan, bits, cls)
        assert off == expect_off
        assert seg == nq * oracle.paper512_chunks(neri, bits) * 64
        expect_off += seg
        if nq == 0:
            continue
        doff, dseg = api.eri_packed_class_offset(plan, bits, cls)
        codes = oracle.unpack_bits(dense[doff // 4:(doff + dseg) // 4], nq * neri, bits)
        mine = cw[off // 4:(off + seg) // 4]
        np.testing.assert_array_equal(oracle.unpack_paper512(mine, nq, neri, bits), codes)
        # the chunk words are exactly the oracle's packing of those codes (padding included)
        np.testing.assert_array_equal(mine, oracle.pack_paper512(codes, nq, neri, bits))
    assert expect_off == total
