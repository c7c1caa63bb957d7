"""Shared helpers of the GPU tests: run the CUDA path through the C ABI and bring its
results back in the caller's quartet order, next to the oracle's."""
import numpy as np
import torch

import oracle
from paper_2303_13632_gb300 import _lib, api, workloads as W


def class_of(shells, q):
    L = np.asarray(shells.L)
    return W.class_id(int(L[q[0]]), int(L[q[1]]), int(L[q[2]]), int(L[q[3]]))


def gpu_fp64(shells, quartets, precision="fp64", pair_table=True):
    """Returns (values in the caller's order as a list of per-quartet arrays)."""
    plan = api.eri_plan_create(shells, quartets, precision=precision, pair_table=pair_table)
    nbytes, _ = api.eri_output_bytes(plan, 0)
    out = torch.empty(max(1, nbytes // 8), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    api.eri_compute(plan, out, stream)
    api.eri_sync(plan, stream)
    host = out.cpu().numpy()
    order = api.eri_plan_quartet_order(plan)
    per = [None] * len(quartets)
    pos = 0
    sizes = oracle.quartet_sizes(shells, np.asarray(quartets)[order]) if len(order) else []
    for i, qi in enumerate(order):
        per[qi] = host[pos:pos + sizes[i]]
        pos += sizes[i]
    return per, plan


def gpu_compressed(shells, quartets, bits, precision="fp64"):
    """Returns (codes per quartet in the caller's order, eps per quartet, raw packed bytes)."""
    plan = api.eri_plan_create(shells, quartets, precision=precision)
    nbytes, sbytes = api.eri_output_bytes(plan, bits)
    packed = torch.full((max(1, nbytes // 4),), -1, dtype=torch.int32, device="cuda")  # garbage fill
    scales = torch.full((max(1, sbytes // 4),), -1.0, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    api.eri_compute_compressed(plan, bits, packed, scales, stream)
    api.eri_sync(plan, stream)
    words = packed.cpu().numpy().view(np.uint32)
    eps_sorted = scales.cpu().numpy()
    order = api.eri_plan_quartet_order(plan)
    q = np.asarray(quartets)
    codes = [None] * len(q)
    eps = np.zeros(len(q), dtype=np.float32)
    for cls in range(_lib.ERI_NUM_CLASS_IDS):
        if W.class_id(*W.class_of_id(cls)) != cls:
            continue  # not a class
        nq, neri, first, _ = api.eri_plan_class_info(plan, cls)
        if nq == 0:
            continue
        off, seg = api.eri_packed_class_offset(plan, bits, cls)
        seg_words = words[off // 4:(off + seg) // 4]
        vals = oracle.unpack_bits(seg_words, nq * neri, bits)
        # padding after the last field must be zero
        tail_bit = nq * neri * bits
        for w in range(tail_bit // 32, len(seg_words)):
            lo = tail_bit - 32 * w
            mask = 0xFFFFFFFF if lo <= 0 else (0xFFFFFFFF ^ ((1 << lo) - 1))
            assert int(seg_words[w]) & mask == 0, ("padding", cls, w)
        for i in range(nq):
            qi = order[first + i]
            codes[qi] = vals[i * neri:(i + 1) * neri]
            eps[qi] = eps_sorted[first + i]
    return codes, eps, plan
