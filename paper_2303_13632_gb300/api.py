"""Python face of the C ABI (include/eri.h): the same entry points, taking numpy arrays,
torch tensors and shell sets.  Argument marshalling only -- every step of the ERI path
runs in the CUDA library.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import (ERI_ALL, ERI_EXPLICIT, ERI_FP64, ERI_MIXED, ERI_QUARTETS_ON_DEVICE, ERI_UNIQUE8,  # noqa: F401
                   EriError, check)

PRECISIONS = {"fp64": ERI_FP64, "mixed": ERI_MIXED}


def _stream_handle(stream) -> ctypes.c_void_p:
    if stream is None:
        return ctypes.c_void_p(0)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)  # torch.cuda.Stream


def _dev_ptr(t) -> ctypes.c_void_p:
    if t is None:
        return ctypes.c_void_p(0)
    if isinstance(t, int):
        return ctypes.c_void_p(t)
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


class Plan:
    """Owns an eri_plan_t; the arrays that back the shell structs are kept alive."""

    def __init__(self, handle: ctypes.c_void_p):
        self.handle = handle

    def destroy(self):
        if self.handle:
            _lib.load().eri_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


MODES = {"explicit": ERI_EXPLICIT, "all": ERI_ALL, "unique8": ERI_UNIQUE8}


def _shell_array(shells):
    """eri_shell_t array of a ShellSet, and the numpy arrays its pointers refer to (keep them
    alive for the call)."""
    n = len(shells.L)
    arr = (_lib.eri_shell_t * max(n, 1))()
    exps = np.ascontiguousarray(shells.exps, dtype=np.float64)
    coefs = np.ascontiguousarray(shells.coefs, dtype=np.float64)
    base_e = exps.ctypes.data
    base_c = coefs.ctypes.data
    for s in range(n):
        sh = arr[s]
        for x in range(3):
            sh.center[x] = float(shells.centers[s][x])
        sh.L = int(shells.L[s])
        sh.nprim = int(shells.nprim[s])
        off = int(shells.pofs[s]) * 8
        sh.exps = ctypes.cast(base_e + off, _lib.c_double_p)
        sh.coefs = ctypes.cast(base_c + off, _lib.c_double_p)
    return arr, (exps, coefs)


def eri_plan_create(shells, quartets=None, precision: str = "fp64", mode: str = "explicit",
                    device: int = 0, pair_table: bool = True, schwarz_threshold: float = 0.0,
                    shard: tuple[int, int] = (0, 0)) -> Plan:
    """shells: a ShellSet (workloads.py); quartets: [n, 4] int32 numpy array (host), a
    contiguous int32 CUDA tensor (device), or None with mode="all" / "unique8"; pair_table=False
    sets ERI_NO_PAIR_TABLE; shard = (shard_index, shard_count) of a unique8 enumeration."""
    lib = _lib.load()
    n = len(shells.L)
    arr, _keep = _shell_array(shells)
    opts = _lib.eri_plan_opts_t(PRECISIONS[precision], MODES[mode], device,
                                0 if pair_table else _lib.ERI_NO_PAIR_TABLE, float(schwarz_threshold),
                                int(shard[0]), int(shard[1]))
    if quartets is None:
        qptr, nq = ctypes.c_void_p(0), 0
    elif isinstance(quartets, np.ndarray):
        q = np.ascontiguousarray(quartets, dtype=np.int32).reshape(-1, 4)
        qptr, nq = ctypes.c_void_p(q.ctypes.data), len(q)
    else:  # torch tensor on the device
        import torch

        if quartets.dtype != torch.int32 or not quartets.is_cuda or not quartets.is_contiguous():
            raise ValueError("device quartets must be a contiguous int32 CUDA tensor")
        qptr, nq = ctypes.c_void_p(quartets.data_ptr()), quartets.numel() // 4
        opts.flags |= ERI_QUARTETS_ON_DEVICE
    handle = ctypes.c_void_p()
    st = lib.eri_plan_create(arr, n, qptr, nq, ctypes.byref(opts), ctypes.byref(handle))
    check(st, "eri_plan_create")
    return Plan(handle)


def eri_plan_destroy(plan: Plan) -> None:
    plan.destroy()


def eri_plan_update_shells(plan: Plan, shells, stream=None) -> None:
    """New centres, exponents and coefficients for the plan's shells (same count, L and nprim
    per shell); the quartet list and everything else of the plan stay."""
    arr, _keep = _shell_array(shells)
    check(_lib.load().eri_plan_update_shells(plan.handle, arr, len(shells.L), _stream_handle(stream)),
          "eri_plan_update_shells")


def eri_plan_set_precision(plan: Plan, precision: str) -> None:
    check(_lib.load().eri_plan_set_precision(plan.handle, PRECISIONS[precision]), "eri_plan_set_precision")


def eri_plan_set_class_precision(plan: Plan, cls: int, precision: str | None) -> None:
    v = -1 if precision is None else PRECISIONS[precision]
    check(_lib.load().eri_plan_set_class_precision(plan.handle, cls, v), "eri_plan_set_class_precision")


def eri_plan_calibrate_precision(plan: Plan, bits: int, sample: int = 4096,
                                 max_err_steps: float = 0.5, stream=None) -> None:
    check(_lib.load().eri_plan_calibrate_precision(plan.handle, bits, sample, max_err_steps,
                                                   _stream_handle(stream)),
          "eri_plan_calibrate_precision")


def eri_plan_class_precision(plan: Plan, cls: int):
    """Returns (precision name, measured mixed error or -1)."""
    p, e = ctypes.c_int32(), ctypes.c_float()
    check(_lib.load().eri_plan_class_precision(plan.handle, cls, ctypes.byref(p), ctypes.byref(e)),
          "eri_plan_class_precision")
    return ("fp64" if p.value == ERI_FP64 else "mixed"), float(e.value)


def eri_plan_class_launches(plan: Plan, cls: int) -> int:
    n = ctypes.c_int32()
    check(_lib.load().eri_plan_class_launches(plan.handle, cls, ctypes.byref(n)), "eri_plan_class_launches")
    return int(n.value)


def eri_plan_class_kernels(plan: Plan, cls: int) -> str:
    buf = ctypes.create_string_buffer(256)
    check(_lib.load().eri_plan_class_kernels(plan.handle, cls, buf, 256), "eri_plan_class_kernels")
    return buf.value.decode()


def eri_fma_probe(precision: str, n_threads: int, iters: int, sink, stream=None) -> None:
    """Launches the FMA throughput probe: 512 * iters * n_threads flops (see include/eri.h)."""
    check(_lib.load().eri_fma_probe(PRECISIONS[precision], n_threads, iters, _dev_ptr(sink),
                                    _stream_handle(stream)), "eri_fma_probe")


def eri_plan_num_quartets(plan: Plan) -> int:
    n = ctypes.c_int64()
    check(_lib.load().eri_plan_num_quartets(plan.handle, ctypes.byref(n)), "eri_plan_num_quartets")
    return n.value


def eri_plan_class_info(plan: Plan, cls: int):
    """Returns (n_quartets, n_eri_per_quartet, first_quartet, fp64_offset)."""
    a, b, c, d = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int64()
    check(_lib.load().eri_plan_class_info(plan.handle, cls, ctypes.byref(a), ctypes.byref(b),
                                          ctypes.byref(c), ctypes.byref(d)), "eri_plan_class_info")
    return a.value, b.value, c.value, d.value


def eri_plan_quartet_order(plan: Plan) -> np.ndarray:
    n = eri_plan_num_quartets(plan)
    out = np.zeros(n, dtype=np.int64)
    check(_lib.load().eri_plan_quartet_order(plan.handle, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))),
          "eri_plan_quartet_order")
    return out


def eri_plan_quartets(plan: Plan) -> np.ndarray:
    """The plan's quartets [n, 4] (int32) in class-sorted order (the order of every output)."""
    n = eri_plan_num_quartets(plan)
    out = np.zeros((n, 4), dtype=np.int32)
    check(_lib.load().eri_plan_quartets(plan.handle, ctypes.c_void_p(out.ctypes.data)), "eri_plan_quartets")
    return out


def eri_plan_screening(plan: Plan):
    """(quartets before Schwarz screening, quartets kept before sharding)."""
    a, b = ctypes.c_int64(), ctypes.c_int64()
    check(_lib.load().eri_plan_screening(plan.handle, ctypes.byref(a), ctypes.byref(b)), "eri_plan_screening")
    return a.value, b.value


def eri_output_bytes(plan: Plan, bits: int):
    """Returns (packed_bytes, scales_bytes); bits = 0 gives the FP64 output size."""
    a, b = ctypes.c_size_t(), ctypes.c_size_t()
    check(_lib.load().eri_output_bytes(plan.handle, bits, ctypes.byref(a), ctypes.byref(b)), "eri_output_bytes")
    return a.value, b.value


def eri_packed_class_offset(plan: Plan, bits: int, cls: int):
    a, b = ctypes.c_size_t(), ctypes.c_size_t()
    check(_lib.load().eri_packed_class_offset(plan.handle, bits, cls, ctypes.byref(a), ctypes.byref(b)),
          "eri_packed_class_offset")
    return a.value, b.value


def eri_paper512_class_offset(plan: Plan, bits: int, cls: int):
    """(byte offset, bytes) of class `cls` in the paper's 512-bit chunk layout; cls =
    ERI_NUM_CLASS_IDS gives (total bytes, 0)."""
    a, b = ctypes.c_size_t(), ctypes.c_size_t()
    check(_lib.load().eri_paper512_class_offset(plan.handle, bits, cls, ctypes.byref(a), ctypes.byref(b)),
          "eri_paper512_class_offset")
    return a.value, b.value


def eri_pack_paper512(plan: Plan, bits: int, packed, chunks, stream=None) -> None:
    check(_lib.load().eri_pack_paper512(plan.handle, bits, _dev_ptr(packed), _dev_ptr(chunks),
                                        _stream_handle(stream)), "eri_pack_paper512")


def eri_pack_paper512_stream(dense, n_quartets: int, n_eri: int, bits: int, chunks, stream=None) -> None:
    check(_lib.load().eri_pack_paper512_stream(_dev_ptr(dense), n_quartets, n_eri, bits, _dev_ptr(chunks),
                                               _stream_handle(stream)), "eri_pack_paper512_stream")


def eri_compute(plan: Plan, out, stream=None) -> None:
    check(_lib.load().eri_compute(plan.handle, _dev_ptr(out), _stream_handle(stream)), "eri_compute")


def eri_compute_class(plan: Plan, cls: int, out, stream=None) -> None:
    check(_lib.load().eri_compute_class(plan.handle, cls, _dev_ptr(out), _stream_handle(stream)),
          "eri_compute_class")


def eri_compute_compressed_to_host(plan: Plan, bits: int, d_packed, d_scales, h_packed, h_scales,
                                   stream=None) -> None:
    """Compressed ERIs streamed class by class to host tensors (pinned for overlap)."""
    check(_lib.load().eri_compute_compressed_to_host(
        plan.handle, bits, _dev_ptr(d_packed), _dev_ptr(d_scales),
        ctypes.c_void_p(h_packed.data_ptr()), ctypes.c_void_p(h_scales.data_ptr()),
        _stream_handle(stream)), "eri_compute_compressed_to_host")


def eri_compute_compressed(plan: Plan, bits: int, packed, scales, stream=None) -> None:
    check(_lib.load().eri_compute_compressed(plan.handle, bits, _dev_ptr(packed), _dev_ptr(scales),
                                             _stream_handle(stream)), "eri_compute_compressed")


def eri_compute_compressed_class(plan: Plan, cls: int, bits: int, packed, scales, stream=None) -> None:
    check(_lib.load().eri_compute_compressed_class(plan.handle, cls, bits, _dev_ptr(packed),
                                                   _dev_ptr(scales), _stream_handle(stream)),
          "eri_compute_compressed_class")


def eri_compute_compressed_batched(plan: Plan, bits: int, packed, scales, stream=None) -> None:
    check(_lib.load().eri_compute_compressed_batched(plan.handle, bits, _dev_ptr(packed), _dev_ptr(scales),
                                                     _stream_handle(stream)), "eri_compute_compressed_batched")


def eri_compute_compressed_queue(plan: Plan, bits: int, packed, scales, stream=None) -> None:
    check(_lib.load().eri_compute_compressed_queue(plan.handle, bits, _dev_ptr(packed), _dev_ptr(scales),
                                                   _stream_handle(stream)), "eri_compute_compressed_queue")


def eri_autotune(plan: Plan, bits: int, packed, scales, cache_path: str | None = None, stream=None) -> None:
    path = cache_path.encode() if cache_path else None
    check(_lib.load().eri_autotune(plan.handle, bits, _dev_ptr(packed), _dev_ptr(scales), path,
                                   _stream_handle(stream)), "eri_autotune")


def eri_backward(plan: Plan, G, dR, dalpha, stream=None) -> None:
    """dR [n_shells, 3] and dalpha [n_prims] (float64 CUDA tensors) receive the gradient of
    E = sum G * ERIs for G laid out like eri_compute's output."""
    check(_lib.load().eri_backward(plan.handle, _dev_ptr(G), _dev_ptr(dR), _dev_ptr(dalpha),
                                   _stream_handle(stream)), "eri_backward")


def eri_compute_class_noalloc(cls: int, precision: str, cx, cy, cz, pofs, nprim, exps, cn, quartets,
                              out, err, stream=None) -> None:
    """No-allocation entry point (every argument a caller-owned CUDA tensor): FP64 or mixed ERIs
    of quartets of one class; see include/eri.h for the contract and its limits."""
    n = quartets.numel() // 4
    check(_lib.load().eri_compute_class_noalloc(
        cls, PRECISIONS[precision], _dev_ptr(cx), _dev_ptr(cy), _dev_ptr(cz), _dev_ptr(pofs),
        _dev_ptr(nprim), _dev_ptr(exps), _dev_ptr(cn), _dev_ptr(quartets), n, _dev_ptr(out),
        _dev_ptr(err), _stream_handle(stream)), "eri_compute_class_noalloc")


def eri_plan_num_basis_functions(plan: Plan) -> int:
    n = ctypes.c_int64()
    check(_lib.load().eri_plan_num_basis_functions(plan.handle, ctypes.byref(n)),
          "eri_plan_num_basis_functions")
    return n.value


def eri_digest_jk(plan: Plan, bits: int, packed, scales, D, J, K, unique8: bool = False,
                  accumulate: bool = False, symmetric: bool = False, stream=None) -> None:
    """J and K (n_bf x n_bf float64 CUDA tensors) from the compressed ERIs and the density D
    (symmetric=True: the caller asserts D is symmetric, see ERI_DIGEST_SYMMETRIC)."""
    flags = ((_lib.ERI_DIGEST_UNIQUE8 if unique8 else 0) | (_lib.ERI_DIGEST_ACCUMULATE if accumulate else 0)
             | (_lib.ERI_DIGEST_SYMMETRIC if symmetric else 0))
    check(_lib.load().eri_digest_jk(plan.handle, bits, _dev_ptr(packed), _dev_ptr(scales), _dev_ptr(D),
                                    _dev_ptr(J), _dev_ptr(K), flags, _stream_handle(stream)),
          "eri_digest_jk")


def eri_sync(plan: Plan, stream=None) -> None:
    check(_lib.load().eri_sync(plan.handle, _stream_handle(stream)), "eri_sync")


def eri_status_string(status: int) -> str:
    return _lib.load().eri_status_string(status).decode()


def eri_boys_device(mmax: int, T, F, stream=None) -> None:
    check(_lib.load().eri_boys_device(mmax, _dev_ptr(T), T.numel(), _dev_ptr(F), _stream_handle(stream)),
          "eri_boys_device")


def eri_rys_device(nroots: int, T, x, w, stream=None) -> None:
    check(_lib.load().eri_rys_device(nroots, _dev_ptr(T), T.numel(), _dev_ptr(x), _dev_ptr(w),
                                     _stream_handle(stream)), "eri_rys_device")


def eri_rys_device_mixed(nroots: int, T, x, w, stream=None) -> None:
    check(_lib.load().eri_rys_device_mixed(nroots, _dev_ptr(T), T.numel(), _dev_ptr(x), _dev_ptr(w),
                                           _stream_handle(stream)), "eri_rys_device_mixed")


def eri_class_id(La: int, Lb: int, Lc: int, Ld: int) -> int:
    return int(_lib.load().eri_class_id(La, Lb, Lc, Ld))


def eri_class_shape(cls: int):
    a, b = ctypes.c_int32(), ctypes.c_int32()
    check(_lib.load().eri_class_shape(cls, ctypes.byref(a), ctypes.byref(b)), "eri_class_shape")
    return a.value, b.value


def eri_convert_device(x, f_out, back_out, stream=None) -> None:
    """Integer-pipe binary64 -> binary32 -> binary64 conversions of the setup stages."""
    check(_lib.load().eri_convert_device(_dev_ptr(x), x.numel(), _dev_ptr(f_out), _dev_ptr(back_out),
                                         _stream_handle(stream)), "eri_convert_device")


class Engine:
    """Shell-quartet access in the style of libint's engine (the library interface the paper's
    conclusion points to): ERIs of a list of shell quartets, returned per quartet as an array of
    shape (n_a, n_b, n_c, n_d) in the caller's order, Cartesian components in the order of
    include/eri.h (a_x from L down, then a_y; libint's Cartesian order).  Each call builds one
    plan of the quartets, runs eri_compute on the device and reorders the class-sorted output on
    the host: a convenience over eri_plan_create / eri_compute / eri_plan_quartet_order for
    integrating callers, not a faster path."""

    def __init__(self, shells, precision: str = "fp64", device: int = 0):
        self.shells = shells
        self.precision = precision
        self.device = device

    def compute(self, quartets, stream=None) -> list:
        import torch

        q = np.ascontiguousarray(quartets, dtype=np.int32).reshape(-1, 4)
        if len(q) == 0:
            return []
        plan = eri_plan_create(self.shells, q, precision=self.precision, device=self.device)
        nbytes, _ = eri_output_bytes(plan, 0)
        out = torch.empty(nbytes // 8, dtype=torch.float64, device=torch.device("cuda", self.device))
        eri_compute(plan, out, stream)
        eri_sync(plan, stream)
        host = out.cpu().numpy()
        order = eri_plan_quartet_order(plan)
        L = np.asarray(self.shells.L)
        dims = [(L[r] + 1) * (L[r] + 2) // 2 for r in q[order].T]
        sizes = dims[0] * dims[1] * dims[2] * dims[3]
        starts = np.concatenate([[0], np.cumsum(sizes)[:-1]])
        res = [None] * len(q)
        for k, i in enumerate(order):
            shape = (int(dims[0][k]), int(dims[1][k]), int(dims[2][k]), int(dims[3][k]))
            res[int(i)] = host[starts[k]:starts[k] + sizes[k]].reshape(shape)
        plan.destroy()
        return res
