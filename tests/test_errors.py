"""Error paths that need no GPU: argument checks before any device call and the injected
allocation failure of eri_plan_create (ERI_INJECT_NOMEM), which must return ERI_E_NOMEM and
leave the output handle untouched."""
import ctypes
import os

import numpy as np
import pytest

from paper_2303_13632_gb300 import _lib, api, workloads as W


def tiny_shells():
    return W.make_shellset(np.zeros((2, 3)), [0, 1], [[1.0], [0.5]], [[1.0], [1.0]])


def test_injected_host_allocation_failure(monkeypatch):
    """k = 1 fails the host plan object, before any device call (so this runs without a GPU)."""
    lib = _lib.load()
    sh = tiny_shells()
    monkeypatch.setenv("ERI_INJECT_NOMEM", "1")
    arr = (_lib.eri_shell_t * 2)()
    exps = np.ascontiguousarray(sh.exps)
    coefs = np.ascontiguousarray(sh.coefs)
    for s in range(2):
        arr[s].L = int(sh.L[s])
        arr[s].nprim = 1
        arr[s].exps = ctypes.cast(exps.ctypes.data + 8 * s, _lib.c_double_p)
        arr[s].coefs = ctypes.cast(coefs.ctypes.data + 8 * s, _lib.c_double_p)
    q = np.array([[0, 1, 0, 1]], dtype=np.int32)
    out = ctypes.c_void_p(12345)
    st = lib.eri_plan_create(arr, 2, ctypes.c_void_p(q.ctypes.data), 1, None, ctypes.byref(out))
    assert st == _lib.ERI_E_NOMEM
    assert out.value == 12345  # untouched
    with pytest.raises(api.EriError) as e:
        api.eri_plan_create(sh, q)
    assert e.value.status == _lib.ERI_E_NOMEM


def test_invalid_shells_fail_before_the_device():
    sh = W.make_shellset(np.zeros((1, 3)), [0], [[-1.0]], [[1.0]])
    with pytest.raises(api.EriError) as e:
        api.eri_plan_create(sh, np.zeros((1, 4), dtype=np.int32))
    assert e.value.status == _lib.ERI_E_INVALID
    sh = W.make_shellset(np.zeros((1, 3)), [5], [[1.0]], [[1.0]])  # h shells: beyond L = 4
    with pytest.raises(api.EriError) as e:
        api.eri_plan_create(sh, np.zeros((1, 4), dtype=np.int32))
    assert e.value.status == _lib.ERI_E_UNSUPPORTED
    sh = W.make_shellset(np.zeros((1, 3)), [-1], [[1.0]], [[1.0]])
    with pytest.raises(api.EriError) as e:
        api.eri_plan_create(sh, np.zeros((1, 4), dtype=np.int32))
    assert e.value.status == _lib.ERI_E_INVALID
    sh = W.make_shellset(np.array([[np.nan, 0.0, 0.0]]), [0], [[1.0]], [[1.0]])
    with pytest.raises(api.EriError) as e:
        api.eri_plan_create(sh, np.zeros((1, 4), dtype=np.int32))
    assert e.value.status == _lib.ERI_E_INVALID


def test_status_names_have_no_timeout():
    assert api.eri_status_string(5) == "ERI_E_UNKNOWN"
    assert api.eri_status_string(_lib.ERI_E_NOMEM) == "ERI_E_NOMEM"
