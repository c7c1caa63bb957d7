"""The C-ABI library builds, loads without a GPU, and exports every function include/eri.h
declares; the host-only helpers answer correctly."""
import os
import re

import pytest

from paper_2303_13632_gb300 import _lib, api
from conftest import ROOT


def header_functions():
    text = open(os.path.join(ROOT, "include", "eri.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(eri_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = header_functions()
    for required in ["eri_plan_create", "eri_compute", "eri_compute_compressed", "eri_plan_destroy",
                     "eri_plan_class_info", "eri_output_bytes", "eri_sync", "eri_status_string"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = _lib.load()
    for name in header_functions():
        assert hasattr(lib, name), name
    assert set(header_functions()) == set(_lib.SIGNATURES)


def test_host_only_helpers():
    assert api.eri_class_id(1, 1, 1, 1) == 85
    assert api.eri_class_id(3, 3, 3, 3) == 255
    assert api.eri_class_shape(api.eri_class_id(3, 3, 3, 3)) == (10000, 7)
    assert api.eri_class_shape(api.eri_class_id(2, 2, 1, 0)) == (108, 3)
    assert api.eri_status_string(_lib.ERI_E_NUMERIC) == "ERI_E_NUMERIC"
    # classes with a g shell: 256 + ((La*5 + Lb)*5 + Lc)*5 + Ld
    assert api.eri_class_id(4, 0, 0, 0) == 256 + 500
    assert api.eri_class_id(4, 4, 4, 4) == 880
    assert api.eri_class_id(0, 1, 2, 4) == 256 + 39
    assert api.eri_class_shape(880) == (50625, 9)
    assert api.eri_class_shape(api.eri_class_id(4, 3, 2, 1)) == (15 * 10 * 6 * 3, 6)
    assert api.eri_class_id(5, 0, 0, 0) == -1
    for bad_id in (256, 256 + 3, 256 + 31, 881, -1):  # slots of no class
        with pytest.raises(_lib.EriError):
            api.eri_class_shape(bad_id)
    assert _lib.ERI_NUM_CLASS_IDS == 881


def test_paper512_stream_validates_before_touching_the_device():
    """Argument errors of the chunk re-layout come back as ERI_E_INVALID from host checks alone
    (no device call is made), and zero quartets is a no-op."""
    lib = _lib.load()
    ok, bad = _lib.ERI_OK, _lib.ERI_E_INVALID
    assert lib.eri_pack_paper512_stream(None, 0, 10, 16, None, None) == ok
    assert lib.eri_pack_paper512_stream(4096, 1, 0, 16, 8192, None) == bad      # n_eri < 1
    assert lib.eri_pack_paper512_stream(4096, 1, 50626, 16, 8192, None) == bad  # n_eri > 50625
    assert lib.eri_pack_paper512_stream(4096, 1, 10, 1, 8192, None) == bad      # bits < 2
    assert lib.eri_pack_paper512_stream(4096, 1, 10, 25, 8192, None) == bad     # bits > 24
    assert lib.eri_pack_paper512_stream(4098, 1, 10, 16, 8192, None) == bad     # misaligned
    assert lib.eri_pack_paper512_stream(None, 1, 10, 16, 8192, None) == bad     # null
    assert lib.eri_pack_paper512_stream(4096, -1, 10, 16, 8192, None) == bad    # negative count


C_CLIENT = r"""
#include <stdio.h>
#include <string.h>
#include "eri.h"
int main(void) {
    int32_t ne = 0, nr = 0;
    if (eri_class_id(3, 3, 3, 3) != 255 || eri_class_id(4, 0, 0, 0) != 756 || eri_class_id(5, 0, 0, 0) != -1) return 1;
    if (eri_class_shape(255, &ne, &nr) != ERI_OK || ne != 10000 || nr != 7) return 2;
    if (eri_class_shape(256, &ne, &nr) != ERI_E_INVALID || ERI_NUM_CLASS_IDS != 881) return 3;
    if (eri_class_shape(ERI_NUM_CLASS_IDS - 1, &ne, &nr) != ERI_OK || ne != 50625 || nr != 9) return 3;
    if (strcmp(eri_status_string(ERI_E_NUMERIC), "ERI_E_NUMERIC") != 0) return 4;
    if (eri_pack_paper512_stream(NULL, 0, 10, 16, NULL, NULL) != ERI_OK) return 5;
    if (eri_pack_paper512_stream((const void *)4096, 1, 10, 25, (void *)8192, NULL) != ERI_E_INVALID)
        return 6;
    if (eri_plan_num_quartets(NULL, NULL) != ERI_E_INVALID) return 7;
    {
        /* option checks happen before any device call */
        eri_plan_opts_t o;
        eri_plan_t p = NULL;
        memset(&o, 0, sizeof o);
        o.quartet_mode = ERI_UNIQUE8;
        o.schwarz_threshold = -1.0;
        if (eri_plan_create(NULL, 0, NULL, 0, &o, &p) != ERI_E_INVALID || p != NULL) return 8;
        o.schwarz_threshold = 1e-10;
        o.shard_count = 4;
        o.shard_index = 4;
        if (eri_plan_create(NULL, 0, NULL, 0, &o, &p) != ERI_E_INVALID) return 9;
        o.quartet_mode = ERI_EXPLICIT;
        o.shard_index = 0;
        if (eri_plan_create(NULL, 0, NULL, 0, &o, &p) != ERI_E_INVALID) return 10;
        o.quartet_mode = 7;
        o.shard_count = 0;
        if (eri_plan_create(NULL, 0, NULL, 0, &o, &p) != ERI_E_INVALID) return 11;
    }
    if (eri_plan_screening(NULL, NULL, NULL) != ERI_E_INVALID) return 12;
    if (eri_plan_num_basis_functions(NULL, NULL) != ERI_E_INVALID) return 13;
    if (eri_digest_jk(NULL, 16, NULL, NULL, NULL, NULL, NULL, ERI_DIGEST_UNIQUE8, NULL) != ERI_E_INVALID)
        return 14;
    eri_plan_destroy(NULL);
    puts("ok");
    return 0;
}
"""


def test_header_is_plain_c_and_links(tmp_path):
    """A C99 program includes eri.h under -pedantic -Werror, links the library by name and calls
    the host-only entry points (no device needed): the boundary is a plain C ABI."""
    import shutil
    import subprocess
    from paper_2303_13632_gb300 import build
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    lib = build.build()
    src = tmp_path / "client.c"
    src.write_text(C_CLIENT)
    exe = tmp_path / "client"
    libdir = os.path.dirname(lib)
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                        "-I", os.path.join(ROOT, "include"), str(src), "-L", libdir, "-leri_gb300",
                        f"-Wl,-rpath,{libdir}", "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", (r.returncode, r.stdout, r.stderr)
