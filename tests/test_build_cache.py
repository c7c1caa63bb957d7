"""The build's object cache: a unit's digest covers its source and every local header it
includes, directly or through other headers, so a changed header rebuilds exactly the units that
include it (a stale object would link old device code into the library)."""
import os

from paper_2303_13632_gb300 import build


def write(path, text):
    with open(path, "w") as f:
        f.write(text)


def test_unit_digest_follows_local_includes(tmp_path, monkeypatch):
    csrc, inc = tmp_path / "csrc", tmp_path / "include"
    csrc.mkdir()
    inc.mkdir()
    monkeypatch.setattr(build, "CSRC", str(csrc))
    monkeypatch.setattr(build, "ROOT", str(tmp_path))
    write(inc / "api.h", "int api;\n")
    write(csrc / "z.h", "int z;\n")
    write(csrc / "x.cuh", '#include "z.h"\n#include <cstdint>\n')
    write(csrc / "a.cu", '#include "x.cuh"\n#include "api.h"\n')
    write(csrc / "b.cu", '  #  include "api.h"\n')
    a0, b0 = build._unit_digest("a.cu", []), build._unit_digest("b.cu", [])
    assert build._unit_digest("a.cu", ["-DK=1"]) != a0  # defines are part of the key
    write(csrc / "z.h", "int z, w;\n")  # two levels below a.cu, not included by b.cu
    a1, b1 = build._unit_digest("a.cu", []), build._unit_digest("b.cu", [])
    assert a1 != a0 and b1 == b0
    write(inc / "api.h", "int api2;\n")  # the public header, included by both
    assert build._unit_digest("a.cu", []) != a1 and build._unit_digest("b.cu", []) != b1


def test_every_unit_of_the_library_has_a_distinct_key():
    keys = {(name, build._unit_digest(src, defs)) for name, src, defs in build._units()}
    names = [k[0] for k in keys]
    assert len(names) == len(set(names)) == len(build._units())
    # the class units share one source and differ only by their define
    class_keys = {h for n, h in keys if n.startswith("eri_classes_")}
    assert len(class_keys) == build.NUM_TU
    assert all(os.path.exists(os.path.join(build.CSRC, src)) for _, src, _ in build._units())
