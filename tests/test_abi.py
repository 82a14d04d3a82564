"""The C-ABI library builds, loads without a GPU and exports every function
that include/ssd.h declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names.update(re.findall(r"\b(sd_[a-z0-9_]+)\s*\(", txt))
    return sorted(names)


@pytest.fixture(scope="module")
def libssd():
    import paper_1503_02198_gb300 as pkg
    pkg.build()
    return pkg.lib()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("sd_create", "sd_set_state", "sd_residual", "sd_step", "sd_get_state", "sd_destroy",
                     "sd_sync", "sd_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(libssd):
    missing = [n for n in _declared() if not hasattr(libssd, n)]
    assert not missing, missing


def test_create_rejects_bad_arguments_without_touching_the_gpu(libssd):
    import paper_1503_02198_gb300 as pkg
    h = ctypes.c_void_p()
    # null mesh / params are rejected on the host before any CUDA call
    rc = libssd.sd_create(None, 2, None, ctypes.byref(h))
    assert rc == pkg.SD_ERR_ARG and not h.value
    assert b"null" in libssd.sd_create_error()


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    import paper_1503_02198_gb300 as pkg
    monkeypatch.setattr(pkg, "_lib", None)
    monkeypatch.setattr(pkg, "LIB_PATH", str(tmp_path / "nope.so"))
    with pytest.raises(RuntimeError):
        pkg.lib()


def test_ctypes_layouts_match_the_header(tmp_path):
    # sizes and field offsets of the public structs, as gcc lays out include/ssd.h
    import subprocess

    import paper_1503_02198_gb300 as pkg
    structs = {"sd_mesh": pkg.sd_mesh, "sd_zone": pkg.sd_zone, "sd_params": pkg.sd_params}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "ssd.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = {}
    for line in subprocess.check_output([str(exe)], text=True).splitlines():
        name, field, val = line.split()
        got[(name, field)] = int(val)
    for name, cls in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, (name, field)
    assert pkg.SD_MAX_ZONES == 4


def test_batched_form_is_held_unless_requested(libssd, monkeypatch):
    # the argument checks come first; then, without SSD_BATCH_ENABLE=1, the
    # batched form refuses to run (host only, no CUDA call)
    import paper_1503_02198_gb300 as pkg
    from ssd_inputs import meshes
    from ssd_inputs.workloads import FlowParams
    monkeypatch.delenv("SSD_BATCH_ENABLE", raising=False)
    m = meshes.periodic_box_mesh(3, 2.0)
    keep = []
    structs = [pkg._mesh_struct(m, keep) for _ in range(2)]
    mptrs = (ctypes.POINTER(pkg.sd_mesh) * 2)(*[ctypes.pointer(x) for x in structs])
    parr = (ctypes.c_int * 2)(2, 3)
    b = ctypes.c_void_p()
    mixed = (pkg.sd_params * 2)(pkg._params_struct(FlowParams(), 0), pkg._params_struct(FlowParams(), 1))
    assert libssd.sd_batch_create(2, mptrs, parr, mixed, 0.0, ctypes.byref(b)) == pkg.SD_ERR_ARG
    same = (pkg.sd_params * 2)(pkg._params_struct(FlowParams(), 1), pkg._params_struct(FlowParams(), 1))
    assert libssd.sd_batch_create(2, mptrs, parr, same, 0.0, ctypes.byref(b)) == pkg.SD_ERR_UNSUPPORTED
    assert not b.value
    assert b"SSD_BATCH_ENABLE" in libssd.sd_create_error()
