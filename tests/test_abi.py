"""Host-side checks of the C-ABI library: it builds, loads without a GPU and exports every
entry point that include/map.h declares.  No compute call is made here."""
import os
import re
import subprocess

import numpy as np
import pytest

import paper_0912_2555_gb300 as pkg
from paper_0912_2555_gb300 import build as gpu_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for hdr in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if hdr.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", hdr)).read()
            names += re.findall(r"^MAP_API\s+[\w\s\*]+?\b(\w+)\s*\(", txt, flags=re.M)
    return names


@pytest.fixture(scope="module")
def lib():
    gpu_build.build()
    return pkg.load()


def test_header_declares_entry_points():
    names = _declared()
    assert {"map_create", "map_run", "map_destroy", "map_last_error"} <= set(names)
    assert set(names) == set(pkg.EXPORTS), "binding and header disagree"


def test_every_declared_symbol_is_exported(lib):
    out = subprocess.check_output(["nm", "-D", "--defined-only", pkg.LIB_PATH], text=True)
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    for name in _declared():
        assert name in exported, f"{name} declared in include/ but not exported"
        assert hasattr(lib, name)


def test_library_is_sm103a(lib):
    # the cubin inside is for sm_103a only (compile flags of the build script)
    assert "arch=compute_103a,code=sm_103a" in " ".join(gpu_build.ARCH)


def test_argument_errors_without_compute(lib):
    import ctypes
    h = ctypes.c_void_p()
    rp = np.array([0, 1], np.uint32)
    ab = np.array([1], np.uint32)
    # n = 0 and n >= 2^31 - 1 are rejected before any CUDA call
    assert lib.map_create(0, rp.ctypes.data, None, ab.ctypes.data, None, ctypes.byref(h)) == pkg.MAP_ERR_ARG
    assert lib.map_create(0x7FFFFFFF, rp.ctypes.data, None, ab.ctypes.data, None, ctypes.byref(h)) == pkg.MAP_ERR_ARG
    assert lib.map_create(1, None, None, ab.ctypes.data, None, ctypes.byref(h)) == pkg.MAP_ERR_ARG
    assert lib.map_run(None, None, None, None) == pkg.MAP_ERR_ARG
    assert "NULL" in pkg.last_error()
    assert lib.map_destroy(None) == pkg.MAP_OK


def test_pack_bits_lsb_first():
    flags = np.zeros(70, np.uint8)
    flags[[0, 31, 32, 69]] = 1
    bits = pkg.pack_bits(flags)
    assert bits.tolist() == [1 | (1 << 31), 1, 1 << 5]


def test_binding_structs_match_the_header(tmp_path):
    """The ctypes mirrors of map_opts, map_result and map_tune_result have the header's size and
    field offsets (compiled with the host compiler against include/map.h)."""
    import ctypes

    structs = {"map_opts": pkg.MapOpts, "map_result": pkg.MapResult, "map_tune_result": pkg.TuneResult}
    src = ["#include <stddef.h>", "#include <stdio.h>", '#include "map.h"', "int main(void) {"]
    for cname, cls in structs.items():
        src.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            src.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    src += ["return 0; }"]
    c = tmp_path / "abi.c"
    c.write_text("\n".join(src))
    exe = tmp_path / "abi"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(c)])
    got = {}
    for line in subprocess.check_output([str(exe)], text=True).splitlines():
        cname, field, value = line.split()
        got[(cname, field)] = int(value)
    for cname, cls in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert got[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)
