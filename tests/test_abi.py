"""The C ABI without a GPU: the library loads, exports every function that
include/augwarp.h declares, the Python descriptor layout matches the C
struct, and host-side argument checks reject bad calls."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "augwarp.h")


@pytest.fixture(scope="module")
def aw():
    from paper_1811_11226_b300 import build
    build.build()
    from paper_1811_11226_b300 import augwarp
    return augwarp


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", text,
                       flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "defined", "__attribute__")))


def test_every_declared_symbol_is_exported(aw):
    names = declared_functions()
    assert "aug_warp_fwd" in names and "iou_loss_fwd_bwd" in names and "aug_warp_bwd" in names
    out = subprocess.run(["nm", "-D", "--defined-only", aw.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    lib = C.CDLL(aw.LIB_PATH)
    for n in names:
        getattr(lib, n)


def test_descriptor_layout_matches_header(aw, tmp_path):
    fields = aw.DESC_DTYPE.names
    src = tmp_path / "layout.c"
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "augwarp.h"',
             'int main(void) {', ' printf("%zu %zu\\n", sizeof(aug_volume_desc), '
             '_Alignof(aug_volume_desc));']
    for f in fields:
        lines.append(f' printf("%zu\\n", offsetof(aug_volume_desc, {f}));')
    lines.append(" return 0; }")
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                           check=True).stdout.split()]
    assert vals[0] == aw.DESC_DTYPE.itemsize == 144 and vals[1] == 16
    assert vals[2:] == [aw.DESC_DTYPE.fields[f][1] for f in fields]


def test_status_strings_and_variants(aw):
    assert aw.status_string(0) == "ok"
    assert "descriptor" in aw.status_string(aw.AUG_ERR_DESCRIPTOR)
    assert aw.status_string(99) == "unknown status"
    for op in (aw.OP_FWD, aw.OP_BWD, aw.OP_IOU):
        n = aw.aug_num_variants(op)
        assert n >= 2
        assert len({aw.aug_variant_name(op, v) for v in range(n)}) == n
        assert aw.aug_variant_name(op, n) == "invalid"
    assert aw.aug_version() >= 10000


def test_host_argument_checks_without_gpu(aw):
    L = aw.lib()
    # Host-side checks happen before any CUDA call.
    assert L.aug_warp_fwd(None, 1, 0, None, 0, None) == aw.AUG_ERR_INVALID_ARG
    assert L.aug_warp_fwd(C.c_void_p(256), 0, 0, None, 0, None) == aw.AUG_ERR_INVALID_ARG
    assert L.aug_warp_fwd(C.c_void_p(256), 1, 0, None, 0, None) == aw.AUG_ERR_WORKSPACE
    assert L.aug_warp_fwd(C.c_void_p(256), 1, 0, C.c_void_p(257), 1 << 30, None) == \
        aw.AUG_ERR_WORKSPACE
    assert L.iou_loss_fwd_bwd(C.c_void_p(256), 1, C.c_void_p(256), 9, C.c_void_p(256), None,
                              C.c_void_p(256), 1 << 30, None) == aw.AUG_ERR_UNSUPPORTED
    assert L.aug_set_variant(0, 10_000) == aw.AUG_ERR_INVALID_ARG
    assert L.aug_set_variant(7, 0) == aw.AUG_ERR_INVALID_ARG
    assert L.aug_philox4x32_10(None, -1, 0, None, None) == aw.AUG_ERR_INVALID_ARG
    assert L.aug_loss_batch_mean(None, 1, C.c_void_p(256), None) == aw.AUG_ERR_INVALID_ARG
    assert L.aug_loss_batch_mean(C.c_void_p(256), 0, C.c_void_p(256), None) == \
        aw.AUG_ERR_INVALID_ARG
    # A host descriptor with a zero dimension is rejected synchronously.
    h = np.zeros(1, aw.DESC_DTYPE)
    assert L.aug_warp_fwd_volume(h.ctypes.data_as(C.c_void_p), 0, None) == \
        aw.AUG_ERR_DESCRIPTOR
    h["in_nx"], h["in_ny"], h["in_nz"] = 4, 4, 4
    h["out_nx"], h["out_ny"], h["out_nz"] = 4, 4, 4
    h["affine"][0, [0, 5, 10]] = 1.0
    h["photo_a"] = 1.0
    h["affine"][0, 0] = np.inf
    assert L.aug_warp_fwd_volume(h.ctypes.data_as(C.c_void_p), 0, None) == \
        aw.AUG_ERR_DESCRIPTOR


def test_struct_sizes_match_the_header():
    import ctypes
    from paper_1811_11226_b300 import augwarp as A
    assert A.DESC_DTYPE.itemsize == 144
    assert ctypes.sizeof(A.ParamSpec) == 128
