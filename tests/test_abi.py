"""The C-ABI library loads and exports every entry point include/*.h declares.

No compute calls: this runs without a GPU.
"""
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(lvr_[a-z0-9_]+)\s*\(", src, re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_1801_01155_gb300 import lvr
    return lvr


def test_headers_declare_the_boundary():
    names = declared()
    for n in ("lvr_voxelize", "lvr_build_lod", "lvr_render", "lvr_create", "lvr_destroy"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    so = lib.LIB_PATH
    out = subprocess.run(["nm", "-D", "--defined-only", so], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = sorted(declared() - exported)
    assert not missing, f"declared but not exported: {missing}"
    for n in declared():
        assert hasattr(lib._L, n)


def test_binding_covers_the_header(lib):
    assert set(lib.ABI_SYMBOLS) <= declared()
    assert declared() <= set(lib.ABI_SYMBOLS), sorted(declared() - set(lib.ABI_SYMBOLS))
    assert lib.lvr_version() == 1


def test_structs_match_header_sizes(lib):
    import ctypes as C
    assert C.sizeof(lib.GridDesc) == 4 * 3 + 4 + 4 + 12 + 4 + 8
    assert C.sizeof(lib.View) == 12 * 3 + 4 + 8 + 16 + 12
    assert C.sizeof(lib.RenderDesc) == 4 + 4096 + 4 + 4 + 4 + 4 + 4 + 4 + 8 + 12 + 8 + 4 + 4 + 4


STRUCTS = {"lvr_grid_desc": "GridDesc", "lvr_lineset_info": "LineSetInfo", "lvr_lod_info": "LodInfo",
           "lvr_view": "View", "lvr_render_desc": "RenderDesc", "lvr_ao_train_desc": "AoTrainDesc",
           "lvr_ao_error": "AoError", "lvr_batch_item": "BatchItem", "lvr_tune": "Tune",
           "lvr_raster_stats": "RasterStats"}


def test_struct_layouts_match_the_c_compiler(lib, tmp_path):
    """Every binding struct has the size and field offsets gcc gives the header's struct."""
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "lvr.h"', "int main(void) {"]
    for cname, pyname in STRUCTS.items():
        lines.append(f'printf("{pyname} size %zu\\n", sizeof({cname}));')
        for f, _ in getattr(lib, pyname)._fields_:
            lines.append(f'printf("{pyname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    for line in filter(None, out):
        pyname, what, val = line.split()
        cls = getattr(lib, pyname)
        got = __import__("ctypes").sizeof(cls) if what == "size" else getattr(cls, what).offset
        assert got == int(val), (pyname, what, got, val)
