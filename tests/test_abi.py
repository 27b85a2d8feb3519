"""The C ABI library builds for sm_103a, loads, and exports every entry point its header declares.
No compute call is made here (no GPU)."""
import ctypes
import os
import re

import pytest

import paper_1907_04229_gb300 as cp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "cptr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cptr_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    cp.build()
    return cp.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(cp._SIGS), set(names) ^ set(cp._SIGS)


def test_bounds_checking_build_exports_the_same_symbols():
    """libcptr_check.so (-DCPTR_CHECK) is the same library with index checks: every declared
    entry point is exported (loaded by path here; the package's own library stays the default)."""
    from paper_1907_04229_gb300 import _build
    path = _build.build(variant="check")
    chk = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(chk, name), name


def test_library_targets_sm103a():
    # the fat binary embeds sm_103a code only; cuobjdump is not needed: nvcc's -gencode list is fixed
    from paper_1907_04229_gb300 import _build
    assert _build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert os.path.getsize(_build.LIB) > 100_000


def test_default_options(lib):
    o = cp.cptr_default_options()
    assert (o.stage1, o.stage2, o.schur, o.smoother) == (0, 0, 0, 0)
    assert abs(o.theta - 0.25) < 1e-15 and abs(o.omega - 2.0 / 3.0) < 1e-15
    assert (o.n_coarse, o.max_levels, o.restart, o.max_it, o.dense_max) == (256, 25, 30, 1000, 1024)
    assert (o.check_every, o.use_graph) == (1, 1)


def test_option_struct_layout_matches_header():
    # cptr_options: 4 int32, 2 doubles, 12 int32, one pointer, 7 int32 (+ padding)
    assert ctypes.sizeof(cp.cptr_options) == 16 + 16 + 48 + 8 + 32
    assert cp.cptr_options.stream.offset == 80
    # cptr_instance: int32 (+ padding), five pointers
    assert ctypes.sizeof(cp.cptr_instance) == 8 + 5 * 8
    assert ctypes.sizeof(cp.cptr_stats) == 24 + 7 * 8


def test_struct_layouts_match_the_c_compiler(tmp_path):
    """The binding's ctypes structures against the C compiler's own layout of the header: the size
    of each struct and the offset of every field."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"cptr_options": cp.cptr_options, "cptr_instance": cp.cptr_instance, "cptr_stats": cp.cptr_stats}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "cptr.h"', "int main(void) {"]
    for name, st in structs.items():
        lines.append(f'printf("{name} sizeof %zu\\n", sizeof({name}));')
        for f in st._fields_:
            lines.append(f'printf("{name} {f[0]} %zu\\n", offsetof({name}, {f[0]}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    seen = 0
    for line in filter(None, out):
        name, field, value = line.split()
        st = structs[name]
        expect = ctypes.sizeof(st) if field == "sizeof" else getattr(st, field).offset
        assert int(value) == expect, (name, field, value, expect)
        seen += 1
    assert seen == sum(len(st._fields_) + 1 for st in structs.values())


def test_invalid_options_are_rejected_before_any_device_work(lib):
    # cptr_create validates its options first and returns CPTR_EINVAL without touching a device
    for kw in (dict(csr_lanes=-1), dict(csr_lanes=3), dict(csr_lanes=64), dict(use_graph=3), dict(restart=0),
               dict(ilu_group=1), dict(ilu_group=5), dict(ilu_group=-1), dict(ilu_lanes=2), dict(ilu_lanes=32)):
        o = cp.cptr_default_options(**kw)
        h = ctypes.c_void_p()
        assert lib.cptr_create(ctypes.byref(h), ctypes.byref(o)) == -1, kw
        assert not h.value


def test_null_context_is_rejected(lib):
    assert lib.cptr_setup(None, 1, 3, None, None, None, None, None, None, 0) == -1
    assert lib.cptr_solve(None, None, None, 1e-6, None, 0) == -1
    assert lib.cptr_last_error(None) == b"null context"
