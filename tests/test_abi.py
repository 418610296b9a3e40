"""The C-ABI library builds, loads and exports every entry point include/*.h declares.
CPU only: no call here touches a GPU."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:gbs_status|void|const char\s*\*)\s+(gbs_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def libpath():
    import __graft_entry__
    return __graft_entry__._build_module().build()


def test_header_declares_entry_points():
    names = _declared()
    assert {"gbs_create", "gbs_select_kth_f32", "gbs_median_f64", "gbs_status_string"} <= names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = _declared() - exported
    assert not missing, missing


def test_binding_covers_header(libpath):
    import paper_1104_2732_gb300 as gbs
    missing = _declared() - set(gbs.EXPORTED)
    assert not missing, missing
    for name in _declared():
        assert callable(getattr(gbs, name))


def test_host_side_checks_need_no_gpu(libpath):
    import paper_1104_2732_gb300 as gbs
    assert gbs.gbs_status_string(0) == b"ok"
    assert gbs.gbs_status_string(2) == b"input contains NaN"
    # NULL context / bad arguments are rejected before any CUDA call
    assert gbs.gbs_select_kth_f32(None, None, 10, 1, None, None) == gbs.GBS_EINVAL
    assert gbs.gbs_median_f64(None, None, 0, None, None) == gbs.GBS_EINVAL
    assert gbs.gbs_cost_pass_f32(None, None, 5, 1, 0.0, 1.0, None, None) == gbs.GBS_EINVAL
    assert gbs.gbs_create(None, 0) == gbs.GBS_EINVAL
    assert gbs.gbs_knn_regress_f32(None, None, 10, 2, None, None, 1, 1, 0, 0.0, None, None, None) == gbs.GBS_EINVAL
    assert gbs.gbs_knn_classify_f32(None, None, 10, 2, None, 3, None, 1, 1, None, None, None, None) == gbs.GBS_EINVAL


def test_struct_sizes_match_header(libpath):
    """The ctypes mirrors of the header's structs have the C layout's sizes."""
    import paper_1104_2732_gb300 as gbs
    assert ctypes.sizeof(gbs.gbs_config) == 8 + 4 * 10
    assert ctypes.sizeof(gbs.gbs_cost_eval) == 48
    assert ctypes.sizeof(gbs.gbs_array_stats) == 88
    assert ctypes.sizeof(gbs.gbs_shard_state) == 3 * 8 + 8 * 4 + 5 * 8 + 5 * 8 + 2 * 4 + 5 * 8
    assert ctypes.sizeof(gbs.gbs_run_stats) == 4 * 8 + 3 * 8 + 64 * 8 * 2 + 72 * 8 + 64 * 8 + 8


def test_struct_layouts_and_constants_match_the_c_compiler(libpath, tmp_path):
    """Every field offset and struct size of the ctypes mirrors, every GBS_* constant of
    the binding and its names of the GBS_HOW_* codes equal what a C compiler reads from
    include/gbselect.h (a field or constant missing from the header fails to compile)."""
    import paper_1104_2732_gb300 as gbs
    structs = [gbs.gbs_config, gbs.gbs_run_stats, gbs.gbs_array_stats, gbs.gbs_cost_eval, gbs.gbs_shard_state,
               gbs.gbs_knn_stats, gbs.gbs_lms_stats]
    consts = sorted(n for n in dir(gbs) if re.fullmatch(r"GBS_[A-Z0-9_]+", n) and isinstance(getattr(gbs, n), int))
    assert consts
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "gbselect.h"', "int main(void) {"]
    want = []
    for s in structs:
        name = s.__name__
        lines.append(f'  printf("{name} sizeof %zu\\n", sizeof({name}));')
        want.append(f"{name} sizeof {ctypes.sizeof(s)}")
        for f, _ in s._fields_:
            lines.append(f'  printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
            want.append(f"{name} {f} {getattr(s, f).offset}")
    for n in consts:
        lines.append(f'  printf("{n} %lld\\n", (long long)({n}));')
        want.append(f"{n} {getattr(gbs, n)}")
    for code, how in sorted(gbs.HOW.items()):   # the binding's names of GBS_HOW_*
        lines.append(f'  printf("GBS_HOW_{how.upper()} %d\\n", (int)GBS_HOW_{how.upper()});')
        want.append(f"GBS_HOW_{how.upper()} {code}")
    lines.append("  return 0;\n}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    got = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")[:-1]
    assert got == want

