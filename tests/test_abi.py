"""The C ABI: the in-tree library builds for sm_103a, loads, and exports every entry point
declared in include/vrte.h. No compute call is made (this runs without a GPU)."""
import ctypes
import os
import re

import pytest

import paper_1707_05882_gb300 as vr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "vrte.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(vrte_[a-z_]+)\s*\(", src)))


def test_header_declares_the_documented_entry_points():
    names = declared_functions()
    for n in ["vrte_plan_create", "vrte_set_layer", "vrte_solve_brdf", "vrte_brdf_backward",
              "vrte_destroy", "vrte_status_string", "vrte_plan_status", "vrte_solve_brdf_host"]:
        assert n in names


def test_library_loads_and_exports_every_declared_symbol():
    lib = vr.load_library(build_if_missing=True)
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def test_status_strings_without_gpu():
    lib = vr.load_library()
    for code in range(9):
        s = lib.vrte_status_string(code)
        assert isinstance(s, bytes) and len(s) > 0
    assert lib.vrte_status_string(0) == b"ok"


def test_null_arguments_are_rejected_without_device_work():
    lib = vr.load_library()
    h = ctypes.c_void_p()
    assert lib.vrte_plan_create(None, ctypes.byref(h)) == 1
    assert lib.vrte_plan_status(None) == 1
    assert lib.vrte_solve_brdf(None, None, 0, None) == 1
    assert lib.vrte_workspace_bytes(None) == 0
    lib.vrte_destroy(None)


def test_plan_descriptor_layout_matches_header(tmp_path):
    """The ctypes mirrors of vrte_plan_desc, vrte_layer and vrte_stage_stat have the sizes and
    field offsets that a C compiler gives the structs of include/vrte.h."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "layout.c"
    src.write_text("""#include <stdio.h>
#include <stddef.h>
#include "vrte.h"
int main(void) {
  printf("%zu %zu %zu %zu\\n", sizeof(vrte_plan_desc), offsetof(vrte_plan_desc, mu_in),
         offsetof(vrte_plan_desc, precision), offsetof(vrte_plan_desc, flags));
  printf("%zu %zu %zu %zu\\n", sizeof(vrte_layer), offsetof(vrte_layer, n_nodes),
         offsetof(vrte_layer, base_albedo), offsetof(vrte_layer, base_mueller));
  printf("%zu %zu\\n", sizeof(vrte_stage_stat), offsetof(vrte_stage_stat, tc_flops));
  return 0;
}
""")
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run([cc, "-I", inc, str(src), "-o", str(exe)], check=True)
    vals = [list(map(int, line.split())) for line in
            subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
            if line.strip()]
    assert vals[0] == [ctypes.sizeof(vr.PlanDesc), vr.PlanDesc.mu_in.offset,
                       vr.PlanDesc.precision.offset, vr.PlanDesc.flags.offset]
    assert vals[1] == [ctypes.sizeof(vr.Layer), vr.Layer.n_nodes.offset, vr.Layer.base_albedo.offset,
                       vr.Layer.base_mueller.offset]
    assert vals[2] == [ctypes.sizeof(vr.StageStat), vr.StageStat.tc_flops.offset]


def test_sliced_gemm_workspace_sizes_without_gpu():
    """Host-side sizing of the sliced GEMM's workspace: rejected shapes give 0 (K outside
    1..1024, slices outside 1..8, empty M, N or batch); valid ones grow with the batch by
    the slice images of one more unit (the epilogue scratch does not grow)."""
    lib = vr.load_library()
    ws = lib.vrte_gemm_sliced_workspace
    assert ws(128, 64, 0, 1, 7) == 0
    assert ws(128, 64, 1025, 1, 7) == 0
    assert ws(128, 64, 64, 1, 0) == 0
    assert ws(128, 64, 64, 1, 9) == 0
    assert ws(0, 64, 64, 1, 7) == 0 and ws(128, 0, 64, 1, 7) == 0 and ws(128, 64, 64, 0, 7) == 0
    one, two, three = ws(200, 100, 300, 1, 7), ws(200, 100, 300, 2, 7), ws(200, 100, 300, 3, 7)
    assert 0 < one < two < three
    # one unit of slices: (256 rows + 128 columns) x 320 K (padded to 32) x 7 slices x 2 bytes,
    # plus the per-row and per-column exponents, each part rounded up to 1 KiB
    unit = 2 * 7 * 320 * (256 + 128) + 4 * (256 + 128)
    assert abs((three - two) - unit) <= 4 * 1024
    assert ws(200, 100, 300, 1, 4) < one
