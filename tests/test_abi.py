"""CPU-side checks of the C ABI: the library builds and loads, exports every
function include/h2eig.h declares, and rejects bad arguments without a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pkg():
    import paper_2311_08618_gb300 as p
    from paper_2311_08618_gb300 import build
    build.build()
    return p


def declared_functions():
    src = open(os.path.join(ROOT, "include", "h2eig.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(h2_\w+)\s*\(", src, flags=re.M)))


def test_exports_every_declared_symbol(pkg):
    names = declared_functions()
    assert len(names) >= 10
    L = pkg.lib()
    for nm in names:
        assert hasattr(L, nm), nm
    assert sorted(pkg.EXPORTED_SYMBOLS) == names


def test_default_options(pkg):
    o = pkg.binding.default_options()
    assert o.precision == 0 and o.admissibility == 0 and o.eps_h2 == 1e-10
    assert o.max_lanes == 64 and o.fill_cap == 0
    # the header's documented defaults of the later options
    assert o.pivot_guard == 1e-3 and o.graphs == 1 and o.hbm_budget == 0
    assert o.tc_schur == 0 and o.lookahead == 0 and o.shifts_per_interval == 16


def test_struct_layouts_match_header(pkg, tmp_path):
    """The ctypes structures have the C compiler's sizes and offsets."""
    import subprocess
    src = tmp_path / "sz.c"
    src.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "h2eig.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(h2_options), offsetof(h2_options, stream),
         offsetof(h2_options, max_lanes), sizeof(h2_stats), offsetof(h2_stats, lanes),
         sizeof(h2_kernel), offsetof(h2_options, hbm_budget), offsetof(h2_stats, cap_bound),
         offsetof(h2_stats, max_residual), sizeof(h2_export_buf), offsetof(h2_export_buf, offsets),
         offsetof(h2_export_buf, B), offsetof(h2_options, tc_schur), offsetof(h2_options, lookahead),
         offsetof(h2_options, shifts_per_interval));
  return 0;
}
""")
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I" + os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    b = pkg.binding
    want = [C.sizeof(b.Options), b.Options.stream.offset, b.Options.max_lanes.offset,
            C.sizeof(b.Stats), b.Stats.lanes.offset, C.sizeof(b.Kernel), b.Options.hbm_budget.offset,
            b.Stats.cap_bound.offset, b.Stats.max_residual.offset, C.sizeof(b.ExportBuf),
            b.ExportBuf.offsets.offset, b.ExportBuf.B.offset, b.Options.tc_schur.offset,
            b.Options.lookahead.offset, b.Options.shifts_per_interval.offset]
    assert got == want


def test_invalid_arguments_rejected_without_gpu(pkg):
    L = pkg.lib()
    k = pkg.Kernel(0, (C.c_double * 4)(1e-3, 0, 0, 0))
    h = C.c_void_p()
    pts = np.zeros((4, 2))
    p = pts.ctypes.data_as(C.c_void_p)
    assert L.h2_build(p, 0, 2, k, 8, 4, 1.0, None, C.byref(h)) == -1
    assert L.h2_build(p, 4, 4, k, 8, 4, 1.0, None, C.byref(h)) == -1
    assert L.h2_build(p, 4, 2, k, 1, 4, 1.0, None, C.byref(h)) == -1
    assert L.h2_build(p, 4, 2, k, 8, 4, -1.0, None, C.byref(h)) == -1
    bad = pkg.Kernel(9, (C.c_double * 4)(0, 0, 0, 0))
    assert L.h2_build(p, 4, 2, bad, 8, 4, 1.0, None, C.byref(h)) == -1
    assert L.h2_build(None, 4, 2, k, 8, 4, 1.0, None, C.byref(h)) == -1
    assert b"null" in L.h2_last_error()
    nanpts = np.full((4, 2), np.nan)
    assert L.h2_build(nanpts.ctypes.data_as(C.c_void_p), 4, 2, k, 8, 4, 1.0, None, C.byref(h)) == -1
    assert L.h2_inertia(None, None, 1, None, None) == -1
    assert L.h2_kth_eig(None, None, 1, 1e-8, None, None) == -1
    assert L.h2_info(None, None) == -1
    L.h2_destroy(None)     # no-op


def test_no_cpu_fallback_without_gpu(pkg):
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    with pytest.raises(pkg.H2Error) as e:
        pkg.H2Matrix(np.random.default_rng(0).random((64, 2)), 0, leaf=16, rank=4)
    assert e.value.code == -6
