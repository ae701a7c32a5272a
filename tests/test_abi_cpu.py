"""The C ABI without a GPU: the library loads, exports every declared entry
point, the ctypes structs match the C layout, and argument checks that run
before any CUDA call return the documented status."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mvs.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mvs_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol(mvs_lib):
    names = _declared()
    assert "mvs_patchmatch" in names and "mvs_plane_infer" in names and "mvs_geo_filter" in names
    out = subprocess.run(["nm", "-D", "--defined-only", mvs_lib.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (mvs_[a-z_0-9]+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, f"not exported: {missing}"
    lib = mvs_lib.load()
    for n in names:
        assert hasattr(lib, n)


def test_ctypes_structs_match_c_layout(mvs_lib):
    prog = r"""
#include <stdio.h>
#include <stddef.h>
#include "mvs.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\n", sizeof(mvs_camera), sizeof(mvs_pm_params), sizeof(mvs_depth_map),
         sizeof(mvs_filter_params), sizeof(mvs_phi_params));
  printf("%zu %zu %zu %zu %zu %zu\n", offsetof(mvs_pm_params, seed), offsetof(mvs_pm_params, precision),
         offsetof(mvs_camera, width), offsetof(mvs_phi_params, hole_cost), offsetof(mvs_pm_params, init_range),
         offsetof(mvs_phi_params, selection));
  printf("%d %d\n", MVS_PHI_SELECT_MRF, MVS_PHI_SELECT_MIN_COST);
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(prog)
        exe = os.path.join(d, "t")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        lines = subprocess.check_output([exe], text=True).split("\n")
    sizes = [int(x) for x in lines[0].split()]
    offs = [int(x) for x in lines[1].split()]
    m = mvs_lib
    assert sizes == [C.sizeof(m.mvs_camera), C.sizeof(m.mvs_pm_params), C.sizeof(m.mvs_depth_map),
                     C.sizeof(m.mvs_filter_params), C.sizeof(m.mvs_phi_params)]
    assert offs == [m.mvs_pm_params.seed.offset, m.mvs_pm_params.precision.offset, m.mvs_camera.width.offset,
                    m.mvs_phi_params.hole_cost.offset, m.mvs_pm_params.init_range.offset,
                    m.mvs_phi_params.selection.offset]
    assert [int(x) for x in lines[2].split()] == [m.MVS_PHI_SELECT_MRF, m.MVS_PHI_SELECT_MIN_COST]


def test_create_rejects_bad_arguments_before_touching_cuda(mvs_lib):
    lib = mvs_lib.load()
    h = C.c_void_p()
    assert lib.mvs_create(None, None, 2, None, C.byref(h)) == mvs_lib.MVS_EINVAL
    assert b"NULL" in lib.mvs_last_error(None)
    cams = (mvs_lib.mvs_camera * 1)()
    ptrs = (C.c_void_p * 1)()
    assert lib.mvs_create(cams, ptrs, 1, None, C.byref(h)) == mvs_lib.MVS_EINVAL
    cams2 = (mvs_lib.mvs_camera * 2)()
    img = np.zeros((4, 4), np.uint8)
    ptrs2 = (C.c_void_p * 2)(img.ctypes.data, img.ctypes.data)
    for c in cams2:
        c.width, c.height = 4, 4
    # singular K
    assert lib.mvs_create(cams2, ptrs2, 2, None, C.byref(h)) == mvs_lib.MVS_EINVAL
    assert b"K" in lib.mvs_last_error(None)
    # non-finite pose
    for c in cams2:
        c.K[0], c.K[4], c.K[8] = 10.0, 10.0, 1.0
    cams2[1].t[0] = float("nan")
    assert lib.mvs_create(cams2, ptrs2, 2, None, C.byref(h)) == mvs_lib.MVS_EINVAL
    # bad sizes
    cams2[1].t[0] = 0.0
    cams2[1].width = 0
    assert lib.mvs_create(cams2, ptrs2, 2, None, C.byref(h)) == mvs_lib.MVS_EINVAL
    assert not h.value


def test_null_context_is_rejected(mvs_lib):
    lib = mvs_lib.load()
    p = mvs_lib.PMParams().c()
    srcs = (C.c_int32 * 1)(1)
    out = mvs_lib.mvs_depth_map(None, None, 0)
    assert lib.mvs_patchmatch(None, 0, srcs, 1, C.byref(p), C.byref(out)) == mvs_lib.MVS_EINVAL
    assert lib.mvs_profile(None, 1) == mvs_lib.MVS_EINVAL
    views = (C.c_int32 * 1)(0)
    n = C.c_int64(0)
    assert lib.mvs_fuse(None, 1, views, None, C.c_float(0.01), None, None, None, 0, C.byref(n), 0) == mvs_lib.MVS_EINVAL
    nbr = np.zeros((2, 1), np.int32)
    assert lib.mvs_select_neighbors(None, 0, None, None, 0.002, 0.1, 1, nbr.ctypes.data, None, None, None,
                                    0) == mvs_lib.MVS_EINVAL
    rng = np.zeros((2, 2, 2), np.float32)
    assert lib.mvs_sparse_depth_range(None, 0, 0, None, None, None, None, 2.0, C.c_float(2.0), C.c_float(8.0),
                                      rng.ctypes.data, 1) == mvs_lib.MVS_EINVAL
    pl = np.zeros((2, 2, 4), np.float32)
    assert lib.mvs_phi_select_min_cost(None, 0, None, None, None, None, pl.ctypes.data_as(C.POINTER(C.c_float)),
                                       1) == mvs_lib.MVS_EINVAL
    lib.mvs_destroy(None)   # NULL-safe


def test_binding_rejects_mixed_memory(mvs_lib):
    torch = pytest.importorskip("torch")
    with pytest.raises(ValueError):
        mvs_lib._mem(np.zeros(4, np.float32), torch.zeros(4).pin_memory() if torch.cuda.is_available() else
                     _FakeCuda())


class _FakeCuda:
    is_cuda = True

    def data_ptr(self):
        return 0

    def is_contiguous(self):
        return True
