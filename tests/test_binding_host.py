"""Host-side marshalling of the Python binding (no GPU): array checks, the
boundary-condition struct, and the argument checks that happen before any
device work."""
import ctypes
import os

import numpy as np
import pytest

from paper_2102_01734_gb300 import build, rt3d


@pytest.fixture(scope="module")
def lib():
    build.build()
    return rt3d.load()


def test_ptr_accepts_contiguous_float64_only():
    a = np.zeros((3, 4))
    assert rt3d._ptr(a) == a.ctypes.data
    assert rt3d._ptr(None) is None
    with pytest.raises(ValueError):
        rt3d._ptr(np.zeros((3, 4), dtype=np.float32))
    with pytest.raises(ValueError):
        rt3d._ptr(np.zeros((4, 3)).T)
    with pytest.raises(TypeError):
        rt3d._ptr([1.0, 2.0])


def test_bc_struct_from_scalars_and_faces():
    keep = []
    assert rt3d._bc(None, keep) is None
    s = rt3d._bc({"I_top": 0.5, "I_bottom": 2.0}, keep)
    assert (s.I_top, s.I_bottom, s.I_irr) == (0.5, 2.0, 0.0)
    assert not s.I_top_face and not s.I_bottom_face
    face = np.arange(12, dtype=np.float64).reshape(3, 4)
    s = rt3d._bc({"I_bottom": face, "I_irr": 3.0}, keep)
    assert s.I_bottom == 0.0 and s.I_bottom_face == keep[-1].ctypes.data
    assert s.I_irr == 3.0
    # a non-contiguous or integer face array is converted, and kept alive
    s = rt3d._bc({"I_bottom": np.arange(12).reshape(4, 3).T}, keep)
    assert keep[-1].dtype == np.float64 and keep[-1].flags.c_contiguous
    assert not s.I_bottom_grad
    # the diffusion gradient face is marshalled as its own pointer
    grad = np.arange(12, dtype=np.float64).reshape(3, 4)
    s = rt3d._bc({"I_bottom": face, "I_bottom_grad": grad}, keep)
    assert s.I_bottom_grad == keep[-1].ctypes.data and s.I_bottom_face == keep[-2].ctypes.data


def test_struct_layouts_match_the_header():
    # rt3d_bc: 2 doubles, 2 pointers, 1 double, 1 pointer
    assert ctypes.sizeof(rt3d.BC) == 6 * 8
    assert rt3d.BC.I_bottom_grad.offset == 5 * 8
    # rt3d_grid_desc: geometry, n[3], ntheta, nphi, interp, precision,
    # nlambda (9 ints, +4 padding), stream pointer, accel (+4), r_in, r_out,
    # cache (+4), stream_bytes
    assert ctypes.sizeof(rt3d.GridDesc) == 9 * 4 + 4 + 8 + 4 + 4 + 2 * 8 + 4 + 4 + 8
    assert rt3d.FS_TUNE_SHAPES == 8


STRUCTS = {"GridDesc": "rt3d_grid_desc", "BC": "rt3d_bc", "SolveStats": "rt3d_solve_stats",
           "FsShape": "rt3d_fs_shape", "GridInfo": "rt3d_grid_info",
           "BatchStats": "rt3d_batch_stats", "LineStats": "rt3d_line_stats"}


def test_every_struct_matches_the_compiled_header(tmp_path):
    """Size and the offset of every field of each ctypes struct against the
    C compiler's layout of include/rt3d.h (gcc on this host)."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "rt3d.h"', "int main(void) {"]
    for py, c in STRUCTS.items():
        lines.append(f'printf("{py} size %zu\\n", sizeof({c}));')
        for name, _ in getattr(rt3d, py)._fields_:
            lines.append(f'printf("{py} {name} %zu\\n", offsetof({c}, {name}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.dirname(rt3d.HEADER), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    seen = 0
    for line in out.splitlines():
        py, key, val = line.split()
        cls = getattr(rt3d, py)
        want = ctypes.sizeof(cls) if key == "size" else getattr(cls, key).offset
        assert int(val) == want, (py, key, int(val), want)
        seen += 1
    assert seen == sum(1 + len(getattr(rt3d, py)._fields_) for py in STRUCTS)


def test_line_solve_checks_lengths_before_the_library(lib):
    with pytest.raises(ValueError):
        rt3d.line_solve(None, np.zeros(8), [1.0, 0.5], [1.0], np.zeros(8), np.zeros(8), None,
                        np.zeros(8))


def test_every_header_function_has_argument_types(lib):
    # the binding declares argtypes for every C entry point it calls, so a
    # wrong argument count fails in ctypes instead of on the device
    src = open(rt3d.__file__).read()
    for name in rt3d.header_functions([rt3d.HEADER]):
        assert f"lib.{name}.argtypes" in src, name
