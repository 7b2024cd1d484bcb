"""Host-side checks of the C ABI (no GPU needed): the library builds, loads,
exports every function include/rt3d.h declares, and rejects bad descriptors
before touching a device."""
import ctypes

import pytest

from paper_2102_01734_gb300 import build, rt3d


@pytest.fixture(scope="module")
def lib():
    build.build()
    return rt3d.load()


def test_header_declares_the_boundary():
    names = rt3d.header_functions()
    for required in ("rt3d_grid_create", "rt3d_grid_destroy", "rt3d_formal_solution",
                     "rt3d_os_solve", "rt3d_ali_step", "rt3d_solve", "rt3d_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in rt3d.header_functions():
        assert hasattr(lib, name), name


@pytest.mark.parametrize("n,nth,nph,interp,prec", [
    ((3, 8, 8), 4, 4, 0, 0),        # nx < 4
    ((8, 8, 0), 4, 4, 0, 0),        # nz < 1
    ((2048, 8, 8), 4, 4, 0, 0),     # nx too large
    ((2047, 2047, 200), 4, 4, 0, 0),  # replicated arrays beyond 2^31 elements
    ((8, 8, 8), 0, 4, 0, 0),        # no angles
    ((8, 8, 8), 4, 4, 7, 0),        # bad interpolation
    ((8, 8, 8), 4, 4, 0, 9),        # bad precision
])
def test_bad_descriptor_is_einval(lib, n, nth, nph, interp, prec):
    with pytest.raises(rt3d.RT3DError) as ei:
        rt3d.grid_create(n, nth, nph, interp, prec, stream=0)
    assert ei.value.status == rt3d.EINVAL
    assert rt3d.last_error()


@pytest.mark.parametrize("geometry,cache,stream_bytes", [
    (rt3d.CARTESIAN_PERIODIC_XY, rt3d.CACHE_HOST_STREAMED, 0),  # host cache: spherical only
    (rt3d.CARTESIAN_PERIODIC_XY, rt3d.CACHE_HOST_MAPPED, 0),
    (rt3d.CARTESIAN_PERIODIC_XY, rt3d.CACHE_HOST_CHORDS, 0),
    (rt3d.SPHERICAL, 4, 0),                                     # no such mode
    (rt3d.SPHERICAL, rt3d.CACHE_HOST_STREAMED, -1),             # negative chunk size
])
def test_bad_cache_mode_is_einval(lib, geometry, cache, stream_bytes):
    with pytest.raises(rt3d.RT3DError) as ei:
        rt3d.grid_create((8, 6, 8), 2, 4, stream=0, geometry=geometry, cache=cache,
                         stream_bytes=stream_bytes)
    assert ei.value.status == rt3d.EINVAL
    assert "cache" in rt3d.last_error() or "stream_bytes" in rt3d.last_error()


def test_null_arguments_are_einval(lib):
    assert lib.rt3d_grid_create(None, None) == rt3d.EINVAL
    assert lib.rt3d_formal_solution(None, None, None, None, None, None) == rt3d.EINVAL
    assert lib.rt3d_solve(None, None, None, None, None, None, 1e-8, 10, None) == rt3d.EINVAL
    st = rt3d.SolveStats()
    # 4 ints, 6 doubles, 1 long long, fs_ff (+4 padding), fsff_ms, rounds,
    # 2 x 16 ints (+4 padding), 2 x 16 doubles, fs_lstar (+4 padding), fs32_lstar_ms
    assert ctypes.sizeof(st) == (4 * 4 + 6 * 8 + 8 + 8 + 8 + 4 + 2 * 16 * 4 + 4 + 2 * 16 * 8
                                 + 4 + 4 + 8)
    assert lib.rt3d_formal_solution_ff(None, None, None, None, None) == rt3d.EINVAL
    # + sm_count, cache, host_bytes, cache_chunks (+4 padding)
    assert ctypes.sizeof(rt3d.GridInfo) == 2 * 4 + 2 * 8 + 4 * 4 + 8 * 4 + 4 + 4 + 8 + 4 + 4
    assert lib.rt3d_grid_set_fs_shape(None, None) == rt3d.EINVAL
    assert lib.rt3d_grid_invalidate_lstar(None) == rt3d.EINVAL
    assert lib.rt3d_grid_set_os_solver(None, rt3d.OS_JACOBI) == rt3d.EINVAL
    assert lib.rt3d_diffusion_bc(None, 1, None, None, None, None) == rt3d.EINVAL
    assert lib.rt3d_line_solve(None, 1, None, None, None, None, None, None, None, 1e-8, 10,
                               None) == rt3d.EINVAL
    # 3 ints (+4 padding), 4 doubles, 1 long long, 1 int (+4 padding), 2 doubles
    assert ctypes.sizeof(rt3d.LineStats) == 3 * 4 + 4 + 4 * 8 + 8 + 4 + 4 + 2 * 8


def test_fs_tune_shapes_are_valid(lib):
    shapes = [rt3d.fs_tune_shape(i) for i in range(rt3d.FS_TUNE_SHAPES)]
    assert len(set(shapes)) == rt3d.FS_TUNE_SHAPES
    for block, rpt, widen, bl in shapes:
        assert block in (64, 128, 256) and rpt in (1, 2, 4) and widen in (0, 1, 2) and bl in (0, 1)
    with pytest.raises(rt3d.RT3DError):
        rt3d.fs_tune_shape(rt3d.FS_TUNE_SHAPES)
