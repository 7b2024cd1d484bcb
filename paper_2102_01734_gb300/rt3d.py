"""Python binding of the C ABI in include/rt3d.h (argument marshalling only).

Every step of the formal solution, Lambda* construction, OS solve and ALI
iteration runs in the CUDA library librt3d.so; this module converts torch
tensors or numpy arrays to pointers and back. There is no CPU fallback: if
the library is missing or cannot be loaded, every call raises.

Arrays are float64, C-contiguous, shape (nz, ny, nx) (x fastest) or flat
(N,). Device tensors are passed through; host arrays are staged by the
library. Lambda* is (27, N) offset-major: [d][v] = dJ_v/dS_{v+d},
d = (dx+1) + 3(dy+1) + 9(dz+1).
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

try:  # torch is the device-memory and stream provider when present
    import torch
except ImportError:  # pragma: no cover
    torch = None

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "librt3d.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "rt3d.h")
HEADERS = [HEADER, os.path.join(os.path.dirname(HERE), "include", "rt3d_nn.h")]

OK, EINVAL, ENOMEM, ECUDA, ENOTCONVERGED, ETIMEOUT, ENUMERIC = range(7)
CARTESIAN_PERIODIC_XY = 0
SPHERICAL = 1
LINEAR, PARABOLIC = 0, 1
FP64, FP32_FS_FP64_ALI, FP32_FS_FF_REFINE = 0, 1, 2
ACCEL_NONE, ACCEL_KRYLOV = 0, 1
OS_JACOBI, OS_GAUSS_SEIDEL, OS_BICGSTAB = 0, 1, 2
CACHE_DEVICE, CACHE_HOST_STREAMED, CACHE_HOST_MAPPED, CACHE_HOST_CHORDS = 0, 1, 2, 3

_c_int, _c_double, _vp = ctypes.c_int, ctypes.c_double, ctypes.c_void_p


class GridDesc(ctypes.Structure):
    _fields_ = [("geometry", _c_int), ("n", _c_int * 3), ("ntheta", _c_int), ("nphi", _c_int),
                ("interp", _c_int), ("precision", _c_int), ("nlambda", _c_int),
                ("cuda_stream", _vp), ("accel", _c_int), ("r_in", _c_double),
                ("r_out", _c_double), ("cache", _c_int), ("stream_bytes", ctypes.c_longlong)]


class BC(ctypes.Structure):
    _fields_ = [("I_top", _c_double), ("I_bottom", _c_double), ("I_top_face", _vp),
                ("I_bottom_face", _vp), ("I_irr", _c_double), ("I_bottom_grad", _vp)]


class SolveStats(ctypes.Structure):
    _fields_ = [("iterations", _c_int), ("fs_fp32", _c_int), ("fs_fp64", _c_int),
                ("jacobi_sweeps", _c_int), ("rel_change", _c_double),
                ("residual64", _c_double), ("est_error", _c_double), ("seconds", _c_double),
                ("fs32_ms", _c_double), ("fs64_ms", _c_double), ("launches", ctypes.c_longlong),
                ("fs_ff", _c_int), ("fsff_ms", _c_double), ("rounds", _c_int), ("round_fp64", _c_int * 16), ("round_fs", _c_int * 16),
                ("round_res", _c_double * 16), ("round_est", _c_double * 16),
                ("fs_lstar", _c_int), ("fs32_lstar_ms", _c_double)]

    def as_dict(self):
        out = {k: getattr(self, k) for k, _ in self._fields_}
        k = min(self.rounds, 16)
        for name in ("round_fp64", "round_fs", "round_res", "round_est"):
            out[name] = list(getattr(self, name))[:k]
        return out


class LineStats(ctypes.Structure):
    _fields_ = [("iterations", _c_int), ("fs_lambda", _c_int), ("jacobi_sweeps", _c_int),
                ("rel_change", _c_double), ("est_error", _c_double), ("seconds", _c_double),
                ("fs64_ms", _c_double), ("launches", ctypes.c_longlong),
                ("fs_lambda32", _c_int), ("fs32_ms", _c_double), ("residual64", _c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class FsShape(ctypes.Structure):
    _fields_ = [("block", _c_int), ("rays_per_thread", _c_int), ("widen", _c_int),
                ("branchless", _c_int)]

    def as_tuple(self):
        return (self.block, self.rays_per_thread, self.widen, self.branchless)


FS_TUNE_SHAPES = 8


class BatchStats(ctypes.Structure):
    _fields_ = [("nlambda", _c_int), ("converged", _c_int), ("iterations", _c_int),
                ("graph_replays", _c_int), ("fs_lambda32", ctypes.c_longlong),
                ("fs_lambda64", ctypes.c_longlong), ("max_est_error", _c_double),
                ("max_residual64", _c_double), ("batch_ms", _c_double), ("fs32_ms", _c_double),
                ("fs64_ms", _c_double), ("seconds", _c_double), ("launches", ctypes.c_longlong),
                ("fs_lambda_ff", ctypes.c_longlong), ("fsff_ms", _c_double),
                ("fs_shape", FsShape), ("fs_tune_ms", ctypes.c_float * FS_TUNE_SHAPES),
                ("recaptures", _c_int), ("fs_batched", ctypes.c_longlong)]

    def as_dict(self):
        out = {k: getattr(self, k) for k, _ in self._fields_}
        out["fs_shape"] = self.fs_shape.as_tuple()
        out["fs_tune_ms"] = list(self.fs_tune_ms)
        return out




class GridInfo(ctypes.Structure):
    _fields_ = [("nangles", _c_int), ("kmax", _c_int), ("segments", ctypes.c_longlong),
                ("device_bytes", ctypes.c_longlong), ("fs_shape", FsShape),
                ("fs_tune_ms", ctypes.c_float * FS_TUNE_SHAPES), ("sm_count", _c_int),
                ("cache", _c_int), ("host_bytes", ctypes.c_longlong), ("cache_chunks", _c_int)]


class RT3DError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"rt3d status {status}: {msg}")
        self.status = status


_lib = None


def load(path: str | None = None):
    """Load librt3d.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"librt3d.so not built ({path}); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER
    lib.rt3d_grid_create.argtypes = [P(GridDesc), P(_vp)]
    lib.rt3d_grid_destroy.argtypes = [_vp]
    lib.rt3d_grid_destroy.restype = None
    lib.rt3d_grid_invalidate_lstar.argtypes = [_vp]
    lib.rt3d_grid_set_os_solver.argtypes = [_vp, _c_int]
    lib.rt3d_grid_get_info.argtypes = [_vp, P(GridInfo)]
    lib.rt3d_grid_set_fs_shape.argtypes = [_vp, ctypes.POINTER(FsShape)]
    lib.rt3d_fs_tune_shape.argtypes = [_c_int, ctypes.POINTER(FsShape)]
    lib.rt3d_grid_template.argtypes = [_vp, _c_int, P(_c_int), _vp, _vp]
    lib.rt3d_formal_solution.argtypes = [_vp, _vp, _vp, P(BC), _vp, _vp]
    lib.rt3d_os_solve.argtypes = [_vp, _vp, _vp, _vp, _vp, _c_int, _c_double, P(_c_int)]
    lib.rt3d_formal_solution_ff.argtypes = [_vp, _vp, _vp, P(BC), _vp]
    lib.rt3d_diffusion_bc.argtypes = [_vp, _c_int, _vp, _vp, _vp, _vp]
    lib.rt3d_ali_step.argtypes = [_vp, _vp, _vp, _vp, P(BC), _vp, P(_c_double)]
    lib.rt3d_solve.argtypes = [_vp, _vp, _vp, _vp, P(BC), _vp, _c_double, _c_int, P(SolveStats)]
    lib.rt3d_os_solve_noalloc.argtypes = [_c_int, _c_int, _c_int, _vp, _vp, _vp, _vp, _c_int,
                                          _c_double, P(_c_int), _vp]
    lib.rt3d_solve_batched.argtypes = [_vp, _c_int, _vp, _vp, _vp, P(BC), _vp, _c_double, _c_int,
                                       _vp, P(BatchStats)]
    lib.rt3d_line_solve.argtypes = [_vp, _c_int, _vp, _vp, _vp, _vp, _vp, P(BC), _vp,
                                    _c_double, _c_int, P(LineStats)]
    lib.rt3d_grid_sph_ray.argtypes = [_vp, _c_int, _c_int, P(_c_int), _vp, _vp, P(_c_int),
                                      P(_c_int)]
    lib.rt3d_last_error.restype = ctypes.c_char_p
    lib.rt3d_last_error.argtypes = []
    _lib = lib
    return lib


def header_functions(paths=None):
    """Names of the functions declared in include/rt3d.h and rt3d_nn.h."""
    names = set()
    for path in (paths or HEADERS):
        src = open(path).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(rt3d_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def last_error() -> str:
    return load().rt3d_last_error().decode()


def _check(status: int):
    if status != OK:
        raise RT3DError(status, last_error())


# ------------------------------------------------------------ marshalling
def _is_torch(x):
    return torch is not None and isinstance(x, torch.Tensor)


def _ptr(x):
    """Pointer of a float64 contiguous tensor/array (None -> NULL)."""
    if x is None:
        return None
    if _is_torch(x):
        if x.dtype != torch.float64 or not x.is_contiguous():
            raise ValueError("arrays must be contiguous float64")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if x.dtype != np.float64 or not x.flags.c_contiguous:
            raise ValueError("arrays must be contiguous float64")
        return x.ctypes.data
    raise TypeError(f"unsupported array type {type(x)}")


def _empty_like(x, shape):
    if _is_torch(x):
        return torch.empty(shape, dtype=torch.float64, device=x.device)
    return np.empty(shape, dtype=np.float64)


def _bc(bc, keep):
    """rt3d_bc from a dict {I_top: float|array, I_bottom: float|array,
    I_bottom_grad: array (optional), I_irr: float (optional)}."""
    if bc is None:
        return None
    s = BC()
    for key, fval, fptr in (("I_top", "I_top", "I_top_face"),
                            ("I_bottom", "I_bottom", "I_bottom_face")):
        val = bc.get(key, 0.0)
        if np.isscalar(val) or (_is_torch(val) and val.dim() == 0):
            setattr(s, fval, float(val))
            setattr(s, fptr, None)
        else:
            if isinstance(val, np.ndarray):
                val = np.ascontiguousarray(val, dtype=np.float64)
            elif _is_torch(val):
                val = val.to(torch.float64).contiguous()
            keep.append(val)
            setattr(s, fval, 0.0)
            setattr(s, fptr, _ptr(val))
    s.I_irr = float(bc.get("I_irr", 0.0))
    grad = bc.get("I_bottom_grad")
    if grad is not None:
        if isinstance(grad, np.ndarray):
            grad = np.ascontiguousarray(grad, dtype=np.float64)
        elif _is_torch(grad):
            grad = grad.to(torch.float64).contiguous()
        keep.append(grad)
        s.I_bottom_grad = _ptr(grad)
    return s


def _stream_handle(stream):
    if stream is not None:
        return int(stream)
    if torch is not None and torch.cuda.is_available():
        return torch.cuda.current_stream().cuda_stream
    return None


# ------------------------------------------------------------- the C ABI
def grid_create(n, ntheta: int, nphi: int, interp: int = LINEAR, precision: int = FP64,
                stream=None, geometry: int = CARTESIAN_PERIODIC_XY, accel: int = ACCEL_KRYLOV,
                r_in: float = 1.0, r_out: float = 1.3, cache: int = CACHE_DEVICE,
                stream_bytes: int = 0):
    lib = load()
    if np.isscalar(n):
        n = (int(n),) * 3
    d = GridDesc()
    d.geometry = geometry
    d.n[0], d.n[1], d.n[2] = (int(v) for v in n)
    d.ntheta, d.nphi = int(ntheta), int(nphi)
    d.interp, d.precision, d.nlambda = int(interp), int(precision), 1
    d.cuda_stream = _stream_handle(stream)
    d.accel = int(accel)
    d.r_in, d.r_out = float(r_in), float(r_out)
    d.cache, d.stream_bytes = int(cache), int(stream_bytes)
    h = _vp()
    _check(lib.rt3d_grid_create(ctypes.byref(d), ctypes.byref(h)))
    return h


def grid_destroy(h):
    load().rt3d_grid_destroy(h)


def grid_get_info(h) -> dict:
    info = GridInfo()
    _check(load().rt3d_grid_get_info(h, ctypes.byref(info)))
    out = {k: getattr(info, k) for k, _ in info._fields_}
    out["fs_tune_ms"] = list(info.fs_tune_ms)
    out["fs_shape"] = info.fs_shape.as_tuple()
    return out


def grid_set_os_solver(h, solver: int) -> None:
    """OS solver of the grid: OS_JACOBI, OS_GAUSS_SEIDEL or OS_BICGSTAB."""
    _check(load().rt3d_grid_set_os_solver(h, int(solver)))


def grid_invalidate_lstar(h) -> None:
    """Drops the grid's Lambda* band: the next solve or ALI step builds it."""
    _check(load().rt3d_grid_invalidate_lstar(h))


def fs_tune_shape(i: int) -> tuple:
    """Candidate i of the FP32 formal solution's autotuner:
    (block, rays_per_thread, widen, branchless)."""
    sh = FsShape()
    _check(load().rt3d_fs_tune_shape(i, ctypes.byref(sh)))
    return sh.as_tuple()


def grid_set_fs_shape(h, shape) -> None:
    """Fixes the FP32 formal solution's ray-bundle shape
    (block, rays_per_thread, widen, branchless); None re-tunes."""
    if shape is None:
        _check(load().rt3d_grid_set_fs_shape(h, None))
    else:
        sh = FsShape(*shape)
        _check(load().rt3d_grid_set_fs_shape(h, ctypes.byref(sh)))


def grid_template(h, angle: int):
    """(vox int32[K], len float64[K]) of the cached characteristic of `angle`."""
    lib = load()
    K = _c_int(0)
    lib.rt3d_grid_template(h, angle, ctypes.byref(K), None, None)  # query the size
    vox = np.zeros(K.value, dtype=np.int32)
    ln = np.zeros(K.value, dtype=np.float64)
    _check(lib.rt3d_grid_template(h, angle, ctypes.byref(K), vox.ctypes.data, ln.ctypes.data))
    return vox, ln


def grid_sph_ray(h, angle: int, index: int, cap: int = 4096):
    """(vox, len, launching voxel, boundary kind) of one cached spherical ray,
    or None past the last ray of the angle."""
    lib = load()
    K = _c_int(cap)
    vox = np.zeros(cap, dtype=np.int32)
    ln = np.zeros(cap)
    launch, kind = _c_int(), _c_int()
    st = lib.rt3d_grid_sph_ray(h, angle, index, ctypes.byref(K), vox.ctypes.data, ln.ctypes.data,
                               ctypes.byref(launch), ctypes.byref(kind))
    if st != OK:
        return None
    return vox[:K.value].copy(), ln[:K.value].copy(), launch.value, kind.value


def formal_solution(h, chi, S, bc=None, J_out=None, lstar_out=None):
    keep = []
    b = _bc(bc, keep)
    _check(load().rt3d_formal_solution(h, _ptr(chi), _ptr(S), ctypes.byref(b) if b else None,
                                       _ptr(J_out), _ptr(lstar_out)))
    return J_out


def formal_solution_ff(h, chi, S, bc=None, J_out=None):
    """Float-float formal solution (FP64-class accuracy on the FP32 pipe)."""
    keep = []
    b = _bc(bc, keep)
    _check(load().rt3d_formal_solution_ff(h, _ptr(chi), _ptr(S), ctypes.byref(b) if b else None,
                                          _ptr(J_out)))
    return J_out


def diffusion_bc(h, chi, B, spherical=False):
    """Bottom-face (I_bottom, I_bottom_grad) of the diffusion inner boundary
    from device tensors chi, B of shape (nz, ny, nx) or (n_lambda, nz, ny, nx);
    returns two device tensors of shape (ny, nx) or (n_lambda, ny, nx). On a
    spherical grid (arrays (nphi, ntheta, nr)) the core faces, (nphi, ntheta)."""
    nl = 1 if chi.dim() == 3 else int(chi.shape[0])
    if spherical:
        face_shape = tuple(chi.shape[:-1])
    else:
        face_shape = tuple(chi.shape[:-3]) + tuple(chi.shape[-2:])
    I_face = torch.empty(face_shape, dtype=torch.float64, device=chi.device)
    grad = torch.empty_like(I_face)
    _check(load().rt3d_diffusion_bc(h, nl, _ptr(chi), _ptr(B), _ptr(I_face), _ptr(grad)))
    return I_face, grad


def os_solve(h, lstar, eps, r, dJ_out, max_sweeps: int = 50, tol: float = 1e-3) -> int:
    m = _c_int(0)
    _check(load().rt3d_os_solve(h, _ptr(lstar), _ptr(eps), _ptr(r), _ptr(dJ_out), max_sweeps,
                                tol, ctypes.byref(m)))
    return m.value


NOALLOC_MAX_VOXELS = 65536


def os_solve_noalloc(n, lstar, eps, r, dJ_out, max_sweeps: int = 50, tol: float = 1e-3,
                     stream=None) -> int:
    """Allocation-free Jacobi OS solve (device arrays only, N <= 65536):
    for callers that cannot allocate device memory. Returns the sweeps."""
    nx, ny, nz = (int(v) for v in n)
    m = _c_int(0)
    _check(load().rt3d_os_solve_noalloc(nx, ny, nz, _ptr(lstar), _ptr(eps), _ptr(r),
                                        _ptr(dJ_out), max_sweeps, tol, ctypes.byref(m),
                                        _stream_handle(stream)))
    return m.value


def ali_step(h, chi, eps, B, bc, J_inout) -> float:
    keep = []
    b = _bc(bc, keep)
    rel = _c_double(0.0)
    _check(load().rt3d_ali_step(h, _ptr(chi), _ptr(eps), _ptr(B), ctypes.byref(b) if b else None,
                                _ptr(J_inout), ctypes.byref(rel)))
    return rel.value


def solve(h, chi, eps, B, bc, J_inout, tol: float = 1e-8, max_iter: int = 2000,
          raise_on_nonconv: bool = True) -> dict:
    keep = []
    b = _bc(bc, keep)
    st = SolveStats()
    status = load().rt3d_solve(h, _ptr(chi), _ptr(eps), _ptr(B), ctypes.byref(b) if b else None,
                               _ptr(J_inout), tol, max_iter, ctypes.byref(st))
    out = st.as_dict()
    out["status"] = status
    if status != OK and (raise_on_nonconv or status != ENOTCONVERGED):
        raise RT3DError(status, last_error())
    return out


def solve_batched(h, chi, eps, B, bc, J_inout, tol: float = 1e-8, max_iter: int = 4000,
                  raise_on_nonconv: bool = True) -> dict:
    """n_lambda problems on one grid: arrays are (n_lambda, nz, ny, nx); bc face
    arrays, when given, (n_lambda, ny, nx)."""
    keep = []
    b = _bc(bc, keep)
    nl = int(J_inout.shape[0])
    st = BatchStats()
    status = np.zeros(nl, dtype=np.int32)
    rc = load().rt3d_solve_batched(h, nl, _ptr(chi), _ptr(eps), _ptr(B),
                                   ctypes.byref(b) if b else None, _ptr(J_inout), tol, max_iter,
                                   status.ctypes.data, ctypes.byref(st))
    out = st.as_dict()
    out["status"] = rc
    out["per_lambda"] = status
    if rc != OK and (raise_on_nonconv or rc != ENOTCONVERGED):
        raise RT3DError(rc, last_error())
    return out


def line_solve(h, chi, scale, wphi, eps, B, bc, Jbar_inout, tol: float = 1e-8,
               max_iter: int = 2000, raise_on_nonconv: bool = True) -> dict:
    """Line transfer: Jbar of nl wavelengths with opacities scale[l] * chi and
    profile weights wphi[l] (host sequences of length nl)."""
    keep = []
    b = _bc(bc, keep)
    sc = np.ascontiguousarray(scale, dtype=np.float64).reshape(-1)
    wp = np.ascontiguousarray(wphi, dtype=np.float64).reshape(-1)
    if sc.size != wp.size:
        raise ValueError("scale and wphi differ in length")
    st = LineStats()
    status = load().rt3d_line_solve(h, int(sc.size), _ptr(chi), sc.ctypes.data, wp.ctypes.data,
                                    _ptr(eps), _ptr(B), ctypes.byref(b) if b else None,
                                    _ptr(Jbar_inout), tol, max_iter, ctypes.byref(st))
    out = st.as_dict()
    out["status"] = status
    if status != OK and (raise_on_nonconv or status != ENOTCONVERGED):
        raise RT3DError(status, last_error())
    return out


class Grid:
    """Owning wrapper of an rt3d_grid handle."""

    def __init__(self, n, ntheta, nphi, interp=LINEAR, precision=FP64, stream=None,
                 accel=ACCEL_KRYLOV, geometry=CARTESIAN_PERIODIC_XY, r_in=1.0, r_out=1.3,
                 cache=CACHE_DEVICE, stream_bytes=0):
        if np.isscalar(n):
            n = (int(n),) * 3
        self.n = tuple(int(v) for v in n)
        self.geometry = geometry
        self.shape = (self.n[2], self.n[1], self.n[0])
        self.N = self.n[0] * self.n[1] * self.n[2]
        self.handle = grid_create(n, ntheta, nphi, interp, precision, stream, geometry=geometry,
                                  accel=accel, r_in=r_in, r_out=r_out, cache=cache,
                                  stream_bytes=stream_bytes)

    def sph_ray(self, angle, index, cap=4096):
        return grid_sph_ray(self.handle, angle, index, cap)

    def close(self):
        if self.handle:
            grid_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        return grid_get_info(self.handle)

    def invalidate_lstar(self):
        grid_invalidate_lstar(self.handle)

    def set_os_solver(self, solver):
        grid_set_os_solver(self.handle, solver)

    def set_fs_shape(self, shape):
        grid_set_fs_shape(self.handle, shape)

    def template(self, angle):
        return grid_template(self.handle, angle)

    def formal_solution(self, chi, S, bc=None, lstar=False, J_out=None, lstar_out=None):
        J = J_out if J_out is not None else _empty_like(chi, self.shape)
        L = None
        if lstar:
            L = lstar_out if lstar_out is not None else _empty_like(chi, (27, self.N))
        formal_solution(self.handle, chi, S, bc, J, L)
        return (J, L) if lstar else J

    def formal_solution_ff(self, chi, S, bc=None, J_out=None):
        J = J_out if J_out is not None else _empty_like(chi, self.shape)
        formal_solution_ff(self.handle, chi, S, bc, J)
        return J

    def diffusion_bc(self, chi, B):
        return diffusion_bc(self.handle, chi, B, spherical=self.geometry == SPHERICAL)

    def os_solve(self, lstar, eps, r, max_sweeps=50, tol=1e-3):
        dJ = _empty_like(r, r.shape)
        m = os_solve(self.handle, lstar, eps, r, dJ, max_sweeps, tol)
        return dJ, m

    def ali_step(self, chi, eps, B, bc, J):
        return ali_step(self.handle, chi, eps, B, bc, J)

    def solve(self, chi, eps, B, bc, J, tol=1e-8, max_iter=2000, raise_on_nonconv=True):
        return solve(self.handle, chi, eps, B, bc, J, tol, max_iter, raise_on_nonconv)

    def solve_batched(self, chi, eps, B, bc, J, tol=1e-8, max_iter=4000, raise_on_nonconv=True):
        return solve_batched(self.handle, chi, eps, B, bc, J, tol, max_iter, raise_on_nonconv)

    def line_solve(self, chi, scale, wphi, eps, B, bc, J, tol=1e-8, max_iter=2000,
                   raise_on_nonconv=True):
        return line_solve(self.handle, chi, scale, wphi, eps, B, bc, J, tol, max_iter,
                          raise_on_nonconv)
