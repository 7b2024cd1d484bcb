"""FP64 CPU oracle of the 3D long-characteristics formal solution and ALI.

TEST INFRASTRUCTURE. Only the tests, ``__graft_entry__.smoke()`` and the CPU
legs of ``bench.py`` may import this package. It shares no code with the CUDA
path (``paper_2102_01734_gb300``) and imports nothing from it.

The C library (``rt3d_oracle.c``) holds the arithmetic; this module only
marshals numpy arrays, plus two plain linear-algebra helpers used as pins:
the brute-force Lambda matrix built column by column from the formal solution
(Eq. frmsol, J = Lambda S) and the direct dense solve of the scattering
problem that the ALI iteration (Eqs. alisol, alo) converges to. The line
transfer functions (profile-averaged mean intensity, Sec. 2) compose the C
routines per wavelength in plain numpy.

Array convention: grids are numpy arrays of shape (nz, ny, nx), x fastest,
so the flat index is v = x + nx (y + ny z). Lambda* is returned as (N, 27)
with d = (dx+1) + 3 (dy+1) + 9 (dz+1).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        c_int, c_double, c_long = ctypes.c_int, ctypes.c_double, ctypes.c_long
        lib.orc_directions.argtypes = [c_int, c_int, _dp, _dp, _dp, _dp]
        lib.orc_trace_cart.argtypes = [c_int, c_int, c_int, _dp, c_int, c_int, c_int, _ip, _dp]
        lib.orc_trace_cart.restype = c_int
        lib.orc_kmax_cart.argtypes = [c_int, c_int, c_int, _dp]
        lib.orc_kmax_cart.restype = c_int
        lib.orc_e012.argtypes = [c_double, _dp, _dp, _dp]
        lib.orc_coef.argtypes = [c_int, c_double, c_double, _dp, _dp, _dp, _dp]
        lib.orc_parab_weight.argtypes = [c_double, c_double]
        lib.orc_parab_weight.restype = c_double
        lib.orc_ray_fs.argtypes = [c_int, _dp, _dp, c_double, c_int, _dp, _dp, _dp, _dp, _dp]
        lib.orc_fs_cart.argtypes = [c_int, c_int, c_int, c_int, c_int, c_int, _dp, _dp,
                                    c_double, _dp, c_double, _dp, _dp, _dp, _dp, c_int]
        lib.orc_fs_cart.restype = c_int
        lib.orc_fs_cart_angles.argtypes = [c_int, c_int, c_int, c_int, c_int, c_int, _dp, _dp,
                                           c_double, _dp, c_double, _dp, _dp, _dp, c_int, _ip,
                                           c_int]
        lib.orc_fs_cart_angles.restype = c_int
        lib.orc_fs_cart_voxel.argtypes = [c_int, c_int, c_int, c_int, c_int, c_int, _dp, _dp,
                                          c_double, _dp, c_double, _dp, _dp, c_long, c_int,
                                          c_int, _dp, _dp]
        lib.orc_fs_cart_voxel.restype = c_int
        lib.orc_os_jacobi.argtypes = [c_int, c_int, c_int, _dp, _dp, _dp, _dp, c_int, c_double]
        lib.orc_os_jacobi.restype = c_int
        lib.orc_os_gauss_seidel.argtypes = [c_int, c_int, c_int, _dp, _dp, _dp, _dp, c_int,
                                            c_double, c_int]
        lib.orc_os_gauss_seidel.restype = c_int
        lib.orc_os_bicgstab.argtypes = [c_int, c_int, c_int, _dp, _dp, _dp, _dp, c_int, c_double]
        lib.orc_os_bicgstab.restype = c_int
        lib.orc_ali_solve.argtypes = [c_int, c_int, c_int, c_int, c_int, c_int, _dp, _dp, _dp,
                                      c_double, _dp, c_double, _dp, _dp, _dp, c_double, c_int,
                                      c_int, c_double, c_int, _dp, _dp]
        lib.orc_diffusion_bc.argtypes = [c_int, c_int, c_int, _dp, _dp, _dp, _dp]
        lib.orc_ali_solve.restype = c_int
        lib.orc_sph_trace_voxel.argtypes = [c_int, c_int, c_int, c_double, c_double, _dp, c_int,
                                            c_int, _ip, _dp, _ip, _dp]
        lib.orc_sph_trace_voxel.restype = c_int
        lib.orc_sph_kcap.argtypes = [c_int, c_int, c_int]
        lib.orc_sph_kcap.restype = c_int
        lib.orc_sph_rays.argtypes = [c_int, c_int, c_int, c_double, c_double, c_int, c_int, c_int,
                                     _ip]
        lib.orc_sph_rays.restype = c_int
        lib.orc_fs_sph.argtypes = [c_int, c_int, c_int, c_double, c_double, c_int, c_int, c_int,
                                   _dp, _dp, _dp, c_double, c_double, _dp, _dp]
        lib.orc_fs_sph.restype = c_int
        lib.orc_fs_sph_bc.argtypes = [c_int, c_int, c_int, c_double, c_double, c_int, c_int,
                                      c_int, _dp, _dp, _dp, _dp, _dp, c_double, c_double, _dp, _dp]
        lib.orc_fs_sph_bc.restype = c_int
        lib.orc_diffusion_bc_sph.argtypes = [c_int, c_int, c_int, c_double, c_double, _dp, _dp,
                                             _dp, _dp]
        _lib = lib
    return _lib


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(_dp)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def default_threads() -> int:
    return max(1, min(os.cpu_count() or 1, 64))


def directions(ntheta: int, nphi: int):
    """Direction set: (mu, phi, dir (n,3), w), angle index o = i*nphi + j."""
    lib = _load()
    n = ntheta * nphi
    mu, phi, w = np.zeros(n), np.zeros(n), np.zeros(n)
    d = np.zeros((n, 3))
    lib.orc_directions(ntheta, nphi, _ptr(mu), _ptr(phi), _ptr(d), _ptr(w))
    return mu, phi, d, w


def trace_cart(shape, d, x0: int = 0, y0: int = 0):
    """Tracker: voxel indices and chords of the characteristic of direction d from
    the centre of inflow-face cell (x0, y0). shape = (nz, ny, nx)."""
    lib = _load()
    nz, ny, nx = shape
    d = _f64(d)
    kmax = lib.orc_kmax_cart(nx, ny, nz, _ptr(d))
    vox = np.zeros(kmax, dtype=np.int32)
    ln = np.zeros(kmax)
    K = lib.orc_trace_cart(nx, ny, nz, _ptr(d), x0, y0, kmax,
                           vox.ctypes.data_as(_ip), _ptr(ln))
    if K < 0:
        raise RuntimeError(f"trace failed ({K})")
    return vox[:K].copy(), ln[:K].copy()


def e012(u: float):
    lib = _load()
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    lib.orc_e012(float(u), ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))
    return a.value, b.value, c.value


def coef(parabolic: bool, u: float, w: float):
    """(E, alpha, beta, gamma) of one interval."""
    lib = _load()
    out = [ctypes.c_double() for _ in range(4)]
    lib.orc_coef(int(parabolic), float(u), float(w), *[ctypes.byref(o) for o in out])
    return tuple(o.value for o in out)


def parab_weight(u: float, w: float) -> float:
    """Weight f of the parabolic against the linear coefficients."""
    return _load().orc_parab_weight(float(u), float(w))


def ray_fs(chil, S, I0: float, parabolic: bool):
    """Formal solution along one characteristic: returns (I, E, alpha, beta, gamma)."""
    lib = _load()
    chil, S = _f64(chil), _f64(S)
    K = chil.size
    outs = [np.zeros(K) for _ in range(5)]
    lib.orc_ray_fs(K, _ptr(chil), _ptr(S), float(I0), int(parabolic), *[_ptr(o) for o in outs])
    return tuple(outs)


def _bc_args(shape, bc):
    """(I_top, top face, I_bottom, bottom face, bottom gradient face): the
    optional "I_bottom_grad" (ny, nx) gives upward characteristics
    I = I_bottom + mu I_bottom_grad (the diffusion inner boundary)."""
    nz, ny, nx = shape
    bc = bc or {}
    top = bc.get("I_top", 0.0)
    bot = bc.get("I_bottom", 0.0)
    grad = bc.get("I_bottom_grad")
    top_face = None if np.isscalar(top) else _f64(np.broadcast_to(top, (ny, nx)))
    bot_face = None if np.isscalar(bot) else _f64(np.broadcast_to(bot, (ny, nx)))
    grad_face = None if grad is None else _f64(np.broadcast_to(grad, (ny, nx)))
    return (float(top) if top_face is None else 0.0, top_face,
            float(bot) if bot_face is None else 0.0, bot_face, grad_face)


def diffusion_bc(chi, B):
    """Bottom-face (I_bottom, I_bottom_grad) of the LTE diffusion inner
    boundary: dB/dtau between the two innermost layers and B carried linearly
    to the bottom face, each (ny, nx)."""
    lib = _load()
    chi, B = _f64(chi), _f64(B)
    nz, ny, nx = chi.shape
    I_face, grad = np.zeros((ny, nx)), np.zeros((ny, nx))
    lib.orc_diffusion_bc(nx, ny, nz, _ptr(chi), _ptr(B), _ptr(I_face), _ptr(grad))
    return I_face, grad


def fs_cart(chi, S, ntheta: int, nphi: int, parabolic: bool = False, bc=None,
            lstar: bool = False, nthreads: int | None = None):
    """J = Lambda S on the periodic box (and Lambda* as (N,27))."""
    lib = _load()
    chi, S = _f64(chi), _f64(S)
    nz, ny, nx = chi.shape
    J = np.zeros(chi.shape)
    L = np.zeros((chi.size, 27)) if lstar else None
    t, tf, b, bf, bg = _bc_args(chi.shape, bc)
    err = lib.orc_fs_cart(nx, ny, nz, ntheta, nphi, int(parabolic), _ptr(chi), _ptr(S),
                          t, _ptr(tf), b, _ptr(bf), _ptr(bg), _ptr(J), _ptr(L),
                          nthreads or default_threads())
    if err:
        raise RuntimeError(f"oracle formal solution failed ({err})")
    return (J, L) if lstar else J


def fs_cart_angles(chi, S, ntheta: int, nphi: int, angles, parabolic: bool = False, bc=None,
                   nthreads: int | None = None):
    """Share of the listed solid angles in J (a bounded sample of a large solve)."""
    lib = _load()
    chi, S = _f64(chi), _f64(S)
    nz, ny, nx = chi.shape
    J = np.zeros(chi.shape)
    ang = np.ascontiguousarray(angles, dtype=np.int32)
    t, tf, b, bf, bg = _bc_args(chi.shape, bc)
    err = lib.orc_fs_cart_angles(nx, ny, nz, ntheta, nphi, int(parabolic), _ptr(chi), _ptr(S),
                                 t, _ptr(tf), b, _ptr(bf), _ptr(bg), _ptr(J),
                                 nthreads or default_threads(), ang.ctypes.data_as(_ip),
                                 int(ang.size))
    if err:
        raise RuntimeError(f"oracle formal solution failed ({err})")
    return J


def fs_cart_voxel(chi, S, ntheta: int, nphi: int, v: int, parabolic: bool = False, bc=None,
                  lstar: bool = False, angles=None):
    """J_v (and the Lambda* row of v) for one voxel, all or a range of angles."""
    lib = _load()
    chi, S = _f64(chi), _f64(S)
    nz, ny, nx = chi.shape
    Jv = ctypes.c_double()
    row = np.zeros(27) if lstar else None
    lo, hi = angles if angles is not None else (0, ntheta * nphi)
    t, tf, b, bf, bg = _bc_args(chi.shape, bc)
    err = lib.orc_fs_cart_voxel(nx, ny, nz, ntheta, nphi, int(parabolic), _ptr(chi), _ptr(S),
                                t, _ptr(tf), b, _ptr(bf), _ptr(bg), int(v), int(lo), int(hi),
                                ctypes.byref(Jv), _ptr(row))
    if err:
        raise RuntimeError(f"oracle voxel formal solution failed ({err})")
    return (Jv.value, row) if lstar else Jv.value


def os_jacobi(lstar, eps, r, max_sweeps: int = 50, tol: float = 1e-3):
    """Jacobi solve of [1 - L*(1-eps)] dJ = r. Returns (dJ, sweeps)."""
    lib = _load()
    eps, r = _f64(eps), _f64(r)
    nz, ny, nx = r.shape
    L = _f64(lstar)
    dJ = np.zeros(r.shape)
    m = lib.orc_os_jacobi(nx, ny, nz, _ptr(L), _ptr(eps), _ptr(r), _ptr(dJ), max_sweeps, tol)
    return dJ, m


def os_gauss_seidel(lstar, eps, r, max_sweeps: int = 50, tol: float = 1e-3,
                    colored: bool = False):
    """Gauss-Seidel solve of [1 - L*(1-eps)] dJ = r (index order, or eight
    parity colors). Returns (dJ, sweeps)."""
    lib = _load()
    eps, r = _f64(eps), _f64(r)
    nz, ny, nx = r.shape
    L = _f64(lstar)
    dJ = np.zeros(r.shape)
    m = lib.orc_os_gauss_seidel(nx, ny, nz, _ptr(L), _ptr(eps), _ptr(r), _ptr(dJ), max_sweeps,
                                tol, int(colored))
    return dJ, m


def os_bicgstab(lstar, eps, r, max_iter: int = 200, tol: float = 1e-10):
    """BiCGStab solve of [1 - L*(1-eps)] dJ = r from 0. Returns (dJ, iterations;
    negative on a breakdown)."""
    lib = _load()
    eps, r = _f64(eps), _f64(r)
    nz, ny, nx = r.shape
    L = _f64(lstar)
    dJ = np.zeros(r.shape)
    k = lib.orc_os_bicgstab(nx, ny, nz, _ptr(L), _ptr(eps), _ptr(r), _ptr(dJ), max_iter, tol)
    return dJ, k


def ali_solve(chi, eps, B, ntheta: int, nphi: int, parabolic: bool = False, bc=None, J0=None,
              tol: float = 1e-13, max_iter: int = 500, max_sweeps: int = 50,
              sweep_tol: float = 1e-3, nthreads: int | None = None):
    """ALI iteration to rel dJ < tol. Returns (J, iterations, history, lstar)."""
    lib = _load()
    chi, eps, B = _f64(chi), _f64(eps), _f64(B)
    nz, ny, nx = chi.shape
    J = _f64(np.zeros(chi.shape) if J0 is None else J0).copy()
    L = np.zeros((chi.size, 27))
    hist = np.zeros(max_iter)
    t, tf, b, bf, bg = _bc_args(chi.shape, bc)
    it = lib.orc_ali_solve(nx, ny, nz, ntheta, nphi, int(parabolic), _ptr(chi), _ptr(eps),
                           _ptr(B), t, _ptr(tf), b, _ptr(bf), _ptr(bg), _ptr(J), tol, max_iter,
                           max_sweeps, sweep_tol, nthreads or default_threads(), _ptr(L),
                           _ptr(hist))
    if it <= -1000000:
        raise RuntimeError(f"oracle ALI failed ({it}): non-finite J or tracing error")
    return J, it, hist[:abs(it)], L


def lambda_matrix(chi, ntheta: int, nphi: int, parabolic: bool = False,
                  nthreads: int | None = None):
    """Brute-force Lambda: column u is J(e_u) with zero boundary intensity."""
    N = chi.size
    M = np.zeros((N, N))
    e = np.zeros(chi.shape)
    flat = e.reshape(-1)
    for u in range(N):
        flat[:] = 0.0
        flat[u] = 1.0
        M[:, u] = fs_cart(chi, e, ntheta, nphi, parabolic, bc=None,
                          nthreads=nthreads).reshape(-1)
    return M


def direct_solve(chi, eps, B, ntheta: int, nphi: int, parabolic: bool = False, bc=None):
    """Fixed point of the scattering problem, J = Lambda((1-eps)J + eps B) + J_bc,
    by a dense LU solve of (1 - Lambda (1-eps)) J = Lambda(eps B) + J_bc."""
    M = lambda_matrix(chi, ntheta, nphi, parabolic)
    eps_f, B_f = _f64(eps).reshape(-1), _f64(B).reshape(-1)
    Jbc = fs_cart(chi, np.zeros(chi.shape), ntheta, nphi, parabolic, bc=bc).reshape(-1)
    rhs = M @ (eps_f * B_f) + Jbc
    A = np.eye(chi.size) - M * (1.0 - eps_f)[None, :]
    return np.linalg.solve(A, rhs).reshape(chi.shape)


# ------------------------------------------------------------ spherical grid
def sph_trace(n, d, v, r_in=1.0, r_out=1.3):
    """Cells, chords, entry-through-core flag and entry point of the ray that
    voxel v launches in direction d on the (nr, nt, np) spherical grid."""
    lib = _load()
    nr, nt, np_ = n
    cap = lib.orc_sph_kcap(nr, nt, np_)
    vox = np.zeros(cap, dtype=np.int32)
    ln = np.zeros(cap)
    ec = ctypes.c_int()
    pin = np.zeros(3)
    d = _f64(d)
    K = lib.orc_sph_trace_voxel(nr, nt, np_, r_in, r_out, _ptr(d), int(v), cap,
                                vox.ctypes.data_as(_ip), _ptr(ln), ctypes.byref(ec), _ptr(pin))
    if K < 0:
        raise RuntimeError("spherical trace failed")
    return vox[:K].copy(), ln[:K].copy(), bool(ec.value), pin


def sph_rays(n, ntheta, nphi, o, r_in=1.0, r_out=1.3):
    """Launching voxels of the ray set of solid angle o."""
    lib = _load()
    nr, nt, np_ = n
    launch = np.zeros(nr * nt * np_, dtype=np.int32)
    k = lib.orc_sph_rays(nr, nt, np_, r_in, r_out, ntheta, nphi, int(o), launch.ctypes.data_as(_ip))
    if k < 0:
        raise RuntimeError("spherical ray set failed")
    return launch[:k].copy()


def fs_sph(chi, S, B, ntheta, nphi, parabolic=False, I_out=0.0, I_irr=0.0, lstar=False,
           r_in=1.0, r_out=1.3, core_face=None, core_grad=None):
    """Formal solution on the spherical grid; arrays shaped (np, nt, nr)
    (r fastest: v = ir + nr (it + nt ip)). Rays from the core start with B of
    their first cell, or, with core_face (np, nt), with core_face + mu
    core_grad (the diffusion condition; core_grad optional)."""
    lib = _load()
    chi, S, B = _f64(chi), _f64(S), _f64(B)
    np_, nt, nr = chi.shape
    J = np.zeros(chi.shape)
    L = np.zeros((chi.size, 27)) if lstar else None
    cf = None if core_face is None else _f64(core_face)
    cg = None if core_grad is None else _f64(core_grad)
    err = lib.orc_fs_sph_bc(nr, nt, np_, r_in, r_out, ntheta, nphi, int(parabolic), _ptr(chi),
                            _ptr(S), _ptr(B), _ptr(cf), _ptr(cg), float(I_out), float(I_irr),
                            _ptr(J), _ptr(L))
    if err:
        raise RuntimeError(f"spherical formal solution failed ({err})")
    return (J, L) if lstar else J


def diffusion_bc_sph(chi, B, r_in=1.0, r_out=1.3):
    """Core-face (I_face, grad) of the LTE diffusion inner boundary on the
    spherical grid, each (np, nt): dB/dtau between the two innermost shells
    and B carried linearly to the core sphere."""
    lib = _load()
    chi, B = _f64(chi), _f64(B)
    np_, nt, nr = chi.shape
    I_face, grad = np.zeros((np_, nt)), np.zeros((np_, nt))
    lib.orc_diffusion_bc_sph(nr, nt, np_, r_in, r_out, _ptr(chi), _ptr(B), _ptr(I_face),
                             _ptr(grad))
    return I_face, grad


# ------------------------------------------------------------ line transfer
# Sec. 2 (with Eq. alisol): for a spectral line the source function is shared
# by the wavelengths l of the line, S = (1 - eps) Jbar + eps B, and couples to
# the radiation field through the profile-averaged mean intensity
# Jbar = int J_l phi_l dl, here the quadrature sum Jbar = sum_l wphi[l] J_l
# (wphi: quadrature weight times profile, summing to 1). Wavelength l sees the
# opacity scale[l] * chi. The OS step of Eq. alo then uses the profile-averaged
# band Lbar* = sum_l wphi[l] Lambda*_l.

def line_lambda_star(chi, scale, wphi, ntheta: int, nphi: int, parabolic: bool = False):
    """Lbar* = sum_l wphi[l] Lambda*_l as (N, 27)."""
    chi = _f64(chi)
    L = np.zeros((chi.size, 27))
    for s_l, w_l in zip(scale, wphi):
        _, Ll = fs_cart(chi * float(s_l), np.ones(chi.shape), ntheta, nphi, parabolic,
                        lstar=True)
        L += float(w_l) * Ll
    return L


def line_fs(chi, scale, wphi, S, ntheta: int, nphi: int, parabolic: bool = False, bc=None):
    """Jbar = sum_l wphi[l] Lambda_l S (+ the boundary terms of each wavelength)."""
    chi = _f64(chi)
    J = np.zeros(chi.shape)
    for s_l, w_l in zip(scale, wphi):
        J += float(w_l) * fs_cart(chi * float(s_l), S, ntheta, nphi, parabolic, bc)
    return J


def line_ali_step(chi, scale, wphi, eps, B, J, ntheta: int, nphi: int,
                  parabolic: bool = False, bc=None, lbar=None, max_sweeps: int = 50,
                  sweep_tol: float = 1e-3):
    """One ALI iteration of the line problem: S from Jbar, Jbar_FS, the Jacobi
    OS solve of [1 - Lbar*(1-eps)] dJ = Jbar_FS - Jbar, Jbar += dJ. Returns
    (Jbar_new, rel, Lbar*) with rel = max |dJ| / |Jbar_new| over dJ != 0."""
    eps, B, J = _f64(eps), _f64(B), _f64(J)
    if lbar is None:
        lbar = line_lambda_star(chi, scale, wphi, ntheta, nphi, parabolic)
    S = (1.0 - eps) * J + eps * B
    Jfs = line_fs(chi, scale, wphi, S, ntheta, nphi, parabolic, bc)
    dJ, _ = os_jacobi(lbar, eps, Jfs - J, max_sweeps, sweep_tol)
    Jn = J + dJ
    nz = dJ != 0.0
    rel = float(np.max(np.abs(dJ[nz]) / np.abs(Jn[nz]))) if nz.any() else 0.0
    return Jn, rel, lbar


def line_ali_solve(chi, scale, wphi, eps, B, ntheta: int, nphi: int, parabolic: bool = False,
                   bc=None, J0=None, tol: float = 1e-13, max_iter: int = 500):
    """Line ALI to rel < tol from J0 (default 0). Returns (Jbar, iterations;
    negative if not converged)."""
    J = np.zeros(np.shape(chi)) if J0 is None else _f64(J0).copy()
    lbar = line_lambda_star(chi, scale, wphi, ntheta, nphi, parabolic)
    for it in range(1, max_iter + 1):
        J, rel, _ = line_ali_step(chi, scale, wphi, eps, B, J, ntheta, nphi, parabolic, bc,
                                  lbar)
        if not np.isfinite(rel):
            raise RuntimeError("oracle line ALI: non-finite Jbar")
        if rel < tol:
            return J, it
    return J, -max_iter


def line_direct_solve(chi, scale, wphi, eps, B, ntheta: int, nphi: int,
                      parabolic: bool = False, bc=None):
    """Fixed point of the line problem by a dense solve of
    (1 - Lbar (1-eps)) Jbar = Lbar(eps B) + Jbar_bc, Lbar = sum_l wphi[l] Lambda_l
    built column by column."""
    chi = _f64(chi)
    eps_f, B_f = _f64(eps).reshape(-1), _f64(B).reshape(-1)
    M = np.zeros((chi.size, chi.size))
    for s_l, w_l in zip(scale, wphi):
        M += float(w_l) * lambda_matrix(chi * float(s_l), ntheta, nphi, parabolic)
    Jbc = line_fs(chi, scale, wphi, np.zeros(chi.shape), ntheta, nphi, parabolic, bc)
    rhs = M @ (eps_f * B_f) + Jbc.reshape(-1)
    A = np.eye(chi.size) - M * (1.0 - eps_f)[None, :]
    return np.linalg.solve(A, rhs).reshape(chi.shape)
