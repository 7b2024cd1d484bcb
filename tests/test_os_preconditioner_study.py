"""What a better OS solver would buy the Krylov solve, on the oracle.

FGMRES (restart 100, right preconditioning, as the library's Krylov solve) on
(1 - Lambda(1-eps)) J = Lambda(eps B) + J_bc with the dense Lambda of a small
field box, preconditioned by the OS operator [1 - Lambda*(1-eps)]^-1 applied
three ways: 50 Jacobi sweeps to 1e-3 (the library's setting), 50 eight-colour
Gauss-Seidel sweeps to 1e-3, and the exact inverse of the band matrix.
Finding: the Jacobi setting already needs no more formal solutions (operator
products) than the exact inverse, so Gauss-Seidel can only save sweeps.
"""
import numpy as np
import pytest

import oracle
from paper_2102_01734_gb300 import inputs

N_BOX, NTH, NPH = 9, 4, 8


@pytest.fixture(scope="module")
def system():
    chi, _, B, bc = inputs.cartesian_config(N_BOX, 1e-2, seed=1)
    M = oracle.lambda_matrix(chi, NTH, NPH, True)
    _, L = oracle.fs_cart(chi, np.ones(chi.shape), NTH, NPH, True, lstar=True)
    Jbc = oracle.fs_cart(chi, np.zeros(chi.shape), NTH, NPH, True, bc=bc).reshape(-1)
    return chi, B, M, L, Jbc


def _band_matrix(L, shape):
    nz, ny, nx = shape
    N = L.shape[0]
    A = np.zeros((N, N))
    for v in range(N):
        x, y, z = v % nx, (v // nx) % ny, v // (nx * ny)
        for c in range(27):
            dx, dy, dz = c % 3 - 1, (c // 3) % 3 - 1, c // 9 - 1
            if 0 <= z + dz < nz:
                A[v, (x + dx) % nx + nx * ((y + dy) % ny + ny * (z + dz))] += L[v, c]
    return A


def _fgmres(A, b, x0, P, tol=1e-8, m=100, max_products=2000):
    """Products with A until ||b - A x|| <= tol ||b|| (Givens-rotated
    least squares, Gram-Schmidt applied twice)."""
    x = x0.copy()
    products = 0
    nb = np.linalg.norm(b)
    while products < max_products:
        r = b - A @ x
        products += 1
        beta = np.linalg.norm(r)
        if beta <= tol * nb:
            return x, products
        V, Z = [r / beta], []
        H = np.zeros((m + 1, m))
        cs, sn, g = np.zeros(m), np.zeros(m), np.zeros(m + 1)
        g[0] = beta
        for j in range(m):
            z = P(V[j])
            Z.append(z)
            w = A @ z
            products += 1
            for _ in range(2):
                for i in range(j + 1):
                    h = w @ V[i]
                    H[i, j] += h
                    w = w - h * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            d = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / d, H[j + 1, j] / d
            H[j, j], H[j + 1, j] = d, 0.0
            g[j + 1], g[j] = -sn[j] * g[j], cs[j] * g[j]
            if abs(g[j + 1]) <= tol * nb or products >= max_products:
                break
            V.append(w / np.linalg.norm(w))
        k = len(Z)
        y = np.linalg.solve(np.triu(H[:k, :k]), g[:k])
        x = x + np.array(Z).T @ y
    return x, products


@pytest.mark.parametrize("eps0", [1e-2, 1e-6])
def test_jacobi_preconditioner_already_reaches_the_exact_os_count(system, eps0):
    chi, B, M, L, Jbc = system
    shape = chi.shape
    eps = np.full(shape, eps0)
    ef, Bf = eps.reshape(-1), B.reshape(-1)
    A = np.eye(chi.size) - M * (1 - ef)[None, :]
    b = M @ (ef * Bf) + Jbc
    Jx = np.linalg.solve(A, b)
    Os = np.eye(chi.size) - _band_matrix(L, shape) * (1 - ef)[None, :]
    Os_inv = np.linalg.inv(Os)
    sweeps = {"jacobi": 0, "gs8": 0}

    def jacobi(r):
        d, m = oracle.os_jacobi(L, eps, r.reshape(shape), 50, 1e-3)
        sweeps["jacobi"] += m
        return d.reshape(-1)

    def gs8(r):
        d, m = oracle.os_gauss_seidel(L, eps, r.reshape(shape), 50, 1e-3, True)
        sweeps["gs8"] += m
        return d.reshape(-1)

    counts = {}
    for name, P in (("jacobi", jacobi), ("gs8", gs8), ("exact", lambda r: Os_inv @ r),
                    ("none", lambda r: r)):
        x, k = _fgmres(A, b, Bf.copy(), P)
        assert np.max(np.abs(x - Jx) / np.abs(Jx)) < 1e-6, name
        counts[name] = k
    assert counts["none"] > 3 * counts["exact"]
    assert counts["jacobi"] <= counts["exact"] + 1
    assert counts["gs8"] <= counts["exact"] + 1
    assert sweeps["gs8"] < sweeps["jacobi"]
