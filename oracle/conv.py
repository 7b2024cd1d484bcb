"""FP64 CPU oracle of the learned warm start's layers (test infrastructure).

Plain numpy, written from the definitions; shares nothing with the CUDA
kernels. Grids are periodic in x and y and zero-padded in z, like the
radiative-transfer box. Activations are (C, nz, ny, nx); weights
(C_out, C_in, 3, 3, 3) indexed [dz+1, dy+1, dx+1].

  conv:      Y[o,z,y,x] = b[o] + sum_{i,dz,dy,dx} W[o,i,dz+1,dy+1,dx+1] X[i,z+dz,y+dy,x+dx]
  pool:      P[c,z,y,x] = mean of X[c, 2z..2z+1, 2y..2y+1, 2x..2x+1]
             (periodic in x, y; a layer beyond the top in z counts as zero)
  upsample:  U[c,z,y,x] = X[c, z//2, y//2, x//2] (cropped to the target size)
  relu:      max(x, 0)
"""
from __future__ import annotations

import numpy as np


def _shift(X, dz, dy, dx):
    """X[..., z+dz, y+dy, x+dx] with periodic x, y and zeros outside in z."""
    S = np.roll(X, shift=(-dy, -dx), axis=(-2, -1))
    out = np.zeros_like(S)
    nz = X.shape[-3]
    if dz == 0:
        out[...] = S
    elif dz > 0:
        out[..., : nz - dz, :, :] = S[..., dz:, :, :]
    else:
        out[..., -dz:, :, :] = S[..., : nz + dz, :, :]
    return out


def conv3d(X, W, b=None):
    X = np.asarray(X, dtype=np.float64)
    W = np.asarray(W, dtype=np.float64)
    Co = W.shape[0]
    Y = np.zeros((Co,) + X.shape[1:])
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                Xs = _shift(X, dz, dy, dx)
                Y += np.einsum("oi,izyx->ozyx", W[:, :, dz + 1, dy + 1, dx + 1], Xs)
    if b is not None:
        Y += np.asarray(b, dtype=np.float64)[:, None, None, None]
    return Y


def conv3d_backward(X, W, dY):
    """(dX, dW, db) of conv3d for the upstream gradient dY."""
    X = np.asarray(X, dtype=np.float64)
    W = np.asarray(W, dtype=np.float64)
    dY = np.asarray(dY, dtype=np.float64)
    dX = np.zeros_like(X)
    dW = np.zeros_like(W)
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                Xs = _shift(X, dz, dy, dx)
                dW[:, :, dz + 1, dy + 1, dx + 1] = np.einsum("ozyx,izyx->oi", dY, Xs)
                # X[v+d] received W[d] dY[v]: scatter back by the opposite shift
                G = np.einsum("oi,ozyx->izyx", W[:, :, dz + 1, dy + 1, dx + 1], dY)
                dX += _shift(G, -dz, -dy, -dx)
    db = dY.sum(axis=(1, 2, 3))
    return dX, dW, db


def _pool_shape(s):
    return tuple((n + 1) // 2 for n in s)


def pool(X):
    X = np.asarray(X, dtype=np.float64)
    C, nz, ny, nx = X.shape
    pz, py, px = _pool_shape((nz, ny, nx))
    P = np.zeros((C, pz, py, px))
    for z in range(pz):
        for y in range(py):
            for x in range(px):
                acc = np.zeros(C)
                for a in (0, 1):
                    zz = 2 * z + a
                    if zz >= nz:
                        continue
                    for b_ in (0, 1):
                        for c in (0, 1):
                            acc += X[:, zz, (2 * y + b_) % ny, (2 * x + c) % nx]
                P[:, z, y, x] = acc / 8.0
    return P


def pool_backward(dP, shape):
    C = dP.shape[0]
    nz, ny, nx = shape
    dX = np.zeros((C, nz, ny, nx))
    pz, py, px = dP.shape[1:]
    for z in range(pz):
        for y in range(py):
            for x in range(px):
                for a in (0, 1):
                    zz = 2 * z + a
                    if zz >= nz:
                        continue
                    for b_ in (0, 1):
                        for c in (0, 1):
                            dX[:, zz, (2 * y + b_) % ny, (2 * x + c) % nx] += dP[:, z, y, x] / 8.0
    return dX


def upsample(X, shape):
    nz, ny, nx = shape
    z = np.arange(nz) // 2
    y = np.arange(ny) // 2
    x = np.arange(nx) // 2
    return np.asarray(X, dtype=np.float64)[:, z][:, :, y][:, :, :, x]


def upsample_backward(dU, small_shape):
    C = dU.shape[0]
    out = np.zeros((C,) + tuple(small_shape))
    nz, ny, nx = dU.shape[1:]
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                out[:, z // 2, y // 2, x // 2] += dU[:, z, y, x]
    return out
