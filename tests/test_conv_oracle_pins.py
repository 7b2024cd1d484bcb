"""Pins of the FP64 CPU oracle of the learned warm start's layers:
brute-force sums on tiny grids, finite-difference gradients, adjoint
identities of pooling and upsampling."""
import numpy as np

from oracle import conv


def _brute_conv(X, W, b):
    C, nz, ny, nx = X.shape
    Co = W.shape[0]
    Y = np.zeros((Co, nz, ny, nx))
    for o in range(Co):
        for z in range(nz):
            for y in range(ny):
                for x in range(nx):
                    s = b[o]
                    for i in range(C):
                        for dz in (-1, 0, 1):
                            zz = z + dz
                            if not 0 <= zz < nz:
                                continue
                            for dy in (-1, 0, 1):
                                for dx in (-1, 0, 1):
                                    s += W[o, i, dz + 1, dy + 1, dx + 1] * \
                                        X[i, zz, (y + dy) % ny, (x + dx) % nx]
                    Y[o, z, y, x] = s
    return Y


def test_conv_matches_brute_force():
    rng = np.random.default_rng(0)
    X = rng.standard_normal((3, 4, 5, 3))
    W = rng.standard_normal((2, 3, 3, 3, 3))
    b = rng.standard_normal(2)
    assert np.max(np.abs(conv.conv3d(X, W, b) - _brute_conv(X, W, b))) < 1e-12


def test_conv_gradients_by_finite_differences():
    rng = np.random.default_rng(1)
    X = rng.standard_normal((2, 4, 3, 5))
    W = rng.standard_normal((3, 2, 3, 3, 3))
    b = rng.standard_normal(3)
    dY = rng.standard_normal((3, 4, 3, 5))
    dX, dW, db = conv.conv3d_backward(X, W, dY)
    f = lambda X_, W_, b_: float(np.sum(conv.conv3d(X_, W_, b_) * dY))
    h = 1e-6
    for idx in [(0, 0, 0, 0), (1, 3, 2, 4), (0, 2, 1, 0)]:
        E = np.zeros_like(X)
        E[idx] = h
        num = (f(X + E, W, b) - f(X - E, W, b)) / (2 * h)
        assert abs(num - dX[idx]) < 1e-7 * max(1, abs(num))
    for idx in [(0, 0, 0, 0, 0), (2, 1, 2, 1, 0), (1, 0, 1, 2, 2)]:
        E = np.zeros_like(W)
        E[idx] = h
        num = (f(X, W + E, b) - f(X, W - E, b)) / (2 * h)
        assert abs(num - dW[idx]) < 1e-7 * max(1, abs(num))
    assert np.allclose(db, dY.sum(axis=(1, 2, 3)))


def test_pool_and_upsample_adjoints_and_constants():
    rng = np.random.default_rng(2)
    for shape in [(5, 6, 7), (4, 4, 4), (3, 5, 2)]:
        X = rng.standard_normal((2,) + shape)
        P = conv.pool(X)
        Q = rng.standard_normal(P.shape)
        assert abs(np.sum(P * Q) - np.sum(X * conv.pool_backward(Q, shape))) < 1e-12
        U = rng.standard_normal(X.shape)
        small = P.shape[1:]
        up = conv.upsample(Q, shape)
        assert abs(np.sum(up * U) - np.sum(Q * conv.upsample_backward(U, small))) < 1e-12
        # constant fields: pooling keeps them away from a ragged top layer
        c = conv.pool(np.ones((1,) + shape))
        assert np.allclose(c[0, : shape[0] // 2], 1.0)
