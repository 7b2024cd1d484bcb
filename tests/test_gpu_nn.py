"""The learned warm start's kernels against the FP64 CPU oracle (oracle/conv.py),
the whole network's gradients against the oracle composition, and what a
trained network gains over starting the solve from J = B."""
import numpy as np
import pytest

from oracle import conv as oc

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ws():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2102_01734_gb300 import build, rt3d, warmstart
    build.build()
    rt3d.load()
    return warmstart


def bf(x):
    """Round to BF16 and back (numpy FP64)."""
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(torch.bfloat16).to(
        torch.float64).numpy()


def to_dev_bf16(x_cl):
    return torch.from_numpy(np.ascontiguousarray(x_cl, dtype=np.float32)).to("cuda").to(torch.bfloat16)


def cl(X):
    """(C, nz, ny, nx) -> (V, C) channel-last."""
    C = X.shape[0]
    return X.reshape(C, -1).T


def cf(Y, shape):
    """(V, C) -> (C, nz, ny, nx)."""
    return Y.T.reshape((Y.shape[1],) + tuple(shape))


def w_oracle(W):
    """Wt[d][ci][co] -> oracle (co, ci, 3, 3, 3)."""
    return np.transpose(W.reshape(3, 3, 3, W.shape[1], W.shape[2]), (4, 3, 0, 1, 2))


def relmax(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-30))


@pytest.mark.parametrize("shape,ci,co", [((4, 5, 6), 16, 16), ((5, 7, 3), 32, 64),
                                         ((3, 4, 5), 48, 16), ((4, 4, 4), 16, 96)])
def test_conv_forward_and_gradients(ws, shape, ci, co):
    lib = ws._lib()
    rng = np.random.default_rng(ci + co)
    X = bf(rng.standard_normal((ci,) + shape))
    W = bf(rng.standard_normal((27, ci, co)) * 0.2)
    b = rng.standard_normal(co).astype(np.float32)
    dY = bf(rng.standard_normal((co,) + shape))
    nz, ny, nx = shape
    Xd = to_dev_bf16(cl(X))[None]
    Wd = to_dev_bf16(W)
    WTd = to_dev_bf16(np.transpose(W, (0, 2, 1)))
    bd = torch.from_numpy(b).to("cuda")
    Yf = torch.empty(1, nx * ny * nz, co, dtype=torch.float32, device="cuda")
    ws._ck(lib.rt3d_nn_conv3d(Xd.data_ptr(), Wd.data_ptr(), bd.data_ptr(), None, Yf.data_ptr(),
                              1, nx, ny, nz, ci, co, 0, 0, None))
    ref = oc.conv3d(X, w_oracle(W), b)
    assert relmax(cf(Yf[0].cpu().numpy(), shape), ref) < 1e-5
    # data gradient: the transposed convolution
    dYd = to_dev_bf16(cl(dY))[None]
    dXf = torch.empty(1, nx * ny * nz, ci, dtype=torch.float32, device="cuda")
    ws._ck(lib.rt3d_nn_conv3d(dYd.data_ptr(), WTd.data_ptr(), None, None, dXf.data_ptr(), 1, nx,
                              ny, nz, co, ci, 0, 1, None))
    dXo, dWo, dbo = oc.conv3d_backward(X, w_oracle(W), dY)
    assert relmax(cf(dXf[0].cpu().numpy(), shape), dXo) < 1e-5
    if (ci // 16) * (co // 16) <= 16:
        dW = torch.zeros(27, ci, co, dtype=torch.float32, device="cuda")
        db = torch.zeros(co, dtype=torch.float32, device="cuda")
        ws._ck(lib.rt3d_nn_conv3d_wgrad(Xd.data_ptr(), dYd.data_ptr(), dW.data_ptr(),
                                        db.data_ptr(), 1, nx, ny, nz, ci, co, None))
        assert relmax(w_oracle(dW.cpu().numpy().astype(np.float64)), dWo) < 1e-5
        assert relmax(db.cpu().numpy(), dbo) < 1e-5


def test_pool_upsample_against_oracle(ws):
    lib = ws._lib()
    rng = np.random.default_rng(5)
    shape = (5, 6, 7)
    nz, ny, nx = shape
    C = 16
    X = bf(rng.standard_normal((C,) + shape))
    Xd = to_dev_bf16(cl(X))[None]
    hs = ws.half(shape)
    P = torch.empty(1, int(np.prod(hs)), C, dtype=torch.bfloat16, device="cuda")
    ws._ck(lib.rt3d_nn_pool(Xd.data_ptr(), P.data_ptr(), 1, nx, ny, nz, C, None))
    Pr = oc.pool(X)
    assert relmax(cf(P[0].float().cpu().numpy(), hs), Pr) < 1e-2  # BF16 output
    dP = bf(rng.standard_normal((C,) + hs))
    dX = torch.zeros(1, nx * ny * nz, C, dtype=torch.float32, device="cuda")
    ws._ck(lib.rt3d_nn_pool_bwd(to_dev_bf16(cl(dP))[None].data_ptr(), dX.data_ptr(), 1, nx, ny,
                                nz, C, None))
    assert relmax(cf(dX[0].cpu().numpy(), shape), oc.pool_backward(dP, shape)) < 1e-6
    S = bf(rng.standard_normal((C,) + hs))
    U = torch.empty(1, nx * ny * nz, 2 * C, dtype=torch.bfloat16, device="cuda")
    ws._ck(lib.rt3d_nn_upsample(to_dev_bf16(cl(S))[None].data_ptr(), U.data_ptr(), 1, nx, ny, nz,
                                C, 2 * C, 0, None))
    assert relmax(cf(U[0, :, :C].float().cpu().numpy(), shape), oc.upsample(S, shape)) == 0.0
    dU = bf(rng.standard_normal((2 * C,) + shape))
    dS = torch.zeros(1, int(np.prod(hs)), C, dtype=torch.float32, device="cuda")
    ws._ck(lib.rt3d_nn_upsample_bwd(to_dev_bf16(cl(dU))[None].data_ptr(), dS.data_ptr(), 1, nx,
                                    ny, nz, C, 2 * C, 0, None))
    assert relmax(cf(dS[0].cpu().numpy(), hs), oc.upsample_backward(dU[:C], hs)) < 1e-6


def _oracle_unet(net, X, shape, target_corr):
    """FP64 forward/backward of the same U-Net with the oracle's layers (BF16
    weights), rounding to BF16 wherever the GPU path stores a tensor in BF16
    (every activation after bias and ReLU, pooled values, the loss gradient,
    every data gradient after a transposed convolution, the small-grid part
    of a concatenation's gradient and the skip sums), so that the remaining
    difference is the compounding of single rounding flips; returns
    (y, {name: dW})."""
    W = {n: w_oracle(net.Wt[n].float().cpu().numpy().astype(np.float64)) for n in net.Wt}
    b = {n: net.b32[n].cpu().numpy().astype(np.float64) for n in net.b32}
    relu = lambda t: np.maximum(t, 0.0)
    s1, s2 = shape, tuple((n + 1) // 2 for n in shape)
    a1 = bf(relu(oc.conv3d(X, W["e1a"], b["e1a"])))
    s1v = bf(relu(oc.conv3d(a1, W["e1b"], b["e1b"])))
    p1 = bf(oc.pool(s1v))
    a2 = bf(relu(oc.conv3d(p1, W["e2a"], b["e2a"])))
    s2v = bf(relu(oc.conv3d(a2, W["e2b"], b["e2b"])))
    p2 = bf(oc.pool(s2v))
    a3 = bf(relu(oc.conv3d(p2, W["b_a"], b["b_a"])))
    bb = bf(relu(oc.conv3d(a3, W["b_b"], b["b_b"])))
    c2 = np.concatenate([oc.upsample(bb, s2), s2v])
    a4 = bf(relu(oc.conv3d(c2, W["d2a"], b["d2a"])))
    u2 = bf(relu(oc.conv3d(a4, W["d2b"], b["d2b"])))
    c1 = np.concatenate([oc.upsample(u2, s1), s1v])
    a5 = bf(relu(oc.conv3d(c1, W["d1a"], b["d1a"])))
    u1 = bf(relu(oc.conv3d(a5, W["d1b"], b["d1b"])))
    y = oc.conv3d(u1, W["out"], b["out"])
    rows = int(np.prod(shape))
    g = np.zeros_like(y)
    g[0] = bf(2.0 * (y[0] - target_corr) / rows)
    gW = {}

    def back(name, Xin, Yout, dY, use_relu=True):
        if use_relu:
            dY = dY * (Yout > 0)
        dXn, dWn, _ = oc.conv3d_backward(Xin, W[name], dY)
        gW[name] = dWn
        return bf(dXn)

    d = back("out", u1, y, g, False)
    d = back("d1b", a5, u1, d)
    d = back("d1a", c1, a5, d)
    d_u2 = bf(oc.upsample_backward(d[:32], s2))
    d_s1 = d[32:]
    d = back("d2b", a4, u2, d_u2)
    d = back("d2a", c2, a4, d)
    d_b = bf(oc.upsample_backward(d[:64], tuple((n + 1) // 2 for n in s2)))
    d_s2 = d[64:]
    d = back("b_b", a3, bb, d_b)
    d = back("b_a", p2, a3, d)
    d_s2 = bf(d_s2 + oc.pool_backward(d, s2))
    d = back("e2b", a2, s2v, d_s2)
    d = back("e2a", p1, a2, d)
    d_s1 = bf(d_s1 + oc.pool_backward(d, s1))
    d = back("e1b", a1, s1v, d_s1)
    back("e1a", X, a1, d)
    return y, gW


# Where the network's layers meet. The GPU path stores activations and data
# gradients in BF16 between layers, so through the whole network its values
# drift from any FP64 composition by BF16 rounding (8-bit mantissa) that
# compounds from layer to layer: an element-wise comparison of the whole
# network is bounded by that budget only. Each layer is therefore checked
# element-wise on the tensors the GPU actually passed it: its forward output
# within one BF16 unit of the oracle layer on the GPU's input (plus the FP32
# accumulation's share; 1e-5 for the FP32 output layer), and its weight
# gradient within 1e-5 of the oracle's on the GPU's input and output gradient
# (FP32 sums of exact BF16 products). The whole network's gradients are
# compared with the FP64 oracle composition by direction and size, which a
# missing or transposed path fails.
FORWARD_PAIRS = [("e1a", "X", "a1"), ("e1b", "a1", "s1"), ("e2a", "p1", "a2"), ("e2b", "a2", "s2"),
                 ("b_a", "p2", "a3"), ("b_b", "a3", "b"), ("d2a", "c2", "a4"), ("d2b", "a4", "u2"),
                 ("d1a", "c1", "a5"), ("d1b", "a5", "u1"), ("out", "u1", "y")]


def test_network_layers_and_gradients_against_oracle(ws):
    net = ws.UNet(seed=3)
    shape = (6, 8, 10)
    rng = np.random.default_rng(7)
    X = np.zeros((16,) + shape)
    X[:4] = bf(rng.standard_normal((4,) + shape))
    corr = rng.standard_normal(shape) * 0.3
    Xd = to_dev_bf16(cl(X))[None]
    Yf = net.forward(Xd, shape)
    c, _ = net.cache
    J0 = torch.ones((1,) + shape, dtype=torch.float64, device="cuda")
    target = torch.from_numpy(np.exp(corr)[None]).to("cuda")
    sse, dY = net.loss_grad(Yf, target, J0)
    gW, gb = net.backward(dY)
    to64 = lambda t: t[0].float().cpu().numpy().astype(np.float64)
    for name, src, dst in FORWARD_PAIRS:
        W = w_oracle(net.Wt[name].float().cpu().numpy().astype(np.float64))
        b = net.b32[name].cpu().numpy().astype(np.float64)
        sh = net.wgrad_inputs[name][2]
        xin = cf(to64(c[src]), sh)
        ref = oc.conv3d(xin, W, b)
        got = cf(to64(c[dst]), sh)
        if name == "out":
            assert relmax(got, ref) < 1e-5, name
        else:
            # one BF16 unit (2^-7 of the value at the bottom of its binade),
            # plus the FP32 accumulation's error, at most a few 1e-7 of the
            # sum of the absolute products (which also bounds a value that
            # the two sums put on different sides of the ReLU's zero)
            absum = oc.conv3d(np.abs(xin), np.abs(W), np.abs(b))
            ref = np.maximum(ref, 0.0)
            assert np.all(np.abs(got - ref) <= 2.0 ** -7 * np.abs(ref) + 1e-5 * absum), name
        Xl, dYl, _ = net.wgrad_inputs[name]
        _, dWo, _ = oc.conv3d_backward(cf(to64(Xl), sh), W, cf(to64(dYl), sh))
        g = w_oracle(gW[name].cpu().numpy().astype(np.float64))
        assert relmax(g, dWo) < 1e-5, (name, relmax(g, dWo))
    # the whole network against the FP64 composition: direction and size
    y_o, gW_o = _oracle_unet(net, X, shape, corr)
    assert relmax(cf(Yf[0].cpu().numpy(), shape)[0], y_o[0]) < 3e-2
    for name, *_ in ws.LAYERS:
        g = w_oracle(gW[name].cpu().numpy().astype(np.float64)).reshape(-1)
        ref = gW_o[name].reshape(-1)
        cos = float(g @ ref / (np.linalg.norm(g) * np.linalg.norm(ref)))
        ratio = float(np.linalg.norm(g) / np.linalg.norm(ref))
        assert cos > 0.98 and abs(ratio - 1.0) < 0.15, (name, cos, ratio)


def test_training_reduces_the_starting_error(ws):
    """Train on solved 16^3 boxes; on three held-out boxes the network's
    prediction is closer to the converged J than J = B is, stays closer after
    the same number of ALI iterations (Eq. alo), and the converged, certified
    solve (FGMRES, the library's default iteration) started from it needs at
    least 15 % fewer formal solutions in total, reaching the same J."""
    from paper_2102_01734_gb300 import inputs, rt3d
    n, nth, nph = 16, 4, 8
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to("cuda")
    data = []
    g = rt3d.Grid(n, nth, nph, rt3d.PARABOLIC, rt3d.FP32_FS_FP64_ALI)
    for seed in range(100, 113):
        chi, eps, B, bc = inputs.cartesian_config(n, 1e-4, seed=seed)
        J = d(B).clone()
        g.solve(d(chi), d(eps), d(B), {"I_top": 0.0, "I_bottom": d(bc["I_bottom"])}, J,
                tol=1e-9, max_iter=3000)
        data.append((d(chi)[None], d(eps)[None], d(B)[None], J[None].clone(), bc))
    train, held = data[:10], data[10:]
    net = ws.UNet(seed=0)
    ws.train(net, train, 500, lr=2e-3, lr_final=2e-4)
    ga = rt3d.Grid(n, nth, nph, rt3d.PARABOLIC, rt3d.FP32_FS_FP64_ALI, accel=rt3d.ACCEL_NONE)
    gk = rt3d.Grid(n, nth, nph, rt3d.PARABOLIC, rt3d.FP32_FS_FP64_ALI, accel=rt3d.ACCEL_KRYLOV)
    fs_b = fs_n = 0
    lmax = lambda A, Jc: float(torch.max(torch.abs(torch.log(A / Jc))))
    for chi, eps, B, J, bc in held:
        pred = net.predict(chi, eps, B, B)
        err_net, err_b = lmax(pred, J), lmax(B, J)
        assert err_net < 0.5 * err_b, (err_net, err_b)
        bcd = {"I_top": 0.0, "I_bottom": d(bc["I_bottom"])}
        # equal work: five ALI iterations from each start
        Jb, Jn = B[0].clone(), pred[0].clone()
        for _ in range(5):
            ga.ali_step(chi[0], eps[0], B[0], bcd, Jb)
            ga.ali_step(chi[0], eps[0], B[0], bcd, Jn)
        e5_b, e5_n = lmax(Jb, J[0]), lmax(Jn, J[0])
        assert e5_n < 0.1 * e5_b, (e5_n, e5_b)
        # the certified solve from each start
        J1 = B[0].clone()
        st_b = gk.solve(chi[0], eps[0], B[0], bcd, J1, tol=1e-9, max_iter=20000)
        J2 = pred[0].clone()
        st_n = gk.solve(chi[0], eps[0], B[0], bcd, J2, tol=1e-9, max_iter=20000)
        assert torch.max(torch.abs(J2 / J1 - 1)) < 1e-8
        fs_b += st_b["fs_fp32"] + st_b["fs_fp64"]
        fs_n += st_n["fs_fp32"] + st_n["fs_fp64"]
        print("warm start: error after 5 ALI iterations", e5_b, e5_n, "formal solutions",
              st_b["fs_fp32"] + st_b["fs_fp64"], st_n["fs_fp32"] + st_n["fs_fp64"])
    assert fs_n <= 0.85 * fs_b, (fs_n, fs_b)
