"""Pins of the FP64 network oracle (oracle/unet_oracle.py) to things other
than itself: a library correlation, brute-force loops, central finite
differences of every layer and of the whole network, and exact special cases."""
from __future__ import annotations

import numpy as np
import pytest
import scipy.signal

from oracle import unet_oracle as U
from paper_2209_01444_gb300 import surrogate, workloads


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def test_conv3x3_matches_scipy_correlation():
    r = _rng(1)
    B, H, W, Ci, Co = 2, 7, 9, 3, 4
    x = r.normal(size=(B, H, W, Ci))
    Wt = r.normal(size=(Co, 9 * Ci))
    b = r.normal(size=Co)
    y = U.conv3x3(x, Wt, b)
    K = Wt.reshape(Co, 3, 3, Ci)
    for bb in range(B):
        for co in range(Co):
            ref = b[co] + sum(scipy.signal.correlate2d(x[bb, :, :, ci], K[co, :, :, ci], mode="same",
                                                       boundary="fill") for ci in range(Ci))
            np.testing.assert_allclose(y[bb, :, :, co], ref, rtol=1e-12, atol=1e-12)


def _fd(f, a, idx, h=1e-6):
    old = a[idx]
    a[idx] = old + h
    fp = f()
    a[idx] = old - h
    fm = f()
    a[idx] = old
    return (fp - fm) / (2 * h)


def _check_fd(f, arr, grad, r, n=12, rtol=1e-6):
    flat = arr.reshape(-1)
    for k in r.choice(flat.size, size=min(n, flat.size), replace=False):
        idx = np.unravel_index(k, arr.shape)
        num = _fd(f, arr, idx)
        assert abs(num - grad[idx]) <= rtol * max(1.0, abs(num)) + 1e-8, (idx, num, grad[idx])


def test_conv3x3_backward_matches_finite_differences():
    r = _rng(2)
    x = r.normal(size=(2, 5, 6, 3))
    Wt = r.normal(size=(4, 27))
    b = r.normal(size=4)
    dy = r.normal(size=(2, 5, 6, 4))
    f = lambda: float((U.conv3x3(x, Wt, b) * dy).sum())
    dx, dW, db = U.conv3x3_bwd(x, Wt, dy)
    _check_fd(f, x, dx, r)
    _check_fd(f, Wt, dW, r)
    _check_fd(f, b, db, r)


def test_maxpool_matches_loops_and_first_maximum_rule():
    r = _rng(3)
    x = r.normal(size=(2, 6, 8, 3))
    x[0, 0, 0, 0] = x[0, 1, 1, 0] = 5.0  # a tie: the first in row-major order wins
    y, arg = U.maxpool(x)
    for b in range(2):
        for i in range(3):
            for j in range(4):
                for c in range(3):
                    win = [x[b, 2 * i + dy, 2 * j + dx, c] for dy in range(2) for dx in range(2)]
                    assert y[b, i, j, c] == max(win)
                    assert arg[b, i, j, c] == win.index(max(win))
    dy_ = r.normal(size=y.shape)
    g = U.maxpool_bwd(dy_, arg, x.shape)
    assert g[0, 0, 0, 0] == dy_[0, 0, 0, 0] and g[0, 1, 1, 0] == 0.0
    assert np.isclose(g.sum(), dy_.sum())


def test_maxpool_backward_matches_finite_differences():
    r = _rng(4)
    x = r.normal(size=(1, 6, 6, 2))
    dy = r.normal(size=(1, 3, 3, 2))
    f = lambda: float((U.maxpool(x)[0] * dy).sum())
    g = U.maxpool_bwd(dy, U.maxpool(x)[1], x.shape)
    _check_fd(f, x, g, r, n=30)


def test_upconv_matches_definition_and_finite_differences():
    r = _rng(5)
    B, H, W, Ci, Co = 2, 3, 4, 6, 3
    x = r.normal(size=(B, H, W, Ci))
    Wt = r.normal(size=(4 * Co, Ci))
    b = r.normal(size=4 * Co)
    y = U.upconv(x, Wt, b)
    assert y.shape == (B, 2 * H, 2 * W, Co)
    for bb in range(B):
        for i in range(2 * H):
            for j in range(2 * W):
                k = (i % 2) * 2 + (j % 2)
                for co in range(Co):
                    ref = b[k * Co + co] + sum(x[bb, i // 2, j // 2, ci] * Wt[k * Co + co, ci] for ci in range(Ci))
                    assert abs(y[bb, i, j, co] - ref) < 1e-12
    dy = r.normal(size=y.shape)
    f = lambda: float((U.upconv(x, Wt, b) * dy).sum())
    dx, dW, db = U.upconv_bwd(x, Wt, dy)
    _check_fd(f, x, dx, r)
    _check_fd(f, Wt, dW, r)
    _check_fd(f, b, db, r)


def test_mse_gradient():
    r = _rng(6)
    y, t = r.normal(size=(2, 3, 4, 5)), r.normal(size=(2, 3, 4, 5))
    loss, g = U.mse(y, t)
    assert np.isclose(loss, ((y - t) ** 2).mean())
    _check_fd(lambda: U.mse(y, t)[0], y, g, r)


@pytest.mark.parametrize("levels", [1, 2, 3])
def test_network_backward_matches_finite_differences(levels):
    r = _rng(10 + levels)
    base, F = 4, 5
    shapes = U.init_shapes(levels, base, 8, F)
    params = {n: r.normal(0.0, np.sqrt(2.0 / s[-1]) if len(s) == 2 else 0.1, s) for n, s in shapes}
    H = W = 2 ** levels * 2
    x = np.zeros((2, H, W, 8))
    x[..., :F] = r.normal(size=(2, H, W, F))
    t = r.normal(size=(2, H, W, F))

    def loss():
        return U.mse(U.forward(params, x, levels, F)[0], t)[0]

    y, cache = U.forward(params, x, levels, F)
    _, dy = U.mse(y, t)
    g = U.backward(params, cache, dy, levels)
    assert set(g) == set(params)
    for n, _ in shapes:
        _check_fd(loss, params[n], g[n], r, n=4, rtol=1e-5)


def test_network_is_identity_with_zero_projection():
    r = _rng(20)
    shapes = U.init_shapes(3, 8, 8, 5)
    params = {n: r.normal(size=s) for n, s in shapes}
    params["out.W"][:] = 0.0
    params["out.b"][:] = 0.0
    x = r.normal(size=(1, 8, 8, 8))
    y, _ = U.forward(params, x, 3, 5)
    np.testing.assert_array_equal(y, x[..., :5])


def test_parameter_order_agrees_with_binding():
    assert U.init_shapes(5, 32, 8, 5) == surrogate.param_shapes(5, 32, 5)
    n = sum(int(np.prod(s)) for _, s in surrogate.param_shapes())
    assert 7_000_000 < n < 9_000_000  # the 32 .. 512 five-level network


def test_bf16_exact_matches_torch_rounding():
    torch = pytest.importorskip("torch")
    r = _rng(7)
    a = np.concatenate([r.normal(size=1000) * 10.0 ** r.integers(-6, 6, 1000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.001953125, 1.005859375]])
    ref = torch.from_numpy(a.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(workloads.bf16_exact(a), ref)


def test_unet_params_seeded_and_bf16_exact():
    shapes = U.init_shapes(2, 8, 8, 5)
    p1 = workloads.unet_params(shapes, 3)
    p2 = workloads.unet_params(shapes, 3)
    for n, s in shapes:
        assert p1[n].shape == s
        np.testing.assert_array_equal(p1[n], p2[n])
        np.testing.assert_array_equal(workloads.bf16_exact(p1[n]), p1[n])


def test_bf16_round_matches_torch_and_quantised_network_is_close():
    torch = pytest.importorskip("torch")
    r = _rng(8)
    a = r.normal(size=2000) * 10.0 ** r.integers(-8, 8, 2000)
    ref = torch.from_numpy(a.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(U.bf16_round(a), ref)
    # with rounding points the network stays within a few BF16 ulps of FP64
    shapes = U.init_shapes(3, 8, 8, 5)
    params = {n: U.bf16_round(r.normal(0.0, np.sqrt(2.0 / s[-1]) if len(s) == 2 else 0.1, s)) for n, s in shapes}
    x = np.zeros((1, 16, 16, 8))
    x[..., :5] = U.bf16_round(r.normal(size=(1, 16, 16, 5)))
    y64, _ = U.forward(params, x, 3, 5)
    yq, _ = U.forward(params, x, 3, 5, q=U.bf16_round)
    d64, dq = y64 - x[..., :5], yq - x[..., :5]
    assert 0 < np.abs(dq - d64).max() <= 0.05 * np.abs(d64).max()


def test_interface_weighted_mse_against_its_definition_and_finite_differences():
    """The weighted loss mean(w d^2), w = 1 + alpha max(0, 1 - phi^2) per
    pixel (phi the input's first field), by brute force over pixels and
    channels, its gradient by central differences, and alpha = 0 (or phi
    outside [-1, 1]) giving the plain mean."""
    rng = np.random.default_rng(7)
    x = rng.uniform(-1, 1, size=(2, 3, 4, 5))
    y, t = rng.normal(size=x.shape), rng.normal(size=x.shape)
    alpha = 12.0
    loss, g = U.mse(y, t, x, alpha)
    acc = 0.0
    for idx in np.ndindex(x.shape):
        w = 1.0 + alpha * max(0.0, 1.0 - x[idx[:3] + (0,)] ** 2)
        acc += w * (y[idx] - t[idx]) ** 2
    assert loss == pytest.approx(acc / x.size, rel=1e-14)
    h = 1e-6
    for idx in [(0, 0, 0, 0), (1, 2, 3, 4), (0, 1, 2, 3)]:
        yp, ym = y.copy(), y.copy()
        yp[idx] += h
        ym[idx] -= h
        fd = (U.mse(yp, t, x, alpha)[0] - U.mse(ym, t, x, alpha)[0]) / (2 * h)
        assert g[idx] == pytest.approx(fd, rel=1e-6)
    assert U.mse(y, t, x, 0.0)[0] == pytest.approx(U.mse(y, t)[0], rel=1e-15)
    # outside [-1, 1] (a prediction's overshoot) the weight stays 1
    xo = x.copy()
    xo[..., 0] = 1.5
    assert U.mse(y, t, xo, alpha)[0] == pytest.approx(U.mse(y, t)[0], rel=1e-15)
