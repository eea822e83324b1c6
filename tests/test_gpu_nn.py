"""Surrogate-network kernels on the GPU against plain PyTorch FP32 references
of the same operation (same BF16 inputs)."""
from __future__ import annotations

import ctypes as ct

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    from paper_2209_01444_gb300 import build_ext, lbm as L

    build_ext.build()
    lib = L.load()
    torch.cuda.init()
    lib.lbm_nn_error(1)
    return torch, lib


def _p(t):
    return ct.c_void_p(t.data_ptr())


@pytest.mark.parametrize("M,N,K,lda", [(256, 128, 64, 64), (300, 64, 200, 200), (1024, 256, 1152, 1152),
                                       (128, 512, 576, 576), (512, 32, 45, 64), (2048, 128, 2304, 2304)])
@pytest.mark.parametrize("out_fp32", [1, 0])
def test_tcgen05_gemm_matches_fp32_matmul(env, M, N, K, lda, out_fp32):
    torch, lib = env
    g = torch.Generator(device="cuda").manual_seed(M * 7 + N + K)
    A = torch.zeros(M, lda, dtype=torch.bfloat16, device="cuda")
    A[:, :K] = torch.randn(M, K, generator=g, device="cuda").to(torch.bfloat16)
    B = torch.zeros(N, lda, dtype=torch.bfloat16, device="cuda")
    B[:, :K] = torch.randn(N, K, generator=g, device="cuda").to(torch.bfloat16)
    bias = torch.randn(N, generator=g, device="cuda")
    D = torch.empty(M, N, dtype=torch.float32 if out_fp32 else torch.bfloat16, device="cuda")
    for relu in (0, 1):
        rc = lib.lbm_nn_gemm(_p(A), lda, _p(B), lda, _p(D), N, _p(bias), M, N, K, out_fp32, relu,
                             ct.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == 0, lib.lbm_last_error(None)
        torch.cuda.synchronize()
        assert lib.lbm_nn_error(1) == 0
        ref = A[:, :K].float() @ B[:, :K].float().T + bias
        if relu:
            ref = torch.clamp(ref, min=0.0)
        scale = float(ref.abs().max())
        err = float((D.float() - ref).abs().max())
        tol = (2e-5 if out_fp32 else 8e-3) * scale
        assert err <= tol, (M, N, K, relu, err, scale)


def test_gemm_rejects_bad_shapes(env):
    torch, lib = env
    A = torch.zeros(128, 64, dtype=torch.bfloat16, device="cuda")
    D = torch.zeros(128, 48, dtype=torch.float32, device="cuda")
    assert lib.lbm_nn_gemm(_p(A), 64, _p(A), 64, _p(D), 48, None, 128, 44, 64, 1, 0, None) != 0  # N % 8
    assert lib.lbm_nn_gemm(_p(A), 60, _p(A), 64, _p(D), 64, None, 128, 64, 64, 1, 0, None) != 0  # lda % 8
    assert lib.lbm_nn_gemm(_p(A), 64, _p(A), 64, _p(D), 48, None, 128, 48, 72, 1, 0, None) != 0  # K > lda
    assert lib.lbm_nn_gemm_split(_p(A), 64, _p(A), 64, _p(D), 48, None, 128, 48, 1024, 1, 0, 4, None,
                                 None) != 0  # split without workspace


def _stream(torch):
    return ct.c_void_p(torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("splits", [1, 3])
def test_gemm_operand_wait_that_runs_out_is_reported_and_recovered(env, splits):
    """A bounded device wait that runs out, made to happen without a fault:
    with the operand-wait bound at 0 the tensor-core issuer gives up its
    first wait for operand tiles (the persistent warp-specialised GEMM,
    splits = 1, and the split-K GEMM).  The GEMM must raise the flag
    lbm_nn_error reports as LBM_ETIMEOUT, leave its output unwritten, drain
    the copies it issued and free its tensor memory; with the default bound
    back, the next GEMM on the same context runs and matches the FP32 matmul."""
    torch, lib = env
    M, N, K = 512, 128, 1024
    g = torch.Generator(device="cuda").manual_seed(5)
    A = torch.randn(M, K, generator=g, device="cuda").to(torch.bfloat16)
    B = torch.randn(N, K, generator=g, device="cuda").to(torch.bfloat16)
    ws = torch.empty(splits * M * N, dtype=torch.float32, device="cuda")
    D = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    args = (_p(A), K, _p(B), K, _p(D), N, None, M, N, K, 1, 0, splits, _p(ws), _stream(torch))
    torch.cuda.synchronize()
    assert lib.lbm_nn_error(1) == 0
    try:
        assert lib.lbm_nn_set_operand_wait(0) == 0
        assert lib.lbm_nn_gemm_split(*args) == 0
        torch.cuda.synchronize()
        assert lib.lbm_nn_error(0) == -5  # LBM_ETIMEOUT
        if splits == 1:
            assert bool(torch.isnan(D).all())  # the epilogue never ran
    finally:
        assert lib.lbm_nn_set_operand_wait(1000000000) == 0
    assert lib.lbm_nn_error(1) == -5  # reported once more, then cleared
    assert lib.lbm_nn_error(0) == 0
    assert lib.lbm_nn_gemm_split(*args) == 0
    torch.cuda.synchronize()
    assert lib.lbm_nn_error(1) == 0
    ref = A.float() @ B.float().T
    assert float((D - ref).abs().max()) <= 2e-5 * float(ref.abs().max())


@pytest.mark.parametrize("M,N,K,splits", [(32, 72, 4096, 16), (64, 288, 2048, 7), (512, 200, 1000, 3),
                                          (128, 264, 640, 1), (96, 8, 512, 2), (1024, 576, 16384, 64)])
def test_gemm_ragged_n_and_split_k(env, M, N, K, splits):
    """Ragged N (multiples of 8 between tile widths) and split-K slices with
    their FP32 reduction, against an FP32 matmul of the same BF16 inputs."""
    torch, lib = env
    g = torch.Generator(device="cuda").manual_seed(M + 3 * N + K)
    ld = (K + 7) // 8 * 8
    A = torch.zeros(M, ld, dtype=torch.bfloat16, device="cuda")
    B = torch.zeros(N, ld, dtype=torch.bfloat16, device="cuda")
    A[:, :K] = torch.randn(M, K, generator=g, device="cuda").to(torch.bfloat16)
    B[:, :K] = torch.randn(N, K, generator=g, device="cuda").to(torch.bfloat16)
    bias = torch.randn(N, generator=g, device="cuda")
    ws = torch.empty(splits * M * N, dtype=torch.float32, device="cuda")
    ref = A[:, :K].float() @ B[:, :K].float().T + bias
    for out_fp32 in (1, 0):
        ldd = N + 8  # pitched output
        D = torch.full((M, ldd), 7.0, dtype=torch.float32 if out_fp32 else torch.bfloat16, device="cuda")
        rc = lib.lbm_nn_gemm_split(_p(A), ld, _p(B), ld, _p(D), ldd, _p(bias), M, N, K, out_fp32, 0, splits,
                                   _p(ws), _stream(torch))
        assert rc == 0
        torch.cuda.synchronize()
        assert lib.lbm_nn_error(1) == 0
        err = float((D[:, :N].float() - ref).abs().max())
        tol = (2e-5 if out_fp32 else 8e-3) * float(ref.abs().max())
        assert err <= tol, (M, N, K, splits, out_fp32, err)
        assert bool((D[:, N:].float() == 7.0).all()), "wrote past N"


def _bf(torch, shape, g, scale=1.0):
    return (torch.randn(*shape, generator=g, device="cuda") * scale).to(torch.bfloat16)


def test_im2col_flip_transpose_exact(env):
    torch, lib = env
    g = torch.Generator(device="cuda").manual_seed(5)
    B, H, W, C, cp = 2, 5, 7, 16, 24
    X = _bf(torch, (B, H, W, cp), g)
    A = torch.empty(B * H * W, 9 * C, dtype=torch.bfloat16, device="cuda")
    assert lib.lbm_nn_im2col3x3(_p(X), B, H, W, C, cp, _p(A), _stream(torch)) == 0
    Xp = torch.nn.functional.pad(X[..., :C].float(), (0, 0, 1, 1, 1, 1))
    ref = torch.stack([Xp[:, ky:ky + H, kx:kx + W, :] for ky in range(3) for kx in range(3)], dim=3)
    assert torch.equal(A.float(), ref.reshape(B * H * W, 9 * C))
    # rotated kernel
    cout, cin = 24, 16
    Wt = _bf(torch, (cout, 9 * cin), g)
    Wf = torch.empty(cin, 9 * cout, dtype=torch.bfloat16, device="cuda")
    assert lib.lbm_nn_flip3x3(_p(Wt), cout, cin, _p(Wf), _stream(torch)) == 0
    ref = Wt.reshape(cout, 9, cin).flip(1).permute(2, 1, 0).reshape(cin, 9 * cout)
    assert torch.equal(Wf, ref)
    # transpose with pitches
    T = torch.empty(40, 80, dtype=torch.bfloat16, device="cuda")
    S = _bf(torch, (70, 48), g)
    assert lib.lbm_nn_transpose(_p(S), 70, 40, 48, _p(T), 80, _stream(torch)) == 0
    torch.cuda.synchronize()
    assert torch.equal(T[:, :70], S[:, :40].T)


def test_pool_and_shuffle_exact(env):
    torch, lib = env
    g = torch.Generator(device="cuda").manual_seed(6)
    # C = 16: the kernels moving 8 channels per 16-byte access; C = 12: the scalar ones
    for C, xp in ((16, 32), (12, 12)):
        _check_pool(torch, lib, g, 2, 6, 8, C, xp)
    _check_shuffle(torch, lib, g, 2)


def _check_pool(torch, lib, g, B, H, W, C, xp):
    X = _bf(torch, (B, H, W, xp), g)
    X[0, 0, 0, 0] = X[0, 1, 1, 0] = 9.0  # tie: the first maximum takes the gradient
    Y = torch.empty(B, H // 2, W // 2, C, dtype=torch.bfloat16, device="cuda")
    assert lib.lbm_nn_maxpool_fwd(_p(X), B, H, W, C, xp, _p(Y), _stream(torch)) == 0
    win = X[..., :C].float().reshape(B, H // 2, 2, W // 2, 2, C).permute(0, 1, 3, 2, 4, 5).reshape(B, H // 2, W // 2, 4, C)
    assert torch.equal(Y.float(), win.max(dim=3).values)
    dY = torch.randn(B, H // 2, W // 2, C, generator=g, device="cuda")
    dX = torch.randn(B, H, W, xp, generator=g, device="cuda")
    base = dX.clone()
    assert lib.lbm_nn_maxpool_bwd(_p(X), B, H, W, C, xp, _p(dY), _p(dX), xp, _stream(torch)) == 0
    torch.cuda.synchronize()
    w = win.cpu().numpy()
    arg = w.argmax(axis=3)  # first maximum
    add = np.zeros(w.shape, np.float32)
    np.put_along_axis(add, arg[:, :, :, None, :], dY.cpu().numpy()[:, :, :, None, :], axis=3)
    add = add.reshape(B, H // 2, W // 2, 2, 2, C).transpose(0, 1, 3, 2, 4, 5).reshape(B, H, W, C)
    ref = base.cpu().numpy()
    ref[..., :C] = ref[..., :C] + add
    assert np.array_equal(dX.cpu().numpy(), ref)


def _check_shuffle(torch, lib, g, B):
    # up-convolution shuffle into the second half of a concatenation buffer and back
    Hl, Wl, c = 3, 4, 8
    U = _bf(torch, (B * Hl * Wl, 4 * c), g)
    Ycat = torch.zeros(B, 2 * Hl, 2 * Wl, 2 * c, dtype=torch.bfloat16, device="cuda")
    assert lib.lbm_nn_shuffle_fwd(_p(U), B, Hl, Wl, c, _p(Ycat), 2 * c, c, _stream(torch)) == 0
    ref = U.reshape(B, Hl, Wl, 2, 2, c).permute(0, 1, 3, 2, 4, 5).reshape(B, 2 * Hl, 2 * Wl, c)
    assert torch.equal(Ycat[..., c:], ref) and bool((Ycat[..., :c] == 0).all())
    dU = torch.empty_like(U)
    dcat = torch.randn(B, 2 * Hl, 2 * Wl, 2 * c, generator=g, device="cuda")
    assert lib.lbm_nn_shuffle_bwd(_p(dcat), 1, 2 * c, c, B, Hl, Wl, c, _p(dU), _stream(torch)) == 0
    torch.cuda.synchronize()
    ref = dcat[..., c:].reshape(B, Hl, 2, Wl, 2, c).permute(0, 1, 3, 2, 4, 5).reshape(B * Hl * Wl, 4 * c)
    assert torch.equal(dU, ref.to(torch.bfloat16))


def test_reductions_projection_and_adam(env):
    torch, lib = env
    g = torch.Generator(device="cuda").manual_seed(7)
    s = _stream(torch)
    rows, C, pitch = 5000, 40, 48
    G = torch.randn(rows, pitch, generator=g, device="cuda")
    out = torch.empty(C, device="cuda")
    part = torch.empty(1 << 20, device="cuda")
    assert lib.lbm_nn_colsum(_p(G), 1, rows, C, pitch, _p(out), _p(part), 300, s) == 0
    torch.cuda.synchronize()
    ref = G[:, :C].double().sum(0)
    assert float((out.double() - ref).abs().max()) <= 1e-4 * float(G[:, :C].abs().sum(0).max())
    # projection with residual, and its backward (C = 32: the vector kernels;
    # C = 20: the scalar ones)
    for P, Cx, O in ((3000, 32, 5), (1001, 20, 3)):
        _check_projection(torch, lib, g, s, part, P, Cx, O)
    _check_mse_and_adam(torch, lib, g, s, part)


def _check_projection(torch, lib, g, s, part, P, Cx, O):
    X = _bf(torch, (P, Cx), g)
    Wt = torch.randn(O, Cx, generator=g, device="cuda")
    b = torch.randn(O, generator=g, device="cuda")
    R = torch.randn(P, O, generator=g, device="cuda")
    Y = torch.empty(P, O, device="cuda")
    assert lib.lbm_nn_proj_fwd(_p(X), P, Cx, Cx, _p(Wt), _p(b), O, _p(R), _p(Y), s) == 0
    torch.cuda.synchronize()
    ref = R.double() + b.double() + X.double() @ Wt.double().T
    assert float((Y.double() - ref).abs().max()) <= 1e-5 * float(ref.abs().max())
    dY = torch.randn(P, O, generator=g, device="cuda")
    dX = torch.empty(P, Cx, device="cuda")
    dW = torch.empty(O, Cx, device="cuda")
    db = torch.empty(O, device="cuda")
    assert lib.lbm_nn_proj_bwd(_p(dY), _p(X), P, Cx, Cx, _p(Wt), O, _p(dX), Cx, _p(dW), _p(db), _p(part), 64, s) == 0
    torch.cuda.synchronize()
    assert float((dX.double() - dY.double() @ Wt.double()).abs().max()) <= 1e-5 * 10
    refW = dY.double().T @ X.double()
    assert float((dW.double() - refW).abs().max()) <= 1e-5 * float(refW.abs().max()) * 10
    assert float((db.double() - dY.double().sum(0)).abs().max()) <= 1e-3


def _check_mse_and_adam(torch, lib, g, s, part):
    # mean squared error
    n = 100_003
    pr, tg = torch.randn(n, generator=g, device="cuda"), torch.randn(n, generator=g, device="cuda")
    grad, loss = torch.empty(n, device="cuda"), torch.empty(1, device="cuda")
    assert lib.lbm_nn_mse(_p(pr), _p(tg), n, _p(grad), _p(loss), _p(part), s) == 0
    torch.cuda.synchronize()
    d = pr.double() - tg.double()
    assert abs(float(loss) - float((d * d).sum())) <= 1e-4 * float((d * d).sum())
    assert float((grad.double() - 2 * d / n).abs().max()) <= 1e-6 * float((2 * d / n).abs().max()) + 1e-12
    # Adam, three steps, against the textbook update in FP64
    m_ = 10_000
    w = torch.randn(m_, generator=g, device="cuda")
    mom, vel = torch.zeros(m_, device="cuda"), torch.zeros(m_, device="cuda")
    wb = torch.empty(m_, dtype=torch.bfloat16, device="cuda")
    wr, mr, vr = w.double().clone(), torch.zeros(m_, dtype=torch.float64, device="cuda"), \
        torch.zeros(m_, dtype=torch.float64, device="cuda")
    for t in (1, 2, 3):
        gr = torch.randn(m_, generator=g, device="cuda")
        assert lib.lbm_nn_adam(_p(w), _p(gr), _p(mom), _p(vel), m_, ct.c_float(1e-2), ct.c_float(0.9),
                               ct.c_float(0.999), ct.c_float(1e-8), t, _p(wb), s) == 0
        gd = gr.double()
        mr = 0.9 * mr + 0.1 * gd
        vr = 0.999 * vr + 0.001 * gd * gd
        wr = wr - 1e-2 * (mr / (1 - 0.9 ** t)) / ((vr / (1 - 0.999 ** t)).sqrt() + 1e-8)
    torch.cuda.synchronize()
    assert float((w.double() - wr).abs().max()) <= 1e-5
    assert torch.equal(wb, w.to(torch.bfloat16))


def test_pack_unpack_cast(env):
    torch, lib = env
    g = torch.Generator(device="cuda").manual_seed(8)
    s = _stream(torch)
    P, F = 1000, 5
    f = torch.randn(P, F, generator=g, device="cuda") * 3 + 1
    mean = torch.tensor([0.5, -1.0, 2.0, 0.0, 0.25], device="cuda")
    std = torch.tensor([2.0, 0.5, 4.0, 1.0, 0.125], device="cuda")
    inv = 1.0 / std
    X = torch.full((P, 8), 3.0, dtype=torch.bfloat16, device="cuda")
    R = torch.empty(P, F, device="cuda")
    assert lib.lbm_nn_pack(_p(f), P, F, _p(mean), _p(inv), _p(X), 8, _p(R), s) == 0
    back = torch.empty(P, F, device="cuda")
    assert lib.lbm_nn_unpack(_p(R), P, F, _p(mean), _p(inv), _p(back), s) == 0
    torch.cuda.synchronize()
    assert torch.equal(R, (f - mean) * inv)
    assert torch.equal(X[:, :F], R.to(torch.bfloat16)) and bool((X[:, F:] == 0).all())
    assert float((back - f).abs().max()) <= 1e-5 * float(f.abs().max())
    A = torch.randn(300, 40, generator=g, device="cuda")
    Bt = torch.zeros(300, 48, dtype=torch.bfloat16, device="cuda")
    assert lib.lbm_nn_cast_bf16(_p(A), 300, 33, 40, _p(Bt), 48, s) == 0
    torch.cuda.synchronize()
    assert torch.equal(Bt[:, :33], A[:, :33].to(torch.bfloat16)) and bool((Bt[:, 33:] == 0).all())


@pytest.mark.parametrize("B,H,W,C,cp,N", [(2, 16, 16, 32, 32, 32), (1, 8, 256, 64, 128, 128), (3, 8, 8, 64, 64, 72),
                                          (1, 4, 4, 96, 96, 64), (2, 32, 32, 128, 128, 256), (1, 2, 2, 512, 512, 512),
                                          (4, 64, 64, 32, 64, 40),
                                          # row reuse (rows of >= 256 pixels, N <= 64): one or two sub-tiles,
                                          # four 32-channel sub-tiles, two 64-channel ones
                                          (1, 6, 256, 32, 40, 64), (2, 4, 512, 64, 64, 40),
                                          (1, 160, 512, 32, 32, 32), (1, 80, 512, 64, 72, 64), (2, 3, 256, 32, 32, 16)])
@pytest.mark.parametrize("out_fp32", [1, 0])
def test_implicit_conv3x3_matches_fp64_conv2d(env, B, H, W, C, cp, N, out_fp32):
    """The implicit convolution (4-D TMA tap shifts, zero padding from the
    out-of-bounds fill) against a CPU FP64 conv2d of the same BF16 values,
    over tiles of whole rows, several rows and several images, 64- and 32-
    channel K blocks, channel pitches wider than C and ragged N; on rows of
    256 pixels or more with N <= 64, the row-reuse form (one box of 130
    pixels per input row serving its three taps)."""
    torch, lib = env
    g = torch.Generator(device="cuda").manual_seed(B * 1000 + H * 10 + C + N)
    X = _bf(torch, (B, H, W, cp), g)
    Wm = _bf(torch, (N, 9 * C), g, scale=1.0 / (3.0 * C ** 0.5))
    bias = torch.randn(N, generator=g, device="cuda")
    D = torch.full((B * H * W, N + 8), 3.0, dtype=torch.float32 if out_fp32 else torch.bfloat16, device="cuda")
    for relu in (0, 1):
        rc = lib.lbm_nn_conv3x3(_p(X), B, H, W, C, cp, _p(Wm), 9 * C, _p(D), N + 8, _p(bias), N, out_fp32, relu,
                                _stream(torch))
        assert rc == 0
        torch.cuda.synchronize()
        assert lib.lbm_nn_error(1) == 0
        x = X[..., :C].double().cpu().permute(0, 3, 1, 2)
        w = Wm.double().cpu().reshape(N, 3, 3, C).permute(0, 3, 1, 2)
        ref = torch.nn.functional.conv2d(x, w, bias.double().cpu(), padding=1).permute(0, 2, 3, 1).reshape(-1, N)
        if relu:
            ref = ref.clamp(min=0.0)
        got = D[:, :N].double().cpu()
        err = float((got - ref).abs().max())
        tol = (2e-5 if out_fp32 else 8e-3) * float(ref.abs().max())
        assert err <= tol, (B, H, W, C, N, relu, err)
        assert bool((D[:, N:].float() == 3.0).all())


def test_implicit_conv3x3_rejects_unsupported_tiles(env):
    torch, lib = env
    X = torch.zeros(1, 48, 48, 32, dtype=torch.bfloat16, device="cuda")
    Wm = torch.zeros(32, 288, dtype=torch.bfloat16, device="cuda")
    D = torch.zeros(48 * 48, 32, device="cuda")
    assert lib.lbm_nn_conv3x3(_p(X), 1, 48, 48, 32, 32, _p(Wm), 288, _p(D), 32, None, 32, 1, 0, None) != 0  # W = 48
    assert lib.lbm_nn_conv3x3(_p(X), 1, 16, 16, 24, 32, _p(Wm), 288, _p(D), 32, None, 32, 1, 0, None) != 0  # C = 24


@pytest.mark.parametrize("B,Hl,Wl,cin,c", [(2, 4, 4, 64, 32), (1, 16, 32, 128, 64), (3, 2, 2, 512, 256)])
def test_upconv2x2_shuffle_epilogue(env, B, Hl, Wl, cin, c):
    torch, lib = env
    g = torch.Generator(device="cuda").manual_seed(B + Hl + cin)
    X = _bf(torch, (B * Hl * Wl, cin), g)
    Wm = _bf(torch, (4 * c, cin), g, scale=cin ** -0.5)
    bias = torch.randn(4 * c, generator=g, device="cuda")
    Y = torch.full((B, 2 * Hl, 2 * Wl, 2 * c), 5.0, dtype=torch.bfloat16, device="cuda")
    assert lib.lbm_nn_upconv2x2(_p(X), cin, _p(Wm), cin, _p(Y), 2 * c, c, _p(bias), B, Hl, Wl, cin, c,
                                _stream(torch)) == 0
    torch.cuda.synchronize()
    U = X.double().cpu() @ Wm.double().cpu().T + bias.double().cpu()
    ref = U.reshape(B, Hl, Wl, 2, 2, c).permute(0, 1, 3, 2, 4, 5).reshape(B, 2 * Hl, 2 * Wl, c)
    err = float((Y[..., c:].double().cpu() - ref).abs().max())
    assert err <= 8e-3 * float(ref.abs().max())
    assert bool((Y[..., :c] == 5.0).all())


@pytest.mark.parametrize("B,H,W,C,cp,taps", [(2, 4, 7, 16, 24, 9), (1, 16, 16, 8, 32, 9), (3, 8, 8, 72, 80, 9),
                                            (2, 6, 10, 40, 48, 1), (1, 1, 1000, 200, 200, 1),
                                            (2, 5, 32, 96, 104, 3), (1, 3, 8, 8, 8, 3), (1, 3, 16, 40, 48, 3)])
def test_gather_transposed_exact(env, B, H, W, C, cp, taps):
    torch, lib = env
    g = torch.Generator(device="cuda").manual_seed(B * H * W + C)
    X = _bf(torch, (B, H, W, cp), g)
    P = B * H * W
    pitch = P + 8
    AT = torch.full((taps * C, pitch), 9.0, dtype=torch.bfloat16, device="cuda")
    assert lib.lbm_nn_gather_t(_p(X), B, H, W, C, cp, taps, _p(AT), pitch, _stream(torch)) == 0
    torch.cuda.synchronize()
    if taps == 9:
        Xp = torch.nn.functional.pad(X[..., :C].float(), (0, 0, 1, 1, 1, 1))
        ref = torch.stack([Xp[:, ky:ky + H, kx:kx + W, :] for ky in range(3) for kx in range(3)], dim=3)
        ref = ref.reshape(P, 9 * C).T
    elif taps == 3:  # the middle row of the nine taps: dy = 0, dx = -1, 0, 1
        Xp = torch.nn.functional.pad(X[..., :C].float(), (0, 0, 1, 1))
        ref = torch.stack([Xp[:, :, kx:kx + W, :] for kx in range(3)], dim=3).reshape(P, 3 * C).T
    else:
        ref = X[..., :C].float().reshape(P, C).T
    assert torch.equal(AT[:, :P].float(), ref)
    assert bool((AT[:, P:] == 9.0).all())


def _wgrad_reference(X, dY):
    """dW[n][t*C + c] = sum over pixels of X shifted by tap t (zero padded) times
    dY, t = ky*3 + kx, in FP64 on the host."""
    B, H, W, C = X.shape
    Xp = np.pad(X.astype(np.float64), ((0, 0), (1, 1), (1, 1), (0, 0)))
    taps = np.stack([Xp[:, ky:ky + H, kx:kx + W, :] for ky in range(3) for kx in range(3)], axis=3)
    return dY.reshape(-1, dY.shape[-1]).astype(np.float64).T @ taps.reshape(-1, 9 * C)


@pytest.mark.parametrize("B,H,W,C,cout,splits", [
    (2, 8, 64, 32, 32, 1),      # 64-pixel K blocks, one box of 32 rows per tap, no split
    (2, 8, 64, 64, 48, 3),      # 64-row boxes, cout not a multiple of the N tile
    (1, 5, 32, 96, 64, 4),      # 32-pixel K blocks, 9C = 864 (a ragged last M tile), odd H
    (3, 4, 32, 128, 32, 7),     # 128-row boxes, more splits than fit evenly
    (1, 2, 96, 160, 16, 2),     # C = 160: 32-row boxes; W = 96: 32-pixel K blocks
    (2, 8, 64, 32, 32, 24),     # many slices: the reduction that splits the slices among threads
])
def test_wgrad_from_three_copies_matches_the_nine_tap_sum(env, B, H, W, C, cout, splits):
    """The weight gradient from three horizontally shifted copies, the vertical
    taps taken by TMA coordinates with zero fill at the top and bottom image
    rows, against the plain nine-tap sum in FP64 (same BF16 inputs)."""
    torch, lib = env
    g = torch.Generator(device="cuda").manual_seed(B * 1000 + H * 100 + W + C + cout)
    X = torch.randn(B, H, W, C, generator=g, device="cuda").to(torch.bfloat16)
    dY = torch.randn(B, H, W, cout, generator=g, device="cuda").to(torch.bfloat16)
    P = B * H * W
    XT3 = torch.full((3 * C, P), 7.0, dtype=torch.bfloat16, device="cuda")
    assert lib.lbm_nn_gather_t(_p(X), B, H, W, C, C, 3, _p(XT3), P, _stream(torch)) == 0
    dYT = dY.reshape(P, cout).T.contiguous()
    ldd = 9 * C + 8
    D = torch.full((cout, ldd), 5.0, dtype=torch.float32, device="cuda")
    ws = torch.empty(splits * 9 * C * cout, dtype=torch.float32, device="cuda")
    rc = lib.lbm_nn_wgrad3x3(_p(XT3), _p(dYT), B, H, W, C, cout, _p(D), ldd, splits, _p(ws), _stream(torch))
    assert rc == 0, lib.lbm_last_error(None)
    torch.cuda.synchronize()
    assert lib.lbm_nn_error(1) == 0
    ref = _wgrad_reference(X.float().cpu().numpy(), dY.float().cpu().numpy())
    got = D[:, :9 * C].double().cpu().numpy()
    # FP32 accumulation of P products of BF16-exact values
    assert np.abs(got - ref).max() <= 4e-6 * np.sqrt(P) * np.abs(ref).max()
    assert bool((D[:, 9 * C:] == 5.0).all())


def test_wgrad_from_three_copies_rejects_unsupported_shapes(env):
    torch, lib = env
    buf = torch.zeros(1 << 16, dtype=torch.float32, device="cuda")
    for (B, H, W, C, cout) in ((1, 4, 48, 32, 32), (1, 4, 64, 40, 32), (1, 4, 64, 32, 12), (1, 4, 16, 32, 32)):
        rc = lib.lbm_nn_wgrad3x3(_p(buf), _p(buf), B, H, W, C, cout, _p(buf), 9 * C, 1, _p(buf), _stream(torch))
        assert rc == -1, (B, H, W, C, cout)
    assert lib.lbm_nn_wgrad3x3(_p(buf), _p(buf), 1, 4, 64, 32, 32, _p(buf), 9 * 32 - 8, 1, _p(buf),
                               _stream(torch)) == -1
