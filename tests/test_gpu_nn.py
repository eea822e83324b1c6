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
    assert lib.lbm_nn_gemm(_p(A), 64, _p(A), 64, _p(D), 48, None, 128, 48, 64, 1, 0, None) != 0  # N = 48
    assert lib.lbm_nn_gemm(_p(A), 60, _p(A), 64, _p(D), 64, None, 128, 64, 64, 1, 0, None) != 0  # lda % 8
