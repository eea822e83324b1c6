// Host-side declarations of the surrogate network's kernels (BF16 operands,
// FP32 accumulation).
#pragma once

#include <cuda_runtime.h>

namespace nn {

// D[M][N] = act(A[M][K] * B[N][K]^T + bias[N]) on tcgen05 tensor cores; A, B
// BF16 row-major with pitches lda, ldb (multiples of 8, >= K); D BF16 or FP32
// with pitch ldd; N a multiple of 8.  splits > 1 divides K into slices whose
// FP32 partials go to `workspace` (splits * M * N floats) and are then summed.
cudaError_t gemm_bf16(const void* A, int lda, const void* B, int ldb, void* D, int ldd, const float* bias, int M,
                      int N, int K, bool out_bf16, bool relu, cudaStream_t s, int splits = 1,
                      float* workspace = nullptr);

// Read (and optionally clear) the flag a GEMM raises when a bounded wait ran out.
cudaError_t gemm_error(int* flag, bool clear);

}  // namespace nn
