// Host-side declarations of the surrogate network's kernels (BF16 operands,
// FP32 accumulation).
#pragma once

#include <cuda_runtime.h>

namespace nn {

// D[M][N] = act(A[M][K] * B[N][K]^T + bias[N]) on tcgen05 tensor cores; A, B
// BF16 row-major with pitches lda, ldb (multiples of 8, >= K); D BF16 or FP32
// with pitch ldd; N a multiple of 8.  splits > 1 divides K into slices whose
// FP32 partials go to `workspace` (splits * M * N floats) and are then summed.
// mask (BF16 [M][mpitch], mpitch a multiple of 8, 16-byte aligned; BF16
// output and one slice only): each output becomes 0 where mask is not
// positive, the gradient through a ReLU whose output was mask.
cudaError_t gemm_bf16(const void* A, int lda, const void* B, int ldb, void* D, int ldd, const float* bias, int M,
                      int N, int K, bool out_bf16, bool relu, cudaStream_t s, int splits = 1,
                      float* workspace = nullptr, const void* mask = nullptr, int mpitch = 0);
// D[n][m] = sum_k A[m][k] B[n][k] (FP32, pitch ldd >= M): the same GEMM with
// its result transposed by the split-K reduction; `workspace` holds
// splits * M * N floats.
cudaError_t gemm_bf16_tout(const void* A, int lda, const void* B, int ldb, float* D, int ldd, int M, int N, int K,
                           cudaStream_t s, int splits, float* workspace);

// Implicit 3 x 3 convolution (zero padding) on tensor cores:
// D[p][n] = act(sum over taps t and channels c < C of X[pixel p shifted by t][c]
// * Wm[n][t * C + c] + bias[n]) with X NHWC BF16 [B][H][W][cpitch] and the
// weight matrix Wm [N][ldw] (ldw >= 9C).  C must be a multiple of 32 and a
// 128-pixel tile whole rows of whole images (W a multiple of 128, or a divisor
// of 128 with matching H); cudaErrorNotSupported otherwise.
// mask: as for gemm_bf16 (BF16 output).
cudaError_t conv3x3_bf16(const void* X, int B, int H, int W, int C, int cpitch, const void* Wm, int ldw, void* D,
                         int ldd, const float* bias, int N, bool out_bf16, bool relu, cudaStream_t s,
                         const void* mask = nullptr, int mpitch = 0);

bool conv3x3_supported(int B, int H, int W, int C);

// 2 x 2 stride-2 up-convolution: the GEMM of X [B*Hl*Wl][cin] with Wm [4c][cin]
// plus bias[4c], stored BF16 straight into Y[b][2y+dy][2x+dx][c0 + co] (pitch
// ypitch) from column (dy * 2 + dx) * c + co; c a multiple of 16.
cudaError_t upconv2x2_bf16(const void* X, int lda, const void* Wm, int ldw, void* Y, int ypitch, int c0,
                           const float* bias, int B, int Hl, int Wl, int cin, int c, cudaStream_t s);

// Weight gradient of a 3 x 3 convolution from three horizontally shifted
// transposed copies of its input (XT3 [3 C][B H W], gatherT with taps 3) and
// the transposed output gradient (dYT [cout][B H W]): D[cout][9 C] (pitch
// ldd >= 9 C) = sum over pixels, the vertical taps taken by TMA coordinates.
// Needs W % 32 == 0, C % 32 == 0, cout % 8 == 0 and a workspace of
// splits x 9 C x cout floats.
bool wgrad3_supported(int B, int H, int W, int C, int cout);
cudaError_t wgrad3_bf16(const void* XT3, const void* dYT, int B, int H, int W, int C, int cout, float* D, int ldd,
                        cudaStream_t s, int splits, float* workspace);

// Read (and optionally clear) the flag a GEMM raises when a bounded wait ran out.
cudaError_t gemm_error(int* flag, bool clear);
// Bound of the GEMMs' waits for their operand tiles on the current device.
cudaError_t set_operand_wait(unsigned long long ns);

}  // namespace nn
