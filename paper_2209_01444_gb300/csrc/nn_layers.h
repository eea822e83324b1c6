// Memory-bound layers of the surrogate network (see nn_layers.cu).
#pragma once

#include <cuda_runtime.h>

namespace nn {

cudaError_t im2col3x3(const void* X, int B, int H, int W, int C, int cpitch, void* A, cudaStream_t s);
cudaError_t col2im3x3(const float* dA, int B, int H, int W, int C, float* dX, int cpitch, cudaStream_t s);
cudaError_t relu_bwd(void* g, bool g_fp32, int gpitch, const void* y, int ypitch, long long rows, int C,
                     cudaStream_t s);
cudaError_t transpose(const void* in, int rows, int cols, int ipitch, void* out, int opitch, cudaStream_t s);
cudaError_t maxpool_fwd(const void* X, int B, int H, int W, int C, int xpitch, void* Y, cudaStream_t s);
cudaError_t maxpool_bwd(const void* X, int B, int H, int W, int C, int xpitch, const float* dY, float* dX, int dpitch,
                        cudaStream_t s);
cudaError_t shuffle_fwd(const void* U, int B, int H, int W, int C, void* Y, int ypitch, int c0, cudaStream_t s);
cudaError_t shuffle_bwd(const void* dY, bool dy_fp32, int ypitch, int c0, int B, int H, int W, int C, void* dU,
                        cudaStream_t s);
cudaError_t proj_fwd(const void* X, int P, int C, int xpitch, const float* Wt, const float* bias, int O,
                     const float* R, float* Y, cudaStream_t s);
cudaError_t proj_bwd(const float* dY, const void* X, int P, int C, int xpitch, const float* Wt, int O, float* dX,
                     int dpitch, float* dW, float* db, float* part, int part_blocks, cudaStream_t s);
cudaError_t flip3x3(const void* W, int cout, int cin, void* Wf, cudaStream_t s);
// Several flips in one launch: job j flips the kernel at W (cout x 9 cin) into
// Wf, its elements numbered from start (jobs in order of start; device table).
struct FlipJob {
    const void* W;
    void* Wf;
    int cout, cin;
    long long start;
};
cudaError_t flip3x3_many(const FlipJob* jobs, int njobs, long long total, cudaStream_t s);
cudaError_t gatherT(const void* X, int B, int H, int W, int C, int cpitch, int taps, void* AT, long long atpitch,
                    cudaStream_t s);
cudaError_t mask_cast(const float* g, int gpitch, const void* y, int ypitch, long long rows, int C, void* out,
                      int opitch, cudaStream_t s);
cudaError_t pad_conv3x3(const void* W, int cout, int cin, int cin_pad, void* Wp, cudaStream_t s);
cudaError_t colsum(const void* g, bool g_fp32, long long rows, int C, int pitch, float* out, float* part,
                   int part_blocks, cudaStream_t s);
// Mean of w (pred - target)^2 over n elements and its gradient; with x (the
// network input, F fields per pixel, phase field first) each pixel's
// elements are weighted by w = 1 + alpha max(0, 1 - phi^2), else w = 1.
cudaError_t mse(const float* pred, const float* target, long long n, float* grad, float* loss, float* part,
                cudaStream_t s, const float* x = nullptr, int F = 1, float alpha = 0.0f);
cudaError_t adam(float* w, const float* g, float* m, float* v, long long n, float lr, float b1, float b2, float eps,
                 int t, void* wb, cudaStream_t s);
cudaError_t pack(const float* f, long long P, int F, const float* mean, const float* inv_std, void* X, int cpitch,
                 float* R, cudaStream_t s);
cudaError_t unpack(const float* Y, long long P, int F, const float* mean, const float* inv_std, float* f,
                   cudaStream_t s);
cudaError_t increment(const float* t, const float* x, long long P, int F, const float* inv_out, float* T,
                      cudaStream_t s);
cudaError_t add_increment(const float* Y, const float* x, long long P, int F, const float* inv_out, float* y,
                          cudaStream_t s);
cudaError_t cast_bf16(const float* a, long long rows, int C, int apitch, void* b, int bpitch, cudaStream_t s);

}  // namespace nn
