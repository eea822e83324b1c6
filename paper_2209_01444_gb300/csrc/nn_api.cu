// C ABI of the surrogate network's kernels (declared in include/lbm.h).
#include <cuda_runtime.h>

#include "lbm.h"
#include "lbm_kernels.h"
#include "nn_kernels.h"
#include "nn_layers.h"

namespace {

int nn_status(cudaError_t e)
{
    if (e == cudaSuccess) return LBM_OK;
    lbm::set_last_error(cudaGetErrorString(e));
    return (e == cudaErrorInvalidValue || e == cudaErrorNotSupported) ? LBM_EINVAL : LBM_ECUDA;
}

}  // namespace

extern "C" {

int lbm_nn_gemm(const void* A, int lda, const void* B, int ldb, void* D, int ldd, const float* bias, int M, int N,
                int K, int out_fp32, int relu, void* stream)
{
    return lbm_nn_gemm_split(A, lda, B, ldb, D, ldd, bias, M, N, K, out_fp32, relu, 1, nullptr, stream);
}

int lbm_nn_gemm_split(const void* A, int lda, const void* B, int ldb, void* D, int ldd, const float* bias, int M,
                      int N, int K, int out_fp32, int relu, int splits, float* workspace, void* stream)
{
    if (!A || !B || !D) {
        lbm::set_last_error("lbm_nn_gemm: NULL operand");
        return LBM_EINVAL;
    }
    return nn_status(nn::gemm_bf16(A, lda, B, ldb, D, ldd, bias, M, N, K, !out_fp32, relu != 0, (cudaStream_t)stream,
                                   splits, workspace));
}

#define NN_S(stream) ((cudaStream_t)(stream))

int lbm_nn_im2col3x3(const void* X, int B, int H, int W, int C, int cpitch, void* A, void* stream)
{
    return nn_status(nn::im2col3x3(X, B, H, W, C, cpitch, A, NN_S(stream)));
}

int lbm_nn_col2im3x3(const float* dA, int B, int H, int W, int C, float* dX, int cpitch, void* stream)
{
    return nn_status(nn::col2im3x3(dA, B, H, W, C, dX, cpitch, NN_S(stream)));
}

int lbm_nn_relu_bwd(void* g, int g_fp32, int gpitch, const void* y, int ypitch, long long rows, int C, void* stream)
{
    return nn_status(nn::relu_bwd(g, g_fp32 != 0, gpitch, y, ypitch, rows, C, NN_S(stream)));
}

int lbm_nn_transpose(const void* in, int rows, int cols, int ipitch, void* out, int opitch, void* stream)
{
    return nn_status(nn::transpose(in, rows, cols, ipitch, out, opitch, NN_S(stream)));
}

int lbm_nn_maxpool_fwd(const void* X, int B, int H, int W, int C, int xpitch, void* Y, void* stream)
{
    return nn_status(nn::maxpool_fwd(X, B, H, W, C, xpitch, Y, NN_S(stream)));
}

int lbm_nn_maxpool_bwd(const void* X, int B, int H, int W, int C, int xpitch, const float* dY, float* dX, int dpitch,
                       void* stream)
{
    return nn_status(nn::maxpool_bwd(X, B, H, W, C, xpitch, dY, dX, dpitch, NN_S(stream)));
}

int lbm_nn_shuffle_fwd(const void* U, int B, int H, int W, int C, void* Y, int ypitch, int c0, void* stream)
{
    return nn_status(nn::shuffle_fwd(U, B, H, W, C, Y, ypitch, c0, NN_S(stream)));
}

int lbm_nn_shuffle_bwd(const void* dY, int dy_fp32, int ypitch, int c0, int B, int H, int W, int C, void* dU,
                       void* stream)
{
    return nn_status(nn::shuffle_bwd(dY, dy_fp32 != 0, ypitch, c0, B, H, W, C, dU, NN_S(stream)));
}

int lbm_nn_proj_fwd(const void* X, int P, int C, int xpitch, const float* Wt, const float* bias, int O, const float* R,
                    float* Y, void* stream)
{
    return nn_status(nn::proj_fwd(X, P, C, xpitch, Wt, bias, O, R, Y, NN_S(stream)));
}

int lbm_nn_proj_bwd(const float* dY, const void* X, int P, int C, int xpitch, const float* Wt, int O, float* dX,
                    int dpitch, float* dW, float* db, float* part, int part_blocks, void* stream)
{
    return nn_status(nn::proj_bwd(dY, X, P, C, xpitch, Wt, O, dX, dpitch, dW, db, part, part_blocks, NN_S(stream)));
}

int lbm_nn_conv3x3(const void* X, int B, int H, int W, int C, int cpitch, const void* Wm, int ldw, void* D, int ldd,
                   const float* bias, int N, int out_fp32, int relu, void* stream)
{
    return nn_status(nn::conv3x3_bf16(X, B, H, W, C, cpitch, Wm, ldw, D, ldd, bias, N, out_fp32 == 0, relu != 0,
                                      NN_S(stream)));
}

int lbm_nn_upconv2x2(const void* X, int lda, const void* Wm, int ldw, void* Y, int ypitch, int c0, const float* bias,
                     int B, int Hl, int Wl, int cin, int c, void* stream)
{
    return nn_status(nn::upconv2x2_bf16(X, lda, Wm, ldw, Y, ypitch, c0, bias, B, Hl, Wl, cin, c, NN_S(stream)));
}

int lbm_nn_gather_t(const void* X, int B, int H, int W, int C, int cpitch, int taps, void* AT, long long atpitch,
                    void* stream)
{
    return nn_status(nn::gatherT(X, B, H, W, C, cpitch, taps, AT, atpitch, NN_S(stream)));
}

int lbm_nn_wgrad3x3(const void* XT3, const void* dYT, int B, int H, int W, int C, int cout, float* D, int ldd,
                    int splits, float* workspace, void* stream)
{
    if (!XT3 || !dYT || !D || !workspace) {
        lbm::set_last_error("lbm_nn_wgrad3x3: NULL argument");
        return LBM_EINVAL;
    }
    return nn_status(nn::wgrad3_bf16(XT3, dYT, B, H, W, C, cout, D, ldd, NN_S(stream), splits, workspace));
}

int lbm_nn_flip3x3(const void* W, int cout, int cin, void* Wf, void* stream)
{
    return nn_status(nn::flip3x3(W, cout, cin, Wf, NN_S(stream)));
}

int lbm_nn_colsum(const void* g, int g_fp32, long long rows, int C, int pitch, float* out, float* part,
                  int part_blocks, void* stream)
{
    return nn_status(nn::colsum(g, g_fp32 != 0, rows, C, pitch, out, part, part_blocks, NN_S(stream)));
}

int lbm_nn_mse(const float* pred, const float* target, long long n, float* grad, float* loss, float* part,
               void* stream)
{
    return nn_status(nn::mse(pred, target, n, grad, loss, part, NN_S(stream)));
}

int lbm_nn_adam(float* w, const float* g, float* m, float* v, long long n, float lr, float b1, float b2, float eps,
                int t, void* w_bf16, void* stream)
{
    return nn_status(nn::adam(w, g, m, v, n, lr, b1, b2, eps, t, w_bf16, NN_S(stream)));
}

int lbm_nn_pack(const float* fields, long long P, int F, const float* mean, const float* inv_std, void* X, int cpitch,
                float* R, void* stream)
{
    return nn_status(nn::pack(fields, P, F, mean, inv_std, X, cpitch, R, NN_S(stream)));
}

int lbm_nn_unpack(const float* Y, long long P, int F, const float* mean, const float* inv_std, float* fields,
                  void* stream)
{
    return nn_status(nn::unpack(Y, P, F, mean, inv_std, fields, NN_S(stream)));
}

int lbm_nn_cast_bf16(const float* a, long long rows, int C, int apitch, void* b, int bpitch, void* stream)
{
    return nn_status(nn::cast_bf16(a, rows, C, apitch, b, bpitch, NN_S(stream)));
}

int lbm_nn_set_operand_wait(unsigned long long ns) { return nn_status(nn::set_operand_wait(ns)); }

int lbm_nn_error(int clear)
{
    int flag = 0;
    cudaError_t e = nn::gemm_error(&flag, clear != 0);
    if (e != cudaSuccess) return nn_status(e);
    return flag ? LBM_ETIMEOUT : LBM_OK;
}

}  // extern "C"
