// C ABI of the surrogate network's kernels (declared in include/lbm.h).
#include <cuda_runtime.h>

#include "lbm.h"
#include "lbm_kernels.h"
#include "nn_kernels.h"

namespace {

int nn_status(cudaError_t e)
{
    if (e == cudaSuccess) return LBM_OK;
    lbm::set_last_error(cudaGetErrorString(e));
    return e == cudaErrorInvalidValue ? LBM_EINVAL : LBM_ECUDA;
}

}  // namespace

extern "C" {

int lbm_nn_gemm(const void* A, int lda, const void* B, int ldb, void* D, int ldd, const float* bias, int M, int N,
                int K, int out_fp32, int relu, void* stream)
{
    if (!A || !B || !D) {
        lbm::set_last_error("lbm_nn_gemm: NULL operand");
        return LBM_EINVAL;
    }
    return nn_status(nn::gemm_bf16(A, lda, B, ldb, D, ldd, bias, M, N, K, !out_fp32, relu != 0, (cudaStream_t)stream));
}

int lbm_nn_error(int clear)
{
    int flag = 0;
    cudaError_t e = nn::gemm_error(&flag, clear != 0);
    if (e != cudaSuccess) return nn_status(e);
    return flag ? LBM_ETIMEOUT : LBM_OK;
}

}  // extern "C"
