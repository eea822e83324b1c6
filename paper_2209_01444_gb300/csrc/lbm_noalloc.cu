// lbm_reduce_noalloc: the reductions of lbm_get_metrics for callers that
// cannot allocate device memory.  The only scratch, one row of partial sums
// per block, is a file-scope device array that every GPU loading the library
// holds until the process exits; nothing here calls cudaMalloc or cudaFree.
#include <cuda_runtime.h>
#include <math.h>

#include <atomic>

#include "lbm.h"
#include "lbm_kernels.h"
#include "lbm_reduce.cuh"

namespace {

using lbm::StepParams;

constexpr int kThreads = lbm::kRedThreadsPerBlock;
constexpr int kNodesPerBlock = lbm::kRedNodesPerBlock;  // 16 nodes per thread
constexpr int kMaxBlocks = 8192;           // 33,554,432 nodes
constexpr int kVals = lbm::kRedValues;     // same partials as the handle's reduction

// 8192 blocks x 7 partials x 8 bytes = 448 KiB per device.
static __device__ __align__(256) double g_reduce_scratch[kMaxBlocks * kVals];

constexpr int kMaxDevices = 64;
std::atomic<double*> g_scratch_ptr[kMaxDevices];

// Device address of the scratch array on the current device.  In host code
// the name g_reduce_scratch is only a host-side stand-in, so the address is
// looked up once per device with that device current.
cudaError_t scratch_for_current_device(double** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    double* p = g_scratch_ptr[dev].load(std::memory_order_acquire);
    if (!p) {
        void* q = nullptr;
        e = cudaGetSymbolAddress(&q, g_reduce_scratch);
        if (e != cudaSuccess) return e;
        p = (double*)q;
        g_scratch_ptr[dev].store(p, std::memory_order_release);
    }
    *out = p;
    return cudaSuccess;
}

// Variant of the handle's node pass: block b folds its chunk of
// kNodesPerBlock nodes with the same arithmetic and order (reduce_chunk) and
// writes its row of partials; every row it writes is overwritten, so nothing
// needs clearing.
template <class Store>
__global__ void __launch_bounds__(kThreads) k_reduce_chunks(const StepParams P, const void* __restrict__ sc,
                                                            const void* __restrict__ fl, double* __restrict__ partials)
{
    lbm::reduce_chunk<Store>(P, sc, fl, partials);
}

int fail(int code, const char* msg)
{
    lbm::set_last_error(msg);
    return code;
}

}  // namespace

extern "C" int lbm_reduce_noalloc(const lbm_params* p, const void* scalar_pops, const void* flow_pops, double cx,
                                  double cy, double orient, double* out, void* stream)
{
    if (!p || !scalar_pops || !flow_pops || !out) return fail(LBM_EINVAL, "lbm_reduce_noalloc: NULL argument");
    if (!isfinite(cx) || !isfinite(cy) || !isfinite(orient))
        return fail(LBM_EINVAL, "lbm_reduce_noalloc: non-finite tip origin");
    StepParams P;
    const char* why = nullptr;
    if (lbm::params_to_step(p, &P, &why) != LBM_OK) return fail(LBM_EINVAL, why);
    const long long N = (long long)P.nx * P.ny;
    const long long blocks = (N + kNodesPerBlock - 1) / kNodesPerBlock;
    if (blocks > kMaxBlocks)
        return fail(LBM_EINVAL, "lbm_reduce_noalloc: grid larger than its 33554432-node limit");
    double* scratch = nullptr;
    cudaError_t e = scratch_for_current_device(&scratch);
    if (e != cudaSuccess) return fail(LBM_ECUDA, cudaGetErrorString(e));
    cudaStream_t s = (cudaStream_t)stream;
    switch (p->storage) {
    case LBM_FP16:
        k_reduce_chunks<lbm::StoreF16><<<(unsigned)blocks, kThreads, 0, s>>>(P, scalar_pops, flow_pops, scratch);
        break;
    case LBM_BF16:
        k_reduce_chunks<lbm::StoreBF16><<<(unsigned)blocks, kThreads, 0, s>>>(P, scalar_pops, flow_pops, scratch);
        break;
    default:
        k_reduce_chunks<lbm::StoreF32><<<(unsigned)blocks, kThreads, 0, s>>>(P, scalar_pops, flow_pops, scratch);
        break;
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(LBM_ECUDA, cudaGetErrorString(e));
    if ((e = lbm::launch_reduce_final(scratch, (int)blocks, out, s)) != cudaSuccess)
        return fail(LBM_ECUDA, cudaGetErrorString(e));
    if ((e = lbm::launch_tips(P, p->storage, scalar_pops, cx, cy, cos(orient), sin(orient), out, s)) != cudaSuccess)
        return fail(LBM_ECUDA, cudaGetErrorString(e));
    return LBM_OK;
}
