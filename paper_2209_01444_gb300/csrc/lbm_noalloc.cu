// lbm_reduce_noalloc: the reductions of lbm_get_metrics for callers that
// cannot allocate device memory.  The only scratch, one row of partial sums
// per block, is a file-scope device array that every GPU loading the library
// holds until the process exits; nothing here calls cudaMalloc or cudaFree.
#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>

#include <mutex>

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

// Device address of the scratch array, per device, with the CUDA context it
// was looked up in: a device reset ends that context, the module is loaded
// again in the next one, and the old address is then stale.
struct ScratchEntry {
    unsigned long long ctx_id = 0;
    double* ptr = nullptr;
};
std::mutex g_scratch_mutex;
ScratchEntry g_scratch[kMaxDevices];

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);
CtxGetCurrentFn g_ctx_current = nullptr;
CtxGetIdFn g_ctx_id = nullptr;

// Identifier of the CUDA context current on this thread (unique for the
// life of the process).  Caller holds g_scratch_mutex.
cudaError_t current_context_id(unsigned long long* id)
{
    if (!g_ctx_current || !g_ctx_id) {
        void* a = nullptr;
        void* b = nullptr;
        cudaDriverEntryPointQueryResult qa, qb;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 4000, cudaEnableDefault, &qa);
        if (e == cudaSuccess) e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb);
        if (e != cudaSuccess) return e;
        if (qa != cudaDriverEntryPointSuccess || qb != cudaDriverEntryPointSuccess || !a || !b)
            return cudaErrorNotSupported;
        g_ctx_current = (CtxGetCurrentFn)a;
        g_ctx_id = (CtxGetIdFn)b;
    }
    CUcontext ctx = nullptr;
    if (g_ctx_current(&ctx) != CUDA_SUCCESS || !ctx) return cudaErrorContextIsDestroyed;
    return g_ctx_id(ctx, id) == CUDA_SUCCESS ? cudaSuccess : cudaErrorContextIsDestroyed;
}

// Device address of the scratch array for a call on `stream`.  In host code
// the name g_reduce_scratch is only a host-side stand-in, so the address is
// looked up with the device current: on every call outside stream capture,
// and kept per device and context for calls made while the stream is being
// captured.  *capture_first is set when a call under capture finds no
// address looked up in the current context.
cudaError_t scratch_for_stream(cudaStream_t stream, double** out, bool* capture_first)
{
    *capture_first = false;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    if ((e = cudaStreamIsCapturing(stream, &st)) != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    ScratchEntry& c = g_scratch[dev];
    if (st != cudaStreamCaptureStatusNone && !c.ptr) {  // nothing looked up yet: refuse before any other call
        *capture_first = true;
        return cudaSuccess;
    }
    unsigned long long id = 0;
    if ((e = current_context_id(&id)) != cudaSuccess) return e;
    if (st == cudaStreamCaptureStatusNone) {
        void* q = nullptr;
        if ((e = cudaGetSymbolAddress(&q, g_reduce_scratch)) != cudaSuccess) return e;
        c.ctx_id = id;
        c.ptr = (double*)q;
    } else if (c.ctx_id != id) {
        *capture_first = true;
        return cudaSuccess;
    }
    *out = c.ptr;
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
    cudaStream_t s = (cudaStream_t)stream;
    double* scratch = nullptr;
    bool capture_first = false;
    cudaError_t e = scratch_for_stream(s, &scratch, &capture_first);
    if (e != cudaSuccess) return fail(LBM_ECUDA, cudaGetErrorString(e));
    if (capture_first)
        return fail(LBM_EINVAL,
                    "lbm_reduce_noalloc: the stream is being captured and no earlier call on this device and "
                    "context looked up the scratch address; make one call before capture");
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
