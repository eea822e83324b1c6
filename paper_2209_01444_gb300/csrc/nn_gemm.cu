// Tensor-core GEMM for the surrogate network (sm_103a, tcgen05):
//   D[M][N] = act(A[M][K] * B[N][K]^T + bias[N])
// with BF16 operands in global memory, both K-major (row-major with K
// contiguous, row pitch a multiple of 8 elements), FP32 accumulation in tensor
// memory, and a BF16 or FP32 result.
//
// One CTA of 128 threads computes a 128 x BN tile.  Thread 0 drives a
// kStages-deep ring: TMA (cp.async.bulk.tensor, 128-byte swizzle) fills a
// stage and completes its `full` mbarrier; four tcgen05.mma (M = 128, N = BN,
// K = 16 each) consume it and tcgen05.commit arrives on its `empty` mbarrier,
// which frees the stage for the load issued kStages - 1 blocks ahead.  The
// accumulator lives in TMEM (BN FP32 columns x 128 lanes); after the last
// commit every warp reads its 32 lanes with tcgen05.ld, adds the bias, applies
// the activation and stores.  Every wait is bounded by a wall-clock limit:
// on expiry the kernel raises the error flag, drains what it issued (again
// bounded), frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include "lbm.h"
#include "nn_kernels.h"

namespace nn {

namespace {

constexpr int kBM = 128;
constexpr int kBK = 64;       // 64 BF16 = 128 bytes: one swizzle row
constexpr int kStages = 4;
constexpr int kThreads = 128;
constexpr unsigned long long kWaitNs = 1000000000ull;  // 1 s per wait

__device__ int g_gemm_error;  // set when a bounded wait expired

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// True once the phase of the given parity has completed; false after kWaitNs.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity)
{
    const uint32_t addr = smem_u32(bar);
    const unsigned long long t0 = global_ns();
    for (uint32_t it = 0;; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(addr), "r"(parity)
            : "memory");
        if (done) return true;
        if ((it & 63) == 63 && global_ns() - t0 > kWaitNs) return false;
    }
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* tm, int c0, int c1, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"((uint64_t)tm), "r"(c0), "r"(c1), "r"(smem_u32(bar))
        : "memory");
}

// Shared-memory matrix descriptor of a K-major tile stored with the 128-byte
// swizzle TMA produces: rows of 128 bytes, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address (16-byte units)
    d |= (uint64_t)1 << 16;                      // leading byte offset (unused with this swizzle)
    d |= (uint64_t)(1024 >> 4) << 32;            // stride byte offset: one 8-row group
    d |= (uint64_t)1 << 46;                      // descriptor version
    d |= (uint64_t)2 << 61;                      // 128-byte swizzle
    return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// blockIdx.z selects a slice of kb_per_split K blocks; with more than one
// slice each writes its FP32 partial tile to D + z * M * ldd (no bias or
// activation) and a reduction kernel finishes.
template <int BN, bool OUT_BF16>
__global__ void __launch_bounds__(kThreads, 1)
    k_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, void* __restrict__ D,
           const float* __restrict__ bias, int M, int N, int K, int ldd, int relu, int kb_per_split)
{
    constexpr int A_BYTES = kBM * kBK * 2;
    constexpr int B_BYTES = BN * kBK * 2;
    constexpr int STAGE = A_BYTES + B_BYTES;
    constexpr uint32_t TMEM_COLS = BN < 32 ? 32 : BN;
    constexpr uint32_t IDESC = idesc_bf16(kBM, BN);
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = (uint64_t*)(smem + kStages * STAGE);
    uint64_t* empty = full + kStages;
    uint64_t* done = empty + kStages;
    uint32_t* tmem_slot = (uint32_t*)(done + 1);
    int* status = (int*)(tmem_slot + 1);  // 0 ok, 1 timed out

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * BN;
    const int kb0 = blockIdx.z * kb_per_split;
    const int nk = min((K + kBK - 1) / kBK - kb0, kb_per_split);  // K blocks of this slice
    if (gridDim.z > 1) {
        D = (float*)D + (size_t)blockIdx.z * M * ldd;
        bias = nullptr;
        relu = 0;
    }

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        *status = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    int issued = 0;  // blocks whose loads were issued (thread 0)
    int consumed = 0;  // blocks whose MMAs were issued (thread 0)
    if (threadIdx.x == 0) {
        bool ok = true;
        for (int kb = 0; kb < nk && kb < kStages - 1; ++kb) {
            mbar_expect_tx(&full[kb], STAGE);
            tma_load_2d(smem + kb * STAGE, &tmA, (kb0 + kb) * kBK, m0, &full[kb]);
            tma_load_2d(smem + kb * STAGE + A_BYTES, &tmB, (kb0 + kb) * kBK, n0, &full[kb]);
            ++issued;
        }
        for (int kb = 0; kb < nk && ok; ++kb) {
            const int pf = kb + kStages - 1;  // block to prefetch now
            if (pf < nk) {
                const int ps = pf % kStages;
                if (pf >= kStages) ok = mbar_wait(&empty[ps], (uint32_t)((pf / kStages - 1) & 1));
                if (!ok) break;
                mbar_expect_tx(&full[ps], STAGE);
                tma_load_2d(smem + ps * STAGE, &tmA, (kb0 + pf) * kBK, m0, &full[ps]);
                tma_load_2d(smem + ps * STAGE + A_BYTES, &tmB, (kb0 + pf) * kBK, n0, &full[ps]);
                ++issued;
            }
            const int s = kb % kStages;
            ok = mbar_wait(&full[s], (uint32_t)((kb / kStages) & 1));
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = smem_u32(smem + s * STAGE), b0 = a0 + A_BYTES;
#pragma unroll
            for (int k = 0; k < kBK / 16; ++k)
                umma(tmem, sw128_desc(a0 + k * 32), sw128_desc(b0 + k * 32), IDESC, (kb > 0 || k > 0) ? 1u : 0u);
            umma_commit(&empty[s]);
            ++consumed;
        }
        umma_commit(done);  // arrives once every MMA issued so far has completed
        if (!ok) {
            *status = 1;
            atomicExch(&g_gemm_error, 1);
            // drain: loads issued but never consumed, bounded
            for (int kb = consumed; kb < issued; ++kb) mbar_wait(&full[kb % kStages], (uint32_t)((kb / kStages) & 1));
        }
    }
    __syncthreads();
    const bool finished = mbar_wait(done, 0);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!finished && threadIdx.x == 0) atomicExch(&g_gemm_error, 1);
    if (finished && *status == 0) {
        const int row = m0 + warp * 32 + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
        for (int c = 0; c < BN; c += 16) {
            uint32_t r[16];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15])
                : "r"(lane_base + (uint32_t)c));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            const int col = n0 + c;
            if (row < M && col < N) {
                float v[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    float x = __uint_as_float(r[j]) + ((bias && col + j < N) ? bias[col + j] : 0.0f);
                    v[j] = relu ? fmaxf(x, 0.0f) : x;
                }
                if (col + 16 > N) {  // ragged last tile: element stores
                    for (int j = 0; col + j < N; ++j) {
                        if (OUT_BF16)
                            ((__nv_bfloat16*)D)[(size_t)row * ldd + col + j] = __float2bfloat16_rn(v[j]);
                        else
                            ((float*)D)[(size_t)row * ldd + col + j] = v[j];
                    }
                } else if (OUT_BF16) {
                    __nv_bfloat162 h[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) h[j] = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
                    uint4* dst = (uint4*)((__nv_bfloat16*)D + (size_t)row * ldd + col);
                    dst[0] = *(uint4*)&h[0];
                    dst[1] = *(uint4*)&h[4];
                } else {
                    float4* dst = (float4*)((float*)D + (size_t)row * ldd + col);
#pragma unroll
                    for (int j = 0; j < 4; ++j) dst[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

cudaError_t encoder()
{
    if (g_encode) return cudaSuccess;
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    return cudaSuccess;
}

// 2-D tensor map of a row-major BF16 matrix [rows][ld] with K = cols valid
// columns, box of 64 columns x box_rows rows, 128-byte swizzle, zero fill.
cudaError_t make_map(CUtensorMap* tm, const void* ptr, int rows, int cols, int ld, int box_rows)
{
    cudaError_t e = encoder();
    if (e != cudaSuccess) return e;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = g_encode(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int BN, bool OUT_BF16>
cudaError_t launch_bn(const CUtensorMap& a, const CUtensorMap& b, void* D, const float* bias, int M, int N, int K,
                      int ldd, int relu, int splits, int kb_per_split, cudaStream_t s)
{
    constexpr int smem = kStages * (kBM * kBK * 2 + BN * kBK * 2) + 1024 + 256;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k_gemm<BN, OUT_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    dim3 grid((M + kBM - 1) / kBM, (N + BN - 1) / BN, splits);
    k_gemm<BN, OUT_BF16><<<grid, kThreads, smem, s>>>(a, b, D, bias, M, N, K, ldd, relu, kb_per_split);
    return cudaGetLastError();
}

// Sum of the FP32 partial tiles of a split-K GEMM, plus bias and activation.
template <bool OUT_BF16>
__global__ void k_split_reduce(const float* __restrict__ part, int splits, int M, int N, int ldp, void* __restrict__ D,
                               int ldd, const float* __restrict__ bias, int relu)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)M * N) return;
    const int row = (int)(i / N), col = (int)(i - (long long)row * N);
    float acc = bias ? bias[col] : 0.0f;
    for (int z = 0; z < splits; ++z) acc += part[(size_t)z * M * ldp + (size_t)row * ldp + col];
    if (relu) acc = fmaxf(acc, 0.0f);
    if (OUT_BF16)
        ((__nv_bfloat16*)D)[(size_t)row * ldd + col] = __float2bfloat16_rn(acc);
    else
        ((float*)D)[(size_t)row * ldd + col] = acc;
}

}  // namespace

cudaError_t gemm_bf16(const void* A, int lda, const void* B, int ldb, void* D, int ldd, const float* bias, int M,
                      int N, int K, bool out_bf16, bool relu, cudaStream_t s, int splits, float* workspace)
{
    const int bn = N >= 256 ? 256 : N > 64 ? 128 : N > 32 ? 64 : 32;
    if (N < 8 || N % 8) return cudaErrorInvalidValue;
    if (lda % 8 || ldb % 8 || ldd % 8 || K > lda || K > ldb || N > ldd || M < 1 || K < 1) return cudaErrorInvalidValue;
    if (((uintptr_t)A | (uintptr_t)B | (uintptr_t)D) & 15) return cudaErrorInvalidValue;
    const int nkb = (K + kBK - 1) / kBK;
    if (splits < 1) splits = 1;
    if (splits > nkb) splits = nkb;
    const int kb_per_split = (nkb + splits - 1) / splits;
    splits = (nkb + kb_per_split - 1) / kb_per_split;
    if (splits > 1 && !workspace) return cudaErrorInvalidValue;
    CUtensorMap ta, tb;
    cudaError_t e = make_map(&ta, A, M, K, lda, kBM);
    if (e == cudaSuccess) e = make_map(&tb, B, N, K, ldb, bn);
    if (e != cudaSuccess) return e;
    const int r = relu ? 1 : 0;
    void* out = splits > 1 ? (void*)workspace : D;
    const int ldo = splits > 1 ? N : ldd;
    const bool ob = splits > 1 ? false : out_bf16;
#define NN_GEMM_CASE(BNV)                                                                                      \
    case BNV:                                                                                                  \
        e = ob ? launch_bn<BNV, true>(ta, tb, out, bias, M, N, K, ldo, r, splits, kb_per_split, s)            \
               : launch_bn<BNV, false>(ta, tb, out, bias, M, N, K, ldo, r, splits, kb_per_split, s);          \
        break;
    switch (bn) {
        NN_GEMM_CASE(32)
        NN_GEMM_CASE(64)
        NN_GEMM_CASE(128)
        NN_GEMM_CASE(256)
    }
#undef NN_GEMM_CASE
    if (e != cudaSuccess || splits == 1) return e;
    const long long n = (long long)M * N;
    const unsigned grid = (unsigned)((n + 255) / 256);
    if (out_bf16)
        k_split_reduce<true><<<grid, 256, 0, s>>>(workspace, splits, M, N, N, D, ldd, bias, r);
    else
        k_split_reduce<false><<<grid, 256, 0, s>>>(workspace, splits, M, N, N, D, ldd, bias, r);
    return cudaGetLastError();
}

cudaError_t gemm_error(int* flag, bool clear)
{
    cudaError_t e = cudaMemcpyFromSymbol(flag, g_gemm_error, sizeof(int));
    if (e == cudaSuccess && clear) {
        const int zero = 0;
        e = cudaMemcpyToSymbol(g_gemm_error, &zero, sizeof(int));
    }
    return e;
}

}  // namespace nn
