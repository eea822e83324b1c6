// Tensor-core GEMM for the surrogate network (sm_103a, tcgen05):
//   D[M][N] = act(A[M][K] * B[N][K]^T + bias[N])
// with BF16 operands in global memory, both K-major (row-major with K
// contiguous, row pitch a multiple of 8 elements), FP32 accumulation in tensor
// memory, and a BF16 or FP32 result.
//
// One CTA of 128 threads computes a 128 x BN tile.  Thread 0 drives an
// S-deep ring (gemm_stages): TMA (cp.async.bulk.tensor, 128- or 64-byte
// swizzle) fills a stage and completes its `full` mbarrier; tcgen05.mma
// (M = 128, N = BN, K = 16 each) consume it and tcgen05.commit arrives on its
// `empty` mbarrier, which frees the stage for the load issued S - 2 blocks
// ahead.  The accumulator lives in TMEM (BN FP32 columns x 128 lanes); after the last
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
constexpr int kThreads = 128;
constexpr unsigned long long kWaitNs = 1000000000ull;  // 1 s per wait

__device__ int g_gemm_error;  // set when a bounded wait expired
// Bound of the MMA issuer's waits for its operand tiles (set_operand_wait);
// every other wait keeps kWaitNs.  0: such a wait gives up at once.
__device__ unsigned long long g_operand_wait_ns = kWaitNs;

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

// The MMA issuer's wait for the operand tiles of one k block: bounded by
// g_operand_wait_ns (0: gives up without waiting).
__device__ __forceinline__ bool mbar_wait_operands(uint64_t* bar, uint32_t parity)
{
    const unsigned long long lim = g_operand_wait_ns;
    if (lim == 0) return false;
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
        if ((it & 63) == 63 && global_ns() - t0 > lim) return false;
    }
}

__device__ __forceinline__ uint32_t mbar_try(uint64_t* bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done;
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

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* tm, int c0, int c1, int c2, int c3,
                                            uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(smem_u32(dst)),
        "l"((uint64_t)tm), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}

// Descriptor of a K-major tile with 64-byte rows (32 BF16) in the 64-byte
// swizzle TMA produces: 8-row groups 512 bytes apart.
__device__ __forceinline__ uint64_t sw64_desc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(512 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)4 << 61;  // 64-byte swizzle
    return d;
}

template <int BK>
__device__ __forceinline__ uint64_t tile_desc(uint32_t saddr)
{
    if constexpr (BK == 64)
        return sw128_desc(saddr);
    else
        return sw64_desc(saddr);
}

// Ring depth: as many stages as fit in about 200 KB of shared memory, 2 to 8
// (a stage holds MT 128-row A tiles and one BN-row B tile of BK columns).
template <int BK, int BN, int MT = 1>
constexpr int stages_for()
{
    constexpr int stage = (MT * kBM + BN) * BK * 2;
    constexpr int n = (200 * 1024) / stage;
    return n < 2 ? 2 : n > 8 ? 8 : n;
}

// Row-reuse form of the implicit 3 x 3 convolution: per stage and sub-tile
// one box of the 128 + 2 pixels of one input row around the sub-tile's 128
// output pixels, kept in a region of kRow3Rows rows (a whole number of swizzle
// patterns), and the three weight tiles of that row's taps.
constexpr int kRow3Rows = 136;

template <int BK, int BN, int MT, bool ROW3>
constexpr int ws_stage_bytes()
{
    return ROW3 ? MT * kRow3Rows * BK * 2 + 3 * BN * BK * 2 : (MT * kBM + BN) * BK * 2;
}

// Ring depth of the persistent kernel: as many stages as fit in about 200 KB,
// 2 to 8.
template <int BK, int BN, int MT, bool ROW3>
constexpr int ws_stages()
{
    constexpr int n = (200 * 1024) / ws_stage_bytes<BK, BN, MT, ROW3>();
    return n < 2 ? 2 : n > 8 ? 8 : n;
}

// Ring depth of the split-K kernel.  Narrow tiles (N <= 64) take at most 4
// stages (about 80 KB), so that two CTAs share an SM: their one issuing thread
// waits on load latency, and two CTAs keep twice the loads in flight (measured:
// 32- and 64-channel weight gradients 1.3x and 1.7x faster); wider tiles keep
// the deeper ring of one CTA per SM, which is faster for them.
template <int BK, int BN>
constexpr int gemm_stages()
{
    return (BN <= 64 && stages_for<BK, BN>() > 4) ? 4 : stages_for<BK, BN>();
}

}  // namespace

// Geometry of an implicit 3 x 3 convolution (the A operand gathered by
// 4-D TMA loads shifted by each tap) and of the up-convolution epilogue.
struct ConvGeo {
    int W = 0, H = 0;      // image size; W == 0: plain 2-D A operand
    int C = 0;             // input channels (a multiple of BK)
    int cblocks = 0;       // C / BK
    int row3 = 0;          // the A map's box is kBM + 2 pixels of one row (row-reuse form)
};
struct ShuffleGeo {
    int Wl = 0, Hl = 0;    // low-resolution image; Wl == 0: plain row-major store
    int c = 0, c0 = 0;     // channels per sub-pixel, first destination channel
    // ReLU mask of a plain store: each output becomes 0 where mask[row][col]
    // (BF16, pitch mpitch) is not positive, as the gradient of a ReLU whose
    // output was mask; null: no mask
    const __nv_bfloat16* mask = nullptr;
    int mpitch = 0;
};

// The ReLU mask of 16 output columns: m[row][col .. col + 15] loaded before
// the accumulator is read (so that the two latencies overlap), then v[j] = 0
// where the mask is not positive.  `all`: the 16 columns lie inside the
// matrix, else only its first n do (loaded element by element).
struct Mask16 {
    uint4 a, b;
};
__device__ __forceinline__ Mask16 load_relu_mask(const __nv_bfloat16* __restrict__ m, bool all)
{
    Mask16 k{};
    if (all) {
        k.a = ((const uint4*)m)[0];
        k.b = ((const uint4*)m)[1];
    }
    return k;
}
__device__ __forceinline__ void apply_relu_mask(float (&v)[16], const Mask16& k, const __nv_bfloat16* __restrict__ m,
                                                bool all, int n)
{
    if (all) {
        const uint32_t w[8] = {k.a.x, k.a.y, k.a.z, k.a.w, k.b.x, k.b.y, k.b.z, k.b.w};
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (!(__uint_as_float(w[j] << 16) > 0.0f)) v[2 * j] = 0.0f;
            if (!(__uint_as_float(w[j] & 0xffff0000u) > 0.0f)) v[2 * j + 1] = 0.0f;
        }
    } else {
        for (int j = 0; j < n && j < 16; ++j)
            if (!(__bfloat162float(m[j]) > 0.0f)) v[j] = 0.0f;
    }
}

namespace {

// One CTA of 128 threads computes a 128 x BN tile of D.  Plain mode: K block
// kb of A is the TMA box at (kb * BK, m0).  Convolution mode (CONV): the M
// tile is 128 consecutive output pixels (whole rows, or 128 pixels of one
// row), K runs over (tap, channel block) and the A box is the input tile
// shifted by the tap, (cb * BK, x0 + kx - 1, y0 + ky - 1, b0); TMA fills what
// lies outside the image with zeros, which is the convolution's zero padding.
// blockIdx.z selects a slice of kb_per_split K blocks; with more than one
// slice each writes its FP32 partial tile to D + z * M * ldd (no bias or
// activation) and a reduction kernel finishes.
//
// WG (weight gradient of a 3 x 3 convolution, dW^T = X_taps^T dY, K = pixels):
// the A rows are (tap t, input channel ci), t = 3 ky + kx, and tmA is a 4-D
// map (x, y, image, row) over three transposed copies of the input shifted
// by dx = kx - 1, row kx * C + ci (geo.C = C input channels); each K block of
// BK pixels lies in one image row, and each tap's rows of the A tile come
// from one box at that row shifted by dy = ky - 1 along y (zero filled
// outside the image, the convolution's padding).  The shift is on the y
// coordinate, so the innermost (x) coordinate stays a multiple of BK.
template <int BN, bool OUT_BF16, int BK, bool CONV, bool WG = false>
__global__ void __launch_bounds__(kThreads, 2)
    k_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, void* __restrict__ D,
           const float* __restrict__ bias, int M, int N, int K, int ldd, int relu, int kb_per_split, ConvGeo geo,
           ShuffleGeo sh)
{
    constexpr int S = gemm_stages<BK, BN>();
    constexpr int A_BYTES = kBM * BK * 2;
    constexpr int B_BYTES = BN * BK * 2;
    constexpr int STAGE = A_BYTES + B_BYTES;
    constexpr uint32_t TMEM_COLS = BN < 32 ? 32 : BN;
    constexpr uint32_t IDESC = idesc_bf16(kBM, BN);
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = (uint64_t*)(smem + S * STAGE);
    uint64_t* empty = full + S;
    uint64_t* done = empty + S;
    uint32_t* tmem_slot = (uint32_t*)(done + 1);
    int* status = (int*)(tmem_slot + 1);  // 0 ok, 1 timed out

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * BN;
    const int kb0 = blockIdx.z * kb_per_split;
    const int nk = min((K + BK - 1) / BK - kb0, kb_per_split);  // K blocks of this slice
    if (gridDim.z > 1) {
        D = (float*)D + (size_t)blockIdx.z * M * ldd;
        bias = nullptr;
        relu = 0;
    }
    int x0 = 0, y0 = 0, b0 = 0;
    if (CONV) {
        x0 = m0 % geo.W;
        y0 = (m0 / geo.W) % geo.H;
        b0 = m0 / (geo.W * geo.H);
    }

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
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

    // WG: the A boxes of this CTA's rows (fixed for the CTA) and the pixel
    // position (x, y, image) of the next K block to load, advanced by one K
    // block per load, so that the thread issuing the loads and MMAs does no
    // division in its loop (load is called with kb = 0, 1, 2, ... in order).
    int wx = 0, wy = 0, wb = 0, nbox = 0;
    int wrow[4] = {0, 0, 0, 0}, wdy[4] = {0, 0, 0, 0};
    if constexpr (WG) {
        const long long pp = (long long)kb0 * BK;  // first pixel of the slice
        wx = (int)(pp % geo.W);
        const long long rw = pp / geo.W;
        wy = (int)(rw % geo.H);
        wb = (int)(rw / geo.H);
        nbox = kBM / geo.cblocks;  // boxes of geo.cblocks rows (128, 64 or 32; divides C)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int row = m0 + j * geo.cblocks;
            const int t = row / geo.C, ci0 = row - t * geo.C;
            const int ky = t / 3, kx = t - 3 * ky;
            // rows past the nine taps: a box outside the map, zero filled
            wrow[j] = t < 9 ? kx * geo.C + ci0 : 3 * geo.C;
            wdy[j] = ky - 1;
        }
    }

    auto load = [&](int kb, int st) {
        uint8_t* a = smem + st * STAGE;
        mbar_expect_tx(&full[st], STAGE);
        if constexpr (WG) {
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (j < nbox)
                    tma_load_4d(a + j * geo.cblocks * BK * 2, &tmA, wx, wy + wdy[j], wb, wrow[j], &full[st]);
            tma_load_2d(a + A_BYTES, &tmB, (kb0 + kb) * BK, n0, &full[st]);
            wx += BK;
            if (wx == geo.W) {
                wx = 0;
                if (++wy == geo.H) {
                    wy = 0;
                    ++wb;
                }
            }
        } else if constexpr (CONV) {
            const int tap = kb / geo.cblocks, cb = kb - tap * geo.cblocks;
            const int ky = tap / 3, kx = tap - 3 * ky;
            tma_load_4d(a, &tmA, cb * BK, x0 + kx - 1, y0 + ky - 1, b0, &full[st]);
            tma_load_2d(a + A_BYTES, &tmB, tap * geo.C + cb * BK, n0, &full[st]);
        } else {
            tma_load_2d(a, &tmA, (kb0 + kb) * BK, m0, &full[st]);
            tma_load_2d(a + A_BYTES, &tmB, (kb0 + kb) * BK, n0, &full[st]);
        }
    };

    int issued = 0;    // blocks whose loads were issued (thread 0)
    int consumed = 0;  // blocks whose MMAs were issued (thread 0)
    // Loads run LA blocks ahead of the MMAs.  With LA = S - 2 the buffer a
    // prefetch reuses was read by the MMAs of two blocks back, which have
    // normally completed, so the thread does not wait for the MMAs it has just
    // issued before it can load again.
    constexpr int LA = S >= 4 ? S - 2 : S - 1;
    if (threadIdx.x == 0) {
        bool ok = true;
        for (int kb = 0; kb < nk && kb < LA; ++kb) {
            load(kb, kb);
            ++issued;
        }
        for (int kb = 0; kb < nk && ok; ++kb) {
            const int pf = kb + LA;  // block to prefetch now
            if (pf < nk) {
                const int ps = pf % S;
                if (pf >= S) ok = mbar_wait(&empty[ps], (uint32_t)((pf / S - 1) & 1));
                if (!ok) break;
                load(pf, ps);
                ++issued;
            }
            const int s = kb % S;
            ok = mbar_wait_operands(&full[s], (uint32_t)((kb / S) & 1));
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = smem_u32(smem + s * STAGE), b0s = a0 + A_BYTES;
#pragma unroll
            for (int k = 0; k < BK / 16; ++k)
                umma(tmem, tile_desc<BK>(a0 + k * 32), tile_desc<BK>(b0s + k * 32), IDESC,
                     (kb > 0 || k > 0) ? 1u : 0u);
            umma_commit(&empty[s]);
            ++consumed;
        }
        umma_commit(done);  // arrives once every MMA issued so far has completed
        if (!ok) {
            *status = 1;
            atomicExch(&g_gemm_error, 1);
            // drain: loads issued but never consumed, bounded
            for (int kb = consumed; kb < issued; ++kb) mbar_wait(&full[kb % S], (uint32_t)((kb / S) & 1));
        }
    }
    __syncthreads();
    const bool finished = mbar_wait(done, 0);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!finished && threadIdx.x == 0) atomicExch(&g_gemm_error, 1);
    if (finished && *status == 0) {
        const int row = m0 + warp * 32 + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
        // destination of this row: plain, or the 2 x 2 pixel shuffle of an up-convolution
        long long rbase = (long long)row * ldd;
        int sy = 0, sx = 0, sb = 0;
        if (sh.Wl) {
            sx = row % sh.Wl;
            sy = (row / sh.Wl) % sh.Hl;
            sb = row / (sh.Wl * sh.Hl);
        }
#pragma unroll 1
        for (int c = 0; c < BN; c += 16) {
            const bool mrow = sh.mask && row < M && n0 + c < N;
            const __nv_bfloat16* mp = mrow ? sh.mask + (long long)row * sh.mpitch + n0 + c : nullptr;
            const Mask16 mk = mrow ? load_relu_mask(mp, n0 + c + 16 <= N) : Mask16{};
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
                if (mrow) apply_relu_mask(v, mk, mp, col + 16 <= N, N - col);
                long long off = rbase + col;
                if (sh.Wl) {  // 16 columns of one sub-pixel (c is a multiple of 16)
                    const int sub = col / sh.c, co = col - sub * sh.c;
                    const long long q = ((long long)sb * 2 * sh.Hl + 2 * sy + (sub >> 1)) * (2LL * sh.Wl) +
                                        2 * sx + (sub & 1);
                    off = q * ldd + sh.c0 + co;
                }
                if (col + 16 > N) {  // ragged last tile: element stores
                    for (int j = 0; col + j < N; ++j) {
                        if (OUT_BF16)
                            ((__nv_bfloat16*)D)[off + j] = __float2bfloat16_rn(v[j]);
                        else
                            ((float*)D)[off + j] = v[j];
                    }
                } else if (OUT_BF16) {
                    __nv_bfloat162 h[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) h[j] = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
                    uint4* dst = (uint4*)((__nv_bfloat16*)D + off);
                    dst[0] = *(uint4*)&h[0];
                    dst[1] = *(uint4*)&h[4];
                } else {
                    float4* dst = (float4*)((float*)D + off);
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

// ----------------------------------------------------------------------------
// Persistent, warp-specialised form of the same tile computation.  Each CTA
// loops over tiles t = blockIdx.x, blockIdx.x + gridDim.x, ... (M fastest, so
// neighbouring CTAs share weight tiles and, for convolutions, input halos in
// L2).  Warp 0 (one lane) issues the TMA loads into an S-deep ring, warp 1
// (one lane) issues the MMAs into one of two TMEM accumulators, and warps
// 2-5 drain the other accumulator (tcgen05.ld, bias, activation, stores), so
// the epilogue of one tile overlaps the main loop of the next.  Every wait is
// bounded; a wait that runs out raises the error flag and a shared abort flag
// that makes the other roles stop, then the CTA drains its copies and MMAs
// (bounded) and frees its TMEM.  For an implicit 3 x 3 convolution a stage is
// one (tap, channel block) pair, or, in the row-reuse form (ROW3), one (input
// row, channel block) pair whose box serves the row's three taps.
constexpr int kWsThreads = 192;

__device__ __forceinline__ bool mbar_wait_abort(uint64_t* bar, uint32_t parity, volatile int* abort_flag)
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
        if ((it & 63) == 63) {
            if (*abort_flag) return false;
            if (global_ns() - t0 > kWaitNs) {
                *abort_flag = 1;
                atomicExch(&g_gemm_error, 1);
                return false;
            }
        }
    }
}

// The warp-specialised MMA issuer's wait for its operand tiles, bounded by
// g_operand_wait_ns; on expiry it raises the error and abort flags as
// mbar_wait_abort does.
__device__ __forceinline__ bool mbar_wait_operands_abort(uint64_t* bar, uint32_t parity, volatile int* abort_flag)
{
    const unsigned long long lim = g_operand_wait_ns;
    const uint32_t addr = smem_u32(bar);
    const unsigned long long t0 = global_ns();
    for (uint32_t it = 0;; ++it) {
        uint32_t done = 0;
        if (lim != 0)
            asm volatile(
                "{\n\t.reg .pred p;\n\t"
                "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                "selp.u32 %0, 1, 0, p;\n\t}"
                : "=r"(done)
                : "r"(addr), "r"(parity)
                : "memory");
        if (done) return true;
        if (lim == 0 || (it & 63) == 63) {
            if (*abort_flag) return false;
            if (lim == 0 || global_ns() - t0 > lim) {
                *abort_flag = 1;
                atomicExch(&g_gemm_error, 1);
                return false;
            }
        }
    }
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

template <int BN, bool OUT_BF16, int BK, bool CONV, int MT, bool ROW3 = false>
__global__ void __launch_bounds__(kWsThreads, 1)
    k_gemm_ws(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, void* __restrict__ D,
              const float* __restrict__ bias, int M, int N, int K, int ldd, int relu, ConvGeo geo, ShuffleGeo sh,
              int tiles_m, int tiles)
{
    static_assert(!ROW3 || CONV, "row reuse is a form of the implicit convolution");
    constexpr int S = ws_stages<BK, BN, MT, ROW3>();
    constexpr int A_BYTES = ROW3 ? kRow3Rows * BK * 2 : kBM * BK * 2;  // one sub-tile's A region
    constexpr int B_BYTES = BN * BK * 2;
    constexpr int NB = ROW3 ? 3 : 1;               // weight tiles per stage
    constexpr int STAGE = MT * A_BYTES + NB * B_BYTES;
    static_assert(STAGE == ws_stage_bytes<BK, BN, MT, ROW3>(), "stage layout");
    // bytes the TMA delivers per stage (ROW3: boxes of kBM + 2 rows)
    constexpr int TX = ROW3 ? MT * (kBM + 2) * BK * 2 + NB * B_BYTES : STAGE;
    constexpr uint32_t SUB_COLS = BN < 32 ? 32 : BN;
    constexpr uint32_t ACC_COLS = MT * SUB_COLS;
    constexpr uint32_t TMEM_COLS = 2 * ACC_COLS;
    constexpr uint32_t IDESC = idesc_bf16(kBM, BN);
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = (uint64_t*)(smem + S * STAGE);
    uint64_t* empty = full + S;
    uint64_t* acc_full = empty + S;
    uint64_t* acc_empty = acc_full + 2;
    uint64_t* done = acc_empty + 2;
    uint32_t* tmem_slot = (uint32_t*)(done + 1);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
    int* counts = (int*)(tmem_slot + 2);  // [0] loads issued, [1] k blocks consumed

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // k blocks: ROW3 takes the three taps of one input row per block
    const int nk = ROW3 ? 3 * geo.cblocks : (K + BK - 1) / BK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&acc_full[a], 1);
            mbar_init(&acc_empty[a], 128);
        }
        mbar_init(done, 1);
        *abort_flag = 0;
        counts[0] = counts[1] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {  // ---------------------------------------- producer
            asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmA) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmB) : "memory");
            int it = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
                const int m0 = (t % tiles_m) * (kBM * MT), n0 = (t / tiles_m) * BN;
                int x0[MT], y0[MT], b0[MT];
#pragma unroll
                for (int i = 0; i < MT; ++i) {
                    const int mi = m0 + i * kBM;
                    x0[i] = y0[i] = b0[i] = 0;
                    if (CONV) {
                        x0[i] = mi % geo.W;
                        y0[i] = (mi / geo.W) % geo.H;
                        b0[i] = mi / (geo.W * geo.H);
                    }
                }
                for (int kb = 0; kb < nk; ++kb, ++it) {
                    const int st = it % S;
                    if (it >= S && !(ok = mbar_wait_abort(&empty[st], (uint32_t)((it / S - 1) & 1), abort_flag)))
                        break;
                    uint8_t* a = smem + st * STAGE;
                    mbar_expect_tx(&full[st], TX);
                    if constexpr (ROW3) {
                        // input row y + ky - 1, pixels x0 - 1 .. x0 + kBM (zero filled outside the image)
                        const int ky = kb / geo.cblocks, cb = kb - ky * geo.cblocks;
#pragma unroll
                        for (int i = 0; i < MT; ++i)
                            tma_load_4d(a + i * A_BYTES, &tmA, cb * BK, x0[i] - 1, y0[i] + ky - 1, b0[i], &full[st]);
#pragma unroll
                        for (int kx = 0; kx < 3; ++kx)
                            tma_load_2d(a + MT * A_BYTES + kx * B_BYTES, &tmB, (3 * ky + kx) * geo.C + cb * BK, n0,
                                        &full[st]);
                    } else if constexpr (CONV) {
                        const int tap = kb / geo.cblocks, cb = kb - tap * geo.cblocks;
                        const int ky = tap / 3, kx = tap - 3 * ky;
#pragma unroll
                        for (int i = 0; i < MT; ++i)
                            tma_load_4d(a + i * A_BYTES, &tmA, cb * BK, x0[i] + kx - 1, y0[i] + ky - 1, b0[i],
                                        &full[st]);
                        tma_load_2d(a + MT * A_BYTES, &tmB, tap * geo.C + cb * BK, n0, &full[st]);
                    } else {
#pragma unroll
                        for (int i = 0; i < MT; ++i) tma_load_2d(a + i * A_BYTES, &tmA, kb * BK, m0 + i * kBM, &full[st]);
                        tma_load_2d(a + MT * A_BYTES, &tmB, kb * BK, n0, &full[st]);
                    }
                    counts[0] = it + 1;
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {  // --------------------------------------------- MMA
            int it = 0, lt = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x, ++lt) {
                const int acc = lt & 1;
                if (lt >= 2 && !(ok = mbar_wait_abort(&acc_empty[acc], (uint32_t)((lt / 2 - 1) & 1), abort_flag)))
                    break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t d = tmem + (uint32_t)(acc * ACC_COLS);
                for (int kb = 0; kb < nk; ++kb, ++it) {
                    const int st = it % S;
                    if (!(ok = mbar_wait_operands_abort(&full[st], (uint32_t)((it / S) & 1), abort_flag))) break;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t a0 = smem_u32(smem + st * STAGE), b0s = a0 + MT * A_BYTES;
                    if constexpr (ROW3) {
                        // tap kx reads the row box from pixel kx on: its A tile starts kx rows in
#pragma unroll
                        for (int kx = 0; kx < 3; ++kx)
#pragma unroll
                            for (int k = 0; k < BK / 16; ++k)
#pragma unroll
                                for (int i = 0; i < MT; ++i)
                                    umma(d + (uint32_t)(i * SUB_COLS),
                                         tile_desc<BK>(a0 + i * A_BYTES + kx * BK * 2 + k * 32),
                                         tile_desc<BK>(b0s + kx * B_BYTES + k * 32), IDESC,
                                         (kb > 0 || kx > 0 || k > 0) ? 1u : 0u);
                    } else {
#pragma unroll
                        for (int k = 0; k < BK / 16; ++k)
#pragma unroll
                            for (int i = 0; i < MT; ++i)
                                umma(d + (uint32_t)(i * SUB_COLS), tile_desc<BK>(a0 + i * A_BYTES + k * 32),
                                     tile_desc<BK>(b0s + k * 32), IDESC, (kb > 0 || k > 0) ? 1u : 0u);
                    }
                    umma_commit(&empty[st]);
                    counts[1] = it + 1;
                }
                if (ok) umma_commit(&acc_full[acc]);
            }
            umma_commit(done);  // completes once every MMA issued has finished
        }
    } else {  // --------------------------------------------------- epilogue
        const int q = warp & 3;  // TMEM lane quarter this warp may access
        const int et = threadIdx.x - 64;
        (void)et;
        int lt = 0;
        for (int t = blockIdx.x; t < tiles; t += gridDim.x, ++lt) {
            const int acc = lt & 1;
            if (!mbar_wait_abort(&acc_full[acc], (uint32_t)((lt / 2) & 1), abort_flag)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int n0 = (t / tiles_m) * BN;
#pragma unroll 1
            for (int sub = 0; sub < MT; ++sub) {
            const int row = (t % tiles_m) * (kBM * MT) + sub * kBM + q * 32 + lane;
            const uint32_t lane_base =
                tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * ACC_COLS + sub * SUB_COLS);
            long long rbase = (long long)row * ldd;
            int sy = 0, sx = 0, sb = 0;
            if (sh.Wl) {
                sx = row % sh.Wl;
                sy = (row / sh.Wl) % sh.Hl;
                sb = row / (sh.Wl * sh.Hl);
            }
#pragma unroll 1
            for (int c = 0; c < BN; c += 16) {
                const bool mrow = sh.mask && row < M && n0 + c < N;
                const __nv_bfloat16* mp = mrow ? sh.mask + (long long)row * sh.mpitch + n0 + c : nullptr;
                const Mask16 mk = mrow ? load_relu_mask(mp, n0 + c + 16 <= N) : Mask16{};
                uint32_t r[16];
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                    "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                      "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                      "=r"(r[14]), "=r"(r[15])
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
                    if (mrow) apply_relu_mask(v, mk, mp, col + 16 <= N, N - col);
                    long long off = rbase + col;
                    if (sh.Wl) {
                        const int sub = col / sh.c, co = col - sub * sh.c;
                        const long long qq = ((long long)sb * 2 * sh.Hl + 2 * sy + (sub >> 1)) * (2LL * sh.Wl) +
                                             2 * sx + (sub & 1);
                        off = qq * ldd + sh.c0 + co;
                    }
                    if (col + 16 > N) {
                        for (int j = 0; col + j < N; ++j) {
                            if (OUT_BF16)
                                ((__nv_bfloat16*)D)[off + j] = __float2bfloat16_rn(v[j]);
                            else
                                ((float*)D)[off + j] = v[j];
                        }
                    } else if (OUT_BF16) {
                        __nv_bfloat162 h[8];
#pragma unroll
                        for (int j = 0; j < 8; ++j) h[j] = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
                        uint4* dst = (uint4*)((__nv_bfloat16*)D + off);
                        dst[0] = *(uint4*)&h[0];
                        dst[1] = *(uint4*)&h[4];
                    } else {
                        float4* dst = (float4*)((float*)D + off);
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            dst[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
                    }
                }
            }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive(&acc_empty[acc]);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        // every issued MMA completes before TMEM is freed; on an abort also
        // every issued copy lands before the CTA's shared memory goes away
        unsigned long long t0 = global_ns();
        bool fin = false;
        while (!(fin = (bool)mbar_try(done, 0)) && global_ns() - t0 < kWaitNs) {
        }
        if (!fin) atomicExch(&g_gemm_error, 1);
        if (*abort_flag)
            for (int it = counts[1]; it < counts[0]; ++it) mbar_wait(&full[it % S], (uint32_t)((it / S) & 1));
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 1)
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
// columns, box of BK columns x box_rows rows, swizzle of BK * 2 bytes, zero fill.
cudaError_t make_map(CUtensorMap* tm, const void* ptr, int rows, int cols, int ld, int box_rows, int bk)
{
    cudaError_t e = encoder();
    if (e != cudaSuccess) return e;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {(cuuint32_t)bk, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = g_encode(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, bk == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// 4-D tensor map of an NHWC BF16 image batch [B][H][W][cpitch] whose first C
// channels are read, with the box (bk channels, bw, bh, bb) of one 128-pixel
// tile.
cudaError_t make_map_4d(CUtensorMap* tm, const void* ptr, int B, int H, int W, int C, int cpitch, int bw, int bh,
                        int bb, int bk)
{
    cudaError_t e = encoder();
    if (e != cudaSuccess) return e;
    cuuint64_t dims[4] = {(cuuint64_t)C, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)B};
    cuuint64_t strides[3] = {(cuuint64_t)cpitch * 2, (cuuint64_t)W * cpitch * 2, (cuuint64_t)H * W * cpitch * 2};
    cuuint32_t box[4] = {(cuuint32_t)bk, (cuuint32_t)bw, (cuuint32_t)bh, (cuuint32_t)bb};
    cuuint32_t es[4] = {1, 1, 1, 1};
    CUresult r = g_encode(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(ptr), dims, strides, box, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, bk == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int BN, bool OUT_BF16, int BK, bool CONV, bool WG = false>
cudaError_t launch_bn(const CUtensorMap& a, const CUtensorMap& b, void* D, const float* bias, int M, int N, int K,
                      int ldd, int relu, int splits, int kb_per_split, const ConvGeo& geo, const ShuffleGeo& sh,
                      cudaStream_t s)
{
    constexpr int smem = gemm_stages<BK, BN>() * (kBM * BK * 2 + BN * BK * 2) + 1024 + 256;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k_gemm<BN, OUT_BF16, BK, CONV, WG>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    dim3 grid((M + kBM - 1) / kBM, (N + BN - 1) / BN, splits);
    k_gemm<BN, OUT_BF16, BK, CONV, WG><<<grid, kThreads, smem, s>>>(a, b, D, bias, M, N, K, ldd, relu,
                                                                    kb_per_split, geo, sh);
    return cudaGetLastError();
}

template <int BN, bool OUT_BF16, int BK, bool CONV, int MT, bool ROW3>
cudaError_t launch_ws_mt(const CUtensorMap& a, const CUtensorMap& b, void* D, const float* bias, int M, int N, int K,
                         int ldd, int relu, const ConvGeo& geo, const ShuffleGeo& sh, cudaStream_t s)
{
    constexpr int smem = ws_stages<BK, BN, MT, ROW3>() * ws_stage_bytes<BK, BN, MT, ROW3>() + 1024 + 256;
    static_assert(smem <= 227 * 1024, "shared memory per CTA");
    static int per_sm = 0, sms = 0;
    if (!per_sm) {
        cudaError_t e = cudaFuncSetAttribute(k_gemm_ws<BN, OUT_BF16, BK, CONV, MT, ROW3>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        int dev = 0;
        if ((e = cudaGetDevice(&dev))) return e;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev))) return e;
        int occ = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_gemm_ws<BN, OUT_BF16, BK, CONV, MT, ROW3>,
                                                               kWsThreads, smem)))
            return e;
        per_sm = occ < 1 ? 1 : occ;
    }
    const int tiles_m = (M + kBM * MT - 1) / (kBM * MT);
    const int tiles = tiles_m * ((N + BN - 1) / BN);
    const int grid = tiles < sms * per_sm ? tiles : sms * per_sm;
    k_gemm_ws<BN, OUT_BF16, BK, CONV, MT, ROW3><<<grid, kWsThreads, smem, s>>>(a, b, D, bias, M, N, K, ldd, relu, geo,
                                                                               sh, tiles_m, tiles);
    return cudaGetLastError();
}

int g_sms = 0;

int sm_count()
{
    if (!g_sms) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            g_sms = 1;
    }
    return g_sms;
}

// Sub-tiles per tile: narrow tiles stack 128-row sub-tiles that share each
// weight tile (four for N = 32 with 32-channel K blocks, two up to N = 128),
// unless that leaves fewer tiles than SMs.
template <int BN, bool OUT_BF16, int BK, bool CONV, bool ROW3>
cudaError_t launch_ws_rows(const CUtensorMap& a, const CUtensorMap& b, void* D, const float* bias, int M, int N,
                           int K, int ldd, int relu, const ConvGeo& geo, const ShuffleGeo& sh, cudaStream_t s)
{
    sm_count();
    constexpr int MTMAX = (BN <= 32 && BK == 32) ? 4 : BN <= 128 ? 2 : 1;
    const long long ntiles_n = (N + BN - 1) / BN;
    auto fills = [&](int mt) { return (M + 128LL * mt - 1) / (128LL * mt) * ntiles_n >= g_sms; };
    if constexpr (MTMAX == 4)
        if (fills(4))
            return launch_ws_mt<BN, OUT_BF16, BK, CONV, 4, ROW3>(a, b, D, bias, M, N, K, ldd, relu, geo, sh, s);
    if constexpr (MTMAX >= 2)
        if (fills(2))
            return launch_ws_mt<BN, OUT_BF16, BK, CONV, 2, ROW3>(a, b, D, bias, M, N, K, ldd, relu, geo, sh, s);
    return launch_ws_mt<BN, OUT_BF16, BK, CONV, 1, ROW3>(a, b, D, bias, M, N, K, ldd, relu, geo, sh, s);
}

// Row reuse (geo.row3, set by conv3x3_bf16 with its matching A map) serves
// tiles up to 64 columns: wider ones would leave a ring of two stages.
template <int BN, bool OUT_BF16, int BK, bool CONV>
cudaError_t launch_ws(const CUtensorMap& a, const CUtensorMap& b, void* D, const float* bias, int M, int N, int K,
                      int ldd, int relu, const ConvGeo& geo, const ShuffleGeo& sh, cudaStream_t s)
{
    if constexpr (CONV && BN <= 64)
        if (geo.row3) return launch_ws_rows<BN, OUT_BF16, BK, CONV, true>(a, b, D, bias, M, N, K, ldd, relu, geo, sh, s);
    return launch_ws_rows<BN, OUT_BF16, BK, CONV, false>(a, b, D, bias, M, N, K, ldd, relu, geo, sh, s);
}

// Widest tile that N allows: narrower tiles with more CTAs re-read A and
// measured slower even where the wide tiles leave SMs idle.
int bn_for(int N) { return N >= 256 ? 256 : N > 64 ? 128 : N > 32 ? 64 : 32; }

template <int BK, bool CONV>
cudaError_t dispatch(int bn, bool ob, const CUtensorMap& ta, const CUtensorMap& tb, void* out, const float* bias, int M,
                     int N, int K, int ldo, int r, int splits, int kbps, const ConvGeo& geo, const ShuffleGeo& sh,
                     cudaStream_t s)
{
#define NN_GEMM_CASE(BNV)                                                                                            \
    case BNV:                                                                                                        \
        if (splits == 1)                                                                                             \
            return ob ? launch_ws<BNV, true, BK, CONV>(ta, tb, out, bias, M, N, K, ldo, r, geo, sh, s)               \
                      : launch_ws<BNV, false, BK, CONV>(ta, tb, out, bias, M, N, K, ldo, r, geo, sh, s);             \
        return ob ? launch_bn<BNV, true, BK, CONV>(ta, tb, out, bias, M, N, K, ldo, r, splits, kbps, geo, sh, s)    \
                  : launch_bn<BNV, false, BK, CONV>(ta, tb, out, bias, M, N, K, ldo, r, splits, kbps, geo, sh, s);
    switch (bn) {
        NN_GEMM_CASE(32)
        NN_GEMM_CASE(64)
        NN_GEMM_CASE(128)
        NN_GEMM_CASE(256)
    }
#undef NN_GEMM_CASE
    return cudaErrorInvalidValue;
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

// The transposed sum with many slices: a CTA takes 32 columns of one row, its
// 8 thread rows slices ty, ty + 8, ... (reads along the columns), and the 8
// partial sums of each column are added through shared memory in a fixed order.
__global__ void k_split_reduce_t_many(const float* __restrict__ part, int splits, int M, int N, int ldp,
                                      float* __restrict__ D, int ldd)
{
    __shared__ float t[8][32];
    const int row = blockIdx.y, col = blockIdx.x * 32 + threadIdx.x;
    float acc = 0.0f;
    if (col < N)
        for (int z = threadIdx.y; z < splits; z += 8) acc += part[(size_t)z * M * ldp + (size_t)row * ldp + col];
    t[threadIdx.y][threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.y == 0 && col < N) {
        float v = 0.0f;
#pragma unroll
        for (int k = 0; k < 8; ++k) v += t[k][threadIdx.x];
        D[(size_t)col * ldd + row] = v;
    }
}

// The transposed sum with few slices: a 32 x 32 tile of (row, col) per CTA,
// summed with reads along col and written through shared memory along row.
__global__ void k_split_reduce_t_tile(const float* __restrict__ part, int splits, int M, int N, int ldp,
                                      float* __restrict__ D, int ldd)
{
    __shared__ float t[32][33];
    const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int row = r0 + ty + 8 * k, col = c0 + tx;
        float acc = 0.0f;
        if (row < M && col < N)
            for (int z = 0; z < splits; ++z) acc += part[(size_t)z * M * ldp + (size_t)row * ldp + col];
        t[ty + 8 * k][tx] = acc;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int col = c0 + ty + 8 * k, row = r0 + tx;
        if (row < M && col < N) D[(size_t)col * ldd + row] = t[tx][ty + 8 * k];
    }
}

// D[col][row] (pitch ldd) = the sum of the slices' partial tiles.
cudaError_t launch_split_reduce_t(const float* part, int splits, int M, int N, float* D, int ldd, cudaStream_t s)
{
    if (splits >= 16 && M <= 65535) {
        const dim3 grid((unsigned)((N + 31) / 32), (unsigned)M);
        k_split_reduce_t_many<<<grid, dim3(32, 8), 0, s>>>(part, splits, M, N, N, D, ldd);
    } else {
        const dim3 grid((unsigned)((N + 31) / 32), (unsigned)((M + 31) / 32));  // M < 2^21 (M = 9 C)
        k_split_reduce_t_tile<<<grid, dim3(32, 8), 0, s>>>(part, splits, M, N, N, D, ldd);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t gemm_bf16_tout(const void* A, int lda, const void* B, int ldb, float* D, int ldd, int M, int N, int K,
                           cudaStream_t s, int splits, float* workspace)
{
    const int bn = bn_for(N);
    if (N < 8 || N % 8 || !workspace) return cudaErrorInvalidValue;
    if (lda % 8 || ldb % 8 || K > lda || K > ldb || M > ldd || M < 1 || K < 1) return cudaErrorInvalidValue;
    if (((uintptr_t)A | (uintptr_t)B | (uintptr_t)D) & 15) return cudaErrorInvalidValue;
    const int nkb = (K + kBK - 1) / kBK;
    if (splits < 1) splits = 1;
    if (splits > nkb) splits = nkb;
    const int kb_per_split = (nkb + splits - 1) / splits;
    splits = (nkb + kb_per_split - 1) / kb_per_split;
    CUtensorMap ta, tb;
    cudaError_t e = make_map(&ta, A, M, K, lda, kBM, kBK);
    if (e == cudaSuccess) e = make_map(&tb, B, N, K, ldb, bn, kBK);
    if (e != cudaSuccess) return e;
    // every split (one included) goes through the workspace; the reduction
    // writes the transpose
    e = dispatch<kBK, false>(bn, false, ta, tb, workspace, nullptr, M, N, K, N, 0, splits, kb_per_split, ConvGeo{},
                             ShuffleGeo{}, s);
    if (e != cudaSuccess) return e;
    return launch_split_reduce_t(workspace, splits, M, N, D, ldd, s);
}

bool wgrad3_supported(int B, int H, int W, int C, int cout)
{
    const long long P = (long long)B * H * W;
    return B >= 1 && H >= 1 && W >= 32 && W % 32 == 0 && C >= 32 && C % 32 == 0 && cout >= 8 && cout % 8 == 0 &&
           P <= 0x7fffffffLL && 9LL * C <= 0x7fffffffLL;
}

cudaError_t wgrad3_bf16(const void* XT3, const void* dYT, int B, int H, int W, int C, int cout, float* D, int ldd,
                        cudaStream_t s, int splits, float* workspace)
{
    if (!wgrad3_supported(B, H, W, C, cout) || !workspace) return cudaErrorInvalidValue;
    if (((uintptr_t)XT3 | (uintptr_t)dYT | (uintptr_t)D) & 15) return cudaErrorInvalidValue;
    const long long P = (long long)B * H * W;
    const int M = 9 * C, N = cout, K = (int)P;
    if (M > ldd) return cudaErrorInvalidValue;
    const int bk = W % 64 == 0 ? 64 : 32;
    // A rows per box: 128, 64 or 32, whichever is the largest to divide C, so
    // that no box straddles two taps
    const int rb = C % 128 == 0 ? 128 : C % 64 == 0 ? 64 : 32;
    cudaError_t e = encoder();
    if (e != cudaSuccess) return e;
    CUtensorMap ta, tb;
    {
        cuuint64_t dims[4] = {(cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)B, (cuuint64_t)(3 * C)};
        cuuint64_t strides[3] = {(cuuint64_t)W * 2, (cuuint64_t)H * W * 2, (cuuint64_t)P * 2};
        cuuint32_t box[4] = {(cuuint32_t)bk, 1, 1, (cuuint32_t)rb};
        cuuint32_t es[4] = {1, 1, 1, 1};
        CUresult r = g_encode(&ta, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(XT3), dims, strides, box, es,
                              CU_TENSOR_MAP_INTERLEAVE_NONE,
                              bk == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    }
    const int bn = bn_for(N);
    if ((e = make_map(&tb, dYT, N, K, K, bn, bk)) != cudaSuccess) return e;
    const int nkb = K / bk;
    if (splits < 1) splits = 1;
    if (splits > nkb) splits = nkb;
    const int kb_per_split = (nkb + splits - 1) / splits;
    splits = (nkb + kb_per_split - 1) / kb_per_split;
    ConvGeo geo;
    geo.W = W;
    geo.H = H;
    geo.C = C;
    geo.cblocks = rb;
#define NN_WG_CASE(BNV)                                                                                        \
    case BNV:                                                                                                  \
        e = bk == 64 ? launch_bn<BNV, false, 64, false, true>(ta, tb, workspace, nullptr, M, N, K, N, 0, splits, \
                                                              kb_per_split, geo, ShuffleGeo{}, s)              \
                     : launch_bn<BNV, false, 32, false, true>(ta, tb, workspace, nullptr, M, N, K, N, 0, splits, \
                                                              kb_per_split, geo, ShuffleGeo{}, s);             \
        break;
    switch (bn) {
        NN_WG_CASE(32)
        NN_WG_CASE(64)
        NN_WG_CASE(128)
        NN_WG_CASE(256)
    default:
        return cudaErrorInvalidValue;
    }
#undef NN_WG_CASE
    if (e != cudaSuccess) return e;
    return launch_split_reduce_t(workspace, splits, M, N, D, ldd, s);
}

// The ReLU-mask epilogue of a single-slice GEMM or convolution storing BF16:
// mask rows of pitch mpitch (a multiple of 8), 16-byte aligned.
static bool mask_ok(const void* mask, int mpitch, bool out_bf16, int N)
{
    return out_bf16 && mpitch % 8 == 0 && mpitch >= N && ((uintptr_t)mask & 15) == 0;
}

cudaError_t gemm_bf16(const void* A, int lda, const void* B, int ldb, void* D, int ldd, const float* bias, int M,
                      int N, int K, bool out_bf16, bool relu, cudaStream_t s, int splits, float* workspace,
                      const void* mask, int mpitch)
{
    const int bn = bn_for(N);
    if (N < 8 || N % 8) return cudaErrorInvalidValue;
    if (mask && (!mask_ok(mask, mpitch, out_bf16, N) || splits > 1)) return cudaErrorInvalidValue;
    if (lda % 8 || ldb % 8 || ldd % 8 || K > lda || K > ldb || N > ldd || M < 1 || K < 1) return cudaErrorInvalidValue;
    if (((uintptr_t)A | (uintptr_t)B | (uintptr_t)D) & 15) return cudaErrorInvalidValue;
    const int nkb = (K + kBK - 1) / kBK;
    if (splits < 1) splits = 1;
    if (splits > nkb) splits = nkb;
    const int kb_per_split = (nkb + splits - 1) / splits;
    splits = (nkb + kb_per_split - 1) / kb_per_split;
    if (splits > 1 && !workspace) return cudaErrorInvalidValue;
    CUtensorMap ta, tb;
    cudaError_t e = make_map(&ta, A, M, K, lda, kBM, kBK);
    if (e == cudaSuccess) e = make_map(&tb, B, N, K, ldb, bn, kBK);
    if (e != cudaSuccess) return e;
    const int r = relu ? 1 : 0;
    void* out = splits > 1 ? (void*)workspace : D;
    const int ldo = splits > 1 ? N : ldd;
    const bool ob = splits > 1 ? false : out_bf16;
    ShuffleGeo sh;
    sh.mask = (const __nv_bfloat16*)mask;
    sh.mpitch = mpitch;
    e = dispatch<kBK, false>(bn, ob, ta, tb, out, bias, M, N, K, ldo, r, splits, kb_per_split, ConvGeo{}, sh, s);
    if (e != cudaSuccess || splits == 1) return e;
    const long long n = (long long)M * N;
    const unsigned grid = (unsigned)((n + 255) / 256);
    if (out_bf16)
        k_split_reduce<true><<<grid, 256, 0, s>>>(workspace, splits, M, N, N, D, ldd, bias, r);
    else
        k_split_reduce<false><<<grid, 256, 0, s>>>(workspace, splits, M, N, N, D, ldd, bias, r);
    return cudaGetLastError();
}

bool conv_tile(int B, int H, int W, int* bw, int* bh, int* bb)
{
    // a 128-pixel tile must be whole rows of whole images, in pixel order
    if (W >= kBM) {
        if (W % kBM) return false;
        *bw = kBM;
        *bh = *bb = 1;
        return true;
    }
    if (kBM % W) return false;
    *bw = W;
    const int rows = kBM / W;
    if (H >= rows) {
        if (H % rows) return false;
        *bh = rows;
        *bb = 1;
        return true;
    }
    if (rows % H) return false;
    *bh = H;
    *bb = rows / H;
    (void)B;
    return true;
}

bool conv3x3_supported(int B, int H, int W, int C)
{
    int bw, bh, bb;
    return C % 32 == 0 && conv_tile(B, H, W, &bw, &bh, &bb);
}

cudaError_t conv3x3_bf16(const void* X, int B, int H, int W, int C, int cpitch, const void* Wm, int ldw, void* D,
                         int ldd, const float* bias, int N, bool out_bf16, bool relu, cudaStream_t s,
                         const void* mask, int mpitch)
{
    const int bk = C % 64 == 0 ? 64 : C % 32 == 0 ? 32 : 0;
    int bw, bh, bb;
    if (!bk || !conv_tile(B, H, W, &bw, &bh, &bb)) return cudaErrorNotSupported;
    if (mask && !mask_ok(mask, mpitch, out_bf16, N)) return cudaErrorInvalidValue;
    if (N < 8 || N % 8 || cpitch % 8 || C > cpitch || ldw % 8 || ldw < 9 * C || ldd % 8 || N > ldd)
        return cudaErrorInvalidValue;
    if (((uintptr_t)X | (uintptr_t)Wm | (uintptr_t)D) & 15) return cudaErrorInvalidValue;
    const int bn = bn_for(N);
    // rows of at least 256 pixels: each stage loads one box of 130 pixels of
    // an input row and serves its three taps from it
    const bool row3 = bw == kBM && W >= 2 * kBM && bn <= 64;
    CUtensorMap ta, tb;
    cudaError_t e = make_map_4d(&ta, X, B, H, W, C, cpitch, row3 ? kBM + 2 : bw, bh, bb, bk);
    if (e == cudaSuccess) e = make_map(&tb, Wm, N, 9 * C, ldw, bn, bk);
    if (e != cudaSuccess) return e;
    ConvGeo geo;
    geo.W = W;
    geo.H = H;
    geo.C = C;
    geo.cblocks = C / bk;
    geo.row3 = row3 ? 1 : 0;
    const int M = B * H * W, K = 9 * C;
    ShuffleGeo sh;
    sh.mask = (const __nv_bfloat16*)mask;
    sh.mpitch = mpitch;
    return bk == 64 ? dispatch<64, true>(bn, out_bf16, ta, tb, D, bias, M, N, K, ldd, relu ? 1 : 0, 1, 1 << 30, geo,
                                         sh, s)
                    : dispatch<32, true>(bn, out_bf16, ta, tb, D, bias, M, N, K, ldd, relu ? 1 : 0, 1, 1 << 30, geo,
                                         sh, s);
}

cudaError_t upconv2x2_bf16(const void* X, int lda, const void* Wm, int ldw, void* Y, int ypitch, int c0,
                           const float* bias, int B, int Hl, int Wl, int cin, int c, cudaStream_t s)
{
    const int N = 4 * c, M = B * Hl * Wl, K = cin;
    if (c % 16 || lda % 8 || ldw % 8 || ypitch % 8 || K > lda || K > ldw || c0 + c > ypitch) return cudaErrorInvalidValue;
    if (((uintptr_t)X | (uintptr_t)Wm | (uintptr_t)Y) & 15) return cudaErrorInvalidValue;
    const int bn = bn_for(N);
    CUtensorMap ta, tb;
    cudaError_t e = make_map(&ta, X, M, K, lda, kBM, kBK);
    if (e == cudaSuccess) e = make_map(&tb, Wm, N, K, ldw, bn, kBK);
    if (e != cudaSuccess) return e;
    ShuffleGeo sh;
    sh.Wl = Wl;
    sh.Hl = Hl;
    sh.c = c;
    sh.c0 = c0;
    return dispatch<kBK, false>(bn, true, ta, tb, Y, bias, M, N, K, ypitch, 0, 1, 1 << 30, ConvGeo{}, sh, s);
}

cudaError_t set_operand_wait(unsigned long long ns)
{
    return cudaMemcpyToSymbol(g_operand_wait_ns, &ns, sizeof(ns));
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
