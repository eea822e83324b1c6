// Memory-bound layers of the surrogate network (NHWC, BF16 activations,
// FP32 where values are summed).  Every kernel here is a plain grid over its
// output elements; the contractions go to the tensor-core GEMM.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "nn_layers.h"

namespace nn {

namespace {

using bf16 = __nv_bfloat16;

__device__ __forceinline__ float bf(bf16 v) { return __bfloat162float(v); }

inline unsigned blocks(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// A[(b, y, x)][(ky, kx, c)] = X[b, y + ky - 1, x + kx - 1, c] (zero outside):
// one thread per (pixel, tap, 8-channel group), 16-byte moves.
__global__ void k_im2col3x3(const bf16* __restrict__ X, int B, int H, int W, int C, int cpitch, bf16* __restrict__ A)
{
    const int groups = C / 8;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long n = (long long)B * H * W * 9 * groups;
    if (i >= n) return;
    const int g = (int)(i % groups);
    long long r = i / groups;
    const int tap = (int)(r % 9);
    const long long p = r / 9;
    const int x = (int)(p % W), y = (int)((p / W) % H), b = (int)(p / ((long long)W * H));
    const int yy = y + tap / 3 - 1, xx = x + tap % 3 - 1;
    uint4 v = make_uint4(0, 0, 0, 0);
    if (yy >= 0 && yy < H && xx >= 0 && xx < W)
        v = *(const uint4*)(X + (((long long)b * H + yy) * W + xx) * cpitch + g * 8);
    *(uint4*)(A + p * (9LL * C) + tap * C + g * 8) = v;
}

// dX[b, y, x, c] = sum over taps of dA[(b, y - ky + 1, x - kx + 1)][(ky, kx, c)].
__global__ void k_col2im3x3(const float* __restrict__ dA, int B, int H, int W, int C, float* __restrict__ dX,
                            int cpitch)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long n = (long long)B * H * W * C;
    if (i >= n) return;
    const int c = (int)(i % C);
    const long long p = i / C;
    const int x = (int)(p % W), y = (int)((p / W) % H), b = (int)(p / ((long long)W * H));
    float acc = 0.0f;
#pragma unroll
    for (int ky = 0; ky < 3; ++ky)
#pragma unroll
        for (int kx = 0; kx < 3; ++kx) {
            const int yo = y - ky + 1, xo = x - kx + 1;
            if (yo < 0 || yo >= H || xo < 0 || xo >= W) continue;
            acc += dA[(((long long)b * H + yo) * W + xo) * (9LL * C) + (ky * 3 + kx) * C + c];
        }
    dX[p * cpitch + c] = acc;
}

// g <- g * (y > 0) on a [rows][C] slice of pitch `pitch` (BF16 or FP32 g).
template <class G>
__global__ void k_relu_bwd(G* __restrict__ g, int gpitch, const bf16* __restrict__ y, int ypitch, long long rows, int C)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= rows * C) return;
    const long long r = i / C;
    const int c = (int)(i - r * C);
    if (!(bf(y[r * ypitch + c]) > 0.0f)) g[r * gpitch + c] = (G)0.0f;
}

// Transposed gather for weight gradients:
//   AT[t * C + c][p] = X[pixel p shifted by tap t][c]   (zero outside)
// with taps 9 (the 3 x 3 neighbourhood, t = ky * 3 + kx), 3 (the middle row
// of it, dy = 0 and dx = -1, 0, 1: tap rows kx * C + c) or 1 (no shift: a
// plain transpose of [P][C] with pitch).  One CTA moves a 64-pixel x
// 64-channel block through shared memory: 16-byte reads along channels (8
// threads per pixel row), then each thread takes a pair of channels for 8
// pixels, reading 32-bit words, splitting them with byte permutes and writing
// 16 bytes along pixels per channel (8 threads per 128-byte line).  The 16-byte
// chunks of tile row r sit at chunk ^ ((r / 8) % 8), so the eight pixel
// groups a warp reads at once fall in different banks.  Each pixel's source
// offset is computed once per CTA.  C and the pitches are multiples of 8; P
// and the AT pitch multiples of 8; P < 2^31.
__global__ void __launch_bounds__(256) k_gatherT(const bf16* __restrict__ X, int B, int H, int W, int C, int cpitch,
                                                 int taps, bf16* __restrict__ AT, long long atpitch)
{
    __shared__ uint4 tile[64][8];   // [pixel][16-byte chunk of 8 channels], chunks permuted per row group
    __shared__ long long src[64];   // element offset of each pixel's shifted source, -1 outside the image
    const int P = B * H * W;
    const int p0 = blockIdx.x * 64;
    const int cblk = blockIdx.y;                 // 64-channel block within (tap, channel)
    const int cpb = (C + 63) / 64;                // channel blocks per tap
    const int t = taps == 9 ? cblk / cpb : taps == 3 ? 3 + cblk / cpb : 4;  // taps 3-5: the middle row; 4: centre
    const int c0 = (cblk % cpb) * 64;
    const int dy = t / 3 - 1, dx = t % 3 - 1;
    if (threadIdx.x < 64) {
        const int p = p0 + threadIdx.x;
        long long off = -1;
        if (p < P) {
            const int x = p % W, r = p / W, y = r % H, b = r / H;
            const int xx = x + dx, yy = y + dy;
            if (xx >= 0 && xx < W && yy >= 0 && yy < H) off = (((long long)b * H + yy) * W + xx) * cpitch;
        }
        src[threadIdx.x] = off;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < 64 * 8; k += 256) {
        const int pi = k >> 3, g = k & 7;
        const int c = c0 + g * 8;
        uint4 v = make_uint4(0, 0, 0, 0);
        const long long off = src[pi];
        if (off >= 0 && c < C) v = *(const uint4*)(X + off + c);
        tile[pi][g ^ ((pi >> 3) & 7)] = v;
    }
    __syncthreads();
    // lane: pixel group g (8 pixels) and one of four channel pairs; warp w
    // holds channel pairs 4w .. 4w + 3 of the block
    const int lane = threadIdx.x & 31, g = lane & 7;
    const int cp = (threadIdx.x >> 5) * 4 + (lane >> 3);  // channel pair 0..31
    const int c = c0 + 2 * cp;
    const int p = p0 + g * 8;
    if (c >= C || p >= P) return;
    uint32_t w[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const uint32_t* row = (const uint32_t*)&tile[g * 8 + j][0];
        w[j] = row[(((cp >> 2) ^ g) << 2) + (cp & 3)];
    }
    uint4 lo, hi;  // channel c and c + 1, pixels p .. p + 7
    lo.x = __byte_perm(w[0], w[1], 0x5410);
    lo.y = __byte_perm(w[2], w[3], 0x5410);
    lo.z = __byte_perm(w[4], w[5], 0x5410);
    lo.w = __byte_perm(w[6], w[7], 0x5410);
    hi.x = __byte_perm(w[0], w[1], 0x7632);
    hi.y = __byte_perm(w[2], w[3], 0x7632);
    hi.z = __byte_perm(w[4], w[5], 0x7632);
    hi.w = __byte_perm(w[6], w[7], 0x7632);
    const long long row = (long long)(taps == 1 ? c : (cblk / cpb) * C + c);
    *(uint4*)(AT + row * atpitch + p) = lo;
    *(uint4*)(AT + (row + 1) * atpitch + p) = hi;
}

// Shifted transposed copies from one staged read of the input: the CTA
// stages pixels p0 - 1 .. p0 + 64 of a 64-channel block, in NR image rows
// (NR = 1: the middle row, taps 3 .. 5 written as rows kx * C + c; NR = 3:
// the rows above, at and below, all nine taps, rows (3 ky + kx) * C + c), and
// writes every tap's copy from that tile.  W is a multiple of 8, so the 8
// pixels a thread writes lie in one image row: only a row's first pixel
// (dx = -1) or last (dx = +1), or a whole group in the first (dy = -1) or last
// (dy = +1) image row, has its source outside the image.
template <int NR>
__global__ void __launch_bounds__(256) k_gather_rows(const bf16* __restrict__ X, int P, int H, int W, int C,
                                                     int cpitch, bf16* __restrict__ AT, long long atpitch)
{
    __shared__ uint4 tile[NR * 66][8];  // [row * 66 + pixel - (p0 - 1)][16-byte chunk], chunks permuted
    const int p0 = blockIdx.x * 64;
    const int c0 = blockIdx.y * 64;
    for (int k = threadIdx.x; k < NR * 66 * 8; k += 256) {
        const int ti = k >> 3, g = k & 7;
        const int rr = ti / 66, pi = ti - rr * 66;
        const long long q = (long long)p0 - 1 + pi + (long long)(NR == 3 ? rr - 1 : 0) * W;
        const int c = c0 + g * 8;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (q >= 0 && q < P && c < C) v = *(const uint4*)(X + q * cpitch + c);
        tile[ti][g ^ ((pi >> 3) & 7)] = v;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, g = lane & 7;
    const int cp = (threadIdx.x >> 5) * 4 + (lane >> 3);  // channel pair 0..31
    const int c = c0 + 2 * cp;
    const int p = p0 + g * 8;
    if (c >= C || p >= P) return;
    const int x = p % W;  // of the first of the 8 pixels
    const int y = (p / W) % H;
#pragma unroll
    for (int rr = 0; rr < NR; ++rr) {
        const bool row_out = NR == 3 && ((rr == 0 && y == 0) || (rr == 2 && y == H - 1));
#pragma unroll
        for (int kx = 0; kx < 3; ++kx) {
            uint32_t w[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int pi = g * 8 + j + kx;  // source pixel p + j + kx - 1 of row rr
                const uint32_t* row = (const uint32_t*)&tile[rr * 66 + pi][0];
                w[j] = row_out ? 0u : row[(((cp >> 2) ^ ((pi >> 3) & 7)) << 2) + (cp & 3)];
            }
            if (kx == 0 && x == 0) w[0] = 0;
            if (kx == 2 && x + 7 == W - 1) w[7] = 0;
            uint4 lo, hi;
            lo.x = __byte_perm(w[0], w[1], 0x5410);
            lo.y = __byte_perm(w[2], w[3], 0x5410);
            lo.z = __byte_perm(w[4], w[5], 0x5410);
            lo.w = __byte_perm(w[6], w[7], 0x5410);
            hi.x = __byte_perm(w[0], w[1], 0x7632);
            hi.y = __byte_perm(w[2], w[3], 0x7632);
            hi.z = __byte_perm(w[4], w[5], 0x7632);
            hi.w = __byte_perm(w[6], w[7], 0x7632);
            const long long r = (long long)(NR == 3 ? 3 * rr + kx : kx) * C + c;
            *(uint4*)(AT + r * atpitch + p) = lo;
            *(uint4*)(AT + (r + 1) * atpitch + p) = hi;
        }
    }
}

// out[r][c] = BF16(y[r][c] > 0 ? g[r][c] : 0): the ReLU mask of an FP32
// gradient and its rounding for the next GEMM, in one pass.
__global__ void k_mask_cast(const float* __restrict__ g, int gpitch, const bf16* __restrict__ y, int ypitch,
                            long long rows, int C, bf16* __restrict__ out, int opitch)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= rows * C) return;
    const long long r = i / C;
    const int c = (int)(i - r * C);
    const float v = bf(y[r * ypitch + c]) > 0.0f ? g[r * gpitch + c] : 0.0f;
    out[r * opitch + c] = __float2bfloat16(v);
}

// The same, eight channels per thread (C, the pitches and the pointers
// aligned to 8 elements; rows * C / 8 < 2^31): 32-byte FP32 and 16-byte BF16
// accesses, 32-bit index arithmetic.
__global__ void k_mask_cast8(const float* __restrict__ g, int gpitch, const bf16* __restrict__ y, int ypitch,
                             int groups, int cg, bf16* __restrict__ out, int opitch)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= groups) return;
    const int r = i / cg, c = (i - r * cg) * 8;
    const float4 g0 = *(const float4*)(g + (long long)r * gpitch + c);
    const float4 g1 = *(const float4*)(g + (long long)r * gpitch + c + 4);
    const uint4 yv = *(const uint4*)(y + (long long)r * ypitch + c);
    const bf16* ys = (const bf16*)&yv;
    const float gv[8] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
    __align__(16) bf16 o[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) o[j] = __float2bfloat16(bf(ys[j]) > 0.0f ? gv[j] : 0.0f);
    *(uint4*)(out + (long long)r * opitch + c) = *(const uint4*)o;
}

// Out[c][r] = In[r][c] (BF16), 32 x 32 tiles through shared memory.
__global__ void k_transpose(const bf16* __restrict__ in, int rows, int cols, int ipitch, bf16* __restrict__ out,
                            int opitch)
{
    __shared__ bf16 t[32][33];
    const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;  // rows on x: up to 2^31 blocks
    for (int k = threadIdx.y; k < 32; k += 8) {
        const int r = r0 + k, c = c0 + threadIdx.x;
        t[k][threadIdx.x] = (r < rows && c < cols) ? in[(long long)r * ipitch + c] : __float2bfloat16(0.0f);
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += 8) {
        const int c = c0 + k, r = r0 + threadIdx.x;
        if (c < cols && r < rows) out[(long long)c * opitch + r] = t[threadIdx.x][k];
    }
}

__global__ void k_maxpool_fwd(const bf16* __restrict__ X, int B, int H, int W, int C, int xpitch, bf16* __restrict__ Y)
{
    const int Ho = H / 2, Wo = W / 2;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)B * Ho * Wo * C) return;
    const int c = (int)(i % C);
    const long long p = i / C;
    const int x = (int)(p % Wo), y = (int)((p / Wo) % Ho), b = (int)(p / ((long long)Wo * Ho));
    const long long base = (((long long)b * H + 2 * y) * W + 2 * x) * xpitch + c;
    float m = bf(X[base]);
    m = fmaxf(m, bf(X[base + xpitch]));
    m = fmaxf(m, bf(X[base + (long long)W * xpitch]));
    m = fmaxf(m, bf(X[base + (long long)W * xpitch + xpitch]));
    Y[p * C + c] = __float2bfloat16(m);
}

// The same, eight channels per thread with 16-byte loads and stores (C and
// xpitch multiples of 8, 16-byte aligned bases).
__global__ void k_maxpool_fwd8(const bf16* __restrict__ X, int B, int H, int W, int C, int xpitch,
                               bf16* __restrict__ Y)
{
    const int Ho = H / 2, Wo = W / 2, G = C / 8;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)B * Ho * Wo * G) return;
    const int g = (int)(i % G);
    const long long p = i / G;
    const int x = (int)(p % Wo), y = (int)((p / Wo) % Ho), b = (int)(p / ((long long)Wo * Ho));
    const bf16* base = X + (((long long)b * H + 2 * y) * W + 2 * x) * xpitch + g * 8;
    const uint4 q[4] = {*(const uint4*)base, *(const uint4*)(base + xpitch), *(const uint4*)(base + (long long)W * xpitch),
                        *(const uint4*)(base + (long long)W * xpitch + xpitch)};
    __nv_bfloat162 r[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        float2 m = __bfloat1622float2(((const __nv_bfloat162*)&q[0])[j]);
#pragma unroll
        for (int k = 1; k < 4; ++k) {
            const float2 v = __bfloat1622float2(((const __nv_bfloat162*)&q[k])[j]);
            m.x = fmaxf(m.x, v.x);
            m.y = fmaxf(m.y, v.y);
        }
        r[j] = __floats2bfloat162_rn(m.x, m.y);
    }
    *(uint4*)(Y + p * C + g * 8) = *(const uint4*)r;
}

// The gradient goes to the first maximum of each 2 x 2 window (row-major order).
__global__ void k_maxpool_bwd(const bf16* __restrict__ X, int B, int H, int W, int C, int xpitch,
                              const float* __restrict__ dY, float* __restrict__ dX, int dpitch)
{
    const int Ho = H / 2, Wo = W / 2;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)B * Ho * Wo * C) return;
    const int c = (int)(i % C);
    const long long p = i / C;
    const int x = (int)(p % Wo), y = (int)((p / Wo) % Ho), b = (int)(p / ((long long)Wo * Ho));
    long long off[4];
    float v[4];
    for (int k = 0; k < 4; ++k) {
        const long long q = ((long long)b * H + 2 * y + k / 2) * W + 2 * x + k % 2;
        off[k] = q;
        v[k] = bf(X[q * xpitch + c]);
    }
    int arg = 0;
    for (int k = 1; k < 4; ++k)
        if (v[k] > v[arg]) arg = k;
    const float g = dY[p * C + c];
    for (int k = 0; k < 4; ++k) dX[off[k] * dpitch + c] += (k == arg) ? g : 0.0f;
}

// The same for C and xpitch multiples of 8 and dpitch a multiple of 4:
// threadIdx.x takes 8 channels of the output pixel blockIdx.x * blockDim.y +
// threadIdx.y, reading each window position's 8 inputs in one 16-byte load and
// adding the gradient to its 8 dX values with two 16-byte read-modify-writes
// (each input position belongs to one window, so no two threads meet).
__global__ void k_maxpool_bwd8(const bf16* __restrict__ X, int B, int H, int W, int C, int xpitch,
                               const float* __restrict__ dY, float* __restrict__ dX, int dpitch)
{
    const int Ho = H / 2, Wo = W / 2;
    const int c = 8 * threadIdx.x;
    const long long p = (long long)blockIdx.x * blockDim.y + threadIdx.y;
    if (p >= (long long)B * Ho * Wo) return;
    const int x = (int)(p % Wo);
    const long long r = p / Wo;
    const int y = (int)(r % Ho), b = (int)(r / Ho);
    float v[4][8];
    long long off[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        off[k] = ((long long)b * H + 2 * y + k / 2) * W + 2 * x + k % 2;
        const uint4 q = *(const uint4*)(X + off[k] * xpitch + c);
        const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            v[k][2 * j] = __uint_as_float(w[j] << 16);
            v[k][2 * j + 1] = __uint_as_float(w[j] & 0xffff0000u);
        }
    }
    const float4 g0 = *(const float4*)(dY + p * C + c), g1 = *(const float4*)(dY + p * C + c + 4);
    const float g[8] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
    int arg[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        arg[j] = 0;
#pragma unroll
        for (int k = 1; k < 4; ++k)
            if (v[k][j] > v[arg[j]][j]) arg[j] = k;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        float4* d = (float4*)(dX + off[k] * dpitch + c);
        float4 a = d[0], e = d[1];
        a.x += arg[0] == k ? g[0] : 0.0f;
        a.y += arg[1] == k ? g[1] : 0.0f;
        a.z += arg[2] == k ? g[2] : 0.0f;
        a.w += arg[3] == k ? g[3] : 0.0f;
        e.x += arg[4] == k ? g[4] : 0.0f;
        e.y += arg[5] == k ? g[5] : 0.0f;
        e.z += arg[6] == k ? g[6] : 0.0f;
        e.w += arg[7] == k ? g[7] : 0.0f;
        d[0] = a;
        d[1] = e;
    }
}

// U[(b, y, x)][(dy, dx, c)] (2 x 2 up-convolution output) -> Y[b, 2y + dy, 2x + dx, c0 + c].
__global__ void k_shuffle_fwd(const bf16* __restrict__ U, int B, int H, int W, int C, bf16* __restrict__ Y,
                              int ypitch, int c0)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)B * H * W * 4 * C) return;
    const int c = (int)(i % C);
    long long r = i / C;
    const int sub = (int)(r % 4);
    const long long p = r / 4;
    const int x = (int)(p % W), y = (int)((p / W) % H), b = (int)(p / ((long long)W * H));
    const long long q = ((long long)b * 2 * H + 2 * y + sub / 2) * (2 * W) + 2 * x + sub % 2;
    Y[q * ypitch + c0 + c] = U[i];
}

// Inverse gather for the gradient: dU[(b, y, x)][(dy, dx, c)] = dY[b, 2y + dy, 2x + dx, c0 + c].
template <class G>
__global__ void k_shuffle_bwd(const G* __restrict__ dY, int ypitch, int c0, int B, int H, int W, int C,
                              bf16* __restrict__ dU)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)B * H * W * 4 * C) return;
    const int c = (int)(i % C);
    long long r = i / C;
    const int sub = (int)(r % 4);
    const long long p = r / 4;
    const int x = (int)(p % W), y = (int)((p / W) % H), b = (int)(p / ((long long)W * H));
    const long long q = ((long long)b * 2 * H + 2 * y + sub / 2) * (2 * W) + 2 * x + sub % 2;
    dU[i] = __float2bfloat16((float)dY[q * ypitch + c0 + c]);
}

// The same, eight channels per thread (C, c0 and the pitch multiples of 8,
// 16-byte aligned pointers; fewer than 2^31 groups): one index computation
// per eight values, 16- or 32-byte loads, a 16-byte store.
template <class G>
__global__ void k_shuffle_bwd8(const G* __restrict__ dY, int ypitch, int c0, int H, int W, int cg, int groups,
                               bf16* __restrict__ dU)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= groups) return;
    const int c = (i % cg) * 8, r = i / cg;
    const int sub = r & 3, p = r >> 2;
    const int x = p % W, t = p / W, y = t % H, b = t / H;
    const long long q = ((long long)b * 2 * H + 2 * y + (sub >> 1)) * (2 * W) + 2 * x + (sub & 1);
    const G* src = dY + q * ypitch + c0 + c;
    __align__(16) bf16 o[8];
    if constexpr (sizeof(G) == 4) {
        const float4 a = *(const float4*)src, d = *(const float4*)(src + 4);
        const float v[8] = {a.x, a.y, a.z, a.w, d.x, d.y, d.z, d.w};
#pragma unroll
        for (int j = 0; j < 8; ++j) o[j] = __float2bfloat16(v[j]);
    } else {
        *(uint4*)o = *(const uint4*)src;
    }
    *(uint4*)(dU + (long long)i * 8) = *(const uint4*)o;
}

// Output projection (1 x 1 convolution to O <= 8 channels) with residual:
// Y[p][o] = R[p][o] + b[o] + sum_c X[p][c] Wt[o][c].
__global__ void k_proj_fwd(const bf16* __restrict__ X, int P, int C, int xpitch, const float* __restrict__ Wt,
                           const float* __restrict__ bias, int O, const float* __restrict__ R, float* __restrict__ Y)
{
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= P) return;
    for (int o = 0; o < O; ++o) {
        float acc = bias[o] + (R ? R[p * O + o] : 0.0f);
        for (int c = 0; c < C; ++c) acc += bf(X[p * xpitch + c]) * Wt[o * C + c];
        Y[p * O + o] = acc;
    }
}

// The same with 16-byte loads of X (C and xpitch multiples of 8) and the
// weights staged in shared memory: one thread per pixel.
__global__ void k_proj_fwd_vec(const bf16* __restrict__ X, int P, int C, int xpitch, const float* __restrict__ Wt,
                               const float* __restrict__ bias, int O, const float* __restrict__ R,
                               float* __restrict__ Y)
{
    extern __shared__ float wsh[];  // O * C weights, then O biases
    for (int i = threadIdx.x; i < O * C; i += blockDim.x) wsh[i] = Wt[i];
    for (int i = threadIdx.x; i < O; i += blockDim.x) wsh[O * C + i] = bias[i];
    __syncthreads();
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= P) return;
    float acc[8];
#pragma unroll
    for (int o = 0; o < 8; ++o) acc[o] = o < O ? wsh[O * C + o] + (R ? R[p * O + o] : 0.0f) : 0.0f;
    const uint4* xp = (const uint4*)(X + p * xpitch);
    for (int c8 = 0; c8 < C / 8; ++c8) {
        const uint4 q = xp[c8];
        const __nv_bfloat162* h = (const __nv_bfloat162*)&q;
        float xv[8];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float2 f = __bfloat1622float2(h[j]);
            xv[2 * j] = f.x;
            xv[2 * j + 1] = f.y;
        }
#pragma unroll
        for (int o = 0; o < 8; ++o) {
            if (o >= O) break;
            const float* w = wsh + o * C + c8 * 8;
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[o] += xv[j] * w[j];
        }
    }
    for (int o = 0; o < O; ++o) Y[p * O + o] = acc[o];
}

// dX[p][c] = sum_o dY[p][o] Wt[o][c] (FP32, pitch dpitch).
__global__ void k_proj_bwd_x(const float* __restrict__ dY, int P, int O, const float* __restrict__ Wt, int C,
                             float* __restrict__ dX, int dpitch)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)P * C) return;
    const long long p = i / C;
    const int c = (int)(i - p * C);
    float acc = 0.0f;
    for (int o = 0; o < O; ++o) acc += dY[p * O + o] * Wt[o * C + c];
    dX[p * dpitch + c] = acc;
}

// Per-block partial sums of dW[o][c] = sum_p dY[p][o] X[p][c] and db[o] =
// sum_p dY[p][o]: block b covers pixels [b * chunk, (b + 1) * chunk).
__global__ void k_proj_bwd_w(const float* __restrict__ dY, const bf16* __restrict__ X, int P, int C, int xpitch, int O,
                             int chunk, float* __restrict__ part)
{
    const int slots = O * (C + 1);
    const int p0 = blockIdx.x * chunk, p1 = min(P, p0 + chunk);
    for (int s = threadIdx.x; s < slots; s += blockDim.x) {
        const int o = s / (C + 1), c = s % (C + 1);
        float acc = 0.0f;
        for (int p = p0; p < p1; ++p) acc += dY[(long long)p * O + o] * (c < C ? bf(X[(long long)p * xpitch + c]) : 1.0f);
        part[(long long)blockIdx.x * slots + s] = acc;
    }
}

// The same sums for C <= 64 and O <= 8, warp-parallel: the block's 8 warps
// take every 8th pixel of its chunk, lane l the channels l and l + 32 of
// all O outputs (lane 0 also the bias), and the warps' sums combine in a
// fixed order through shared memory into the block's row of partials.
__global__ void __launch_bounds__(256) k_proj_bwd_w_warps(const float* __restrict__ dY, const bf16* __restrict__ X,
                                                          int P, int C, int xpitch, int O, int chunk,
                                                          float* __restrict__ part)
{
    __shared__ float sm[8][8 * 65];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int slots = O * (C + 1);
    const int p0 = blockIdx.x * chunk, p1 = min(P, p0 + chunk);
    float acc[2][8], accb[8];
#pragma unroll
    for (int o = 0; o < 8; ++o) acc[0][o] = acc[1][o] = accb[o] = 0.0f;
    for (int p = p0 + warp; p < p1; p += 8) {
        float d[8];
#pragma unroll
        for (int o = 0; o < 8; ++o) d[o] = o < O ? dY[(long long)p * O + o] : 0.0f;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int c = lane + 32 * k;
            const float x = c < C ? bf(X[(long long)p * xpitch + c]) : 0.0f;
#pragma unroll
            for (int o = 0; o < 8; ++o) acc[k][o] += d[o] * x;
        }
#pragma unroll
        for (int o = 0; o < 8; ++o) accb[o] += d[o];
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int c = lane + 32 * k;
        if (c < C)
            for (int o = 0; o < O; ++o) sm[warp][o * (C + 1) + c] = acc[k][o];
    }
    if (lane == 0)
        for (int o = 0; o < O; ++o) sm[warp][o * (C + 1) + C] = accb[o];
    __syncthreads();
    for (int s = threadIdx.x; s < slots; s += 256) {
        float v = 0.0f;
        for (int w = 0; w < 8; ++w) v += sm[w][s];
        part[(long long)blockIdx.x * slots + s] = v;
    }
}

// dX[p][c] = sum_o dY[p][o] Wt[o][c] for C a multiple of 4: threadIdx.x takes
// four channels, threadIdx.y a pixel, so that every store is 16 bytes and no
// thread divides.
__global__ void k_proj_bwd_x4(const float* __restrict__ dY, int P, int O, const float* __restrict__ Wt, int C,
                              float* __restrict__ dX, int dpitch)
{
    const int c = 4 * threadIdx.x;
    const long long p = (long long)blockIdx.x * blockDim.y + threadIdx.y;
    if (p >= P) return;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int o = 0; o < O; ++o) {
        const float d = dY[p * O + o];
        const float4 w = *(const float4*)(Wt + o * C + c);
        acc.x += d * w.x;
        acc.y += d * w.y;
        acc.z += d * w.z;
        acc.w += d * w.w;
    }
    *(float4*)(dX + p * dpitch + c) = acc;
}

// Per-block partial sums of dW[o][c] = sum_p dY[p][o] X[p][c] and db[o] =
// sum_p dY[p][o] for C = 8 G with G in {1, 2, 4, 8}: thread t adds channels
// 8 (t % G) .. + 7 of every (256 / G)-th pixel of the block's chunk from one
// 16-byte load; the threads of one channel group are added by shuffles within
// each warp and then over the warps through shared memory, in a fixed order.
template <int O>
__global__ void __launch_bounds__(256) k_proj_bwd_w8(const float* __restrict__ dY, const bf16* __restrict__ X, int P,
                                                     int C, int xpitch, int chunk, float* __restrict__ part)
{
    __shared__ float sm[8][8][O * 9];  // [warp][group][o * 9 + k], k = 8: the bias
    const int G = C >> 3, lanes = 256 / G;
    const int cg = threadIdx.x % G, pl = threadIdx.x / G;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int p0 = blockIdx.x * chunk, p1 = min(P, p0 + chunk);
    float acc[O][9];
#pragma unroll
    for (int o = 0; o < O; ++o)
#pragma unroll
        for (int k = 0; k < 9; ++k) acc[o][k] = 0.0f;
    for (int p = p0 + pl; p < p1; p += lanes) {
        const uint4 v = *(const uint4*)(X + (long long)p * xpitch + 8 * cg);
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
        float x[8];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            x[2 * k] = __uint_as_float(w[k] << 16);
            x[2 * k + 1] = __uint_as_float(w[k] & 0xffff0000u);
        }
#pragma unroll
        for (int o = 0; o < O; ++o) {
            const float d = dY[(long long)p * O + o];
#pragma unroll
            for (int k = 0; k < 8; ++k) acc[o][k] += d * x[k];
            acc[o][8] += d;
        }
    }
    // lanes with the same group differ in the bits above log2(G)
#pragma unroll
    for (int o = 0; o < O; ++o)
#pragma unroll
        for (int k = 0; k < 9; ++k)
            for (int off = G; off < 32; off <<= 1) acc[o][k] += __shfl_xor_sync(0xffffffffu, acc[o][k], off);
    if (lane < G)
#pragma unroll
        for (int o = 0; o < O; ++o)
#pragma unroll
            for (int k = 0; k < 9; ++k) sm[warp][lane][o * 9 + k] = acc[o][k];
    __syncthreads();
    const int slots = O * (C + 1);
    for (int s = threadIdx.x; s < slots; s += 256) {
        const int o = s / (C + 1), c = s - o * (C + 1);
        // the bias (c == C) is the same sum in every group: take group 0's
        const int g = c < C ? c >> 3 : 0, k = c < C ? c & 7 : 8;
        float v = 0.0f;
        for (int w = 0; w < 8; ++w) v += sm[w][g][o * 9 + k];
        part[(long long)blockIdx.x * slots + s] = v;
    }
}

// Weights of the transposed 3 x 3 convolution that carries the gradient back
// to the input: Wf[ci][t * cout + co] = W[co][(8 - t) * cin + ci] (the
// kernel rotated by 180 degrees, input and output channels swapped).
__global__ void k_flip3x3(const bf16* __restrict__ W, int cout, int cin, bf16* __restrict__ Wf)
{
    // one thread per output element, so that the writes are contiguous; the
    // scattered reads come from a kernel small enough to stay in L2
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)cout * 9 * cin) return;
    const int co = (int)(i % cout);
    const long long r = i / cout;
    const int tf = (int)(r % 9), ci = (int)(r / 9);
    Wf[i] = W[((long long)co * 9 + (8 - tf)) * cin + ci];
}

// Every kernel of a network in one launch: element i belongs to the last job
// whose start is <= i (at most a few tens of jobs, scanned in order).
__global__ void k_flip3x3_many(const FlipJob* __restrict__ jobs, int njobs, long long total)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= total) return;
    int j = 0;
    while (j + 1 < njobs && jobs[j + 1].start <= i) ++j;
    const FlipJob jb = jobs[j];
    const long long k = i - jb.start;
    const int co = (int)(k % jb.cout);
    const long long r = k / jb.cout;
    const int tf = (int)(r % 9), ci = (int)(r / 9);
    ((bf16*)jb.Wf)[k] = ((const bf16*)jb.W)[((long long)co * 9 + (8 - tf)) * jb.cin + ci];
}

// Wp[co][t * cin_pad + ci] = W[co][t * cin + ci] for ci < cin, else 0: the
// kernel of a convolution whose input carries cin_pad channels, the extra ones zero.
__global__ void k_pad_conv3x3(const bf16* __restrict__ W, int cout, int cin, int cin_pad, bf16* __restrict__ Wp)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)cout * 9 * cin_pad) return;
    const int ci = (int)(i % cin_pad);
    const long long r = i / cin_pad;
    const int t = (int)(r % 9), co = (int)(r / 9);
    Wp[i] = ci < cin ? W[((long long)co * 9 + t) * cin + ci] : __float2bfloat16(0.0f);
}

// Column sums of a [rows][C] matrix (pitch), as per-block partials over row chunks.
template <class G>
__global__ void k_colsum_part(const G* __restrict__ g, long long rows, int C, int pitch, int chunk,
                              float* __restrict__ part)
{
    // the block's 128 threads split into 128 / L row lanes of L = min(C, 128)
    // column threads; each column's row lanes are then added in shared memory
    __shared__ float sm[128];
    const int L = C < 128 ? C : 128;
    const int lanes = 128 / L;
    const int cl = threadIdx.x % L, rl = threadIdx.x / L;
    const long long r0 = (long long)blockIdx.x * chunk;
    const long long r1 = r0 + chunk < rows ? r0 + chunk : rows;
    for (int cb = 0; cb < C; cb += L) {
        const int c = cb + cl;
        float acc = 0.0f;
        if (rl < lanes && c < C)
            for (long long r = r0 + rl; r < r1; r += lanes) acc += (float)g[r * pitch + c];
        sm[threadIdx.x] = acc;
        __syncthreads();
        if (threadIdx.x < L && cb + threadIdx.x < C) {
            float v = 0.0f;
            for (int k = 0; k < lanes; ++k) v += sm[k * L + threadIdx.x];
            part[(long long)blockIdx.x * C + cb + threadIdx.x] = v;
        }
        __syncthreads();
    }
}

// The same partial sums for a BF16 matrix with C and the pitch multiples of 8
// and at most 1024 columns: each thread adds 8 columns of a row from one
// 16-byte load; the block's 128 threads are 128 / G row lanes of G = C / 8
// column groups, whose lanes are then added in shared memory in a fixed order.
__global__ void k_colsum_part8(const bf16* __restrict__ g, long long rows, int C, int pitch, int chunk,
                               float* __restrict__ part)
{
    __shared__ float sm[128][8];
    const int G = C >> 3;
    const int lanes = 128 / G;
    const int cg = threadIdx.x % G, rl = threadIdx.x / G;
    const long long r0 = (long long)blockIdx.x * chunk;
    const long long r1 = r0 + chunk < rows ? r0 + chunk : rows;
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (rl < lanes)
        for (long long r = r0 + rl; r < r1; r += lanes) {
            const uint4 v = *(const uint4*)(g + r * pitch + 8 * cg);
            const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                acc[2 * k] += __uint_as_float(w[k] << 16);
                acc[2 * k + 1] += __uint_as_float(w[k] & 0xffff0000u);
            }
        }
#pragma unroll
    for (int k = 0; k < 8; ++k) sm[threadIdx.x][k] = acc[k];
    __syncthreads();
    if (threadIdx.x < G) {
        float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int l = 0; l < lanes; ++l)
#pragma unroll
            for (int k = 0; k < 8; ++k) v[k] += sm[l * G + threadIdx.x][k];
#pragma unroll
        for (int k = 0; k < 8; ++k) part[(long long)blockIdx.x * C + 8 * threadIdx.x + k] = v[k];
    }
}

// dW[o][c] and db[o] from the nb partial rows of O x (C + 1) slots: one warp
// per slot, lanes over the partial rows, a shuffle tree (a fixed order).
__global__ void k_proj_sum(const float* __restrict__ part, int nb, int O, int C, float* __restrict__ dW,
                           float* __restrict__ db)
{
    const int s = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    const int slots = O * (C + 1);
    if (s >= slots) return;
    float acc = 0.0f;
    for (int b = lane; b < nb; b += 32) acc += part[(long long)b * slots + s];
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, d);
    if (lane) return;
    const int o = s / (C + 1), c = s % (C + 1);
    if (c < C)
        dW[o * C + c] = acc;
    else
        db[o] = acc;
}

// out[s] = sum over the nb partial rows: one warp per slot, lanes take
// partial rows b = lane, lane + 32, ... and a shuffle tree adds the lanes
// (a fixed order, so the result is reproducible).
__global__ void k_sum_parts(const float* __restrict__ part, int nb, int slots, float* __restrict__ out)
{
    const int s = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (s >= slots) return;
    float acc = 0.0f;
    for (int b = lane; b < nb; b += 32) acc += part[(long long)b * slots + s];
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, d);
    if (lane == 0) out[s] = acc;
}

// out[0] = the sum of part[0 .. nb): 1024 threads add strided subsets, then a
// shared-memory tree adds the threads (a fixed order, so the result is
// reproducible).
__global__ void __launch_bounds__(1024) k_sum_one(const float* __restrict__ part, int nb, float* __restrict__ out)
{
    __shared__ float sm[1024];
    float acc = 0.0f;
    for (int b = threadIdx.x; b < nb; b += 1024) acc += part[b];
    sm[threadIdx.x] = acc;
    __syncthreads();
    for (int h = 512; h > 0; h >>= 1) {
        if (threadIdx.x < h) sm[threadIdx.x] += sm[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = sm[0];
}

// Weighted squared error: d[i] = pred - target, weight w = 1 + alpha max(0,
// 1 - phi^2) with phi = x[pixel * F] the phase field of the input at the
// element's pixel (w = 1 without x); per-block partial sums of w d^2 and the
// gradient 2 w d / n.
__global__ void k_mse(const float* __restrict__ pred, const float* __restrict__ target, long long n,
                      const float* __restrict__ x, int F, float alpha, float* __restrict__ grad,
                      float* __restrict__ part)
{
    __shared__ float sm[256];
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    float d = 0.0f, w = 1.0f;
    if (i < n) {
        d = pred[i] - target[i];
        if (x) {
            const float phi = x[(i / F) * F];
            w = 1.0f + alpha * fmaxf(0.0f, 1.0f - phi * phi);
        }
        grad[i] = 2.0f * w * d / (float)n;
    }
    sm[threadIdx.x] = w * d * d;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sm[0];
}

// Adam with bias correction on FP32 master weights; writes the BF16 copy.
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       long long n, float lr, float b1, float b2, float eps, float c1, float c2,
                       bf16* __restrict__ wb)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    if (wb) wb[i] = __float2bfloat16(wi);
}

// FP32 [P][F] fields -> BF16 NHWC [P][cpitch] with (x - mean) / std per field
// and zero extra channels.
// One thread per pixel: F <= 8 fields in, cpitch BF16 channels out as
// 16-byte stores (cpitch a multiple of 8, X 16-byte aligned).
__global__ void k_pack_px(const float* __restrict__ f, long long P, int F, const float* __restrict__ mean,
                          const float* __restrict__ inv_std, bf16* __restrict__ X, int cpitch)
{
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= P) return;
    __nv_bfloat162 h[4];
    float v[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) v[c] = c < F ? (f[p * F + c] - mean[c]) * inv_std[c] : 0.0f;
#pragma unroll
    for (int j = 0; j < 4; ++j) h[j] = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
    uint4* dst = (uint4*)(X + p * cpitch);
    dst[0] = *(const uint4*)h;
    const uint4 z = make_uint4(0, 0, 0, 0);
    for (int g = 1; g < cpitch / 8; ++g) dst[g] = z;
}

// R (optional) receives the same normalised fields in FP32 [P][F].
__global__ void k_pack(const float* __restrict__ f, long long P, int F, const float* __restrict__ mean,
                       const float* __restrict__ inv_std, bf16* __restrict__ X, int cpitch, float* __restrict__ R)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= P * cpitch) return;
    const long long p = i / cpitch;
    const int c = (int)(i - p * cpitch);
    const float v = c < F ? (f[p * F + c] - mean[c]) * inv_std[c] : 0.0f;
    if (X) X[i] = __float2bfloat16(v);
    if (R && c < F) R[p * F + c] = v;
}

// FP32 [rows][C] (pitch apitch) -> BF16 [rows][C] (pitch bpitch).
__global__ void k_cast_bf16(const float* __restrict__ a, long long rows, int C, int apitch, bf16* __restrict__ b,
                            int bpitch)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= rows * C) return;
    const long long r = i / C;
    const int c = (int)(i - r * C);
    b[r * bpitch + c] = __float2bfloat16(a[r * apitch + c]);
}

// T[p][c] = (t[p][c] - x[p][c]) * inv_out[c]: the K-step increment in the
// network's output units.
__global__ void k_increment(const float* __restrict__ t, const float* __restrict__ x, long long P, int F,
                            const float* __restrict__ inv_out, float* __restrict__ T)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= P * F) return;
    T[i] = (t[i] - x[i]) * inv_out[(int)(i % F)];
}

// y[p][c] = x[p][c] + Y[p][c] / inv_out[c]; a block covers a contiguous run
// of elements, and the per-field scale comes from a shared table.
__global__ void k_add_increment(const float* __restrict__ Y, const float* __restrict__ x, long long P, int F,
                                const float* __restrict__ inv_out, float* __restrict__ y)
{
    __shared__ float so[8];
    if (threadIdx.x < F) so[threadIdx.x] = 1.0f / inv_out[threadIdx.x];
    __syncthreads();
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= P * F) return;
    y[i] = x[i] + Y[i] * so[(int)(i % F)];
}

// FP32 fields [P][F] = mean + std * Y[P][F] (undo the normalisation).
__global__ void k_unpack(const float* __restrict__ Y, long long P, int F, const float* __restrict__ mean,
                         const float* __restrict__ inv_std, float* __restrict__ f)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= P * F) return;
    const int c = (int)(i % F);
    f[i] = mean[c] + Y[i] / inv_std[c];
}

}  // namespace

cudaError_t im2col3x3(const void* X, int B, int H, int W, int C, int cpitch, void* A, cudaStream_t s)
{
    if (C % 8 || cpitch % 8) return cudaErrorInvalidValue;
    const long long n = (long long)B * H * W * 9 * (C / 8);
    k_im2col3x3<<<blocks(n), 256, 0, s>>>((const bf16*)X, B, H, W, C, cpitch, (bf16*)A);
    return cudaGetLastError();
}

cudaError_t col2im3x3(const float* dA, int B, int H, int W, int C, float* dX, int cpitch, cudaStream_t s)
{
    const long long n = (long long)B * H * W * C;
    k_col2im3x3<<<blocks(n), 256, 0, s>>>(dA, B, H, W, C, dX, cpitch);
    return cudaGetLastError();
}

cudaError_t relu_bwd(void* g, bool g_fp32, int gpitch, const void* y, int ypitch, long long rows, int C, cudaStream_t s)
{
    if (g_fp32)
        k_relu_bwd<float><<<blocks(rows * C), 256, 0, s>>>((float*)g, gpitch, (const bf16*)y, ypitch, rows, C);
    else
        k_relu_bwd<bf16><<<blocks(rows * C), 256, 0, s>>>((bf16*)g, gpitch, (const bf16*)y, ypitch, rows, C);
    return cudaGetLastError();
}

cudaError_t transpose(const void* in, int rows, int cols, int ipitch, void* out, int opitch, cudaStream_t s)
{
    if ((cols + 31) / 32 > 65535) return cudaErrorInvalidValue;
    dim3 grid((rows + 31) / 32, (cols + 31) / 32), block(32, 8);
    k_transpose<<<grid, block, 0, s>>>((const bf16*)in, rows, cols, ipitch, (bf16*)out, opitch);
    return cudaGetLastError();
}

cudaError_t maxpool_fwd(const void* X, int B, int H, int W, int C, int xpitch, void* Y, cudaStream_t s)
{
    if (H % 2 || W % 2) return cudaErrorInvalidValue;
    if (C % 8 == 0 && xpitch % 8 == 0 && (((uintptr_t)X | (uintptr_t)Y) & 15) == 0)
        k_maxpool_fwd8<<<blocks((long long)B * (H / 2) * (W / 2) * (C / 8)), 256, 0, s>>>((const bf16*)X, B, H, W, C,
                                                                                        xpitch, (bf16*)Y);
    else
        k_maxpool_fwd<<<blocks((long long)B * (H / 2) * (W / 2) * C), 256, 0, s>>>((const bf16*)X, B, H, W, C, xpitch,
                                                                                 (bf16*)Y);
    return cudaGetLastError();
}

cudaError_t maxpool_bwd(const void* X, int B, int H, int W, int C, int xpitch, const float* dY, float* dX, int dpitch,
                        cudaStream_t s)
{
    const long long Po = (long long)B * (H / 2) * (W / 2);
    const bool vec = C % 8 == 0 && C / 8 <= 256 && xpitch % 8 == 0 && dpitch % 4 == 0 &&
                     (((uintptr_t)X | (uintptr_t)dY | (uintptr_t)dX) & 15) == 0;
    if (vec) {
        const dim3 b(C / 8, 256 / (C / 8));
        k_maxpool_bwd8<<<(unsigned)((Po + b.y - 1) / b.y), b, 0, s>>>((const bf16*)X, B, H, W, C, xpitch, dY, dX,
                                                                         dpitch);
    } else {
        k_maxpool_bwd<<<blocks(Po * C), 256, 0, s>>>((const bf16*)X, B, H, W, C, xpitch, dY, dX, dpitch);
    }
    return cudaGetLastError();
}

cudaError_t shuffle_fwd(const void* U, int B, int H, int W, int C, void* Y, int ypitch, int c0, cudaStream_t s)
{
    k_shuffle_fwd<<<blocks((long long)B * H * W * 4 * C), 256, 0, s>>>((const bf16*)U, B, H, W, C, (bf16*)Y, ypitch,
                                                                      c0);
    return cudaGetLastError();
}

cudaError_t shuffle_bwd(const void* dY, bool dy_fp32, int ypitch, int c0, int B, int H, int W, int C, void* dU,
                        cudaStream_t s)
{
    const long long n = (long long)B * H * W * 4 * C;
    const bool vec = C % 8 == 0 && c0 % 8 == 0 && ypitch % 8 == 0 && n / 8 < 0x7fffffffLL &&
                     (((uintptr_t)dY | (uintptr_t)dU) & 15) == 0;
    if (vec) {
        const int groups = (int)(n / 8);
        if (dy_fp32)
            k_shuffle_bwd8<float><<<(groups + 255) / 256, 256, 0, s>>>((const float*)dY, ypitch, c0, H, W, C / 8,
                                                                       groups, (bf16*)dU);
        else
            k_shuffle_bwd8<bf16><<<(groups + 255) / 256, 256, 0, s>>>((const bf16*)dY, ypitch, c0, H, W, C / 8,
                                                                      groups, (bf16*)dU);
    } else if (dy_fp32) {
        k_shuffle_bwd<float><<<blocks(n), 256, 0, s>>>((const float*)dY, ypitch, c0, B, H, W, C, (bf16*)dU);
    } else {
        k_shuffle_bwd<bf16><<<blocks(n), 256, 0, s>>>((const bf16*)dY, ypitch, c0, B, H, W, C, (bf16*)dU);
    }
    return cudaGetLastError();
}

cudaError_t proj_fwd(const void* X, int P, int C, int xpitch, const float* Wt, const float* bias, int O,
                     const float* R, float* Y, cudaStream_t s)
{
    if (O > 8) return cudaErrorInvalidValue;
    const size_t sh = (size_t)(O * C + O) * sizeof(float);
    if (C % 8 == 0 && xpitch % 8 == 0 && ((uintptr_t)X & 15) == 0 && sh <= 48 * 1024)
        k_proj_fwd_vec<<<blocks(P, 128), 128, sh, s>>>((const bf16*)X, P, C, xpitch, Wt, bias, O, R, Y);
    else
        k_proj_fwd<<<blocks(P), 256, 0, s>>>((const bf16*)X, P, C, xpitch, Wt, bias, O, R, Y);
    return cudaGetLastError();
}

cudaError_t proj_bwd(const float* dY, const void* X, int P, int C, int xpitch, const float* Wt, int O, float* dX,
                     int dpitch, float* dW, float* db, float* part, int part_blocks, cudaStream_t s)
{
    if (dX) {
        const bool vec = C % 4 == 0 && C / 4 <= 256 && dpitch % 4 == 0 &&
                         (((uintptr_t)dX | (uintptr_t)Wt) & 15) == 0;
        if (vec) {
            const dim3 b(C / 4, 256 / (C / 4));
            k_proj_bwd_x4<<<(unsigned)((P + b.y - 1) / b.y), b, 0, s>>>(dY, P, O, Wt, C, dX, dpitch);
        } else {
            k_proj_bwd_x<<<blocks((long long)P * C), 256, 0, s>>>(dY, P, O, Wt, C, dX, dpitch);
        }
    }
    const int chunk = (P + part_blocks - 1) / part_blocks;
    const int nb = (P + chunk - 1) / chunk;
    const bool vec = (C == 8 || C == 16 || C == 32 || C == 64) && O >= 1 && O <= 8 && xpitch % 8 == 0 &&
                     ((uintptr_t)X & 15) == 0;
    if (vec) {
        switch (O) {
#define NN_PROJ_W8(OV) \
    case OV: k_proj_bwd_w8<OV><<<nb, 256, 0, s>>>(dY, (const bf16*)X, P, C, xpitch, chunk, part); break;
            NN_PROJ_W8(1)
            NN_PROJ_W8(2)
            NN_PROJ_W8(3)
            NN_PROJ_W8(4)
            NN_PROJ_W8(5)
            NN_PROJ_W8(6)
            NN_PROJ_W8(7)
            NN_PROJ_W8(8)
#undef NN_PROJ_W8
        }
    } else if (C <= 64 && O <= 8) {
        k_proj_bwd_w_warps<<<nb, 256, 0, s>>>(dY, (const bf16*)X, P, C, xpitch, O, chunk, part);
    } else {
        k_proj_bwd_w<<<nb, 128, 0, s>>>(dY, (const bf16*)X, P, C, xpitch, O, chunk, part);
    }
    const int slots = O * (C + 1);
    k_proj_sum<<<(unsigned)((slots + 7) / 8), 256, 0, s>>>(part, nb, O, C, dW, db);
    return cudaGetLastError();
}

cudaError_t gatherT(const void* X, int B, int H, int W, int C, int cpitch, int taps, void* AT, long long atpitch,
                    cudaStream_t s)
{
    const long long P = (long long)B * H * W;
    if ((taps != 9 && taps != 3 && taps != 1) || C % 8 || cpitch % 8 || atpitch % 8 || P % 8)
        return cudaErrorInvalidValue;
    if (P > 0x7fffffffLL) return cudaErrorInvalidValue;
    if (((uintptr_t)X | (uintptr_t)AT) & 15) return cudaErrorInvalidValue;
    if ((taps == 3 || taps == 9) && W % 8 == 0) {
        const dim3 grid((unsigned)((P + 63) / 64), (unsigned)((C + 63) / 64));
        if (grid.y > 65535) return cudaErrorInvalidValue;
        if (taps == 3)
            k_gather_rows<1><<<grid, 256, 0, s>>>((const bf16*)X, (int)P, H, W, C, cpitch, (bf16*)AT, atpitch);
        else
            k_gather_rows<3><<<grid, 256, 0, s>>>((const bf16*)X, (int)P, H, W, C, cpitch, (bf16*)AT, atpitch);
        return cudaGetLastError();
    }
    const long long cblocks = (long long)((C + 63) / 64) * taps;
    if (cblocks > 65535) return cudaErrorInvalidValue;
    dim3 grid((unsigned)((P + 63) / 64), (unsigned)cblocks);
    k_gatherT<<<grid, 256, 0, s>>>((const bf16*)X, B, H, W, C, cpitch, taps, (bf16*)AT, atpitch);
    return cudaGetLastError();
}

cudaError_t mask_cast(const float* g, int gpitch, const void* y, int ypitch, long long rows, int C, void* out,
                      int opitch, cudaStream_t s)
{
    const bool vec = C % 8 == 0 && gpitch % 8 == 0 && ypitch % 8 == 0 && opitch % 8 == 0 &&
                     (((uintptr_t)g | (uintptr_t)y | (uintptr_t)out) & 31) == 0 && rows * (C / 8) < 0x7fffffffLL;
    if (vec) {
        const int groups = (int)(rows * (C / 8));
        k_mask_cast8<<<(groups + 255) / 256, 256, 0, s>>>(g, gpitch, (const bf16*)y, ypitch, groups, C / 8,
                                                          (bf16*)out, opitch);
    } else {
        k_mask_cast<<<blocks(rows * C), 256, 0, s>>>(g, gpitch, (const bf16*)y, ypitch, rows, C, (bf16*)out,
                                                     opitch);
    }
    return cudaGetLastError();
}

cudaError_t pad_conv3x3(const void* W, int cout, int cin, int cin_pad, void* Wp, cudaStream_t s)
{
    if (cin_pad < cin) return cudaErrorInvalidValue;
    k_pad_conv3x3<<<blocks((long long)cout * 9 * cin_pad), 256, 0, s>>>((const bf16*)W, cout, cin, cin_pad, (bf16*)Wp);
    return cudaGetLastError();
}

cudaError_t flip3x3_many(const FlipJob* jobs, int njobs, long long total, cudaStream_t s)
{
    if (njobs < 1 || total < 1) return cudaSuccess;
    k_flip3x3_many<<<blocks(total), 256, 0, s>>>(jobs, njobs, total);
    return cudaGetLastError();
}

cudaError_t flip3x3(const void* W, int cout, int cin, void* Wf, cudaStream_t s)
{
    k_flip3x3<<<blocks((long long)cout * 9 * cin), 256, 0, s>>>((const bf16*)W, cout, cin, (bf16*)Wf);
    return cudaGetLastError();
}

cudaError_t colsum(const void* g, bool g_fp32, long long rows, int C, int pitch, float* out, float* part,
                   int part_blocks, cudaStream_t s)
{
    if (rows < 1 || C < 1 || part_blocks < 1) return cudaErrorInvalidValue;
    // at most part_blocks partial rows; a block's rows are split among its
    // row lanes, and a block takes about 32 rows per lane (fewer, longer blocks
    // for short matrices: less to add afterwards, without starving the grid)
    const bool vec = !g_fp32 && C % 8 == 0 && pitch % 8 == 0 && C <= 1024 && ((uintptr_t)g & 15) == 0;
    const int G = vec ? C / 8 : (C < 128 ? C : 128);
    const long long lanes = G < 128 ? 128 / G : 1;
    long long chunk = (rows + part_blocks - 1) / part_blocks;
    if (chunk < 32 * lanes) chunk = 32 * lanes;
    const int nb = (int)((rows + chunk - 1) / chunk);
    if (g_fp32)
        k_colsum_part<float><<<nb, 128, 0, s>>>((const float*)g, rows, C, pitch, (int)chunk, part);
    else if (vec)
        k_colsum_part8<<<nb, 128, 0, s>>>((const bf16*)g, rows, C, pitch, (int)chunk, part);
    else
        k_colsum_part<bf16><<<nb, 128, 0, s>>>((const bf16*)g, rows, C, pitch, (int)chunk, part);
    k_sum_parts<<<(unsigned)((C + 7) / 8), 256, 0, s>>>(part, nb, C, out);
    return cudaGetLastError();
}

cudaError_t mse(const float* pred, const float* target, long long n, float* grad, float* loss, float* part,
                cudaStream_t s, const float* x, int F, float alpha)
{
    const int nb = (int)((n + 255) / 256);
    k_mse<<<nb, 256, 0, s>>>(pred, target, n, x, F, alpha, grad, part);
    k_sum_one<<<1, 1024, 0, s>>>(part, nb, loss);
    return cudaGetLastError();
}

cudaError_t adam(float* w, const float* g, float* m, float* v, long long n, float lr, float b1, float b2, float eps,
                 int t, void* wb, cudaStream_t s)
{
    const float c1 = 1.0f - powf(b1, (float)t), c2 = 1.0f - powf(b2, (float)t);
    k_adam<<<blocks(n), 256, 0, s>>>(w, g, m, v, n, lr, b1, b2, eps, c1, c2, (bf16*)wb);
    return cudaGetLastError();
}

cudaError_t pack(const float* f, long long P, int F, const float* mean, const float* inv_std, void* X, int cpitch,
                 float* R, cudaStream_t s)
{
    if (F > cpitch) return cudaErrorInvalidValue;
    if (X && !R && F <= 8 && cpitch % 8 == 0 && ((uintptr_t)X & 15) == 0)
        k_pack_px<<<blocks(P), 256, 0, s>>>(f, P, F, mean, inv_std, (bf16*)X, cpitch);
    else
        k_pack<<<blocks(P * cpitch), 256, 0, s>>>(f, P, F, mean, inv_std, (bf16*)X, cpitch, R);
    return cudaGetLastError();
}

cudaError_t unpack(const float* Y, long long P, int F, const float* mean, const float* inv_std, float* f,
                   cudaStream_t s)
{
    k_unpack<<<blocks(P * F), 256, 0, s>>>(Y, P, F, mean, inv_std, f);
    return cudaGetLastError();
}

cudaError_t increment(const float* t, const float* x, long long P, int F, const float* inv_out, float* T,
                      cudaStream_t s)
{
    k_increment<<<blocks(P * F), 256, 0, s>>>(t, x, P, F, inv_out, T);
    return cudaGetLastError();
}

cudaError_t add_increment(const float* Y, const float* x, long long P, int F, const float* inv_out, float* y,
                          cudaStream_t s)
{
    k_add_increment<<<blocks(P * F), 256, 0, s>>>(Y, x, P, F, inv_out, y);
    return cudaGetLastError();
}

cudaError_t cast_bf16(const float* a, long long rows, int C, int apitch, void* b, int bpitch, cudaStream_t s)
{
    k_cast_bf16<<<blocks(rows * C), 256, 0, s>>>(a, rows, C, apitch, (bf16*)b, bpitch);
    return cudaGetLastError();
}

}  // namespace nn
