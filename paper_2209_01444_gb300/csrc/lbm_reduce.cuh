// Node pass of the metrics reduction, shared by the handle's reduction
// (lbm_aux.cu) and its allocation-free variant (lbm_noalloc.cu), which
// therefore give the same partials bit for bit.
//
// Block b folds the nodes [b * kRedNodesPerBlock, (b + 1) * kRedNodesPerBlock)
// (row-major over the nx x ny grid, pitch skipped), thread t the nodes
// t, t + kRedThreadsPerBlock, ... of that chunk (16 of them).  A thread sums
// its nodes' small deviations in FP32 (phi + 1, C - 1, H - H_ref, the nine
// flow deviations, max |u|, non-finite count) and adds the constant
// reference terms once, in FP64, with its exact node count; warps and the
// block then combine FP64 values in a fixed order.  GB300 issues FP64 at a
// small fraction of its FP32 rate, so per-node FP64 arithmetic would bound
// this pass well below the memory bandwidth.
//
// Partials per block (kRedValues doubles): sum (1 + phi)/2, sum C, sum H,
// sum of the flow populations, max |u|, non-finite count, sum phi.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

constexpr int kRedValues = 7;
constexpr int kRedThreadsPerBlock = 256;
constexpr int kRedNodesPerBlock = 4096;  // 16 nodes per thread

// Blocks of the node pass for an nx x ny grid.
__host__ __device__ inline long long reduce_chunk_blocks(long long nodes)
{
    return (nodes + kRedNodesPerBlock - 1) / kRedNodesPerBlock;
}

__device__ __forceinline__ double red_warp_sum(double v)
{
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
    return v;
}
__device__ __forceinline__ double red_warp_max(double v)
{
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, d));
    return v;
}

template <class Store>
__device__ __forceinline__ void reduce_chunk(const StepParams& P, const void* __restrict__ sc,
                                             const void* __restrict__ fl, double* __restrict__ partials)
{
    const long long N = (long long)P.nx * P.ny;
    const long long first = (long long)blockIdx.x * kRedNodesPerBlock;
    const long long last = min(first + kRedNodesPerBlock, N);
    float sp1 = 0.0f, sdC = 0.0f, sdH = 0.0f, sh = 0.0f, umax = 0.0f;
    int bad = 0, count = 0;
    for (long long t = first + threadIdx.x; t < last; t += kRedThreadsPerBlock) {
        const int y = (int)(t / P.nx), x = (int)(t - (long long)y * P.nx);
        const long long o = (long long)y * P.pitch + x;
        float f[5], n[5], g[5], h[9];
#pragma unroll
        for (int i = 0; i < 5; ++i) f[i] = Store::load(sc, fl, kF + i, o, P);
#pragma unroll
        for (int i = 0; i < 5; ++i) n[i] = Store::load(sc, fl, kN + i, o, P);
#pragma unroll
        for (int i = 0; i < 5; ++i) g[i] = Store::load(sc, fl, kG + i, o, P);
#pragma unroll
        for (int i = 0; i < 9; ++i) h[i] = Store::load(sc, fl, kH + i, o, P);
        const Macro m = node_macros(f, n, g, h, P);
        float s9 = 0.0f;
#pragma unroll
        for (int i = 0; i < 9; ++i) s9 += h[i];
        const float u = sqrtf(m.ux * m.ux + m.uy * m.uy);
        sp1 += m.p1;
        sdC += m.dC;
        sdH += m.dH;
        sh += s9;
        umax = fmaxf(umax, u);
        bad += (isfinite(m.p1) && isfinite(m.dC) && isfinite(m.dth) && isfinite(u)) ? 0 : 1;
        ++count;
    }
    const double c = (double)count;
    double acc[kRedValues];
    acc[0] = 0.5 * (double)sp1;
    acc[1] = c + (double)sdC;
    acc[2] = c * ((double)P.theta_ref + (double)P.latent) + (double)sdH;
    acc[3] = c * (double)P.rho0 + (double)sh;
    acc[4] = (double)umax;
    acc[5] = (double)bad;
    acc[6] = (double)sp1 - c;
    __shared__ double sm[kRedValues][kRedThreadsPerBlock / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < kRedValues; ++k) {
        const double v = k == 4 ? red_warp_max(acc[k]) : red_warp_sum(acc[k]);
        if (lane == 0) sm[k][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < kRedValues) {
        const int k = threadIdx.x;
        double v = sm[k][0];
        for (int w = 1; w < kRedThreadsPerBlock / 32; ++w) v = (k == 4) ? fmax(v, sm[k][w]) : v + sm[k][w];
        partials[(long long)blockIdx.x * kRedValues + k] = v;
    }
}

}  // namespace lbm
