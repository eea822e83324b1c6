// Initialisation, field extraction, state codecs and the metrics reductions.
#include <cuda_runtime.h>
#include <math.h>

#include <cooperative_groups.h>

#include "lbm_kernels.h"
#include "lbm_reduce.cuh"

namespace lbm {

namespace {

template <class Store>
__device__ __forceinline__ void load_node(const StepParams& P, const void* sc, const void* fl, long long o, float* f,
                                          float* n, float* g, float* h)
{
#pragma unroll
    for (int i = 0; i < 5; ++i) f[i] = Store::load(sc, fl, kF + i, o, P);
#pragma unroll
    for (int i = 0; i < 5; ++i) n[i] = Store::load(sc, fl, kN + i, o, P);
#pragma unroll
    for (int i = 0; i < 5; ++i) g[i] = Store::load(sc, fl, kG + i, o, P);
#pragma unroll
    for (int i = 0; i < 9; ++i) h[i] = Store::load(sc, fl, kH + i, o, P);
}

__device__ __forceinline__ double min_image(double d, int L, int periodic)
{
    if (!periodic) return d;
    while (d > 0.5 * L) d -= L;
    while (d < -0.5 * L) d += L;
    return d;
}

// Row bands.  Whole-grid transfers go through a bounded scratch buffer one
// band of rows [y0, y0 + rows) at a time; a band's scratch holds its planes
// one after another, rows * pitch elements each, node (x, y) at
// (y - y0) * pitch + x.

// Seeds (Sec. 4): phi = max_j tanh[(R_j - d_j)/(sqrt2 W0)], grain = nearest
// centre (ties to the lower index); FP64 so that both choices match an FP64
// evaluation.  fields: 6 FP64 band planes (phi, U, theta, ux, uy, p), lattice
// units; grain: the whole grid's plane.
__global__ void k_seed_fields(const StepParams P, const double* __restrict__ seeds, int ns, double U0,
                              double theta0, double W, double* __restrict__ fields, uint8_t* __restrict__ grain,
                              int y0, int rows)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = y0 + blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= P.nx || y >= y0 + rows || y >= P.ny) return;
    const long long o = (long long)y * P.pitch + x;
    const long long ob = (long long)(y - y0) * P.pitch + x, bp = (long long)rows * P.pitch;
    // phi is the largest of the seeds' profiles; tanh increases, so that is
    // the profile of the largest argument: one tanh per node (ns >= 1)
    double best_arg = -1e300, best_d2 = 1e300;
    int best = 0;
    const double inv = 1.0 / (sqrt(2.0) * W);
    for (int j = 0; j < ns; ++j) {
        const double dx = min_image(x - seeds[4 * j + 0], P.nx, P.periodic_x);
        const double dy = min_image(y - seeds[4 * j + 1], P.ny, P.periodic_y);
        const double d2 = dx * dx + dy * dy;
        const double a = (seeds[4 * j + 2] - sqrt(d2)) * inv;
        if (a > best_arg) best_arg = a;
        if (d2 < best_d2) {
            best_d2 = d2;
            best = j;
        }
    }
    fields[0 * bp + ob] = tanh(best_arg);
    fields[1 * bp + ob] = U0;
    fields[2 * bp + ob] = theta0;
    fields[3 * bp + ob] = 0.0;
    fields[4 * bp + ob] = 0.0;
    fields[5 * bp + ob] = 0.0;
    if (grain) grain[o] = (uint8_t)best;
}

// Equilibrium populations of node o for the macro deviations (phi + 1,
// C - 1, U, theta - theta_ref, u in flow lattice units, p), then history = the
// macros recovered from the stored populations (so the first backward
// differences vanish).
template <class Store>
__device__ void init_node(const StepParams& P, long long o, float p1, float dC, float Uf, float dth, float ux,
                          float uy, float p, void* __restrict__ sc, void* __restrict__ fl, float* __restrict__ hist,
                          float heqx, float heqy)
{
    const float hp1 = h_plus_1(P.h_kind, p1);
    const float H = (P.theta_ref + P.latent) + dth - P.latent * hp1;
    const float C = 1.0f + dC;
    const float sx = ux * P.nsub, sy = uy * P.nsub;
    float e[9];
    deq_phi(p1, e);
#pragma unroll
    for (int i = 0; i < 5; ++i) Store::store(sc, fl, kF + i, o, e[i], P);
    deq_C(dC, (1.0f - 0.5f * p1) * Uf, C * sx, C * sy, e);
#pragma unroll
    for (int i = 0; i < 5; ++i) Store::store(sc, fl, kN + i, o, e[i], P);
    deq_H(dth, P.latent * hp1, H * sx, H * sy, e);
#pragma unroll
    for (int i = 0; i < 5; ++i) Store::store(sc, fl, kG + i, o, e[i], P);
    deq_flow(p, heqx, heqy, e);
#pragma unroll
    for (int i = 0; i < 9; ++i) Store::store(sc, fl, kH + i, o, e[i], P);

    float f[5], n[5], g[5], h[9];
    load_node<Store>(P, sc, fl, o, f, n, g, h);
    const Macro m = node_macros(f, n, g, h, P);
    const float usx = m.ux * P.nsub, usy = m.uy * P.nsub;
    hist_at(hist, 0, o) = m.phi;
    hist_at(hist, 1, o) = coupling_Q(m.phi, P.theta_ref + m.dth, m.U, P);
    hist_at(hist, 2, o) = (1.0f + m.dC) * usx;
    hist_at(hist, 3, o) = (1.0f + m.dC) * usy;
    hist_at(hist, 4, o) = m.H * usx;
    hist_at(hist, 5, o) = m.H * usy;
}

template <class Store>
__global__ void k_init(const StepParams P, const double* __restrict__ fields, void* __restrict__ sc,
                       void* __restrict__ fl, float* __restrict__ hist, int y0, int rows)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = y0 + blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= P.nx || y >= y0 + rows || y >= P.ny) return;
    const long long o = (long long)y * P.pitch + x;
    const long long ob = (long long)(y - y0) * P.pitch + x, bp = (long long)rows * P.pitch;
    // macro deviations from the reference state, formed in FP64
    const double phi = fields[0 * bp + ob], U = fields[1 * bp + ob];
    const double k = P.k;
    const float p1 = (float)(phi + 1.0);
    const float dC = (float)(0.5 * (1.0 + k - (1.0 - k) * phi) * (1.0 + (1.0 - k) * U) - 1.0);
    const float dth = (float)(fields[2 * bp + ob] - (double)P.theta_ref);
    const float ux = (float)fields[3 * bp + ob], uy = (float)fields[4 * bp + ob];
    init_node<Store>(P, o, p1, dC, (float)U, dth, ux, uy, (float)fields[5 * bp + ob], sc, fl, hist, ux, uy);
}

// Fields of every node, pixel-interleaved for the surrogate network:
// dst[(y * nx + x) * 5 + c] for c = phi, C, theta, u_x, u_y (velocities in
// the paper's units: flow lattice units times inv_vf).
template <class Store>
__global__ void k_fields_nhwc(const StepParams P, const void* __restrict__ sc, const void* __restrict__ fl,
                              float inv_vf, float* __restrict__ dst)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= P.nx || y >= P.ny) return;
    const long long o = (long long)y * P.pitch + x;
    float f[5], n[5], g[5], h[9];
    load_node<Store>(P, sc, fl, o, f, n, g, h);
    const Macro m = node_macros(f, n, g, h, P);
    float* d = dst + ((long long)y * P.nx + x) * 5;
    d[0] = m.phi;
    d[1] = 1.0f + m.dC;
    d[2] = P.theta_ref + m.dth;
    d[3] = m.ux * inv_vf;
    d[4] = m.uy * inv_vf;
}

// Replaces every node's populations by the equilibrium of the given fields
// (layout of k_fields_nhwc; phi clamped to [-1, 1], U recovered from C and
// phi by the definition of U), keeping the node's current pressure.  Each
// thread reads and writes only its own node, so this works in place.
template <class Store>
__global__ void k_set_fields_nhwc(const StepParams P, const float* __restrict__ src, float vf, void* __restrict__ sc,
                                  void* __restrict__ fl, float* __restrict__ hist, const float* __restrict__ prev,
                                  float inv_k)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= P.nx || y >= P.ny) return;
    const long long o = (long long)y * P.pitch + x;
    float f[5], n[5], g[5], h[9];
    load_node<Store>(P, sc, fl, o, f, n, g, h);
    const float p = node_macros(f, n, g, h, P).p;
    const float* d = src + ((long long)y * P.nx + x) * 5;
    const float phi = fminf(1.0f, fmaxf(-1.0f, d[0]));
    const float C = d[1];
    const float k = P.k;
    const float U = (2.0f * C / (1.0f + k - (1.0f - k) * phi) - 1.0f) / (1.0f - k);
    const float p1 = phi + 1.0f, dC = C - 1.0f, dth = d[2] - P.theta_ref;
    const float ux = d[3] * vf, uy = d[4] * vf;
    // The stored momentum j is what the macro recovery turns into
    // u = (j + F/2)(1 + q~)/2 (Guo forcing and the fluid-solid force, q~ =
    // (1 - phi)/2), so the flow equilibrium takes j = 2u/(1 + q~) - F/2; its
    // pressure argument compensates the |j|^2 - |u|^2 the recovery removes.
    const float a = 0.5f * (1.0f + (1.0f - 0.5f * p1));
    const float Fx = P.Fx, Fy = P.Fy + P.gbT * dth + P.gbC * (dC + P.dC_ref);
    const float jx = ux / a - 0.5f * Fx, jy = uy / a - 0.5f * Fy;
    const float peq = p - 0.4f * (jx * jx + jy * jy - ux * ux - uy * uy);
    init_node<Store>(P, o, p1, dC, U, dth, ux, uy, peq, sc, fl, hist, jx, jy);
    if (!prev) return;
    // History one step back on the straight line from the fields K steps
    // earlier (prev), so that the first backward differences after the
    // rebuild carry the window's mean rate of change.
    const float* q = prev + ((long long)y * P.nx + x) * 5;
    const float phi_b = phi - (phi - fminf(1.0f, fmaxf(-1.0f, q[0]))) * inv_k;
    const float C_b = C - (C - q[1]) * inv_k;
    const float th_b = d[2] - (d[2] - q[2]) * inv_k;
    const float ux_b = ux - (ux - q[3] * vf) * inv_k, uy_b = uy - (uy - q[4] * vf) * inv_k;
    const float U_b = (2.0f * C_b / (1.0f + k - (1.0f - k) * phi_b) - 1.0f) / (1.0f - k);
    const float H_b = th_b - 0.5f * (h_plus_1(P.h_kind, phi_b + 1.0f) - 1.0f);  // H = theta - h/2
    hist_at(hist, 0, o) = phi_b;
    hist_at(hist, 1, o) = coupling_Q(phi_b, th_b, U_b, P);
    hist_at(hist, 2, o) = C_b * ux_b * P.nsub;
    hist_at(hist, 3, o) = C_b * uy_b * P.nsub;
    hist_at(hist, 4, o) = H_b * ux_b * P.nsub;
    hist_at(hist, 5, o) = H_b * uy_b * P.nsub;
}

// Interface mismatch between two pixel-interleaved field sets (stride 5,
// phi first): out[0] += nodes where the signs of phi differ, out[1] = max
// |phi_a - phi_b| (as the bits of a non-negative float, so integer maximum
// orders them).
__global__ void k_phi_mismatch(const float* __restrict__ a, const float* __restrict__ b, long long n,
                               unsigned long long* __restrict__ out)
{
    unsigned long long cnt = 0;
    float mx = 0.0f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float pa = a[i * 5], pb = b[i * 5];
        cnt += ((pa > 0.0f) != (pb > 0.0f)) ? 1ull : 0ull;
        const float d = fabsf(pa - pb);
        mx = (d > mx || d != d) ? d : mx;
    }
    for (int s = 16; s > 0; s >>= 1) {
        cnt += __shfl_down_sync(0xffffffffu, cnt, s);
        mx = fmaxf(mx, __shfl_down_sync(0xffffffffu, mx, s));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&out[0], cnt);
        atomicMax(&out[1], (unsigned long long)__float_as_uint(mx));
    }
}

// out[0] += the number of values of a[0 .. n) that are not finite.
__global__ void k_count_nonfinite(const float* __restrict__ a, long long n, unsigned long long* __restrict__ out)
{
    unsigned long long cnt = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        cnt += isfinite(a[i]) ? 0ull : 1ull;
    for (int s = 16; s > 0; s >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, s);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(&out[0], cnt);
}

// Macro deviations of every node: phi + 1, C - 1, U, theta - theta_ref, ux,
// uy, p (flow lattice units); the host adds the reference values in FP64.
template <class Store>
__global__ void k_macros(const StepParams P, const void* __restrict__ sc, const void* __restrict__ fl,
                         float* __restrict__ out, int y0, int rows)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = y0 + blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= P.nx || y >= y0 + rows || y >= P.ny) return;
    const long long o = (long long)y * P.pitch + x;
    float f[5], n[5], g[5], h[9];
    load_node<Store>(P, sc, fl, o, f, n, g, h);
    const Macro m = node_macros(f, n, g, h, P);
    const long long ob = (long long)(y - y0) * P.pitch + x, bp = (long long)rows * P.pitch;
    out[0 * bp + ob] = m.p1;
    out[1 * bp + ob] = m.dC;
    out[2 * bp + ob] = m.U;
    out[3 * bp + ob] = m.dth;
    out[4 * bp + ob] = m.ux;
    out[5 * bp + ob] = m.uy;
    out[6 * bp + ob] = m.p;
}

// The selected fields of the rows [y0, y0 + rows) in their final FP32 form,
// plane k of the band at out + k * rows * nx with rows of nx values (the
// layout of the caller's array, so each plane of the band is one contiguous
// copy): field = deviation * scale + offset, the deviations of k_macros.
template <class Store>
__global__ void k_fields_f32(const StepParams P, const void* __restrict__ sc, const void* __restrict__ fl,
                             const FieldsF32 spec, float* __restrict__ out, int y0, int rows)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = y0 + blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= P.nx || y >= y0 + rows || y >= P.ny) return;
    const long long o = (long long)y * P.pitch + x;
    float f[5], n[5], g[5], h[9];
    load_node<Store>(P, sc, fl, o, f, n, g, h);
    const Macro m = node_macros(f, n, g, h, P);
    const float v[7] = {m.p1, m.dC, m.U, m.dth, m.ux, m.uy, m.p};
    const long long ob = (long long)(y - y0) * P.nx + x, bp = (long long)rows * P.nx;
    for (int k = 0; k < spec.n; ++k) {
        float d = v[0];
#pragma unroll
        for (int q = 1; q < 7; ++q)
            if (spec.sel[k] == q) d = v[q];
        out[k * bp + ob] = fmaf(d, spec.scale[k], spec.offset[k]);
    }
}

// Deviations of every population as FP32 band planes 0..23 and the history
// as planes 24..29 (and back).
template <class Store>
__global__ void k_decode(const StepParams P, const void* __restrict__ sc, const void* __restrict__ fl,
                         const float* __restrict__ hist, float* __restrict__ out, int y0, int rows)
{
    const long long bp = (long long)rows * P.pitch;
    const long long ib = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (ib >= bp) return;
    const long long i = (long long)y0 * P.pitch + ib;
#pragma unroll
    for (int q = 0; q < kPlanes; ++q) out[q * bp + ib] = Store::load(sc, fl, q, i, P);
#pragma unroll
    for (int k = 0; k < kHist; ++k) out[(kPlanes + k) * bp + ib] = hist_at(hist, k, i);
}

template <class Store>
__global__ void k_encode(const StepParams P, const float* __restrict__ in, void* __restrict__ sc,
                         void* __restrict__ fl, float* __restrict__ hist, int y0, int rows)
{
    const long long bp = (long long)rows * P.pitch;
    const long long ib = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (ib >= bp) return;
    const long long i = (long long)y0 * P.pitch + ib;
#pragma unroll
    for (int q = 0; q < kPlanes; ++q) Store::store(sc, fl, q, i, in[q * bp + ib], P);
#pragma unroll
    for (int k = 0; k < kHist; ++k) hist_at(hist, k, i) = in[(kPlanes + k) * bp + ib];
}

// ------------------------------------------------------------- reductions
constexpr int kRedThreads = 256;
constexpr int kTipThreads = 256;
constexpr int kTipCluster = 8;  // CTAs per ray
constexpr int kRedVals = kRedValues;

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
    return v;
}
__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, d));
    return v;
}

// Pass 1: block b folds its chunk of nodes into kRedVals partials
// (reduce_chunk: FP32 per thread, FP64 across threads, fixed order).
template <class Store>
__global__ void __launch_bounds__(kRedThreadsPerBlock) k_reduce_nodes(const StepParams P, const void* __restrict__ sc,
                                                                      const void* __restrict__ fl,
                                                                      double* __restrict__ partials)
{
    reduce_chunk<Store>(P, sc, fl, partials);
}

// Pass 2: one warp per value folds the partials: lane l takes blocks
// l, l + 32, ..., then a shuffle tree adds the lanes (a fixed order).
__global__ void k_reduce_final(const double* __restrict__ partials, int nblocks, double* __restrict__ out)
{
    const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (k >= kRedVals) return;
    double v = 0.0;
    for (int b = lane; b < nblocks; b += 32) {
        const double p = partials[(long long)b * kRedVals + k];
        v = (k == 4) ? fmax(v, p) : v + p;
    }
    v = (k == 4) ? warp_max(v) : warp_sum(v);
    if (lane == 0) out[k] = v;
}

// Hydrodynamic force and torque on the solid (Eq. 27, weighted by 1 - q~ =
// (1 + phi)/2, the share of the fluid-solid force the flow feels): per-block
// FP64 partials of -sum w f_x, -sum w f_y and -sum ((x - cx) w f_y - (y - cy) w f_x).
template <class Store>
__global__ void __launch_bounds__(kRedThreads) k_force(const StepParams P, const void* __restrict__ sc,
                                                       const void* __restrict__ fl, double cx, double cy,
                                                       double* __restrict__ partials)
{
    double acc[3] = {0, 0, 0};
    const long long N = (long long)P.nx * P.ny;
    for (long long t = blockIdx.x * (long long)kRedThreads + threadIdx.x; t < N;
         t += (long long)gridDim.x * kRedThreads) {
        const int y = (int)(t / P.nx), x = (int)(t - (long long)y * P.nx);
        const long long o = (long long)y * P.pitch + x;
        float f[5], n[5], g[5], h[9];
        load_node<Store>(P, sc, fl, o, f, n, g, h);
        const Macro m = node_macros(f, n, g, h, P);
        const double w = 0.5 * (double)m.p1;
        const double fx = w * (double)m.fsx, fy = w * (double)m.fsy;
        acc[0] -= fx;
        acc[1] -= fy;
        acc[2] -= (x - cx) * fy - (y - cy) * fx;
    }
    __shared__ double sm[3][kRedThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double v = warp_sum(acc[k]);
        if (lane == 0) sm[k][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double v = 0.0;
        for (int w = 0; w < kRedThreads / 32; ++w) v += sm[threadIdx.x][w];
        partials[(long long)blockIdx.x * 3 + threadIdx.x] = v;
    }
}

__global__ void k_force_final(const double* __restrict__ partials, int nblocks, double* __restrict__ out)
{
    const int k = threadIdx.x;
    if (k >= 3) return;
    double v = 0.0;
    for (int b = 0; b < nblocks; ++b) v += partials[(long long)b * 3 + k];
    out[k] = v;
}

// Frozen inputs of flow-only steps: phi and the body force F_y of every node.
template <class Store>
__global__ void k_flow_inputs(const StepParams P, const void* __restrict__ sc, const void* __restrict__ fl,
                              float* __restrict__ phi, float* __restrict__ fy)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= P.nx || y >= P.ny) return;
    const long long o = (long long)y * P.pitch + x;
    float f[5], n[5], g[5], h[9];
    load_node<Store>(P, sc, fl, o, f, n, g, h);
    const Macro m = node_macros(f, n, g, h, P);
    phi[o] = m.phi;
    fy[o] = m.Fy;
}

template <class Store>
__device__ __forceinline__ double phi_at(const StepParams& P, const void* sc, int x, int y)
{
    const long long o = (long long)y * P.pitch + x;
    float s = 0.0f;  // phi + 1
#pragma unroll
    for (int i = 0; i < 5; ++i) s += Store::load(sc, nullptr, kF + i, o, P);
    return (double)s - 1.0;
}

template <class Store>
__device__ double phi_bilinear(const StepParams& P, const void* sc, double px, double py)
{
    int i = (int)floor(px), j = (int)floor(py);
    if (i > P.nx - 2) i = P.nx - 2;
    if (j > P.ny - 2) j = P.ny - 2;
    const double fx = px - i, fy = py - j;
    return (1 - fx) * (1 - fy) * phi_at<Store>(P, sc, i, j) + fx * (1 - fy) * phi_at<Store>(P, sc, i + 1, j) +
           (1 - fx) * fy * phi_at<Store>(P, sc, i, j + 1) + fx * fy * phi_at<Store>(P, sc, i + 1, j + 1);
}

template <class Store>
__device__ __forceinline__ float phi_at_f(const StepParams& P, const void* sc, int x, int y)
{
    const long long o = (long long)y * P.pitch + x;
    float s = 0.0f;  // phi + 1
#pragma unroll
    for (int i = 0; i < 5; ++i) s += Store::load(sc, nullptr, kF + i, o, P);
    return s - 1.0f;
}

// Tip distance along three rays from (cx, cy).  A cluster of kTipCluster
// CTAs handles one ray; its threads take the half-node samples j in turn.  A
// sample counts while its position (FP64) is inside the grid; phi there is
// interpolated bilinearly in FP32 to decide phi > 0 (the FP64 pipe of
// GB300 would otherwise bound this kernel).  The CTAs combine the outermost
// positive sample and the first outside one through distributed shared
// memory, and rank 0 interpolates between that sample and its successor
// to phi = 0 in FP64.
template <class Store>
__global__ void __cluster_dims__(kTipCluster, 1, 1) __launch_bounds__(kTipThreads)
    k_tips(const StepParams P, const void* __restrict__ sc, double cx, double cy, double c, double s,
           double* __restrict__ out)
{
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int r = blockIdx.x / kTipCluster;
    const double ex = r == 0 ? c : (r == 1 ? -c : -s);
    const double ey = r == 0 ? s : (r == 1 ? -s : c);
    const int jmax = 2 * (P.nx + P.ny) + 4;
    int last = -1, first_out = jmax;
    for (int j = rank * kTipThreads + threadIdx.x; j < jmax; j += kTipCluster * kTipThreads) {
        const double px = cx + j * 0.5 * ex, py = cy + j * 0.5 * ey;
        const bool inside = !(px < 0 || py < 0 || px > P.nx - 1 || py > P.ny - 1);
        if (!inside) {
            first_out = min(first_out, j);
            continue;
        }
        int i0 = (int)floor(px), j0 = (int)floor(py);
        if (i0 > P.nx - 2) i0 = P.nx - 2;
        if (j0 > P.ny - 2) j0 = P.ny - 2;
        const float fx = (float)(px - i0), fy = (float)(py - j0);
        const float v = (1.0f - fx) * (1.0f - fy) * phi_at_f<Store>(P, sc, i0, j0) +
                        fx * (1.0f - fy) * phi_at_f<Store>(P, sc, i0 + 1, j0) +
                        (1.0f - fx) * fy * phi_at_f<Store>(P, sc, i0, j0 + 1) +
                        fx * fy * phi_at_f<Store>(P, sc, i0 + 1, j0 + 1);
        if (v > 0.0f) last = max(last, j);
    }
    __shared__ int s_last[kTipThreads / 32], s_out[kTipThreads / 32];
    __shared__ int c_last, c_out;  // this CTA's result, read by rank 0
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        last = max(last, __shfl_down_sync(0xffffffffu, last, d));
        first_out = min(first_out, __shfl_down_sync(0xffffffffu, first_out, d));
    }
    if ((threadIdx.x & 31) == 0) {
        s_last[threadIdx.x >> 5] = last;
        s_out[threadIdx.x >> 5] = first_out;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kTipThreads / 32; ++w) {
            last = max(last, s_last[w]);
            first_out = min(first_out, s_out[w]);
        }
        c_last = last;
        c_out = first_out;
    }
    cluster.sync();
    if (rank == 0 && threadIdx.x == 0) {
        for (int q = 1; q < kTipCluster; ++q) {
            last = max(last, *cluster.map_shared_rank(&c_last, q));
            first_out = min(first_out, *cluster.map_shared_rank(&c_out, q));
        }
        // samples past the first outside one never count (the ray leaves a
        // rectangle once), so clip `last` to the inside run
        double tip;
        if (last < 0 || last >= first_out) {
            tip = nan("");
        } else if (last + 1 >= first_out) {
            tip = last * 0.5;
        } else {
            const double v0 = phi_bilinear<Store>(P, sc, cx + last * 0.5 * ex, cy + last * 0.5 * ey);
            const double v1 = phi_bilinear<Store>(P, sc, cx + (last + 1) * 0.5 * ex, cy + (last + 1) * 0.5 * ey);
            tip = (last + v0 / (v0 - v1)) * 0.5;
        }
        out[7 + r] = tip;
    }
    cluster.sync();  // rank 0 has read the other CTAs' shared memory
}

template <class Store>
cudaError_t init_t(const StepParams& P, const double* fields, void* sc, void* fl, float* hist, int y0, int rows,
                   cudaStream_t s)
{
    const dim3 b(64, 4), g((P.nx + 63) / 64, (rows + 3) / 4);
    k_init<Store><<<g, b, 0, s>>>(P, fields, sc, fl, hist, y0, rows);
    return cudaGetLastError();
}

template <class Store>
cudaError_t fields_nhwc_t(const StepParams& P, const void* sc, const void* fl, float inv_vf, float* dst,
                          cudaStream_t s)
{
    const dim3 b(64, 4), g((P.nx + 63) / 64, (P.ny + 3) / 4);
    k_fields_nhwc<Store><<<g, b, 0, s>>>(P, sc, fl, inv_vf, dst);
    return cudaGetLastError();
}

template <class Store>
cudaError_t set_fields_nhwc_t(const StepParams& P, const float* src, float vf, void* sc, void* fl, float* hist,
                              const float* prev, int K, cudaStream_t s)
{
    const dim3 b(64, 4), g((P.nx + 63) / 64, (P.ny + 3) / 4);
    k_set_fields_nhwc<Store><<<g, b, 0, s>>>(P, src, vf, sc, fl, hist, prev, 1.0f / (float)(K > 0 ? K : 1));
    return cudaGetLastError();
}

template <class Store>
cudaError_t macros_t(const StepParams& P, const void* sc, const void* fl, float* out, int y0, int rows,
                     cudaStream_t s)
{
    const dim3 b(64, 4), g((P.nx + 63) / 64, (rows + 3) / 4);
    k_macros<Store><<<g, b, 0, s>>>(P, sc, fl, out, y0, rows);
    return cudaGetLastError();
}

template <class Store>
cudaError_t fields_f32_t(const StepParams& P, const void* sc, const void* fl, const FieldsF32& spec, float* out,
                         int y0, int rows, cudaStream_t s)
{
    const dim3 b(64, 4), g((P.nx + 63) / 64, (rows + 3) / 4);
    k_fields_f32<Store><<<g, b, 0, s>>>(P, sc, fl, spec, out, y0, rows);
    return cudaGetLastError();
}

template <class Store>
cudaError_t decode_t(const StepParams& P, const void* sc, const void* fl, const float* hist, float* out, int y0,
                     int rows, cudaStream_t s)
{
    const long long n = (long long)rows * P.pitch;
    k_decode<Store><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(P, sc, fl, hist, out, y0, rows);
    return cudaGetLastError();
}

template <class Store>
cudaError_t encode_t(const StepParams& P, const float* in, void* sc, void* fl, float* hist, int y0, int rows,
                     cudaStream_t s)
{
    const long long n = (long long)rows * P.pitch;
    k_encode<Store><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(P, in, sc, fl, hist, y0, rows);
    return cudaGetLastError();
}

template <class Store>
cudaError_t reduce_t(const StepParams& P, const void* sc, const void* fl, double cx, double cy, double c, double s,
                     double* partials, double* out, cudaStream_t st)
{
    const int nb = reduce_blocks(P);
    k_reduce_nodes<Store><<<nb, kRedThreadsPerBlock, 0, st>>>(P, sc, fl, partials);
    k_reduce_final<<<1, 32 * kRedVals, 0, st>>>(partials, nb, out);
    k_tips<Store><<<3 * kTipCluster, kTipThreads, 0, st>>>(P, sc, cx, cy, c, s, out);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_seed_fields(const StepParams& P, const double* seeds, int ns, double U0, double theta0, double W,
                               double* fields, uint8_t* grain, int y0, int rows, cudaStream_t s)
{
    const dim3 b(64, 4), g((P.nx + 63) / 64, (rows + 3) / 4);
    k_seed_fields<<<g, b, 0, s>>>(P, seeds, ns, U0, theta0, W, fields, grain, y0, rows);
    return cudaGetLastError();
}

cudaError_t launch_init_from_fields(const StepParams& P, int storage, const double* fields, void* sc, void* fl,
                                    float* hist, int y0, int rows, cudaStream_t s)
{
    switch (storage) {
    case kStoreF16: return init_t<StoreF16>(P, fields, sc, fl, hist, y0, rows, s);
    case kStoreBF16: return init_t<StoreBF16>(P, fields, sc, fl, hist, y0, rows, s);
    default: return init_t<StoreF32>(P, fields, sc, fl, hist, y0, rows, s);
    }
}

cudaError_t launch_fields_nhwc(const StepParams& P, int storage, const void* sc, const void* fl, float inv_vf,
                               float* dst, cudaStream_t s)
{
    switch (storage) {
    case kStoreF16: return fields_nhwc_t<StoreF16>(P, sc, fl, inv_vf, dst, s);
    case kStoreBF16: return fields_nhwc_t<StoreBF16>(P, sc, fl, inv_vf, dst, s);
    default: return fields_nhwc_t<StoreF32>(P, sc, fl, inv_vf, dst, s);
    }
}

cudaError_t launch_set_fields_nhwc(const StepParams& P, int storage, const float* src, float vf, void* sc, void* fl,
                                   float* hist, const float* prev, int K, cudaStream_t s)
{
    switch (storage) {
    case kStoreF16: return set_fields_nhwc_t<StoreF16>(P, src, vf, sc, fl, hist, prev, K, s);
    case kStoreBF16: return set_fields_nhwc_t<StoreBF16>(P, src, vf, sc, fl, hist, prev, K, s);
    default: return set_fields_nhwc_t<StoreF32>(P, src, vf, sc, fl, hist, prev, K, s);
    }
}

cudaError_t launch_force(const StepParams& P, int storage, const void* sc, const void* fl, double cx, double cy,
                         double* partials, double* out, cudaStream_t st)
{
    const int nb = reduce_blocks(P);
    switch (storage) {
    case kStoreF16: k_force<StoreF16><<<nb, kRedThreads, 0, st>>>(P, sc, fl, cx, cy, partials); break;
    case kStoreBF16: k_force<StoreBF16><<<nb, kRedThreads, 0, st>>>(P, sc, fl, cx, cy, partials); break;
    default: k_force<StoreF32><<<nb, kRedThreads, 0, st>>>(P, sc, fl, cx, cy, partials); break;
    }
    k_force_final<<<1, 32, 0, st>>>(partials, nb, out);
    return cudaGetLastError();
}

cudaError_t launch_flow_inputs(const StepParams& P, int storage, const void* sc, const void* fl, float* phi, float* fy,
                               cudaStream_t st)
{
    const dim3 b(64, 4), g((P.nx + 63) / 64, (P.ny + 3) / 4);
    switch (storage) {
    case kStoreF16: k_flow_inputs<StoreF16><<<g, b, 0, st>>>(P, sc, fl, phi, fy); break;
    case kStoreBF16: k_flow_inputs<StoreBF16><<<g, b, 0, st>>>(P, sc, fl, phi, fy); break;
    default: k_flow_inputs<StoreF32><<<g, b, 0, st>>>(P, sc, fl, phi, fy); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_count_nonfinite(const float* a, long long n, unsigned long long* out, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    long long blocks = (n + 255) / 256;
    if (blocks > 1216) blocks = 1216;
    if (blocks < 1) blocks = 1;
    k_count_nonfinite<<<(unsigned)blocks, 256, 0, s>>>(a, n, out);
    return cudaGetLastError();
}

cudaError_t launch_phi_mismatch(const float* a, const float* b, long long n, unsigned long long* out, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(out, 0, 2 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    long long blocks = (n + 255) / 256;
    if (blocks > 1216) blocks = 1216;
    if (blocks < 1) blocks = 1;
    k_phi_mismatch<<<(unsigned)blocks, 256, 0, s>>>(a, b, n, out);
    return cudaGetLastError();
}

cudaError_t launch_macros(const StepParams& P, int storage, const void* sc, const void* fl, float* out, int y0,
                          int rows, cudaStream_t s)
{
    switch (storage) {
    case kStoreF16: return macros_t<StoreF16>(P, sc, fl, out, y0, rows, s);
    case kStoreBF16: return macros_t<StoreBF16>(P, sc, fl, out, y0, rows, s);
    default: return macros_t<StoreF32>(P, sc, fl, out, y0, rows, s);
    }
}

cudaError_t launch_fields_f32(const StepParams& P, int storage, const void* sc, const void* fl,
                              const FieldsF32& spec, float* out, int y0, int rows, cudaStream_t s)
{
    switch (storage) {
    case kStoreF16: return fields_f32_t<StoreF16>(P, sc, fl, spec, out, y0, rows, s);
    case kStoreBF16: return fields_f32_t<StoreBF16>(P, sc, fl, spec, out, y0, rows, s);
    default: return fields_f32_t<StoreF32>(P, sc, fl, spec, out, y0, rows, s);
    }
}

cudaError_t launch_decode(const StepParams& P, int storage, const void* sc, const void* fl, const float* hist,
                          float* out, int y0, int rows, cudaStream_t s)
{
    switch (storage) {
    case kStoreF16: return decode_t<StoreF16>(P, sc, fl, hist, out, y0, rows, s);
    case kStoreBF16: return decode_t<StoreBF16>(P, sc, fl, hist, out, y0, rows, s);
    default: return decode_t<StoreF32>(P, sc, fl, hist, out, y0, rows, s);
    }
}

cudaError_t launch_encode(const StepParams& P, int storage, const float* in, void* sc, void* fl, float* hist, int y0,
                          int rows, cudaStream_t s)
{
    switch (storage) {
    case kStoreF16: return encode_t<StoreF16>(P, in, sc, fl, hist, y0, rows, s);
    case kStoreBF16: return encode_t<StoreBF16>(P, in, sc, fl, hist, y0, rows, s);
    default: return encode_t<StoreF32>(P, in, sc, fl, hist, y0, rows, s);
    }
}

int reduce_blocks(const StepParams& P) { return (int)reduce_chunk_blocks((long long)P.nx * P.ny); }

size_t reduce_partials_size(const StepParams& P) { return (size_t)reduce_blocks(P) * kRedVals; }

cudaError_t launch_reduce(const StepParams& P, int storage, const void* sc, const void* fl, double cx, double cy,
                          double c, double s, double* partials, double* out, cudaStream_t st)
{
    switch (storage) {
    case kStoreF16: return reduce_t<StoreF16>(P, sc, fl, cx, cy, c, s, partials, out, st);
    case kStoreBF16: return reduce_t<StoreBF16>(P, sc, fl, cx, cy, c, s, partials, out, st);
    default: return reduce_t<StoreF32>(P, sc, fl, cx, cy, c, s, partials, out, st);
    }
}

cudaError_t launch_reduce_final(const double* partials, int nblocks, double* out, cudaStream_t st)
{
    k_reduce_final<<<1, 32 * kRedVals, 0, st>>>(partials, nblocks, out);
    return cudaGetLastError();
}

cudaError_t launch_tips(const StepParams& P, int storage, const void* sc, double cx, double cy, double c, double s,
                        double* out, cudaStream_t st)
{
    switch (storage) {
    case kStoreF16: k_tips<StoreF16><<<3 * kTipCluster, kTipThreads, 0, st>>>(P, sc, cx, cy, c, s, out); break;
    case kStoreBF16: k_tips<StoreBF16><<<3 * kTipCluster, kTipThreads, 0, st>>>(P, sc, cx, cy, c, s, out); break;
    default: k_tips<StoreF32><<<3 * kTipCluster, kTipThreads, 0, st>>>(P, sc, cx, cy, c, s, out); break;
    }
    return cudaGetLastError();
}

}  // namespace lbm
