// Device-side building blocks of the coupled MRT lattice Boltzmann step
// (arXiv 2209.01444): storage codecs, node macros, anisotropy and the four
// collisions written in moment space.  Everything here is FP32 arithmetic.
//
// Lattices (Appendix B):
//   D2Q5  directions 0:(0,0) 1:(1,0) 2:(0,1) 3:(-1,0) 4:(0,-1), weights 1/3, 1/6
//         (forced by cs^2 = 1/3), moments m = (sum f, f1 - f3, f2 - f4, f1 + f3,
//         f2 + f4) = M f of Eq. (B.1);
//   D2Q9  directions 0..4 as above, 5:(1,1) 6:(-1,1) 7:(-1,-1) 8:(1,-1),
//         raw moments of Eq. (B.2).
// Relaxation: D2Q5 S = diag(1, s1, s1, 1, 1); D2Q9 S = diag(1, 1, 1, s2, s2,
// s2, 1, 1, 1) (Sec. 4: every rate not tied to a transport coefficient is 1).
//
// Deviation form.  Every population is held as its deviation d_i = f_i -
// f_i^ref from the equilibrium of a constant reference state, the liquid at
// rest (phi = -1, C = 1 so U = 0, theta = theta_ref, u = 0, p = 0):
//   phi:  f^ref = (-1/3, -1/6, -1/6, -1/6, -1/6)       (sum -1)
//   C:    n^ref = (1, 0, 0, 0, 0)                       (sum 1)
//   H:    g^ref = (theta_ref/3 + L, theta_ref/6 x 4)    (sum theta_ref + L)
//   flow: h^ref = (rho0, 0, ..., 0)                     (sum rho0)
// The references are isotropic, so first moments are unchanged and the macro
// (L = 1/2 is the latent-heat factor of H = theta - h(phi)/2, Eq. 21; L = 0
// in the isothermal mode, where H = theta).  The macro
// deviations phi + 1, C - 1, theta - theta_ref follow from sums of small
// numbers without cancellation; the MRT collision and the modified streaming
// of Eq. (13) are linear and carry over unchanged to deviations.  16-bit
// storage rounds the same deviations.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>
#include <string.h>

namespace lbm {

constexpr int TX = 32;  // tile width of the fused kernel (one warp along x)
constexpr int TY = 4;   // tile height: four warps per CTA, so that fewer warps wait at each tile
                        // barrier than with eight (measured faster in every storage format)
constexpr float kGradEps2 = 1e-12f;  // |grad phi|^2 below which n, N, J_at vanish

// Population slot of model/direction q: phi 0..4, C 5..9, H 10..14, flow 15..23.
constexpr int kF = 0, kN = 5, kG = 10, kH = 15, kPlanes = 24;
// History planes: phi, Q, (Cu)_x, (Cu)_y, (Hu)_x, (Hu)_y.
constexpr int kHist = 6;

struct StepParams {
    int nx, ny, pitch;
    long long plane;          // elements per plane (pitch * ny)
    int periodic_x, periodic_y;
    int h_kind;
    int grad_local;           // 0: nine-point stencil, 1: local scheme of Sec. 3.1
    float kappa3;             // 3 W0^2/tau0: s1^phi = 1/(kappa3 a_s^2 + 1/2)
    float inv_tau;            // 1/tau0 (lattice)
    float eps;                // anisotropy strength
    float lambda, k, Mc;      // Eq. (5), Eq. (20)
    float W;                  // W0 in lattice units
    float inv_D;              // 1/D (lattice)
    float s1C, s1T, s2u;      // relaxation rates of Sec. 4
    float rho0;
    float Fx, Fy, gbT, gbC;   // body force and buoyancy (flow lattice units)
    float theta_ref;          // buoyancy reference = reference state of the deviations
    float latent;             // L in H = theta - L h(phi): 1/2 (Eq. 21), 0 when isothermal
    float dC_ref;             // 1 - C_ref: buoyancy offset of the solute term
    float nsub;               // flow-lattice velocity -> scalar-lattice velocity
    float cos_o, sin_o;       // orientation when the whole domain is one grain
    const float2* grain_cs;   // (cos, sin) per grain id
    // boundary data
    int bc[4];
    float uin_x, uin_y;
    float dir_phi, dir_U, dir_theta;
};

// ------------------------------------------------------------------ layout
// Node blocks.  Every per-node buffer (populations, history) keeps its values
// in blocks of 32 nodes along x: node o = y * pitch + x (pitch a multiple of
// 32, so no block spans two rows) is lane o & 31 of block o >> 5, and the
// block holds plane q of its 32 nodes contiguously at [block][q][lane].  A
// warp's 32 nodes still read or write each plane as one contiguous segment,
// and all planes of one node lie in one block: a kernel forms one address per
// node and reaches every plane at a compile-time offset from it.
// Element index of plane 0 of node o in a buffer of np planes per block.
__device__ __forceinline__ long long block_index(long long o, int np)
{
    return (long long)((unsigned long long)(unsigned)(o >> 5) * (unsigned)(np * 32)) + (long long)(o & 31);
}

// The same index split into a row term and a column term, so that the
// pushes of one node to its neighbours share three row and three column terms:
// block_index(y * pitch + x, np) = block_row(y, pitch, np) + block_col(x, np).
// (Grids hold fewer than 2^31 nodes, so y * pitch / 32 fits in 32 bits.)
__device__ __forceinline__ long long block_row(int y, int pitch, int np)
{
    return (long long)((unsigned long long)(unsigned)(y * (pitch >> 5)) * (unsigned)(np * 32));
}
__device__ __forceinline__ int block_col(int x, int np) { return (x >> 5) * (np * 32) + (x & 31); }

// History value k (phi, Q, (Cu)_x, (Cu)_y, (Hu)_x, (Hu)_y) of node o.
__device__ __forceinline__ float& hist_at(float* hist, int k, long long o)
{
    return hist[block_index(o, kHist) + 32 * k];
}
__device__ __forceinline__ float hist_at(const float* hist, int k, long long o)
{
    return hist[block_index(o, kHist) + 32 * k];
}

// ------------------------------------------------------------------ codecs
// A state is two buffers: the scalar populations (phi, C, H) and the flow
// populations, each in node blocks.  FP32 storage keeps all 15 scalar planes
// in FP32.  16-bit storage keeps the 12 moving scalar planes and the 9 flow
// planes in FP16 or BF16 (scaled, rounded to nearest even) and the three
// scalar rest planes (q = 0, 5, 10), which carry the O(1) solid/liquid
// contrast and the smallest per-step increments, in FP32: a scalar block is
// 12 x 32 16-bit values followed by 3 x 32 FP32 values (1152 bytes).  q is
// always a compile-time constant at the call sites, so the plane mapping
// folds into address offsets.
struct StoreF32 {
    using T = float;
    static constexpr int kScalarBytes = 15 * 4;  // per node
    static constexpr int kFlowBytes = 9 * 4;
    static constexpr int kSS = 1, kSF = 1;       // scales of the moving scalar and the flow planes
    static __device__ __forceinline__ float load(const void* sc, const void* fl, int q, long long o,
                                                 const StepParams& P)
    {
        return q < kH ? ((const float*)sc)[block_index(o, 15) + 32 * q]
                      : ((const float*)fl)[block_index(o, 9) + 32 * (q - kH)];
    }
    static __device__ __forceinline__ void store(void* sc, void* fl, int q, long long o, float v,
                                                 const StepParams& P)
    {
        if (q < kH)
            ((float*)sc)[block_index(o, 15) + 32 * q] = v;
        else
            ((float*)fl)[block_index(o, 9) + 32 * (q - kH)] = v;
    }
    // Pushes: element index of node (x, y) in the moving scalar planes
    // (row + column terms) and in the flow buffer; q a moving scalar plane.
    static __device__ __forceinline__ long long mov_row(int y, const StepParams& P) { return block_row(y, P.pitch, 15); }
    static __device__ __forceinline__ int mov_col(int x) { return block_col(x, 15); }
    static __device__ __forceinline__ long long flow_row(int y, const StepParams& P) { return block_row(y, P.pitch, 9); }
    static __device__ __forceinline__ int flow_col(int x) { return block_col(x, 9); }
    static __device__ __forceinline__ void store_mov(void* sc, int q, long long e, float v) { ((float*)sc)[e + 32 * q] = v; }
    static __device__ __forceinline__ void store_flow(void* fl, int i, long long e, float v) { ((float*)fl)[e + 32 * i] = v; }
    static __device__ __forceinline__ float load_flow(const void* fl, int i, long long o)
    {
        return ((const float*)fl)[block_index(o, 9) + 32 * i];
    }
    // n_i and g_i (i = 1..4), which stream to the same neighbour: the moving
    // scalar index serves both (16-bit storage keeps them in one word)
    static __device__ __forceinline__ long long pair_row(int y, const StepParams& P) { return mov_row(y, P); }
    static __device__ __forceinline__ int pair_col(int x) { return mov_col(x); }
    static __device__ __forceinline__ void load_pair(const void* sc, int i, long long o, float& n, float& g)
    {
        const long long b = block_index(o, 15);
        n = ((const float*)sc)[b + 32 * (kN + i)];
        g = ((const float*)sc)[b + 32 * (kG + i)];
    }
    static __device__ __forceinline__ void store_pair(void* sc, int i, long long e, float n, float g)
    {
        ((float*)sc)[e + 32 * (kN + i)] = n;
        ((float*)sc)[e + 32 * (kG + i)] = g;
    }
};

template <class H>
struct Conv;
template <>
struct Conv<__half> {
    static __device__ __forceinline__ float to(__half v) { return __half2float(v); }
    static __device__ __forceinline__ __half from(float v) { return __float2half_rn(v); }
    // a 32-bit word of two values (low half first)
    static __device__ __forceinline__ float2 to2(uint32_t w)
    {
        __half2 h;
        memcpy(&h, &w, 4);
        return __half22float2(h);
    }
    static __device__ __forceinline__ uint32_t from2(float a, float b)
    {
        const __half2 h = __floats2half2_rn(a, b);
        uint32_t w;
        memcpy(&w, &h, 4);
        return w;
    }
};
template <>
struct Conv<__nv_bfloat16> {
    static __device__ __forceinline__ float to(__nv_bfloat16 v) { return __bfloat162float(v); }
    static __device__ __forceinline__ __nv_bfloat16 from(float v) { return __float2bfloat16_rn(v); }
    static __device__ __forceinline__ float2 to2(uint32_t w)
    {
        __nv_bfloat162 h;
        memcpy(&h, &w, 4);
        return __bfloat1622float2(h);
    }
    static __device__ __forceinline__ uint32_t from2(float a, float b)
    {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        uint32_t w;
        memcpy(&w, &h, 4);
        return w;
    }
};

// S_SC, S_FL: power-of-two scales of the scalar and flow deviations before
// rounding (FP16 keeps the smallest deviations out of its subnormal range).
// A scalar block (1152 bytes = 288 32-bit words) holds, for its 32 nodes:
// words 0..63 the phase-field planes f_1..f_4 in 16 bits (f_i at 16-bit index
// 32 (i - 1) + lane); words 64..191 the pairs (n_i, g_i), i = 1..4, one word
// per node (n in the low half; pair i at word 64 + 32 (i - 1) + lane), since
// both go to the same neighbour; words 192..287 the FP32 rest planes f_0,
// n_0, g_0 (word 192 + 32 r + lane).
// load/store take and give deviations.  The push stores (store_mov,
// store_pair, store_flow) take, and load_pair and load_flow give, values in
// units of the plane's scale (kSS for the moving scalar planes, kSF for the
// flow planes): the fused step folds the scale into the constants of its
// moment transforms, which is exact for a power of two.
template <class H, int S_SC, int S_FL>
struct Store16 {
    using T = H;
    static constexpr int kSS = S_SC, kSF = S_FL;
    static __device__ __forceinline__ float scale(int q) { return q >= kH ? (float)S_FL : (float)S_SC; }
    static __device__ __forceinline__ float inv_scale(int q) { return q >= kH ? 1.0f / S_FL : 1.0f / S_SC; }
    static constexpr int kScalarBytes = 12 * 2 + 3 * 4;
    static constexpr int kFlowBytes = 9 * 2;
    static __device__ __forceinline__ bool rest(int q) { return q == kF || q == kN || q == kG; }
    // word index of word 0 of node o's block plus its lane
    static __device__ __forceinline__ long long word_index(long long o)
    {
        return (long long)((unsigned long long)(unsigned)(o >> 5) * 288u) + (long long)(o & 31);
    }
    // 16-bit index of f_1 of node o
    static __device__ __forceinline__ long long moving_index(long long o)
    {
        return (long long)((unsigned long long)(unsigned)(o >> 5) * 576u) + (long long)(o & 31);
    }
    // 16-bit index of the value of scalar population q (moving, not rest) of node o
    static __device__ __forceinline__ long long half_index(int q, long long o)
    {
        if (q < kN) return moving_index(o) + 32 * (q - 1);
        const int i = q < kG ? q - kN : q - kG;
        return 2 * (word_index(o) + 64 + 32 * (i - 1)) + (q < kG ? 0 : 1);
    }
    static __device__ __forceinline__ float load(const void* sc, const void* fl, int q, long long o,
                                                 const StepParams& P)
    {
        if (q >= kH) return Conv<H>::to(((const H*)fl)[block_index(o, 9) + 32 * (q - kH)]) * inv_scale(q);
        if (rest(q)) return ((const float*)sc)[word_index(o) + 192 + 32 * (q / 5)];
        return Conv<H>::to(((const H*)sc)[half_index(q, o)]) * inv_scale(q);
    }
    static __device__ __forceinline__ void store(void* sc, void* fl, int q, long long o, float v,
                                                 const StepParams& P)
    {
        if (q >= kH)
            ((H*)fl)[block_index(o, 9) + 32 * (q - kH)] = Conv<H>::from(v * scale(q));
        else if (rest(q))
            ((float*)sc)[word_index(o) + 192 + 32 * (q / 5)] = v;
        else
            ((H*)sc)[half_index(q, o)] = Conv<H>::from(v * scale(q));
    }
    // pushes: the moving phase-field planes (16-bit index, row + column terms),
    // the (n_i, g_i) words (word index) and the flow planes
    static __device__ __forceinline__ long long mov_row(int y, const StepParams& P)
    {
        return (long long)((unsigned long long)(unsigned)(y * (P.pitch >> 5)) * 576u);
    }
    static __device__ __forceinline__ int mov_col(int x) { return (x >> 5) * 576 + (x & 31); }
    static __device__ __forceinline__ long long pair_row(int y, const StepParams& P)
    {
        return (long long)((unsigned long long)(unsigned)(y * (P.pitch >> 5)) * 288u);
    }
    static __device__ __forceinline__ int pair_col(int x) { return (x >> 5) * 288 + (x & 31) + 64; }
    static __device__ __forceinline__ long long flow_row(int y, const StepParams& P) { return block_row(y, P.pitch, 9); }
    static __device__ __forceinline__ int flow_col(int x) { return block_col(x, 9); }
    static __device__ __forceinline__ void store_mov(void* sc, int q, long long e, float vs)  // q = f_1..f_4
    {
        ((H*)sc)[e + 32 * (q - 1)] = Conv<H>::from(vs);
    }
    static __device__ __forceinline__ void store_flow(void* fl, int i, long long e, float vs)
    {
        ((H*)fl)[e + 32 * i] = Conv<H>::from(vs);
    }
    static __device__ __forceinline__ float load_flow(const void* fl, int i, long long o)
    {
        return Conv<H>::to(((const H*)fl)[block_index(o, 9) + 32 * i]);
    }
    static __device__ __forceinline__ void load_pair(const void* sc, int i, long long o, float& ns, float& gs)
    {
        const float2 v = Conv<H>::to2(((const uint32_t*)sc)[word_index(o) + 64 + 32 * (i - 1)]);
        ns = v.x;
        gs = v.y;
    }
    static __device__ __forceinline__ void store_pair(void* sc, int i, long long e, float ns, float gs)
    {
        ((uint32_t*)sc)[e + 32 * (i - 1)] = Conv<H>::from2(ns, gs);
    }
};
using StoreF16 = Store16<__half, 16, 1024>;
using StoreBF16 = Store16<__nv_bfloat16, 1, 1>;

__device__ __forceinline__ int wrap(int v, int n)
{
    v %= n;
    return v < 0 ? v + n : v;
}

// h(phi) + 1 as a function of p = phi + 1 (Sec. 2): kind 0 is h = phi, kind 1
// is 15/8 (phi - 2 phi^3/3 + phi^5/5), whose h + 1 = 15/8 p^3 (4/3 - p + p^2/5).
__device__ __forceinline__ float h_plus_1(int kind, float p)
{
    if (kind == 1) return 1.875f * p * p * p * (4.0f / 3.0f - p + 0.2f * p * p);
    return p;
}

// Eq. (20) with C = 1 + dC and phi = p - 1:
// U = [2C/(1 + k - (1 - k) phi) - 1]/(1 - k) = (2 dC + (1 - k) p) / ((2 - (1 - k) p)(1 - k)).
// (The denominator is at least 2k(1 - k) for p in [0, 2]: the fast division,
// within 2 ulp, is safe and saves the exact division's instruction sequence.)
__device__ __forceinline__ float U_of(float dC, float p, float k)
{
    return __fdividef(2.0f * dC + (1.0f - k) * p, (2.0f - (1.0f - k) * p) * (1.0f - k));
}
// Its inverse: C - 1 = (2 - (1 - k) p)(1 + (1 - k) U)/2 - 1.
__device__ __forceinline__ float dC_of(float U, float p, float k)
{
    return 0.5f * (2.0f - (1.0f - k) * p) * (1.0f - k) * U - 0.5f * (1.0f - k) * p;
}

// Eq. (5).
__device__ __forceinline__ float coupling_Q(float phi, float theta, float U, const StepParams& P)
{
    float w = 1.0f - phi * phi;
    return phi * w - P.lambda * (theta + P.Mc * U) * w * w;
}

// Macroscopic values of one node from its 24 population deviations
// (Eqs. 15, 20, 23, 26).
struct Macro {
    float p1;             // phi + 1
    float phi, dC, U, dth, hp1;   // phi, C - 1, U, theta - theta_ref, h(phi) + 1
    float H, dH;          // H = theta - L h(phi) and its deviation H - (theta_ref + L)
    float ux, uy, p;      // corrected velocity and pressure (flow lattice units)
    float Fx, Fy;         // external force F (flow lattice units)
    float fsx, fsy;       // fluid-solid force f = -u*
};

// SN, SF: n_1..n_4, g_1..g_4 given in units of 1/SN, h in units of 1/SF (a
// power of two, so every sum below equals the unscaled one bit for bit).
template <int SN, int SF>
__device__ __forceinline__ float scaled_rest_sum(const float* v)
{
    if constexpr (SN == 1) {
        return v[0] + v[1] + v[2] + v[3] + v[4];
    } else {
        constexpr float iN = 1.0f / SN;
        return fmaf(v[4], iN, fmaf(v[3], iN, fmaf(v[2], iN, fmaf(v[1], iN, v[0]))));
    }
}

template <int SN = 1, int SF = 1>
__device__ __forceinline__ Macro node_macros(const float* f, const float* n, const float* g, const float* h,
                                             const StepParams& P)
{
    constexpr float iF = 1.0f / SF;
    Macro m;
    m.p1 = f[0] + f[1] + f[2] + f[3] + f[4];
    m.phi = m.p1 - 1.0f;
    m.dC = scaled_rest_sum<SN, SF>(n);
    const float dH = scaled_rest_sum<SN, SF>(g);
    m.hp1 = h_plus_1(P.h_kind, m.p1);
    m.dth = dH + P.latent * m.hp1;             // theta = H + L h
    m.dH = dH;
    m.H = (P.theta_ref + P.latent) + dH;
    m.U = U_of(m.dC, m.p1, P.k);
    m.Fx = P.Fx;
    m.Fy = P.Fy + P.gbT * m.dth + P.gbC * (m.dC + P.dC_ref);
    float jx = (h[1] - h[3] + h[5] - h[6] - h[7] + h[8]) * iF;
    float jy = (h[2] - h[4] + h[5] + h[6] - h[7] - h[8]) * iF;
    float rest = (h[1] + h[2] + h[3] + h[4] + h[5] + h[6] + h[7] + h[8]) * iF;
    float usx = jx + 0.5f * m.Fx, usy = jy + 0.5f * m.Fy;   // u*
    float qt = 1.0f - 0.5f * m.p1;                         // q~ = (1 - phi)/2
    m.fsx = -usx;
    m.fsy = -usy;
    m.ux = usx + 0.5f * (1.0f - qt) * m.fsx;
    m.uy = usy + 0.5f * (1.0f - qt) * m.fsy;
    // p = cs^2/(1 - w0) (sum_{i!=0} h_i - w0 |u|^2/(2 cs^2)) with w0 = 4/9
    m.p = 0.6f * (rest - (2.0f / 3.0f) * (m.ux * m.ux + m.uy * m.uy));
    return m;
}

// Eqs. (2)-(3) for the gradient (gx, gy) of a grain rotated by (c, s):
// a_s and the anisotropic vector N in lattice axes.
__device__ __forceinline__ void anisotropy(float gx, float gy, float eps, float c, float s, float& as, float& Nx,
                                           float& Ny)
{
    float px = c * gx + s * gy;
    float py = -s * gx + c * gy;
    float px2 = px * px, py2 = py * py;
    float m2 = px2 + py2;
    if (m2 < kGradEps2) {
        as = 1.0f;
        Nx = 0.0f;
        Ny = 0.0f;
        return;
    }
    float inv = __fdividef(1.0f, m2 * m2);  // m2^2 in [1e-24, 1e20]: fast division within 2 ulp
    float a = 1.0f - 3.0f * eps + 4.0f * eps * (px2 * px2 + py2 * py2) * inv;
    float t = 16.0f * eps * a * px * py * (px2 - py2) * inv;  // N'_x = t py, N'_y = -t px
    float nx_ = t * py, ny_ = -t * px;
    Nx = c * nx_ - s * ny_;
    Ny = s * nx_ + c * ny_;
    as = a;
}

// ------------------------------------------------------------- equilibria
// Deviation of the population-form equilibria from the reference state (used
// by initialisation and the wall scheme).
// Eq. (14): w_i phi - w_i (-1) = w_i (phi + 1).
__device__ __forceinline__ void deq_phi(float p1, float* e)
{
    e[0] = p1 * (1.0f / 3.0f);
    e[1] = e[2] = e[3] = e[4] = p1 * (1.0f / 6.0f);
}
// Eq. (19) with qU = q~ U and (jx, jy) = C u.
__device__ __forceinline__ void deq_C(float dC, float qU, float jx, float jy, float* e)
{
    e[0] = dC - (2.0f / 3.0f) * qU;
    float b = qU * (1.0f / 6.0f);
    e[1] = b + 0.5f * jx;
    e[3] = b - 0.5f * jx;
    e[2] = b + 0.5f * jy;
    e[4] = b - 0.5f * jy;
}
// Eq. (22) with dth = theta - theta_ref, lhp1 = L (h(phi) + 1) and (jx, jy) = H u.
__device__ __forceinline__ void deq_H(float dth, float lhp1, float jx, float jy, float* e)
{
    e[0] = dth * (1.0f / 3.0f) - lhp1;
    float b = dth * (1.0f / 6.0f);
    e[1] = b + 0.5f * jx;
    e[3] = b - 0.5f * jx;
    e[2] = b + 0.5f * jy;
    e[4] = b - 0.5f * jy;
}
// Eq. (25): h_i^eq = sigma_i + w_i [3 c.u + 9/2 (c.u)^2 - 3/2 |u|^2], minus rho0 on i = 0.
__device__ __forceinline__ void deq_flow(float p, float ux, float uy, float* e)
{
    float uu = 1.5f * (ux * ux + uy * uy);
    e[0] = -(5.0f / 3.0f) * p - (4.0f / 9.0f) * uu;
    const float w1 = 1.0f / 9.0f, w5 = 1.0f / 36.0f;
    float cx[4] = {ux, uy, -ux, -uy};
#pragma unroll
    for (int i = 0; i < 4; ++i) e[1 + i] = w1 * (3.0f * p + 3.0f * cx[i] + 4.5f * cx[i] * cx[i] - uu);
    float d[4] = {ux + uy, -ux + uy, -ux - uy, ux - uy};
#pragma unroll
    for (int i = 0; i < 4; ++i) e[5 + i] = w5 * (3.0f * p + 3.0f * d[i] + 4.5f * d[i] * d[i] - uu);
}

// ------------------------------------------------------------- collisions
// D2Q5 MRT with S = diag(1, s1, s1, 1, 1) on deviations.  Equilibrium moments
// (A, Bx, By, Cv/3, Cv/3) enter as the deviations dA = A - A_ref and
// dCv = Cv - Cv_ref of the reference state; (Gx, Gy) are the first moments of
// the auxiliary term, weighted by (1 - s1/2); S0 is an isotropic source added
// with weights w_i.  The post-collision deviations follow through the inverse
// of Eq. (B.1).  SI, SO: d_1..d_4 are given, and out_1..out_4 returned, in
// units of 1/SI and 1/SO (powers of two; d_0 and out_0 unscaled).
template <int SI = 1, int SO = 1>
__device__ __forceinline__ void collide_d2q5(const float* d, float dA, float Bx, float By, float dCv, float s1,
                                             float Gx, float Gy, float S0, float* out)
{
    constexpr float iI = 1.0f / SI, hO = 0.5f * SO;
    float m1 = (d[1] - d[3]) * iI, m2 = (d[2] - d[4]) * iI;
    float k1 = 1.0f - 0.5f * s1;
    float r1 = m1 - s1 * (m1 - Bx) + k1 * Gx;
    float r2 = m2 - s1 * (m2 - By) + k1 * Gy;
    float e = (dCv + S0) * (1.0f / 3.0f);   // deviation of each post-collision second moment
    out[0] = dA + S0 - 2.0f * e;
    out[1] = hO * (e + r1);
    out[3] = hO * (e - r1);
    out[2] = hO * (e + r2);
    out[4] = hO * (e - r2);
}

// D2Q9 raw-moment MRT of Eq. (24): m* = m - S (m - m^eq) + (I - S/2) m_F with
// m^eq and m_F of Eq. (B.3) (varphi = 0) and F' = F + [1 - q~] f; returns the
// post-collision deviations through the inverse of Eq. (B.2) (m0* = rho0).
// SI, SO: h given and out returned in units of 1/SI and 1/SO (powers of two).
template <int SI = 1, int SO = 1>
__device__ __forceinline__ void collide_flow(const float* h, const Macro& m, float s2, float* out)
{
    constexpr float iI = 1.0f / SI, hO = 0.5f * SO, qO = 0.25f * SO;
    float qt = 1.0f - 0.5f * m.p1;
    float Fpx = m.Fx + (1.0f - qt) * m.fsx;
    float Fpy = m.Fy + (1.0f - qt) * m.fsy;
    float u = m.ux, v = m.uy, p = m.p;
    // pre-collision second-order moments that relax with s2
    float mxx = (h[1] + h[3] + h[5] + h[6] + h[7] + h[8]) * iI;
    float myy = (h[2] + h[4] + h[5] + h[6] + h[7] + h[8]) * iI;
    float mxy = (h[5] - h[6] + h[7] - h[8]) * iI;
    // post-collision moments
    float r1 = u + 0.5f * Fpx;
    float r2 = v + 0.5f * Fpy;
    float r3 = mxx - s2 * (mxx - (p + u * u));
    float r4 = myy - s2 * (myy - (p + v * v));
    float r5 = mxy - s2 * (mxy - u * v);
    float r6 = (v + 0.5f * Fpy) * (1.0f / 3.0f);
    float r7 = (u + 0.5f * Fpx) * (1.0f / 3.0f);
    float r8 = (p + u * u + v * v) * (1.0f / 3.0f);
    // inverse of the tensor-product raw-moment matrix (r0 - rho0 = 0)
    if constexpr (SO == 1)
        out[0] = -r3 - r4 + r8;
    else
        out[0] = (float)SO * (-r3 - r4 + r8);
    out[1] = hO * (r1 + r3 - r7 - r8);
    out[3] = hO * (-r1 + r3 + r7 - r8);
    out[2] = hO * (r2 + r4 - r6 - r8);
    out[4] = hO * (-r2 + r4 + r6 - r8);
    out[5] = qO * (r5 + r6 + r7 + r8);
    out[6] = qO * (-r5 + r6 - r7 + r8);
    out[7] = qO * (r5 - r6 - r7 + r8);
    out[8] = qO * (-r5 - r6 + r7 + r8);
}

}  // namespace lbm
