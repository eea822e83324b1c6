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
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace lbm {

constexpr int TX = 32;  // tile width of the fused kernel (one warp along x)
constexpr int TY = 8;   // tile height
constexpr float kGradEps2 = 1e-12f;  // |grad phi|^2 below which n, N, J_at vanish

// Population slot of model/direction q in a state buffer of 24 planes:
// phi 0..4, C 5..9, H 10..14, flow 15..23.
constexpr int kF = 0, kN = 5, kG = 10, kH = 15, kPlanes = 24;
// History planes: phi, Q, (Cu)_x, (Cu)_y, (Hu)_x, (Hu)_y.
constexpr int kHist = 6;

struct StepParams {
    int nx, ny, pitch;
    long long plane;          // elements per plane (pitch * ny)
    int periodic_x, periodic_y;
    int h_kind;
    float kappa3;             // 3 W0^2/tau0: s1^phi = 1/(kappa3 a_s^2 + 1/2)
    float inv_tau;            // 1/tau0 (lattice)
    float eps;                // anisotropy strength
    float lambda, k, Mc;      // Eq. (5), Eq. (20)
    float W;                  // W0 in lattice units
    float inv_D;              // 1/D (lattice)
    float s1C, s1T, s2u;      // relaxation rates of Sec. 4
    float rho0;
    float Fx, Fy, gbT, gbC, theta_ref, C_ref;  // body force and buoyancy (flow lattice units)
    float nsub;               // flow-lattice velocity -> scalar-lattice velocity
    float cos_o, sin_o;       // orientation when the whole domain is one grain
    const float2* grain_cs;   // (cos, sin) per grain id
    // boundary data
    int bc[4];
    float uin_x, uin_y;
    float dir_phi, dir_U, dir_theta;
    // reduced-precision codec: reference equilibrium and scale per plane
    float ref[kPlanes];
    float scale[kPlanes], inv_scale[kPlanes];
};

// ------------------------------------------------------------------ codecs
// FP32 stores populations as they are; FP16/BF16 store s (f - f_ref).
struct StoreF32 {
    using T = float;
    static __device__ __forceinline__ float load(const T* p, long long i, int, const StepParams&) { return p[i]; }
    static __device__ __forceinline__ void store(T* p, long long i, int, float v, const StepParams&) { p[i] = v; }
};
struct StoreF16 {
    using T = __half;
    static __device__ __forceinline__ float load(const T* p, long long i, int q, const StepParams& P)
    {
        return P.ref[q] + __half2float(p[i]) * P.inv_scale[q];
    }
    static __device__ __forceinline__ void store(T* p, long long i, int q, float v, const StepParams& P)
    {
        p[i] = __float2half_rn((v - P.ref[q]) * P.scale[q]);
    }
};
struct StoreBF16 {
    using T = __nv_bfloat16;
    static __device__ __forceinline__ float load(const T* p, long long i, int q, const StepParams& P)
    {
        return P.ref[q] + __bfloat162float(p[i]) * P.inv_scale[q];
    }
    static __device__ __forceinline__ void store(T* p, long long i, int q, float v, const StepParams& P)
    {
        p[i] = __float2bfloat16_rn((v - P.ref[q]) * P.scale[q]);
    }
};

__device__ __forceinline__ int wrap(int v, int n)
{
    v %= n;
    return v < 0 ? v + n : v;
}

// h(phi) of Sec. 2.
__device__ __forceinline__ float h_of_phi(int kind, float phi)
{
    if (kind == 1) {
        float p2 = phi * phi;
        return 1.875f * phi * (1.0f - p2 * (2.0f / 3.0f) + p2 * p2 * 0.2f);
    }
    return phi;
}

// Eq. (20) and its inverse.
__device__ __forceinline__ float U_of_C(float C, float phi, float k)
{
    return (2.0f * C / (1.0f + k - (1.0f - k) * phi) - 1.0f) / (1.0f - k);
}
__device__ __forceinline__ float C_of_U(float U, float phi, float k)
{
    return 0.5f * (1.0f + k - (1.0f - k) * phi) * (1.0f + (1.0f - k) * U);
}

// Eq. (5).
__device__ __forceinline__ float coupling_Q(float phi, float theta, float U, const StepParams& P)
{
    float w = 1.0f - phi * phi;
    return phi * w - P.lambda * (theta + P.Mc * U) * w * w;
}

// Macroscopic values of one node from its 24 populations (Eqs. 15, 20, 23, 26).
struct Macro {
    float phi, C, U, theta, H;
    float ux, uy, p;      // corrected velocity and pressure (flow lattice units)
    float Fx, Fy;         // external force F (flow lattice units)
    float fsx, fsy;       // fluid-solid force f = -u*
};

__device__ __forceinline__ Macro node_macros(const float* f, const float* n, const float* g, const float* h,
                                             const StepParams& P)
{
    Macro m;
    m.phi = f[0] + f[1] + f[2] + f[3] + f[4];
    m.C = n[0] + n[1] + n[2] + n[3] + n[4];
    m.H = g[0] + g[1] + g[2] + g[3] + g[4];
    m.theta = m.H + 0.5f * h_of_phi(P.h_kind, m.phi);
    m.U = U_of_C(m.C, m.phi, P.k);
    m.Fx = P.Fx;
    m.Fy = P.Fy + P.gbT * (m.theta - P.theta_ref) + P.gbC * (m.C - P.C_ref);
    float jx = h[1] - h[3] + h[5] - h[6] - h[7] + h[8];
    float jy = h[2] - h[4] + h[5] + h[6] - h[7] - h[8];
    float rest = h[1] + h[2] + h[3] + h[4] + h[5] + h[6] + h[7] + h[8];
    float usx = jx + 0.5f * m.Fx, usy = jy + 0.5f * m.Fy;   // u*
    float qt = 0.5f * (1.0f - m.phi);
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
    float inv = 1.0f / (m2 * m2);
    float a = 1.0f - 3.0f * eps + 4.0f * eps * (px2 * px2 + py2 * py2) * inv;
    float t = 16.0f * eps * a * px * py * (px2 - py2) * inv;  // N'_x = t py, N'_y = -t px
    float nx_ = t * py, ny_ = -t * px;
    Nx = c * nx_ - s * ny_;
    Ny = s * nx_ + c * ny_;
    as = a;
}

// ------------------------------------------------------------- equilibria
// Population forms (used by initialisation and the wall scheme).
__device__ __forceinline__ void feq_phi(float phi, float* e)
{
    e[0] = phi * (1.0f / 3.0f);
    e[1] = e[2] = e[3] = e[4] = phi * (1.0f / 6.0f);
}
// Eq. (19) with qU = q~ U and (jx, jy) = C u.
__device__ __forceinline__ void feq_C(float C, float qU, float jx, float jy, float* e)
{
    e[0] = C - (2.0f / 3.0f) * qU;
    float b = qU * (1.0f / 6.0f);
    e[1] = b + 0.5f * jx;
    e[3] = b - 0.5f * jx;
    e[2] = b + 0.5f * jy;
    e[4] = b - 0.5f * jy;
}
// Eq. (22) with (jx, jy) = H u.
__device__ __forceinline__ void feq_H(float theta, float hphi, float jx, float jy, float* e)
{
    e[0] = theta * (1.0f / 3.0f) - 0.5f * hphi;
    float b = theta * (1.0f / 6.0f);
    e[1] = b + 0.5f * jx;
    e[3] = b - 0.5f * jx;
    e[2] = b + 0.5f * jy;
    e[4] = b - 0.5f * jy;
}
// Eq. (25): h_i^eq = sigma_i + w_i [3 c.u + 9/2 (c.u)^2 - 3/2 |u|^2].
__device__ __forceinline__ void feq_flow(float p, float ux, float uy, float rho0, float* e)
{
    float uu = 1.5f * (ux * ux + uy * uy);
    e[0] = rho0 - (5.0f / 3.0f) * p + (4.0f / 9.0f) * (-uu);
    const float w1 = 1.0f / 9.0f, w5 = 1.0f / 36.0f;
    float cx[4] = {ux, uy, -ux, -uy};
#pragma unroll
    for (int i = 0; i < 4; ++i) e[1 + i] = w1 * (3.0f * p + 3.0f * cx[i] + 4.5f * cx[i] * cx[i] - uu);
    float d[4] = {ux + uy, -ux + uy, -ux - uy, ux - uy};
#pragma unroll
    for (int i = 0; i < 4; ++i) e[5 + i] = w5 * (3.0f * p + 3.0f * d[i] + 4.5f * d[i] * d[i] - uu);
}

// ------------------------------------------------------------- collisions
// D2Q5 MRT with S = diag(1, s1, s1, 1, 1), equilibrium moments (A, Bx, By,
// Cv/3, Cv/3), auxiliary first moments (Gx, Gy) weighted by (1 - s1/2) and an
// isotropic source S0 added with weights w_i:
//   f*_0 = (A + S0 - 2 (Cv + S0)/3) ... written through the inverse of Eq. (B.1).
__device__ __forceinline__ void collide_d2q5(const float* f, float A, float Bx, float By, float Cv, float s1,
                                             float Gx, float Gy, float S0, float* out)
{
    float m1 = f[1] - f[3], m2 = f[2] - f[4];
    float k1 = 1.0f - 0.5f * s1;
    float r1 = m1 - s1 * (m1 - Bx) + k1 * Gx;
    float r2 = m2 - s1 * (m2 - By) + k1 * Gy;
    float e = (Cv + S0) * (1.0f / 3.0f);   // post-collision second moments (each)
    out[0] = A + S0 - 2.0f * e;
    out[1] = 0.5f * (e + r1);
    out[3] = 0.5f * (e - r1);
    out[2] = 0.5f * (e + r2);
    out[4] = 0.5f * (e - r2);
}

// D2Q9 raw-moment MRT of Eq. (24): m* = m - S (m - m^eq) + (I - S/2) m_F with
// m^eq and m_F of Eq. (B.3) (varphi = 0) and F' = F + [1 - q~] f; returns the
// post-collision populations through the inverse of Eq. (B.2).
__device__ __forceinline__ void collide_flow(const float* h, const Macro& m, float s2, float rho0, float* out)
{
    float qt = 0.5f * (1.0f - m.phi);
    float Fpx = m.Fx + (1.0f - qt) * m.fsx;
    float Fpy = m.Fy + (1.0f - qt) * m.fsy;
    float u = m.ux, v = m.uy, p = m.p;
    // pre-collision second-order moments that relax with s2
    float mxx = h[1] + h[3] + h[5] + h[6] + h[7] + h[8];
    float myy = h[2] + h[4] + h[5] + h[6] + h[7] + h[8];
    float mxy = h[5] - h[6] + h[7] - h[8];
    // post-collision moments
    float r0 = rho0;
    float r1 = u + 0.5f * Fpx;
    float r2 = v + 0.5f * Fpy;
    float r3 = mxx - s2 * (mxx - (p + u * u));
    float r4 = myy - s2 * (myy - (p + v * v));
    float r5 = mxy - s2 * (mxy - u * v);
    float r6 = (v + 0.5f * Fpy) * (1.0f / 3.0f);
    float r7 = (u + 0.5f * Fpx) * (1.0f / 3.0f);
    float r8 = (p + u * u + v * v) * (1.0f / 3.0f);
    // inverse of the tensor-product raw-moment matrix
    out[0] = r0 - r3 - r4 + r8;
    out[1] = 0.5f * (r1 + r3 - r7 - r8);
    out[3] = 0.5f * (-r1 + r3 + r7 - r8);
    out[2] = 0.5f * (r2 + r4 - r6 - r8);
    out[4] = 0.5f * (-r2 + r4 + r6 - r8);
    out[5] = 0.25f * (r5 + r6 + r7 + r8);
    out[6] = 0.25f * (-r5 + r6 - r7 + r8);
    out[7] = 0.25f * (r5 - r6 - r7 + r8);
    out[8] = 0.25f * (-r5 - r6 + r7 + r8);
}

}  // namespace lbm
