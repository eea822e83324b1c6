// Per-node contribution to the metrics reduction, shared by the handle's
// reduction (lbm_aux.cu) and its allocation-free variant (lbm_noalloc.cu) so
// that both give the same numbers.  The node's own arithmetic is FP32 (the
// macros, the sum of its nine flow deviations, |u|); the running sums over
// nodes are FP64, with the constant reference terms (C = 1 + dC, H =
// theta_ref + L + dH with L the latent-heat factor, sum h = rho0 + sum of
// deviations) added per node in FP64 so that long sums keep their digits.  FP64 work per node is a few
// additions: GB300's FP64 rate is a small fraction of its FP32 rate.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

constexpr int kRedValues = 7;  // sum (1+phi)/2, sum C, sum H, sum h, max |u|, non-finite count, sum phi

__device__ __forceinline__ void reduce_accumulate(const StepParams& P, const Macro& m, const float* h, double* acc)
{
    float s9 = 0.0f;
#pragma unroll
    for (int i = 0; i < 9; ++i) s9 += h[i];
    const float u = sqrtf(m.ux * m.ux + m.uy * m.uy);
    acc[0] += 0.5 * (double)m.p1;
    acc[1] += 1.0 + (double)m.dC;
    acc[2] += ((double)P.theta_ref + (double)P.latent) + (double)m.dH;
    acc[3] += (double)P.rho0 + (double)s9;
    acc[4] = fmax(acc[4], (double)u);
    acc[5] += (isfinite(m.p1) && isfinite(m.dC) && isfinite(m.dth) && isfinite(u)) ? 0.0 : 1.0;
    acc[6] += (double)m.p1 - 1.0;
}

}  // namespace lbm
