// Fused coupled step (phase field, solute, heat, flow), wall kernel and flow
// sub-step kernel for sm_103a.
//
// One coupled step n -> n+1 (Sec. 3, time-n macros for every model):
//   1. macros of Eqs. (15), (20), (23), (26) from the node's populations;
//   2. grad(phi) by the isotropic nine-point stencil on phi^n, which each CTA
//      builds in shared memory from the phi populations of its tile and a
//      one-node halo;
//   3. a_s and N of Eqs. (2)-(3) in the grain's crystal frame; Q of Eq. (5);
//      J_at of Eq. (7);
//   4. MRT collisions of the four models in moment space (Appendix B);
//   5. push streaming; phi uses the modified streaming of Eq. (13)/Remark 2,
//      f_i(x+c_i, t+1) = [f*_i(x) - (1 - a_s^2(x)) f_i(x+c_i, t)] / a_s^2(x),
//      whose f_i(x+c_i, t) is read from the same shared tile;
//   6. history (phi, Q, Cu, Hu at time n) is written in place for the
//      backward time differences of the next step.
// Periodic wrap is applied to every streaming destination; on non-periodic
// sides the wrapped values land on wall nodes, which the wall scheme then
// overwrites completely: the wall kernel after the step, or, for the left and
// right walls of steps inside a captured step graph, the next step as it
// loads them (coupled_tile).
#include <cuda_runtime.h>
#include <stddef.h>

#include <type_traits>

#include "lbm_kernels.h"

namespace lbm {

namespace {

constexpr int kLocalGradIters = 2;  // fixed-point passes of the local grad(phi) scheme

__device__ __forceinline__ int mirror_or_wrap_local(int g, int n, int periodic, int local, int d)
{
    // Neighbour g = node + d seen from local index `local` of the node: a
    // periodic neighbour (or one inside the domain) is in the halo at
    // local + d; a non-periodic ghost is the mirror image at local - d.
    if (!periodic && (g < 0 || g >= n)) return local - d;
    return local + d;
}

#ifndef LBM_BATCH_WARPS
#define LBM_BATCH_WARPS 32  // resident warps per SM the batched kernel's register budget is sized for
#endif

#ifndef LBM_STEP_MIN_BLOCKS
#define LBM_STEP_MIN_BLOCKS 9  // resident CTAs of 128 threads per SM the register budget is sized for
                               // (56 registers; 36 warps hide more of the memory latency than 32)
#endif

// Non-equilibrium extrapolation (Guo et al.) on one side pair, applied to the
// freshly streamed buffer: pop(b) = pop^eq(boundary macros) + pop(f) -
// pop^eq(macros of f), f the first interior node.  `axis` 1: bottom/top rows
// over x in [xlo, xhi]; `axis` 0: left/right columns over every y.  The
// result depends on the interior node alone, so applying it twice changes
// nothing.
//
// Phase-field part: boundary populations fb from the interior populations ff,
// whose sum (node_macros' order) is p1f = phi_f + 1.
__device__ __forceinline__ void wall_phi(const StepParams& P, int type, const float (&ff)[5], float p1f,
                                         float (&fb)[5])
{
    const float p1b = type == 5 ? P.dir_phi + 1.0f : p1f;  // Dirichlet far field, else zero gradient
    float eb[5], ef[5];
    deq_phi(p1b, eb);
    deq_phi(p1f, ef);
#pragma unroll
    for (int i = 0; i < 5; ++i) fb[i] = eb[i] + ff[i] - ef[i];
}

// Flow, solute and heat parts from the interior node's macros m and
// populations n, g, h; the scalar parts only when !flow_only.
__device__ __forceinline__ void wall_rest(const StepParams& P, int axis, int type, const Macro& m,
                                          const float (&n)[5], const float (&g)[5], const float (&h)[9],
                                          float (&nb)[5], float (&gb)[5], float (&hb)[9], int flow_only)
{
    float ubx = 0.0f, uby = 0.0f, pb = m.p;
    if (type == 1) {  // inflow
        ubx = P.uin_x;
        uby = P.uin_y;
    } else if (type == 2) {  // outflow
        ubx = m.ux;
        uby = m.uy;
        pb = 0.0f;
    } else if (type == 3) {  // symmetry
        ubx = axis == 0 ? 0.0f : m.ux;
        uby = axis == 0 ? m.uy : 0.0f;
    }
    float eb[9], ef[9];
    deq_flow(pb, ubx, uby, eb);
    deq_flow(m.p, m.ux, m.uy, ef);
#pragma unroll
    for (int i = 0; i < 9; ++i) hb[i] = eb[i] + h[i] - ef[i];
    if (flow_only) return;

    float p1b = m.p1, dCb = m.dC, Ub = m.U, dthb = m.dth;
    if (type == 5) {  // Dirichlet far field
        p1b = P.dir_phi + 1.0f;
        Ub = P.dir_U;
        dCb = dC_of(Ub, p1b, P.k);
        dthb = P.dir_theta - P.theta_ref;
    }
    const float hp1b = h_plus_1(P.h_kind, p1b);
    const float Hb = (P.theta_ref + P.latent) + dthb - P.latent * hp1b;
    const float Cb = 1.0f + dCb, Cf = 1.0f + m.dC;
    const float sc = P.nsub;
    deq_C(dCb, (1.0f - 0.5f * p1b) * Ub, Cb * ubx * sc, Cb * uby * sc, eb);
    deq_C(m.dC, (1.0f - 0.5f * m.p1) * m.U, Cf * m.ux * sc, Cf * m.uy * sc, ef);
#pragma unroll
    for (int i = 0; i < 5; ++i) nb[i] = eb[i] + n[i] - ef[i];
    deq_H(dthb, P.latent * hp1b, Hb * ubx * sc, Hb * uby * sc, eb);
    deq_H(m.dth, P.latent * m.hp1, m.H * m.ux * sc, m.H * m.uy * sc, ef);
#pragma unroll
    for (int i = 0; i < 5; ++i) gb[i] = eb[i] + g[i] - ef[i];
}

// Per-node part of the coupled step for node (x, y) = tile-local (lx - 1, ly - 1):
// f, n, g, h are its populations at time n (n_1..n_4 and g_1..g_4 in units
// of 1/Store::kSS, h in units of 1/Store::kSF: the codec's push scales), the
// *_prev values its history;
// fs holds the tile's phi populations with a one-node halo, node (x, y) at
// column fx = lx - 1 + XO of rows of FW floats; ps holds phi on the tile and
// halo with node (x, y) at [ly][lx].  Collides, push-streams (the phase field
// by the modified streaming of Eq. 13) and writes the history.
template <class Store, bool GRAIN, bool WRITE_FB, int TYV, int FW, int XO>
__device__ __forceinline__ void coupled_node(const StepParams& P, void* __restrict__ dst, void* __restrict__ dstf,
                                             float* __restrict__ hist, float* __restrict__ fb, int x, int y,
                                             int lx, int ly, const float (&f)[5], const float (&n)[5],
                                             const float (&g)[5], const float (&h)[9], float phi_prev,
                                             float Q_prev, float Cux_prev, float Cuy_prev, float Hux_prev,
                                             float Huy_prev, bool grain_on, uint8_t gid,
                                             const float (&fs)[5][TYV + 2][FW],
                                             const float (&ps)[TYV + 2][TX + 2])
{
    const long long o = (long long)y * P.pitch + x;
    const int fx = lx - 1 + XO;

    constexpr int SS = Store::kSS, SF = Store::kSF;
    const Macro m = node_macros<SS, SF>(f, n, g, h, P);
    const float usx = m.ux * P.nsub, usy = m.uy * P.nsub;  // velocity of the scalar lattice

    float co = P.cos_o, so = P.sin_o;
    if (GRAIN && grain_on) {
        const float2 cs = P.grain_cs[gid];
        co = cs.x;
        so = cs.y;
    }
    float gx, gy;
    if (!P.grad_local) {
        // grad(phi): (1/cs^2) sum_i w_i c_i phi(x + c_i) over the D2Q9 neighbours
        const int xl = mirror_or_wrap_local(x - 1, P.nx, P.periodic_x, lx, -1);
        const int xr = mirror_or_wrap_local(x + 1, P.nx, P.periodic_x, lx, +1);
        const int yd = mirror_or_wrap_local(y - 1, P.ny, P.periodic_y, ly, -1);
        const int yu = mirror_or_wrap_local(y + 1, P.ny, P.periodic_y, ly, +1);
        const float pE = ps[ly][xr], pW = ps[ly][xl], pN = ps[yu][lx], pS = ps[yd][lx];
        const float pNE = ps[yu][xr], pNW = ps[yu][xl], pSE = ps[yd][xr], pSW = ps[yd][xl];
        // paired differences, so that mirror-symmetric neighbourhoods (a wall
        // ghost, a symmetric seed) give an exactly zero component
        gx = (pE - pW) * (1.0f / 3.0f) + ((pNE - pNW) + (pSE - pSW)) * (1.0f / 12.0f);
        gy = (pN - pS) * (1.0f / 3.0f) + ((pNE - pSE) + (pNW - pSW)) * (1.0f / 12.0f);
    } else {
        // local scheme of Sec. 3.1: grad(phi) = -(s1/cs^2)(sum_i c_i f_i + W0^2 N/tau0)
        // with s1 and N taken at grad(phi): two fixed-point passes from a_s = 1, N = 0
        const float jx = f[1] - f[3], jy = f[2] - f[4];
        const float k0 = P.kappa3 * (1.0f / 3.0f);
        float s1 = __fdividef(1.0f, P.kappa3 + 0.5f);
        gx = -3.0f * s1 * jx;
        gy = -3.0f * s1 * jy;
#pragma unroll
        for (int it = 0; it < kLocalGradIters; ++it) {
            float a1, nx_, ny_;
            anisotropy(gx, gy, P.eps, co, so, a1, nx_, ny_);
            s1 = __fdividef(1.0f, P.kappa3 * a1 * a1 + 0.5f);
            gx = -3.0f * s1 * (jx + k0 * nx_);
            gy = -3.0f * s1 * (jy + k0 * ny_);
        }
    }
    float as, Nx, Ny;
    anisotropy(gx, gy, P.eps, co, so, as, Nx, Ny);
    const float as2 = as * as;
    // 1/a_s^2 (a_s^2 within (1 - 3 eps)^2 .. (1 + eps)^2) and the phase-field
    // rate, by fast division (within 2 ulp; both denominators are O(1))
    const float ia = __fdividef(1.0f, as2);
    const float g2 = gx * gx + gy * gy;
    const float Q = coupling_Q(m.phi, P.theta_ref + m.dth, m.U, P);

    // ---- phase field: Eqs. (13)-(14), relaxation rate of Sec. 3.1
    float fo[5];
    {
        const float s1 = __fdividef(1.0f, P.kappa3 * as2 + 0.5f);
        const float S0 = (Q + 0.5f * as2 * (Q - Q_prev)) * P.inv_tau;
        const float ga = -(1.0f / 3.0f) * ia;
        collide_d2q5<1, SS>(f, m.p1, 0.0f, 0.0f, m.p1, s1, ga * Nx, ga * Ny, S0, fo);
    }
    // ---- solute: Eqs. (17)-(19) with J_at of Eq. (7)
    float no[5];
    {
        float Jx = 0.0f, Jy = 0.0f;
        if (!(g2 < kGradEps2)) {
            const float a = -0.35355339059327373f * P.W * (1.0f + (1.0f - P.k) * m.U) * (m.phi - phi_prev) *
                            rsqrtf(g2);
            Jx = a * gx;
            Jy = a * gy;
        }
        const float qt = 1.0f - 0.5f * m.p1;
        const float C = 1.0f + m.dC;
        const float Cux = C * usx, Cuy = C * usy;
        // sum_i c_i G_i = d_t(Cu) + cs^2 (U grad q~ + J_at/D), grad q~ = -grad(phi)/2
        const float Gx = (Cux - Cux_prev) + (1.0f / 3.0f) * (-0.5f * m.U * gx + Jx * P.inv_D);
        const float Gy = (Cuy - Cuy_prev) + (1.0f / 3.0f) * (-0.5f * m.U * gy + Jy * P.inv_D);
        collide_d2q5<SS, SS>(n, m.dC, Cux, Cuy, qt * m.U, P.s1C, Gx, Gy, 0.0f, no);
    }
    // ---- heat: Eqs. (21)-(23)
    float go[5];
    {
        const float Hux = m.H * usx, Huy = m.H * usy;
        collide_d2q5<SS, SS>(g, m.dH, Hux, Huy, m.dth, P.s1T, Hux - Hux_prev, Huy - Huy_prev, 0.0f, go);
    }
    // ---- flow: Eqs. (24)-(26)
    float ho[9];
    collide_flow<SF, SF>(h, m, P.s2u, ho);

    // ---- push streaming: the rest populations stay at o; every moving one
    // goes to the neighbour node (x + c_x, y + c_y), whose element index is a
    // row term plus a column term (three of each)
    const int xp = (x + 1 == P.nx) ? 0 : x + 1, xm = (x == 0) ? P.nx - 1 : x - 1;
    const int yp = (y + 1 == P.ny) ? 0 : y + 1, ym = (y == 0) ? P.ny - 1 : y - 1;
    {
        const long long rY = Store::mov_row(y, P), rP = Store::mov_row(yp, P), rM = Store::mov_row(ym, P);
        const int c0 = Store::mov_col(x), cP = Store::mov_col(xp), cM = Store::mov_col(xm);
        const long long d5[5] = {0, rY + cP, rP + c0, rY + cM, rM + c0};
        // modified streaming of the phase field: the destination's time-n
        // population sits in the shared tile (its halo is periodic-wrapped)
        const float ib = ia - 1.0f, ibs = ib * (float)SS;
        const float fd[5] = {fs[0][ly][fx], fs[1][ly][fx + 1], fs[2][ly + 1][fx], fs[3][ly][fx - 1],
                             fs[4][ly - 1][fx]};
        Store::store(dst, dstf, kF, o, fo[0] * ia - ib * fd[0], P);
        Store::store(dst, dstf, kN, o, no[0], P);
        Store::store(dst, dstf, kG, o, go[0], P);
#pragma unroll
        for (int i = 1; i < 5; ++i) Store::store_mov(dst, kF + i, d5[i], fo[i] * ia - ibs * fd[i]);
        // n_i and g_i go to the same neighbour (one word in 16-bit storage)
        const long long qY = Store::pair_row(y, P), qP = Store::pair_row(yp, P), qM = Store::pair_row(ym, P);
        const int p0 = Store::pair_col(x), pP = Store::pair_col(xp), pM = Store::pair_col(xm);
        const long long e5[5] = {0, qY + pP, qP + p0, qY + pM, qM + p0};
#pragma unroll
        for (int i = 1; i < 5; ++i) Store::store_pair(dst, i, e5[i], no[i], go[i]);
    }
    {
        const long long rY = Store::flow_row(y, P), rP = Store::flow_row(yp, P), rM = Store::flow_row(ym, P);
        const int c0 = Store::flow_col(x), cP = Store::flow_col(xp), cM = Store::flow_col(xm);
        const long long d9[9] = {rY + c0, rY + cP, rP + c0, rY + cM, rM + c0, rP + cP, rP + cM, rM + cM, rM + cP};
#pragma unroll
        for (int i = 0; i < 9; ++i) Store::store_flow(dstf, i, d9[i], ho[i]);
    }

    // ---- history of the backward differences
    hist_at(hist, 0, o) = m.phi;
    hist_at(hist, 1, o) = Q;
    hist_at(hist, 2, o) = (1.0f + m.dC) * usx;
    hist_at(hist, 3, o) = (1.0f + m.dC) * usy;
    hist_at(hist, 4, o) = m.H * usx;
    hist_at(hist, 5, o) = m.H * usy;
    if (WRITE_FB) fb[o] = m.Fy;
}


// One tile of the coupled step: the CTA (TX x TYV threads) updates the nodes
// [x0, x0 + TX) x [y0, y0 + TYV) of one domain.  GRAIN: the domain may carry a
// grain map (read when `grain` is not null).  All threads reach the barriers,
// so callers may loop over tiles.
//
// XWALL with xfix set: the left and right walls of a domain that is not
// periodic in x were not updated after the previous step (the wall scheme's
// column pass was skipped); the tile applies that update to the wall cells it
// loads instead.  Extrapolation depends on the first interior node alone, and
// the tile holding a wall column also holds that node (x = 1 or nx - 2), so
// the result is the column pass's, without its strided sweep over 24 planes.
// Rows (bottom/top walls) are still updated by their own pass after each step,
// before the columns, as the corners belong to the columns.
template <class Store, bool GRAIN, bool WRITE_FB, int TYV, bool XWALL = false>
__device__ __forceinline__ void coupled_tile(const StepParams& P, const void* __restrict__ src,
                                             const void* __restrict__ srcf, void* __restrict__ dst,
                                             void* __restrict__ dstf, float* __restrict__ hist,
                                             const uint8_t* __restrict__ grain, float* __restrict__ fb, int x0,
                                             int y0, float (&fs)[5][TYV + 2][TX + 2], float (&ps)[TYV + 2][TX + 2],
                                             int xfix = 0)
{
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int x = x0 + tx, y = y0 + ty;
    const bool active = x < P.nx && y < P.ny;
    // XWALL: C, H and flow populations of the tile's own wall nodes, computed
    // first, while no other values are held in registers
    const bool xwall_tile = XWALL && xfix && !P.periodic_x && (x0 == 0 || x0 + TX + 1 >= P.nx);
    __shared__ float wnb[XWALL ? 2 : 1][XWALL ? TYV : 1][19];
    if constexpr (XWALL) {
        static_assert(2 * (TYV + 2) <= TX * TYV && 2 * TYV <= TX * TYV, "wall-repair thread ranges");
        const int tid = ty * TX + tx;
        if (xwall_tile && tid < 2 * TYV) {
            const int side = tid / TYV, r = tid % TYV;
            const int xw = side == 0 ? 0 : P.nx - 1, xi = side == 0 ? 1 : P.nx - 2;
            const int yw = y0 + r;
            if (xw >= x0 && xw < x0 + TX && yw < P.ny) {
                const long long oi = (long long)yw * P.pitch + xi;
                float fi[5], ni[5], gi[5], hi[9], nbw[5], gbw[5], hbw[9];
#pragma unroll
                for (int i = 0; i < 5; ++i) fi[i] = Store::load(src, srcf, kF + i, oi, P);
#pragma unroll
                for (int i = 0; i < 5; ++i) ni[i] = Store::load(src, srcf, kN + i, oi, P);
#pragma unroll
                for (int i = 0; i < 5; ++i) gi[i] = Store::load(src, srcf, kG + i, oi, P);
#pragma unroll
                for (int i = 0; i < 9; ++i) hi[i] = Store::load(src, srcf, kH + i, oi, P);
                const Macro mi = node_macros(fi, ni, gi, hi, P);
                wall_rest(P, 0, P.bc[side], mi, ni, gi, hi, nbw, gbw, hbw, 0);
                // in the units the node update takes (rest populations unscaled)
                wnb[side][r][0] = nbw[0];
                wnb[side][r][5] = gbw[0];
#pragma unroll
                for (int i = 1; i < 5; ++i) wnb[side][r][i] = nbw[i] * (float)Store::kSS;
#pragma unroll
                for (int i = 1; i < 5; ++i) wnb[side][r][5 + i] = gbw[i] * (float)Store::kSS;
#pragma unroll
                for (int i = 0; i < 9; ++i) wnb[side][r][10 + i] = hbw[i] * (float)Store::kSF;
            }
        }
        if (xwall_tile) __syncthreads();  // keeps the loads below after the repair
    }
    // own-node loads first, so that they are in flight while the halo loads.
    // Every thread loads its own tile cell (x, y), wrapped into the grid when
    // the tile reaches past it (such cells serve as periodic neighbours of
    // the edge nodes); the first 2 (TX + 2) + 2 TYV threads load the halo ring.
    const long long o = active ? (long long)y * P.pitch + x : 0;
    int cx = x, cy = y;
    if (!active) {
        cx = cx >= P.nx ? wrap(cx, P.nx) : cx;
        cy = cy >= P.ny ? wrap(cy, P.ny) : cy;
    }
    const long long oc = active ? o : (long long)cy * P.pitch + cx;
    float f[5], n[5], g[5], h[9];
#pragma unroll
    for (int i = 0; i < 5; ++i) f[i] = Store::load(src, srcf, kF + i, oc, P);
    n[0] = Store::load(src, srcf, kN, o, P);
    g[0] = Store::load(src, srcf, kG, o, P);
#pragma unroll
    for (int i = 1; i < 5; ++i) Store::load_pair(src, i, o, n[i], g[i]);
#pragma unroll
    for (int i = 0; i < 9; ++i) h[i] = Store::load_flow(srcf, i, o);
    const float* hn = hist;
    const float phi_prev = hist_at(hn, 0, o);
    const float Q_prev = hist_at(hn, 1, o);
    const float Cux_prev = hist_at(hn, 2, o), Cuy_prev = hist_at(hn, 3, o);
    const float Hux_prev = hist_at(hn, 4, o), Huy_prev = hist_at(hn, 5, o);
    uint8_t gid = 0;
    if (GRAIN && grain) gid = grain[o];

    static_assert(2 * (TX + 2) + 2 * TYV <= TX * TYV, "halo ring thread range");
    const int tid = ty * TX + tx;
    if (tid < 2 * (TX + 2) + 2 * TYV) {
        int hx, hy;
        if (tid < 2 * (TX + 2)) {  // the rows below and above the tile, corners included
            hy = tid < TX + 2 ? 0 : TYV + 1;
            hx = tid < TX + 2 ? tid : tid - (TX + 2);
        } else {  // the columns left and right of it
            const int r = tid - 2 * (TX + 2);
            hx = r < TYV ? 0 : TX + 1;
            hy = 1 + (r < TYV ? r : r - TYV);
        }
        int gx = x0 - 1 + hx, gy = y0 - 1 + hy;
        gx = (gx < 0) ? gx + P.nx : (gx >= P.nx ? gx - P.nx : gx);
        gy = (gy < 0) ? gy + P.ny : (gy >= P.ny ? gy - P.ny : gy);
        if (gx >= P.nx) gx = wrap(gx, P.nx);  // domains narrower than a tile
        if (gy >= P.ny) gy = wrap(gy, P.ny);
        const long long oh = (long long)gy * P.pitch + gx;
        float sum = 0.0f;
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            const float v = Store::load(src, srcf, kF + i, oh, P);
            fs[i][hy][hx] = v;
            sum += v;
        }
        ps[hy][hx] = sum;
    }
    {
        float sum = 0.0f;
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            fs[i][ty + 1][tx + 1] = f[i];
            sum += f[i];
        }
        ps[ty + 1][tx + 1] = sum;
    }
    __syncthreads();

    if constexpr (XWALL) {
        if (xwall_tile) {
            // (side, row) of each wall column the tile holds: x = 0 (side 0)
            // at tile column 1 - x0, x = nx - 1 (side 1) at nx - x0
            const int tid = ty * TX + tx;
            if (tid < 2 * (TYV + 2)) {
                // phase-field populations and phi of a wall cell of the tile or its halo rows
                const int side = tid / (TYV + 2), hy = tid % (TYV + 2);
                const int hx = side == 0 ? 1 - x0 : P.nx - x0;
                if (hx >= 0 && hx <= TX + 1) {
                    const int hf = side == 0 ? hx + 1 : hx - 1;  // the interior node, never a wall (nx >= 4)
                    float ff[5], fbw[5];
#pragma unroll
                    for (int i = 0; i < 5; ++i) ff[i] = fs[i][hy][hf];
                    wall_phi(P, P.bc[side], ff, ff[0] + ff[1] + ff[2] + ff[3] + ff[4], fbw);
                    float sum = 0.0f;
#pragma unroll
                    for (int i = 0; i < 5; ++i) {
                        fs[i][hy][hx] = fbw[i];
                        sum += fbw[i];
                    }
                    ps[hy][hx] = sum;
                }
            }
            __syncthreads();
            if (active && (x == 0 || x == P.nx - 1)) {
                const int side = x == 0 ? 0 : 1;
#pragma unroll
                for (int i = 0; i < 5; ++i) f[i] = fs[i][ty + 1][tx + 1];  // as the repair left the tile
#pragma unroll
                for (int i = 0; i < 5; ++i) n[i] = wnb[side][ty][i];
#pragma unroll
                for (int i = 0; i < 5; ++i) g[i] = wnb[side][ty][5 + i];
#pragma unroll
                for (int i = 0; i < 9; ++i) h[i] = wnb[side][ty][10 + i];
            }
        }
    }

    if (!active) return;
    coupled_node<Store, GRAIN, WRITE_FB, TYV, TX + 2, 1>(P, dst, dstf, hist, fb, x, y, tx + 1, ty + 1, f, n, g, h,
                                                          phi_prev, Q_prev, Cux_prev, Cuy_prev, Hux_prev, Huy_prev,
                                                          grain != nullptr, gid, fs, ps);
}

template <class Store, bool GRAIN, bool WRITE_FB, bool XWALL = false>
__global__ void __launch_bounds__(TX* TY, LBM_STEP_MIN_BLOCKS)
    k_coupled_step(const StepParams P, const void* __restrict__ src, const void* __restrict__ srcf,
                   void* __restrict__ dst, void* __restrict__ dstf, float* __restrict__ hist,
                   const uint8_t* __restrict__ grain, float* __restrict__ fb, int xfix = 0)
{
    __shared__ float fs[5][TY + 2][TX + 2];
    __shared__ float ps[TY + 2][TX + 2];
    coupled_tile<Store, GRAIN, WRITE_FB, TY, XWALL>(P, src, srcf, dst, dstf, hist, grain, fb, blockIdx.x * TX,
                                                    blockIdx.y * TY, fs, ps, xfix);
}

// Descriptors of the batch being stepped, in constant memory: the domain
// index is uniform across a CTA, so parameter reads are broadcast from the
// constant cache as in the single-domain kernel.  launch_batch_step copies the
// batch's table in before each step.
__constant__ DomainDesc c_batch_desc[kMaxBatchDomains];

// Batched coupled step: one persistent grid sweeps the tile table of every
// domain; each CTA takes a contiguous run of tiles, so consecutive tiles share
// the domain and their halos stay in L2.  A kernel boundary separates steps.
template <class Store, int TYV>
__global__ void __launch_bounds__(TX* TYV, (LBM_BATCH_WARPS / TYV > 0 ? LBM_BATCH_WARPS / TYV : 1))
    k_batch_step(const int4* __restrict__ tiles, int ntiles, int chunk, int parity, int xfix)
{
    __shared__ float fs[5][TYV + 2][TX + 2];
    __shared__ float ps[TYV + 2][TX + 2];
    const int t_end = min(ntiles, (blockIdx.x + 1) * chunk);
    for (int t = blockIdx.x * chunk; t < t_end; ++t) {
        const int4 tl = tiles[t];
        const DomainDesc& d = c_batch_desc[tl.x];
        coupled_tile<Store, true, false, TYV, true>(d.P, d.sc[parity], d.fl[parity], d.sc[1 - parity],
                                                    d.fl[1 - parity], d.hist, d.grain, nullptr, tl.y, tl.z, fs, ps,
                                                    xfix);
        __syncthreads();  // the tile arrays are reused by the next tile
    }
}

// v as a store to flow plane q and a load would return it (16-bit storage
// rounds; FP32 keeps v).
template <class Store>
__device__ __forceinline__ float stored_flow(int q, float v)
{
    if constexpr (std::is_same<Store, StoreF32>::value) {
        return v;
    } else {
        return Conv<typename Store::T>::to(Conv<typename Store::T>::from(v * Store::scale(q))) * Store::inv_scale(q);
    }
}

// Flow populations the flow-only wall pass gives a wall node of `side` (axis
// 0: left/right columns, 1: bottom/top rows) from its interior node at offset
// oi, whose flow populations are hi: extrapolation with that node's macros,
// its scalar populations read from sc.
template <class Store>
__device__ __forceinline__ void flow_wall_from(const StepParams& P, const void* __restrict__ sc, int axis, int side,
                                               long long oi, const float (&hi)[9], float (&hb)[9])
{
    float fi[5], ni[5], gi[5], nb[5], gb[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) fi[i] = Store::load(sc, nullptr, kF + i, oi, P);
#pragma unroll
    for (int i = 0; i < 5; ++i) ni[i] = Store::load(sc, nullptr, kN + i, oi, P);
#pragma unroll
    for (int i = 0; i < 5; ++i) gi[i] = Store::load(sc, nullptr, kG + i, oi, P);
    const Macro m = node_macros(fi, ni, gi, hi, P);
    wall_rest(P, axis, P.bc[side], m, ni, gi, hi, nb, gb, hb, 1);
}

// The flow populations the flow-only wall pass (rows, then columns) would
// have left at wall node (x, y) after the previous flow step, which skipped
// it: a row node from its interior node; a column node from its interior
// node; a corner from the row node beside it as the row pass leaves it.
template <class Store>
__device__ __forceinline__ void flow_wall_repair(const StepParams& P, const void* __restrict__ sc,
                                              const void* __restrict__ src, int x, int y, bool wx, bool wy,
                                              float (&h)[9])
{
    const int xi = x == 0 ? 1 : P.nx - 2, yi = y == 0 ? 1 : P.ny - 2;
    const int row_side = y == 0 ? 2 : 3, col_side = x == 0 ? 0 : 1;
    float hi[9];
    if (!wx) {
        const long long oi = (long long)yi * P.pitch + x;
#pragma unroll
        for (int i = 0; i < 9; ++i) hi[i] = Store::load(nullptr, src, kH + i, oi, P);
        flow_wall_from<Store>(P, sc, 1, row_side, oi, hi, h);
    } else {
        const long long oc = (long long)y * P.pitch + xi;
        if (wy) {
            const long long oi = (long long)yi * P.pitch + xi;
            float hr[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) hr[i] = Store::load(nullptr, src, kH + i, oi, P);
            flow_wall_from<Store>(P, sc, 1, row_side, oi, hr, hi);
#pragma unroll
            for (int i = 0; i < 9; ++i) hi[i] = stored_flow<Store>(kH + i, hi[i]);  // as the row pass stores it
        } else {
#pragma unroll
            for (int i = 0; i < 9; ++i) hi[i] = Store::load(nullptr, src, kH + i, oc, P);
        }
        flow_wall_from<Store>(P, sc, 0, col_side, oc, hi, h);
    }
    // as the wall pass would store them and this step's load return them
#pragma unroll
    for (int i = 0; i < 9; ++i) h[i] = stored_flow<Store>(kH + i, h[i]);
}

// Flow sub-step (two-time-scaling of Sec. 4): collide and stream h with phi
// and the force frozen at time n.  repair: the previous flow step skipped the
// flow-only wall pass, so wall nodes first take the populations it would have
// given them (flow_wall_repair; sc holds the newest scalar populations, whose
// macros the wall scheme uses).
// phi: plane 0 of a node-block array of phi_np planes (the history, or the
// frozen phi of flow-only steps, phi_np = 1: a plain plane).
template <class Store>
__global__ void __launch_bounds__(256, 8) k_flow_substep(const StepParams P, const void* __restrict__ src,
                                                      void* __restrict__ dst, const float* __restrict__ phi,
                                                      int phi_np, const float* __restrict__ fb,
                                                      const void* __restrict__ sc, int repair)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= P.nx || y >= P.ny) return;
    const long long o = (long long)y * P.pitch + x;
    float h[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) h[i] = Store::load(nullptr, src, kH + i, o, P);
    if (repair) {
        const bool wx = !P.periodic_x && (x == 0 || x == P.nx - 1);
        const bool wy = !P.periodic_y && (y == 0 || y == P.ny - 1);
        if (wx || wy) flow_wall_repair<Store>(P, sc, src, x, y, wx, wy, h);
    }
    Macro m;
    m.phi = phi[block_index(o, phi_np)];
    m.p1 = m.phi + 1.0f;
    m.Fx = P.Fx;
    m.Fy = fb[o];
    float jx = h[1] - h[3] + h[5] - h[6] - h[7] + h[8];
    float jy = h[2] - h[4] + h[5] + h[6] - h[7] - h[8];
    float rest = h[1] + h[2] + h[3] + h[4] + h[5] + h[6] + h[7] + h[8];
    float usx = jx + 0.5f * m.Fx, usy = jy + 0.5f * m.Fy;
    float qt = 1.0f - 0.5f * m.p1;
    m.fsx = -usx;
    m.fsy = -usy;
    m.ux = usx + 0.5f * (1.0f - qt) * m.fsx;
    m.uy = usy + 0.5f * (1.0f - qt) * m.fsy;
    m.p = 0.6f * (rest - (2.0f / 3.0f) * (m.ux * m.ux + m.uy * m.uy));
    float ho[9];
    collide_flow<1, Store::kSF>(h, m, P.s2u, ho);
    const int xp = (x + 1 == P.nx) ? 0 : x + 1, xm = (x == 0) ? P.nx - 1 : x - 1;
    const int yp = (y + 1 == P.ny) ? 0 : y + 1, ym = (y == 0) ? P.ny - 1 : y - 1;
    const long long rY = Store::flow_row(y, P), rP = Store::flow_row(yp, P), rM = Store::flow_row(ym, P);
    const int c0 = Store::flow_col(x), cP = Store::flow_col(xp), cM = Store::flow_col(xm);
    const long long d9[9] = {rY + c0, rY + cP, rP + c0, rY + cM, rM + c0, rP + cP, rP + cM, rM + cM, rM + cP};
#pragma unroll
    for (int i = 0; i < 9; ++i) Store::store_flow(dst, i, d9[i], ho[i]);
}

template <class Store>
__device__ __forceinline__ void wall_node(const StepParams& P, void* __restrict__ pop, void* __restrict__ popf,
                                          int axis, int which, int j, int flow_only)
{
    const int side = axis == 0 ? which : 2 + which;
    if (P.bc[side] == 0) return;
    int xb, yb, xf, yf;
    if (axis == 0) {
        yb = yf = j;
        xb = which ? P.nx - 1 : 0;
        xf = which ? P.nx - 2 : 1;
    } else {
        xb = xf = j;
        yb = which ? P.ny - 1 : 0;
        yf = which ? P.ny - 2 : 1;
    }
    const long long ob = (long long)yb * P.pitch + xb, of = (long long)yf * P.pitch + xf;
    float f[5], n[5], g[5], h[9];
#pragma unroll
    for (int i = 0; i < 5; ++i) f[i] = Store::load(pop, popf, kF + i, of, P);
#pragma unroll
    for (int i = 0; i < 5; ++i) n[i] = Store::load(pop, popf, kN + i, of, P);
#pragma unroll
    for (int i = 0; i < 5; ++i) g[i] = Store::load(pop, popf, kG + i, of, P);
#pragma unroll
    for (int i = 0; i < 9; ++i) h[i] = Store::load(pop, popf, kH + i, of, P);
    const Macro m = node_macros(f, n, g, h, P);
    const int type = P.bc[side];
    float fb[5], nb[5], gb[5], hb[9];
    wall_rest(P, axis, type, m, n, g, h, nb, gb, hb, flow_only);
#pragma unroll
    for (int i = 0; i < 9; ++i) Store::store(pop, popf, kH + i, ob, hb[i], P);
    if (flow_only) return;
    wall_phi(P, type, f, m.p1, fb);
#pragma unroll
    for (int i = 0; i < 5; ++i) Store::store(pop, popf, kF + i, ob, fb[i], P);
#pragma unroll
    for (int i = 0; i < 5; ++i) Store::store(pop, popf, kN + i, ob, nb[i], P);
#pragma unroll
    for (int i = 0; i < 5; ++i) Store::store(pop, popf, kG + i, ob, gb[i], P);
}

template <class Store>
__global__ void k_walls(const StepParams P, void* __restrict__ pop, void* __restrict__ popf, int axis, int lo,
                        int count, int flow_only)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * count) return;
    const int which = t / count;           // 0: low side, 1: high side
    wall_node<Store>(P, pop, popf, axis, which, lo + (t - which * count), flow_only);
}

// Batched walls: one thread per entry {domain, axis, side, index} of a list
// holding one axis of every domain.
template <class Store>
__global__ void k_batch_walls(const DomainDesc* __restrict__ descs, const int4* __restrict__ nodes, int count,
                              int parity)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    const int4 e = nodes[t];
    const DomainDesc& d = descs[e.x];
    wall_node<Store>(d.P, d.sc[parity], d.fl[parity], e.y, e.z, e.w, 0);
}

// Rows (bottom/top walls, x in [1, nx - 2] when x is not periodic), then,
// with `columns`, the left/right columns over every y (corners included).
template <class Store>
cudaError_t walls(const StepParams& P, void* sc, void* fl, int flow_only, cudaStream_t s, bool columns = true)
{
    if (!P.periodic_y) {
        const int lo = P.periodic_x ? 0 : 1, hi = P.periodic_x ? P.nx - 1 : P.nx - 2;
        const int count = hi - lo + 1;
        k_walls<Store><<<(2 * count + 127) / 128, 128, 0, s>>>(P, sc, fl, 1, lo, count, flow_only);
    }
    if (!P.periodic_x && columns) {
        k_walls<Store><<<(2 * P.ny + 127) / 128, 128, 0, s>>>(P, sc, fl, 0, 0, P.ny, flow_only);
    }
    return cudaGetLastError();
}

template <class Store>
cudaError_t flow_steps_t(const StepParams& P, int n, void* sc, void* const fl[2], int* cf, const float* phi,
                         const float* fy, cudaStream_t s)
{
    const dim3 fblock(64, 4), fgrid((P.nx + 63) / 64, (P.ny + 3) / 4);
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < n; ++k) {
        // wall pass after the last step only; each later step repairs the wall
        // nodes it loads instead
        k_flow_substep<Store><<<fgrid, fblock, 0, s>>>(P, fl[*cf], fl[1 - *cf], phi, 1, fy, sc, k > 0);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (k + 1 == n && (e = walls<Store>(P, sc, fl[1 - *cf], 1, s)) != cudaSuccess) return e;
        *cf = 1 - *cf;
    }
    return e;
}

template <class Store>
cudaError_t coupled_step(const StepParams& P, int n_sub, StepBuffers& B, cudaStream_t s, int repair, int skip_columns)
{
    const dim3 block(TX, TY), grid((P.nx + TX - 1) / TX, (P.ny + TY - 1) / TY);
    const void* src = B.sc[B.cs];
    const void* srcf = B.fl[B.cf];
    void* dst = B.sc[1 - B.cs];
    void* dstf = B.fl[1 - B.cf];
    const bool grain = B.grain != nullptr, wfb = n_sub > 1;
    if (B.ev_begin && !B.ev_substeps) cudaEventRecord(B.ev_begin, s);
    // left/right walls: with skip_columns their column pass is left out and
    // the next step, launched with `repair`, updates them at its load
    // (coupled_tile); only steps with one flow step per coupled step do
    // that, with flow sub-steps the column pass stays
    const bool xwall = !wfb && !P.periodic_x;
    const int xfix = xwall ? repair : 0;
    if (xwall && grain)
        k_coupled_step<Store, true, false, true>
            <<<grid, block, 0, s>>>(P, src, srcf, dst, dstf, B.hist, B.grain, B.fb, xfix);
    else if (xwall)
        k_coupled_step<Store, false, false, true>
            <<<grid, block, 0, s>>>(P, src, srcf, dst, dstf, B.hist, B.grain, B.fb, xfix);
    else if (grain && wfb)
        k_coupled_step<Store, true, true><<<grid, block, 0, s>>>(P, src, srcf, dst, dstf, B.hist, B.grain, B.fb);
    else if (grain)
        k_coupled_step<Store, true, false><<<grid, block, 0, s>>>(P, src, srcf, dst, dstf, B.hist, B.grain, B.fb);
    else if (wfb)
        k_coupled_step<Store, false, true><<<grid, block, 0, s>>>(P, src, srcf, dst, dstf, B.hist, B.grain, B.fb);
    else
        k_coupled_step<Store, false, false><<<grid, block, 0, s>>>(P, src, srcf, dst, dstf, B.hist, B.grain, B.fb);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (B.ev_end && !B.ev_substeps) cudaEventRecord(B.ev_end, s);
    if ((e = walls<Store>(P, dst, dstf, 0, s, !(xwall && skip_columns))) != cudaSuccess) return e;
    B.cs = 1 - B.cs;
    B.cf = 1 - B.cf;
    const dim3 fblock(64, 4), fgrid((P.nx + 63) / 64, (P.ny + 3) / 4);
    for (int sub = 1; sub < n_sub; ++sub) {
        // phi and the force of time n come from hist/fb; the wall scheme reads
        // the scalar macros of time n+1 from the newest scalar buffer.  The
        // flow-only wall pass runs after the last sub-step only: each later
        // sub-step repairs the wall nodes it loads instead.
        if (sub == 1 && B.ev_begin && B.ev_substeps) cudaEventRecord(B.ev_begin, s);
        k_flow_substep<Store><<<fgrid, fblock, 0, s>>>(P, B.fl[B.cf], B.fl[1 - B.cf], B.hist, kHist, B.fb,
                                                       B.sc[B.cs], sub > 1);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (sub + 1 == n_sub && B.ev_end && B.ev_substeps) cudaEventRecord(B.ev_end, s);
        if (sub + 1 == n_sub && (e = walls<Store>(P, B.sc[B.cs], B.fl[1 - B.cf], 1, s)) != cudaSuccess) return e;
        B.cf = 1 - B.cf;
    }
    return cudaSuccess;
}

// run: tiles per CTA; 0 makes the grid persistent (one contiguous run of
// tiles per resident CTA).
// repair / skip_columns: as for the single-domain step; the column list holds
// the left/right walls of every domain that is not periodic in x.
template <class Store, int TYV>
cudaError_t batch_step_t(const BatchTables& T, int parity, int ctas, int run, cudaStream_t s, int repair,
                         int skip_columns)
{
    const int k = TYV == 4 ? 0 : TYV == 8 ? 1 : 2;
    const int chunk = run > 0 ? run : (T.ntiles[k] + ctas - 1) / ctas;
    const int grid = (T.ntiles[k] + chunk - 1) / chunk;
    if (T.ev_begin) cudaEventRecord(T.ev_begin, s);
    k_batch_step<Store, TYV><<<grid, dim3(TX, TYV), 0, s>>>(T.tiles[k], T.ntiles[k], chunk, parity, repair);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (T.ev_end) cudaEventRecord(T.ev_end, s);
    // the fused kernel wrote buffers 1 - parity; walls act on those (rows, then columns)
    if (T.nwall[0])
        k_batch_walls<Store><<<(T.nwall[0] + 127) / 128, 128, 0, s>>>(T.descs, T.walls[0], T.nwall[0], 1 - parity);
    if (T.nwall[1] && !skip_columns)
        k_batch_walls<Store><<<(T.nwall[1] + 127) / 128, 128, 0, s>>>(T.descs, T.walls[1], T.nwall[1], 1 - parity);
    return cudaGetLastError();
}

template <class Store>
cudaError_t batch_step_store(const BatchTables& T, int ty, int parity, int ctas, int run, cudaStream_t s,
                             int repair, int skip_columns)
{
    cudaError_t e = cudaMemcpyToSymbolAsync(c_batch_desc, T.descs, sizeof(DomainDesc) * T.ndomains, 0,
                                            cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    switch (ty) {
    case 4: return batch_step_t<Store, 4>(T, parity, ctas, run, s, repair, skip_columns);
    case 16: return batch_step_t<Store, 16>(T, parity, ctas, run, s, repair, skip_columns);
    default: return batch_step_t<Store, 8>(T, parity, ctas, run, s, repair, skip_columns);
    }
}

template <class Store, int TYV>
int batch_ctas_t()
{
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch_step<Store, TYV>, TX * TYV, 0);
    return sms * (per > 0 ? per : 1);
}

}  // namespace

cudaError_t launch_batch_step(const BatchTables& T, int storage, int ty, int run, int parity, int ctas,
                              cudaStream_t s, int repair, int skip_columns)
{
    switch (storage) {
    case kStoreF16: return batch_step_store<StoreF16>(T, ty, parity, ctas, run, s, repair, skip_columns);
    case kStoreBF16: return batch_step_store<StoreBF16>(T, ty, parity, ctas, run, s, repair, skip_columns);
    default: return batch_step_store<StoreF32>(T, ty, parity, ctas, run, s, repair, skip_columns);
    }
}

int batch_resident_ctas(int storage, int ty)
{
    if (storage == kStoreF16) return ty == 4 ? batch_ctas_t<StoreF16, 4>() : ty == 16 ? batch_ctas_t<StoreF16, 16>() : batch_ctas_t<StoreF16, 8>();
    if (storage == kStoreBF16) return ty == 4 ? batch_ctas_t<StoreBF16, 4>() : ty == 16 ? batch_ctas_t<StoreBF16, 16>() : batch_ctas_t<StoreBF16, 8>();
    return ty == 4 ? batch_ctas_t<StoreF32, 4>() : ty == 16 ? batch_ctas_t<StoreF32, 16>() : batch_ctas_t<StoreF32, 8>();
}

cudaError_t flow_steps(const StepParams& P, int storage, int n, void* sc, void* const fl[2], int* cf, const float* phi,
                       const float* fy, cudaStream_t s)
{
    switch (storage) {
    case kStoreF16: return flow_steps_t<StoreF16>(P, n, sc, fl, cf, phi, fy, s);
    case kStoreBF16: return flow_steps_t<StoreBF16>(P, n, sc, fl, cf, phi, fy, s);
    default: return flow_steps_t<StoreF32>(P, n, sc, fl, cf, phi, fy, s);
    }
}

cudaError_t launch_coupled_step(const StepParams& P, int storage, int n_sub, StepBuffers& B, cudaStream_t s,
                                int repair, int skip_columns)
{
    switch (storage) {
    case kStoreF16: return coupled_step<StoreF16>(P, n_sub, B, s, repair, skip_columns);
    case kStoreBF16: return coupled_step<StoreBF16>(P, n_sub, B, s, repair, skip_columns);
    default: return coupled_step<StoreF32>(P, n_sub, B, s, repair, skip_columns);
    }
}

}  // namespace lbm
