/*
 * FP64 CPU oracle of the diffuse-interface MRT lattice Boltzmann method of
 * Zhan, Chai, Shi, Jiang, Geng and Sun, "A diffuse-interface lattice
 * Boltzmann method for the dendritic growth with thermosolutal convection"
 * (arXiv 2209.01444).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA path is checked against.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark load it.  It shares no code, header,
 * table or constant with the CUDA library; it is written straight from the
 * paper, node by node, in population space: every collision is the paper's
 * Eq. (10) form  f* = f - Lambda (f - f^eq) + sources + (I - Lambda/2) G  with
 * Lambda = M^-1 S M built numerically from the printed transformation
 * matrices (Appendix B), never in moment space.
 *
 * Readings of points the paper leaves open (each is also listed in the design
 * notes of the repository):
 *   R1  seed profile  phi = tanh[(R - d)/(sqrt(2) W0)]  (Sec. 4, garbled there),
 *       several seeds: maximum over seeds, minimum-image distance on periodic
 *       axes;
 *   R2  a_s^2 in the modified phi streaming (Eq. 13, Remark 2) is taken at the
 *       source node x, time t;
 *   R3  time derivatives (dF/dt in Eq. 13, dphi/dt in Eq. 7, d(Cu)/dt in
 *       Eq. 19, d(Hu)/dt in Eq. 22) are first-order backward differences with
 *       the history initialised to the time-0 values (zero at the first step);
 *   R4  grad(phi) by the isotropic nine-point stencil
 *       grad(phi) = (1/cs^2) sum_i w_i c_i phi(x + c_i) (D2Q9 weights),
 *       mirror ghosts at non-periodic walls;
 *   R21 the local scheme of Sec. 3.1 (grad_mode 1): grad(phi) =
 *       -(s1/(cs^2 dt)) (sum_i c_i f_i + W0^2 N / tau0) with the node's own
 *       pre-collision f; s1 and N depend on grad(phi), so the formula is
 *       solved by fixed-point iteration from the isotropic guess (a_s = 1,
 *       N = 0), LOCAL_GRAD_ITERS passes;
 *   R22 the isothermal alloy of Sec. 4.3 (isothermal 1) drops the latent
 *       heat from the enthalpy, H = theta, so a uniform theta0 = 0 stays
 *       0 exactly and the phase field sees only the solute;
 *   R5  |grad(phi)|^2 < 1e-12 (lattice units): n = N = J_at = 0, a_s = 1;
 *   R6  D2Q5 weights 1/3, 1/6 (forced by cs^2 = 1/3), D2Q9 weights 4/9, 1/9,
 *       1/36;
 *   R7  fluid-solid force f = (u_s - u*)/dt with u_s = 0 (Sec. 3.4);
 *   R8  "other relaxation rates = 1": D2Q5 s0 = s2 = 1, D2Q9 s0 = s1 = s3 =
 *       s4 = 1, varphi = 0 so K is unused (Sec. 4);
 *   R9  external force F = constant body force + Boussinesq buoyancy
 *       (0, gbT (theta - theta_ref) + gbC (C - C_ref)), gravity along -y;
 *   R10 two-time-scaling (Sec. 4): the flow takes n_sub sub-steps of
 *       dt/n_sub per coupled step with phi, C, theta frozen; the scalar models
 *       see the velocity in their own lattice units, n_sub * u_flow;
 *   R11 boundaries: Guo's non-equilibrium extrapolation on the first/last node
 *       rows; the non-equilibrium part is taken from the first interior node
 *       with its macros of Eqs. (15)-(26) evaluated from the populations it
 *       holds after streaming; y walls are applied first, then x walls (the
 *       corners belong to the x walls);
 *   R12 Jacobi coupling: every model in step n uses time-n macros.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "lbm_oracle.h"

/* ---------------------------------------------------------------- lattices */
/* D2Q5, direction order fixed by the columns of M in Appendix B (Eq. B.1). */
static const int C5[5][2] = {{0, 0}, {1, 0}, {0, 1}, {-1, 0}, {0, -1}};
static const double W5[5] = {1.0 / 3.0, 1.0 / 6.0, 1.0 / 6.0, 1.0 / 6.0, 1.0 / 6.0};
/* D2Q9, direction order fixed by rows 2-3 of M in Appendix B (Eq. B.2). */
static const int C9[9][2] = {{0, 0}, {1, 0}, {0, 1}, {-1, 0}, {0, -1},
                             {1, 1}, {-1, 1}, {-1, -1}, {1, -1}};
static const double W9[9] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const double CS2 = 1.0 / 3.0; /* c_s^2 = c^2/3 with c = dx/dt = 1 (App. B) */
static const double GRAD_EPS2 = 1e-12; /* reading R5 */

/* ------------------------------------------------------- small linear algebra */
/* Gauss-Jordan inverse with partial pivoting of an n x n row-major matrix. */
static int mat_inverse(int n, const double* a, double* inv)
{
    double w[81 * 2];
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < 2 * n; ++c)
            w[r * 2 * n + c] = c < n ? a[r * n + c] : (c - n == r ? 1.0 : 0.0);
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r = col + 1; r < n; ++r)
            if (fabs(w[r * 2 * n + col]) > fabs(w[piv * 2 * n + col])) piv = r;
        if (fabs(w[piv * 2 * n + col]) < 1e-300) return -1;
        if (piv != col)
            for (int c = 0; c < 2 * n; ++c) {
                double t = w[col * 2 * n + c];
                w[col * 2 * n + c] = w[piv * 2 * n + c];
                w[piv * 2 * n + c] = t;
            }
        double d = w[col * 2 * n + col];
        for (int c = 0; c < 2 * n; ++c) w[col * 2 * n + c] /= d;
        for (int r = 0; r < n; ++r) {
            if (r == col) continue;
            double m = w[r * 2 * n + col];
            if (m == 0.0) continue;
            for (int c = 0; c < 2 * n; ++c) w[r * 2 * n + c] -= m * w[col * 2 * n + c];
        }
    }
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) inv[r * n + c] = w[r * 2 * n + n + c];
    return 0;
}

/* Lambda = M^-1 diag(S) M  (Appendix B). */
static void build_lambda(int n, const double* M, const double* Minv, const double* S, double* L)
{
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double acc = 0.0;
            for (int k = 0; k < n; ++k) acc += Minv[i * n + k] * S[k] * M[k * n + j];
            L[i * n + j] = acc;
        }
}

/* Moment rows of the D2Q5 matrix M (Eq. B.1): 1, c_x, c_y, c_x^2, c_y^2. */
void orc_lattice_M5(double* M)
{
    for (int i = 0; i < 5; ++i) {
        double cx = C5[i][0], cy = C5[i][1];
        M[0 * 5 + i] = 1.0;
        M[1 * 5 + i] = cx;
        M[2 * 5 + i] = cy;
        M[3 * 5 + i] = cx * cx;
        M[4 * 5 + i] = cy * cy;
    }
}

/* Moment rows of the D2Q9 raw-moment matrix M (Eq. B.2):
 * 1, c_x, c_y, c_x^2, c_y^2, c_x c_y, c_x^2 c_y, c_x c_y^2, c_x^2 c_y^2. */
void orc_lattice_M9(double* M)
{
    for (int i = 0; i < 9; ++i) {
        double cx = C9[i][0], cy = C9[i][1];
        M[0 * 9 + i] = 1.0;
        M[1 * 9 + i] = cx;
        M[2 * 9 + i] = cy;
        M[3 * 9 + i] = cx * cx;
        M[4 * 9 + i] = cy * cy;
        M[5 * 9 + i] = cx * cy;
        M[6 * 9 + i] = cx * cx * cy;
        M[7 * 9 + i] = cx * cy * cy;
        M[8 * 9 + i] = cx * cx * cy * cy;
    }
}

/* D2Q5 collision matrix for S = diag(s0, s1, s1, s2, s2) (Eq. B.1). */
int orc_lambda5(double s0, double s1, double s2, double* L)
{
    double M[25], Minv[25], S[5] = {s0, s1, s1, s2, s2};
    orc_lattice_M5(M);
    if (mat_inverse(5, M, Minv)) return -1;
    build_lambda(5, M, Minv, S, L);
    return 0;
}

/* D2Q9 collision matrix for a diagonal S given as 9 entries (App. B). */
int orc_lambda9(const double* S, double* L)
{
    double M[81], Minv[81];
    orc_lattice_M9(M);
    if (mat_inverse(9, M, Minv)) return -1;
    build_lambda(9, M, Minv, S, L);
    return 0;
}

/* -------------------------------------------- equilibria and source terms */
/* Eq. (14): f_i^eq = w_i phi. */
void orc_feq_phi(double phi, double* out)
{
    for (int i = 0; i < 5; ++i) out[i] = W5[i] * phi;
}

/* Eq. (14): dt F_i^phi = w_i Q_phi / tau0 (tau0 in time steps). */
void orc_F_phi(double Q, double tau, double* out)
{
    for (int i = 0; i < 5; ++i) out[i] = W5[i] * Q / tau;
}

/* Eq. (14): G_i^phi = -w_i c_i . N / a_s^2. */
void orc_G_phi(double Nx, double Ny, double as2, double* out)
{
    for (int i = 0; i < 5; ++i) out[i] = -W5[i] * (C5[i][0] * Nx + C5[i][1] * Ny) / as2;
}

/* Eq. (19): n_0^eq = C + (w_0 - 1) q U,  n_i^eq = w_i q U + w_i c_i . (C u) / cs^2
 * with qU = q~(phi) U and (Cux, Cuy) = C u. */
void orc_neq(double C, double qU, double Cux, double Cuy, double* out)
{
    out[0] = C + (W5[0] - 1.0) * qU;
    for (int i = 1; i < 5; ++i) out[i] = W5[i] * qU + W5[i] * (C5[i][0] * Cux + C5[i][1] * Cuy) / CS2;
}

/* Eq. (19): G_i^C = w_i c_i . [ d_t(C u)/cs^2 + U grad q~ + J_at / D ]. */
void orc_G_C(double dCux, double dCuy, double U, double gqx, double gqy, double Jx, double Jy, double D,
             double* out)
{
    double vx = dCux / CS2 + U * gqx + Jx / D;
    double vy = dCuy / CS2 + U * gqy + Jy / D;
    for (int i = 0; i < 5; ++i) out[i] = W5[i] * (C5[i][0] * vx + C5[i][1] * vy);
}

/* Eq. (22): g_0^eq = w_0 theta - L h(phi),  g_i^eq = w_i theta + w_i c_i . (H u)/cs^2,
 * with the latent term Lh = L h(phi): L = 1/2 as printed, L = 0 in the
 * isothermal mode (reading R22). */
void orc_geq(double theta, double Lh, double Hux, double Huy, double* out)
{
    out[0] = W5[0] * theta - Lh;
    for (int i = 1; i < 5; ++i) out[i] = W5[i] * theta + W5[i] * (C5[i][0] * Hux + C5[i][1] * Huy) / CS2;
}

/* Eq. (22): G_i^theta = w_i c_i . d_t(H u) / cs^2. */
void orc_G_theta(double dHux, double dHuy, double* out)
{
    for (int i = 0; i < 5; ++i) out[i] = W5[i] * (C5[i][0] * dHux + C5[i][1] * dHuy) / CS2;
}

/* Eq. (25): h_i^eq = sigma_i + w_i [ c_i.u/cs^2 + uu:(c_i c_i - cs^2 I)/(2 cs^4) ],
 * sigma_0 = (w_0 - 1) p/cs^2 + rho0, sigma_i = w_i p / cs^2. */
void orc_heq(double p, double ux, double uy, double rho0, double* out)
{
    for (int i = 0; i < 9; ++i) {
        double cu = C9[i][0] * ux + C9[i][1] * uy;
        double uu = ux * ux + uy * uy;
        double sigma = (i == 0) ? (W9[0] - 1.0) * p / CS2 + rho0 : W9[i] * p / CS2;
        out[i] = sigma + W9[i] * (cu / CS2 + (cu * cu - CS2 * uu) / (2.0 * CS2 * CS2));
    }
}

/* Eq. (25) with varphi = 0: F_i^u = w_i c_i . F' / cs^2,  F' = F + [1 - q~] f. */
void orc_F_u(double Fx, double Fy, double* out)
{
    for (int i = 0; i < 9; ++i) out[i] = W9[i] * (C9[i][0] * Fx + C9[i][1] * Fy) / CS2;
}

/* Eq. (2)-(3) for a gradient g = grad(phi) of a grain whose crystal axes are
 * rotated by `orient` (radians) from the lattice axes: the gradient is taken
 * into the crystal frame, a_s and N follow Eqs. (2)-(3) there, and N is rotated
 * back.  Degenerate gradients follow reading R5. */
void orc_anisotropy(double gx, double gy, double eps, double orient, double* as, double* Nx, double* Ny)
{
    double c = cos(orient), s = sin(orient);
    double px = c * gx + s * gy;  /* crystal-frame components of grad(phi) */
    double py = -s * gx + c * gy;
    double m2 = px * px + py * py; /* |grad phi|^2 */
    if (m2 < GRAD_EPS2) {
        *as = 1.0;
        *Nx = 0.0;
        *Ny = 0.0;
        return;
    }
    /* n = -grad(phi)/|grad(phi)|, so sum_a n_a^4 = (px^4 + py^4)/|g|^4. */
    double sum4 = (px * px * px * px + py * py * py * py) / (m2 * m2);
    double a = (1.0 - 3.0 * eps) * (1.0 + 4.0 * eps / (1.0 - 3.0 * eps) * sum4);
    /* d a_s / d(d_x phi) = 4 eps d/dpx[(px^4+py^4)/(px^2+py^2)^2]
     *                    = 16 eps px py^2 (px^2 - py^2) / |g|^6, likewise for y. */
    double dax = 16.0 * eps * px * py * py * (px * px - py * py) / (m2 * m2 * m2);
    double day = 16.0 * eps * py * px * px * (py * py - px * px) / (m2 * m2 * m2);
    double npx = m2 * a * dax; /* Eq. (3) in the crystal frame */
    double npy = m2 * a * day;
    *Nx = c * npx - s * npy;
    *Ny = s * npx + c * npy;
    *as = a;
}

/* Eq. (5). */
static double coupling_Q(double phi, double theta, double U, double lambda, double Mc)
{
    double w = 1.0 - phi * phi;
    return phi * w - lambda * (theta + Mc * U) * w * w;
}

/* h(phi) of Sec. 2: kind 0 is h = phi, kind 1 is 15/8 (phi - 2 phi^3/3 + phi^5/5). */
static double h_of_phi(int kind, double phi)
{
    if (kind == 1) {
        double p3 = phi * phi * phi;
        return 15.0 / 8.0 * (phi - 2.0 * p3 / 3.0 + p3 * phi * phi / 5.0);
    }
    return phi;
}

/* Eq. (4a)/(20): U from C and phi, and its inverse. */
static double U_of_C(double C, double phi, double k)
{
    return (2.0 * C / (1.0 + k - (1.0 - k) * phi) - 1.0) / (1.0 - k);
}
static double C_of_U(double U, double phi, double k)
{
    return 0.5 * (1.0 + k - (1.0 - k) * phi) * (1.0 + (1.0 - k) * U);
}

/* ----------------------------------------------------------------- the run */
struct orc_sim {
    orc_params P;
    int nx, ny, N;
    /* lattice-unit parameters */
    double W, tau, kappa0, Dl, s1C, s1T, s2u, vf, ff, nsub_scale;
    double uin_x, uin_y, Fx, Fy, gbT, gbC;
    double M5[25], M5inv[25];
    double LamC[25], LamT[25], LamU[81];
    /* populations at time n (pre-collision) and the next buffers */
    double *f, *nC, *g, *h;
    double *f2, *n2, *g2, *h2;
    /* history (time n-1 values) */
    double *phi_prev, *Q_prev, *Cu_prev, *Hu_prev;
    double* orient;
    /* macros at time n */
    double *phi, *C, *U, *theta, *H, *ux, *uy, *p;
    long long steps;
};

/* Latent-heat factor L of H = theta - L h(phi): 1/2 (Eq. 21), 0 in the
 * isothermal mode (reading R22). */
static double latent(const orc_sim* s) { return s->P.isothermal ? 0.0 : 0.5; }

static int is_periodic_x(const orc_sim* s) { return s->P.bc[0] == ORC_BC_PERIODIC; }
static int is_periodic_y(const orc_sim* s) { return s->P.bc[2] == ORC_BC_PERIODIC; }

/* Fixed-point passes of the local gradient scheme (reading R21). */
#define LOCAL_GRAD_ITERS 2

/* Index of (x + dx, y + dy) for the gradient stencil: periodic wrap, or a
 * mirror ghost about the wall node (reading R4). */
static int stencil_index(const orc_sim* s, int x, int y)
{
    if (x < 0) x = is_periodic_x(s) ? x + s->nx : -x;
    if (x >= s->nx) x = is_periodic_x(s) ? x - s->nx : 2 * (s->nx - 1) - x;
    if (y < 0) y = is_periodic_y(s) ? y + s->ny : -y;
    if (y >= s->ny) y = is_periodic_y(s) ? y - s->ny : 2 * (s->ny - 1) - y;
    return y * s->nx + x;
}

/* Destination of streaming from (x, y) along c: -1 when it leaves a
 * non-periodic domain (such values are replaced by the boundary scheme). */
static int stream_index(const orc_sim* s, int x, int y, int cx, int cy)
{
    int xx = x + cx, yy = y + cy;
    if (xx < 0 || xx >= s->nx) {
        if (!is_periodic_x(s)) return -1;
        xx = (xx + s->nx) % s->nx;
    }
    if (yy < 0 || yy >= s->ny) {
        if (!is_periodic_y(s)) return -1;
        yy = (yy + s->ny) % s->ny;
    }
    return yy * s->nx + xx;
}

static int valid_bc(int b) { return b >= ORC_BC_PERIODIC && b <= ORC_BC_DIRICHLET; }

orc_sim* orc_create(const orc_params* P)
{
    if (!P || P->nx < 4 || P->ny < 4) return NULL;
    if (P->W0 <= 0 || P->tau0 <= 0 || P->dx <= 0 || P->dt <= 0) return NULL;
    if (P->eps_s < 0 || P->eps_s >= 1.0 / 3.0 || P->k <= 0 || P->k >= 1) return NULL;
    if (P->D <= 0 || P->alpha <= 0 || P->nu <= 0 || P->n_sub < 1) return NULL;
    if (P->grad_mode != 0 && P->grad_mode != 1) return NULL;
    if (P->isothermal != 0 && P->isothermal != 1) return NULL;
    for (int b = 0; b < 4; ++b)
        if (!valid_bc(P->bc[b])) return NULL;
    if ((P->bc[0] == ORC_BC_PERIODIC) != (P->bc[1] == ORC_BC_PERIODIC)) return NULL;
    if ((P->bc[2] == ORC_BC_PERIODIC) != (P->bc[3] == ORC_BC_PERIODIC)) return NULL;

    orc_sim* s = (orc_sim*)calloc(1, sizeof(orc_sim));
    if (!s) return NULL;
    s->P = *P;
    s->nx = P->nx;
    s->ny = P->ny;
    s->N = P->nx * P->ny;
    /* Lattice units: dx = dt = 1 for the scalar models, dt/n_sub for the flow. */
    double dtf = P->dt / P->n_sub;
    s->W = P->W0 / P->dx;
    s->tau = P->tau0 / P->dt;
    s->kappa0 = s->W * s->W / s->tau;         /* W0^2 / tau0 */
    s->Dl = P->D * P->dt / (P->dx * P->dx);   /* D in lattice units */
    double al = P->alpha * P->dt / (P->dx * P->dx);
    double nul = P->nu * dtf / (P->dx * P->dx);
    /* Relaxation rates of Sec. 4. */
    s->s1C = 1.0 / (s->Dl * (1.0 - P->k) / CS2 + 0.5);
    s->s1T = 1.0 / (al / CS2 + 0.5);
    s->s2u = 1.0 / (nul / CS2 + 0.5);
    s->vf = dtf / P->dx;        /* paper velocity -> flow lattice velocity */
    s->ff = dtf * dtf / P->dx;  /* paper force/mass -> flow lattice force */
    s->nsub_scale = (double)P->n_sub; /* flow lattice velocity -> scalar lattice velocity */
    s->uin_x = P->u_in[0] * s->vf;
    s->uin_y = P->u_in[1] * s->vf;
    s->Fx = P->force[0] * s->ff;
    s->Fy = P->force[1] * s->ff;
    s->gbT = P->gbetaT * s->ff;
    s->gbC = P->gbetaC * s->ff;
    if (orc_lambda5(1.0, s->s1C, 1.0, s->LamC) || orc_lambda5(1.0, s->s1T, 1.0, s->LamT)) {
        free(s);
        return NULL;
    }
    orc_lattice_M5(s->M5);
    if (mat_inverse(5, s->M5, s->M5inv)) {
        free(s);
        return NULL;
    }
    double Su[9] = {1, 1, 1, s->s2u, s->s2u, s->s2u, 1, 1, 1};
    if (orc_lambda9(Su, s->LamU)) {
        free(s);
        return NULL;
    }
    size_t N = (size_t)s->N;
    double** arrays[] = {&s->f, &s->nC, &s->g, &s->f2, &s->n2, &s->g2};
    for (int a = 0; a < 6; ++a) *arrays[a] = (double*)calloc(5 * N, sizeof(double));
    s->h = (double*)calloc(9 * N, sizeof(double));
    s->h2 = (double*)calloc(9 * N, sizeof(double));
    s->phi_prev = (double*)calloc(N, sizeof(double));
    s->Q_prev = (double*)calloc(N, sizeof(double));
    s->Cu_prev = (double*)calloc(2 * N, sizeof(double));
    s->Hu_prev = (double*)calloc(2 * N, sizeof(double));
    s->orient = (double*)calloc(N, sizeof(double));
    double** macro[] = {&s->phi, &s->C, &s->U, &s->theta, &s->H, &s->ux, &s->uy, &s->p};
    for (int a = 0; a < 8; ++a) *macro[a] = (double*)calloc(N, sizeof(double));
    return s;
}

void orc_destroy(orc_sim* s)
{
    if (!s) return;
    double* all[] = {s->f, s->nC, s->g, s->h, s->f2, s->n2, s->g2, s->h2, s->phi_prev, s->Q_prev,
                     s->Cu_prev, s->Hu_prev, s->orient, s->phi, s->C, s->U, s->theta, s->H,
                     s->ux, s->uy, s->p};
    for (size_t a = 0; a < sizeof(all) / sizeof(all[0]); ++a) free(all[a]);
    free(s);
}

/* Flow lattice force of reading R9 at a node. */
static void body_force(const orc_sim* s, double theta, double C, double* Fx, double* Fy)
{
    *Fx = s->Fx;
    *Fy = s->Fy + s->gbT * (theta - s->P.theta_ref) + s->gbC * (C - s->P.C_ref);
}

/* Eq. (26): u* = sum c_i h_i + F/2, f = (u_s - u*)/dt with u_s = 0,
 * u = u* + [1 - q~] f / 2, and the pressure (varphi = 0). */
static void flow_macros(const double* hn, double phi, double Fx, double Fy, double* ux, double* uy,
                        double* fsx, double* fsy, double* p)
{
    double mx = 0, my = 0, rest = 0;
    for (int i = 0; i < 9; ++i) {
        mx += C9[i][0] * hn[i];
        my += C9[i][1] * hn[i];
        if (i) rest += hn[i];
    }
    double usx = mx + 0.5 * Fx, usy = my + 0.5 * Fy;
    double qt = 0.5 * (1.0 - phi);
    *fsx = (0.0 - usx);
    *fsy = (0.0 - usy);
    *ux = usx + 0.5 * (1.0 - qt) * (*fsx);
    *uy = usy + 0.5 * (1.0 - qt) * (*fsy);
    *p = CS2 / (1.0 - W9[0]) * (rest - W9[0] * ((*ux) * (*ux) + (*uy) * (*uy)) / (2.0 * CS2));
}

/* Macroscopic values of one node (Eqs. 15, 20, 23, 26) from population
 * arrays f, n, g [5][N] and h [9][N]. */
typedef struct {
    double phi, C, U, theta, H, ux, uy, p;
} node_macro;

static node_macro macros_at(const orc_sim* s, const double* f, const double* n, const double* g,
                            const double* h, int x)
{
    const int N = s->N;
    node_macro m;
    double phi = 0, C = 0, H = 0, hn[9];
    for (int i = 0; i < 5; ++i) {
        phi += f[i * N + x];
        C += n[i * N + x];
        H += g[i * N + x];
    }
    for (int i = 0; i < 9; ++i) hn[i] = h[i * N + x];
    double theta = H + latent(s) * h_of_phi(s->P.h_kind, phi);
    double Fx, Fy, fsx, fsy;
    body_force(s, theta, C, &Fx, &Fy);
    flow_macros(hn, phi, Fx, Fy, &m.ux, &m.uy, &fsx, &fsy, &m.p);
    m.phi = phi;
    m.C = C;
    m.U = U_of_C(C, phi, s->P.k);
    m.theta = theta;
    m.H = H;
    return m;
}

/* All macroscopic fields at the current time level. */
static void compute_macros(orc_sim* s)
{
    const int N = s->N;
#pragma omp parallel for schedule(static)
    for (int x = 0; x < N; ++x) {
        node_macro m = macros_at(s, s->f, s->nC, s->g, s->h, x);
        s->phi[x] = m.phi;
        s->C[x] = m.C;
        s->U[x] = m.U;
        s->theta[x] = m.theta;
        s->H[x] = m.H;
        s->ux[x] = m.ux;
        s->uy[x] = m.uy;
        s->p[x] = m.p;
    }
}

/* Generic population-space MRT collision of Eq. (10):
 * out_i = f_i - sum_j L_ij (f_j - feq_j) + sum_j (delta_ij - L_ij/2) G_j. */
static void collide(int q, const double* L, const double* fn, const double* feq, const double* G,
                    double* out)
{
    for (int i = 0; i < q; ++i) {
        double coll = 0.0, aux = 0.0;
        for (int j = 0; j < q; ++j) {
            coll += L[i * q + j] * (fn[j] - feq[j]);
            aux += ((i == j ? 1.0 : 0.0) - 0.5 * L[i * q + j]) * G[j];
        }
        out[i] = fn[i] - coll + aux;
    }
}

/* Flow collision, Eq. (24)-(25), then push streaming into h2. */
static void collide_stream_flow(orc_sim* s, int x, int y, double phi, double Fx, double Fy)
{
    const int N = s->N, idx = y * s->nx + x;
    double hn[9], heq[9], Fu[9], hs[9];
    for (int i = 0; i < 9; ++i) hn[i] = s->h[i * N + idx];
    double ux, uy, fsx, fsy, p;
    flow_macros(hn, phi, Fx, Fy, &ux, &uy, &fsx, &fsy, &p);
    double qt = 0.5 * (1.0 - phi);
    orc_heq(p, ux, uy, s->P.rho0, heq);
    orc_F_u(Fx + (1.0 - qt) * fsx, Fy + (1.0 - qt) * fsy, Fu);
    collide(9, s->LamU, hn, heq, Fu, hs);
    for (int i = 0; i < 9; ++i) {
        int d = stream_index(s, x, y, C9[i][0], C9[i][1]);
        if (d >= 0) s->h2[i * N + d] = hs[i];
    }
}

/* --------------------------------------------------------------- boundaries */
/* Guo's non-equilibrium extrapolation (Sec. 4, reading R11) at boundary node
 * b with first interior node f on side `side` (0 left, 1 right, 2 bottom,
 * 3 top), on the freshly streamed buffers f2/n2/g2/h2:
 *   pop(b) = pop^eq(boundary macros) + [pop(f) - pop^eq(macros of f)],
 * where the macros of f are those of Eqs. (15), (20), (23), (26) evaluated
 * from the populations held at f. */
static void nee_node(orc_sim* s, double* fp, double* np_, double* gp, int b, int f, int side, int flow_only)
{
    const int N = s->N;
    const int type = s->P.bc[side];
    const double k = s->P.k;
    const node_macro mf = macros_at(s, fp, np_, gp, s->h2, f);
    double ubx, uby, pb = mf.p;
    switch (type) {
    case ORC_BC_INFLOW:
        ubx = s->uin_x;
        uby = s->uin_y;
        break;
    case ORC_BC_OUTFLOW:
        ubx = mf.ux;
        uby = mf.uy;
        pb = 0.0;
        break;
    case ORC_BC_SYMMETRY:
        ubx = (side < 2) ? 0.0 : mf.ux;
        uby = (side < 2) ? mf.uy : 0.0;
        break;
    default: /* no-slip and Dirichlet walls */
        ubx = 0.0;
        uby = 0.0;
        break;
    }
    double eb[9], ef[9];
    orc_heq(pb, ubx, uby, s->P.rho0, eb);
    orc_heq(mf.p, mf.ux, mf.uy, s->P.rho0, ef);
    for (int i = 0; i < 9; ++i) s->h2[i * N + b] = eb[i] + s->h2[i * N + f] - ef[i];
    if (flow_only) return;

    /* scalars: zero gradient, or the Dirichlet far field of Sec. 4.4 */
    double phib = mf.phi, Cb = mf.C, Ub = mf.U, thetab = mf.theta;
    if (type == ORC_BC_DIRICHLET) {
        phib = s->P.dir_phi;
        Ub = s->P.dir_U;
        Cb = C_of_U(Ub, phib, k);
        thetab = s->P.dir_theta;
    }
    const double hb = h_of_phi(s->P.h_kind, phib), hf = h_of_phi(s->P.h_kind, mf.phi);
    const double L = latent(s);
    const double Hb = thetab - L * hb;
    const double sc = s->nsub_scale;
    orc_feq_phi(phib, eb);
    orc_feq_phi(mf.phi, ef);
    for (int i = 0; i < 5; ++i) fp[i * N + b] = eb[i] + fp[i * N + f] - ef[i];
    orc_neq(Cb, 0.5 * (1.0 - phib) * Ub, Cb * ubx * sc, Cb * uby * sc, eb);
    orc_neq(mf.C, 0.5 * (1.0 - mf.phi) * mf.U, mf.C * mf.ux * sc, mf.C * mf.uy * sc, ef);
    for (int i = 0; i < 5; ++i) np_[i * N + b] = eb[i] + np_[i * N + f] - ef[i];
    orc_geq(thetab, L * hb, Hb * ubx * sc, Hb * uby * sc, eb);
    orc_geq(mf.theta, L * hf, mf.H * mf.ux * sc, mf.H * mf.uy * sc, ef);
    for (int i = 0; i < 5; ++i) gp[i * N + b] = eb[i] + gp[i * N + f] - ef[i];
}

/* The scalar arrays passed in are the newest scalar populations: the freshly
 * streamed f2/n2/g2 in the coupled step, f/nC/g (time n+1) during the flow
 * sub-steps.  The flow populations are always the freshly streamed h2. */
static void apply_boundaries(orc_sim* s, double* fp, double* np_, double* gp, int flow_only)
{
    const int nx = s->nx, ny = s->ny;
    if (!is_periodic_y(s)) {
        int xlo = is_periodic_x(s) ? 0 : 1, xhi = is_periodic_x(s) ? nx - 1 : nx - 2;
        for (int x = xlo; x <= xhi; ++x) {
            nee_node(s, fp, np_, gp, 0 * nx + x, 1 * nx + x, 2, flow_only);
            nee_node(s, fp, np_, gp, (ny - 1) * nx + x, (ny - 2) * nx + x, 3, flow_only);
        }
    }
    if (!is_periodic_x(s)) {
        for (int y = 0; y < ny; ++y) {
            nee_node(s, fp, np_, gp, y * nx + 0, y * nx + 1, 0, flow_only);
            nee_node(s, fp, np_, gp, y * nx + nx - 1, y * nx + nx - 2, 1, flow_only);
        }
    }
}

static void swap_ptr(double** a, double** b)
{
    double* t = *a;
    *a = *b;
    *b = t;
}

/* grad(phi) at node (x, y) of the current state (phi from compute_macros):
 * the nine-point stencil of reading R4, or the local scheme of Sec. 3.1
 * (reading R21) from the node's own pre-collision f. */
static void grad_phi(const orc_sim* s, int x, int y, double* gxo, double* gyo)
{
    const orc_params* P = &s->P;
    const int N = s->N, idx = y * s->nx + x;
    double gx = 0.0, gy = 0.0;
    if (P->grad_mode == 1) {
        double jx = 0.0, jy = 0.0;
        for (int i = 1; i < 5; ++i) {
            jx += C5[i][0] * s->f[i * N + idx];
            jy += C5[i][1] * s->f[i * N + idx];
        }
        double a1 = 1.0, nx_ = 0.0, ny_ = 0.0;
        for (int it = 0; it <= LOCAL_GRAD_ITERS; ++it) {
            if (it > 0) orc_anisotropy(gx, gy, P->eps_s, s->orient[idx], &a1, &nx_, &ny_);
            const double s1 = 1.0 / (a1 * a1 * s->kappa0 / CS2 + 0.5);
            gx = -s1 / CS2 * (jx + s->kappa0 * nx_);
            gy = -s1 / CS2 * (jy + s->kappa0 * ny_);
        }
    } else {
        for (int i = 1; i < 9; ++i) {
            double ph = s->phi[stencil_index(s, x + C9[i][0], y + C9[i][1])];
            gx += W9[i] * C9[i][0] * ph;
            gy += W9[i] * C9[i][1] * ph;
        }
        gx /= CS2;
        gy /= CS2;
    }
    *gxo = gx;
    *gyo = gy;
}

/* grad(phi) of every node by the given scheme (0 stencil, 1 local), out =
 * [2][ny][nx] in lattice units (per lattice spacing). */
int orc_grad_phi(orc_sim* s, int mode, double* out)
{
    if (!s || !out || (mode != 0 && mode != 1)) return -1;
    compute_macros(s);
    const int keep = s->P.grad_mode;
    s->P.grad_mode = mode;
    for (int y = 0; y < s->ny; ++y)
        for (int x = 0; x < s->nx; ++x) {
            const int idx = y * s->nx + x;
            grad_phi(s, x, y, &out[idx], &out[s->N + idx]);
        }
    s->P.grad_mode = keep;
    return 0;
}

/* One coupled step n -> n+1 (the order of reading R12). */
static void coupled_step(orc_sim* s)
{
    const int nx = s->nx, ny = s->ny, N = s->N;
    const orc_params* P = &s->P;
    compute_macros(s);

#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            const int idx = y * nx + x;
            const double phi = s->phi[idx], C = s->C[idx], U = s->U[idx];
            const double theta = s->theta[idx], H = s->H[idx];
            /* velocity seen by the scalar models (reading R10) */
            const double usx = s->ux[idx] * s->nsub_scale, usy = s->uy[idx] * s->nsub_scale;

            double gx, gy;
            grad_phi(s, x, y, &gx, &gy);
            double as, Nx, Ny;
            orc_anisotropy(gx, gy, P->eps_s, s->orient[idx], &as, &Nx, &Ny);
            const double as2 = as * as;
            const double g2 = gx * gx + gy * gy;
            const double Q = coupling_Q(phi, theta, U, P->lambda, P->Mc_inf);

            /* ---- phase field, Eqs. (13)-(14) */
            double fn[5], feq[5], F[5], dF[5], G[5], Lphi[25], fs[5];
            for (int i = 0; i < 5; ++i) fn[i] = s->f[i * N + idx];
            orc_feq_phi(phi, feq);
            orc_F_phi(Q, s->tau, F);
            orc_F_phi(Q - s->Q_prev[idx], s->tau, dF); /* dt * d_t F by backward difference */
            orc_G_phi(Nx, Ny, as2, G);
            const double s1phi = 1.0 / (as2 * s->kappa0 / CS2 + 0.5); /* Sec. 3.1 */
            const double Sphi[5] = {1.0, s1phi, s1phi, 1.0, 1.0};
            build_lambda(5, s->M5, s->M5inv, Sphi, Lphi);
            collide(5, Lphi, fn, feq, G, fs);
            for (int i = 0; i < 5; ++i) fs[i] += F[i] + 0.5 * as2 * dF[i];
            /* modified streaming, Eq. (13) with Remark 2:
             * a_s^2 f_i(x+c_i, t+1) = f*_i(x) - [1 - a_s^2] f_i(x+c_i, t) */
            for (int i = 0; i < 5; ++i) {
                int d = stream_index(s, x, y, C5[i][0], C5[i][1]);
                if (d >= 0) s->f2[i * N + d] = (fs[i] - (1.0 - as2) * s->f[i * N + d]) / as2;
            }

            /* ---- solute, Eqs. (17)-(19) with J_at of Eq. (7) */
            const double qt = 0.5 * (1.0 - phi);
            const double Cux = C * usx, Cuy = C * usy;
            double Jx = 0.0, Jy = 0.0;
            if (!(g2 < GRAD_EPS2)) {
                double gn = sqrt(g2);
                double a = -1.0 / (2.0 * sqrt(2.0)) * s->W * (1.0 + (1.0 - P->k) * U) *
                           (phi - s->phi_prev[idx]);
                Jx = a * gx / gn;
                Jy = a * gy / gn;
            }
            double nn[5], neq[5], GC[5], ns[5];
            for (int i = 0; i < 5; ++i) nn[i] = s->nC[i * N + idx];
            orc_neq(C, qt * U, Cux, Cuy, neq);
            orc_G_C(Cux - s->Cu_prev[idx], Cuy - s->Cu_prev[N + idx], U, -0.5 * gx, -0.5 * gy, Jx, Jy,
                    s->Dl, GC);
            collide(5, s->LamC, nn, neq, GC, ns);
            for (int i = 0; i < 5; ++i) {
                int d = stream_index(s, x, y, C5[i][0], C5[i][1]);
                if (d >= 0) s->n2[i * N + d] = ns[i];
            }

            /* ---- heat, Eqs. (21)-(23) */
            const double Hux = H * usx, Huy = H * usy;
            double gg[5], geq[5], GT[5], gs[5];
            for (int i = 0; i < 5; ++i) gg[i] = s->g[i * N + idx];
            orc_geq(theta, latent(s) * h_of_phi(P->h_kind, phi), Hux, Huy, geq);
            orc_G_theta(Hux - s->Hu_prev[idx], Huy - s->Hu_prev[N + idx], GT);
            collide(5, s->LamT, gg, geq, GT, gs);
            for (int i = 0; i < 5; ++i) {
                int d = stream_index(s, x, y, C5[i][0], C5[i][1]);
                if (d >= 0) s->g2[i * N + d] = gs[i];
            }

            /* ---- flow, Eqs. (24)-(26), first sub-step */
            double Fx, Fy;
            body_force(s, theta, C, &Fx, &Fy);
            collide_stream_flow(s, x, y, phi, Fx, Fy);
        }
    }
    apply_boundaries(s, s->f2, s->n2, s->g2, 0);

    /* history for the backward differences (reading R3) */
#pragma omp parallel for schedule(static)
    for (int idx = 0; idx < N; ++idx) {
        const double usx = s->ux[idx] * s->nsub_scale, usy = s->uy[idx] * s->nsub_scale;
        s->phi_prev[idx] = s->phi[idx];
        s->Q_prev[idx] = coupling_Q(s->phi[idx], s->theta[idx], s->U[idx], P->lambda, P->Mc_inf);
        s->Cu_prev[idx] = s->C[idx] * usx;
        s->Cu_prev[N + idx] = s->C[idx] * usy;
        s->Hu_prev[idx] = s->H[idx] * usx;
        s->Hu_prev[N + idx] = s->H[idx] * usy;
    }
    swap_ptr(&s->f, &s->f2);
    swap_ptr(&s->nC, &s->n2);
    swap_ptr(&s->g, &s->g2);
    swap_ptr(&s->h, &s->h2);

    /* remaining flow sub-steps with phi, C, theta frozen at time n (reading R10) */
    for (int sub = 1; sub < P->n_sub; ++sub) {
#pragma omp parallel for schedule(static)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const int idx = y * nx + x;
                double Fx, Fy;
                body_force(s, s->theta[idx], s->C[idx], &Fx, &Fy);
                collide_stream_flow(s, x, y, s->phi[idx], Fx, Fy);
            }
        apply_boundaries(s, s->f, s->nC, s->g, 1);
        swap_ptr(&s->h, &s->h2);
    }
    s->steps++;
}

/* Flow-only steps with phi, C and theta frozen: the flow model of Sec. 3.4
 * alone, as in the stationary-cylinder problem of Sec. 4.1 (the phase field
 * does not evolve there).  Each step is one collision + streaming of h with
 * the fluid-solid force and the body force of the frozen fields, then the
 * flow boundaries (the same operations as a two-time-scaling sub-step).  The
 * coupled-step count does not change. */
int orc_step_flow(orc_sim* s, int nsteps)
{
    if (!s || nsteps < 0) return -1;
    const int nx = s->nx, ny = s->ny;
    compute_macros(s);
    for (int n = 0; n < nsteps; ++n) {
#pragma omp parallel for schedule(static)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const int idx = y * nx + x;
                double Fx, Fy;
                body_force(s, s->theta[idx], s->C[idx], &Fx, &Fy);
                collide_stream_flow(s, x, y, s->phi[idx], Fx, Fy);
            }
        apply_boundaries(s, s->f, s->nC, s->g, 1);
        swap_ptr(&s->h, &s->h2);
    }
    return 0;
}

/* Hydrodynamic force and torque on the solid, Eq. (27) (HDforce): the paper
 * sums f over the nodes covered by the solid; in the diffuse interface the
 * force the flow feels at a node is [1 - q~] f (Eq. 24), so the sum here is
 * weighted by 1 - q~ = (1 + phi)/2 (reading).  With dx = 1 in flow lattice
 * units: out[0..1] = F_f = -sum (1 - q~) f, out[2] = T_f = -sum (x - xs) x
 * (1 - q~) f about (cx, cy), in flow lattice units. */
int orc_force(orc_sim* s, double cx, double cy, double* out)
{
    if (!s || !out) return -1;
    compute_macros(s);
    const int nx = s->nx, ny = s->ny, N = s->N;
    double Fx = 0, Fy = 0, T = 0;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            const int idx = y * nx + x;
            double hn[9];
            for (int i = 0; i < 9; ++i) hn[i] = s->h[i * N + idx];
            double bx, by, ux, uy, fsx, fsy, p;
            body_force(s, s->theta[idx], s->C[idx], &bx, &by);
            flow_macros(hn, s->phi[idx], bx, by, &ux, &uy, &fsx, &fsy, &p);
            const double w = 0.5 * (1.0 + s->phi[idx]);
            Fx -= w * fsx;
            Fy -= w * fsy;
            T -= (x - cx) * w * fsy - (y - cy) * w * fsx;
        }
    out[0] = Fx;
    out[1] = Fy;
    out[2] = T;
    return 0;
}

int orc_step(orc_sim* s, int nsteps)
{
    if (!s || nsteps < 0) return -1;
    for (int n = 0; n < nsteps; ++n) coupled_step(s);
    return 0;
}

long long orc_step_count(const orc_sim* s) { return s ? s->steps : -1; }

/* ------------------------------------------------------------ initial state */
/* Populations at equilibrium of the given lattice-unit macros, then history
 * = the time-0 macros recovered from those populations (reading R3). */
static void set_equilibrium_state(orc_sim* s, const double* phi, const double* U, const double* theta,
                                  const double* ux, const double* uy, const double* p)
{
    const int N = s->N;
    const double k = s->P.k, sc = s->nsub_scale;
#pragma omp parallel for schedule(static)
    for (int x = 0; x < N; ++x) {
        double C = C_of_U(U[x], phi[x], k);
        double hphi = h_of_phi(s->P.h_kind, phi[x]);
        double H = theta[x] - latent(s) * hphi;
        double e[9];
        orc_feq_phi(phi[x], e);
        for (int i = 0; i < 5; ++i) s->f[i * N + x] = e[i];
        orc_neq(C, 0.5 * (1.0 - phi[x]) * U[x], C * ux[x] * sc, C * uy[x] * sc, e);
        for (int i = 0; i < 5; ++i) s->nC[i * N + x] = e[i];
        orc_geq(theta[x], latent(s) * hphi, H * ux[x] * sc, H * uy[x] * sc, e);
        for (int i = 0; i < 5; ++i) s->g[i * N + x] = e[i];
        orc_heq(p[x], ux[x], uy[x], s->P.rho0, e);
        for (int i = 0; i < 9; ++i) s->h[i * N + x] = e[i];
    }
    compute_macros(s);
#pragma omp parallel for schedule(static)
    for (int x = 0; x < N; ++x) {
        s->phi_prev[x] = s->phi[x];
        s->Q_prev[x] = coupling_Q(s->phi[x], s->theta[x], s->U[x], s->P.lambda, s->P.Mc_inf);
        s->Cu_prev[x] = s->C[x] * s->ux[x] * sc;
        s->Cu_prev[N + x] = s->C[x] * s->uy[x] * sc;
        s->Hu_prev[x] = s->H[x] * s->ux[x] * sc;
        s->Hu_prev[N + x] = s->H[x] * s->uy[x] * sc;
    }
    s->steps = 0;
}

/* Minimum-image offset along an axis of length L. */
static double axis_offset(double d, int L, int periodic)
{
    if (!periodic) return d;
    while (d > 0.5 * L) d -= L;
    while (d < -0.5 * L) d += L;
    return d;
}

/* Seeds [x, y, R, orientation] in lattice units/radians (reading R1; grain map
 * = nearest seed centre, ties to the lower index), placed on a window of a
 * larger gnx x gny domain: node (i, j) of this grid is node (gx0 + i, gy0 + j)
 * of the large one, whose periodicity is (gpx, gpy).  The plain seeded start
 * is the window covering the whole domain. */
int orc_init_seeds_window(orc_sim* s, const double* seeds, int ns, double U0, double theta0, int gx0, int gy0,
                          int gnx, int gny, int gpx, int gpy)
{
    if (!s || ns < 1 || !seeds) return -1;
    const int N = s->N, nx = s->nx;
    double* buf = (double*)malloc(6 * (size_t)N * sizeof(double));
    if (!buf) return -1;
    double *phi = buf, *U = buf + N, *th = buf + 2 * N, *ux = buf + 3 * N, *uy = buf + 4 * N,
           *p = buf + 5 * N;
#pragma omp parallel for schedule(static)
    for (int idx = 0; idx < N; ++idx) {
        int x = (gx0 + idx % nx) % gnx, y = (gy0 + idx / nx) % gny;
        double best_phi = -2.0, best_d2 = 1e300;
        int best = 0;
        for (int j = 0; j < ns; ++j) {
            double dxs = axis_offset(x - seeds[4 * j + 0], gnx, gpx);
            double dys = axis_offset(y - seeds[4 * j + 1], gny, gpy);
            double d2 = dxs * dxs + dys * dys;
            double ph = tanh((seeds[4 * j + 2] - sqrt(d2)) / (sqrt(2.0) * s->W));
            if (ph > best_phi) best_phi = ph;
            if (d2 < best_d2) {
                best_d2 = d2;
                best = j;
            }
        }
        phi[idx] = best_phi;
        s->orient[idx] = seeds[4 * best + 3];
        U[idx] = U0;
        th[idx] = theta0;
        ux[idx] = uy[idx] = p[idx] = 0.0;
    }
    set_equilibrium_state(s, phi, U, th, ux, uy, p);
    free(buf);
    return 0;
}

int orc_init_seeds(orc_sim* s, const double* seeds, int ns, double U0, double theta0)
{
    if (!s) return -1;
    return orc_init_seeds_window(s, seeds, ns, U0, theta0, 0, 0, s->nx, s->ny, is_periodic_x(s),
                                 is_periodic_y(s));
}

/* fields [6][N]: phi, U, theta, ux, uy, p with velocity and pressure in paper
 * units; orient [N] in radians or NULL for 0. */
int orc_init_fields(orc_sim* s, const double* fields, const double* orient)
{
    if (!s || !fields) return -1;
    const int N = s->N;
    double* buf = (double*)malloc(3 * (size_t)N * sizeof(double));
    if (!buf) return -1;
    double dtf = s->P.dt / s->P.n_sub;
    double pscale = dtf * dtf / (s->P.dx * s->P.dx);
    for (int x = 0; x < N; ++x) {
        buf[x] = fields[3 * N + x] * s->vf;
        buf[N + x] = fields[4 * N + x] * s->vf;
        buf[2 * N + x] = fields[5 * N + x] * pscale;
        s->orient[x] = orient ? orient[x] : 0.0;
    }
    set_equilibrium_state(s, fields, fields + N, fields + 2 * N, buf, buf + N, buf + 2 * N);
    free(buf);
    return 0;
}

/* out [7][N]: phi, C, U, theta, ux, uy, p (velocity and pressure in paper units). */
int orc_get_fields(orc_sim* s, double* out)
{
    if (!s || !out) return -1;
    compute_macros(s);
    const int N = s->N;
    double dtf = s->P.dt / s->P.n_sub;
    double pscale = (s->P.dx * s->P.dx) / (dtf * dtf);
    for (int x = 0; x < N; ++x) {
        out[0 * N + x] = s->phi[x];
        out[1 * N + x] = s->C[x];
        out[2 * N + x] = s->U[x];
        out[3 * N + x] = s->theta[x];
        out[4 * N + x] = s->ux[x] / s->vf;
        out[5 * N + x] = s->uy[x] / s->vf;
        out[6 * N + x] = s->p[x] * pscale;
    }
    return 0;
}

/* State [30][N]: f(5), n(5), g(5), h(9), phi_prev, Q_prev, Cu_prev(2), Hu_prev(2). */
int orc_get_state(const orc_sim* s, double* out)
{
    if (!s || !out) return -1;
    size_t N = (size_t)s->N;
    memcpy(out, s->f, 5 * N * sizeof(double));
    memcpy(out + 5 * N, s->nC, 5 * N * sizeof(double));
    memcpy(out + 10 * N, s->g, 5 * N * sizeof(double));
    memcpy(out + 15 * N, s->h, 9 * N * sizeof(double));
    memcpy(out + 24 * N, s->phi_prev, N * sizeof(double));
    memcpy(out + 25 * N, s->Q_prev, N * sizeof(double));
    memcpy(out + 26 * N, s->Cu_prev, 2 * N * sizeof(double));
    memcpy(out + 28 * N, s->Hu_prev, 2 * N * sizeof(double));
    return 0;
}

int orc_set_state(orc_sim* s, const double* in)
{
    if (!s || !in) return -1;
    size_t N = (size_t)s->N;
    memcpy(s->f, in, 5 * N * sizeof(double));
    memcpy(s->nC, in + 5 * N, 5 * N * sizeof(double));
    memcpy(s->g, in + 10 * N, 5 * N * sizeof(double));
    memcpy(s->h, in + 15 * N, 9 * N * sizeof(double));
    memcpy(s->phi_prev, in + 24 * N, N * sizeof(double));
    memcpy(s->Q_prev, in + 25 * N, N * sizeof(double));
    memcpy(s->Cu_prev, in + 26 * N, 2 * N * sizeof(double));
    memcpy(s->Hu_prev, in + 28 * N, 2 * N * sizeof(double));
    return 0;
}

int orc_get_orient(const orc_sim* s, double* out)
{
    if (!s || !out) return -1;
    memcpy(out, s->orient, (size_t)s->N * sizeof(double));
    return 0;
}

/* ----------------------------------------------------------------- metrics */
static double bilinear(const orc_sim* s, const double* a, double px, double py)
{
    int i = (int)floor(px), j = (int)floor(py);
    if (i > s->nx - 2) i = s->nx - 2;
    if (j > s->ny - 2) j = s->ny - 2;
    double fx = px - i, fy = py - j;
    const double* r0 = a + (size_t)j * s->nx;
    const double* r1 = r0 + s->nx;
    return (1 - fx) * (1 - fy) * r0[i] + fx * (1 - fy) * r0[i + 1] + (1 - fx) * fy * r1[i] +
           fx * fy * r1[i + 1];
}

/* Tip distance (lattice units) from (cx, cy) along the unit vector (ex, ey):
 * phi is sampled bilinearly every half node while the sample stays inside the
 * grid; the outermost sample with phi > 0 and its outward neighbour are
 * interpolated linearly to phi = 0.  NaN if no sample is solid.  (The paper
 * uses tip positions without defining them; this is the definition used
 * throughout this repository.) */
static double tip_along(const orc_sim* s, double cx, double cy, double ex, double ey)
{
    const double ds = 0.5;
    int last = -1;
    double vlast = 0, vnext = 0;
    int have_next = 0;
    for (int j = 0;; ++j) {
        double px = cx + j * ds * ex, py = cy + j * ds * ey;
        if (px < 0 || py < 0 || px > s->nx - 1 || py > s->ny - 1) break;
        double v = bilinear(s, s->phi, px, py);
        if (v > 0) {
            last = j;
            vlast = v;
            have_next = 0;
        } else if (last == j - 1 && last >= 0) {
            vnext = v;
            have_next = 1;
        }
    }
    if (last < 0) return NAN;
    if (!have_next) return last * ds;
    return (last + vlast / (vlast - vnext)) * ds;
}

/* out[10]: tip +x, tip -x, tip +y (crystal axes of orientation `orient`
 * through (cx, cy), lattice units), solid fraction sum((1+phi)/2)/N,
 * sum C, sum H, sum of all h_i, max |u| (paper units), non-finite flag,
 * sum phi.  Sums run over nodes in row-major order. */
int orc_metrics(orc_sim* s, double cx, double cy, double orient, double* out)
{
    if (!s || !out) return -1;
    compute_macros(s);
    const int N = s->N;
    double c = cos(orient), sn = sin(orient);
    out[0] = tip_along(s, cx, cy, c, sn);
    out[1] = tip_along(s, cx, cy, -c, -sn);
    out[2] = tip_along(s, cx, cy, -sn, c);
    double sf = 0, sC = 0, sH = 0, sh = 0, umax = 0, sphi = 0;
    int bad = 0;
    for (int x = 0; x < N; ++x) {
        sf += 0.5 * (1.0 + s->phi[x]);
        sC += s->C[x];
        sH += s->H[x];
        sphi += s->phi[x];
        for (int i = 0; i < 9; ++i) sh += s->h[i * N + x];
        double u = sqrt(s->ux[x] * s->ux[x] + s->uy[x] * s->uy[x]) / s->vf;
        if (u > umax) umax = u;
        if (!isfinite(s->phi[x]) || !isfinite(s->C[x]) || !isfinite(s->theta[x]) || !isfinite(u)) bad = 1;
    }
    out[3] = sf / N;
    out[4] = sC;
    out[5] = sH;
    out[6] = sh;
    out[7] = umax;
    out[8] = bad;
    out[9] = sphi;
    return 0;
}

/* Lattice-unit parameters derived in orc_create, for inspection:
 * [W, tau, kappa0, D, s1C, s1T, s2u, velocity scale, force scale]. */
int orc_lattice_params(const orc_sim* s, double* out)
{
    if (!s || !out) return -1;
    out[0] = s->W;
    out[1] = s->tau;
    out[2] = s->kappa0;
    out[3] = s->Dl;
    out[4] = s->s1C;
    out[5] = s->s1T;
    out[6] = s->s2u;
    out[7] = s->vf;
    out[8] = s->ff;
    return 0;
}
