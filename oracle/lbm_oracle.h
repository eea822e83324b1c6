/*
 * Interface of the FP64 CPU oracle (test infrastructure only; see
 * lbm_oracle.c).  This header belongs to the oracle alone: the CUDA library
 * neither includes nor links anything declared here.
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_BC_PERIODIC = 0, ORC_BC_INFLOW = 1, ORC_BC_OUTFLOW = 2, ORC_BC_SYMMETRY = 3,
       ORC_BC_NOSLIP = 4, ORC_BC_DIRICHLET = 5 };

/* The problem as the paper states it (Secs. 2-4), in W0/tau0 units. */
typedef struct {
    int nx, ny;                    /* lattice nodes */
    double W0, tau0, dx, dt;       /* dx in W0 units, dt in tau0 units */
    double eps_s, lambda, k, Mc_inf;
    double D, alpha, nu, rho0;
    int n_sub, h_kind;
    double gbetaT, gbetaC, theta_ref, C_ref;
    double force[2];               /* constant body force */
    int bc[4];                     /* left, right, bottom, top */
    double u_in[2];
    double dir_phi, dir_U, dir_theta;
    int grad_mode;                 /* 0: nine-point stencil (reading R4), 1: local scheme of Sec. 3.1 */
    int isothermal;                /* 0: H = theta - h(phi)/2 (Eq. 21); 1: H = theta (Sec. 4.3, reading R22) */
} orc_params;

typedef struct orc_sim orc_sim;

orc_sim* orc_create(const orc_params* p);
void orc_destroy(orc_sim* s);
int orc_init_seeds(orc_sim* s, const double* seeds, int ns, double U0, double theta0);
int orc_init_seeds_window(orc_sim* s, const double* seeds, int ns, double U0, double theta0, int gx0, int gy0,
                          int gnx, int gny, int gpx, int gpy);
int orc_init_fields(orc_sim* s, const double* fields, const double* orient);
int orc_step(orc_sim* s, int nsteps);
int orc_step_flow(orc_sim* s, int nsteps);
int orc_force(orc_sim* s, double cx, double cy, double* out);
int orc_grad_phi(orc_sim* s, int mode, double* out);
long long orc_step_count(const orc_sim* s);
int orc_get_fields(orc_sim* s, double* out);
int orc_get_state(const orc_sim* s, double* out);
int orc_set_state(orc_sim* s, const double* in);
int orc_get_orient(const orc_sim* s, double* out);
int orc_metrics(orc_sim* s, double cx, double cy, double orient, double* out);
int orc_lattice_params(const orc_sim* s, double* out);

/* building blocks, exposed for the pins */
void orc_lattice_M5(double* M);
void orc_lattice_M9(double* M);
int orc_lambda5(double s0, double s1, double s2, double* L);
int orc_lambda9(const double* S, double* L);
void orc_feq_phi(double phi, double* out);
void orc_F_phi(double Q, double tau, double* out);
void orc_G_phi(double Nx, double Ny, double as2, double* out);
void orc_neq(double C, double qU, double Cux, double Cuy, double* out);
void orc_G_C(double dCux, double dCuy, double U, double gqx, double gqy, double Jx, double Jy, double D,
             double* out);
void orc_geq(double theta, double Lh, double Hux, double Huy, double* out);
void orc_G_theta(double dHux, double dHuy, double* out);
void orc_heq(double p, double ux, double uy, double rho0, double* out);
void orc_F_u(double Fx, double Fy, double* out);
void orc_anisotropy(double gx, double gy, double eps, double orient, double* as, double* Nx, double* Ny);

#ifdef __cplusplus
}
#endif
#endif
