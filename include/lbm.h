/*
 * lbm.h - C ABI of the GB300 (sm_103a) diffuse-interface MRT lattice
 * Boltzmann library for dendritic growth with thermosolutal convection.
 *
 * The library advances the coupled update of four distribution functions of
 * Zhan et al., "A diffuse-interface lattice Boltzmann method for the dendritic
 * growth with thermosolutal convection" (arXiv 2209.01444):
 *   - the anisotropic phase field phi       (D2Q5, Sec. 3.1, Eqs. 13-15),
 *   - the concentration C / supersaturation (D2Q5, Sec. 3.2, Eqs. 17-20),
 *   - the enthalpy H / temperature theta    (D2Q5, Sec. 3.3, Eqs. 21-23),
 *   - the melt flow                         (D2Q9 MRT, Sec. 3.4, Eqs. 24-26)
 *     with the order-parameter-weighted fluid-solid force and buoyancy,
 * with the relaxation rates, seed profile, non-equilibrium-extrapolation
 * boundaries and two-time-scaling of Sec. 4 and the matrices of Appendix B.
 *
 * Conventions shared by every call:
 *   - Every call returns LBM_OK (0) or a negative LBM_E* code and never
 *     throws; lbm_last_error() gives a human-readable reason.
 *   - The library owns all device memory of a handle (allocated in
 *     lbm_create, released in lbm_destroy).  The caller owns every host buffer
 *     and seed array passed in; the library copies what it needs and keeps no
 *     pointer to caller memory after a call returns.
 *   - Fields and states are row-major planes of ny rows by nx columns, node
 *     (x, y) at index y*nx + x, x along the first lattice axis.
 *   - Lengths and seed data are in lattice units (nodes); velocities,
 *     pressures and forces in the paper's W0/tau0 units.
 *   - Work is queued on the handle's CUDA stream (default: the legacy default
 *     stream).  Calls that return host data synchronise that stream.
 *   - Handles are not thread-safe; use one handle per host thread.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>

#if defined(__GNUC__)
#define LBM_API __attribute__((visibility("default")))
#else
#define LBM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ----------------------------------------------------------- status codes */
#define LBM_OK 0
#define LBM_EINVAL (-1)   /* bad argument or parameter set            */
#define LBM_ENOMEM (-2)   /* device or host allocation failed         */
#define LBM_ECUDA (-3)    /* a CUDA runtime call failed               */
#define LBM_ENUMERIC (-4) /* non-finite value found in the state      */
#define LBM_ETIMEOUT (-5) /* a bounded device wait ran out            */
#define LBM_ESTATE (-6)   /* call out of order (e.g. step before init) */

/* --------------------------------------------------------- enumerations */
/* Wall types (Sec. 4: non-equilibrium extrapolation on the walls).
 *   PERIODIC  : both opposite sides must be periodic.
 *   INFLOW    : flow u = u_in, p from the interior; scalars zero-gradient.
 *   OUTFLOW   : flow u from the interior, p = 0; scalars zero-gradient.
 *   SYMMETRY  : normal velocity 0, tangential from the interior; scalars
 *               zero-gradient.
 *   NOSLIP    : u = 0; scalars zero-gradient.
 *   DIRICHLET : u = 0; phi = dir_phi, U = dir_U, theta = dir_theta (the
 *               far-field condition of Sec. 4.4). */
enum { LBM_BC_PERIODIC = 0, LBM_BC_INFLOW = 1, LBM_BC_OUTFLOW = 2, LBM_BC_SYMMETRY = 3,
       LBM_BC_NOSLIP = 4, LBM_BC_DIRICHLET = 5 };

/* Population storage precision.  Collisions always run in FP32.  FP16/BF16
 * store equilibrium-shifted deviations d_i = s (f_i - f_i^ref) from the
 * equilibrium of a constant reference state (liquid at rest, phi = -1,
 * C = 1, theta = theta_ref, p = 0); the history fields stay FP32. */
enum { LBM_FP32 = 0, LBM_FP16 = 1, LBM_BF16 = 2 };
enum { LBM_GRAD_FD9 = 0, LBM_GRAD_LOCAL = 1 };
/* Field indices for lbm_get_fields (bit i of the mask selects field i). */
enum { LBM_FIELD_PHI = 0, LBM_FIELD_C = 1, LBM_FIELD_U = 2, LBM_FIELD_THETA = 3,
       LBM_FIELD_UX = 4, LBM_FIELD_UY = 5, LBM_FIELD_P = 6, LBM_NUM_FIELDS = 7 };

/* Number of planes in the FP64 state of lbm_get_state/lbm_set_state:
 * f_0..4 (phi), n_0..4 (C), g_0..4 (H), h_0..8 (flow), then the history
 * phi^{n-1}, Q^{n-1}, (Cu)^{n-1}_x, (Cu)^{n-1}_y, (Hu)^{n-1}_x, (Hu)^{n-1}_y. */
#define LBM_STATE_PLANES 30

/* --------------------------------------------------------------- problem */
/* The problem as the paper states it (Secs. 2-4).  All doubles are in the
 * paper's units (lengths in W0, times in tau0). */
typedef struct lbm_params {
    int nx, ny;            /* lattice nodes along x and y (each >= 4; ny <= 262140,
                              nx <= 2^30)                                       */
    double W0, tau0;       /* interface width and kinetic time, Eq. (1)          */
    double dx, dt;         /* lattice spacing (W0 units) and coupled time step   */
    double eps_s;          /* anisotropy strength, Eq. (2), 0 <= eps_s < 1/3     */
    double lambda;         /* coupling constant, Eq. (5)                         */
    double k;              /* partition coefficient, Eq. (4a), 0 < k < 1         */
    double Mc_inf;         /* M c_inf, Eq. (5)                                   */
    double D, alpha, nu;   /* solute / thermal diffusivity, viscosity (> 0)      */
    double rho0;           /* reference density of Eq. (25)                      */
    int n_sub;             /* flow sub-steps per coupled step (Sec. 4; >= 1)     */
    int h_kind;            /* 0: h = phi, 1: 15/8 (phi - 2phi^3/3 + phi^5/5)     */
    double gbetaT, gbetaC; /* Boussinesq buoyancy along +y per unit theta and C  */
    double theta_ref, C_ref; /* buoyancy reference values; theta_ref also sets the
                                FP16/BF16 reference state                        */
    double force[2];       /* constant body force                                */
    int bc[4];             /* wall types: left, right, bottom, top               */
    double u_in[2];        /* inflow velocity                                    */
    double dir_phi, dir_U, dir_theta; /* Dirichlet far-field values             */
    int storage;           /* LBM_FP32, LBM_FP16 or LBM_BF16                     */
    int grad_mode;         /* LBM_GRAD_FD9 (nine-point stencil) or LBM_GRAD_LOCAL
                              (the local scheme of Sec. 3.1: grad(phi) from the
                              node's own first moment, solved by two
                              fixed-point passes from a_s = 1, N = 0)      */
    int isothermal;        /* 0: enthalpy H = theta - h(phi)/2 (Eq. 21, latent
                              heat released at the interface); 1: H = theta,
                              no latent heat, the isothermal alloy of Sec. 4.3:
                              a start at uniform theta0 = 0 keeps theta = 0
                              exactly; a uniform theta0 != 0 stays uniform up
                              to the flow's O(Ma^2) divergence                */
} lbm_params;

/* A seed (Sec. 4): centre and radius in lattice units, crystal-axis
 * orientation in radians.  phi = max over seeds of tanh[(R - d)/(sqrt2 W0)]
 * with d the minimum-image distance on periodic axes; each node belongs to
 * the grain of its nearest seed centre (ties to the lower index). */
typedef struct lbm_seed {
    double x, y, R, orient;
} lbm_seed;

/* Reductions of lbm_get_metrics, on the device: each thread sums the
 * deviations of 16 nodes from the reference state in FP32 and adds the
 * reference terms in FP64; threads and blocks combine in FP64, in a fixed
 * order (the same result on every call). */
typedef struct lbm_metrics {
    double tip[3];         /* tip distance (lattice units) from the given centre
                              along the grain's +x, -x and +y axes: phi sampled
                              bilinearly every half node, outermost sample with
                              phi > 0 interpolated to phi = 0; NaN if none     */
    double solid_fraction; /* sum((1 + phi)/2) / (nx ny)                       */
    double sum_C;          /* sum over nodes of C = sum_i n_i                  */
    double sum_H;          /* sum over nodes of H = sum_i g_i                  */
    double sum_h;          /* sum over nodes and directions of h_i             */
    double max_u;          /* max |u| in paper units                           */
    double nonfinite;      /* 1 if any node holds a NaN/Inf macro, else 0      */
    double sum_phi;        /* sum over nodes of phi                            */
    long long step;        /* coupled steps taken since initialisation         */
} lbm_metrics;

typedef struct lbm_handle lbm_handle;

/* ------------------------------------------------------------- life cycle */
/* Fill *p with the thermosolutal parameter set of Sec. 4.4 on an nx x ny
 * periodic box (W0 = tau0 = 1, dx = 1, dt = 0.05, eps_s = 0.05, alpha = D = 2,
 * k = 0.15, Mc_inf = 0.5325, lambda = 3.1913, nu = 2, rho0 = 1, FP32). */
LBM_API int lbm_params_default(lbm_params* p, int nx, int ny);

/* Validate *p, derive the lattice-unit parameters and relaxation rates of
 * Sec. 4, and allocate the device state (double-buffered populations, history,
 * grain map).  On success *out receives a new handle.  LBM_EINVAL, with the
 * reason in lbm_last_error(NULL) and nothing allocated, for a value outside
 * the ranges stated in lbm_params or a real parameter that is NaN or
 * infinite; LBM_ENOMEM when the device memory does not suffice. */
LBM_API int lbm_create(const lbm_params* p, lbm_handle** out);

/* Release every resource of h (NULL is a no-op). */
LBM_API void lbm_destroy(lbm_handle* h);

/* Queue all later work of h on `stream` (a cudaStream_t, e.g. the handle of
 * torch.cuda.current_stream(); NULL selects the legacy default stream). */
LBM_API int lbm_set_stream(lbm_handle* h, void* stream);

/* --------------------------------------------------------- initial state */
/* Seeded start (Sec. 4): phi from the seeds, U = U0, theta = theta0, u = 0,
 * p = 0, populations at equilibrium, history = the time-0 macros.  At most 256
 * seeds. */
LBM_API int lbm_init_seeds(lbm_handle* h, const lbm_seed* seeds, int n_seeds, double U0, double theta0);

/* Start from given macroscopic fields: `fields` holds 6 planes (phi, U,
 * theta, u_x, u_y, p), velocities and pressure in paper units; `orient` is
 * one plane of grain orientations in radians (NULL: 0 everywhere, at most 256
 * distinct values).  Populations at equilibrium, history = time-0 macros. */
LBM_API int lbm_init_fields(lbm_handle* h, const double* fields, const double* orient);

/* ------------------------------------------------------------------ steps */
/* Queue `nsteps` coupled time steps (the fused stream-collide kernel of all
 * four models, then the wall kernels, then n_sub - 1 flow-only sub-steps) on
 * the handle's stream and return without waiting.  Long runs are replayed
 * from captured 16-step CUDA graphs; inside one (n_sub = 1) the
 * left/right walls of a step are updated by the next step as it loads them,
 * and the last step of the graph runs the wall kernels in full, so the state
 * seen between calls is always complete.  The graph is captured,
 * instantiated and uploaded when a state is set (lbm_init_seeds,
 * lbm_init_fields, lbm_load_state), so the first lbm_step pays none of it. */
LBM_API int lbm_step(lbm_handle* h, int nsteps);

/* Wait for all queued work of h; reports an asynchronous CUDA error. */
LBM_API int lbm_synchronize(lbm_handle* h);

/* Size limit, in bytes, of the device buffer that whole-grid transfers
 * (lbm_init_seeds, lbm_init_fields, lbm_get_fields, lbm_get_state,
 * lbm_get_state_region, lbm_set_state) work through, one band of rows at a
 * time (default 64 MiB; at least one row of the widest transfer, 120 bytes per
 * node, is always used).  The buffer is allocated on the first such call, so
 * a handle holds only its state (about 217 bytes per node in FP32, 133 in
 * FP16/BF16, plus O(nx + ny) tables) and the grid can fill most of the
 * device.  Results do not depend on the band size. */
LBM_API int lbm_set_io_chunk(lbm_handle* h, size_t bytes);

/* Number of coupled steps taken since the last initialisation. */
LBM_API long long lbm_step_count(const lbm_handle* h);

/* ---------------------------------------------------------------- output */
/* Write the fields selected by `mask` (bit LBM_FIELD_*) into `out`, in
 * increasing field order, nx*ny doubles each: phi, C, U (Eq. 20), theta
 * (Eq. 23), u_x, u_y (corrected velocity of Eq. 26, paper units), p (Eq. 26,
 * paper units).  Only the selected planes are copied to the host (as FP32,
 * band by band through a pinned staging buffer of at most 64 MiB that the
 * process's handles share, allocated on the first call and kept until exit),
 * and converted there on up to 16 host threads while the next band is
 * copied.  Synchronous. */
LBM_API int lbm_get_fields(lbm_handle* h, unsigned mask, double* out);

/* The same fields in FP32, the precision the device computes them in: `out`
 * receives nx*ny floats per selected field, in increasing field order (the
 * macros of Eqs. 15, 20, 23 and 26 as for lbm_get_fields, each rounded once
 * to FP32 from deviation * scale + offset).  The fields are formed on the
 * device band by band.  Page-locked `out` (cudaHostAlloc, cudaHostRegister)
 * receives each band's planes straight from the device, at the host link's
 * rate, and no host thread touches the values; pageable `out` receives them
 * through the pinned staging buffer lbm_get_fields uses, copied on up to 16
 * host threads while the next band crosses.  Synchronous; the caller owns
 * `out`.  LBM_EINVAL for a NULL out or an unknown mask bit, LBM_ENOMEM when
 * the staging buffer cannot be allocated. */
LBM_API int lbm_get_fields_f32(lbm_handle* h, unsigned mask, float* out);

/* FP64 copy of the decoded state: LBM_STATE_PLANES planes of nx*ny
 * (populations in lattice units, history as stored).  Synchronous. */
LBM_API int lbm_get_state(lbm_handle* h, double* out);

/* FP64 copy of the decoded state restricted to the w x hgt window with
 * lower-left node (x0, y0): LBM_STATE_PLANES planes of w*hgt, row-major.
 * The window must lie inside the grid.  Synchronous. */
LBM_API int lbm_get_state_region(lbm_handle* h, int x0, int y0, int w, int hgt, double* out);

/* Overwrite the state from LBM_STATE_PLANES FP64 planes (rounded to the
 * storage precision).  The grain map and step counter are kept. */
LBM_API int lbm_set_state(lbm_handle* h, const double* in);

/* Flow-only steps: the flow model alone (collision, streaming, flow walls)
 * with phi, C and theta frozen at their current values, as in the stationary-
 * cylinder problem of Sec. 4.1.  The coupled-step count does not change.
 * Queued on the handle's stream; the flow populations alternate buffers as in
 * lbm_step. */
LBM_API int lbm_step_flow(lbm_handle* h, int nsteps);
/* Hydrodynamic force and torque on the solid, Eq. (27): out[0..1] = F_f =
 * -sum (1 - q~) f, out[2] = T_f = -sum (x - (cx, cy)) x (1 - q~) f, summed in
 * FP64 over all nodes in flow lattice units, with f = (u_s - u*)/dt, u_s = 0
 * and the diffuse-interface weight 1 - q~ = (1 + phi)/2 of Eq. (24).
 * Synchronous. */
LBM_API int lbm_get_force(lbm_handle* h, double cx, double cy, double* out);

/* Periodic reductions (the paper measures tip velocities from tip positions
 * over time): with every > 0, lbm_step stops at every multiple of `every`
 * steps and queues the lbm_metrics reduction (tips from cx, cy along the
 * orientation `orient`) into a device ring of `capacity` records, without
 * host synchronisation; every = 0 turns it off.  Enabling frees the previous
 * ring, synchronises, and records the current state if its step count is a
 * multiple of `every`.
 * lbm_get_monitor copies the newest min(max, recorded, capacity) records,
 * oldest first, into out[] and, if v_tip is not NULL, the tip velocities
 * v_tip[3 i + a] = (tip_a(record i) - tip_a(record before)) dx / elapsed time,
 * in W0/tau0 (NaN where the earlier record is gone); synchronous. */
LBM_API int lbm_set_monitor(lbm_handle* h, int every, int capacity, double cx, double cy, double orient);
LBM_API int lbm_get_monitor(lbm_handle* h, lbm_metrics* out, double* v_tip, int max, int* count);

/* Reductions at the current step (see lbm_metrics) with tips measured from
 * (cx, cy) along the axes of a grain of orientation `orient`.  Synchronous;
 * returns LBM_ENUMERIC (with *m filled) when a non-finite value is found. */
LBM_API int lbm_get_metrics(lbm_handle* h, double cx, double cy, double orient, lbm_metrics* m);

/* ------------------------------------------------------------- checkpoint */
/* Size in bytes of a checkpoint of h (raw storage-precision populations,
 * history, grain map and orientation table, step counter, parameters). */
LBM_API size_t lbm_checkpoint_bytes(const lbm_handle* h);

/* Write a checkpoint into `host` (`bytes` >= lbm_checkpoint_bytes).  Synchronous. */
LBM_API int lbm_save_state(lbm_handle* h, void* host, size_t bytes);

/* Restore a checkpoint written by a handle with identical parameters;
 * resuming is bit-exact.  LBM_EINVAL if the size or parameters differ. */
LBM_API int lbm_load_state(lbm_handle* h, const void* host, size_t bytes);

/* ------------------------------------------------------------------ batch */
/* Many independent domains advanced together: each has its own size and
 * parameters (one storage type for all, n_sub = 1).  One persistent kernel
 * per coupled step sweeps the tiles of every domain, batched wall kernels
 * follow, and lbm_batch_step replays 16-step sequences from captured CUDA
 * graphs.  The tile height (4, 8 or 16 rows of 32 nodes) is chosen by
 * lbm_batch_tune.  Domains are indexed 0..n-1; per-domain results use the
 * single-domain conventions above. */
typedef struct lbm_batch lbm_batch;

/* Create n domains (1 <= n <= 256) from params[0..n-1] (validated as
 * lbm_create does).  Batches stepped concurrently on different streams of one
 * device share the constant-memory copy of the domain table and must not
 * overlap. */
LBM_API int lbm_batch_create(const lbm_params* params, int n, lbm_batch** out);
LBM_API void lbm_batch_destroy(lbm_batch* b);
LBM_API int lbm_batch_set_stream(lbm_batch* b, void* stream);
/* Seeded start of one domain (lbm_init_seeds semantics). */
LBM_API int lbm_batch_init_seeds(lbm_batch* b, int dom, const lbm_seed* seeds, int n_seeds, double U0,
                                 double theta0);
/* Queue nsteps coupled steps of every domain; all must be initialised. */
LBM_API int lbm_batch_step(lbm_batch* b, int nsteps);
LBM_API int lbm_batch_synchronize(lbm_batch* b);
LBM_API int lbm_batch_get_fields(lbm_batch* b, int dom, unsigned mask, double* out);
LBM_API int lbm_batch_get_metrics(lbm_batch* b, int dom, double cx, double cy, double orient, lbm_metrics* m);
/* Total nodes of all domains; current tiling (tile height, tiles per CTA). */
LBM_API long long lbm_batch_nodes(const lbm_batch* b);
LBM_API int lbm_batch_tile_height(const lbm_batch* b);
LBM_API int lbm_batch_tiles_per_cta(const lbm_batch* b);
/* Force the tiling instead of tuning it: tile height 4, 8 or 16 rows of 32
 * nodes; tiles per CTA >= 1, or 0 for a persistent grid of as many CTAs as fit
 * on the GPU at once, each taking one contiguous run of tiles.  Default (8, 1). */
LBM_API int lbm_batch_set_tiling(lbm_batch* b, int tile_height, int tiles_per_cta);
/* Autotuner: pick the fastest tiling for this batch on this GPU among tile
 * heights {4, 8, 16} x tiles per CTA {1, 4, persistent}.  A cache file (one
 * "key height tiles_per_cta" line per GPU name, storage, size class and domain
 * count; NULL for none) is read first and appended to after a measurement.
 * Measuring times 12 steps per tiling on a device copy of the current state,
 * which is restored afterwards (needs that much free memory); the step counter
 * does not move. */
LBM_API int lbm_batch_tune(lbm_batch* b, const char* cache_path, int* tile_height);
/* Kernel timing of the batched step, as lbm_set_profiling does for a handle:
 * while enabled, lbm_batch_step launches every step directly (no graph) and
 * brackets the batched fused kernel with CUDA events on the batch's stream;
 * lbm_batch_kernel_time returns the total device time (ms) of the kernels
 * timed since profiling was enabled, and their number (synchronises the
 * pending events).  Enabling or disabling resets the accumulated time. */
LBM_API int lbm_batch_set_profiling(lbm_batch* b, int enable);
LBM_API int lbm_batch_kernel_time(lbm_batch* b, double* total_ms, long long* launches);
LBM_API const char* lbm_batch_last_error(const lbm_batch* b);

/* ------------------------------------------------------- surrogate network */
/* Building blocks of the learned surrogate (a convolutional network that
 * advances the fields K steps at a time; the paper has no counterpart).  All
 * tensors are device memory owned by the caller; work is queued on `stream`.
 *
 * Tensor-core GEMM: D[M][N] = act(A[M][K] B[N][K]^T + bias[N]) with A and B
 * BF16, row-major with K contiguous and row pitches lda, ldb (multiples of 8
 * elements, >= K, 16-byte aligned bases); FP32 accumulation; D BF16
 * (out_fp32 = 0) or FP32 with pitch ldd; bias FP32[N] or NULL; relu != 0
 * clamps at zero.  N must be a multiple of 8.  Runs on
 * tcgen05 (sm_103a).  LBM_EINVAL for unsupported shapes or alignment. */
LBM_API int lbm_nn_gemm(const void* A, int lda, const void* B, int ldb, void* D, int ldd, const float* bias, int M,
                        int N, int K, int out_fp32, int relu, void* stream);

/* lbm_nn_gemm with K split into `splits` slices computed by separate CTAs
 * (for long reductions such as weight gradients over every pixel); their FP32
 * partial tiles go to `workspace` (splits * M * N floats) and a reduction adds
 * them, the bias and the activation. */
LBM_API int lbm_nn_gemm_split(const void* A, int lda, const void* B, int ldb, void* D, int ldd, const float* bias,
                              int M, int N, int K, int out_fp32, int relu, int splits, float* workspace,
                              void* stream);

/* Implicit 3 x 3 convolution with zero padding (no gathered copy: the tensor
 * cores read shifted tiles of X through 4-D TMA loads): D[p][n] =
 * act(sum_{tap, c < C} X[p shifted by tap][c] * Wm[n][tap*C + c] + bias[n]),
 * X NHWC BF16 [B][H][W][cpitch], Wm BF16 [N][ldw] (ldw >= 9C, tap = ky*3+kx),
 * D [B*H*W][ldd] BF16 or FP32.  C a multiple of 32; a 128-pixel tile must be
 * whole rows of whole images (W a multiple of 128, or W and H dividing 128
 * appropriately): LBM_EINVAL otherwise. */
LBM_API int lbm_nn_conv3x3(const void* X, int B, int H, int W, int C, int cpitch, const void* Wm, int ldw, void* D,
                           int ldd, const float* bias, int N, int out_fp32, int relu, void* stream);
/* 2 x 2 stride-2 up-convolution stored straight into a concatenation buffer:
 * Y[b][2y+dy][2x+dx][c0+co] = bias[k] + sum_i X[(b,y,x)][i] Wm[k][i] with
 * k = (dy*2+dx)*c + co; X [B*Hl*Wl][lda], Wm [4c][ldw] BF16, Y BF16 pitch
 * ypitch; c a multiple of 16. */
LBM_API int lbm_nn_upconv2x2(const void* X, int lda, const void* Wm, int ldw, void* Y, int ypitch, int c0,
                             const float* bias, int B, int Hl, int Wl, int cin, int c, void* stream);

/* Layers around the GEMM.  Activations are NHWC: [B][H][W][channels] with a
 * channel pitch (the row length of one pixel), BF16 unless named FP32.
 * im2col3x3: A[(b,y,x)][(ky,kx,c)] = X[b, y+ky-1, x+kx-1, c], zero outside
 *   the image (C and cpitch multiples of 8; A has 9C columns).
 * col2im3x3: FP32 dX[b,y,x,c] = sum over taps of dA[(b,y-ky+1,x-kx+1)][(ky,kx,c)].
 * relu_bwd: g[r][c] = 0 where y[r][c] <= 0 (g FP32 or BF16).
 * transpose: out[c][r] = in[r][c] (BF16).
 * maxpool_fwd / _bwd: 2 x 2 max pooling; the backward adds the FP32 gradient
 *   to the first maximum of each window.
 * shuffle_fwd / _bwd: the 2 x 2 stride-2 up-convolution's GEMM output
 *   U[(b,y,x)][(dy,dx,c)] <-> Y[b, 2y+dy, 2x+dx, c0+c].
 * proj_fwd: FP32 Y[p][o] = R[p][o] + b[o] + sum_c X[p][c] Wt[o][c] (O <= 8
 *   outputs, R the residual or NULL); proj_bwd: FP32 dX (skipped when NULL),
 *   dW (O x C) and db (O) from per-block partials `part` (part_blocks * O *
 *   (C + 1) floats).
 * flip3x3: weights of the gradient-to-input convolution, Wf[ci][t*cout+co] =
 *   W[co][(8-t)*cin+ci] (BF16; W is [cout][9*cin]).
 * colsum: out[c] = sum_r g[r][c] through `part` (part_blocks * C floats).
 * mse: loss[0] = sum (pred - target)^2, grad = 2 (pred - target)/n; `part`
 *   holds n/256 + 1 floats.
 * adam: one Adam step (bias-corrected, step t >= 1) on FP32 weights; writes
 *   their BF16 copy when w_bf16 is not NULL.
 * pack: FP32 fields [P][F] -> BF16 [P][cpitch], (x - mean)/std, zero padded;
 *   R (FP32 [P][F], or NULL) receives the normalised fields unrounded.
 * unpack: FP32 fields [P][F] = mean + std * Y.
 * cast_bf16: FP32 [rows][C] (pitch apitch) -> BF16 (pitch bpitch). */
LBM_API int lbm_nn_im2col3x3(const void* X, int B, int H, int W, int C, int cpitch, void* A, void* stream);
LBM_API int lbm_nn_col2im3x3(const float* dA, int B, int H, int W, int C, float* dX, int cpitch, void* stream);
LBM_API int lbm_nn_relu_bwd(void* g, int g_fp32, int gpitch, const void* y, int ypitch, long long rows, int C,
                            void* stream);
LBM_API int lbm_nn_transpose(const void* in, int rows, int cols, int ipitch, void* out, int opitch, void* stream);
LBM_API int lbm_nn_maxpool_fwd(const void* X, int B, int H, int W, int C, int xpitch, void* Y, void* stream);
LBM_API int lbm_nn_maxpool_bwd(const void* X, int B, int H, int W, int C, int xpitch, const float* dY, float* dX,
                               int dpitch, void* stream);
LBM_API int lbm_nn_shuffle_fwd(const void* U, int B, int H, int W, int C, void* Y, int ypitch, int c0, void* stream);
LBM_API int lbm_nn_shuffle_bwd(const void* dY, int dy_fp32, int ypitch, int c0, int B, int H, int W, int C, void* dU,
                               void* stream);
LBM_API int lbm_nn_proj_fwd(const void* X, int P, int C, int xpitch, const float* Wt, const float* bias, int O,
                            const float* R, float* Y, void* stream);
LBM_API int lbm_nn_proj_bwd(const float* dY, const void* X, int P, int C, int xpitch, const float* Wt, int O,
                            float* dX, int dpitch, float* dW, float* db, float* part, int part_blocks,
                            void* stream);
LBM_API int lbm_nn_flip3x3(const void* W, int cout, int cin, void* Wf, void* stream);
/* Transposed gather for weight gradients: AT[t*C + c][p] = X[pixel p shifted
 * by tap t][c] (zero outside the image) for taps = 9 (t = ky*3 + kx); for
 * taps = 3 the middle row of those taps only, AT[kx*C + c][p] = X[p shifted by
 * (dy, dx) = (0, kx - 1)][c]; AT[c][p] = X[p][c] for taps = 1; BF16, row pitch
 * atpitch; C, cpitch, atpitch and B*H*W multiples of 8. */
LBM_API int lbm_nn_gather_t(const void* X, int B, int H, int W, int C, int cpitch, int taps, void* AT,
                            long long atpitch, void* stream);
/* Weight gradient of a 3 x 3 zero-padded convolution from three copies of its
 * input: D[n][t*C + c] = sum_p X[p shifted by tap t][c] dY[p][n] (t = ky*3 +
 * kx), FP32 with row pitch ldd >= 9C, from XT3 = lbm_nn_gather_t(X, taps = 3)
 * (BF16 [3C][B*H*W], pitch B*H*W) and dYT = dY transposed (BF16 [cout][B*H*W],
 * pitch B*H*W).  The vertical shifts are taken by the tensor-core GEMM's TMA
 * coordinates, zero filled outside the image.  K = B*H*W is split into
 * `splits` slices whose partial sums go to `workspace` (splits * 9C * cout
 * floats).  W and C multiples of 32, cout a multiple of 8: LBM_EINVAL
 * otherwise. */
LBM_API int lbm_nn_wgrad3x3(const void* XT3, const void* dYT, int B, int H, int W, int C, int cout, float* D,
                            int ldd, int splits, float* workspace, void* stream);
LBM_API int lbm_nn_colsum(const void* g, int g_fp32, long long rows, int C, int pitch, float* out, float* part,
                          int part_blocks, void* stream);
LBM_API int lbm_nn_mse(const float* pred, const float* target, long long n, float* grad, float* loss, float* part,
                       void* stream);
LBM_API int lbm_nn_adam(float* w, const float* g, float* m, float* v, long long n, float lr, float b1, float b2,
                        float eps, int t, void* w_bf16, void* stream);
LBM_API int lbm_nn_pack(const float* fields, long long P, int F, const float* mean, const float* inv_std, void* X,
                        int cpitch, float* R, void* stream);
LBM_API int lbm_nn_unpack(const float* Y, long long P, int F, const float* mean, const float* inv_std, float* fields,
                          void* stream);
LBM_API int lbm_nn_cast_bf16(const float* a, long long rows, int C, int apitch, void* b, int bpitch, void* stream);

/* The surrogate network as one object (the paper has no counterpart): a
 * convolutional U-Net with `levels` levels of widths base * 2^l (3 x 3
 * convolutions, two per level and side, ReLU, 2 x 2 max pooling, 2 x 2
 * stride-2 up-convolutions, skip concatenation) and a 1 x 1 output projection
 * added to the input fields (residual), run on tensor cores in BF16 with FP32
 * accumulation.  It is sized at creation for `batch` images of
 * height x width pixels with `fields` <= 8 fields per pixel; height and width
 * must be multiples of 2^(levels-1) and batch*height*width/4^(levels-1) a
 * multiple of 8.  The object owns every device buffer it uses.
 *
 * Parameters are one FP32 vector (lbm_unet_param_count values): the tensors
 * in the order enc{l}a.W, enc{l}a.b, enc{l}b.W, enc{l}b.b for l = 0 ..
 * levels-1, then up{l}.W, up{l}.b, dec{l}a.W, dec{l}a.b, dec{l}b.W, dec{l}b.b
 * for l = levels-2 .. 0, then out.W, out.b, each row-major: conv weight
 * [cout][9*cin] with column (ky*3+kx)*cin+ci (enc0a has cin = 8, the padded
 * field count), bias [cout]; up-convolution weight [4c][2c] with row
 * (dy*2+dx)*c+co and bias [4c]; out.W [fields][base], out.b [fields].
 *
 * Fields x, targets and predictions are FP32 device arrays [batch][height]
 * [width][fields].  The network reads the inputs as (x - mean)/std_in and its
 * output is the increment in units of std_out: the prediction is
 * y = x + std_out * out (lbm_unet_set_norm; default mean 0, both scales 1);
 * the loss is the mean squared error of out against (target - x)/std_out
 * (weighted at the interface with lbm_unet_set_loss_weight).  All calls queue work on the object's stream and
 * return without waiting, except set_params, get_params, get_grads, set_norm
 * and loss, which synchronise.  Errors: LBM_EINVAL for bad arguments,
 * LBM_ENOMEM / LBM_ECUDA from CUDA; lbm_unet_last_error gives the reason. */
typedef struct lbm_unet lbm_unet;
LBM_API int lbm_unet_create(int levels, int base, int fields, int batch, int height, int width, lbm_unet** out);
LBM_API void lbm_unet_destroy(lbm_unet* u);
LBM_API int lbm_unet_set_stream(lbm_unet* u, void* stream);
LBM_API long long lbm_unet_param_count(const lbm_unet* u);
LBM_API long long lbm_unet_device_bytes(const lbm_unet* u);
/* Loads parameters (host, FP32) and resets the Adam moments and step. */
LBM_API int lbm_unet_set_params(lbm_unet* u, const float* host);
LBM_API int lbm_unet_get_params(lbm_unet* u, float* host);
/* Gradients of the loss from the last lbm_unet_backward / train_step. */
LBM_API int lbm_unet_get_grads(lbm_unet* u, float* host);
LBM_API int lbm_unet_set_norm(lbm_unet* u, const float* mean, const float* std_in, const float* std_out);
/* Interface weight of the training loss (not in the paper, which has no
 * network): each pixel's squared errors are weighted by 1 + alpha max(0, 1 - phi^2),
 * phi the phase field of the input x (field 0, physical units), so that the
 * pixels where the interface moves, a few per cent of a field, weigh in the
 * loss as the far field does; the loss is sum w d^2 / n.  alpha >= 0; 0 (the
 * default) is the plain mean squared error. */
LBM_API int lbm_unet_set_loss_weight(lbm_unet* u, float alpha);
/* Writes the FP32 parameters and the normalisation to a file (magic
 * "LBMUNET1", int32 levels, base, fields, 0, int64 parameter count, FP32 mean,
 * std_in, std_out and parameters, little-endian); synchronous.  The Adam
 * moments are not saved. */
LBM_API int lbm_unet_save(lbm_unet* u, const char* path);
/* Reads such a file into u, whose levels, base and fields must match (batch,
 * height and width may differ: train on patches, infer on whole fields);
 * LBM_EINVAL with the reason in lbm_unet_last_error for a missing, truncated,
 * mismatched or non-finite file.  Resets the Adam moments. */
LBM_API int lbm_unet_load(lbm_unet* u, const char* path);
/* Prediction y (physical units, may be NULL) for the fields x. */
LBM_API int lbm_unet_forward(lbm_unet* u, const float* x, float* y);
/* Forward, loss against `target` and the gradients of every parameter. */
LBM_API int lbm_unet_backward(lbm_unet* u, const float* x, const float* target);
/* One Adam step (bias-corrected) on the current gradients; refreshes the BF16
 * weights the kernels read. */
LBM_API int lbm_unet_adam(lbm_unet* u, float lr, float beta1, float beta2, float eps);
/* backward + adam(lr, 0.9, 0.999, 1e-8). */
LBM_API int lbm_unet_train_step(lbm_unet* u, const float* x, const float* target, float lr);
/* Mean squared error of the last backward (output units). */
LBM_API int lbm_unet_loss(lbm_unet* u, double* out);
/* Copies the last network output (the increment in units of std_out). */
LBM_API int lbm_unet_output(lbm_unet* u, float* y_norm);
LBM_API const char* lbm_unet_last_error(const lbm_unet* u);
LBM_API int lbm_unet_shape(const lbm_unet* u, int* batch, int* height, int* width, int* fields);

/* ------------------------------------------- device-side field exchange */
/* Device snapshots of a handle's state (populations, history, step count) in
 * library-owned memory, slot 0 or 1 (allocated on first use; queued on the
 * handle's stream).  lbm_surrogate_advance with audit != 0 overwrites slot 1.
 * Restoring an empty slot gives LBM_ESTATE. */
LBM_API int lbm_snapshot_save(lbm_handle* h, int slot);
LBM_API int lbm_snapshot_restore(lbm_handle* h, int slot);

/* The fields of every node as one FP32 device array [ny][nx][5], per node
 * phi, C, theta, u_x, u_y (the paper's units), for the surrogate network;
 * and the reverse: every node's populations replaced by the equilibrium of
 * the given fields (phi clamped to [-1, 1], U recovered from C and phi, the
 * node's pressure kept; the stored flow momentum chosen so that the recovered
 * velocity, with the forcing and the fluid-solid force, is the given one).
 * With prev (the fields K steps earlier, same layout) the history is set one
 * step back on the line between prev and src; with prev NULL it equals the
 * new macros.  Both queue on the handle's stream. */
LBM_API int lbm_fields_nhwc(lbm_handle* h, float* dst);
LBM_API int lbm_set_fields_nhwc(lbm_handle* h, const float* src, const float* prev, int K);
LBM_API int lbm_batch_fields_nhwc(lbm_batch* b, int dom, float* dst);

/* One surrogate window of K steps (the paper has no counterpart).  The network
 * (sized for one ny x nx image of 5 fields, run on the handle's stream)
 * predicts the fields K steps ahead.  audit == 0: if every predicted value is
 * finite, the state becomes the equilibrium of the prediction, the step count
 * advances by K and accepted = 1; otherwise nothing changes, accepted = 0 and
 * tip_err = infinity (the caller runs the window with the plain LB).  audit !=
 * 0: the plain LB also runs the window from the same state and its result is
 * kept; the report compares the two: the largest tip difference over the
 * three rays of lbm_metrics (origin cx, cy, orientation `orient`), the nodes
 * whose phi sign differs and the largest |phi| difference; accepted = tip
 * error <= tip_tol (a non-finite prediction is never accepted).
 * Synchronises. */
typedef struct lbm_surrogate_report {
    int audited, accepted;
    double tip_err;     /* lattice units */
    double tip[3];      /* tips of the LB result (audited windows) */
    long long mismatch; /* nodes where the sign of phi differs */
    double max_dphi;
} lbm_surrogate_report;
LBM_API int lbm_surrogate_advance(lbm_handle* h, lbm_unet* net, int K, double tip_tol, int audit, double cx,
                                  double cy, double orient, lbm_surrogate_report* rep);

/* LBM_ETIMEOUT if a network kernel gave up a bounded wait since the flag was
 * last cleared (clear != 0 clears it), else LBM_OK.  Synchronous. */
LBM_API int lbm_nn_error(int clear);

/* Bound, in nanoseconds, on how long the GEMMs' tensor-core issuer waits for
 * the TMA copies of each k block's operand tiles (default 1e9, one second;
 * for the current device, from the next launch on).  Every other wait of the
 * GEMMs keeps its one-second bound.  When a wait runs out the GEMM raises the
 * flag that lbm_nn_error reports (LBM_ETIMEOUT), leaves its output unwritten,
 * waits (bounded) for every copy and MMA it already issued, frees its tensor
 * memory and returns.  0 makes the first such wait give up at once, which
 * exercises that path without a fault.  Synchronous. */
LBM_API int lbm_nn_set_operand_wait(unsigned long long ns);

/* ------------------------------------------------ allocation-free reduction */
/* The reductions of lbm_get_metrics, computed straight from population
 * buffers the caller owns, without allocating anything.  The paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc, such as a process whose device memory is owned by another
 * allocator (a framework's caching pool that must see every allocation) or a
 * long-running loop that may only allocate at start-up.  Those callers still
 * need the per-block scratch of the reduction; here it lives in one static
 * device array of 448 KiB (8192 blocks x 7 partials) that every GPU loading
 * the library holds until the process exits.
 *
 * Inputs (device memory, read only): the scalar and flow population buffers of
 * a state for the problem *p, in the layout the library keeps (the two buffers
 * that lbm_save_state writes right after its header).  Each buffer holds the
 * deviations of its populations from the reference equilibrium for
 * pitch*ny nodes, pitch = nx rounded up to a multiple of 32, in blocks of 32
 * nodes: node (x, y) is lane (y*pitch + x) % 32 of block (y*pitch + x) / 32,
 * and a block stores each of its planes as 32 consecutive values, plane after
 * plane.  A scalar block has the 15 FP32 planes f_0..4, n_0..4, g_0..4
 * (LBM_FP32; 1920 bytes), or (LBM_FP16/LBM_BF16; 1152 bytes) the planes
 * f_1..4 in 16 bits, then four planes of 32-bit words holding (n_i, g_i) for
 * i = 1..4 (n_i in the low half), then the FP32 rest planes f_0, n_0, g_0; a
 * flow block has the 9 planes h_0..8 of the storage type.  Output: `out`, 10 doubles in device memory: sum (1 + phi)/2,
 * sum C, sum H, sum of all h_i, max |u| in flow lattice units, number of nodes
 * with a non-finite macro, sum phi, and the three tip distances of
 * lbm_metrics.tip.  The work is queued on `stream` (a cudaStream_t, NULL for the
 * legacy default stream) and the call returns without waiting.
 *
 * Limits and sharing: grids larger than 33,554,432 nodes are rejected with
 * LBM_EINVAL.  A call made outside stream capture looks up the device
 * address of the static array (cudaGetSymbolAddress, with the device current)
 * and keeps it for that device and CUDA context (a device reset ends the
 * context; the next call outside capture looks the address up again).  A call
 * made while `stream` is being captured, with no address kept for the current
 * context, is refused with LBM_EINVAL: make the first call on a device before
 * any stream capture.  Every call shares the one array and leaves
 * its partial sums in it (each call overwrites every row it reads, so nothing
 * needs clearing), so calls whose kernels overlap on the GPU, for example on two
 * streams at once, race.  Errors: LBM_EINVAL for bad arguments or parameters,
 * LBM_ECUDA for a failed CUDA call; lbm_last_error(NULL) gives the reason. */
LBM_API int lbm_reduce_noalloc(const lbm_params* p, const void* scalar_pops, const void* flow_pops, double cx,
                               double cy, double orient, double* out, void* stream);

/* ------------------------------------------------------------ diagnostics */
/* Kernel timing for roofline measurements: while enabled, lbm_step launches
 * every coupled step directly (no graph) and brackets kernels with CUDA events
 * on the handle's stream.  enable = 1: the fused stream-collide kernel of each
 * coupled step; enable = 2: the n_sub - 1 flow sub-step kernels of each
 * coupled step (two-time-scaling, Sec. 4; LBM_EINVAL when n_sub = 1), their
 * final wall pass excluded; 0 disables.  Enabling or disabling resets the
 * accumulated time. */
LBM_API int lbm_set_profiling(lbm_handle* h, int enable);

/* Total device time (ms) of the kernel launches timed since profiling was
 * enabled, and their number (fused kernels, or flow sub-step kernels).
 * Synchronises the pending events. */
LBM_API int lbm_kernel_time(lbm_handle* h, double* total_ms, long long* launches);

/* Reason for the last failing call on h (or of lbm_create when h is NULL). */
LBM_API const char* lbm_last_error(const lbm_handle* h);

/* Library version string. */
LBM_API const char* lbm_version(void);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
