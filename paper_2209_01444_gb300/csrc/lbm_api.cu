// C ABI of the library (declared in include/lbm.h): parameter validation and
// lattice-unit conversion (Sec. 4), device state, CUDA-graph replay of the
// coupled step, field extraction, reductions and checkpoints.
#include <cuda_runtime.h>

#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "lbm.h"
#include "lbm_kernels.h"
#include "trace.h"

using lbm::StepParams;

namespace {

thread_local std::string g_create_error;

// Steps per captured graph: even, so every buffer returns to its parity.
constexpr int kGraphSteps = 16;

struct GraphKey {
    int cs, cf;
    bool operator<(const GraphKey& o) const { return cs != o.cs ? cs < o.cs : cf < o.cf; }
};

}  // namespace

struct lbm_handle {
    lbm_params prm;
    StepParams P;
    int storage = 0;
    size_t sc_bytes = 0, fl_bytes = 0;  // bytes of one scalar / flow population buffer
    cudaStream_t stream = nullptr;
    lbm::StepBuffers B{};
    uint8_t* grain = nullptr;          // device grain ids
    float2* grain_cs = nullptr;        // device (cos, sin) table
    std::vector<float2> grain_table;   // host copy of the table
    bool uniform = true;               // one orientation everywhere
    double* d_partials = nullptr;
    double* d_red = nullptr;
    void* scratch = nullptr;           // band buffer of the whole-grid transfers (allocated on first use)
    size_t scratch_bytes = 0;
    size_t io_chunk = (size_t)64 << 20;  // its size limit (lbm_set_io_chunk)
    double* d_seeds = nullptr;
    long long steps = 0;
    bool initialised = false;
    std::string err;
    std::map<GraphKey, cudaGraphExec_t> graphs;
    // kernel timing (lbm_set_profiling)
    bool profiling = false;
    int prof_substeps = 0;         // 1: time the flow sub-step kernels instead of the fused kernel
    std::vector<cudaEvent_t> ev;   // begin/end pairs of pending fused-kernel launches
    size_t ev_used = 0;
    double prof_ms = 0.0;
    long long prof_launches = 0;
    // lattice conversion
    double vf = 1, pscale = 1;  // paper velocity -> flow lattice, lattice pressure -> paper
    double ref[lbm::kPlanes];   // reference equilibrium of the stored deviations
    // device snapshots (lbm_snapshot_save) and surrogate scratch, allocated on first use
    void* snap_sc[2] = {nullptr, nullptr};
    void* snap_fl[2] = {nullptr, nullptr};
    float* snap_hist[2] = {nullptr, nullptr};
    long long snap_steps[2] = {-1, -1};
    float *sur_x = nullptr, *sur_y = nullptr, *sur_l = nullptr;
    unsigned long long* d_mis = nullptr;
    // periodic reductions (lbm_set_monitor): device ring of 10-double records
    int mon_every = 0, mon_cap = 0;
    double mon_cx = 0, mon_cy = 0, mon_c = 1, mon_s = 0;
    double* d_ring = nullptr;
    std::vector<long long> mon_steps;  // step of each record, in order of recording
    // flow-only steps: frozen phi and F_y
    float *flow_phi = nullptr, *flow_fy = nullptr;
    // events of the two halves of the shared pinned staging buffer (lbm_get_fields)
    cudaEvent_t pin_ev[2] = {nullptr, nullptr};
};

namespace {

int fail(lbm_handle* h, int code, const std::string& msg)
{
    if (h)
        h->err = msg;
    else
        g_create_error = msg;
    return code;
}

int cuda_fail(lbm_handle* h, cudaError_t e, const char* where)
{
    return fail(h, LBM_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define LBM_CUDA(h, call)                                  \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
    } while (0)

void drop_graphs(lbm_handle* h)
{
    for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
    h->graphs.clear();
}

bool valid_bc(int b) { return b >= LBM_BC_PERIODIC && b <= LBM_BC_DIRICHLET; }

std::string validate(const lbm_params* p)
{
    if (!p) return "params is NULL";
    if (p->nx < 4 || p->ny < 4) return "nx and ny must be >= 4";
    // the row-tiled kernels put 4 rows per CTA along grid.y (at most 65535)
    if (p->ny > 4 * 65535) return "ny must be <= 262140";
    if (p->nx > (1 << 30)) return "nx must be <= 2^30";
    if (p->isothermal != 0 && p->isothermal != 1) return "isothermal must be 0 or 1";
    if ((long long)p->nx * p->ny > (1LL << 31)) return "grid too large";
    const double reals[] = {p->W0,     p->tau0,  p->dx,        p->dt,    p->eps_s,     p->lambda,
                            p->k,      p->Mc_inf, p->D,        p->alpha, p->nu,        p->rho0,
                            p->gbetaT, p->gbetaC, p->theta_ref, p->C_ref, p->force[0],  p->force[1],
                            p->u_in[0], p->u_in[1], p->dir_phi, p->dir_U, p->dir_theta};
    for (double v : reals)
        if (!std::isfinite(v)) return "every real parameter must be finite";
    if (!(p->W0 > 0 && p->tau0 > 0 && p->dx > 0 && p->dt > 0)) return "W0, tau0, dx, dt must be > 0";
    if (!(p->eps_s >= 0 && p->eps_s < 1.0 / 3.0)) return "eps_s must be in [0, 1/3)";
    if (!(p->k > 0 && p->k < 1)) return "k must be in (0, 1)";
    if (!(p->D > 0 && p->alpha > 0 && p->nu > 0)) return "D, alpha, nu must be > 0";
    if (!(p->rho0 > 0)) return "rho0 must be > 0";
    if (p->n_sub < 1 || p->n_sub > 1000) return "n_sub must be in [1, 1000]";
    if (p->h_kind != 0 && p->h_kind != 1) return "h_kind must be 0 or 1";
    for (int b = 0; b < 4; ++b)
        if (!valid_bc(p->bc[b])) return "unknown wall type";
    if ((p->bc[0] == LBM_BC_PERIODIC) != (p->bc[1] == LBM_BC_PERIODIC)) return "left/right periodicity must match";
    if ((p->bc[2] == LBM_BC_PERIODIC) != (p->bc[3] == LBM_BC_PERIODIC)) return "bottom/top periodicity must match";
    if (p->storage < LBM_FP32 || p->storage > LBM_BF16) return "unknown storage";
    if (p->grad_mode != LBM_GRAD_FD9 && p->grad_mode != LBM_GRAD_LOCAL) return "unknown grad_mode";
    return "";
}

// Lattice-unit parameters (Sec. 4): dx = dt = 1 for the scalar models,
// dt/n_sub for the flow.
void derive(lbm_handle* h)
{
    const lbm_params& p = h->prm;
    StepParams& P = h->P;
    memset(&P, 0, sizeof(P));
    P.nx = p.nx;
    P.ny = p.ny;
    const size_t align = 32;  // 128-byte rows in FP32, 64-byte rows in 16-bit
    P.pitch = (int)((p.nx + align - 1) / align * align);
    P.plane = (long long)P.pitch * p.ny;
    P.periodic_x = p.bc[0] == LBM_BC_PERIODIC;
    P.periodic_y = p.bc[2] == LBM_BC_PERIODIC;
    P.h_kind = p.h_kind;
    const double W = p.W0 / p.dx, tau = p.tau0 / p.dt;
    const double dtf = p.dt / p.n_sub;
    const double Dl = p.D * p.dt / (p.dx * p.dx);
    const double al = p.alpha * p.dt / (p.dx * p.dx);
    const double nul = p.nu * dtf / (p.dx * p.dx);
    P.kappa3 = (float)(3.0 * W * W / tau);
    P.grad_local = p.grad_mode == LBM_GRAD_LOCAL ? 1 : 0;
    P.latent = p.isothermal ? 0.0f : 0.5f;
    P.inv_tau = (float)(1.0 / tau);
    P.eps = (float)p.eps_s;
    P.lambda = (float)p.lambda;
    P.k = (float)p.k;
    P.Mc = (float)p.Mc_inf;
    P.W = (float)W;
    P.inv_D = (float)(1.0 / Dl);
    P.s1C = (float)(1.0 / (3.0 * Dl * (1.0 - p.k) + 0.5));
    P.s1T = (float)(1.0 / (3.0 * al + 0.5));
    P.s2u = (float)(1.0 / (3.0 * nul + 0.5));
    P.rho0 = (float)p.rho0;
    h->vf = dtf / p.dx;
    const double ff = dtf * dtf / p.dx;
    h->pscale = (p.dx * p.dx) / (dtf * dtf);
    P.Fx = (float)(p.force[0] * ff);
    P.Fy = (float)(p.force[1] * ff);
    P.gbT = (float)(p.gbetaT * ff);
    P.gbC = (float)(p.gbetaC * ff);
    P.theta_ref = (float)p.theta_ref;
    P.dC_ref = (float)(1.0 - p.C_ref);
    P.nsub = (float)p.n_sub;
    P.cos_o = 1.0f;
    P.sin_o = 0.0f;
    for (int b = 0; b < 4; ++b) P.bc[b] = p.bc[b];
    P.uin_x = (float)(p.u_in[0] * h->vf);
    P.uin_y = (float)(p.u_in[1] * h->vf);
    P.dir_phi = (float)p.dir_phi;
    P.dir_U = (float)p.dir_U;
    P.dir_theta = (float)p.dir_theta;
    // Reference equilibrium whose deviations are stored (liquid at rest:
    // phi = -1, C = 1, theta = theta_ref, p = 0, H = theta_ref + L), kept in FP64 for the state
    // interface.
    const double w5[5] = {1.0 / 3, 1.0 / 6, 1.0 / 6, 1.0 / 6, 1.0 / 6};
    const double th = (double)P.theta_ref;
    for (int i = 0; i < 5; ++i) {
        h->ref[lbm::kF + i] = -w5[i];
        h->ref[lbm::kN + i] = i == 0 ? 1.0 : 0.0;
        h->ref[lbm::kG + i] = w5[i] * th + (i == 0 ? (double)P.latent : 0.0);
    }
    for (int i = 0; i < 9; ++i) h->ref[lbm::kH + i] = i == 0 ? (double)P.rho0 : 0.0;
}

int ensure_initialised(lbm_handle* h)
{
    if (!h) return LBM_EINVAL;
    if (!h->initialised) return fail(h, LBM_ESTATE, "state not initialised (call lbm_init_seeds or lbm_init_fields)");
    return LBM_OK;
}

int set_grains(lbm_handle* h, const std::vector<double>& orient_of_id, const std::vector<uint8_t>* host_ids)
{
    // one orientation everywhere: no grain plane is read by the step kernel
    h->grain_table.assign(256, make_float2(1.0f, 0.0f));
    for (size_t j = 0; j < orient_of_id.size(); ++j)
        h->grain_table[j] = make_float2((float)cos(orient_of_id[j]), (float)sin(orient_of_id[j]));
    bool uniform = true;
    for (size_t j = 1; j < orient_of_id.size(); ++j)
        if (orient_of_id[j] != orient_of_id[0]) uniform = false;
    h->uniform = uniform;
    h->P.cos_o = h->grain_table[0].x;
    h->P.sin_o = h->grain_table[0].y;
    LBM_CUDA(h, cudaMemcpyAsync(h->grain_cs, h->grain_table.data(), 256 * sizeof(float2), cudaMemcpyHostToDevice,
                                h->stream));
    if (host_ids)
        LBM_CUDA(h, cudaMemcpyAsync(h->grain, host_ids->data(), (size_t)h->P.plane, cudaMemcpyHostToDevice,
                                    h->stream));
    h->P.grain_cs = h->grain_cs;
    h->B.grain = uniform ? nullptr : h->grain;
    return LBM_OK;
}

// Rows per band for a transfer that keeps `node_bytes` per node in the band
// buffer, which is allocated (or grown) here: at most io_chunk bytes, at
// least one row of the widest transfer (96 bytes per node), never more than
// the whole grid needs.
int band_rows(lbm_handle* h, size_t node_bytes, int* rows)
{
    const size_t row_max = (size_t)h->P.pitch * (LBM_STATE_PLANES * sizeof(float));  // the widest transfer
    size_t want = std::min(h->io_chunk, row_max * (size_t)h->P.ny);
    want = std::max(want, row_max);
    if (h->scratch_bytes != want) {
        LBM_CUDA(h, cudaStreamSynchronize(h->stream));
        if (h->scratch) cudaFree(h->scratch);
        h->scratch = nullptr;
        h->scratch_bytes = 0;
        cudaError_t e = cudaMalloc(&h->scratch, want);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(h, LBM_ENOMEM, std::string("band buffer: ") + cudaGetErrorString(e));
        }
        h->scratch_bytes = want;
    }
    const size_t r = h->scratch_bytes / ((size_t)h->P.pitch * node_bytes);
    *rows = (int)std::max<size_t>(1, std::min<size_t>(r, (size_t)h->P.ny));
    return LBM_OK;
}

// Decoded state of the rows [y0, y0 + hgt) in bands: deliver(y, r, pops,
// hist) receives each band's 24 FP32 population-deviation planes and 6
// history planes in host memory (r * pitch values each).
template <class Deliver>
int decode_rows(lbm_handle* h, int y0, int hgt, Deliver deliver)
{
    int rows, rc;
    if ((rc = band_rows(h, LBM_STATE_PLANES * sizeof(float), &rows))) return rc;
    const size_t pitch = (size_t)h->P.pitch;
    float* dev = (float*)h->scratch;
    std::vector<float> planes((size_t)rows * pitch * LBM_STATE_PLANES);
    for (int y = y0; y < y0 + hgt; y += rows) {
        const int r = std::min(rows, y0 + hgt - y);
        const size_t band = (size_t)r * pitch;
        LBM_CUDA(h, lbm::launch_decode(h->P, h->storage, h->B.sc[h->B.cs], h->B.fl[h->B.cf], h->B.hist, dev, y, r,
                                       h->stream));
        LBM_CUDA(h, cudaMemcpyAsync(planes.data(), dev, band * LBM_STATE_PLANES * sizeof(float),
                                    cudaMemcpyDeviceToHost, h->stream));
        LBM_CUDA(h, cudaStreamSynchronize(h->stream));
        if ((rc = deliver(y, r, planes.data(), planes.data() + lbm::kPlanes * band))) return rc;
    }
    return LBM_OK;
}

int graph_for(lbm_handle* h, cudaGraphExec_t* out);

// The step graph of the current buffer parity, built when a state is set so
// that its capture, instantiation and upload belong to initialisation, not to
// the first lbm_step.  Best effort: a capture that fails here is retried, and
// reported, by lbm_step.
void prebuild_graph(lbm_handle* h)
{
    if (h->profiling) return;
    cudaGraphExec_t ex;
    if (graph_for(h, &ex) != LBM_OK || cudaGraphUpload(ex, h->stream) != cudaSuccess) cudaGetLastError();
}

// Initial state, band by band: fill(y0, rows, fields) writes the band's six
// FP64 macro planes (lattice units) into `fields`, then the equilibrium
// populations and the history of those rows follow from them.
template <class Fill>
int init_bands(lbm_handle* h, Fill fill)
{
    h->B.cs = 0;
    h->B.cf = 0;
    h->steps = 0;
    drop_graphs(h);
    int rows, rc;
    if ((rc = band_rows(h, 6 * sizeof(double), &rows))) return rc;
    double* fields = (double*)h->scratch;
    for (int y0 = 0; y0 < h->P.ny; y0 += rows) {
        const int r = std::min(rows, h->P.ny - y0);
        if ((rc = fill(y0, r, fields))) return rc;
        LBM_CUDA(h, lbm::launch_init_from_fields(h->P, h->storage, fields, h->B.sc[0], h->B.fl[0], h->B.hist, y0, r,
                                                 h->stream));
    }
    LBM_CUDA(h, cudaStreamSynchronize(h->stream));
    h->initialised = true;
    prebuild_graph(h);
    return LBM_OK;
}

int collect_profile(lbm_handle* h)
{
    if (!h->ev_used) return LBM_OK;
    LBM_CUDA(h, cudaEventSynchronize(h->ev[h->ev_used - 1]));
    for (size_t i = 0; i + 1 < h->ev_used; i += 2) {
        float ms = 0.0f;
        LBM_CUDA(h, cudaEventElapsedTime(&ms, h->ev[i], h->ev[i + 1]));
        h->prof_ms += ms;
        h->prof_launches += h->prof_substeps ? h->prm.n_sub - 1 : 1;
    }
    h->ev_used = 0;
    return LBM_OK;
}

int run_steps_direct(lbm_handle* h, int n)
{
    for (int i = 0; i < n; ++i) {
        if (h->profiling) {
            if (h->ev_used + 2 > h->ev.size()) {
                int rc = collect_profile(h);
                if (rc) return rc;
                while (h->ev.size() < 512) {
                    cudaEvent_t e;
                    LBM_CUDA(h, cudaEventCreate(&e));
                    h->ev.push_back(e);
                }
            }
            h->B.ev_begin = h->ev[h->ev_used++];
            h->B.ev_end = h->ev[h->ev_used++];
            h->B.ev_substeps = h->prof_substeps;
        }
        cudaError_t e = lbm::launch_coupled_step(h->P, h->storage, h->prm.n_sub, h->B, h->stream);
        h->B.ev_begin = h->B.ev_end = nullptr;
        if (e != cudaSuccess) return cuda_fail(h, e, "coupled step");
    }
    return LBM_OK;
}

int graph_for(lbm_handle* h, cudaGraphExec_t* out)
{
    const GraphKey key{h->B.cs, h->B.cf};
    auto it = h->graphs.find(key);
    if (it != h->graphs.end()) {
        *out = it->second;
        return LBM_OK;
    }
    cudaStream_t cap;
    LBM_CUDA(h, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    lbm::StepBuffers saved = h->B;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        // the left/right walls of all but the last step are updated by the
        // next step as it loads them (see launch_coupled_step); the graph's
        // first step takes the state as stored and its last leaves it complete
        for (int i = 0; i < kGraphSteps && e == cudaSuccess; ++i)
            e = lbm::launch_coupled_step(h->P, h->storage, h->prm.n_sub, h->B, cap, i > 0, i + 1 < kGraphSteps);
        cudaError_t e2 = cudaStreamEndCapture(cap, &g);
        if (e == cudaSuccess) e = e2;
    }
    h->B = saved;  // the capture only recorded the launches
    cudaStreamDestroy(cap);
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(h, e, "graph capture");
    }
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(h, e, "graph instantiate");
    h->graphs[key] = ex;
    *out = ex;
    return LBM_OK;
}

// Pinned host staging buffer of lbm_get_fields (and of lbm_get_fields_f32 into
// pageable memory), shared by every handle of the process (at most 2 x
// kPinHalf bytes, allocated on first use, kept until exit); a call holds the
// mutex while it uses it.
constexpr size_t kPinHalf = (size_t)32 << 20;
struct PinnedStaging {
    std::mutex mu;
    float* p = nullptr;
    size_t bytes = 0;
} g_pinned;

// The shared staging buffer, grown to at least `bytes`; the caller holds
// g_pinned.mu for as long as it uses the buffer.  Null (with h's error set)
// when page-locked memory cannot be had.
float* staging_buffer(lbm_handle* h, size_t bytes)
{
    if (g_pinned.bytes < bytes) {
        if (g_pinned.p) cudaFreeHost(g_pinned.p);
        g_pinned.p = nullptr;
        g_pinned.bytes = 0;
        cudaError_t e = cudaHostAlloc((void**)&g_pinned.p, bytes, cudaHostAllocPortable);
        if (e != cudaSuccess) {
            cudaGetLastError();
            fail(h, LBM_ENOMEM, std::string("pinned band buffer: ") + cudaGetErrorString(e));
            return nullptr;
        }
        g_pinned.bytes = bytes;
    }
    return g_pinned.p;
}

// Runs fn(r0, r1) over the row range [0, rows) on up to 16 host threads.
template <class Fn>
void parallel_rows(int rows, Fn fn)
{
    const int nt = std::max(1, std::min({(int)std::thread::hardware_concurrency(), 16, rows / 8}));
    if (nt == 1) {
        fn(0, rows);
        return;
    }
    std::vector<std::thread> pool;
    for (int t = 0; t < nt; ++t) pool.emplace_back(fn, rows * t / nt, rows * (t + 1) / nt);
    for (std::thread& th : pool) th.join();
}

}  // namespace

extern "C" {

int lbm_params_default(lbm_params* p, int nx, int ny)
{
    if (!p) return LBM_EINVAL;
    memset(p, 0, sizeof(*p));
    p->nx = nx;
    p->ny = ny;
    p->W0 = 1.0;
    p->tau0 = 1.0;
    p->dx = 1.0;
    p->dt = 0.05;
    p->eps_s = 0.05;
    p->lambda = 3.1913;
    p->k = 0.15;
    p->Mc_inf = 0.5325;
    p->D = 2.0;
    p->alpha = 2.0;
    p->nu = 2.0;
    p->rho0 = 1.0;
    p->n_sub = 1;
    p->h_kind = 0;
    p->theta_ref = -0.55;
    p->C_ref = 1.0;
    for (int b = 0; b < 4; ++b) p->bc[b] = LBM_BC_PERIODIC;
    p->dir_phi = -1.0;
    p->dir_U = 0.0;
    p->dir_theta = -0.55;
    p->storage = LBM_FP32;
    p->grad_mode = LBM_GRAD_FD9;
    p->isothermal = 0;
    return LBM_OK;
}

int lbm_create(const lbm_params* p, lbm_handle** out)
{
    if (!out) return fail(nullptr, LBM_EINVAL, "out is NULL");
    *out = nullptr;
    std::string why = validate(p);
    if (!why.empty()) return fail(nullptr, LBM_EINVAL, why);
    lbm_handle* h = new (std::nothrow) lbm_handle();
    if (!h) return fail(nullptr, LBM_ENOMEM, "host allocation failed");
    h->prm = *p;
    h->storage = p->storage;
    derive(h);
    h->sc_bytes = (size_t)h->P.plane * lbm::scalar_node_bytes(p->storage);
    h->fl_bytes = (size_t)h->P.plane * lbm::flow_node_bytes(p->storage);
    const size_t fp = (size_t)h->P.plane * sizeof(float);
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void** ptr, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(ptr, bytes);
    };
    for (int b = 0; b < 2; ++b) {
        alloc(&h->B.sc[b], h->sc_bytes);
        alloc(&h->B.fl[b], h->fl_bytes);
    }
    alloc((void**)&h->B.hist, fp * lbm::kHist);
    if (p->n_sub > 1) alloc((void**)&h->B.fb, fp);
    alloc((void**)&h->grain, (size_t)h->P.plane);
    alloc((void**)&h->grain_cs, 256 * sizeof(float2));
    alloc((void**)&h->d_partials, lbm::reduce_partials_size(h->P) * sizeof(double));
    alloc((void**)&h->d_red, 16 * sizeof(double));
    alloc((void**)&h->d_seeds, 256 * 4 * sizeof(double));
    if (e == cudaSuccess) e = cudaMemset(h->grain, 0, (size_t)h->P.plane);
    if (e != cudaSuccess) {
        std::string msg = std::string("device allocation: ") + cudaGetErrorString(e);
        lbm_destroy(h);
        cudaGetLastError();
        return fail(nullptr, e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, msg);
    }
    h->P.grain_cs = h->grain_cs;
    *out = h;
    return LBM_OK;
}

int lbm_set_io_chunk(lbm_handle* h, size_t bytes)
{
    if (!h) return LBM_EINVAL;
    if (bytes < 1) return fail(h, LBM_EINVAL, "io chunk of 0 bytes");
    h->io_chunk = bytes;
    return LBM_OK;
}

void lbm_destroy(lbm_handle* h)
{
    if (!h) return;
    drop_graphs(h);
    for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
    void* ptrs[] = {h->B.sc[0], h->B.sc[1], h->B.fl[0], h->B.fl[1], h->B.hist, h->B.fb, h->grain,
                    h->grain_cs, h->d_partials, h->d_red, h->scratch, h->d_seeds,
                    h->snap_sc[0], h->snap_sc[1], h->snap_fl[0], h->snap_fl[1], h->snap_hist[0], h->snap_hist[1],
                    h->sur_x, h->sur_y, h->sur_l, h->d_mis, h->d_ring, h->flow_phi, h->flow_fy};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    for (cudaEvent_t e : h->pin_ev)
        if (e) cudaEventDestroy(e);
    delete h;
}

int lbm_set_stream(lbm_handle* h, void* stream)
{
    if (!h) return LBM_EINVAL;
    h->stream = (cudaStream_t)stream;
    return LBM_OK;
}

int lbm_init_seeds(lbm_handle* h, const lbm_seed* seeds, int n, double U0, double theta0)
{
    if (!h) return LBM_EINVAL;
    if (!seeds || n < 1 || n > 256) return fail(h, LBM_EINVAL, "need 1..256 seeds");
    std::vector<double> s(4 * (size_t)n);
    std::vector<double> orient(n);
    for (int j = 0; j < n; ++j) {
        s[4 * j + 0] = seeds[j].x;
        s[4 * j + 1] = seeds[j].y;
        s[4 * j + 2] = seeds[j].R;
        s[4 * j + 3] = seeds[j].orient;
        orient[j] = seeds[j].orient;
        if (!isfinite(seeds[j].x) || !isfinite(seeds[j].y) || !isfinite(seeds[j].R) || !isfinite(seeds[j].orient))
            return fail(h, LBM_EINVAL, "non-finite seed");
    }
    LBM_CUDA(h, cudaMemcpyAsync(h->d_seeds, s.data(), s.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    int rc = set_grains(h, orient, nullptr);
    if (rc) return rc;
    const double W = h->prm.W0 / h->prm.dx;
    return init_bands(h, [&](int y0, int r, double* fields) {
        LBM_CUDA(h, lbm::launch_seed_fields(h->P, h->d_seeds, n, U0, theta0, W, fields, h->grain, y0, r, h->stream));
        return LBM_OK;
    });
}

int lbm_init_fields(lbm_handle* h, const double* fields, const double* orient)
{
    if (!h) return LBM_EINVAL;
    if (!fields) return fail(h, LBM_EINVAL, "fields is NULL");
    const int nx = h->P.nx, ny = h->P.ny, pitch = h->P.pitch;
    const size_t N = (size_t)nx * ny;
    std::vector<double> f64((size_t)h->P.plane * 6, 0.0);
    const double scale[6] = {1, 1, 1, h->vf, h->vf, 1.0 / h->pscale};
    for (int q = 0; q < 6; ++q)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                double v = fields[q * N + (size_t)y * nx + x];
                if (!isfinite(v)) return fail(h, LBM_EINVAL, "non-finite initial field");
                f64[(size_t)q * h->P.plane + (size_t)y * pitch + x] = v * scale[q];
            }
    std::vector<double> table;
    std::vector<uint8_t> ids((size_t)h->P.plane, 0);
    if (orient) {
        std::map<double, int> index;
        for (size_t i = 0; i < N; ++i) {
            double o = orient[i];
            if (!isfinite(o)) return fail(h, LBM_EINVAL, "non-finite orientation");
            auto it = index.find(o);
            if (it == index.end()) {
                if (index.size() == 256) return fail(h, LBM_EINVAL, "more than 256 distinct orientations");
                it = index.emplace(o, (int)table.size()).first;
                table.push_back(o);
            }
            ids[(i / nx) * pitch + (i % nx)] = (uint8_t)it->second;
        }
    } else {
        table.push_back(0.0);
    }
    int rc = set_grains(h, table, &ids);
    if (rc) return rc;
    const size_t plane = (size_t)h->P.plane;
    return init_bands(h, [&](int y0, int r, double* fields) {
        const size_t band = (size_t)r * pitch;
        for (int q = 0; q < 6; ++q)
            LBM_CUDA(h, cudaMemcpyAsync(fields + q * band, f64.data() + q * plane + (size_t)y0 * pitch,
                                        band * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        return LBM_OK;
    });
}

namespace {

int step_chunk(lbm_handle* h, int nsteps)
{
    int rc;
    int left = nsteps;
    while (!h->profiling && left >= kGraphSteps) {
        cudaGraphExec_t ex;
        if ((rc = graph_for(h, &ex))) return rc;
        LBM_CUDA(h, cudaGraphLaunch(ex, h->stream));
        left -= kGraphSteps;
        h->steps += kGraphSteps;
    }
    if ((rc = run_steps_direct(h, left))) return rc;
    h->steps += left;
    return LBM_OK;
}

// Queues the metrics reduction of the current state into the next ring slot.
int monitor_record(lbm_handle* h)
{
    const int slot = (int)(h->mon_steps.size() % (size_t)h->mon_cap);
    LBM_CUDA(h, lbm::launch_reduce(h->P, h->storage, h->B.sc[h->B.cs], h->B.fl[h->B.cf], h->mon_cx, h->mon_cy,
                                   h->mon_c, h->mon_s, h->d_partials, h->d_ring + (size_t)slot * 10, h->stream));
    h->mon_steps.push_back(h->steps);
    return LBM_OK;
}

}  // namespace

int lbm_step(lbm_handle* h, int nsteps)
{
    trace::Range range("lbm_step");
    int rc = ensure_initialised(h);
    if (rc) return rc;
    if (nsteps < 0) return fail(h, LBM_EINVAL, "nsteps < 0");
    if (!h->mon_every) return step_chunk(h, nsteps);
    // with a monitor: stop at every multiple of the period and record
    int left = nsteps;
    while (left > 0) {
        const int to_next = h->mon_every - (int)(h->steps % h->mon_every);
        const int n = left < to_next ? left : to_next;
        if ((rc = step_chunk(h, n))) return rc;
        left -= n;
        if (h->steps % h->mon_every == 0 && (rc = monitor_record(h))) return rc;
    }
    return LBM_OK;
}

int lbm_step_flow(lbm_handle* h, int nsteps)
{
    trace::Range range("lbm_step_flow");
    int rc = ensure_initialised(h);
    if (rc) return rc;
    if (nsteps < 0) return fail(h, LBM_EINVAL, "nsteps < 0");
    if (!h->flow_phi) {
        LBM_CUDA(h, cudaMalloc((void**)&h->flow_phi, (size_t)h->P.plane * sizeof(float)));
        LBM_CUDA(h, cudaMalloc((void**)&h->flow_fy, (size_t)h->P.plane * sizeof(float)));
    }
    LBM_CUDA(h, lbm::launch_flow_inputs(h->P, h->storage, h->B.sc[h->B.cs], h->B.fl[h->B.cf], h->flow_phi, h->flow_fy,
                                        h->stream));
    void* const fl[2] = {h->B.fl[0], h->B.fl[1]};
    LBM_CUDA(h, lbm::flow_steps(h->P, h->storage, nsteps, h->B.sc[h->B.cs], fl, &h->B.cf, h->flow_phi, h->flow_fy,
                                h->stream));
    return LBM_OK;
}

int lbm_get_force(lbm_handle* h, double cx, double cy, double* out)
{
    int rc = ensure_initialised(h);
    if (rc) return rc;
    if (!out) return fail(h, LBM_EINVAL, "out is NULL");
    if (!isfinite(cx) || !isfinite(cy)) return fail(h, LBM_EINVAL, "non-finite centre");
    LBM_CUDA(h, lbm::launch_force(h->P, h->storage, h->B.sc[h->B.cs], h->B.fl[h->B.cf], cx, cy, h->d_partials,
                                  h->d_red, h->stream));
    LBM_CUDA(h, cudaMemcpyAsync(out, h->d_red, 3 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    LBM_CUDA(h, cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

int lbm_set_monitor(lbm_handle* h, int every, int capacity, double cx, double cy, double orient)
{
    int rc = ensure_initialised(h);
    if (rc) return rc;
    if (every < 0 || (every > 0 && (capacity < 2 || capacity > (1 << 20))))
        return fail(h, LBM_EINVAL, "monitor: every >= 0 and 2 <= capacity <= 2^20");
    if (!isfinite(cx) || !isfinite(cy) || !isfinite(orient)) return fail(h, LBM_EINVAL, "non-finite tip origin");
    LBM_CUDA(h, cudaStreamSynchronize(h->stream));
    if (h->d_ring) {
        cudaFree(h->d_ring);
        h->d_ring = nullptr;
    }
    h->mon_steps.clear();
    h->mon_every = every;
    h->mon_cap = capacity;
    if (!every) return LBM_OK;
    h->mon_cx = cx;
    h->mon_cy = cy;
    h->mon_c = cos(orient);
    h->mon_s = sin(orient);
    LBM_CUDA(h, cudaMalloc((void**)&h->d_ring, (size_t)capacity * 10 * sizeof(double)));
    if (h->steps % every == 0) return monitor_record(h);
    return LBM_OK;
}

int lbm_get_monitor(lbm_handle* h, lbm_metrics* out, double* v_tip, int max, int* count)
{
    if (!h || !count || (max > 0 && !out)) return LBM_EINVAL;
    *count = 0;
    if (!h->mon_every) return LBM_OK;
    const size_t total = h->mon_steps.size();
    const size_t avail = total < (size_t)h->mon_cap ? total : (size_t)h->mon_cap;
    std::vector<double> ring((size_t)h->mon_cap * 10);
    LBM_CUDA(h, cudaMemcpyAsync(ring.data(), h->d_ring, ring.size() * sizeof(double), cudaMemcpyDeviceToHost,
                                h->stream));
    LBM_CUDA(h, cudaStreamSynchronize(h->stream));
    const size_t first = total - avail;  // oldest record still in the ring
    const size_t n = avail < (size_t)max ? avail : (size_t)(max > 0 ? max : 0);
    const size_t start = total - n;      // the newest n records, oldest first
    const double N = (double)h->P.nx * h->P.ny;
    for (size_t i = 0; i < n; ++i) {
        const size_t k = start + i;
        const double* r = &ring[(k % (size_t)h->mon_cap) * 10];
        lbm_metrics& m = out[i];
        m.tip[0] = r[7];
        m.tip[1] = r[8];
        m.tip[2] = r[9];
        m.solid_fraction = r[0] / N;
        m.sum_C = r[1];
        m.sum_H = r[2];
        m.sum_h = r[3];
        m.max_u = r[4] / h->vf;
        m.nonfinite = r[5] > 0 ? 1.0 : 0.0;
        m.sum_phi = r[6];
        m.step = h->mon_steps[k];
        if (v_tip) {
            for (int a = 0; a < 3; ++a) {
                double v = NAN;
                if (i > 0 || k > first) {
                    const double* p = &ring[((k - 1) % (size_t)h->mon_cap) * 10];
                    const double dt = (double)(h->mon_steps[k] - h->mon_steps[k - 1]) * h->prm.dt;
                    v = (r[7 + a] - p[7 + a]) * h->prm.dx / dt;
                }
                v_tip[i * 3 + a] = v;
            }
        }
    }
    *count = (int)n;
    return LBM_OK;
}

int lbm_synchronize(lbm_handle* h)
{
    if (!h) return LBM_EINVAL;
    LBM_CUDA(h, cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

long long lbm_step_count(const lbm_handle* h) { return h ? h->steps : -1; }

int lbm_get_fields(lbm_handle* h, unsigned mask, double* out)
{
    int rc = ensure_initialised(h);
    if (rc) return rc;
    if (!out) return fail(h, LBM_EINVAL, "out is NULL");
    if (mask >> LBM_NUM_FIELDS) return fail(h, LBM_EINVAL, "unknown field bit");
    const int nx = h->P.nx, ny = h->P.ny, pitch = h->P.pitch;
    // device planes hold phi + 1, C - 1, U, theta - theta_ref, ux, uy, p
    const double scale[LBM_NUM_FIELDS] = {1, 1, 1, 1, 1.0 / h->vf, 1.0 / h->vf, h->pscale};
    const double offset[LBM_NUM_FIELDS] = {-1.0, 1.0, 0, (double)h->P.theta_ref, 0, 0, 0};
    int rows;
    if ((rc = band_rows(h, LBM_NUM_FIELDS * sizeof(float), &rows))) return rc;
    float* dev = (float*)h->scratch;
    int sel[LBM_NUM_FIELDS], nsel = 0;
    for (int q = 0; q < LBM_NUM_FIELDS; ++q)
        if (mask & (1u << q)) sel[nsel++] = q;
    if (!nsel) return LBM_OK;
    // two pinned halves: the host converts one band while the next is computed and copied
    rows = std::max(1, std::min<int>(rows, (int)(kPinHalf / ((size_t)pitch * nsel * sizeof(float)))));
    const size_t half = (size_t)rows * pitch * nsel;
    std::lock_guard<std::mutex> lock(g_pinned.mu);
    float* pin = staging_buffer(h, 2 * half * sizeof(float));
    if (!pin) return LBM_ENOMEM;
    for (cudaEvent_t& e : h->pin_ev)
        if (!e) LBM_CUDA(h, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    auto convert = [&](int y0, int r, const float* src) {
        const size_t band = (size_t)r * pitch;
        parallel_rows(r, [&](int r0, int r1) {
            for (int k = 0; k < nsel; ++k) {
                const int q = sel[k];
                const double sq = scale[q], oq = offset[q];
                for (int y = r0; y < r1; ++y) {
                    const float* in = src + (size_t)k * band + (size_t)y * pitch;
                    double* o = out + (size_t)k * nx * ny + (size_t)(y0 + y) * nx;
                    for (int x = 0; x < nx; ++x) o[x] = (double)in[x] * sq + oq;
                }
            }
        });
    };
    int prev_y0 = -1, prev_r = 0, slot = 0;
    for (int y0 = 0; y0 < ny; y0 += rows, slot ^= 1) {
        const int r = std::min(rows, ny - y0);
        const size_t band = (size_t)r * pitch;
        float* dst = pin + (size_t)slot * half;
        LBM_CUDA(h, lbm::launch_macros(h->P, h->storage, h->B.sc[h->B.cs], h->B.fl[h->B.cf], dev, y0, r, h->stream));
        // only the requested planes cross to the host
        for (int k = 0; k < nsel; ++k)
            LBM_CUDA(h, cudaMemcpyAsync(dst + k * band, dev + (size_t)sel[k] * band, band * sizeof(float),
                                        cudaMemcpyDeviceToHost, h->stream));
        LBM_CUDA(h, cudaEventRecord(h->pin_ev[slot], h->stream));
        if (prev_y0 >= 0) {
            LBM_CUDA(h, cudaEventSynchronize(h->pin_ev[slot ^ 1]));
            convert(prev_y0, prev_r, pin + (size_t)(slot ^ 1) * half);
        }
        prev_y0 = y0;
        prev_r = r;
    }
    LBM_CUDA(h, cudaEventSynchronize(h->pin_ev[slot ^ 1]));
    convert(prev_y0, prev_r, pin + (size_t)(slot ^ 1) * half);
    return LBM_OK;
}

int lbm_get_fields_f32(lbm_handle* h, unsigned mask, float* out)
{
    int rc = ensure_initialised(h);
    if (rc) return rc;
    if (!out) return fail(h, LBM_EINVAL, "out is NULL");
    if (mask >> LBM_NUM_FIELDS) return fail(h, LBM_EINVAL, "unknown field bit");
    const int nx = h->P.nx, ny = h->P.ny;
    // device planes hold phi + 1, C - 1, U, theta - theta_ref, ux, uy, p
    const double scale[LBM_NUM_FIELDS] = {1, 1, 1, 1, 1.0 / h->vf, 1.0 / h->vf, h->pscale};
    const double offset[LBM_NUM_FIELDS] = {-1.0, 1.0, 0, (double)h->P.theta_ref, 0, 0, 0};
    lbm::FieldsF32 spec{};
    for (int q = 0; q < LBM_NUM_FIELDS; ++q)
        if (mask & (1u << q)) {
            spec.sel[spec.n] = q;
            spec.scale[spec.n] = (float)scale[q];
            spec.offset[spec.n] = (float)offset[q];
            ++spec.n;
        }
    if (!spec.n) return LBM_OK;
    int rows;
    if ((rc = band_rows(h, spec.n * sizeof(float), &rows))) return rc;
    float* dev = (float*)h->scratch;
    // page-locked output takes the copies directly; pageable output goes through
    // the pinned staging halves, a host copy of one band overlapping the next
    cudaPointerAttributes at{};
    const bool locked = cudaPointerGetAttributes(&at, out) == cudaSuccess && at.type == cudaMemoryTypeHost;
    cudaGetLastError();
    std::unique_lock<std::mutex> lock(g_pinned.mu, std::defer_lock);
    float* pin = nullptr;
    size_t half = 0;
    if (!locked) {
        rows = std::max(1, std::min<int>(rows, (int)(kPinHalf / ((size_t)nx * spec.n * sizeof(float)))));
        half = (size_t)rows * nx * spec.n;
        lock.lock();
        if (!(pin = staging_buffer(h, 2 * half * sizeof(float)))) return LBM_ENOMEM;
        for (cudaEvent_t& e : h->pin_ev)
            if (!e) LBM_CUDA(h, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    auto unstage = [&](int y0, int r, const float* src) {
        const size_t band = (size_t)r * nx;
        parallel_rows(r, [&](int r0, int r1) {
            for (int k = 0; k < spec.n; ++k)
                memcpy(out + (size_t)k * nx * ny + (size_t)(y0 + r0) * nx, src + k * band + (size_t)r0 * nx,
                       (size_t)(r1 - r0) * nx * sizeof(float));
        });
    };
    int prev_y0 = -1, prev_r = 0, slot = 0;
    for (int y0 = 0; y0 < ny; y0 += rows, slot ^= 1) {
        const int r = std::min(rows, ny - y0);
        const size_t band = (size_t)r * nx;
        LBM_CUDA(h, lbm::launch_fields_f32(h->P, h->storage, h->B.sc[h->B.cs], h->B.fl[h->B.cf], spec, dev, y0, r,
                                           h->stream));
        if (locked) {
            // plane k of the band is one contiguous run of the caller's array
            for (int k = 0; k < spec.n; ++k)
                LBM_CUDA(h, cudaMemcpyAsync(out + (size_t)k * nx * ny + (size_t)y0 * nx, dev + k * band,
                                            band * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
            continue;
        }
        LBM_CUDA(h, cudaMemcpyAsync(pin + (size_t)slot * half, dev, band * spec.n * sizeof(float),
                                    cudaMemcpyDeviceToHost, h->stream));
        LBM_CUDA(h, cudaEventRecord(h->pin_ev[slot], h->stream));
        if (prev_y0 >= 0) {
            LBM_CUDA(h, cudaEventSynchronize(h->pin_ev[slot ^ 1]));
            unstage(prev_y0, prev_r, pin + (size_t)(slot ^ 1) * half);
        }
        prev_y0 = y0;
        prev_r = r;
    }
    if (locked) {
        LBM_CUDA(h, cudaStreamSynchronize(h->stream));
        return LBM_OK;
    }
    LBM_CUDA(h, cudaEventSynchronize(h->pin_ev[slot ^ 1]));
    unstage(prev_y0, prev_r, pin + (size_t)(slot ^ 1) * half);
    return LBM_OK;
}

int lbm_get_state(lbm_handle* h, double* out)
{
    int rc = ensure_initialised(h);
    if (rc) return rc;
    if (!out) return fail(h, LBM_EINVAL, "out is NULL");
    const int nx = h->P.nx, ny = h->P.ny;
    const size_t pitch = (size_t)h->P.pitch;
    return decode_rows(h, 0, ny, [&](int y0, int r, const float* pops, const float* hist) {
        const size_t band = (size_t)r * pitch;
        for (int q = 0; q < LBM_STATE_PLANES; ++q) {
            const bool pop = q < lbm::kPlanes;
            const double ref = pop ? h->ref[q] : 0.0;
            const float* src = pop ? pops + q * band : hist + (q - lbm::kPlanes) * band;
            for (int y = 0; y < r; ++y)
                for (int x = 0; x < nx; ++x)
                    out[(size_t)q * nx * ny + (size_t)(y0 + y) * nx + x] = ref + (double)src[(size_t)y * pitch + x];
        }
        return LBM_OK;
    });
}

int lbm_get_state_region(lbm_handle* h, int x0, int y0, int w, int hgt, double* out)
{
    int rc = ensure_initialised(h);
    if (rc) return rc;
    if (!out) return fail(h, LBM_EINVAL, "out is NULL");
    if (w < 1 || hgt < 1 || x0 < 0 || y0 < 0 || x0 + w > h->P.nx || y0 + hgt > h->P.ny)
        return fail(h, LBM_EINVAL, "window outside the grid");
    const size_t pitch = (size_t)h->P.pitch, wn = (size_t)w * hgt;
    return decode_rows(h, y0, hgt, [&](int yb, int r, const float* pops, const float* hist) {
        const size_t band = (size_t)r * pitch;
        for (int q = 0; q < LBM_STATE_PLANES; ++q) {
            const bool pop = q < lbm::kPlanes;
            const double ref = pop ? h->ref[q] : 0.0;
            const float* src = pop ? pops + q * band : hist + (q - lbm::kPlanes) * band;
            for (int y = 0; y < r; ++y)
                for (int x = 0; x < w; ++x)
                    out[q * wn + (size_t)(yb - y0 + y) * w + x] = ref + (double)src[(size_t)y * pitch + x0 + x];
        }
        return LBM_OK;
    });
}

int lbm_set_state(lbm_handle* h, const double* in)
{
    int rc = ensure_initialised(h);
    if (rc) return rc;
    if (!in) return fail(h, LBM_EINVAL, "in is NULL");
    const int nx = h->P.nx, ny = h->P.ny;
    const size_t pitch = (size_t)h->P.pitch, N = (size_t)nx * ny;
    for (size_t i = 0; i < N * LBM_STATE_PLANES; ++i)  // the whole input first: a refusal changes nothing
        if (!isfinite(in[i])) return fail(h, LBM_EINVAL, "non-finite state value");
    int rows;
    if ((rc = band_rows(h, LBM_STATE_PLANES * sizeof(float), &rows))) return rc;
    float* dev = (float*)h->scratch;
    std::vector<float> host((size_t)rows * pitch * LBM_STATE_PLANES, 0.0f);
    for (int y0 = 0; y0 < ny; y0 += rows) {
        const int r = std::min(rows, ny - y0);
        const size_t band = (size_t)r * pitch;
        for (int q = 0; q < LBM_STATE_PLANES; ++q) {
            const double ref = q < lbm::kPlanes ? h->ref[q] : 0.0;
            for (int y = 0; y < r; ++y)
                for (int x = 0; x < nx; ++x)
                    host[q * band + (size_t)y * pitch + x] =
                        (float)(in[(size_t)q * N + (size_t)(y0 + y) * nx + x] - ref);
        }
        LBM_CUDA(h, cudaMemcpyAsync(dev, host.data(), band * LBM_STATE_PLANES * sizeof(float),
                                    cudaMemcpyHostToDevice, h->stream));
        LBM_CUDA(h, lbm::launch_encode(h->P, h->storage, dev, h->B.sc[h->B.cs], h->B.fl[h->B.cf], h->B.hist, y0, r,
                                       h->stream));
        // the host band buffer is refilled for the next band
        LBM_CUDA(h, cudaStreamSynchronize(h->stream));
    }
    return LBM_OK;
}

int lbm_get_metrics(lbm_handle* h, double cx, double cy, double orient, lbm_metrics* m)
{
    int rc = ensure_initialised(h);
    if (rc) return rc;
    if (!m) return fail(h, LBM_EINVAL, "m is NULL");
    if (!isfinite(cx) || !isfinite(cy) || !isfinite(orient)) return fail(h, LBM_EINVAL, "non-finite tip origin");
    LBM_CUDA(h, lbm::launch_reduce(h->P, h->storage, h->B.sc[h->B.cs], h->B.fl[h->B.cf], cx, cy, cos(orient),
                                   sin(orient), h->d_partials, h->d_red, h->stream));
    double r[10];
    LBM_CUDA(h, cudaMemcpyAsync(r, h->d_red, sizeof(r), cudaMemcpyDeviceToHost, h->stream));
    LBM_CUDA(h, cudaStreamSynchronize(h->stream));
    const double N = (double)h->P.nx * h->P.ny;
    m->tip[0] = r[7];
    m->tip[1] = r[8];
    m->tip[2] = r[9];
    m->solid_fraction = r[0] / N;
    m->sum_C = r[1];
    m->sum_H = r[2];
    m->sum_h = r[3];
    m->max_u = r[4] / h->vf;
    m->nonfinite = r[5] > 0 ? 1.0 : 0.0;
    m->sum_phi = r[6];
    m->step = h->steps;
    if (r[5] > 0) return fail(h, LBM_ENUMERIC, "non-finite value in the state");
    return LBM_OK;
}

// Checkpoint layout: header, then the newest scalar and flow buffers (raw
// storage precision), history, grain ids, orientation table.
struct CkptHeader {
    char magic[8];
    lbm_params prm;
    long long steps;
    int uniform;
    int pad;
};

size_t lbm_checkpoint_bytes(const lbm_handle* h)
{
    if (!h) return 0;
    const size_t plane = (size_t)h->P.plane;
    return sizeof(CkptHeader) + h->sc_bytes + h->fl_bytes + plane * sizeof(float) * lbm::kHist + plane +
           256 * sizeof(float2);
}

int lbm_save_state(lbm_handle* h, void* host, size_t bytes)
{
    int rc = ensure_initialised(h);
    if (rc) return rc;
    if (!host || bytes < lbm_checkpoint_bytes(h)) return fail(h, LBM_EINVAL, "checkpoint buffer too small");
    char* p = (char*)host;
    CkptHeader hd;
    memset(&hd, 0, sizeof(hd));
    memcpy(hd.magic, "LBMCKPT3", 8);
    hd.prm = h->prm;
    hd.steps = h->steps;
    hd.uniform = h->uniform ? 1 : 0;
    memcpy(p, &hd, sizeof(hd));
    p += sizeof(hd);
    const size_t plane = (size_t)h->P.plane;
    const size_t sb = h->sc_bytes, fbz = h->fl_bytes;
    LBM_CUDA(h, cudaMemcpyAsync(p, h->B.sc[h->B.cs], sb, cudaMemcpyDeviceToHost, h->stream));
    p += sb;
    LBM_CUDA(h, cudaMemcpyAsync(p, h->B.fl[h->B.cf], fbz, cudaMemcpyDeviceToHost, h->stream));
    p += fbz;
    LBM_CUDA(h, cudaMemcpyAsync(p, h->B.hist, plane * sizeof(float) * lbm::kHist, cudaMemcpyDeviceToHost, h->stream));
    p += plane * sizeof(float) * lbm::kHist;
    LBM_CUDA(h, cudaMemcpyAsync(p, h->grain, plane, cudaMemcpyDeviceToHost, h->stream));
    p += plane;
    memcpy(p, h->grain_table.data(), 256 * sizeof(float2));
    LBM_CUDA(h, cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

int lbm_load_state(lbm_handle* h, const void* host, size_t bytes)
{
    if (!h) return LBM_EINVAL;
    if (!host || bytes != lbm_checkpoint_bytes(h)) return fail(h, LBM_EINVAL, "checkpoint size mismatch");
    const char* p = (const char*)host;
    CkptHeader hd;
    memcpy(&hd, p, sizeof(hd));
    if (memcmp(hd.magic, "LBMCKPT3", 8) != 0) return fail(h, LBM_EINVAL, "not a checkpoint of this layout");
    if (memcmp(&hd.prm, &h->prm, sizeof(lbm_params)) != 0) return fail(h, LBM_EINVAL, "checkpoint parameters differ");
    p += sizeof(hd);
    const size_t plane = (size_t)h->P.plane;
    const size_t sb = h->sc_bytes, fbz = h->fl_bytes;
    h->B.cs = 0;
    h->B.cf = 0;
    drop_graphs(h);
    LBM_CUDA(h, cudaMemcpyAsync(h->B.sc[0], p, sb, cudaMemcpyHostToDevice, h->stream));
    p += sb;
    LBM_CUDA(h, cudaMemcpyAsync(h->B.fl[0], p, fbz, cudaMemcpyHostToDevice, h->stream));
    p += fbz;
    LBM_CUDA(h, cudaMemcpyAsync(h->B.hist, p, plane * sizeof(float) * lbm::kHist, cudaMemcpyHostToDevice, h->stream));
    p += plane * sizeof(float) * lbm::kHist;
    LBM_CUDA(h, cudaMemcpyAsync(h->grain, p, plane, cudaMemcpyHostToDevice, h->stream));
    p += plane;
    h->grain_table.resize(256);
    memcpy(h->grain_table.data(), p, 256 * sizeof(float2));
    LBM_CUDA(h, cudaMemcpyAsync(h->grain_cs, h->grain_table.data(), 256 * sizeof(float2), cudaMemcpyHostToDevice,
                                h->stream));
    LBM_CUDA(h, cudaStreamSynchronize(h->stream));
    h->uniform = hd.uniform != 0;
    h->P.cos_o = h->grain_table[0].x;
    h->P.sin_o = h->grain_table[0].y;
    h->B.grain = h->uniform ? nullptr : h->grain;
    h->steps = hd.steps;
    h->initialised = true;
    prebuild_graph(h);
    return LBM_OK;
}

// ------------------------------------------------ device snapshots, surrogate
int lbm_snapshot_save(lbm_handle* h, int slot)
{
    int rc = ensure_initialised(h);
    if (rc) return rc;
    if (slot < 0 || slot > 1) return fail(h, LBM_EINVAL, "snapshot slot must be 0 or 1");
    const size_t hb = (size_t)h->P.plane * sizeof(float) * lbm::kHist;
    if (!h->snap_sc[slot]) {
        LBM_CUDA(h, cudaMalloc(&h->snap_sc[slot], h->sc_bytes));
        LBM_CUDA(h, cudaMalloc(&h->snap_fl[slot], h->fl_bytes));
        LBM_CUDA(h, cudaMalloc((void**)&h->snap_hist[slot], hb));
    }
    LBM_CUDA(h, cudaMemcpyAsync(h->snap_sc[slot], h->B.sc[h->B.cs], h->sc_bytes, cudaMemcpyDeviceToDevice, h->stream));
    LBM_CUDA(h, cudaMemcpyAsync(h->snap_fl[slot], h->B.fl[h->B.cf], h->fl_bytes, cudaMemcpyDeviceToDevice, h->stream));
    LBM_CUDA(h, cudaMemcpyAsync(h->snap_hist[slot], h->B.hist, hb, cudaMemcpyDeviceToDevice, h->stream));
    h->snap_steps[slot] = h->steps;
    return LBM_OK;
}

int lbm_snapshot_restore(lbm_handle* h, int slot)
{
    int rc = ensure_initialised(h);
    if (rc) return rc;
    if (slot < 0 || slot > 1) return fail(h, LBM_EINVAL, "snapshot slot must be 0 or 1");
    if (h->snap_steps[slot] < 0) return fail(h, LBM_ESTATE, "no snapshot in this slot");
    const size_t hb = (size_t)h->P.plane * sizeof(float) * lbm::kHist;
    LBM_CUDA(h, cudaMemcpyAsync(h->B.sc[h->B.cs], h->snap_sc[slot], h->sc_bytes, cudaMemcpyDeviceToDevice, h->stream));
    LBM_CUDA(h, cudaMemcpyAsync(h->B.fl[h->B.cf], h->snap_fl[slot], h->fl_bytes, cudaMemcpyDeviceToDevice, h->stream));
    LBM_CUDA(h, cudaMemcpyAsync(h->B.hist, h->snap_hist[slot], hb, cudaMemcpyDeviceToDevice, h->stream));
    h->steps = h->snap_steps[slot];
    return LBM_OK;
}

int lbm_fields_nhwc(lbm_handle* h, float* dst)
{
    int rc = ensure_initialised(h);
    if (rc) return rc;
    if (!dst) return fail(h, LBM_EINVAL, "dst is NULL");
    LBM_CUDA(h, lbm::launch_fields_nhwc(h->P, h->storage, h->B.sc[h->B.cs], h->B.fl[h->B.cf], (float)(1.0 / h->vf),
                                        dst, h->stream));
    return LBM_OK;
}

int lbm_set_fields_nhwc(lbm_handle* h, const float* src, const float* prev, int K)
{
    int rc = ensure_initialised(h);
    if (rc) return rc;
    if (!src) return fail(h, LBM_EINVAL, "src is NULL");
    if (prev && K < 1) return fail(h, LBM_EINVAL, "K must be >= 1 with prev");
    LBM_CUDA(h, lbm::launch_set_fields_nhwc(h->P, h->storage, src, (float)h->vf, h->B.sc[h->B.cs], h->B.fl[h->B.cf],
                                            h->B.hist, prev, K, h->stream));
    return LBM_OK;
}

namespace {

int tips_now(lbm_handle* h, double cx, double cy, double orient, double tip[3])
{
    lbm_metrics m;
    int rc = lbm_get_metrics(h, cx, cy, orient, &m);
    if (rc) return rc;
    for (int r = 0; r < 3; ++r) tip[r] = m.tip[r];
    return LBM_OK;
}

}  // namespace

int lbm_surrogate_advance(lbm_handle* h, lbm_unet* net, int K, double tip_tol, int audit, double cx, double cy,
                          double orient, lbm_surrogate_report* rep)
{
    trace::Range range("lbm_surrogate_advance");
    int rc = ensure_initialised(h);
    if (rc) return rc;
    if (!net || !rep || K < 1) return fail(h, LBM_EINVAL, "need a network, a report and K >= 1");
    int nb = 0, nh = 0, nw = 0, nf = 0;
    lbm_unet_shape(net, &nb, &nh, &nw, &nf);
    if (nb != 1 || nh != h->P.ny || nw != h->P.nx || nf != 5)
        return fail(h, LBM_EINVAL, "network must be sized for one ny x nx image of 5 fields");
    const size_t n5 = (size_t)h->P.nx * h->P.ny * 5;
    if (!h->sur_x) {
        LBM_CUDA(h, cudaMalloc((void**)&h->sur_x, n5 * sizeof(float)));
        LBM_CUDA(h, cudaMalloc((void**)&h->sur_y, n5 * sizeof(float)));
        LBM_CUDA(h, cudaMalloc((void**)&h->sur_l, n5 * sizeof(float)));
        LBM_CUDA(h, cudaMalloc((void**)&h->d_mis, 2 * sizeof(unsigned long long)));
    }
    memset(rep, 0, sizeof(*rep));
    if ((rc = lbm_unet_set_stream(net, h->stream))) return fail(h, rc, "lbm_unet_set_stream failed");
    if ((rc = lbm_fields_nhwc(h, h->sur_x))) return rc;
    if ((rc = lbm_unet_forward(net, h->sur_x, h->sur_y)))
        return fail(h, rc, std::string("network: ") + lbm_unet_last_error(net));
    if (!audit) {
        // a prediction that is not finite is not applied: the state stays at
        // the window's start and the report says so (the caller runs the
        // window with the LB)
        unsigned long long bad = 0;
        LBM_CUDA(h, lbm::launch_count_nonfinite(h->sur_y, (long long)n5, h->d_mis, h->stream));
        LBM_CUDA(h, cudaMemcpyAsync(&bad, h->d_mis, sizeof bad, cudaMemcpyDeviceToHost, h->stream));
        LBM_CUDA(h, cudaStreamSynchronize(h->stream));
        if (bad) {
            rep->tip_err = INFINITY;
            return LBM_OK;
        }
        if ((rc = lbm_set_fields_nhwc(h, h->sur_y, nullptr, 0))) return rc;
        h->steps += K;
        rep->accepted = 1;
        return LBM_OK;
    }
    // audit: the plain LB over the same window decides; its result is kept
    rep->audited = 1;
    if ((rc = lbm_step(h, K))) return rc;
    if ((rc = lbm_fields_nhwc(h, h->sur_l))) return rc;
    LBM_CUDA(h, lbm::launch_phi_mismatch(h->sur_y, h->sur_l, (long long)h->P.nx * h->P.ny, h->d_mis, h->stream));
    double tl[3], ts[3];
    if ((rc = tips_now(h, cx, cy, orient, tl))) return rc;
    if ((rc = lbm_snapshot_save(h, 1))) return rc;
    if ((rc = lbm_set_fields_nhwc(h, h->sur_y, nullptr, 0))) return rc;
    rc = tips_now(h, cx, cy, orient, ts);
    const int rr = lbm_snapshot_restore(h, 1);
    if (rc == LBM_ENUMERIC) {
        ts[0] = ts[1] = ts[2] = INFINITY;  // the prediction is not finite: reject it
        rc = LBM_OK;
    }
    if (rc) return rc;
    if (rr) return rr;
    unsigned long long mis[2];
    LBM_CUDA(h, cudaMemcpyAsync(mis, h->d_mis, sizeof mis, cudaMemcpyDeviceToHost, h->stream));
    LBM_CUDA(h, cudaStreamSynchronize(h->stream));
    double err = 0.0;
    for (int r = 0; r < 3; ++r) {
        rep->tip[r] = tl[r];
        const double d = fabs(ts[r] - tl[r]);
        err = (d > err || d != d) ? d : err;
    }
    rep->tip_err = err;
    rep->mismatch = (long long)mis[0];
    uint32_t bits = (uint32_t)mis[1];
    float mx;
    memcpy(&mx, &bits, sizeof mx);
    rep->max_dphi = mx;
    rep->accepted = err <= tip_tol ? 1 : 0;
    return LBM_OK;
}

int lbm_set_profiling(lbm_handle* h, int enable)
{
    if (!h) return LBM_EINVAL;
    int rc = collect_profile(h);
    if (rc) return rc;
    if (enable < 0 || enable > 2) return fail(h, LBM_EINVAL, "profiling mode must be 0, 1 or 2");
    if (enable == 2 && h->prm.n_sub < 2) return fail(h, LBM_EINVAL, "no flow sub-steps to time (n_sub = 1)");
    h->profiling = enable != 0;
    h->prof_substeps = enable == 2;
    h->prof_ms = 0.0;
    h->prof_launches = 0;
    return LBM_OK;
}

int lbm_kernel_time(lbm_handle* h, double* total_ms, long long* launches)
{
    if (!h || !total_ms || !launches) return LBM_EINVAL;
    int rc = collect_profile(h);
    if (rc) return rc;
    *total_ms = h->prof_ms;
    *launches = h->prof_launches;
    return LBM_OK;
}

const char* lbm_last_error(const lbm_handle* h) { return h ? h->err.c_str() : g_create_error.c_str(); }

const char* lbm_version(void) { return "lbm-gb300 0.1 (sm_103a)"; }

}  // extern "C"

namespace lbm {

// Lattice-unit parameters of a problem statement without creating a handle
// (the temporary handle below holds no heap or device memory).
int params_to_step(const lbm_params* p, StepParams* out, const char** why)
{
    static thread_local std::string msg;
    msg = validate(p);
    if (!msg.empty()) {
        *why = msg.c_str();
        return LBM_EINVAL;
    }
    lbm_handle tmp;
    tmp.prm = *p;
    derive(&tmp);
    *out = tmp.P;
    return LBM_OK;
}

// Message returned by lbm_last_error(NULL) for calls that take no handle.
void set_last_error(const char* msg) { g_create_error = msg; }

}  // namespace lbm

// ===================================================================== batch
// Many independent domains (their own sizes and parameters, one storage type,
// n_sub = 1) advanced together: each domain keeps the buffers of a
// single-domain handle; one persistent kernel per step sweeps the tiles of all
// of them, batched wall kernels follow, and 16-step sequences replay from
// captured CUDA graphs.

struct lbm_batch {
    std::vector<lbm_handle*> dom;
    int storage = 0;
    int parity = 0;          // buffer index holding the newest populations of every domain
    int ty = 8;              // tile height of the batched kernel
    int run = 1;             // tiles per CTA (0: persistent grid)
    int ctas[3] = {0, 0, 0}; // resident CTAs for tile heights 4, 8, 16
    cudaStream_t stream = nullptr;
    lbm::DomainDesc* d_descs = nullptr;
    int4* d_tiles[3] = {nullptr, nullptr, nullptr};
    int ntiles[3] = {0, 0, 0};
    int4* d_walls[2] = {nullptr, nullptr};
    int nwall[2] = {0, 0};
    std::map<std::pair<int, int>, cudaGraphExec_t> graphs;  // (parity, ty * 1000 + run)
    long long steps = 0, nodes = 0;
    std::string err;
    // kernel timing (lbm_batch_set_profiling): begin/end pairs of pending launches
    bool profiling = false;
    std::vector<cudaEvent_t> ev;
    size_t ev_used = 0;
    double prof_ms = 0.0;
    long long prof_launches = 0;
};

namespace {

thread_local std::string g_batch_error;

int bfail(lbm_batch* b, int code, const std::string& msg)
{
    if (b)
        b->err = msg;
    else
        g_batch_error = msg;
    return code;
}

#define LBM_BCUDA(b, call)                                                              \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) return bfail(b, LBM_ECUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
    } while (0)

int tyk(int ty) { return ty == 4 ? 0 : ty == 8 ? 1 : 2; }

void drop_batch_graphs(lbm_batch* b)
{
    for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
    b->graphs.clear();
}

lbm::BatchTables tables(const lbm_batch* b)
{
    lbm::BatchTables T;
    T.descs = b->d_descs;
    T.ndomains = (int)b->dom.size();
    for (int k = 0; k < 3; ++k) {
        T.tiles[k] = b->d_tiles[k];
        T.ntiles[k] = b->ntiles[k];
    }
    for (int k = 0; k < 2; ++k) {
        T.walls[k] = b->d_walls[k];
        T.nwall[k] = b->nwall[k];
    }
    return T;
}

// Descriptor table from the domains' current parameters and buffers.
int upload_descs(lbm_batch* b)
{
    std::vector<lbm::DomainDesc> d(b->dom.size());
    for (size_t i = 0; i < b->dom.size(); ++i) {
        lbm_handle* h = b->dom[i];
        d[i].P = h->P;
        for (int k = 0; k < 2; ++k) {
            d[i].sc[k] = h->B.sc[k];
            d[i].fl[k] = h->B.fl[k];
        }
        d[i].hist = h->B.hist;
        d[i].grain = h->B.grain;
    }
    LBM_BCUDA(b, cudaMemcpyAsync(b->d_descs, d.data(), d.size() * sizeof(lbm::DomainDesc), cudaMemcpyHostToDevice,
                                 b->stream));
    LBM_BCUDA(b, cudaStreamSynchronize(b->stream));
    drop_batch_graphs(b);
    return LBM_OK;
}

int batch_graph(lbm_batch* b, cudaGraphExec_t* out)
{
    const auto key = std::make_pair(b->parity, b->ty * 1000 + b->run);
    auto it = b->graphs.find(key);
    if (it != b->graphs.end()) {
        *out = it->second;
        return LBM_OK;
    }
    cudaStream_t cap;
    LBM_BCUDA(b, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    const lbm::BatchTables T = tables(b);
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    int par = b->parity;
    for (int i = 0; i < kGraphSteps && e == cudaSuccess; ++i) {
        // left/right walls as in the single-domain graphs
        e = lbm::launch_batch_step(T, b->storage, b->ty, b->run, par, b->ctas[tyk(b->ty)], cap, i > 0,
                                   i + 1 < kGraphSteps);
        par = 1 - par;
    }
    cudaError_t e2 = cudaStreamEndCapture(cap, &g);
    if (e == cudaSuccess) e = e2;
    cudaStreamDestroy(cap);
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return bfail(b, LBM_ECUDA, std::string("batch graph capture: ") + cudaGetErrorString(e));
    }
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return bfail(b, LBM_ECUDA, std::string("batch graph instantiate: ") + cudaGetErrorString(e));
    b->graphs[key] = ex;
    *out = ex;
    return LBM_OK;
}

int batch_ready(lbm_batch* b)
{
    if (!b) return LBM_EINVAL;
    for (lbm_handle* h : b->dom)
        if (!h->initialised) return bfail(b, LBM_ESTATE, "every domain must be initialised before stepping");
    return LBM_OK;
}

int batch_collect_profile(lbm_batch* b)
{
    if (!b->ev_used) return LBM_OK;
    LBM_BCUDA(b, cudaEventSynchronize(b->ev[b->ev_used - 1]));
    for (size_t i = 0; i + 1 < b->ev_used; i += 2) {
        float ms = 0.0f;
        LBM_BCUDA(b, cudaEventElapsedTime(&ms, b->ev[i], b->ev[i + 1]));
        b->prof_ms += ms;
        b->prof_launches += 1;
    }
    b->ev_used = 0;
    return LBM_OK;
}

int batch_run_direct(lbm_batch* b, int n)
{
    lbm::BatchTables T = tables(b);
    for (int i = 0; i < n; ++i) {
        if (b->profiling) {
            if (b->ev_used + 2 > b->ev.size()) {
                int rc = batch_collect_profile(b);
                if (rc) return rc;
                while (b->ev.size() < 512) {
                    cudaEvent_t e;
                    LBM_BCUDA(b, cudaEventCreate(&e));
                    b->ev.push_back(e);
                }
            }
            T.ev_begin = b->ev[b->ev_used++];
            T.ev_end = b->ev[b->ev_used++];
        }
        LBM_BCUDA(b, lbm::launch_batch_step(T, b->storage, b->ty, b->run, b->parity, b->ctas[tyk(b->ty)], b->stream));
        b->parity = 1 - b->parity;
    }
    return LBM_OK;
}

void sync_domain_parity(lbm_batch* b)
{
    for (lbm_handle* h : b->dom) {
        h->B.cs = b->parity;
        h->B.cf = b->parity;
        h->steps = b->steps;
    }
}

}  // namespace

extern "C" {

int lbm_batch_create(const lbm_params* params, int n, lbm_batch** out)
{
    if (!out) return bfail(nullptr, LBM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!params || n < 1) return bfail(nullptr, LBM_EINVAL, "need at least one domain");
    if (n > lbm::kMaxBatchDomains) return bfail(nullptr, LBM_EINVAL, "at most 256 domains per batch");
    for (int i = 0; i < n; ++i) {
        if (params[i].storage != params[0].storage) return bfail(nullptr, LBM_EINVAL, "domains must share one storage");
        if (params[i].n_sub != 1) return bfail(nullptr, LBM_EINVAL, "batched domains need n_sub = 1");
    }
    lbm_batch* b = new (std::nothrow) lbm_batch();
    if (!b) return bfail(nullptr, LBM_ENOMEM, "host allocation failed");
    b->storage = params[0].storage;
    for (int i = 0; i < n; ++i) {
        lbm_handle* h = nullptr;
        int rc = lbm_create(&params[i], &h);
        if (rc != LBM_OK) {
            std::string why = "domain " + std::to_string(i) + ": " + lbm_last_error(nullptr);
            lbm_batch_destroy(b);
            return bfail(nullptr, rc, why);
        }
        b->dom.push_back(h);
        b->nodes += (long long)params[i].nx * params[i].ny;
    }
    // tile tables for each tile height, domain-major
    const int tys[3] = {4, 8, 16};
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
        std::vector<int4> t;
        for (int i = 0; i < n; ++i)
            for (int y0 = 0; y0 < params[i].ny; y0 += tys[k])
                for (int x0 = 0; x0 < params[i].nx; x0 += lbm::TX) t.push_back(make_int4(i, x0, y0, 0));
        b->ntiles[k] = (int)t.size();
        e = cudaMalloc(&b->d_tiles[k], t.size() * sizeof(int4));
        if (e == cudaSuccess) e = cudaMemcpy(b->d_tiles[k], t.data(), t.size() * sizeof(int4), cudaMemcpyHostToDevice);
    }
    // wall lists: y walls (axis 1) and x walls (axis 0), same node sets as the single-domain walls
    std::vector<int4> w[2];
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        const lbm_params& p = params[i];
        const bool px = p.bc[0] == LBM_BC_PERIODIC, py = p.bc[2] == LBM_BC_PERIODIC;
        if (!py) {
            const int lo = px ? 0 : 1, hi = px ? p.nx - 1 : p.nx - 2;
            for (int which = 0; which < 2; ++which)
                for (int j = lo; j <= hi; ++j) w[0].push_back(make_int4(i, 1, which, j));
        }
        if (!px)
            for (int which = 0; which < 2; ++which)
                for (int j = 0; j < p.ny; ++j) w[1].push_back(make_int4(i, 0, which, j));
    }
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        b->nwall[k] = (int)w[k].size();
        if (w[k].empty()) continue;
        e = cudaMalloc(&b->d_walls[k], w[k].size() * sizeof(int4));
        if (e == cudaSuccess)
            e = cudaMemcpy(b->d_walls[k], w[k].data(), w[k].size() * sizeof(int4), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMalloc(&b->d_descs, n * sizeof(lbm::DomainDesc));
    if (e != cudaSuccess) {
        std::string why = std::string("batch tables: ") + cudaGetErrorString(e);
        lbm_batch_destroy(b);
        return bfail(nullptr, LBM_ECUDA, why);
    }
    for (int k = 0; k < 3; ++k) b->ctas[k] = lbm::batch_resident_ctas(b->storage, tys[k]);
    *out = b;
    return upload_descs(b);
}

void lbm_batch_destroy(lbm_batch* b)
{
    if (!b) return;
    drop_batch_graphs(b);
    for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
    for (lbm_handle* h : b->dom) lbm_destroy(h);
    for (int k = 0; k < 3; ++k)
        if (b->d_tiles[k]) cudaFree(b->d_tiles[k]);
    for (int k = 0; k < 2; ++k)
        if (b->d_walls[k]) cudaFree(b->d_walls[k]);
    if (b->d_descs) cudaFree(b->d_descs);
    delete b;
}

int lbm_batch_set_stream(lbm_batch* b, void* stream)
{
    if (!b) return LBM_EINVAL;
    b->stream = (cudaStream_t)stream;
    for (lbm_handle* h : b->dom) h->stream = b->stream;
    return LBM_OK;
}

int lbm_batch_init_seeds(lbm_batch* b, int dom, const lbm_seed* seeds, int n, double U0, double theta0)
{
    if (!b) return LBM_EINVAL;
    if (dom < 0 || dom >= (int)b->dom.size()) return bfail(b, LBM_EINVAL, "domain index out of range");
    lbm_handle* h = b->dom[dom];
    int rc = lbm_init_seeds(h, seeds, n, U0, theta0);
    if (rc) return bfail(b, rc, h->err);
    // the handle initialised buffer 0; the batch may be at the other parity
    if (b->parity == 1) {
        LBM_BCUDA(b, cudaMemcpyAsync(h->B.sc[1], h->B.sc[0], h->sc_bytes, cudaMemcpyDeviceToDevice, b->stream));
        LBM_BCUDA(b, cudaMemcpyAsync(h->B.fl[1], h->B.fl[0], h->fl_bytes, cudaMemcpyDeviceToDevice, b->stream));
    }
    h->B.cs = h->B.cf = b->parity;
    return upload_descs(b);
}

int lbm_batch_step(lbm_batch* b, int nsteps)
{
    trace::Range range("lbm_batch_step");
    int rc = batch_ready(b);
    if (rc) return rc;
    if (nsteps < 0) return bfail(b, LBM_EINVAL, "nsteps < 0");
    int left = nsteps;
    while (!b->profiling && left >= kGraphSteps) {
        cudaGraphExec_t ex;
        if ((rc = batch_graph(b, &ex))) return rc;
        LBM_BCUDA(b, cudaGraphLaunch(ex, b->stream));
        left -= kGraphSteps;  // even: the parity is unchanged
    }
    if ((rc = batch_run_direct(b, left))) return rc;
    b->steps += nsteps;
    sync_domain_parity(b);
    return LBM_OK;
}

int lbm_batch_set_profiling(lbm_batch* b, int enable)
{
    if (!b) return LBM_EINVAL;
    int rc = batch_collect_profile(b);
    if (rc) return rc;
    b->profiling = enable != 0;
    b->prof_ms = 0.0;
    b->prof_launches = 0;
    return LBM_OK;
}

int lbm_batch_kernel_time(lbm_batch* b, double* total_ms, long long* launches)
{
    if (!b || !total_ms || !launches) return LBM_EINVAL;
    int rc = batch_collect_profile(b);
    if (rc) return rc;
    *total_ms = b->prof_ms;
    *launches = b->prof_launches;
    return LBM_OK;
}

int lbm_batch_synchronize(lbm_batch* b)
{
    if (!b) return LBM_EINVAL;
    LBM_BCUDA(b, cudaStreamSynchronize(b->stream));
    return LBM_OK;
}

int lbm_batch_get_fields(lbm_batch* b, int dom, unsigned mask, double* out)
{
    if (!b) return LBM_EINVAL;
    if (dom < 0 || dom >= (int)b->dom.size()) return bfail(b, LBM_EINVAL, "domain index out of range");
    int rc = lbm_get_fields(b->dom[dom], mask, out);
    return rc ? bfail(b, rc, b->dom[dom]->err) : LBM_OK;
}

int lbm_batch_fields_nhwc(lbm_batch* b, int dom, float* dst)
{
    if (!b) return LBM_EINVAL;
    if (dom < 0 || dom >= (int)b->dom.size()) return bfail(b, LBM_EINVAL, "domain index out of range");
    int rc = lbm_fields_nhwc(b->dom[dom], dst);
    return rc ? bfail(b, rc, b->dom[dom]->err) : LBM_OK;
}

int lbm_batch_get_metrics(lbm_batch* b, int dom, double cx, double cy, double orient, lbm_metrics* m)
{
    if (!b) return LBM_EINVAL;
    if (dom < 0 || dom >= (int)b->dom.size()) return bfail(b, LBM_EINVAL, "domain index out of range");
    int rc = lbm_get_metrics(b->dom[dom], cx, cy, orient, m);
    return rc ? bfail(b, rc, b->dom[dom]->err) : LBM_OK;
}

long long lbm_batch_nodes(const lbm_batch* b) { return b ? b->nodes : -1; }

int lbm_batch_tile_height(const lbm_batch* b) { return b ? b->ty : -1; }

int lbm_batch_tiles_per_cta(const lbm_batch* b) { return b ? b->run : -1; }

int lbm_batch_set_tiling(lbm_batch* b, int tile_height, int tiles_per_cta)
{
    if (!b) return LBM_EINVAL;
    if (tile_height != 4 && tile_height != 8 && tile_height != 16)
        return bfail(b, LBM_EINVAL, "tile height must be 4, 8 or 16");
    if (tiles_per_cta < 0) return bfail(b, LBM_EINVAL, "tiles per CTA must be >= 0");
    b->ty = tile_height;
    b->run = tiles_per_cta;
    return LBM_OK;
}

int lbm_batch_tune(lbm_batch* b, const char* cache_path, int* tile_height)
{
    int rc = batch_ready(b);
    if (rc) return rc;
    cudaDeviceProp prop;
    int dev = 0;
    LBM_BCUDA(b, cudaGetDevice(&dev));
    LBM_BCUDA(b, cudaGetDeviceProperties(&prop, dev));
    // size class: total nodes to two significant digits
    long long cls = b->nodes;
    long long scale = 1;
    while (cls >= 100) {
        cls /= 10;
        scale *= 10;
    }
    char key[512];  // the device name (up to 256 characters) and the batch's class
    snprintf(key, sizeof(key), "%s|storage%d|nodes%lld|domains%zu", prop.name, b->storage, cls * scale, b->dom.size());
    for (char* c = key; *c; ++c)
        if (*c == ' ') *c = '_';
    if (cache_path) {
        if (FILE* f = fopen(cache_path, "r")) {
            char k[512];
            int v, r;
            while (fscanf(f, "%511s %d %d", k, &v, &r) == 3)
                if (strcmp(k, key) == 0 && (v == 4 || v == 8 || v == 16) && r >= 0) {
                    b->ty = v;
                    b->run = r;
                    fclose(f);
                    if (tile_height) *tile_height = v;
                    return LBM_OK;
                }
            fclose(f);
        }
    }
    // time each tile height on a snapshot of the state, then restore it
    std::vector<void*> backup;
    for (lbm_handle* h : b->dom) {
        void* p = nullptr;
        cudaError_t e = cudaMalloc(&p, h->sc_bytes + h->fl_bytes + (size_t)h->P.plane * sizeof(float) * lbm::kHist);
        if (e != cudaSuccess) {
            for (void* q : backup) cudaFree(q);
            return bfail(b, LBM_ENOMEM, "no device memory for the tuning snapshot");
        }
        char* c = (char*)p;
        cudaMemcpyAsync(c, h->B.sc[b->parity], h->sc_bytes, cudaMemcpyDeviceToDevice, b->stream);
        cudaMemcpyAsync(c + h->sc_bytes, h->B.fl[b->parity], h->fl_bytes, cudaMemcpyDeviceToDevice, b->stream);
        cudaMemcpyAsync(c + h->sc_bytes + h->fl_bytes, h->B.hist, (size_t)h->P.plane * sizeof(float) * lbm::kHist,
                        cudaMemcpyDeviceToDevice, b->stream);
        backup.push_back(p);
    }
    const int start_parity = b->parity;
    const int tys[3] = {4, 8, 16};
    const int runs[3] = {1, 4, 0};
    float best_ms = 1e30f;
    int best = b->ty, best_run = b->run;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const lbm::BatchTables T = tables(b);
    for (int k = 0; k < 3; ++k)
        for (int r = 0; r < 3; ++r) {
            // steps as inside the captured graphs: left/right walls updated at
            // the next step's load (the state is restored below)
            int par = start_parity;
            for (int i = 0; i < 2; ++i, par = 1 - par)
                lbm::launch_batch_step(T, b->storage, tys[k], runs[r], par, b->ctas[k], b->stream, i > 0, 1);
            cudaEventRecord(e0, b->stream);
            for (int i = 0; i < 10; ++i, par = 1 - par)
                lbm::launch_batch_step(T, b->storage, tys[k], runs[r], par, b->ctas[k], b->stream, 1, 1);
            cudaEventRecord(e1, b->stream);
            cudaEventSynchronize(e1);
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best_ms) {
                best_ms = ms;
                best = tys[k];
                best_run = runs[r];
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (size_t i = 0; i < b->dom.size(); ++i) {
        lbm_handle* h = b->dom[i];
        char* c = (char*)backup[i];
        cudaMemcpyAsync(h->B.sc[start_parity], c, h->sc_bytes, cudaMemcpyDeviceToDevice, b->stream);
        cudaMemcpyAsync(h->B.fl[start_parity], c + h->sc_bytes, h->fl_bytes, cudaMemcpyDeviceToDevice, b->stream);
        cudaMemcpyAsync(h->B.hist, c + h->sc_bytes + h->fl_bytes, (size_t)h->P.plane * sizeof(float) * lbm::kHist,
                        cudaMemcpyDeviceToDevice, b->stream);
    }
    cudaError_t e = cudaStreamSynchronize(b->stream);
    for (void* q : backup) cudaFree(q);
    if (e != cudaSuccess) return bfail(b, LBM_ECUDA, std::string("tuning: ") + cudaGetErrorString(e));
    e = cudaGetLastError();
    if (e != cudaSuccess) return bfail(b, LBM_ECUDA, std::string("tuning: ") + cudaGetErrorString(e));
    b->parity = start_parity;
    b->ty = best;
    b->run = best_run;
    drop_batch_graphs(b);
    if (cache_path)
        if (FILE* f = fopen(cache_path, "a")) {
            fprintf(f, "%s %d %d\n", key, best, best_run);
            fclose(f);
        }
    if (tile_height) *tile_height = best;
    return LBM_OK;
}

const char* lbm_batch_last_error(const lbm_batch* b) { return b ? b->err.c_str() : g_batch_error.c_str(); }

}  // extern "C"
