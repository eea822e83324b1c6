// Host-side declarations of the kernel launchers shared by the C-ABI
// translation unit and the kernel translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lbm.h"
#include "lbm_device.cuh"

namespace lbm {

// Storage kinds (same values as LBM_FP32/LBM_FP16/LBM_BF16).
enum Storage { kStoreF32 = 0, kStoreF16 = 1, kStoreBF16 = 2 };

// Bytes per node of the scalar and flow population buffers (see the codecs in
// lbm_device.cuh: 16-bit storage keeps the three scalar rest planes in FP32).
inline size_t scalar_node_bytes(int storage) { return storage == kStoreF32 ? 15 * 4 : 12 * 2 + 3 * 4; }
inline size_t flow_node_bytes(int storage) { return storage == kStoreF32 ? 9 * 4 : 9 * 2; }

// One coupled step (Sec. 3 + Sec. 4): the fused kernel, the wall kernels and
// the n_sub - 1 flow-only sub-steps; on return cs/cf name the newest buffers.
struct StepBuffers {
    void* sc[2];           // scalar populations (phi, C, H): planes 0..14, node blocks
    void* fl[2];           // flow populations: planes 15..23, node blocks
    float* hist;           // kHist planes, node blocks
    float* fb;             // force plane for flow sub-steps (n_sub > 1) or null
    const uint8_t* grain;  // grain id plane or null (uniform orientation)
    int cs, cf;            // indices of the buffers holding the newest populations
    cudaEvent_t ev_begin = nullptr, ev_end = nullptr;  // recorded around the timed kernels when set
    int ev_substeps = 0;   // 0: the events bracket the fused kernel; 1: the n_sub - 1 flow sub-step kernels
};

// One coupled step.  skip_columns: leave out the column pass of the left/right
// walls (n_sub = 1 and walls in x; ignored otherwise);
// the next step must then be launched with `repair`, which applies that
// update to the wall cells as they are loaded.  A state read or kept between
// launches must come from a step without skip_columns.
cudaError_t launch_coupled_step(const StepParams& P, int storage, int n_sub, StepBuffers& B, cudaStream_t s,
                                int repair = 0, int skip_columns = 0);

// One domain of a batch as the batched kernels see it: its parameters and the
// two parities of its population buffers (n_sub = 1).
struct DomainDesc {
    StepParams P;
    void* sc[2];
    void* fl[2];
    float* hist;
    const uint8_t* grain;  // null when the domain is one grain
};

// Device tables of a batch: tiles {domain, x0, y0, 0} for tile heights 4, 8,
// 16 (index 0, 1, 2), wall nodes {domain, axis, side, index} for the y walls
// (0) and the x walls (1).
// Domains per batch: the batched kernel reads its descriptors from constant
// memory (64 KiB).
constexpr int kMaxBatchDomains = 256;

struct BatchTables {
    const DomainDesc* descs;  // device copy, loaded into constant memory before each step
    int ndomains;
    const int4* tiles[3];
    int ntiles[3];
    const int4* walls[2];
    int nwall[2];
    cudaEvent_t ev_begin = nullptr, ev_end = nullptr;  // recorded around the batched kernel when set
};

// One coupled step of every domain: buffers `parity` -> 1 - parity, then walls.
// ty: tile height 4, 8 or 16; run: tiles per CTA (0: persistent grid of
// `ctas` CTAs, each taking one contiguous run).  repair, skip_columns: as for
// launch_coupled_step.
cudaError_t launch_batch_step(const BatchTables& T, int storage, int ty, int run, int parity, int ctas,
                              cudaStream_t s, int repair = 0, int skip_columns = 0);
// CTAs of the persistent batched kernel that fit on the current device at once.
int batch_resident_ctas(int storage, int ty);

// Row bands: the whole-grid transfers below work on the rows [y0, y0 + rows)
// and keep their planes in a band buffer, rows * pitch elements per plane,
// node (x, y) at (y - y0) * pitch + x.

// Initialisation of a band: equilibrium populations from lattice-unit macros
// (phi, U, theta, ux, uy, p) in FP64 band planes, then history = time-0 macros.
cudaError_t launch_init_from_fields(const StepParams& P, int storage, const double* fields, void* sc, void* fl,
                                    float* hist, int y0, int rows, cudaStream_t s);

// Seeded initial fields of a band: phi, U = U0, theta = theta0 (FP64 band
// planes) and the grain ids (the whole grid's plane).
cudaError_t launch_seed_fields(const StepParams& P, const double* seeds, int ns, double U0, double theta0,
                               double W, double* fields, uint8_t* grain, int y0, int rows, cudaStream_t s);

// Fields of every node pixel-interleaved for the network (FP32 NHWC), and back.
cudaError_t launch_fields_nhwc(const StepParams& P, int storage, const void* sc, const void* fl, float inv_vf,
                               float* dst, cudaStream_t s);
cudaError_t launch_set_fields_nhwc(const StepParams& P, int storage, const float* src, float vf, void* sc, void* fl,
                                   float* hist, const float* prev, int K, cudaStream_t s);
cudaError_t launch_force(const StepParams& P, int storage, const void* sc, const void* fl, double cx, double cy,
                         double* partials, double* out, cudaStream_t st);
cudaError_t launch_flow_inputs(const StepParams& P, int storage, const void* sc, const void* fl, float* phi, float* fy,
                               cudaStream_t st);
// n flow-only steps (collide + stream h, flow walls) with frozen phi and F_y;
// *cf is the flow buffer parity, updated.
cudaError_t flow_steps(const StepParams& P, int storage, int n, void* sc, void* const fl[2], int* cf, const float* phi,
                       const float* fy, cudaStream_t s);
cudaError_t launch_phi_mismatch(const float* a, const float* b, long long n, unsigned long long* out, cudaStream_t s);
// out[0] = the number of values of a[0 .. n) that are not finite (queued on s).
cudaError_t launch_count_nonfinite(const float* a, long long n, unsigned long long* out, cudaStream_t s);
// Macros of a band (FP32 band planes phi + 1, C - 1, U, theta - theta_ref,
// ux, uy, p; lattice units).
cudaError_t launch_macros(const StepParams& P, int storage, const void* sc, const void* fl, float* out, int y0,
                          int rows, cudaStream_t s);
// Fields of a band in their final FP32 form: field k (of n) is the macro
// plane sel[k] of launch_macros times scale[k] plus offset[k], written at
// out + k * rows * nx in rows of nx values.
struct FieldsF32 {
    int n;
    int sel[7];
    float scale[7], offset[7];
};
cudaError_t launch_fields_f32(const StepParams& P, int storage, const void* sc, const void* fl,
                              const FieldsF32& spec, float* out, int y0, int rows, cudaStream_t s);

// Decode a band's populations and history to FP32 band planes (24
// population deviations, then the kHist history values) / encode them back.
cudaError_t launch_decode(const StepParams& P, int storage, const void* sc, const void* fl, const float* hist,
                          float* out, int y0, int rows, cudaStream_t s);
cudaError_t launch_encode(const StepParams& P, int storage, const float* in, void* sc, void* fl, float* hist, int y0,
                          int rows, cudaStream_t s);

// Metrics reductions (FP64 results): out[0..6] = solid fraction sum, sum C, sum H, sum h,
// max |u| (flow lattice units), non-finite count, sum phi; then out[7..9] =
// the three tip distances.  `partials` must hold reduce_partials_size()
// doubles.
int reduce_blocks(const StepParams& P);
size_t reduce_partials_size(const StepParams& P);
cudaError_t launch_reduce(const StepParams& P, int storage, const void* sc, const void* fl, double cx, double cy,
                          double c, double s, double* partials, double* out, cudaStream_t st);

// Building blocks of the reduction, for callers that bring their own partials:
// fold `nblocks` rows of 7 partials into out[0..6]; tips into out[7..9].
cudaError_t launch_reduce_final(const double* partials, int nblocks, double* out, cudaStream_t st);
cudaError_t launch_tips(const StepParams& P, int storage, const void* sc, double cx, double cy, double c, double s,
                        double* out, cudaStream_t st);

// Validation and lattice-unit conversion of lbm_create, for calls without a
// handle; *why receives the reason on LBM_EINVAL.
int params_to_step(const lbm_params* p, StepParams* out, const char** why);
void set_last_error(const char* msg);

}  // namespace lbm
