// The surrogate network as one object: a convolutional U-Net over NHWC BF16
// activations whose forward, backward and Adam update are sequences of the
// tensor-core GEMM (nn_gemm.cu) and the layer kernels (nn_layers.cu) on one
// stream.  The host code here only plans buffers and issues launches.
//
// Network (levels L, base width w, level l has c_l = w * 2^l channels):
//   encoder l = 0 .. L-1: a_l = relu(conv3x3(in_l)), s_l = relu(conv3x3(a_l)),
//     in_{l+1} = maxpool2x2(s_l);
//   decoder l = L-2 .. 0: u_l = upconv2x2(h_{l+1}) (h_{L-1} = s_{L-1},
//     otherwise the decoder output d_{l+1}), cat_l = [s_l, u_l],
//     d_l = relu(conv3x3(relu(conv3x3(cat_l))));
//   output: the K-step increment proj1x1(d_0) in output units, so that the
//   prediction is y = x + std_out * proj1x1(d_0), with the inputs normalised
//   as (x - mean) / std_in.
// A 3 x 3 convolution is an im2col gather followed by a GEMM with the bias and
// ReLU in its epilogue; its input gradient is the same gather of the output
// gradient times the 180-degree-rotated kernel; its weight gradient is a
// split-K GEMM over all pixels.  s_l is written straight into the first half
// of the concatenation buffer cat_l and u_l into the second half, so the
// concatenation costs nothing.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "lbm.h"
#include "nn_kernels.h"
#include "nn_layers.h"
#include "trace.h"

namespace {

using bf16 = __nv_bfloat16;

constexpr int kInPitch = 8;   // input channels the first convolution's weights see (fields, zero padded)
constexpr int kX0Pitch = 32;  // stored input pitch: the first convolution runs as a 32-channel implicit one
constexpr int kPartBlocks = 1024;

struct Conv {
    int cin = 0, cout = 0;
    long long w = 0, b = 0;  // offsets in the padded parameter vector
    bf16* wf = nullptr;      // [cin][9 cout] rotated kernel for the input gradient
    bf16* wpad = nullptr;    // [cout][9 cin_pad] kernel with zero channels (first convolution only)
    int cin_pad = 0;
};

struct Up {
    int cin = 0, cout = 0;  // cin = 2 cout
    long long w = 0, b = 0;
    bf16* wt = nullptr;  // [cin][4 cout] transpose for the input gradient
};

struct Level {
    int c = 0, H = 0, W = 0;
    long long P = 0;
    Conv ea, eb, da, db;
    Up up;
    bf16* a = nullptr;     // [P][c]
    bf16* s = nullptr;     // cat_l [P][2c] (s in the first half) or, at the bottom, [P][c]
    int spitch = 0;
    bf16* pool = nullptr;  // [P/4][c]
    bf16* dA = nullptr;    // decoder activations [P][c]
    bf16* dD = nullptr;
    float* dcat = nullptr;  // gradient of cat_l, FP32 [P][2c]
};

struct Tensor {
    long long packed, padded, n;
};

long long round_up(long long x, long long m) { return (x + m - 1) / m * m; }

}  // namespace

struct lbm_unet {
    int L = 0, base = 0, F = 0, B = 0, H = 0, W = 0;
    long long P0 = 0;
    std::vector<Tensor> tensors;  // in the order of the network definition
    long long n_packed = 0, n_padded = 0;
    long long out_w = 0, out_b = 0;
    std::vector<Level> lv;
    float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
    bf16* wb = nullptr;
    int t = 0;
    float *mean = nullptr, *inv_std = nullptr, *inv_out = nullptr;
    float iface_w = 0.0f;  // interface weight of the loss (lbm_unet_set_loss_weight)
    std::vector<float> norm_h;  // host copy: mean, std_in, std_out (F each)
    bf16* x0 = nullptr;
    float *Y = nullptr, *T = nullptr, *G = nullptr;
    float *loss = nullptr, *part = nullptr;
    bf16 *col = nullptr, *colT = nullptr, *tA = nullptr, *tB = nullptr;
    bf16 *gA = nullptr, *gB = nullptr, *dU = nullptr;
    float* g32 = nullptr;
    float* ws = nullptr;
    long long ws_n = 0;
    nn::FlipJob* flip_jobs = nullptr;  // device table of the kernel flips (derive)
    int n_flip = 0;
    long long flip_total = 0;
    cudaStream_t s = nullptr;
    std::vector<void*> allocs;
    long long bytes = 0;
    std::string err;
};

namespace {

int fail(lbm_unet* u, int code, const std::string& what)
{
    if (u) u->err = what;
    return code;
}

int cuda_fail(lbm_unet* u, cudaError_t e, const char* where)
{
    return fail(u, LBM_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define UN_CHECK(u, call)                                           \
    do {                                                            \
        cudaError_t e_ = (call);                                    \
        if (e_ != cudaSuccess) return cuda_fail((u), e_, #call);    \
    } while (0)

template <class T>
cudaError_t alloc(lbm_unet* u, T** p, long long n)
{
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, (size_t)std::max<long long>(n, 1) * sizeof(T));
    if (e != cudaSuccess) return e;
    u->allocs.push_back(q);
    u->bytes += std::max<long long>(n, 1) * (long long)sizeof(T);
    *p = (T*)q;
    return cudaMemset(q, 0, (size_t)std::max<long long>(n, 1) * sizeof(T));
}

// Streaming multiprocessors of the current device (152 on a GB300).
int sm_count()
{
    static int n = 0;
    if (n == 0) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
            n = v;
        else
            return 152;
    }
    return n;
}

// K slices so that the weight-gradient GEMM runs as one wave of CTAs (one
// per SM for wide tiles, two for tiles up to 64 columns, which the split-K
// kernel runs two to an SM), each with the longest K loop that allows:
// measured on the U-Net's shapes, one wave takes 10 to 30 % less time than
// two, whose partial tiles are twice as many to write and add, and whose last
// CTAs often start a third, nearly empty wave.
int splits_for(int M, int N, long long K)
{
    const int bn = N >= 256 ? 256 : N > 64 ? 128 : N > 32 ? 64 : 32;
    const long long tiles = (long long)((M + 127) / 128) * ((N + bn - 1) / bn);
    const long long nkb = (K + 63) / 64;
    // narrow tiles run two CTAs per SM (the split-K kernel's shallower ring)
    long long sp = (bn <= 64 ? 2 : 1) * sm_count() / tiles;
    sp = std::min<long long>(sp, nkb);
    sp = std::min<long long>(sp, 256);
    return (int)std::max<long long>(sp, 1);
}

long long split_ws(int M, int N, long long K) { return (long long)splits_for(M, N, K) * M * N; }

// The planned shapes and offsets, before any allocation.
void plan(lbm_unet* u)
{
    long long packed = 0, padded = 0;
    auto add = [&](long long n) {
        Tensor t{packed, padded, n};
        u->tensors.push_back(t);
        packed += n;
        padded = round_up(padded + n, 64);
        return t.padded;
    };
    u->lv.resize(u->L);
    int cprev = kInPitch;
    long long P = u->P0;
    int H = u->H, W = u->W;
    for (int l = 0; l < u->L; ++l) {
        Level& L = u->lv[l];
        L.c = u->base << l;
        L.H = H;
        L.W = W;
        L.P = P;
        L.ea.cin = cprev;
        L.ea.cout = L.c;
        L.ea.w = add(9LL * cprev * L.c);
        L.ea.b = add(L.c);
        L.eb.cin = L.c;
        L.eb.cout = L.c;
        L.eb.w = add(9LL * L.c * L.c);
        L.eb.b = add(L.c);
        cprev = L.c;
        H /= 2;
        W /= 2;
        P /= 4;
    }
    for (int l = u->L - 2; l >= 0; --l) {
        Level& L = u->lv[l];
        const int c = L.c;
        L.up.cin = 2 * c;
        L.up.cout = c;
        L.up.w = add(4LL * c * 2 * c);
        L.up.b = add(4LL * c);
        L.da.cin = 2 * c;
        L.da.cout = c;
        L.da.w = add(9LL * 2 * c * c);
        L.da.b = add(c);
        L.db.cin = c;
        L.db.cout = c;
        L.db.w = add(9LL * c * c);
        L.db.b = add(c);
    }
    u->out_w = add((long long)u->F * u->base);
    u->out_b = add(u->F);
    u->n_packed = packed;
    u->n_padded = padded;
}

cudaError_t allocate(lbm_unet* u)
{
    cudaError_t e = cudaSuccess;
#define UN_ALLOC(p, n)                        \
    do {                                      \
        if ((e = alloc(u, &(p), (n)))) return e; \
    } while (0)
    const long long np = u->n_padded;
    UN_ALLOC(u->w, np);
    UN_ALLOC(u->g, np);
    UN_ALLOC(u->m, np);
    UN_ALLOC(u->v, np);
    UN_ALLOC(u->wb, np);
    UN_ALLOC(u->mean, kInPitch);
    UN_ALLOC(u->inv_std, kInPitch);
    UN_ALLOC(u->inv_out, kInPitch);
    const long long P0 = u->P0;
    UN_ALLOC(u->x0, P0 * kX0Pitch);
    UN_ALLOC(u->Y, P0 * u->F);
    UN_ALLOC(u->T, P0 * u->F);
    UN_ALLOC(u->G, P0 * u->F);
    UN_ALLOC(u->loss, 4);
    const long long part_n = std::max<long long>((long long)kPartBlocks * (u->base + 1) * 8, P0 * u->F / 256 + 2);
    UN_ALLOC(u->part, std::max<long long>(part_n, (long long)kPartBlocks * 4 * (u->base << (u->L - 1))));
    const int L = u->L;
    for (int l = 0; l < L; ++l) {
        Level& v = u->lv[l];
        const long long P = v.P;
        const int c = v.c;
        UN_ALLOC(v.a, P * c);
        if (l < L - 1) {
            v.spitch = 2 * c;
            UN_ALLOC(v.s, P * 2 * c);
            UN_ALLOC(v.pool, P / 4 * c);
            UN_ALLOC(v.dA, P * c);
            UN_ALLOC(v.dD, P * c);
        } else {
            v.spitch = c;
            UN_ALLOC(v.s, P * c);
        }
        for (Conv* cv : {&v.ea, &v.eb, &v.da, &v.db})
            if (cv->cout) UN_ALLOC(cv->wf, 9LL * cv->cin * cv->cout);
        if (l == 0 && nn::conv3x3_supported(u->B, v.H, v.W, kX0Pitch)) {
            v.ea.cin_pad = kX0Pitch;
            UN_ALLOC(v.ea.wpad, 9LL * kX0Pitch * v.ea.cout);
        }
        if (v.up.cout) UN_ALLOC(v.up.wt, 8LL * c * c);
    }
    // gathered-copy buffer for the convolutions the implicit kernel does not
    // take (the first one, 8 input channels; any level of an odd image size)
    long long col_n = 9LL * P0 * kInPitch;
    for (const Level& v : u->lv)
        for (const Conv* cv : {&v.ea, &v.eb, &v.da, &v.db})
            if (cv->cout && !nn::conv3x3_supported(u->B, v.H, v.W, cv->cin)) col_n = std::max(col_n, 9 * v.P * cv->cin);
    UN_ALLOC(u->col, col_n);
    // the table of kernel flips derive() runs in one launch (the weight and
    // flipped-weight buffers stay where they are for the network's life)
    std::vector<nn::FlipJob> jobs;
    long long total = 0;
    for (Level& v : u->lv)
        for (Conv* cv : {&v.ea, &v.eb, &v.da, &v.db})
            if (cv->cout) {
                jobs.push_back({u->wb + cv->w, cv->wf, cv->cout, cv->cin, total});
                total += 9LL * cv->cout * cv->cin;
            }
    nn::FlipJob* table = nullptr;
    UN_ALLOC(table, (long long)jobs.size());
    if ((e = cudaMemcpy(table, jobs.data(), jobs.size() * sizeof(nn::FlipJob), cudaMemcpyHostToDevice))) return e;
    u->flip_jobs = table;
    u->n_flip = (int)jobs.size();
    u->flip_total = total;
#undef UN_ALLOC
    return e;
}

// Buffers only training needs, allocated at the first backward pass.
cudaError_t allocate_backward(lbm_unet* u)
{
    if (u->ws) return cudaSuccess;
    cudaError_t e = cudaSuccess;
#define UN_ALLOC(p, n)                           \
    do {                                         \
        if ((e = alloc(u, &(p), (n)))) return e; \
    } while (0)
    long long col_n = 9LL * u->P0 * kInPitch, ws_n = 0, t_n = 0, g_n = u->P0 * u->base;
    const int L = u->L;
    for (int l = 0; l < L; ++l) {
        Level& v = u->lv[l];
        const long long P = v.P;
        const int c = v.c;
        if (l < L - 1) UN_ALLOC(v.dcat, P * 2 * c);
        for (Conv* cv : {&v.ea, &v.eb, &v.da, &v.db}) {
            if (!cv->cout) continue;
            col_n = std::max(col_n, 9 * P * std::max(cv->cin, cv->cout));
            ws_n = std::max(ws_n, split_ws(9 * cv->cin, cv->cout, P));
            t_n = std::max(t_n, P * std::max(cv->cout, cv->cin));
            g_n = std::max(g_n, P * std::max(cv->cout, cv->cin));
        }
        if (v.up.cout) {
            const long long Pl = P / 4;
            ws_n = std::max(ws_n, split_ws(4 * c, 2 * c, Pl));
            t_n = std::max(t_n, Pl * 4 * c);
            g_n = std::max(g_n, Pl * 4 * c);
        }
    }
    bf16* col = nullptr;
    UN_ALLOC(col, col_n);
    u->col = col;  // the forward's smaller buffer stays allocated until destroy
    UN_ALLOC(u->colT, col_n);
    UN_ALLOC(u->tA, t_n);
    UN_ALLOC(u->tB, t_n);
    UN_ALLOC(u->gA, g_n);
    UN_ALLOC(u->gB, g_n);
    UN_ALLOC(u->dU, g_n);
    UN_ALLOC(u->g32, g_n);
    UN_ALLOC(u->ws, ws_n);
    u->ws_n = ws_n;
#undef UN_ALLOC
    return e;
}

// BF16 copy-derived weights: the rotated conv kernels and transposed
// up-convolution matrices used by the backward pass.
cudaError_t derive(lbm_unet* u)
{
    cudaError_t e = cudaSuccess;
    if ((e = nn::flip3x3_many(u->flip_jobs, u->n_flip, u->flip_total, u->s))) return e;
    for (Level& v : u->lv) {
        for (Conv* cv : {&v.ea, &v.eb, &v.da, &v.db}) {
            if (cv->cout && cv->wpad &&
                (e = nn::pad_conv3x3(u->wb + cv->w, cv->cout, cv->cin, cv->cin_pad, cv->wpad, u->s)))
                return e;
        }
        if (v.up.cout) {
            const int c = v.c;
            if ((e = nn::transpose(u->wb + v.up.w, 4 * c, 2 * c, 2 * c, v.up.wt, 4 * c, u->s))) return e;
        }
    }
    return e;
}

cudaError_t conv_fwd(lbm_unet* u, const Level& v, const Conv& cv, const bf16* in, int inpitch, bf16* out,
                     int outpitch)
{
    cudaError_t e;
    if (cv.wpad)  // zero channels cin .. cin_pad-1 of the input meet zero weights
        e = nn::conv3x3_bf16(in, u->B, v.H, v.W, cv.cin_pad, inpitch, cv.wpad, 9 * cv.cin_pad, out, outpitch,
                             u->w + cv.b, cv.cout, true, true, u->s);
    else
        e = nn::conv3x3_bf16(in, u->B, v.H, v.W, cv.cin, inpitch, u->wb + cv.w, 9 * cv.cin, out, outpitch,
                             u->w + cv.b, cv.cout, true, true, u->s);
    if (e != cudaErrorNotSupported) return e;
    // layouts the implicit convolution does not take (cin = 8): gathered copy + GEMM
    if ((e = nn::im2col3x3(in, u->B, v.H, v.W, cv.cin, inpitch, u->col, u->s))) return e;
    return nn::gemm_bf16(u->col, 9 * cv.cin, u->wb + cv.w, 9 * cv.cin, out, outpitch, u->w + cv.b, (int)v.P, cv.cout,
                         9 * cv.cin, true, true, u->s);
}

// Weight and bias gradients of one convolution from its input `in` and the
// (masked) BF16 output gradient dY [P][cout]; the FP32 input gradient goes to
// dx (pitch dxpitch) when dx is not NULL.
// g32 [rows][C] (pitch) masked by y > 0, then rounded into BF16 [rows][C].
cudaError_t mask_cast(lbm_unet* u, float* g32, int gpitch, const bf16* y, int ypitch, long long rows, int C, bf16* out)
{
    return nn::mask_cast(g32, gpitch, y, ypitch, rows, C, out, C, u->s);
}

// Gradients of a 3 x 3 convolution: weights and bias, and the input gradient
// into dx (FP32, pitch dxpitch) or, with dxb, masked by the convolution's
// input (the output of a ReLU) and rounded to BF16 [P][cin] in the GEMM's
// epilogue (dx then only serves a shape the implicit convolution lacks).
cudaError_t conv_bwd(lbm_unet* u, const Level& v, const Conv& cv, const bf16* in, int inpitch, const bf16* dY,
                     float* dx, int dxpitch, bf16* dxb = nullptr)
{
    const long long P = v.P;
    const int K9 = 9 * cv.cin;
    cudaError_t e;
    // dW [cout][9 cin] = dY^T X_taps, computed as its transpose so that the
    // 9 cin taps fill the MMA's 128 rows and cout (as small as 32) is the N
    // width; the split-K reduction writes it back as [cout][9 cin].  Where the
    // shapes allow, only the three horizontal shifts of X are written out and
    // the GEMM takes the vertical ones by TMA coordinates (a third of the
    // gathered bytes); otherwise all nine taps are gathered.
    const bool three = nn::wgrad3_supported(u->B, v.H, v.W, cv.cin, cv.cout);
    if ((e = nn::gatherT(in, u->B, v.H, v.W, cv.cin, inpitch, three ? 3 : 9, u->colT, P, u->s))) return e;
    if ((e = nn::gatherT(dY, u->B, v.H, v.W, cv.cout, cv.cout, 1, u->tA, P, u->s))) return e;
    const int sp = splits_for(K9, cv.cout, P);
    if (three)
        e = nn::wgrad3_bf16(u->colT, u->tA, u->B, v.H, v.W, cv.cin, cv.cout, u->g + cv.w, K9, u->s, sp, u->ws);
    else
        e = nn::gemm_bf16_tout(u->colT, (int)P, u->tA, (int)P, u->g + cv.w, K9, K9, cv.cout, (int)P, u->s, sp, u->ws);
    if (e) return e;
    if ((e = nn::colsum(dY, false, P, cv.cout, cv.cout, u->g + cv.b, u->part, kPartBlocks, u->s))) return e;
    if (!dx) return cudaSuccess;
    if (dxb) {
        e = nn::conv3x3_bf16(dY, u->B, v.H, v.W, cv.cout, cv.cout, cv.wf, 9 * cv.cout, dxb, cv.cin, nullptr, cv.cin,
                             true, false, u->s, in, inpitch);
        if (e != cudaErrorNotSupported) return e;
    } else {
        e = nn::conv3x3_bf16(dY, u->B, v.H, v.W, cv.cout, cv.cout, cv.wf, 9 * cv.cout, dx, dxpitch, nullptr, cv.cin,
                             false, false, u->s);
        if (e != cudaErrorNotSupported) return e;
    }
    if ((e = nn::im2col3x3(dY, u->B, v.H, v.W, cv.cout, cv.cout, u->col, u->s))) return e;
    if ((e = nn::gemm_bf16(u->col, 9 * cv.cout, cv.wf, 9 * cv.cout, dx, dxpitch, nullptr, (int)P, cv.cin,
                           9 * cv.cout, false, false, u->s)))
        return e;
    return dxb ? mask_cast(u, dx, dxpitch, in, inpitch, P, cv.cin, dxb) : cudaSuccess;
}


cudaError_t forward(lbm_unet* u, const float* x)
{
    cudaError_t e;
    if ((e = nn::pack(x, u->P0, u->F, u->mean, u->inv_std, u->x0, kX0Pitch, nullptr, u->s))) return e;
    const bf16* in = u->x0;
    int inpitch = kX0Pitch;
    const int L = u->L;
    for (int l = 0; l < L; ++l) {
        Level& v = u->lv[l];
        if ((e = conv_fwd(u, v, v.ea, in, inpitch, v.a, v.c))) return e;
        if ((e = conv_fwd(u, v, v.eb, v.a, v.c, v.s, v.spitch))) return e;
        if (l < L - 1) {
            if ((e = nn::maxpool_fwd(v.s, u->B, v.H, v.W, v.c, v.spitch, v.pool, u->s))) return e;
            in = v.pool;
            inpitch = v.c;
        }
    }
    const bf16* h = u->lv[L - 1].s;
    for (int l = L - 2; l >= 0; --l) {
        Level& v = u->lv[l];
        const Level& lo = u->lv[l + 1];
        const int c = v.c;
        if ((e = nn::upconv2x2_bf16(h, 2 * c, u->wb + v.up.w, 2 * c, v.s, 2 * c, c, u->w + v.up.b, u->B, lo.H, lo.W,
                                    2 * c, c, u->s)))
            return e;
        if ((e = conv_fwd(u, v, v.da, v.s, 2 * c, v.dA, c))) return e;
        if ((e = conv_fwd(u, v, v.db, v.dA, c, v.dD, c))) return e;
        h = v.dD;
    }
    const bf16* top = L > 1 ? u->lv[0].dD : u->lv[0].s;
    return nn::proj_fwd(top, (int)u->P0, u->base, u->base, u->w + u->out_w, u->w + u->out_b, u->F, nullptr, u->Y,
                        u->s);
}

// Loss and parameter gradients for the target t (physical units); forward(x) ran.
cudaError_t backward(lbm_unet* u, const float* x, const float* t)
{
    cudaError_t e;
    const long long P0 = u->P0;
    const int L = u->L, F = u->F, w0 = u->base;
    if ((e = nn::increment(t, x, P0, F, u->inv_out, u->T, u->s))) return e;
    if ((e = nn::mse(u->Y, u->T, P0 * F, u->G, u->loss, u->part, u->s, u->iface_w != 0.0f ? x : nullptr, F,
                     u->iface_w)))
        return e;
    const bf16* top = L > 1 ? u->lv[0].dD : u->lv[0].s;
    if ((e = nn::proj_bwd(u->G, top, (int)P0, w0, w0, u->w + u->out_w, F, u->g32, w0, u->g + u->out_w, u->g + u->out_b,
                          u->part, kPartBlocks, u->s)))
        return e;
    if ((e = mask_cast(u, u->g32, w0, top, L > 1 ? w0 : u->lv[0].spitch, P0, w0, u->gA))) return e;
    // decoder, top level first; gA holds the masked gradient of the level's output
    for (int l = 0; l < L - 1; ++l) {
        Level& v = u->lv[l];
        const Level& lo = u->lv[l + 1];
        const int c = v.c;
        if ((e = conv_bwd(u, v, v.db, v.dA, c, u->gA, u->g32, c, u->gB))) return e;
        if ((e = conv_bwd(u, v, v.da, v.s, 2 * c, u->gB, v.dcat, 2 * c))) return e;
        // up-convolution: gradient of u_l is the second half of dcat
        if ((e = nn::shuffle_bwd(v.dcat, true, 2 * c, c, u->B, lo.H, lo.W, c, u->dU, u->s))) return e;
        if ((e = nn::colsum(u->dU, false, lo.P, 4 * c, 4 * c, u->g + v.up.b, u->part, kPartBlocks, u->s))) return e;
        const bf16* hlow = (l + 1 < L - 1) ? lo.dD : lo.s;
        if ((e = nn::gatherT(u->dU, u->B, lo.H, lo.W, 4 * c, 4 * c, 1, u->tA, lo.P, u->s))) return e;
        if ((e = nn::gatherT(hlow, u->B, lo.H, lo.W, 2 * c, 2 * c, 1, u->tB, lo.P, u->s))) return e;
        const int sp = splits_for(4 * c, 2 * c, lo.P);
        if ((e = nn::gemm_bf16(u->tA, (int)lo.P, u->tB, (int)lo.P, u->g + v.up.w, 2 * c, nullptr, 4 * c, 2 * c,
                               (int)lo.P, false, false, u->s, sp, u->ws)))
            return e;
        // gradient of the up-convolution's input, masked by that input (a ReLU
        // output) and rounded to BF16 in the GEMM's epilogue
        if ((e = nn::gemm_bf16(u->dU, 4 * c, v.up.wt, 4 * c, u->gA, 2 * c, nullptr, (int)lo.P, 2 * c, 4 * c, true,
                               false, u->s, 1, nullptr, hlow, 2 * c)))
            return e;
    }
    // encoder, bottom level first
    for (int l = L - 1; l >= 0; --l) {
        Level& v = u->lv[l];
        const int c = v.c;
        if (l < L - 1) {
            // skip gradient (first half of dcat) plus the pooled path's gradient in g32
            if ((e = nn::maxpool_bwd(v.s, u->B, v.H, v.W, c, 2 * c, u->g32, v.dcat, 2 * c, u->s))) return e;
            if ((e = mask_cast(u, v.dcat, 2 * c, v.s, 2 * c, v.P, c, u->gA))) return e;
        }
        if ((e = conv_bwd(u, v, v.eb, v.a, c, u->gA, u->g32, c, u->gB))) return e;
        const bf16* in = l == 0 ? u->x0 : u->lv[l - 1].pool;
        const int inpitch = l == 0 ? kX0Pitch : u->lv[l - 1].c;
        if ((e = conv_bwd(u, v, v.ea, in, inpitch, u->gB, l == 0 ? nullptr : u->g32, v.ea.cin))) return e;
    }
    return cudaSuccess;
}

}  // namespace

extern "C" {

int lbm_unet_create(int levels, int base, int fields, int batch, int height, int width, lbm_unet** out)
{
    if (!out) return LBM_EINVAL;
    *out = nullptr;
    if (levels < 1 || levels > 8 || base < 8 || base % 8 || fields < 1 || fields > kInPitch || batch < 1)
        return LBM_EINVAL;
    const int div = 1 << (levels - 1);
    if (height < div || width < div || height % div || width % div) return LBM_EINVAL;
    const long long P0 = (long long)batch * height * width;
    const long long Pb = P0 >> (2 * (levels - 1));
    if (Pb % 8 || P0 > (1LL << 30)) return LBM_EINVAL;
    lbm_unet* u = new lbm_unet;
    u->L = levels;
    u->base = base;
    u->F = fields;
    u->B = batch;
    u->H = height;
    u->W = width;
    u->P0 = P0;
    plan(u);
    cudaError_t e = allocate(u);
    if (e == cudaSuccess) {
        float ones[kInPitch], zeros[kInPitch] = {0};
        for (float& o : ones) o = 1.0f;
        e = cudaMemcpy(u->mean, zeros, sizeof zeros, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(u->inv_std, ones, sizeof ones, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(u->inv_out, ones, sizeof ones, cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        lbm_unet_destroy(u);
        return e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA;
    }
    *out = u;
    return LBM_OK;
}

void lbm_unet_destroy(lbm_unet* u)
{
    if (!u) return;
    for (void* p : u->allocs) cudaFree(p);
    delete u;
}

int lbm_unet_set_stream(lbm_unet* u, void* stream)
{
    if (!u) return LBM_EINVAL;
    u->s = (cudaStream_t)stream;
    return LBM_OK;
}

long long lbm_unet_param_count(const lbm_unet* u) { return u ? u->n_packed : -1; }

int lbm_unet_shape(const lbm_unet* u, int* batch, int* height, int* width, int* fields)
{
    if (!u || !batch || !height || !width || !fields) return LBM_EINVAL;
    *batch = u->B;
    *height = u->H;
    *width = u->W;
    *fields = u->F;
    return LBM_OK;
}

long long lbm_unet_device_bytes(const lbm_unet* u) { return u ? u->bytes : -1; }

int lbm_unet_set_params(lbm_unet* u, const float* host)
{
    if (!u || !host) return LBM_EINVAL;
    std::vector<float> pad((size_t)u->n_padded, 0.0f);
    for (const Tensor& t : u->tensors) std::memcpy(&pad[t.padded], host + t.packed, (size_t)t.n * sizeof(float));
    UN_CHECK(u, cudaMemcpyAsync(u->w, pad.data(), pad.size() * sizeof(float), cudaMemcpyHostToDevice, u->s));
    UN_CHECK(u, cudaMemsetAsync(u->m, 0, pad.size() * sizeof(float), u->s));
    UN_CHECK(u, cudaMemsetAsync(u->v, 0, pad.size() * sizeof(float), u->s));
    UN_CHECK(u, nn::cast_bf16(u->w, 1, (int)u->n_padded, (int)u->n_padded, u->wb, (int)u->n_padded, u->s));
    UN_CHECK(u, derive(u));
    UN_CHECK(u, cudaStreamSynchronize(u->s));
    u->t = 0;
    return LBM_OK;
}

static int get_vec(lbm_unet* u, const float* dev, float* host)
{
    if (!u || !host) return LBM_EINVAL;
    std::vector<float> pad((size_t)u->n_padded);
    UN_CHECK(u, cudaStreamSynchronize(u->s));
    UN_CHECK(u, cudaMemcpy(pad.data(), dev, pad.size() * sizeof(float), cudaMemcpyDeviceToHost));
    for (const Tensor& t : u->tensors) std::memcpy(host + t.packed, &pad[t.padded], (size_t)t.n * sizeof(float));
    return LBM_OK;
}

int lbm_unet_get_params(lbm_unet* u, float* host) { return get_vec(u, u ? u->w : nullptr, host); }

int lbm_unet_get_grads(lbm_unet* u, float* host) { return get_vec(u, u ? u->g : nullptr, host); }

int lbm_unet_set_loss_weight(lbm_unet* u, float alpha)
{
    if (!u || !(alpha >= 0.0f) || !isfinite(alpha)) return LBM_EINVAL;
    u->iface_w = alpha;
    return LBM_OK;
}

int lbm_unet_set_norm(lbm_unet* u, const float* mean, const float* std_in, const float* std_out)
{
    if (!u || !mean || !std_in) return LBM_EINVAL;
    if (!std_out) std_out = std_in;
    float mu[kInPitch] = {0}, is[kInPitch], io[kInPitch];
    for (int c = 0; c < kInPitch; ++c) is[c] = io[c] = 1.0f;
    for (int c = 0; c < u->F; ++c) {
        if (!(std_in[c] > 0.0f) || !(std_out[c] > 0.0f)) return fail(u, LBM_EINVAL, "scales must be positive");
        mu[c] = mean[c];
        is[c] = 1.0f / std_in[c];
        io[c] = 1.0f / std_out[c];
    }
    u->norm_h.assign(3 * (size_t)u->F, 0.0f);
    for (int c = 0; c < u->F; ++c) {
        u->norm_h[c] = mean[c];
        u->norm_h[u->F + c] = std_in[c];
        u->norm_h[2 * u->F + c] = std_out[c];
    }
    UN_CHECK(u, cudaMemcpyAsync(u->mean, mu, sizeof mu, cudaMemcpyHostToDevice, u->s));
    UN_CHECK(u, cudaMemcpyAsync(u->inv_std, is, sizeof is, cudaMemcpyHostToDevice, u->s));
    UN_CHECK(u, cudaMemcpyAsync(u->inv_out, io, sizeof io, cudaMemcpyHostToDevice, u->s));
    UN_CHECK(u, cudaStreamSynchronize(u->s));
    return LBM_OK;
}

// Weight file: "LBMUNET1", int32 levels, base, fields, 0, int64 parameter
// count, FP32 mean, std_in, std_out (fields each), FP32 parameters; all
// little-endian, as the hosts this builds for store them.
static const char kUnetMagic[8] = {'L', 'B', 'M', 'U', 'N', 'E', 'T', '1'};

int lbm_unet_save(lbm_unet* u, const char* path)
{
    if (!u || !path) return LBM_EINVAL;
    std::vector<float> p((size_t)lbm_unet_param_count(u));
    int rc = lbm_unet_get_params(u, p.data());
    if (rc) return rc;
    std::vector<float> norm = u->norm_h;
    if (norm.empty()) {  // never set: mean 0, scales 1
        norm.assign(3 * (size_t)u->F, 1.0f);
        std::fill(norm.begin(), norm.begin() + u->F, 0.0f);
    }
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(u, LBM_EINVAL, std::string("cannot open ") + path + " for writing");
    const int32_t shape[4] = {u->L, u->base, u->F, 0};
    const int64_t n = (int64_t)p.size();
    bool ok = std::fwrite(kUnetMagic, 1, 8, f) == 8 && std::fwrite(shape, sizeof shape, 1, f) == 1 &&
              std::fwrite(&n, sizeof n, 1, f) == 1 && std::fwrite(norm.data(), sizeof(float), norm.size(), f) == norm.size() &&
              std::fwrite(p.data(), sizeof(float), p.size(), f) == p.size();
    ok = (std::fclose(f) == 0) && ok;
    return ok ? LBM_OK : fail(u, LBM_EINVAL, std::string("write to ") + path + " failed");
}

int lbm_unet_load(lbm_unet* u, const char* path)
{
    if (!u || !path) return LBM_EINVAL;
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(u, LBM_EINVAL, std::string("cannot open ") + path);
    char magic[8];
    int32_t shape[4];
    int64_t n = 0;
    std::vector<float> norm(3 * (size_t)u->F), p((size_t)lbm_unet_param_count(u));
    std::string why;
    if (std::fread(magic, 1, 8, f) != 8 || std::memcmp(magic, kUnetMagic, 8) != 0)
        why = "not a network weight file";
    else if (std::fread(shape, sizeof shape, 1, f) != 1 || std::fread(&n, sizeof n, 1, f) != 1)
        why = "truncated header";
    else if (shape[0] != u->L || shape[1] != u->base || shape[2] != u->F || n != (int64_t)p.size())
        why = "the file holds a network of another shape";
    else if (std::fread(norm.data(), sizeof(float), norm.size(), f) != norm.size() ||
             std::fread(p.data(), sizeof(float), p.size(), f) != p.size())
        why = "truncated weights";
    else if (std::fgetc(f) != EOF)
        why = "trailing bytes after the weights";
    std::fclose(f);
    if (!why.empty()) return fail(u, LBM_EINVAL, std::string(path) + ": " + why);
    for (float x : p)
        if (!std::isfinite(x)) return fail(u, LBM_EINVAL, std::string(path) + ": non-finite weight");
    int rc = lbm_unet_set_params(u, p.data());
    if (rc) return rc;
    return lbm_unet_set_norm(u, norm.data(), norm.data() + u->F, norm.data() + 2 * u->F);
}

int lbm_unet_forward(lbm_unet* u, const float* x, float* y)
{
    trace::Range range("lbm_unet_forward");
    if (!u || !x) return LBM_EINVAL;
    UN_CHECK(u, forward(u, x));
    if (y) UN_CHECK(u, nn::add_increment(u->Y, x, u->P0, u->F, u->inv_out, y, u->s));
    return LBM_OK;
}

int lbm_unet_backward(lbm_unet* u, const float* x, const float* target)
{
    trace::Range range("lbm_unet_backward");
    if (!u || !x || !target) return LBM_EINVAL;
    UN_CHECK(u, allocate_backward(u));
    UN_CHECK(u, forward(u, x));
    UN_CHECK(u, backward(u, x, target));
    return LBM_OK;
}

int lbm_unet_adam(lbm_unet* u, float lr, float beta1, float beta2, float eps)
{
    if (!u || !(lr >= 0.0f)) return LBM_EINVAL;
    ++u->t;
    UN_CHECK(u, nn::adam(u->w, u->g, u->m, u->v, u->n_padded, lr, beta1, beta2, eps, u->t, u->wb, u->s));
    UN_CHECK(u, derive(u));
    return LBM_OK;
}

int lbm_unet_train_step(lbm_unet* u, const float* x, const float* target, float lr)
{
    trace::Range range("lbm_unet_train_step");
    int r = lbm_unet_backward(u, x, target);
    if (r != LBM_OK) return r;
    return lbm_unet_adam(u, lr, 0.9f, 0.999f, 1e-8f);
}

int lbm_unet_loss(lbm_unet* u, double* out)
{
    if (!u || !out) return LBM_EINVAL;
    float l = 0.0f;
    UN_CHECK(u, cudaStreamSynchronize(u->s));
    UN_CHECK(u, cudaMemcpy(&l, u->loss, sizeof l, cudaMemcpyDeviceToHost));
    *out = (double)l / (double)(u->P0 * u->F);
    return LBM_OK;
}

int lbm_unet_output(lbm_unet* u, float* y_norm)
{
    if (!u || !y_norm) return LBM_EINVAL;
    UN_CHECK(u, cudaMemcpyAsync(y_norm, u->Y, (size_t)u->P0 * u->F * sizeof(float), cudaMemcpyDeviceToDevice, u->s));
    return LBM_OK;
}

const char* lbm_unet_last_error(const lbm_unet* u) { return u ? u->err.c_str() : "null network"; }

}  // extern "C"
