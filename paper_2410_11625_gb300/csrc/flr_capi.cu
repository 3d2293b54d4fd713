// flr_capi.cu -- the extern "C" boundary of libflr.so (declared in include/flr.h):
// argument validation, handle and workspace management, and the launch sequences
//   fused forward kernel (moments, solve, averaging, apply) -> FP64 correction of flagged
//   pixels, for the compiled (q, r, rc) instances with 16-byte rows (flr_fused.cu);
//   otherwise forward kernel -> FP64 re-solve of flagged pixels -> averaging + apply.
// No exception and no abort crosses the ABI: every failure is a negative flr_status.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <algorithm>
#include <vector>

#include "flr.h"
#include "flr_internal.cuh"

namespace {

thread_local char g_cuda_error[256] = "no error";

int cuda_fail(cudaError_t e, const char *what)
{
    std::snprintf(g_cuda_error, sizeof(g_cuda_error), "%s: %s", what, cudaGetErrorString(e));
    return FLR_ERR_CUDA;
}

#define FLR_CUDA(call, what)                          \
    do {                                              \
        cudaError_t e_ = (call);                      \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace

namespace flr {
namespace host {

// Rows per segment of the forward kernel: minimise (waves of CTAs) x (rows walked,
// including the 2r warm-up rows of every segment).
int choose_segment_rows(int H, int W, int r, int n_sm)
{
    const int strips = (W + flr::kTW - 1) / flr::kTW;
    int best_th = H, best_cost = -1;
    for (int segs = 1; segs <= 256; ++segs) {
        int th = (H + segs - 1) / segs;
        th = (th + flr::kB - 1) / flr::kB * flr::kB;
        const int real_segs = (H + th - 1) / th;
        const long long waves = ((long long)strips * real_segs + n_sm - 1) / n_sm;
        const long long cost = waves * (th + 2 * r);
        if (best_cost < 0 || cost < best_cost) { best_cost = (int)cost; best_th = th; }
        if (th <= flr::kB) break;
    }
    return best_th;
}

// Launch plan of the fused forward kernel over `rows` output rows: strips of TW columns, and
// the segment height that minimises (waves of CTAs, one CTA per SM) x (rows walked per
// segment, including the 2 (r + rc) warm-up rows).
FusedPlan fused_plan(int rows, int W, int r, int rc, int n_sm)
{
    FusedPlan p;
    p.TW = flr::fused_tile_width(rc);
    p.strips = (W + p.TW - 1) / p.TW;
    int best_th = rows;
    long long best = -1;
    for (int segs = 1; segs <= 512; ++segs) {
        int th = (rows + segs - 1) / segs;
        th = (th + 3) / 4 * 4;
        const int real = (rows + th - 1) / th;
        const long long waves = ((long long)p.strips * real + n_sm - 1) / n_sm;
        const long long cost = waves * (th + 2 * r + 2 * rc);
        if (best < 0 || cost < best) { best = cost; best_th = th; }
        if (th <= 4) break;
    }
    p.TH = best_th;
    p.segs = (rows + p.TH - 1) / p.TH;
    p.cap = (p.TW + 2 * rc) * (p.TH + 2 * rc);
    return p;
}

// Whether a call can take the fused path: a compiled instance, rows of 16-byte multiples
// (TMA), 16-byte aligned images, and images whose element offsets fit in 32 bits.
bool fused_ok(const flr_params &p, int H, int W, const void *g, const void *mg, const void *rad, const void *out)
{
    return flr::fused_supported(p.q, p.radius, p.coef_radius) && (W % 4) == 0 && aligned16(g) && aligned16(rad) &&
           aligned16(out) && (!mg || aligned16(mg)) && (long long)H * W * (p.q + 3) < 0x7fffffffLL;
}

int validate_params(const flr_params *p)
{
    if (!p) return FLR_ERR_ARG;
    if ((p->flags & ~FLR_FLAG_TIMING) != 0u || !(p->eps >= 0.f) || p->radius < 0 || p->coef_radius < 0) return FLR_ERR_ARG;
    if (p->pivot_ratio != p->pivot_ratio) return FLR_ERR_ARG;
    if (p->q < 1 || p->q > FLR_MAX_Q || p->radius > FLR_MAX_RADIUS ||
        p->coef_radius > FLR_MAX_COEF_RADIUS)
        return FLR_ERR_UNSUPPORTED;
    return FLR_OK;
}

}  // namespace host
}  // namespace flr

struct flr_handle {
    flr_params p;
    int device = 0;
    int n_sm = 0;
    unsigned long long *d_count = nullptr;  // [0] flagged pixels, [1] non-finite output values
    int *d_status = nullptr;                // set by a kernel whose bounded wait ran out
    float *d_shift = nullptr;               // frame reference shift, Q+3 floats
    int *d_flags = nullptr;                 // flag list
    int flag_cap = 0;
    float *d_coef = nullptr;  // (Q+1)*3 coefficient planes (coef_radius > 0)
    size_t coef_px = 0;
    float *stage = nullptr;  // host-path staging: guide, map guide, radiance, out
    size_t stage_px = 0;
    // host-path pipeline: copy-in and copy-out streams, per-band events, re-solve start index
    cudaStream_t s_in = nullptr, s_out = nullptr;
    std::vector<cudaEvent_t> band_ev;
    unsigned long long *d_fstart = nullptr;
    float *bwd = nullptr;  // backward workspace: models, fields/averaged models, G(A), GS, BS
    size_t bwd_px = 0;
    size_t adj_smem = 0;
    size_t fwd_smem = 0;
    cudaStream_t last_stream = nullptr;
    // instrumentation: launch counts, and event quadruples per call with FLR_FLAG_TIMING
    unsigned long long n_fwd = 0, n_fp64 = 0, n_apply = 0;
    std::vector<cudaEvent_t> events;
    size_t events_used = 0;
    // fused path (flr_fused.cu): per-CTA flag lists, entry counts and reference shifts
    int *d_flist = nullptr;
    size_t flist_ints = 0;
    int *d_fcount = nullptr;
    float *d_fshift = nullptr;
    int fcta = 0;
    bool last_fused = false;  // the last forward call took the fused path
    // asynchronous host path (flr_denoise_host_async): two device staging slots (guide, map
    // guide, radiance, out), per slot the events "inputs copied in", "kernels done" and
    // "result copied out", and the slot the next frame takes
    float *aslot[2] = {nullptr, nullptr};
    size_t aslot_px[2] = {0, 0};
    cudaEvent_t a_in[2] = {}, a_comp[2] = {}, a_out[2] = {};
    int a_next = 0;
    bool a_pending = false;
};

namespace {

using flr::host::FusedPlan;
using flr::host::choose_segment_rows;
using flr::host::fused_ok;
using flr::host::fused_plan;
using flr::host::validate_params;

int grow(flr_handle *h, int H, int W)
{
    const size_t px = (size_t)H * W;
    if ((size_t)h->flag_cap < px && h->p.pivot_ratio > 0.f) {
        if (h->d_flags) cudaFree(h->d_flags);
        h->d_flags = nullptr;
        h->flag_cap = 0;
        if (px > (size_t)0x7fffffff) return FLR_ERR_ARG;
        if (cudaMalloc(&h->d_flags, px * sizeof(int)) != cudaSuccess) return FLR_ERR_NOMEM;
        h->flag_cap = (int)px;
    }
    if (h->p.coef_radius > 0 && h->coef_px < px) {
        if (h->d_coef) cudaFree(h->d_coef);
        h->d_coef = nullptr;
        h->coef_px = 0;
        if (cudaMalloc(&h->d_coef, px * (size_t)(h->p.q + 1) * 3 * sizeof(float)) != cudaSuccess)
            return FLR_ERR_NOMEM;
        h->coef_px = px;
    }
    return FLR_OK;
}

// With FLR_FLAG_TIMING: the next event of the handle's pool, recorded on stream s.
cudaError_t mark(flr_handle *h, cudaStream_t s)
{
    if (!(h->p.flags & FLR_FLAG_TIMING)) return cudaSuccess;
    if (h->events_used == h->events.size()) {
        cudaEvent_t ev;
        cudaError_t e = cudaEventCreate(&ev);
        if (e != cudaSuccess) return e;
        h->events.push_back(ev);
    }
    return cudaEventRecord(h->events[h->events_used++], s);
}

int grow_fused(flr_handle *h, const FusedPlan &pl)
{
    const int ncta = pl.strips * pl.segs;
    const size_t ints = (size_t)ncta * pl.cap;
    if (ncta > h->fcta) {
        cudaFree(h->d_fcount);
        cudaFree(h->d_fshift);
        h->d_fcount = nullptr;
        h->d_fshift = nullptr;
        h->fcta = 0;
        if (cudaMalloc(&h->d_fcount, ncta * sizeof(int)) != cudaSuccess ||
            cudaMalloc(&h->d_fshift, (size_t)ncta * (FLR_MAX_Q + 3) * sizeof(float)) != cudaSuccess)
            return FLR_ERR_NOMEM;
        h->fcta = ncta;
    }
    if (ints > h->flist_ints && h->p.pivot_ratio > 0.f) {
        cudaFree(h->d_flist);
        h->d_flist = nullptr;
        h->flist_ints = 0;
        if (cudaMalloc(&h->d_flist, ints * sizeof(int)) != cudaSuccess) return FLR_ERR_NOMEM;
        h->flist_ints = ints;
    }
    return FLR_OK;
}

// The fused forward kernel over output rows [row_lo, row_hi), then (pivot test on) the FP64
// correction of its flagged pixels.  Timing marks bracket each kernel (apply: none).
int run_fused(flr_handle *h, const float *guide, const float *map_guide, const float *radiance, float *out, int H,
              int W, int row_lo, int row_hi, cudaStream_t s)
{
    const FusedPlan pl = fused_plan(row_hi - row_lo, W, h->p.radius, h->p.coef_radius, h->n_sm);
    int st = grow_fused(h, pl);
    if (st != FLR_OK) return st;
    flr::FusedArgs fa;
    fa.guide = guide;
    fa.map_guide = map_guide;
    fa.rad = radiance;
    fa.out = out;
    fa.H = H;
    fa.W = W;
    fa.r = h->p.radius;
    fa.rc = h->p.coef_radius;
    fa.eps = h->p.eps;
    fa.tau = h->p.pivot_ratio;
    fa.TH = pl.TH;
    fa.row_lo = row_lo;
    fa.row_hi = row_hi;
    fa.list = h->d_flist;
    fa.list_cap = h->p.pivot_ratio > 0.f ? pl.cap : 0;
    fa.list_count = h->d_fcount;
    fa.cta_shift = h->d_fshift;
    fa.flag_count = h->d_count;
    fa.nonfinite = h->d_count + 1;
    fa.status = h->d_status;
    const dim3 grid(pl.strips, pl.segs);
    FLR_CUDA(mark(h, s), "timing event");
    FLR_CUDA(flr::launch_fused(h->p.q, fa, grid, s), "fused forward kernel launch");
    ++h->n_fwd;
    FLR_CUDA(mark(h, s), "timing event");
    if (h->p.pivot_ratio > 0.f) {
        FLR_CUDA(flr::launch_fused_fix(h->p.q, fa, grid, s), "fp64 correction launch");
        ++h->n_fp64;
    }
    FLR_CUDA(mark(h, s), "timing event");
    FLR_CUDA(mark(h, s), "timing event");
    h->last_fused = true;
    return FLR_OK;
}

// Row bands of the host entry point (see flr_denoise_host): band k computes the models of
// rows [c_k, c_k+1), needs input rows below in_end_k+1 (copied in as rows [in_end_k,
// in_end_k+1)) and writes output rows [o_k, o_k+1).  Returns the number of bands K; the
// arrays hold K + 1 entries (K <= FLR_HOST_MAX_BANDS).  Bands of about 360 rows: a band's
// kernels lose efficiency as it gets shorter (each segment re-fills its window and a short
// band fills fewer CTAs), while fewer bands expose more of the first copy; at 1920x1080
// three bands measured 0.74 ms per frame against 0.96 (one), 0.79 (two), 0.75 (four) and
// 0.93 (eight).
int band_plan(int H, int r, int rc, int *c, int *in_end, int *o)
{
    const int K = std::max(1, std::min(FLR_HOST_MAX_BANDS, (H + 180) / 360));
    for (int k = 0; k <= K; ++k) c[k] = k == K ? H : (int)((long long)H * k / K) / flr::kB * flr::kB;
    for (int k = 0; k <= K; ++k) {
        in_end[k] = std::min(H, c[k] + r);
        o[k] = (k == 0 || k == K || rc == 0) ? c[k] : std::max(0, c[k] - rc);
    }
    in_end[0] = 0;
    return K;
}

// Device staging of the host paths: guide (q planes), map guide (q), radiance (3) and output
// (3) of a px-pixel frame, each region starting 16-byte aligned (planes px floats apart).
size_t staging_floats(size_t px, int q)
{
    const size_t pxa = (px + 3) & ~(size_t)3;
    return pxa * (2 * (size_t)q + 6);
}
void staging_regions(float *base, size_t px, int q, float **dg, float **dm, float **dr, float **dout)
{
    auto up = [](size_t n) { return (n + 3) & ~(size_t)3; };
    *dg = base;
    *dm = *dg + up((size_t)q * px);
    *dr = *dm + up((size_t)q * px);
    *dout = *dr + up(3 * px);
}

// The handle's copy-in and copy-out streams (created on first use).
int copy_streams(flr_handle *h)
{
    if (!h->s_in) FLR_CUDA(cudaStreamCreateWithFlags(&h->s_in, cudaStreamNonBlocking), "copy stream");
    if (!h->s_out) FLR_CUDA(cudaStreamCreateWithFlags(&h->s_out, cudaStreamNonBlocking), "copy stream");
    return FLR_OK;
}

}  // namespace

extern "C" {

const char *flr_status_string(int status)
{
    switch (status) {
    case FLR_OK: return "FLR_OK";
    case FLR_ERR_ARG: return "FLR_ERR_ARG: invalid argument";
    case FLR_ERR_ALIGN: return "FLR_ERR_ALIGN: device pointer not 16-byte aligned";
    case FLR_ERR_CUDA: return "FLR_ERR_CUDA: CUDA runtime error";
    case FLR_ERR_UNSUPPORTED: return "FLR_ERR_UNSUPPORTED: parameter outside the built range";
    case FLR_ERR_NOMEM: return "FLR_ERR_NOMEM: workspace allocation failed";
    case FLR_ERR_TIMEOUT: return "FLR_ERR_TIMEOUT: a device-side wait ran out of time";
    default: return "unknown flr status";
    }
}

const char *flr_last_cuda_error(void) { return g_cuda_error; }

int flr_create(const flr_params *params, flr_handle **out)
{
    if (!out) return FLR_ERR_ARG;
    *out = nullptr;
    int st = validate_params(params);
    if (st != FLR_OK) return st;
    flr_handle *h = new (std::nothrow) flr_handle();
    if (!h) return FLR_ERR_NOMEM;
    h->p = *params;
    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, h->device);
    if (e == cudaSuccess) e = cudaMalloc(&h->d_count, 2 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&h->d_shift, sizeof(float) * (FLR_MAX_Q + 3));
    if (e == cudaSuccess) e = cudaMemset(h->d_count, 0, 2 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&h->d_status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(h->d_status, 0, sizeof(int));
    if (e == cudaSuccess) {
        h->fwd_smem = flr::fwd_smem_bytes(h->p.q, h->p.radius);
        e = flr::fwd_prepare(h->p.q, h->p.radius, h->fwd_smem);
    }
    if (e == cudaSuccess) {
        h->adj_smem = flr::adj_smem_bytes(h->p.q, h->p.radius);
        e = flr::adj_prepare(h->p.q, h->p.radius, h->adj_smem);
    }
    if (e != cudaSuccess) {
        cuda_fail(e, "flr_create");
        flr_destroy(h);
        return FLR_ERR_CUDA;
    }
    *out = h;
    return FLR_OK;
}

int flr_destroy(flr_handle *h)
{
    if (!h) return FLR_OK;
    cudaDeviceSynchronize();
    cudaFree(h->d_count);
    cudaFree(h->d_status);
    cudaFree(h->d_fstart);
    for (cudaEvent_t e : h->band_ev) cudaEventDestroy(e);
    if (h->s_in) cudaStreamDestroy(h->s_in);
    if (h->s_out) cudaStreamDestroy(h->s_out);
    cudaFree(h->d_shift);
    cudaFree(h->d_flags);
    cudaFree(h->d_coef);
    cudaFree(h->stage);
    cudaFree(h->bwd);
    cudaFree(h->d_flist);
    cudaFree(h->d_fcount);
    cudaFree(h->d_fshift);
    for (cudaEvent_t ev : h->events) cudaEventDestroy(ev);
    for (int k = 0; k < 2; ++k) {
        cudaFree(h->aslot[k]);
        for (cudaEvent_t ev : {h->a_in[k], h->a_comp[k], h->a_out[k]})
            if (ev) cudaEventDestroy(ev);
    }
    delete h;
    return FLR_OK;
}

int flr_reserve(flr_handle *h, int H, int W)
{
    if (!h || H <= 0 || W <= 0) return FLR_ERR_ARG;
    if (flr::fused_supported(h->p.q, h->p.radius, h->p.coef_radius) && W % 4 == 0)
        return grow_fused(h, fused_plan(H, W, h->p.radius, h->p.coef_radius, h->n_sm));
    return grow(h, H, W);
}

int flr_denoise(flr_handle *h, const float *guide, const float *map_guide, const float *radiance,
                float *out, int H, int W, void *stream)
{
    if (!h || !guide || !radiance || !out || H <= 0 || W <= 0) return FLR_ERR_ARG;
    if ((long long)H * W > 0x7fffffffLL) return FLR_ERR_ARG;
    if (!aligned16(guide) || !aligned16(radiance) || !aligned16(out) ||
        (map_guide && !aligned16(map_guide)))
        return FLR_ERR_ALIGN;
    const int q = h->p.q;
    const size_t px = (size_t)H * W;
    // the output must not overlap any input
    auto overlaps = [&](const float *p, size_t n) {
        return p && (const char *)out < (const char *)(p + n) && (const char *)p < (const char *)(out + 3 * px);
    };
    if (overlaps(guide, q * px) || overlaps(map_guide, q * px) || overlaps(radiance, 3 * px))
        return FLR_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    h->last_stream = s;
    FLR_CUDA(cudaMemsetAsync(h->d_count, 0, 2 * sizeof(unsigned long long), s), "reset counters");
    if (fused_ok(h->p, H, W, guide, map_guide, radiance, out))
        return run_fused(h, guide, map_guide, radiance, out, H, W, 0, H, s);
    h->last_fused = false;
    int st = grow(h, H, W);
    if (st != FLR_OK) return st;

    flr::FwdArgs fa;
    fa.guide = guide;
    fa.map_guide = map_guide;
    fa.rad = radiance;
    fa.out = out;
    fa.coef = h->d_coef;
    fa.H = H;
    fa.W = W;
    fa.r = h->p.radius;
    fa.rc = h->p.coef_radius;
    fa.eps = h->p.eps;
    fa.tau = h->p.pivot_ratio;
    fa.TH = choose_segment_rows(H, W, h->p.radius, h->n_sm);
    fa.flag_count = h->d_count;
    fa.flag_list = h->d_flags;
    fa.flag_cap = h->flag_cap;
    fa.shift_out = h->d_shift;
    fa.force_coef = 0;
    fa.gA = nullptr;
    fa.gS = nullptr;
    fa.geps = nullptr;
    fa.status = h->d_status;
    fa.nonfinite = h->d_count + 1;
    dim3 grid((W + flr::kTW - 1) / flr::kTW, (H + fa.TH - 1) / fa.TH);
    FLR_CUDA(mark(h, s), "timing event");
    FLR_CUDA(flr::launch_fwd(q, fa, grid, h->fwd_smem, s), "forward kernel launch");
    ++h->n_fwd;
    FLR_CUDA(mark(h, s), "timing event");

    if (h->p.pivot_ratio > 0.f) {
        flr::Fp64Args da;
        da.guide = guide;
        da.map_guide = map_guide;
        da.rad = radiance;
        da.shift = h->d_shift;
        da.out = out;
        da.coef = h->d_coef;
        da.H = H;
        da.W = W;
        da.r = h->p.radius;
        da.rc = h->p.coef_radius;
        da.eps = (double)h->p.eps;
        da.flag_count = h->d_count;
        da.flag_list = h->d_flags;
        da.flag_cap = h->flag_cap;
        da.force_coef = 0;
        da.nonfinite = h->d_count + 1;
        FLR_CUDA(flr::launch_fp64(q, da, h->n_sm, s), "fp64 re-solve launch");
        ++h->n_fp64;
    }
    FLR_CUDA(mark(h, s), "timing event");
    if (h->p.coef_radius > 0) {
        flr::ApplyArgs aa;
        aa.coef = h->d_coef;
        aa.map_guide = map_guide ? map_guide : guide;
        aa.shift = h->d_shift;
        aa.out = out;
        aa.H = H;
        aa.W = W;
        aa.rc = h->p.coef_radius;
        aa.status = h->d_status;
        aa.nonfinite = h->d_count + 1;
        FLR_CUDA(flr::launch_apply(q, aa, s), "apply kernel launch");
        ++h->n_apply;
    }
    FLR_CUDA(mark(h, s), "timing event");
    return FLR_OK;
}

int flr_backward(flr_handle *h, const float *guide, const float *map_guide, const float *radiance,
                 const float *grad_out, float *grad_guide, float *grad_map_guide, float *grad_radiance,
                 double *grad_eps, int H, int W, void *stream)
{
    if (!h || !guide || !radiance || !grad_out || !grad_guide || !grad_radiance || H <= 0 || W <= 0)
        return FLR_ERR_ARG;
    if ((long long)H * W > 0x7fffffffLL) return FLR_ERR_ARG;
    if (!aligned16(guide) || !aligned16(radiance) || !aligned16(grad_out) || !aligned16(grad_guide) ||
        !aligned16(grad_radiance) || (map_guide && !aligned16(map_guide)) ||
        (grad_map_guide && !aligned16(grad_map_guide)))
        return FLR_ERR_ALIGN;
    const int q = h->p.q;
    const int nch = q + 3 + q * (q + 1) / 2 + 3 * q;
    const int ncf = 3 * (q + 1);
    const size_t px = (size_t)H * W;
    int st = grow(h, H, W);
    if (st != FLR_OK) return st;
    if (h->bwd_px < px || !h->bwd) {
        cudaFree(h->bwd);
        h->bwd = nullptr;
        h->bwd_px = 0;
        const size_t planes = 3 * (size_t)(3 * (FLR_MAX_Q + 1)) + 2 * (size_t)(FLR_MAX_Q + 3 + FLR_MAX_Q * (FLR_MAX_Q + 1) / 2 + 3 * FLR_MAX_Q);
        if (cudaMalloc(&h->bwd, px * planes * sizeof(float)) != cudaSuccess) return FLR_ERR_NOMEM;
        h->bwd_px = px;
    }
    float *Acoef = h->bwd;                 // per-pixel models A_k
    float *F = Acoef + (size_t)ncf * px;   // fields, later the box-averaged models
    float *GA = F + (size_t)ncf * px;      // G(A_k)
    float *GS = GA + (size_t)ncf * px;     // per-pixel moment gradients
    float *BS = GS + (size_t)nch * px;     // their window sums
    cudaStream_t s = (cudaStream_t)stream;
    h->last_stream = s;
    const int r = h->p.radius, rc = h->p.coef_radius;

    // 1. the frame reference shift (the fields need it before the adjoint kernel runs)
    FLR_CUDA(cudaMemsetAsync(h->d_count, 0, 2 * sizeof(unsigned long long), s), "reset counters");
    FLR_CUDA(flr::launch_frame_shift(q, guide, radiance, H, W, 0, h->d_shift, s), "backward: frame shift launch");
    flr::FwdArgs fa;
    fa.guide = guide;
    fa.map_guide = map_guide;
    fa.rad = radiance;
    fa.out = nullptr;
    fa.coef = Acoef;
    fa.H = H;
    fa.W = W;
    fa.r = r;
    fa.rc = rc;
    fa.eps = h->p.eps;
    fa.tau = h->p.pivot_ratio;
    fa.TH = choose_segment_rows(H, W, r, h->n_sm);
    fa.flag_count = h->d_count;
    fa.flag_list = h->d_flags;
    fa.flag_cap = h->flag_cap;
    fa.shift_out = h->d_shift;
    fa.force_coef = 1;
    fa.gA = nullptr;
    fa.gS = nullptr;
    fa.geps = nullptr;
    fa.status = h->d_status;
    dim3 grid((W + flr::kTW - 1) / flr::kTW, (H + fa.TH - 1) / fa.TH);
    flr::Fp64Args da;
    const bool fp64_fix = h->p.pivot_ratio > 0.f;
    if (fp64_fix) {
        da.guide = guide;
        da.map_guide = map_guide;
        da.rad = radiance;
        da.shift = h->d_shift;
        da.out = nullptr;
        da.coef = Acoef;
        da.H = H;
        da.W = W;
        da.r = r;
        da.rc = rc;
        da.eps = (double)h->p.eps;
        da.flag_count = h->d_count;
        da.flag_list = h->d_flags;
        da.flag_cap = h->flag_cap;
        da.force_coef = 1;
    }
    // 2. adjoint of the apply and of the average: G(A_k)
    const float *z = map_guide ? map_guide : guide;
    FLR_CUDA(flr::launch_bwd_fields(q, grad_out, z, h->d_shift, F, H, W, rc, s), "backward: fields launch");
    const float *gA = F;
    if (rc > 0) {
        FLR_CUDA(flr::launch_box_sum(F, GA, ncf, H, W, rc, s, h->d_status), "backward: average adjoint launch");
        gA = GA;
    }
    // 3. per-pixel adjoint solve (moments recomputed) -> GS, d/d eps
    if (grad_eps) FLR_CUDA(cudaMemsetAsync(grad_eps, 0, sizeof(double), s), "backward: reset eps gradient");
    double *geps = grad_eps;
    if (!geps) {
        geps = (double *)(BS + (size_t)nch * px);  // unused slot at the end of the workspace
    }
    fa.gA = gA;
    fa.gS = GS;
    fa.geps = geps;
    fa.status = h->d_status;
    fa.force_coef = 0;
    // the adjoint kernel also writes each pixel's model A_k (coefficients relative to the frame
    // reference) and lists the pixels whose pivot fell low, whose models the FP64 re-solve
    // then replaces (these feed only the averaged models of the applied guide)
    FLR_CUDA(flr::launch_adj(q, fa, grid, h->adj_smem, s), "backward: adjoint kernel launch");
    if (fp64_fix) FLR_CUDA(flr::launch_fp64(q, da, h->n_sm, s), "backward: fp64 re-solve launch");
    // 4. adjoint of the window sums, the averaged models for the applied guide, contraction
    FLR_CUDA(flr::launch_box_sum(GS, BS, nch, H, W, r, s, h->d_status), "backward: window-sum adjoint launch");
    const float *BA = Acoef;
    if (rc > 0) {  // the averaged a (planes 3 .. ncf - 1); the contraction reads no averaged bias
        FLR_CUDA(flr::launch_box_sum(Acoef + 3 * px, F + 3 * px, ncf - 3, H, W, rc, s, h->d_status),
                 "backward: model average launch");
        BA = F;
    }
    flr::BwdArgs ba;
    ba.guide = guide;
    ba.rad = radiance;
    ba.shift = h->d_shift;
    ba.g = grad_out;
    ba.BS = BS;
    ba.BA = BA;
    ba.grad_guide = grad_guide;
    ba.grad_map = grad_map_guide;
    ba.grad_rad = grad_radiance;
    ba.H = H;
    ba.W = W;
    ba.rc = rc;
    ba.separate_map = map_guide != nullptr;
    FLR_CUDA(flr::launch_bwd_contract(q, ba, s), "backward: contraction launch");
    return FLR_OK;
}

int flr_denoise_batch(flr_handle *h, int n, const flr_frame *frames, void *stream)
{
    if (!h || n <= 0 || !frames) return FLR_ERR_ARG;
    for (int i = 0; i < n; ++i) {
        const flr_frame &f = frames[i];
        int st = flr_denoise(h, f.guide, f.map_guide, f.radiance, f.out, f.H, f.W, stream);
        if (st != FLR_OK) return st;
    }
    return FLR_OK;
}

int flr_denoise_host(flr_handle *h, const float *guide, const float *map_guide,
                     const float *radiance, float *out, int H, int W, void *stream)
{
    if (!h || !guide || !radiance || !out || H <= 0 || W <= 0) return FLR_ERR_ARG;
    if ((long long)H * W > 0x7fffffffLL) return FLR_ERR_ARG;
    const int q = h->p.q, r = h->p.radius, rc = h->p.coef_radius;
    const size_t px = (size_t)H * W;
    if (int st = flr_host_wait(h)) return st;  // frames queued by flr_denoise_host_async
    if (h->stage_px < px || !h->stage) {
        cudaFree(h->stage);
        h->stage = nullptr;
        h->stage_px = 0;
        if (cudaMalloc(&h->stage, staging_floats(px, FLR_MAX_Q) * sizeof(float)) != cudaSuccess)
            return FLR_ERR_NOMEM;
        h->stage_px = px;
    }
    cudaStream_t s = (cudaStream_t)stream;
    float *dg, *dm, *dr, *dout;
    staging_regions(h->stage, px, q, &dg, &dm, &dr, &dout);
    // Row bands: the copy of band k + 1 overlaps the kernels of band k, whose output copy
    // overlaps the kernels of band k + 1 (separate copy-in and copy-out streams).  Band k's
    // kernels compute the models of rows [c_k, c_k+1) from input rows up to c_k+1 + r and
    // apply the averaged models to rows [c_k - rc, c_k+1 - rc); each band has its own segment
    // height.  One band (small frames) is exactly flr_denoise.  The bands: band_plan.
    int c[FLR_HOST_MAX_BANDS + 1], in_end[FLR_HOST_MAX_BANDS + 1], o[FLR_HOST_MAX_BANDS + 1];
    const int K = band_plan(H, r, rc, c, in_end, o);
    if (K == 1) {
        FLR_CUDA(cudaMemcpyAsync(dg, guide, sizeof(float) * q * px, cudaMemcpyHostToDevice, s), "h2d guide");
        if (map_guide)
            FLR_CUDA(cudaMemcpyAsync(dm, map_guide, sizeof(float) * q * px, cudaMemcpyHostToDevice, s), "h2d map guide");
        FLR_CUDA(cudaMemcpyAsync(dr, radiance, sizeof(float) * 3 * px, cudaMemcpyHostToDevice, s), "h2d radiance");
        int st = flr_denoise(h, dg, map_guide ? dm : nullptr, dr, dout, H, W, stream);
        if (st != FLR_OK) return st;
        FLR_CUDA(cudaMemcpyAsync(out, dout, sizeof(float) * 3 * px, cudaMemcpyDeviceToHost, s), "d2h out");
        FLR_CUDA(cudaStreamSynchronize(s), "host-path synchronise");
        return FLR_OK;
    }
    if (!fused_ok(h->p, H, W, dg, map_guide ? dm : nullptr, dr, dout)) {
        int st = grow(h, H, W);
        if (st != FLR_OK) return st;
    }
    if (!h->d_fstart) {
        if (int st = copy_streams(h)) return st;
        FLR_CUDA(cudaMalloc(&h->d_fstart, sizeof(unsigned long long)), "re-solve index");
        h->band_ev.resize(2 * FLR_HOST_MAX_BANDS + 1);
        for (auto &e : h->band_ev) FLR_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "band event");
    }
    const size_t plane_b = px * sizeof(float);
    cudaEvent_t e_start = h->band_ev[2 * FLR_HOST_MAX_BANDS];
    // the copies start after the work already queued on the caller's stream
    FLR_CUDA(cudaEventRecord(e_start, s), "band event");
    FLR_CUDA(cudaStreamWaitEvent(h->s_in, e_start, 0), "band wait");
    FLR_CUDA(cudaMemsetAsync(h->d_count, 0, 2 * sizeof(unsigned long long), s), "reset counters");
    FLR_CUDA(cudaMemsetAsync(h->d_fstart, 0, sizeof(unsigned long long), s), "reset counter");
    h->last_stream = s;
    for (int k = 0; k < K; ++k) {
        // copy in input rows [in_end[k], in_end[k+1]) of every plane (2-D copies: rows of
        // one band across the planes of a tensor)
        const int ra = in_end[k], rb = in_end[k + 1];
        if (rb > ra) {
            const size_t off = (size_t)ra * W * sizeof(float), bytes = (size_t)(rb - ra) * W * sizeof(float);
            FLR_CUDA(cudaMemcpy2DAsync((char *)dg + off, plane_b, (const char *)guide + off, plane_b, bytes, q,
                                       cudaMemcpyHostToDevice, h->s_in), "h2d guide band");
            if (map_guide)
                FLR_CUDA(cudaMemcpy2DAsync((char *)dm + off, plane_b, (const char *)map_guide + off, plane_b, bytes, q,
                                           cudaMemcpyHostToDevice, h->s_in), "h2d map guide band");
            FLR_CUDA(cudaMemcpy2DAsync((char *)dr + off, plane_b, (const char *)radiance + off, plane_b, bytes, 3,
                                       cudaMemcpyHostToDevice, h->s_in), "h2d radiance band");
        }
        FLR_CUDA(cudaEventRecord(h->band_ev[2 * k], h->s_in), "band event");
        FLR_CUDA(cudaStreamWaitEvent(s, h->band_ev[2 * k], 0), "band wait");
        if (fused_ok(h->p, H, W, dg, map_guide ? dm : nullptr, dr, dout)) {  // outputs [o_k, o_k+1) in one pass
            int sf = run_fused(h, dg, map_guide ? dm : nullptr, dr, dout, H, W, o[k], o[k + 1], s);
            if (sf != FLR_OK) return sf;
            FLR_CUDA(cudaEventRecord(h->band_ev[2 * k + 1], s), "band event");
            FLR_CUDA(cudaStreamWaitEvent(h->s_out, h->band_ev[2 * k + 1], 0), "band wait");
            const int oa = o[k], ob = o[k + 1];
            if (ob > oa) {
                const size_t off = (size_t)oa * W * sizeof(float), bytes = (size_t)(ob - oa) * W * sizeof(float);
                FLR_CUDA(cudaMemcpy2DAsync((char *)out + off, plane_b, (const char *)dout + off, plane_b, bytes, 3,
                                           cudaMemcpyDeviceToHost, h->s_out), "d2h out band");
            }
            continue;
        }
        h->last_fused = false;
        // models of rows [c_k, c_k+1)
        flr::FwdArgs fa;
        fa.guide = dg;
        fa.map_guide = map_guide ? dm : nullptr;
        fa.rad = dr;
        fa.out = dout;
        fa.coef = h->d_coef;
        fa.H = H;
        fa.W = W;
        fa.r = r;
        fa.rc = rc;
        fa.eps = h->p.eps;
        fa.tau = h->p.pivot_ratio;
        fa.TH = choose_segment_rows(c[k + 1] - c[k], W, r, h->n_sm);
        fa.flag_count = h->d_count;
        fa.flag_list = h->d_flags;
        fa.flag_cap = h->flag_cap;
        fa.shift_out = h->d_shift;
        fa.force_coef = 0;
        fa.gA = nullptr;
        fa.gS = nullptr;
        fa.geps = nullptr;
        fa.status = h->d_status;
        fa.nonfinite = h->d_count + 1;
        fa.row_lo = c[k];
        fa.row_hi = c[k + 1];
        fa.ref_rows = in_end[1];  // the reference comes from the first band's rows
        dim3 grid((W + flr::kTW - 1) / flr::kTW, (c[k + 1] - c[k] + fa.TH - 1) / fa.TH);
        FLR_CUDA(flr::launch_fwd(q, fa, grid, h->fwd_smem, s), "forward kernel launch");
        ++h->n_fwd;
        if (h->p.pivot_ratio > 0.f) {
            flr::Fp64Args da;
            da.guide = dg;
            da.map_guide = map_guide ? dm : nullptr;
            da.rad = dr;
            da.shift = h->d_shift;
            da.out = dout;
            da.coef = h->d_coef;
            da.H = H;
            da.W = W;
            da.r = r;
            da.rc = rc;
            da.eps = (double)h->p.eps;
            da.flag_count = h->d_count;
            da.flag_list = h->d_flags;
            da.flag_cap = h->flag_cap;
            da.force_coef = 0;
            da.nonfinite = h->d_count + 1;
            da.flag_start = h->d_fstart;  // only this band's flags
            FLR_CUDA(flr::launch_fp64(q, da, h->n_sm, s), "fp64 re-solve launch");
            FLR_CUDA(cudaMemcpyAsync(h->d_fstart, h->d_count, sizeof(unsigned long long), cudaMemcpyDeviceToDevice, s),
                     "re-solve index");
            ++h->n_fp64;
        }
        if (rc > 0) {  // averaged models applied to rows [o_k, o_k+1)
            flr::ApplyArgs aa;
            aa.coef = h->d_coef;
            aa.map_guide = map_guide ? dm : dg;
            aa.shift = h->d_shift;
            aa.out = dout;
            aa.H = H;
            aa.W = W;
            aa.rc = rc;
            aa.status = h->d_status;
            aa.nonfinite = h->d_count + 1;
            aa.row_lo = o[k];
            aa.row_hi = o[k + 1];
            FLR_CUDA(flr::launch_apply(q, aa, s), "apply kernel launch");
            ++h->n_apply;
        }
        FLR_CUDA(cudaEventRecord(h->band_ev[2 * k + 1], s), "band event");
        // copy out output rows [o_k, o_k+1)
        FLR_CUDA(cudaStreamWaitEvent(h->s_out, h->band_ev[2 * k + 1], 0), "band wait");
        const int oa = o[k], ob = o[k + 1];
        if (ob > oa) {
            const size_t off = (size_t)oa * W * sizeof(float), bytes = (size_t)(ob - oa) * W * sizeof(float);
            FLR_CUDA(cudaMemcpy2DAsync((char *)out + off, plane_b, (const char *)dout + off, plane_b, bytes, 3,
                                       cudaMemcpyDeviceToHost, h->s_out), "d2h out band");
        }
    }
    FLR_CUDA(cudaStreamSynchronize(h->s_out), "host-path synchronise");
    FLR_CUDA(cudaStreamSynchronize(s), "host-path synchronise");
    return FLR_OK;
}

int flr_denoise_host_async(flr_handle *h, const float *guide, const float *map_guide,
                           const float *radiance, float *out, int H, int W, void *stream)
{
    if (!h || !guide || !radiance || !out || H <= 0 || W <= 0) return FLR_ERR_ARG;
    if ((long long)H * W > 0x7fffffffLL) return FLR_ERR_ARG;
    const int q = h->p.q;
    const size_t px = (size_t)H * W;
    cudaStream_t s = (cudaStream_t)stream;
    if (int st = copy_streams(h)) return st;
    for (int k = 0; k < 2; ++k)
        for (cudaEvent_t *ev : {&h->a_in[k], &h->a_comp[k], &h->a_out[k]})
            if (!*ev) FLR_CUDA(cudaEventCreateWithFlags(ev, cudaEventDisableTiming), "host-path event");
    const int k = h->a_next;
    if (h->aslot_px[k] < px) {
        // a larger frame: the frames in flight may still use the slot, so they finish first
        if (int st = flr_host_wait(h)) return st;
        cudaFree(h->aslot[k]);
        h->aslot[k] = nullptr;
        h->aslot_px[k] = 0;
        if (cudaMalloc(&h->aslot[k], staging_floats(px, q) * sizeof(float)) != cudaSuccess) return FLR_ERR_NOMEM;
        h->aslot_px[k] = px;
    }
    float *dg, *dm, *dr, *dout;
    staging_regions(h->aslot[k], px, q, &dg, &dm, &dr, &dout);
    h->a_pending = true;
    // inputs: into the slot once the frame that used it last has been computed
    FLR_CUDA(cudaStreamWaitEvent(h->s_in, h->a_comp[k], 0), "host-path wait");
    FLR_CUDA(cudaMemcpyAsync(dg, guide, sizeof(float) * q * px, cudaMemcpyHostToDevice, h->s_in), "h2d guide");
    if (map_guide)
        FLR_CUDA(cudaMemcpyAsync(dm, map_guide, sizeof(float) * q * px, cudaMemcpyHostToDevice, h->s_in),
                 "h2d map guide");
    FLR_CUDA(cudaMemcpyAsync(dr, radiance, sizeof(float) * 3 * px, cudaMemcpyHostToDevice, h->s_in), "h2d radiance");
    FLR_CUDA(cudaEventRecord(h->a_in[k], h->s_in), "host-path event");
    // kernels: after the inputs, and after the slot's previous result has been copied out
    FLR_CUDA(cudaStreamWaitEvent(s, h->a_in[k], 0), "host-path wait");
    FLR_CUDA(cudaStreamWaitEvent(s, h->a_out[k], 0), "host-path wait");
    int st = flr_denoise(h, dg, map_guide ? dm : nullptr, dr, dout, H, W, stream);
    if (st != FLR_OK) return st;
    FLR_CUDA(cudaEventRecord(h->a_comp[k], s), "host-path event");
    // result: copied out while the next frame's kernels run
    FLR_CUDA(cudaStreamWaitEvent(h->s_out, h->a_comp[k], 0), "host-path wait");
    FLR_CUDA(cudaMemcpyAsync(out, dout, sizeof(float) * 3 * px, cudaMemcpyDeviceToHost, h->s_out), "d2h out");
    FLR_CUDA(cudaEventRecord(h->a_out[k], h->s_out), "host-path event");
    h->a_next = k ^ 1;
    return FLR_OK;
}

int flr_host_wait(flr_handle *h)
{
    if (!h) return FLR_ERR_ARG;
    if (!h->a_pending) return FLR_OK;
    h->a_pending = false;
    // every result copy follows its frame's kernels, which follow its input copies; the
    // events of both slots cover a frame whose call returned early with an error
    for (int k = 0; k < 2; ++k)
        for (cudaEvent_t ev : {h->a_in[k], h->a_comp[k], h->a_out[k]})
            if (ev) FLR_CUDA(cudaEventSynchronize(ev), "host-path wait");
    return FLR_OK;
}

int flr_host_band_plan(int H, int radius, int coef_radius, int *c, int *in_end, int *out_lo)
{
    if (H <= 0 || radius < 0 || coef_radius < 0 || !c || !in_end || !out_lo) return FLR_ERR_ARG;
    return band_plan(H, radius, coef_radius, c, in_end, out_lo);
}

int flr_get_kernel_times(flr_handle *h, flr_kernel_times *out, int reset)
{
    if (!h || !out) return FLR_ERR_ARG;
    std::memset(out, 0, sizeof(*out));
    out->fwd_n = h->n_fwd;
    out->fp64_n = h->n_fp64;
    out->apply_n = h->n_apply;
    if (h->events_used >= 4) FLR_CUDA(cudaEventSynchronize(h->events[h->events_used - 1]), "timing sync");
    for (size_t i = 0; i + 4 <= h->events_used; i += 4) {
        float t[3];
        for (int k = 0; k < 3; ++k)
            FLR_CUDA(cudaEventElapsedTime(&t[k], h->events[i + k], h->events[i + k + 1]), "timing read");
        out->fwd_ms += t[0];
        out->fp64_ms += t[1];
        out->apply_ms += t[2];
    }
    if (reset) {
        h->events_used = 0;
        h->n_fwd = h->n_fp64 = h->n_apply = 0;
    }
    return FLR_OK;
}

int flr_get_stats(flr_handle *h, flr_stats *out)
{
    if (!h || !out) return FLR_ERR_ARG;
    unsigned long long cnt[2] = {0ull, 0ull};
    FLR_CUDA(cudaStreamSynchronize(h->last_stream), "stats synchronise");
    FLR_CUDA(cudaMemcpy(cnt, h->d_count, sizeof(cnt), cudaMemcpyDeviceToHost), "stats copy");
    const unsigned long long n = cnt[0];
    out->flagged = n;
    out->nonfinite = cnt[1];
    if (h->last_fused)  // the fused path lists every flagged pixel: no capacity limit
        out->resolved = h->p.pivot_ratio > 0.f ? n : 0ull;
    else
        out->resolved = h->p.pivot_ratio > 0.f ? (n < (unsigned long long)h->flag_cap ? n : (unsigned long long)h->flag_cap) : 0ull;
    int status = 0;
    FLR_CUDA(cudaMemcpy(&status, h->d_status, sizeof(int), cudaMemcpyDeviceToHost), "stats copy");
    if (status != 0) {
        FLR_CUDA(cudaMemset(h->d_status, 0, sizeof(int)), "stats reset");
        return FLR_ERR_TIMEOUT;
    }
    return FLR_OK;
}

}  // extern "C"
