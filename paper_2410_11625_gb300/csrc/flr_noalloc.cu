// flr_noalloc.cu -- flr_denoise_noalloc: the FLR pass for callers that cannot allocate
// device memory.
//
// flr_denoise needs a handle, and a handle allocates its workspace (flag lists, coefficient
// planes) with cudaMalloc.  Some callers cannot do that: code running where the device
// allocator must not be touched (inside a custom allocator or a memory-pool callback, under a
// host that forbids late allocations after start-up, or a plugin that only receives buffers
// from its host application).  This entry point takes the same inputs and output but keeps
// its workspace in one file-scope __device__ array, so no call allocates or frees anything.
// The array lives in every GPU that loads the library until the process exits.
//
// It runs the same kernels as flr_denoise: the fused forward kernel and its FP64 correction
// where that path applies, otherwise the forward, FP64 re-solve and apply kernels; the two
// paths share the array's large region (only one runs per call).
//
// Limits and sharing: frames of at most FLR_NOALLOC_MAX_PIXELS pixels; every call on a device
// uses the same array and leaves the last call's contents in it, so calls that overlap on the
// GPU (two streams, two threads) race and must be serialised by the caller.  The counters and
// the status word, the parts that must start at zero, are cleared by every call.
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <mutex>

#include "flr.h"
#include "flr_internal.cuh"

namespace {

// workspace layout inside the array (byte offsets, each 256-byte aligned)
constexpr size_t kMaxPx = FLR_NOALLOC_MAX_PIXELS;
constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kOffCount = 0;    // 2 x u64: flagged pixels, non-finite output values
constexpr size_t kOffStatus = 16;  // int: a bounded device wait ran out
constexpr size_t kOffShift = 256;  // FLR_MAX_Q + 3 floats (frame reference of the unfused path)
constexpr size_t kOffFlags = 512;  // kMaxPx ints (flag list of the unfused path)
constexpr size_t kOffBig = align256(kOffFlags + kMaxPx * sizeof(int));
// the large region: the unfused path's (Q+1)*3 coefficient planes, or the fused path's
// per-CTA entry counts, reference shifts and flag lists
constexpr size_t kBigBytes = kMaxPx * (FLR_MAX_Q + 1) * 3 * sizeof(float);
constexpr size_t kBytes = align256(kOffBig + kBigBytes);
constexpr int kMaxFusedCta = 2048;
constexpr size_t kFusedCountBytes = align256(kMaxFusedCta * sizeof(int));
constexpr size_t kFusedShiftBytes = align256((size_t)kMaxFusedCta * (FLR_MAX_Q + 3) * sizeof(float));
constexpr size_t kFusedListInts = (kBigBytes - kFusedCountBytes - kFusedShiftBytes) / sizeof(int);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char *g_scratch_ptr[kMaxDevices];  // device address of the array, per device
int g_n_sm[kMaxDevices];

// Once per device, with that device current: the device address of the array (the host
// symbol is only a stand-in and must never reach a kernel) and the SM count.
int setup_device(int dev)
{
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (g_scratch_ptr[dev]) return FLR_OK;
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return FLR_ERR_CUDA;
    int n_sm = 0;
    e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return FLR_ERR_CUDA;
    g_n_sm[dev] = n_sm;
    g_scratch_ptr[dev] = (unsigned char *)p;
    return FLR_OK;
}

}  // namespace

extern "C" int flr_denoise_noalloc(const flr_params *p, const float *guide, const float *map_guide,
                                   const float *radiance, float *out, int H, int W, void *stream)
{
    if (!p || !guide || !radiance || !out || H <= 0 || W <= 0) return FLR_ERR_ARG;
    int st = flr::host::validate_params(p);
    if (st != FLR_OK) return st;
    if ((long long)H * W > (long long)kMaxPx) return FLR_ERR_UNSUPPORTED;  // beyond the array
    if (((uintptr_t)guide | (uintptr_t)radiance | (uintptr_t)out | (uintptr_t)map_guide) & 15u)
        return FLR_ERR_ALIGN;
    const size_t px = (size_t)H * W;
    auto overlaps = [&](const float *a, size_t n) {
        return a && (const char *)out < (const char *)(a + n) && (const char *)a < (const char *)(out + 3 * px);
    };
    if (overlaps(guide, (size_t)p->q * px) || overlaps(map_guide, (size_t)p->q * px) ||
        overlaps(radiance, 3 * px))
        return FLR_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return FLR_ERR_CUDA;
    st = setup_device(dev);
    if (st != FLR_OK) return st;
    const int q = p->q;
    unsigned char *base = g_scratch_ptr[dev];
    auto *count = (unsigned long long *)(base + kOffCount);
    auto *status = (int *)(base + kOffStatus);
    auto *shift = (float *)(base + kOffShift);
    auto *flags = (int *)(base + kOffFlags);
    unsigned char *big = base + kOffBig;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemsetAsync(base, 0, 32, s) != cudaSuccess) return FLR_ERR_CUDA;  // counters and status

    if (flr::host::fused_ok(*p, H, W, guide, map_guide, radiance, out)) {
        const flr::host::FusedPlan pl = flr::host::fused_plan(H, W, p->radius, p->coef_radius, g_n_sm[dev]);
        const int ncta = pl.strips * pl.segs;
        if (ncta <= kMaxFusedCta && (size_t)ncta * pl.cap <= kFusedListInts) {
            flr::FusedArgs fa;
            fa.guide = guide;
            fa.map_guide = map_guide;
            fa.rad = radiance;
            fa.out = out;
            fa.H = H;
            fa.W = W;
            fa.r = p->radius;
            fa.rc = p->coef_radius;
            fa.eps = p->eps;
            fa.tau = p->pivot_ratio;
            fa.TH = pl.TH;
            fa.row_lo = 0;
            fa.row_hi = H;
            fa.list_count = (int *)big;
            fa.cta_shift = (float *)(big + kFusedCountBytes);
            fa.list = (int *)(big + kFusedCountBytes + kFusedShiftBytes);
            fa.list_cap = p->pivot_ratio > 0.f ? pl.cap : 0;
            fa.flag_count = count;
            fa.nonfinite = count + 1;
            fa.status = status;
            const dim3 grid(pl.strips, pl.segs);
            if (flr::launch_fused(q, fa, grid, s) != cudaSuccess) return FLR_ERR_CUDA;
            if (p->pivot_ratio > 0.f && flr::launch_fused_fix(q, fa, grid, s) != cudaSuccess) return FLR_ERR_CUDA;
            return FLR_OK;
        }
    }

    auto *coef = (float *)big;
    const size_t smem = flr::fwd_smem_bytes(q, p->radius);
    if (flr::fwd_prepare(q, p->radius, smem) != cudaSuccess) return FLR_ERR_CUDA;
    flr::FwdArgs fa;
    fa.guide = guide;
    fa.map_guide = map_guide;
    fa.rad = radiance;
    fa.out = out;
    fa.coef = coef;
    fa.H = H;
    fa.W = W;
    fa.r = p->radius;
    fa.rc = p->coef_radius;
    fa.eps = p->eps;
    fa.tau = p->pivot_ratio;
    fa.TH = flr::host::choose_segment_rows(H, W, p->radius, g_n_sm[dev]);
    fa.flag_count = count;
    fa.flag_list = flags;
    fa.flag_cap = (int)kMaxPx;
    fa.shift_out = shift;
    fa.force_coef = 0;
    fa.gA = nullptr;
    fa.gS = nullptr;
    fa.geps = nullptr;
    fa.status = status;
    fa.nonfinite = count + 1;
    dim3 grid((W + flr::kTW - 1) / flr::kTW, (H + fa.TH - 1) / fa.TH);
    if (flr::launch_fwd(q, fa, grid, smem, s) != cudaSuccess) return FLR_ERR_CUDA;
    if (p->pivot_ratio > 0.f) {
        flr::Fp64Args da;
        da.guide = guide;
        da.map_guide = map_guide;
        da.rad = radiance;
        da.shift = shift;
        da.out = out;
        da.coef = coef;
        da.H = H;
        da.W = W;
        da.r = p->radius;
        da.rc = p->coef_radius;
        da.eps = (double)p->eps;
        da.flag_count = count;
        da.flag_list = flags;
        da.flag_cap = (int)kMaxPx;
        da.force_coef = 0;
        da.nonfinite = count + 1;
        if (flr::launch_fp64(q, da, g_n_sm[dev], s) != cudaSuccess) return FLR_ERR_CUDA;
    }
    if (p->coef_radius > 0) {
        flr::ApplyArgs aa;
        aa.coef = coef;
        aa.map_guide = map_guide ? map_guide : guide;
        aa.shift = shift;
        aa.out = out;
        aa.H = H;
        aa.W = W;
        aa.rc = p->coef_radius;
        aa.status = status;
        aa.nonfinite = count + 1;
        if (flr::launch_apply(q, aa, s) != cudaSuccess) return FLR_ERR_CUDA;
    }
    return FLR_OK;
}
