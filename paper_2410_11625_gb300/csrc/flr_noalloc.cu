// flr_noalloc.cu -- flr_denoise_noalloc: the FLR pass for callers that cannot allocate
// device memory.
//
// flr_denoise needs a handle, and a handle allocates its workspace (the coefficient planes
// and the flag list) with cudaMalloc.  Some callers cannot do that: code running where the
// device allocator must not be touched (inside a custom allocator or a memory-pool
// callback, under a host that forbids late allocations after start-up, or a plugin that
// only receives buffers from its host application).  This entry point takes the same
// inputs and output but keeps its workspace in one file-scope __device__ array, so no call
// allocates or frees anything.  The array lives in every GPU that loads the library until
// the process exits.
//
// Limits and sharing: frames of at most FLR_NOALLOC_MAX_PIXELS pixels; every call on a
// device uses the same array and leaves the last call's contents in it, so calls that
// overlap on the GPU (two streams, two threads) race and must be serialised by the caller.
// The flag counter, the only part that must start at zero, is cleared by every call.
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
constexpr size_t kOffCount = 0;                                                // 1 x u64
constexpr size_t kOffShift = 256;                                              // FLR_MAX_Q + 3 floats
constexpr size_t kOffFlags = 512;                                              // kMaxPx ints
constexpr size_t kOffCoef = align256(kOffFlags + kMaxPx * sizeof(int));        // (Q+1)*3 planes
constexpr size_t kBytes = align256(kOffCoef + kMaxPx * (FLR_MAX_Q + 1) * 3 * sizeof(float));

static __device__ __align__(256) unsigned char g_noalloc_scratch[kBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char *g_scratch_ptr[kMaxDevices];  // device address of the array, per device
int g_n_sm[kMaxDevices];
size_t g_smem_ready[kMaxDevices][FLR_MAX_Q + 1];  // forward-kernel shared memory configured
int g_smem_radius[kMaxDevices][FLR_MAX_Q + 1];     // ... for the kernel of this radius

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

int segment_rows(int H, int W, int r, int n_sm)
{
    const int strips = (W + flr::kTW - 1) / flr::kTW;
    int best_th = H;
    long long best = -1;
    for (int segs = 1; segs <= 256; ++segs) {
        int th = (H + segs - 1) / segs;
        th = (th + flr::kB - 1) / flr::kB * flr::kB;
        const long long waves = ((long long)strips * ((H + th - 1) / th) + n_sm - 1) / n_sm;
        const long long cost = waves * (th + 2 * r);
        if (best < 0 || cost < best) { best = cost; best_th = th; }
        if (th <= flr::kB) break;
    }
    return best_th;
}

}  // namespace

extern "C" int flr_denoise_noalloc(const flr_params *p, const float *guide, const float *map_guide,
                                   const float *radiance, float *out, int H, int W, void *stream)
{
    if (!p || !guide || !radiance || !out || H <= 0 || W <= 0) return FLR_ERR_ARG;
    if ((p->flags & ~FLR_FLAG_TIMING) != 0u || !(p->eps >= 0.f) || p->radius < 0 || p->coef_radius < 0 ||
        p->pivot_ratio != p->pivot_ratio)
        return FLR_ERR_ARG;
    if (p->q < 1 || p->q > FLR_MAX_Q || p->radius > FLR_MAX_RADIUS || p->coef_radius > FLR_MAX_COEF_RADIUS)
        return FLR_ERR_UNSUPPORTED;
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
    int st = setup_device(dev);
    if (st != FLR_OK) return st;
    const int q = p->q;
    const size_t smem = flr::fwd_smem_bytes(q, p->radius);
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (g_smem_ready[dev][q] < smem || g_smem_radius[dev][q] != p->radius) {
            if (flr::fwd_prepare(q, p->radius, smem) != cudaSuccess) return FLR_ERR_CUDA;
            g_smem_ready[dev][q] = smem;
            g_smem_radius[dev][q] = p->radius;
        }
    }
    unsigned char *base = g_scratch_ptr[dev];
    auto *count = (unsigned long long *)(base + kOffCount);
    auto *shift = (float *)(base + kOffShift);
    auto *flags = (int *)(base + kOffFlags);
    auto *coef = (float *)(base + kOffCoef);
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemsetAsync(count, 0, sizeof(unsigned long long), s) != cudaSuccess) return FLR_ERR_CUDA;

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
    fa.TH = segment_rows(H, W, p->radius, g_n_sm[dev]);
    fa.flag_count = count;
    fa.flag_list = flags;
    fa.flag_cap = (int)kMaxPx;
    fa.shift_out = shift;
    fa.force_coef = 0;
    fa.gA = nullptr;
    fa.gS = nullptr;
    fa.geps = nullptr;
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
        aa.status = nullptr;
        if (flr::launch_apply(q, aa, s) != cudaSuccess) return FLR_ERR_CUDA;
    }
    return FLR_OK;
}
