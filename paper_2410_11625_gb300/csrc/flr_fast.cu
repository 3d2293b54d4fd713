// flr_fast.cu -- the paper's fast FLR (Sec. 3.2) and its joint denoising and upsampling
// (Sec. 3.2.1) on sm_103a, behind the flr_fast_* entry points of include/flr.h.
//
// The paper's four steps, as four kernels:
//   1. block_moments: outer products of the shifted inputs summed over F x F blocks of the
//      input grid (the strided box filter);  one thread per input column walks the F rows
//      of its block row, then a shuffle tree over the F lanes of a block reduces them;
//   2. blur_h:  horizontal Gaussian over the block grid (one thread per channel and block);
//   3. blur_v_solve: vertical Gaussian, then the centred ridge model of every block in
//      registers (the window sums staged per thread in shared memory); a block whose
//      Cholesky pivot ratio falls to tau or below is re-solved in FP64 from the same sums;
//   4. apply: bilinear interpolation of the block models at every output pixel (output
//      grid s times finer than the input grid) and application to the map guide.
// Only step 1 and step 4 touch full-resolution data: the input is read once (44 B per
// input pixel for Q = 8), the map guide once and the output written once (32 + 12 B per
// output pixel); everything in between lives in (F^2)-times smaller planes that stay in L2.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <utility>
#include <vector>

#include "flr.h"
#include "flr_fast_stages.cuh"

namespace flr {
namespace {

using fast::FastArgs;
using fast::kMaxTaps;

template <int Q, int F>
__global__ void __launch_bounds__(256) block_moments_kernel(const FastArgs a)
{
    fast::stage_moments<Q, F>(a, blockIdx.y, blockIdx.x);
}

template <int Q>
__global__ void __launch_bounds__(128) blur_h_kernel(const FastArgs a)
{
    fast::stage_blur_h<Q>(a, (size_t)blockIdx.x * blockDim.x + threadIdx.x);
}

template <int Q>
__global__ void __launch_bounds__(128) blur_v_solve_kernel(const FastArgs a)
{
    extern __shared__ float sS[];  // [NCH][blockDim.x]
    fast::stage_blur_v_solve<Q>(a, (size_t)blockIdx.x * blockDim.x + threadIdx.x, sS + threadIdx.x, blockDim.x);
}

template <int Q>
__global__ void __launch_bounds__(256) fast_apply_kernel(const FastArgs a)
{
    const size_t runs = (size_t)a.Ho * (a.Wo / (a.F * a.s) + 2);
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < runs; t += (size_t)gridDim.x * blockDim.x)
        fast::stage_apply<Q>(a, t);
}

template <int Q>
cudaError_t launch_fast_q(const FastArgs &a, cudaStream_t st)
{
    dim3 g1((a.Wi + 255) / 256, a.Hb);
    switch (a.F) {
    case 2: block_moments_kernel<Q, 2><<<g1, 256, 0, st>>>(a); break;
    case 4: block_moments_kernel<Q, 4><<<g1, 256, 0, st>>>(a); break;
    case 8: block_moments_kernel<Q, 8><<<g1, 256, 0, st>>>(a); break;
    default: return cudaErrorInvalidValue;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t nb = (size_t)a.Hb * a.Wb;
    blur_h_kernel<Q><<<(unsigned)((nb + 127) / 128), 128, 0, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    blur_v_solve_kernel<Q><<<(unsigned)((nb + 127) / 128), 128, sizeof(float) * Chan<Q>::NCH * 128, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const size_t runs = (size_t)a.Ho * (a.Wo / (a.F * a.s) + 2);
    fast_apply_kernel<Q><<<(unsigned)((runs + 255) / 256 < 16384 ? (runs + 255) / 256 : 16384), 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_fast(int q, const FastArgs &a, cudaStream_t st)
{
    switch (q) {
    case 1: return launch_fast_q<1>(a, st);
    case 2: return launch_fast_q<2>(a, st);
    case 3: return launch_fast_q<3>(a, st);
    case 4: return launch_fast_q<4>(a, st);
    case 5: return launch_fast_q<5>(a, st);
    case 6: return launch_fast_q<6>(a, st);
    case 7: return launch_fast_q<7>(a, st);
    case 8: return launch_fast_q<8>(a, st);
    default: return cudaErrorInvalidValue;
    }
}

thread_local char g_fast_err[256] = "no error";

}  // namespace
}  // namespace flr

struct flr_fast_handle {
    flr_fast_params p;
    float w[2 * flr::fast::kMaxTaps + 1];
    float *ws = nullptr;  // block moments, blur temporary, block models
    size_t ws_blocks = 0;
    float *shift = nullptr;
    unsigned long long *count = nullptr;
    cudaStream_t last_stream = nullptr;
    // batch path: per-frame workspace, barrier words, status word
    float *bws = nullptr;
    size_t bws_floats = 0;
    unsigned *bar = nullptr;  // [0] count, [1] generation, [2] status
};

namespace {

size_t block_floats(int q) { return 2 * (size_t)(q + 3 + q * (q + 1) / 2 + 3 * q) + (size_t)(q + 3) + 1 + 3 * (size_t)(q + 1); }

// Fill one frame's arguments; ws points at its per-block workspace.
void frame_args(const flr_fast_handle *h, const flr_frame &fr, float *ws, flr::fast::FastArgs &a)
{
    const int q = h->p.q, F = h->p.factor, s = h->p.scale;
    const int Hb = (fr.H + F - 1) / F, Wb = (fr.W + F - 1) / F;
    const size_t nb = (size_t)Hb * Wb;
    const int nch = q + 3 + q * (q + 1) / 2 + 3 * q;
    a.guide = fr.guide;
    a.rad = fr.radiance;
    a.map_guide = fr.map_guide ? fr.map_guide : fr.guide;
    a.out = fr.out;
    a.blk = ws;
    a.tmp = ws + nb * (nch + q + 3);
    a.coef = a.tmp + nb * (nch + 1);
    a.shift = h->shift;  // replaced per frame by the caller
    a.flag_count = h->count;
    a.Hi = fr.H;
    a.Wi = fr.W;
    a.Ho = fr.H * s;
    a.Wo = fr.W * s;
    a.Hb = Hb;
    a.Wb = Wb;
    a.F = F;
    a.s = s;
    a.taps = h->p.taps;
    a.eps = h->p.eps;
    a.tau = h->p.pivot_ratio;
    std::memcpy(a.w, h->w, sizeof(a.w));
}

int check_frames(const flr_fast_handle *h, int n, const flr_frame *frames, size_t *floats)
{
    if (!h || n <= 0 || n > FLR_MAX_BATCH || !frames) return FLR_ERR_ARG;
    if (!flr::batch_supported(h->p.q, h->p.factor)) return FLR_ERR_UNSUPPORTED;
    size_t total = 0;
    for (int i = 0; i < n; ++i) {
        const flr_frame &f = frames[i];
        if (!f.guide || !f.radiance || !f.out || f.H <= 0 || f.W <= 0) return FLR_ERR_ARG;
        if (h->p.scale > 1 && !f.map_guide) return FLR_ERR_ARG;
        if ((long long)f.H * h->p.scale * f.W * h->p.scale > 0x7fffffffLL) return FLR_ERR_ARG;
        if (((uintptr_t)f.guide | (uintptr_t)f.radiance | (uintptr_t)f.out | (uintptr_t)f.map_guide) & 15u)
            return FLR_ERR_ALIGN;
        const size_t nb = (size_t)((f.H + h->p.factor - 1) / h->p.factor) * ((f.W + h->p.factor - 1) / h->p.factor);
        total += nb * block_floats(h->p.q) + 64;  // + room for the frame's reference shift
    }
    *floats = total;
    return FLR_OK;
}

}  // namespace

extern "C" {

int flr_fast_create(const flr_fast_params *p, flr_fast_handle **out)
{
    if (!out || !p) return FLR_ERR_ARG;
    *out = nullptr;
    if (p->flags != 0u || !(p->eps >= 0.f) || !(p->sigma > 0.f) || p->taps < 0 || p->scale < 1 ||
        p->pivot_ratio != p->pivot_ratio)
        return FLR_ERR_ARG;
    if (p->q < 1 || p->q > FLR_MAX_Q || p->taps > flr::fast::kMaxTaps || p->scale > 8 ||
        (p->factor != 2 && p->factor != 4 && p->factor != 8))
        return FLR_ERR_UNSUPPORTED;
    flr_fast_handle *h = new (std::nothrow) flr_fast_handle();
    if (!h) return FLR_ERR_NOMEM;
    h->p = *p;
    for (int d = -p->taps; d <= p->taps; ++d)
        h->w[d + p->taps] = (float)std::exp(-(double)d * d / (2.0 * (double)p->sigma * p->sigma));
    if (cudaMalloc(&h->shift, sizeof(float) * (FLR_MAX_Q + 3)) != cudaSuccess ||
        cudaMalloc(&h->count, sizeof(unsigned long long)) != cudaSuccess) {
        flr_fast_destroy(h);
        return FLR_ERR_NOMEM;
    }
    *out = h;
    return FLR_OK;
}

int flr_fast_destroy(flr_fast_handle *h)
{
    if (!h) return FLR_OK;
    cudaDeviceSynchronize();
    cudaFree(h->ws);
    cudaFree(h->bws);
    cudaFree(h->bar);
    cudaFree(h->shift);
    cudaFree(h->count);
    delete h;
    return FLR_OK;
}

int flr_fast_denoise(flr_fast_handle *h, const float *guide, const float *map_guide, const float *radiance,
                     float *out, int Hi, int Wi, void *stream)
{
    if (!h || !guide || !radiance || !out || Hi <= 0 || Wi <= 0) return FLR_ERR_ARG;
    const int s = h->p.scale, F = h->p.factor, q = h->p.q;
    if (s > 1 && !map_guide) return FLR_ERR_ARG;
    if ((long long)Hi * s * Wi * s > 0x7fffffffLL) return FLR_ERR_ARG;
    if (((uintptr_t)guide | (uintptr_t)radiance | (uintptr_t)out | (uintptr_t)map_guide) & 15u) return FLR_ERR_ALIGN;
    const int Hb = (Hi + F - 1) / F, Wb = (Wi + F - 1) / F;
    const size_t nb = (size_t)Hb * Wb;
    const int nch = q + 3 + q * (q + 1) / 2 + 3 * q;
    if (h->ws_blocks < nb || !h->ws) {
        cudaFree(h->ws);
        h->ws = nullptr;
        h->ws_blocks = 0;
        if (cudaMalloc(&h->ws, nb * sizeof(float) * (2 * (size_t)nch + (size_t)(q + 3) + 1 + 3 * (size_t)(q + 1))) != cudaSuccess)
            return FLR_ERR_NOMEM;
        h->ws_blocks = nb;
    }
    flr::fast::FastArgs a;
    a.guide = guide;
    a.rad = radiance;
    a.map_guide = map_guide ? map_guide : guide;
    a.out = out;
    a.blk = h->ws;
    a.tmp = h->ws + nb * (nch + q + 3);
    a.coef = a.tmp + nb * (nch + 1);
    a.shift = h->shift;
    a.flag_count = h->count;
    a.Hi = Hi;
    a.Wi = Wi;
    a.Ho = Hi * s;
    a.Wo = Wi * s;
    a.Hb = Hb;
    a.Wb = Wb;
    a.F = F;
    a.s = s;
    a.taps = h->p.taps;
    a.eps = h->p.eps;
    a.tau = h->p.pivot_ratio;
    std::memcpy(a.w, h->w, sizeof(a.w));
    cudaStream_t st = (cudaStream_t)stream;
    h->last_stream = st;
    cudaError_t e = cudaMemsetAsync(h->count, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = flr::launch_fast(q, a, st);
    if (e != cudaSuccess) {
        std::snprintf(flr::g_fast_err, sizeof(flr::g_fast_err), "%s", cudaGetErrorString(e));
        return FLR_ERR_CUDA;
    }
    return FLR_OK;
}

int flr_fast_reserve_batch(flr_fast_handle *h, int n, const flr_frame *frames)
{
    size_t floats = 0;
    int st = check_frames(h, n, frames, &floats);
    if (st != FLR_OK) return st;
    if (!h->bar && cudaMalloc(&h->bar, 4 * sizeof(unsigned)) != cudaSuccess) return FLR_ERR_NOMEM;
    if (h->bws_floats < floats || !h->bws) {
        cudaFree(h->bws);
        h->bws = nullptr;
        h->bws_floats = 0;
        if (cudaMalloc(&h->bws, floats * sizeof(float)) != cudaSuccess) return FLR_ERR_NOMEM;
        h->bws_floats = floats;
    }
    return FLR_OK;
}

int flr_fast_denoise_batch(flr_fast_handle *h, int n, const flr_frame *frames, void *stream)
{
    size_t floats = 0;
    int st = check_frames(h, n, frames, &floats);
    if (st != FLR_OK) return st;
    if (h->bws_floats < floats || !h->bar) {
        st = flr_fast_reserve_batch(h, n, frames);
        if (st != FLR_OK) return st;
    }
    flr::fast::FastArgs fa[FLR_MAX_BATCH];
    float *ws = h->bws;
    for (int i = 0; i < n; ++i) {
        frame_args(h, frames[i], ws + 64, fa[i]);
        fa[i].shift = ws;  // this frame's reference shift
        const size_t nb = (size_t)fa[i].Hb * fa[i].Wb;
        ws += nb * block_floats(h->p.q) + 64;
    }
    std::vector<unsigned char> args(flr::batch_args_size());
    flr::fill_batch_args(args.data(), n, fa, h->bar, h->bar + 1, (int *)(h->bar + 2));
    cudaStream_t s = (cudaStream_t)stream;
    h->last_stream = s;
    cudaError_t e = cudaMemsetAsync(h->count, 0, sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->bar, 0, 3 * sizeof(unsigned), s);
    if (e == cudaSuccess) e = flr::launch_batch(h->p.q, h->p.factor, args.data(), s);
    if (e != cudaSuccess) {
        std::snprintf(flr::g_fast_err, sizeof(flr::g_fast_err), "%s", cudaGetErrorString(e));
        return FLR_ERR_CUDA;
    }
    return FLR_OK;
}

int flr_fast_batch_status(flr_fast_handle *h)
{
    if (!h || !h->bar) return FLR_ERR_ARG;
    int status = 0;
    if (cudaStreamSynchronize(h->last_stream) != cudaSuccess ||
        cudaMemcpy(&status, h->bar + 2, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return FLR_ERR_CUDA;
    return status == 0 ? FLR_OK : FLR_ERR_TIMEOUT;
}

int flr_barrier_selftest(int ctas, unsigned long long timeout_ns, int *status)
{
    if (ctas <= 0 || ctas > 1024 || !status || timeout_ns > 10000000000ull) return FLR_ERR_ARG;
    unsigned *w = nullptr;
    if (cudaMalloc(&w, 4 * sizeof(unsigned)) != cudaSuccess) return FLR_ERR_NOMEM;
    cudaError_t e = cudaMemset(w, 0, 4 * sizeof(unsigned));
    if (e == cudaSuccess) e = flr::launch_barrier_selftest(w, w + 1, (unsigned)ctas + 1, (int *)(w + 2), timeout_ns, ctas, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(status, w + 2, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(w);
    return e == cudaSuccess ? FLR_OK : FLR_ERR_CUDA;
}

int flr_fast_get_stats(flr_fast_handle *h, flr_stats *out)
{
    if (!h || !out) return FLR_ERR_ARG;
    unsigned long long n = 0;
    if (cudaStreamSynchronize(h->last_stream) != cudaSuccess ||
        cudaMemcpy(&n, h->count, sizeof(n), cudaMemcpyDeviceToHost) != cudaSuccess)
        return FLR_ERR_CUDA;
    out->flagged = n;
    out->resolved = h->p.pivot_ratio > 0.f ? n : 0ull;
    return FLR_OK;
}

}  // extern "C"
