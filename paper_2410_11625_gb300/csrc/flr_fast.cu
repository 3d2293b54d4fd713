// flr_fast.cu -- the paper's fast FLR (Sec. 3.2) and its joint denoising and upsampling
// (Sec. 3.2.1) on sm_103a, behind the flr_fast_* entry points of include/flr.h.
//
// The paper's four steps, as four kernels:
//   1. block_moments: outer products of the shifted inputs summed over F x F blocks of the
//      input grid (the strided box filter);  one thread per pair of input columns walks the
//      F rows of its block row, then a shuffle tree over the F / 2 lanes of a block reduces
//      them;
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
#include "tma.cuh"

namespace flr {
namespace {

using fast::FastArgs;
using fast::kMaxTaps;

template <int Q, int F>
__global__ void __launch_bounds__(256, 2) block_moments_kernel(const FastArgs a)
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

// ---- parameter gradients (sigma and the regularisation terms) ---------------------------
template <int Q>
__global__ void __launch_bounds__(128) blur_v_tangent_kernel(const FastArgs a)
{
    extern __shared__ float sS[];  // [2][NCH][blockDim.x]: blurred sums, their sigma-derivative
    fast::stage_blur_v_tangent<Q>(a, (size_t)blockIdx.x * blockDim.x + threadIdx.x, sS + threadIdx.x,
                                  sS + Chan<Q>::NCH * blockDim.x + threadIdx.x, blockDim.x);
}

// Deterministic dot product: kDotBlocks partial sums in double (each thread strides through
// the data in a fixed order, then a fixed tree per CTA), summed by one CTA in a fixed tree.
constexpr int kDotBlocks = 256;
__global__ void __launch_bounds__(256) dot_partial_kernel(const float *x, const float *y, size_t n, double *part)
{
    __shared__ double sp[256];
    double acc = 0.0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        acc += (double)x[i] * (double)y[i];
    sp[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sp[threadIdx.x] += sp[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sp[0];
}

__global__ void __launch_bounds__(256) dot_final_kernel(const double *part, double *out)
{
    __shared__ double sp[kDotBlocks];
    sp[threadIdx.x] = part[threadIdx.x];
    __syncthreads();
    for (int o = kDotBlocks / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sp[threadIdx.x] += sp[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sp[0];
}

// ---- TMA version of the apply stage (rows 16-byte aligned) ------------------------------
//
// Persistent CTAs walk work items of kFW output columns; each item's map-guide rows arrive
// by one TMA box copy into a two-stage ring (the next item loads while the current one is
// computed), so the bytes in flight do not depend on registers per thread.  The copy
// engine zero-fills outside the image.  Waits are bounded (1 s) and report through the
// status word.
constexpr int kFW = 128;
constexpr unsigned long long kFastTimeoutNs = 1000000000ull;

struct alignas(128) FastKArgs {
    CUtensorMap t0;  // map-guide planes [Q][Ho][Wo], box (kFW, P, Q)
    FastArgs a;
};

__device__ __forceinline__ float *align128(float *p)
{
    return p + (((128 - (tma::smem_addr(p) & 127)) & 127) >> 2);
}

// Stage 4 with TMA: item (cell row i, column chunk cx).  Cell row i is the P = F s output
// rows [P i - P/2, P i + P/2), which all interpolate between the same two block rows; the
// item loads those rows of the Q map-guide planes.  Thread t owns output column kFW cx + t:
// it interpolates its corner models horizontally once per item (top and bottom block row),
// then for each row vertically, and applies them.  The coordinates are the exact rational
// ones of fast::stage_apply.
template <int Q>
__global__ void __launch_bounds__(kFW, 3) apply_tma_kernel(const __grid_constant__ FastKArgs k)
{
    constexpr int NC = 3 * (Q + 1), PMAX = 8, STAGE = Q * PMAX * kFW;
    const FastArgs &a = k.a;
    extern __shared__ __align__(16) float smem[];
    float *base = align128(smem);
    uint64_t *bar = reinterpret_cast<uint64_t *>(base + 2 * STAGE);
    __shared__ int s_abort;
    const int tid = threadIdx.x, lane = tid & 31;
    const int P = a.F * a.s, den = 2 * P;
    const int ncx = (a.Wo + kFW - 1) / kFW, nitems = (a.Hb + 1) * ncx;
    const size_t oplane = (size_t)a.Ho * a.Wo, bplane = (size_t)a.Hb * a.Wb;
    if (tid == 0) {
        s_abort = 0;
        tma::mbar_init(bar, 1);
        tma::mbar_init(bar + 1, 1);
        tma::mbar_init_fence();
    }
    __syncthreads();
    auto issue = [&](int item, int st) {
        const int ci = item / ncx, cx = item % ncx;
        tma::mbar_expect_tx(bar + st, (unsigned)(Q * P * kFW * 4));
        tma::load_3d_hint(base + st * STAGE, &k.t0, cx * kFW, P * ci - P / 2, 0, bar + st, fast::l2_policy_stream());
    };
    if (tid == 0 && (int)blockIdx.x < nitems) issue(blockIdx.x, 0);
    float sh[Q + 3];
#pragma unroll
    for (int q = 0; q < Q + 3; ++q) sh[q] = a.shift[q];
    int it = 0;
    for (int item = blockIdx.x; item < nitems; item += gridDim.x, ++it) {
        const int st = it & 1;
        if (tid == 0 && item + (int)gridDim.x < nitems) {
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            issue(item + gridDim.x, st ^ 1);
        }
        if (!tma::wait_warp(bar + st, (uint32_t)((it >> 1) & 1), kFastTimeoutNs) && lane == 0) {
            s_abort = 1;
            if (a.status) atomicExch(a.status, 1);
        }
        __syncthreads();
        if (s_abort) break;
        const float *T = base + st * STAGE;  // [Q][P][kFW]
        const int ci = item / ncx, cx = item % ncx;
        const int x = cx * kFW + tid;
        const int ya = P * ci - P / 2;       // first output row of the cell (may be < 0)
        if (x < a.Wo) {
            // block rows of the cell (the same for all its rows)
            const int yfirst = max(ya, 0);
            const int ny0 = min(max(2 * yfirst + 1 - P, 0), (a.Hb - 1) * den);
            const int i0 = min(ny0 / den, max(a.Hb - 2, 0)), i1 = min(i0 + 1, a.Hb - 1);
            // block columns and weight of this column
            const int r = (x + P / 2) / P;
            const int jl = min(max(r - 1, 0), a.Wb - 1), jr = min(max(r, 0), a.Wb - 1);
            const int nx = min(max(2 * x + 1 - P, 0), (a.Wb - 1) * den);
            const float fx = fminf(fmaxf((float)(nx - (r - 1) * den) / (float)den, 0.f), 1.f);
            float top[NC], dtb[NC];  // horizontally interpolated top row, bottom minus top
            {
                const size_t t0 = (size_t)i0 * a.Wb, t1 = (size_t)i1 * a.Wb;
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    const float *pc = a.coef + c * bplane;
                    const float l0 = __ldg(pc + t0 + jl), l1 = __ldg(pc + t1 + jl);
                    const float d0 = __ldg(pc + t0 + jr) - l0, d1 = __ldg(pc + t1 + jr) - l1;
                    top[c] = fmaf(fx, d0, l0);
                    dtb[c] = fmaf(fx, d1, l1) - top[c];
                }
            }
            for (int t = 0; t < P; ++t) {
                const int yo = ya + t;
                if (yo < 0 || yo >= a.Ho) continue;
                const int ny = min(max(2 * yo + 1 - P, 0), (a.Hb - 1) * den);
                const float fy = (float)(ny - i0 * den) / (float)den;
                float z[Q];
#pragma unroll
                for (int i = 0; i < Q; ++i) z[i] = T[(i * P + t) * kFW + tid] - sh[i];
                const size_t off = (size_t)yo * a.Wo + x;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    float o = fmaf(fy, dtb[c], top[c]);
#pragma unroll
                    for (int i = 0; i < Q; ++i) {
                        const int kk = 3 * (i + 1) + c;
                        o = fmaf(fmaf(fy, dtb[kk], top[kk]), z[i], o);
                    }
                    __stcs(a.out + c * oplane + off, o + sh[Q + c]);  // streamed: not kept in L2
                }
            }
        }
        __syncthreads();  // stage st is read; the next iteration may refill it
    }
}

template <int Q>
size_t apply_tma_smem()
{
    return 128 + sizeof(float) * 2 * (size_t)Q * 8 * kFW + 16;
}

int fast_n_sm()
{
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            n = 1;
    }
    return n;
}

template <int Q, int F>
cudaError_t launch_moments(const FastArgs &a, cudaStream_t st)
{
    dim3 g1(fast::moment_chunks(a.Wi), a.Hb);
    block_moments_kernel<Q, F><<<g1, 256, 0, st>>>(a);
    return cudaGetLastError();
}

template <int Q>
cudaError_t launch_apply_fast(const FastArgs &a, cudaStream_t st)
{
    const int P = a.F * a.s;
    const bool aligned = (a.Wo & 3) == 0 && ((uintptr_t)a.map_guide & 15) == 0 && P <= 8;
    if (aligned) {
        FastKArgs k;
        std::memset(&k, 0, sizeof(k));
        k.a = a;
        if (tma::encode_planes_f32(&k.t0, a.map_guide, a.Wo, a.Ho, Q, kFW, P, Q) == cudaSuccess) {
            const size_t smem = apply_tma_smem<Q>();
            cudaError_t e = cudaFuncSetAttribute(apply_tma_kernel<Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            // three CTAs per SM need the whole unified L1 / shared array as shared memory
            e = cudaFuncSetAttribute(apply_tma_kernel<Q>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)cudaSharedmemCarveoutMaxShared);
            if (e != cudaSuccess) return e;
            const int nitems = (a.Hb + 1) * ((a.Wo + kFW - 1) / kFW);
            const int grid = nitems < 3 * fast_n_sm() ? nitems : 3 * fast_n_sm();  // three CTAs per SM
            apply_tma_kernel<Q><<<grid, kFW, smem, st>>>(k);
            return cudaGetLastError();
        }
    }
    const size_t runs = (size_t)a.Ho * (a.Wo / (a.F * a.s) + 2);
    fast_apply_kernel<Q><<<(unsigned)((runs + 255) / 256 < 16384 ? (runs + 255) / 256 : 16384), 256, 0, st>>>(a);
    return cudaGetLastError();
}

template <int Q>
cudaError_t launch_fast_q(const FastArgs &a, cudaStream_t st)
{
    cudaError_t e;
    switch (a.F) {
    case 2: e = launch_moments<Q, 2>(a, st); break;
    case 4: e = launch_moments<Q, 4>(a, st); break;
    case 8: e = launch_moments<Q, 8>(a, st); break;
    default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    const size_t nb = (size_t)a.Hb * a.Wb;
    blur_h_kernel<Q><<<(unsigned)((nb + 127) / 128), 128, 0, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    blur_v_solve_kernel<Q><<<(unsigned)((nb + 127) / 128), 128, sizeof(float) * Chan<Q>::NCH * 128, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return launch_apply_fast<Q>(a, st);
}

// Parameter gradients of one frame: the forward's moments and horizontal blur, the
// horizontal blur with the weights' sigma-derivative, the tangent solve, then per parameter
// the apply of its model tangents (frame reference without the radiance offset, tshift) and
// the dot product with grad_out into grad[t].  dout: [3][Ho][Wo] scratch; part: kDotBlocks
// doubles.
template <int Q>
cudaError_t launch_param_grad_q(const FastArgs &a, float *tshift, const float *grad_out, float *dout,
                                double *part, double *grad, cudaStream_t st)
{
    cudaError_t e;
    switch (a.F) {
    case 2: e = launch_moments<Q, 2>(a, st); break;
    case 4: e = launch_moments<Q, 4>(a, st); break;
    case 8: e = launch_moments<Q, 8>(a, st); break;
    default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    const size_t nb = (size_t)a.Hb * a.Wb;
    const unsigned gb = (unsigned)((nb + 127) / 128);
    blur_h_kernel<Q><<<gb, 128, 0, st>>>(a);
    FastArgs ad = a;  // the horizontal blur with w' = dw/dsigma into tmp2
    ad.tmp = a.tmp2;
    std::memcpy(ad.w, a.wd, sizeof(ad.w));
    blur_h_kernel<Q><<<gb, 128, 0, st>>>(ad);
    const size_t smem = sizeof(float) * 2 * Chan<Q>::NCH * 128;
    static bool attr_set = false;
    if (!attr_set) {
        if ((e = cudaFuncSetAttribute(blur_v_tangent_kernel<Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
            cudaSuccess)
            return e;
        attr_set = true;
    }
    blur_v_tangent_kernel<Q><<<gb, 128, smem, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // the frame reference the moments wrote, with the radiance offset zero: a tangent of the
    // output carries no constant
    if ((e = cudaMemcpyAsync(tshift, a.shift, sizeof(float) * Q, cudaMemcpyDeviceToDevice, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(tshift + Q, 0, sizeof(float) * 3, st)) != cudaSuccess) return e;
    const size_t runs = (size_t)a.Ho * (a.Wo / (a.F * a.s) + 2);
    const size_t npx = 3 * (size_t)a.Ho * a.Wo;
    for (int t = 0; t < 3; ++t) {
        FastArgs at = a;
        at.coef = a.dcoef + (size_t)t * 3 * (Q + 1) * nb;
        at.shift = tshift;
        at.out = dout;
        fast_apply_kernel<Q><<<(unsigned)((runs + 255) / 256 < 16384 ? (runs + 255) / 256 : 16384), 256, 0, st>>>(at);
        dot_partial_kernel<<<kDotBlocks, 256, 0, st>>>(dout, grad_out, npx, part);
        dot_final_kernel<<<1, kDotBlocks, 0, st>>>(part, grad + t);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_param_grad(int q, const FastArgs &a, float *tshift, const float *grad_out, float *dout,
                              double *part, double *grad, cudaStream_t st)
{
    switch (q) {
    case 1: return launch_param_grad_q<1>(a, tshift, grad_out, dout, part, grad, st);
    case 2: return launch_param_grad_q<2>(a, tshift, grad_out, dout, part, grad, st);
    case 3: return launch_param_grad_q<3>(a, tshift, grad_out, dout, part, grad, st);
    case 4: return launch_param_grad_q<4>(a, tshift, grad_out, dout, part, grad, st);
    case 5: return launch_param_grad_q<5>(a, tshift, grad_out, dout, part, grad, st);
    case 6: return launch_param_grad_q<6>(a, tshift, grad_out, dout, part, grad, st);
    case 7: return launch_param_grad_q<7>(a, tshift, grad_out, dout, part, grad, st);
    case 8: return launch_param_grad_q<8>(a, tshift, grad_out, dout, part, grad, st);
    default: return cudaErrorInvalidValue;
    }
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

// Self-test of the bounded mbarrier wait the TMA and tensor-core kernels use: barrier 0
// expects two arrivals and receives one, so its phase never completes and every warp's wait
// must run out (status bit 0); barrier 1 expects one arrival and receives it, so the wait
// must succeed (a timeout there sets bit 1).
__global__ void mbarrier_selftest_kernel(int *status, unsigned long long timeout_ns)
{
    __shared__ uint64_t bar[2];
    if (threadIdx.x == 0) {
        tma::mbar_init(&bar[0], 2);
        tma::mbar_init(&bar[1], 1);
        tma::mbar_init_fence();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(tma::smem_addr(&bar[0])) : "memory");
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(tma::smem_addr(&bar[1])) : "memory");
    }
    __syncthreads();
    const bool done0 = tma::wait_warp(&bar[0], 0, timeout_ns);
    const bool done1 = tma::wait_warp(&bar[1], 0, timeout_ns);
    if ((threadIdx.x & 31) == 0) {
        if (!done0) atomicOr(status, 1);
        if (!done1) atomicOr(status, 2);
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
    int *status = nullptr;  // set by a kernel whose bounded wait ran out
    cudaStream_t last_stream = nullptr;
    // parameter gradients: sigma-derivative of the weights, workspace (second horizontal
    // blur, model tangents, frame reference without radiance offset, output tangent), partials
    float wd[2 * flr::fast::kMaxTaps + 1];
    float *gws = nullptr;
    size_t gws_floats = 0;
    double *gpart = nullptr;
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
    a.appendix = (h->p.flags & FLR_FAST_APPENDIX) ? 1 : 0;
    a.eps_mul = h->p.eps_mul;
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
    if ((p->flags & ~FLR_FAST_APPENDIX) != 0u || !(p->eps >= 0.f) || !(p->sigma > 0.f) || p->taps < 0 ||
        p->scale < 1 || p->pivot_ratio != p->pivot_ratio || !(p->eps_mul >= 0.f && p->eps_mul <= 1.f) ||
        (!(p->flags & FLR_FAST_APPENDIX) && p->eps_mul != 0.f))
        return FLR_ERR_ARG;
    if (p->q < 1 || p->q > FLR_MAX_Q || p->taps > flr::fast::kMaxTaps || p->scale > 8 ||
        (p->factor != 2 && p->factor != 4 && p->factor != 8))
        return FLR_ERR_UNSUPPORTED;
    flr_fast_handle *h = new (std::nothrow) flr_fast_handle();
    if (!h) return FLR_ERR_NOMEM;
    h->p = *p;
    for (int d = -p->taps; d <= p->taps; ++d) {
        const double sg = (double)p->sigma, wv = std::exp(-(double)d * d / (2.0 * sg * sg));
        h->w[d + p->taps] = (float)wv;
        h->wd[d + p->taps] = (float)(wv * (double)d * d / (sg * sg * sg));  // d w / d sigma
    }
    if (cudaMalloc(&h->shift, sizeof(float) * (FLR_MAX_Q + 3)) != cudaSuccess ||
        cudaMalloc(&h->count, sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc(&h->status, sizeof(int)) != cudaSuccess || cudaMemset(h->status, 0, sizeof(int)) != cudaSuccess) {
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
    cudaFree(h->gws);
    cudaFree(h->gpart);
    cudaFree(h->bws);
    cudaFree(h->bar);
    cudaFree(h->shift);
    cudaFree(h->count);
    cudaFree(h->status);
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
    a.appendix = (h->p.flags & FLR_FAST_APPENDIX) ? 1 : 0;
    a.eps_mul = h->p.eps_mul;
    a.status = h->status;
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

int flr_mbarrier_selftest(int ctas, unsigned long long timeout_ns, int *status)
{
    if (ctas <= 0 || ctas > 1024 || !status || timeout_ns > 10000000000ull) return FLR_ERR_ARG;
    int *d = nullptr;
    if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) return FLR_ERR_NOMEM;
    cudaError_t e = cudaMemset(d, 0, sizeof(int));
    if (e == cudaSuccess) {
        flr::mbarrier_selftest_kernel<<<ctas, 64>>>(d, timeout_ns);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(status, d, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(d);
    return e == cudaSuccess ? FLR_OK : FLR_ERR_CUDA;
}

int flr_fast_param_grad(flr_fast_handle *h, const float *guide, const float *map_guide, const float *radiance,
                        const float *grad_out, double *grad, int Hi, int Wi, void *stream)
{
    if (!h || !guide || !radiance || !grad_out || !grad || Hi <= 0 || Wi <= 0) return FLR_ERR_ARG;
    const int s = h->p.scale, F = h->p.factor, q = h->p.q;
    if (s > 1 && !map_guide) return FLR_ERR_ARG;
    if ((long long)Hi * s * Wi * s > 0x7fffffffLL) return FLR_ERR_ARG;
    if (((uintptr_t)guide | (uintptr_t)radiance | (uintptr_t)grad_out | (uintptr_t)map_guide) & 15u ||
        ((uintptr_t)grad & 7u))
        return FLR_ERR_ALIGN;
    const int Hb = (Hi + F - 1) / F, Wb = (Wi + F - 1) / F;
    const size_t nb = (size_t)Hb * Wb, npx = (size_t)Hi * s * Wi * s;
    const int nch = q + 3 + q * (q + 1) / 2 + 3 * q;
    if (h->ws_blocks < nb || !h->ws) {
        cudaFree(h->ws);
        h->ws = nullptr;
        h->ws_blocks = 0;
        if (cudaMalloc(&h->ws, nb * sizeof(float) * (2 * (size_t)nch + (size_t)(q + 3) + 1 + 3 * (size_t)(q + 1))) != cudaSuccess)
            return FLR_ERR_NOMEM;
        h->ws_blocks = nb;
    }
    // gradient workspace: tmp2, dcoef, tshift (32 floats), dout
    const size_t off_dc = (size_t)(nch + 1) * nb, off_ts = off_dc + 9 * (size_t)(q + 1) * nb;
    const size_t off_out = (off_ts + 32 + 3) & ~(size_t)3, need = off_out + 3 * npx;
    if (h->gws_floats < need || !h->gws) {
        cudaFree(h->gws);
        h->gws = nullptr;
        h->gws_floats = 0;
        if (cudaMalloc(&h->gws, need * sizeof(float)) != cudaSuccess) return FLR_ERR_NOMEM;
        h->gws_floats = need;
    }
    if (!h->gpart && cudaMalloc(&h->gpart, sizeof(double) * flr::kDotBlocks) != cudaSuccess) return FLR_ERR_NOMEM;
    flr::fast::FastArgs a;
    std::memset(&a, 0, sizeof(a));
    a.guide = guide;
    a.rad = radiance;
    a.map_guide = map_guide ? map_guide : guide;
    a.out = nullptr;
    a.blk = h->ws;
    a.tmp = h->ws + nb * (nch + q + 3);
    a.coef = a.tmp + nb * (nch + 1);
    a.tmp2 = h->gws;
    a.dcoef = h->gws + off_dc;
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
    a.appendix = (h->p.flags & FLR_FAST_APPENDIX) ? 1 : 0;
    a.eps_mul = h->p.eps_mul;
    a.status = h->status;
    std::memcpy(a.w, h->w, sizeof(a.w));
    std::memcpy(a.wd, h->wd, sizeof(a.wd));
    cudaStream_t st = (cudaStream_t)stream;
    h->last_stream = st;
    cudaError_t e = cudaMemsetAsync(h->count, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess)
        e = flr::launch_param_grad(q, a, h->gws + off_ts, grad_out, h->gws + off_out, h->gpart, grad, st);
    if (e != cudaSuccess) {
        std::snprintf(flr::g_fast_err, sizeof(flr::g_fast_err), "%s", cudaGetErrorString(e));
        return FLR_ERR_CUDA;
    }
    return FLR_OK;
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
    out->nonfinite = 0ull;  // not counted by the fast path
    int status = 0;
    if (cudaMemcpy(&status, h->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return FLR_ERR_CUDA;
    if (status != 0) {
        if (cudaMemset(h->status, 0, sizeof(int)) != cudaSuccess) return FLR_ERR_CUDA;
        return FLR_ERR_TIMEOUT;
    }
    return FLR_OK;
}

}  // extern "C"
