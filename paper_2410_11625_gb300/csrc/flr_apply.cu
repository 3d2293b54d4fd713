// flr_apply.cu -- FLR coefficient averaging and model application (sm_103a).
//
// Input: the per-pixel models A_k = (b_k, a_k) written by the forward kernel, as
// (Q+1)*3 planes (plane 3*i + c holds row i, column c of A_k; row 0 is the bias), with
// the bias expressed relative to the frame reference shift s.  Output, per pixel i:
//     I_i = (1, z_i - s) * mean_{k in T'_i} A_k  + s_y,
// where T'_i is the clipped square window of radius rc and z the map guide (Sec. 3.1
// applies the model to the centre pixel, I_k = x_k A_k; the averaging over T'_i is the
// coefficient box-average of the guided-filter family that Sec. 3.2 contrasts FLR with).
//
// This kernel is bound by HBM: it reads (Q+1)*3 coefficient planes plus the Q map-guide
// planes and writes 3 planes, and does ~6 flops per value read.  A CTA owns a 64 x 32
// output tile; for each coefficient plane it stages the tile plus a radius-rc halo in
// shared memory with asynchronous copies, double-buffered so plane p+1 is in flight while
// plane p is summed (zero outside the image, which is what clipping the window means for
// a sum), slides a horizontal then a vertical radius-rc sum, and accumulates
// sum_k A_k[i][c] * (z_i - s_i) in registers.  Division by the window size happens once
// at the end, so the 27 averaged coefficients are never materialised.
#include "flr_internal.cuh"

namespace flr {
namespace {

constexpr int kAW = 64, kAH = 32, kAThreads = 256, kARun = 8;
static_assert(kAW * (kAH / kARun) == kAThreads, "one thread per (column, 8-row run)");

__device__ __forceinline__ void cp_async4(float *dst, const float *src, bool valid)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src),
                 "r"(valid ? 4 : 0));
}

// Copy the tile + halo of one coefficient plane into shared memory (zero outside the
// image), asynchronously: each warp copies whole rows, lanes along the row.
__device__ __forceinline__ void load_tile(float *T, int TS, const float *src, int H, int W, int ty0,
                                          int tx0, int rc, int THh, int TWh, int warp, int lane)
{
    for (int row = warp; row < THh; row += kAThreads / 32) {
        const int sy = ty0 - rc + row;
        const bool row_ok = sy >= 0 && sy < H;
        const float *srow = src + (size_t)(row_ok ? sy : 0) * W;
        for (int col = lane; col < TWh; col += 32) {
            const int sx = tx0 - rc + col;
            const bool ok = row_ok && sx >= 0 && sx < W;
            cp_async4(T + row * TS + col, ok ? srow + sx : src, ok);
        }
    }
    asm volatile("cp.async.commit_group;\n" ::);
}

template <int Q>
__global__ void __launch_bounds__(kAThreads) flr_apply_kernel(const ApplyArgs a)
{
    extern __shared__ float sm[];
    const int H = a.H, W = a.W, rc = a.rc;
    const int TWh = kAW + 2 * rc, THh = kAH + 2 * rc;
    const int TS = TWh + 1, HS = kAW + 1;
    float *T0 = sm;             // [THh][TS]   coefficient plane tile + halo, double-buffered
    float *T1 = T0 + THh * TS;
    float *Hb = T1 + THh * TS;  // [THh][HS]   horizontal sums
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tx0 = blockIdx.x * kAW, ty0 = blockIdx.y * kAH;
    const int x = tid % kAW, run = tid / kAW;
    const int gx = tx0 + x;
    const size_t plane = (size_t)H * W;
    constexpr int NP = 3 * (Q + 1);

    float acc[3][kARun];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int t = 0; t < kARun; ++t) acc[c][t] = 0.f;

    load_tile(T0, TS, a.coef, H, W, ty0, tx0, rc, THh, TWh, warp, lane);
    for (int i = 0; i <= Q; ++i) {
        float zf[kARun];
#pragma unroll
        for (int t = 0; t < kARun; ++t) {
            const int gy = ty0 + run * kARun + t;
            zf[t] = 1.f;
            if (i > 0) {
                zf[t] = (gx < W && gy < H)
                            ? __ldg(a.map_guide + (size_t)(i - 1) * plane + (size_t)gy * W + gx) - a.shift[i - 1]
                            : 0.f;
            }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int p = 3 * i + c;
            float *Tc = (p & 1) ? T1 : T0;
            if (p + 1 < NP) {
                load_tile((p & 1) ? T0 : T1, TS, a.coef + (size_t)(p + 1) * plane, H, W, ty0, tx0, rc,
                          THh, TWh, warp, lane);
                asm volatile("cp.async.wait_group 1;\n" ::);
            } else {
                asm volatile("cp.async.wait_group 0;\n" ::);
            }
            __syncthreads();  // plane p is in Tc for every thread
            for (int item = tid; item < THh * 4; item += kAThreads) {
                const int row = item >> 2, xr = (item & 3) * 16;
                const float *q = Tc + row * TS + xr;
                float *h = Hb + row * HS + xr;
                float s = 0.f;
                for (int k = 0; k <= 2 * rc; ++k) s += q[k];
                h[0] = s;
#pragma unroll
                for (int t = 1; t < 16; ++t) {
                    s += q[t + 2 * rc] - q[t - 1];
                    h[t] = s;
                }
            }
            __syncthreads();  // Hb complete; Tc may be refilled from here on
            {
                const float *q = Hb + (run * kARun) * HS + x;
                float s = 0.f;
                for (int k = 0; k <= 2 * rc; ++k) s += q[k * HS];
                acc[c][0] = fmaf(s, zf[0], acc[c][0]);
#pragma unroll
                for (int t = 1; t < kARun; ++t) {
                    s += q[(t + 2 * rc) * HS] - q[(t - 1) * HS];
                    acc[c][t] = fmaf(s, zf[t], acc[c][t]);
                }
            }
        }
    }
    if (gx < W) {
        const float nx = (float)(min(gx + rc, W - 1) - max(gx - rc, 0) + 1);
#pragma unroll
        for (int t = 0; t < kARun; ++t) {
            const int gy = ty0 + run * kARun + t;
            if (gy < H) {
                const float ny = (float)(min(gy + rc, H - 1) - max(gy - rc, 0) + 1);
                const float inv_m = 1.0f / (nx * ny);
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    a.out[c * plane + (size_t)gy * W + gx] = fmaf(acc[c][t], inv_m, a.shift[Q + c]);
            }
        }
    }
}

template <int Q>
cudaError_t launch_apply_q(const ApplyArgs &a, cudaStream_t st)
{
    const int TWh = kAW + 2 * a.rc, THh = kAH + 2 * a.rc;
    const size_t smem = sizeof(float) * ((size_t)2 * THh * (TWh + 1) + (size_t)THh * (kAW + 1));
    cudaError_t e = cudaFuncSetAttribute(flr_apply_kernel<Q>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((a.W + kAW - 1) / kAW, (a.H + kAH - 1) / kAH);
    flr_apply_kernel<Q><<<grid, kAThreads, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_apply(int q, const ApplyArgs &a, cudaStream_t st)
{
    switch (q) {
    case 1: return launch_apply_q<1>(a, st);
    case 2: return launch_apply_q<2>(a, st);
    case 3: return launch_apply_q<3>(a, st);
    case 4: return launch_apply_q<4>(a, st);
    case 5: return launch_apply_q<5>(a, st);
    case 6: return launch_apply_q<6>(a, st);
    case 7: return launch_apply_q<7>(a, st);
    case 8: return launch_apply_q<8>(a, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace flr
