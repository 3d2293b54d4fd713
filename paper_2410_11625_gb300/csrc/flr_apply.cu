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
// shared memory, double-buffered so plane p+1 is in flight while plane p is summed (zero
// outside the image, which is what clipping the window means for a sum), slides a
// horizontal then a vertical radius-rc sum, and accumulates sum_k A_k[i][c] * (z_i - s_i)
// in registers.  Division by the window size happens once at the end, so the 27 averaged
// coefficients are never materialised.  When rows are 16-byte aligned (W % 4 == 0) one
// thread stages each plane tile with a single TMA box copy (the copy engine zero-fills
// the halo outside the image) completing on an mbarrier; otherwise every thread issues
// 4-byte asynchronous copies.
#include <cstring>

#include "flr_internal.cuh"
#include "tma.cuh"

namespace flr {
namespace {

constexpr int kAW = 64, kAH = 32, kAThreads = 256, kARun = 8;
static_assert(kAW * (kAH / kARun) == kAThreads, "one thread per (column, 8-row run)");

__device__ __forceinline__ void cp_async4(float *dst, const float *src, bool valid)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 4 : 0));
}
__device__ __forceinline__ void cp_async16(float *dst, const float *src, bool valid)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src),
                 "r"(valid ? 16 : 0));
}

// Tile geometry: the tile covers rows ty0 - rc .. ty0 + kAH + rc and columns starting at
// tx0 - RCA (RCA = rc rounded up to a multiple of 4, so rows start 16-byte aligned).
struct ApplyGeom {
    int RCA, TWa, THh, TS, HS;
    __host__ __device__ ApplyGeom(int rc)
    {
        RCA = (rc + 3) & ~3;
        TWa = kAW + 2 * RCA;
        THh = kAH + 2 * rc;
        TS = TWa + 4;   // 16-byte aligned rows (also the TMA box width)
        HS = kAW + 1;   // odd: the column walks of the vertical pass are conflict-free
    }
    __host__ __device__ int tile_floats() const { return (THh * TS + 31) / 32 * 32; }  // 128-byte multiple
    __host__ __device__ size_t floats() const
    {
        return 32 + (size_t)2 * tile_floats() + (size_t)THh * HS + 8;  // alignment slack, tiles, Hb, mbarriers
    }
};

constexpr unsigned long long kApplyTimeoutNs = 1000000000ull;  // 1 s per wait

// Kernel parameters: the TMA map of the coefficient planes (valid when use_tma) and the
// apply arguments.
struct alignas(128) ApplyKArgs {
    CUtensorMap tm;
    ApplyArgs a;
    int use_tma;
};

// Copy the tile + halo of one coefficient plane into shared memory (zero outside the
// image), asynchronously: each warp copies whole rows, lanes along the row.
__device__ __forceinline__ void load_tile(float *T, const ApplyGeom &g, const float *src, int H, int W,
                                          int ty0, int tx0, int rc, int warp, int lane)
{
    const int xs0 = tx0 - g.RCA;
    const bool vec = (W & 3) == 0;
    for (int row = warp; row < g.THh; row += kAThreads / 32) {
        const int sy = ty0 - rc + row;
        const bool row_ok = sy >= 0 && sy < H;
        const float *srow = src + (size_t)(row_ok ? sy : 0) * W;
        float *trow = T + row * g.TS;
        if (vec) {
            for (int c = lane; c < (g.TWa >> 2); c += 32) {
                const int sx = xs0 + 4 * c;
                const bool ok = row_ok && sx >= 0 && sx < W;
                cp_async16(trow + 4 * c, ok ? srow + sx : src, ok);
            }
        } else {
            for (int col = lane; col < g.TWa; col += 32) {
                const int sx = xs0 + col;
                const bool ok = row_ok && sx >= 0 && sx < W;
                cp_async4(trow + col, ok ? srow + sx : src, ok);
            }
        }
    }
    asm volatile("cp.async.commit_group;\n" ::);
}

template <int Q, int RT>
__global__ void __launch_bounds__(kAThreads, 4) flr_apply_kernel(const __grid_constant__ ApplyKArgs ka)
{
    extern __shared__ __align__(16) float sm[];
    const ApplyArgs &a = ka.a;
    const bool use_tma = ka.use_tma != 0;
    const int H = a.H, W = a.W;
    const int rc = RT >= 0 ? RT : a.rc;
    const ApplyGeom g(rc);
    float *base = sm + (((128 - (tma::smem_addr(sm) & 127)) & 127) >> 2);  // 128-byte aligned
    float *T0 = base;               // [THh][TS]   coefficient plane tile + halo, double-buffered
    float *T1 = T0 + g.tile_floats();
    float *Hb = T1 + g.tile_floats();  // [THh][HS]   horizontal sums
    uint64_t *bar = reinterpret_cast<uint64_t *>(Hb + ((g.THh * g.HS + 1) & ~1));  // [2] TMA arrivals
    __shared__ int s_abort;
    __shared__ float s_shift[Q + 3];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int row_hi = a.row_hi < 0 ? H : min(a.row_hi, H);
    const int tx0 = blockIdx.x * kAW, ty0 = a.row_lo + blockIdx.y * kAH;
    const int x = tid % kAW, run = tid / kAW;
    const int gx = tx0 + x;
    const size_t plane = (size_t)H * W;
    const int xoff = g.RCA - rc;  // tile column of output column 0's window start
    constexpr int NP = 3 * (Q + 1);

    float acc[3][kARun];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int t = 0; t < kARun; ++t) acc[c][t] = 0.f;

    // stage plane p of the tile into T: one TMA box copy, or asynchronous copies
    auto stage = [&](float *T, int p) {
        if (use_tma) {
            if (tid == 0) {
                uint64_t *b = bar + (p & 1);
                tma::mbar_expect_tx(b, (unsigned)(g.THh * g.TS * 4));
                tma::load_3d(T, &ka.tm, tx0 - g.RCA, ty0 - rc, p, b);
            }
        } else {
            load_tile(T, g, a.coef + (size_t)p * plane, H, W, ty0, tx0, rc, warp, lane);
        }
    };
    if (tid == 0) {
        s_abort = 0;
        if (use_tma) {
            tma::mbar_init(bar, 1);
            tma::mbar_init(bar + 1, 1);
            tma::mbar_init_fence();
        }
    }
    if (tid < Q + 3) s_shift[tid] = a.shift[tid];
    __syncthreads();
    stage(T0, 0);
    // the map-guide values of model row i + 1 are prefetched into L1 while row i is summed
    auto prefetch_z = [&](int i) {
        if (i < 1 || i > Q || gx >= W) return;
#pragma unroll
        for (int t = 0; t < kARun; ++t) {
            const int gy = ty0 + run * kARun + t;
            if (gy < H)
                asm volatile("prefetch.global.L1 [%0];\n" ::"l"(a.map_guide + (size_t)(i - 1) * plane + (size_t)gy * W + gx));
        }
    };
    prefetch_z(1);
    for (int i = 0; i <= Q; ++i) {
        float zf[kARun];
#pragma unroll
        for (int t = 0; t < kARun; ++t) {
            const int gy = ty0 + run * kARun + t;
            zf[t] = 1.f;
            if (i > 0) {
                zf[t] = (gx < W && gy < H)
                            ? __ldg(a.map_guide + (size_t)(i - 1) * plane + (size_t)gy * W + gx) - s_shift[i - 1]
                            : 0.f;
            }
        }
        prefetch_z(i + 1);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int p = 3 * i + c;
            float *Tc = (p & 1) ? T1 : T0;
            if (p + 1 < NP) stage((p & 1) ? T0 : T1, p + 1);
            if (use_tma) {
                if (!tma::wait_warp(bar + (p & 1), (uint32_t)((p >> 1) & 1), kApplyTimeoutNs) && lane == 0) {
                    s_abort = 1;
                    if (a.status) atomicExch(a.status, 1);
                }
            } else if (p + 1 < NP) {
                asm volatile("cp.async.wait_group 1;\n" ::);
            } else {
                asm volatile("cp.async.wait_group 0;\n" ::);
            }
            __syncthreads();  // plane p is in Tc for every thread
            if (s_abort) {  // let a copy still in flight land before the CTA exits, then stop
                if (use_tma && p + 1 < NP && warp == 0)
                    tma::wait_warp(bar + ((p + 1) & 1), (uint32_t)(((p + 1) >> 1) & 1), kApplyTimeoutNs);
                return;
            }
            // horizontal sums: 16 outputs per item, operands held in registers; consecutive
            // lanes take consecutive rows (16-byte loads, row stride = 4 mod 8 floats: the
            // eight lanes of each 128-bit phase hit distinct banks)
            for (int item = tid; item < g.THh * 4; item += kAThreads) {
                const int xr = (item / g.THh) * 16, row = item % g.THh;
                const float *q = Tc + row * g.TS + xr;  // 16-byte aligned
                float *h = Hb + row * g.HS + xr;
                if constexpr (RT >= 0) {
                    constexpr int RCA = (RT + 3) & ~3, XO = RCA - RT;
                    constexpr int N = 16 + 2 * RCA;
                    float v[N];
#pragma unroll
                    for (int k = 0; k < N; k += 4) {
                        const float4 f = *reinterpret_cast<const float4 *>(q + k);
                        v[k] = f.x;
                        v[k + 1] = f.y;
                        v[k + 2] = f.z;
                        v[k + 3] = f.w;
                    }
                    float s4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                    for (int k = 0; k <= 2 * RT; ++k) s4[k & 3] += v[XO + k];
                    float s = (s4[0] + s4[1]) + (s4[2] + s4[3]);
                    h[0] = s;
#pragma unroll
                    for (int t = 1; t < 16; ++t) {
                        s += v[XO + t + 2 * RT] - v[XO + t - 1];
                        h[t] = s;
                    }
                } else {
                    const float *qq = q + xoff;
                    float s = 0.f;
                    for (int k = 0; k <= 2 * rc; ++k) s += qq[k];
                    h[0] = s;
#pragma unroll
                    for (int t = 1; t < 16; ++t) {
                        s += qq[t + 2 * rc] - qq[t - 1];
                        h[t] = s;
                    }
                }
            }
            __syncthreads();  // Hb complete; Tc may be refilled from here on
            if (use_tma && tid == 0) asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            {
                const float *q = Hb + (run * kARun) * g.HS + x;
                if constexpr (RT >= 0) {
                    constexpr int N = kARun + 2 * RT;
                    float v[N];
#pragma unroll
                    for (int k = 0; k < N; ++k) v[k] = q[k * g.HS];
                    float s2[2] = {0.f, 0.f};
#pragma unroll
                    for (int k = 0; k <= 2 * RT; ++k) s2[k & 1] += v[k];
                    float s = s2[0] + s2[1];
                    acc[c][0] = fmaf(s, zf[0], acc[c][0]);
#pragma unroll
                    for (int t = 1; t < kARun; ++t) {
                        s += v[t + 2 * RT] - v[t - 1];
                        acc[c][t] = fmaf(s, zf[t], acc[c][t]);
                    }
                } else {
                    float s = 0.f;
                    for (int k = 0; k <= 2 * rc; ++k) s += q[k * g.HS];
                    acc[c][0] = fmaf(s, zf[0], acc[c][0]);
#pragma unroll
                    for (int t = 1; t < kARun; ++t) {
                        s += q[(t + 2 * rc) * g.HS] - q[(t - 1) * g.HS];
                        acc[c][t] = fmaf(s, zf[t], acc[c][t]);
                    }
                }
            }
        }
    }
    if (gx < W) {
        const float nx = (float)(min(gx + rc, W - 1) - max(gx - rc, 0) + 1);
        int bad = 0;
#pragma unroll
        for (int t = 0; t < kARun; ++t) {
            const int gy = ty0 + run * kARun + t;
            if (gy < row_hi) {
                const float ny = (float)(min(gy + rc, H - 1) - max(gy - rc, 0) + 1);
                const float inv_m = 1.0f / (nx * ny);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float o = fmaf(acc[c][t], inv_m, s_shift[Q + c]);
                    a.out[c * plane + (size_t)gy * W + gx] = o;
                    bad += !isfinite(o);
                }
            }
        }
        if (bad && a.nonfinite) atomicAdd(a.nonfinite, (unsigned long long)bad);
    }
}

template <int Q, int RT>
cudaError_t launch_apply_qr(const ApplyArgs &a, cudaStream_t st)
{
    const ApplyGeom g(a.rc);
    const size_t smem = sizeof(float) * g.floats();
    cudaError_t e = cudaFuncSetAttribute(flr_apply_kernel<Q, RT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    // four CTAs per SM (64 registers each) need most of the unified L1 / shared array
    e = cudaFuncSetAttribute(flr_apply_kernel<Q, RT>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    const int rows = (a.row_hi < 0 ? a.H : a.row_hi) - a.row_lo;
    if (rows <= 0) return cudaSuccess;
    dim3 grid((a.W + kAW - 1) / kAW, (rows + kAH - 1) / kAH);
    ApplyKArgs ka;
    std::memset(&ka, 0, sizeof(ka));
    ka.a = a;
    ka.use_tma = ((a.W & 3) == 0 && ((uintptr_t)a.coef & 15) == 0 &&
                  tma::encode_planes_f32(&ka.tm, a.coef, a.W, a.H, 3 * (Q + 1), g.TS, g.THh, 1) == cudaSuccess)
                     ? 1
                     : 0;
    flr_apply_kernel<Q, RT><<<grid, kAThreads, smem, st>>>(ka);
    return cudaGetLastError();
}

template <int Q>
cudaError_t launch_apply_q(const ApplyArgs &a, cudaStream_t st)
{
    if constexpr (Q == 8) {
        if (a.rc == 8) return launch_apply_qr<8, 8>(a, st);
        if (a.rc == 5) return launch_apply_qr<8, 5>(a, st);
    }
    return launch_apply_qr<Q, -1>(a, st);
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
