// flr_bwd.cu -- kernels of the FLR backward pass that are not the per-pixel adjoint solve
// (that one is the forward kernel in adjoint mode, flr_fwd.cu).  sm_103a.
//
// The backward pass is the reverse-mode derivative of the forward's steps (the paper
// trains through FLR by backpropagation, Sec. 3.2-3.3; it prints no adjoint).  With
// g = dL/dI and m_i the size of the clipped averaging window T'_i:
//   fields    F_i = (1, z_i - s) g_i^T / m_i                       (adjoint of the apply)
//   G(A_k)    = sum_{i in T'_k} F_i                                (adjoint of the average)
//   adjoint   per pixel k: the moment gradients GS_k               (flr_fwd.cu, ADJ = true)
//   BS_j      = sum_{k in T_j} GS_k                                (adjoint of the window sums)
//   contract  dx_j = BS_x + 2 BS_xx (x_j - s) + BS_xy (y_j - s_y)
//             dy_j = BS_y + BS_xy^T (x_j - s)
//             dz_j = Abar_j g_j                                    (the applied guide)
// j in T_k <=> k in T_j for clipped square windows of one radius, so every adjoint of a
// window sum is the same clipped box sum.
#include <cstring>

#include "flr_internal.cuh"
#include "tma.cuh"

namespace flr {
namespace {

constexpr int kBW = 64, kBH = 32, kBThreads = 256;

template <int Q>
__global__ void bwd_fields_kernel(const float *__restrict__ g, const float *__restrict__ z,
                                  const float *__restrict__ shift, float *__restrict__ F, int H, int W, int rc)
{
    const size_t plane = (size_t)H * W;
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < plane; p += (size_t)gridDim.x * blockDim.x) {
        const int y = (int)(p / W), x = (int)(p % W);
        float inv_m = 1.f;
        if (rc > 0) {
            const float ny = (float)(min(y + rc, H - 1) - max(y - rc, 0) + 1);
            const float nx = (float)(min(x + rc, W - 1) - max(x - rc, 0) + 1);
            inv_m = 1.0f / (ny * nx);
        }
        float gc[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            gc[c] = g[c * plane + p] * inv_m;
            F[c * plane + p] = gc[c];
        }
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const float zi = z[i * plane + p] - shift[i];
#pragma unroll
            for (int c = 0; c < 3; ++c) F[(3 * (i + 1) + c) * plane + p] = zi * gc[c];
        }
    }
}

// out[plane] = sum over the clipped radius-rad window of in[plane]; blockIdx.z = plane.
__global__ void __launch_bounds__(kBThreads) box_sum_kernel(const float *__restrict__ in, float *__restrict__ out,
                                                           int H, int W, int rad)
{
    extern __shared__ float sm[];
    const int TWh = kBW + 2 * rad, THh = kBH + 2 * rad;
    const int TS = TWh + 1, HS = kBW + 1;
    float *T = sm;
    float *Hb = T + THh * TS;
    const size_t plane = (size_t)H * W;
    const float *src = in + (size_t)blockIdx.z * plane;
    float *dst = out + (size_t)blockIdx.z * plane;
    const int tx0 = blockIdx.x * kBW, ty0 = blockIdx.y * kBH;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int row = warp; row < THh; row += kBThreads / 32) {
        const int sy = ty0 - rad + row;
        for (int col = lane; col < TWh; col += 32) {
            const int sx = tx0 - rad + col;
            T[row * TS + col] = (sy >= 0 && sy < H && sx >= 0 && sx < W) ? __ldg(src + (size_t)sy * W + sx) : 0.f;
        }
    }
    __syncthreads();
    for (int item = tid; item < THh * 4; item += kBThreads) {
        const int row = item % THh, xr = (item / THh) * 16;
        const float *q = T + row * TS + xr;
        float *h = Hb + row * HS + xr;
        float s = 0.f;
        for (int k = 0; k <= 2 * rad; ++k) s += q[k];
        h[0] = s;
#pragma unroll
        for (int t = 1; t < 16; ++t) {
            s += q[t + 2 * rad] - q[t - 1];
            h[t] = s;
        }
    }
    __syncthreads();
    const int x = tid % kBW, run = tid / kBW;
    const int gx = tx0 + x;
    const float *q = Hb + (run * 8) * HS + x;
    float s = 0.f;
    for (int k = 0; k <= 2 * rad; ++k) s += q[k * HS];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        if (t > 0) s += q[(t + 2 * rad) * HS] - q[(t - 1) * HS];
        const int gy = ty0 + run * 8 + t;
        if (gx < W && gy < H) dst[(size_t)gy * W + gx] = s;
    }
}

// The same clipped box sum over many planes with TMA staging (rows 16-byte aligned): one CTA
// per 64 x 32 output tile walks every plane; each plane's tile + halo arrives by one TMA box
// copy (the copy engine zero-fills outside the image) into a double-buffered ring, so the
// next plane loads while the current one is summed.  Waits are bounded (1 s).
struct alignas(128) BoxKArgs {
    CUtensorMap tm;  // [nplanes][H][W] float32, box (TS, THh, 1)
    float *out;
    int H, W, rad, nplanes;
    int *status;
};

struct BoxGeom {
    int RCA, TWa, THh, TS, HS;
    __host__ __device__ BoxGeom(int rad)
    {
        RCA = (rad + 3) & ~3;  // staged columns start 16-byte aligned
        TWa = kBW + 2 * RCA;
        THh = kBH + 2 * rad;
        TS = TWa + 4;          // row stride = 4 (mod 8) floats: conflict-free 128-bit phases
        HS = kBW + 1;
    }
    __host__ __device__ int tile_floats() const { return (THh * TS + 31) / 32 * 32; }
    __host__ __device__ size_t floats() const { return 32 + (size_t)2 * tile_floats() + (size_t)THh * HS + 8; }
};

constexpr unsigned long long kBoxTimeoutNs = 1000000000ull;

template <int RT>
__global__ void __launch_bounds__(kBThreads, 4) box_sum_tma_kernel(const __grid_constant__ BoxKArgs k)
{
    extern __shared__ __align__(16) float sm[];
    const int rad = RT >= 0 ? RT : k.rad;
    const BoxGeom g(rad);
    float *base = sm + (((128 - (tma::smem_addr(sm) & 127)) & 127) >> 2);
    float *T0 = base, *T1 = base + g.tile_floats();
    float *Hb = T1 + g.tile_floats();
    uint64_t *bar = reinterpret_cast<uint64_t *>(Hb + ((g.THh * g.HS + 1) & ~1));
    __shared__ int s_abort;
    const int tid = threadIdx.x, lane = tid & 31;
    const int tx0 = blockIdx.x * kBW, ty0 = blockIdx.y * kBH;
    const size_t plane = (size_t)k.H * k.W;
    auto stage = [&](float *T, int p) {
        if (tid == 0) {
            uint64_t *b = bar + (p & 1);
            tma::mbar_expect_tx(b, (unsigned)(g.THh * g.TS * 4));
            tma::load_3d(T, &k.tm, tx0 - g.RCA, ty0 - rad, p, b);
        }
    };
    if (tid == 0) {
        s_abort = 0;
        tma::mbar_init(bar, 1);
        tma::mbar_init(bar + 1, 1);
        tma::mbar_init_fence();
    }
    __syncthreads();
    stage(T0, 0);
    const int x = tid % kBW, run = tid / kBW;
    const int gx = tx0 + x;
    for (int p = 0; p < k.nplanes; ++p) {
        float *Tc = (p & 1) ? T1 : T0;
        if (p + 1 < k.nplanes) stage((p & 1) ? T0 : T1, p + 1);
        if (!tma::wait_warp(bar + (p & 1), (uint32_t)((p >> 1) & 1), kBoxTimeoutNs) && lane == 0) {
            s_abort = 1;
            if (k.status) atomicExch(k.status, 1);
        }
        __syncthreads();
        if (s_abort) {  // let a copy still in flight land before the CTA exits, then stop
            if (p + 1 < k.nplanes && tid < 32)
                tma::wait_warp(bar + ((p + 1) & 1), (uint32_t)(((p + 1) >> 1) & 1), kBoxTimeoutNs);
            return;
        }
        // horizontal sums: 16 outputs per item, operands in registers; consecutive lanes take
        // consecutive rows (16-byte loads at row stride 4 mod 8 floats: distinct banks)
        for (int item = tid; item < g.THh * 4; item += kBThreads) {
            const int xr = (item / g.THh) * 16, row = item % g.THh;
            const float *q = Tc + row * g.TS + xr;
            float *h = Hb + row * g.HS + xr;
            if constexpr (RT >= 0) {
                constexpr int RCA = (RT + 3) & ~3, XO = RCA - RT, N = 16 + 2 * RCA;
                float v[N];
#pragma unroll
                for (int kk = 0; kk < N; kk += 4) {
                    const float4 f = *reinterpret_cast<const float4 *>(q + kk);
                    v[kk] = f.x;
                    v[kk + 1] = f.y;
                    v[kk + 2] = f.z;
                    v[kk + 3] = f.w;
                }
                float s4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int kk = 0; kk <= 2 * RT; ++kk) s4[kk & 3] += v[XO + kk];
                float s = (s4[0] + s4[1]) + (s4[2] + s4[3]);
                h[0] = s;
#pragma unroll
                for (int t = 1; t < 16; ++t) {
                    s += v[XO + t + 2 * RT] - v[XO + t - 1];
                    h[t] = s;
                }
            } else {
                const float *qq = q + (g.RCA - rad);
                float s = 0.f;
                for (int kk = 0; kk <= 2 * rad; ++kk) s += qq[kk];
                h[0] = s;
#pragma unroll
                for (int t = 1; t < 16; ++t) {
                    s += qq[t + 2 * rad] - qq[t - 1];
                    h[t] = s;
                }
            }
        }
        __syncthreads();  // Hb complete; Tc may be refilled from here on
        if (tid == 0) asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        // vertical sums: thread = (column, run of 8 rows)
        const float *q = Hb + (run * 8) * g.HS + x;
        float s = 0.f;
        for (int kk = 0; kk <= 2 * rad; ++kk) s += q[kk * g.HS];
        float *dst = k.out + (size_t)p * plane;
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            if (t > 0) s += q[(t + 2 * rad) * g.HS] - q[(t - 1) * g.HS];
            const int gy = ty0 + run * 8 + t;
            if (gx < k.W && gy < k.H) dst[(size_t)gy * k.W + gx] = s;
        }
    }
}

template <int Q>
__global__ void __launch_bounds__(256) bwd_contract_kernel(const BwdArgs a)
{
    using C = Chan<Q>;
    const int H = a.H, W = a.W;
    const size_t plane = (size_t)H * W;
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < plane; p += (size_t)gridDim.x * blockDim.x) {
        const int y = (int)(p / W), x = (int)(p % W);
        // every input of this pixel is read once, up front (the outputs may not alias them)
        float xs[Q], ys[3], gc[3];
#pragma unroll
        for (int i = 0; i < Q; ++i) xs[i] = __ldg(a.guide + i * plane + p) - a.shift[i];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            ys[c] = __ldg(a.rad + c * plane + p) - a.shift[Q + c];
            gc[c] = __ldg(a.g + c * plane + p);
        }
        float inv_m = 1.f;
        if (a.rc > 0) {
            const float ny = (float)(min(y + a.rc, H - 1) - max(y - a.rc, 0) + 1);
            const float nx = (float)(min(x + a.rc, W - 1) - max(x - a.rc, 0) + 1);
            inv_m = 1.0f / (ny * nx);
        }
        const float *BS = a.BS;
        float bxx[C::NXX];
#pragma unroll
        for (int t = 0; t < C::NXX; ++t) bxx[t] = __ldg(BS + (C::XX0 + t) * plane + p);
        float bxy[Q][3];
#pragma unroll
        for (int i = 0; i < Q; ++i)
#pragma unroll
            for (int c = 0; c < 3; ++c) bxy[i][c] = __ldg(BS + C::xy(i, c) * plane + p);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            float d = __ldg(BS + (C::X0 + i) * plane + p);
#pragma unroll
            for (int j = 0; j < Q; ++j) {
                const int t = (i <= j ? C::xx(i, j) : C::xx(j, i)) - C::XX0;
                d = fmaf(2.f * bxx[t], xs[j], d);
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) d = fmaf(bxy[i][c], ys[c], d);
            // the applied guide: dz_i = sum_c Abar[i][c] g_c
            float dz = 0.f;
#pragma unroll
            for (int c = 0; c < 3; ++c) dz = fmaf(__ldg(a.BA + (3 * (i + 1) + c) * plane + p), gc[c], dz);
            dz *= inv_m;
            if (a.separate_map) {
                a.grad_guide[i * plane + p] = d;
                if (a.grad_map) a.grad_map[i * plane + p] = dz;
            } else {
                a.grad_guide[i * plane + p] = d + dz;
            }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float d = __ldg(BS + (C::Y0 + c) * plane + p);
#pragma unroll
            for (int i = 0; i < Q; ++i) d = fmaf(bxy[i][c], xs[i], d);
            a.grad_rad[c * plane + p] = d;
        }
    }
}

// The same contraction for four consecutive pixels of a row per thread (W a multiple of 4,
// every plane 16-byte aligned): one 16-byte load per plane and four pixels instead of four
// 4-byte loads, and each output channel's gradient formed from its own planes in turn, so
// that a thread holds four pixels' inputs and one channel's operands at a time.  Every
// pixel's arithmetic (operands, order of the fused multiply-adds) is that of
// bwd_contract_kernel, so the results are the same bit for bit.
__device__ __forceinline__ float4 ld4(const float *p) { return __ldg(reinterpret_cast<const float4 *>(p)); }
__device__ __forceinline__ void st4(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }
__device__ __forceinline__ float4 fma4(float4 a, float4 b, float4 c)
{
    return make_float4(fmaf(a.x, b.x, c.x), fmaf(a.y, b.y, c.y), fmaf(a.z, b.z, c.z), fmaf(a.w, b.w, c.w));
}

template <int Q>
__global__ void __launch_bounds__(256) bwd_contract4_kernel(const BwdArgs a)
{
    using C = Chan<Q>;
    const int H = a.H, W = a.W;
    const size_t plane = (size_t)H * W;
    const size_t nq = plane / 4;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += (size_t)gridDim.x * blockDim.x) {
        const size_t p = 4 * q;
        const int y = (int)(p / W), x0 = (int)(p % W);
        float4 xs[Q], ys[3], gc[3];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const float4 v = ld4(a.guide + i * plane + p);
            const float s = a.shift[i];
            xs[i] = make_float4(v.x - s, v.y - s, v.z - s, v.w - s);
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float4 v = ld4(a.rad + c * plane + p);
            const float s = a.shift[Q + c];
            ys[c] = make_float4(v.x - s, v.y - s, v.z - s, v.w - s);
            gc[c] = ld4(a.g + c * plane + p);
        }
        float inv_m[4] = {1.f, 1.f, 1.f, 1.f};
        if (a.rc > 0) {
            const float ny = (float)(min(y + a.rc, H - 1) - max(y - a.rc, 0) + 1);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int x = x0 + k;
                const float nx = (float)(min(x + a.rc, W - 1) - max(x - a.rc, 0) + 1);
                inv_m[k] = 1.0f / (ny * nx);
            }
        }
        const float *BS = a.BS;
#pragma unroll 1
        for (int i = 0; i < Q; ++i) {  // one guide channel's 15 planes in flight at a time
            float4 d = ld4(BS + (C::X0 + i) * plane + p);
#pragma unroll
            for (int j = 0; j < Q; ++j) {
                const int t = (i <= j ? C::xx(i, j) : C::xx(j, i));
                const float4 b = ld4(BS + t * plane + p);
                d = fma4(make_float4(2.f * b.x, 2.f * b.y, 2.f * b.z, 2.f * b.w), xs[j], d);
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) d = fma4(ld4(BS + C::xy(i, c) * plane + p), ys[c], d);
            float4 dz = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int c = 0; c < 3; ++c) dz = fma4(ld4(a.BA + (3 * (i + 1) + c) * plane + p), gc[c], dz);
            dz = make_float4(dz.x * inv_m[0], dz.y * inv_m[1], dz.z * inv_m[2], dz.w * inv_m[3]);
            if (a.separate_map) {
                st4(a.grad_guide + i * plane + p, d);
                if (a.grad_map) st4(a.grad_map + i * plane + p, dz);
            } else {
                st4(a.grad_guide + i * plane + p, make_float4(d.x + dz.x, d.y + dz.y, d.z + dz.z, d.w + dz.w));
            }
        }
#pragma unroll 1
        for (int c = 0; c < 3; ++c) {
            float4 d = ld4(BS + (C::Y0 + c) * plane + p);
#pragma unroll
            for (int i = 0; i < Q; ++i) d = fma4(ld4(BS + C::xy(i, c) * plane + p), xs[i], d);
            st4(a.grad_rad + c * plane + p, d);
        }
    }
}

int elem_grid(size_t n) { return (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096); }

}  // namespace

cudaError_t launch_bwd_fields(int q, const float *g, const float *z, const float *shift, float *F, int H, int W,
                              int rc, cudaStream_t st)
{
    const int grid = elem_grid((size_t)H * W);
    switch (q) {
    case 1: bwd_fields_kernel<1><<<grid, 256, 0, st>>>(g, z, shift, F, H, W, rc); break;
    case 2: bwd_fields_kernel<2><<<grid, 256, 0, st>>>(g, z, shift, F, H, W, rc); break;
    case 3: bwd_fields_kernel<3><<<grid, 256, 0, st>>>(g, z, shift, F, H, W, rc); break;
    case 4: bwd_fields_kernel<4><<<grid, 256, 0, st>>>(g, z, shift, F, H, W, rc); break;
    case 5: bwd_fields_kernel<5><<<grid, 256, 0, st>>>(g, z, shift, F, H, W, rc); break;
    case 6: bwd_fields_kernel<6><<<grid, 256, 0, st>>>(g, z, shift, F, H, W, rc); break;
    case 7: bwd_fields_kernel<7><<<grid, 256, 0, st>>>(g, z, shift, F, H, W, rc); break;
    case 8: bwd_fields_kernel<8><<<grid, 256, 0, st>>>(g, z, shift, F, H, W, rc); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int RT>
cudaError_t launch_box_sum_tma(const BoxKArgs &k, cudaStream_t st)
{
    const BoxGeom g(k.rad);
    const size_t smem = sizeof(float) * g.floats();
    cudaError_t e = cudaFuncSetAttribute(box_sum_tma_kernel<RT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // four CTAs per SM need most of the unified L1 / shared array as shared memory
    e = cudaFuncSetAttribute(box_sum_tma_kernel<RT>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    dim3 grid((k.W + kBW - 1) / kBW, (k.H + kBH - 1) / kBH);
    box_sum_tma_kernel<RT><<<grid, kBThreads, smem, st>>>(k);
    return cudaGetLastError();
}

cudaError_t launch_box_sum(const float *in, float *out, int nplanes, int H, int W, int rad, cudaStream_t st, int *status)
{
    if ((W & 3) == 0 && ((uintptr_t)in & 15) == 0 && nplanes > 0) {
        BoxKArgs k;
        std::memset(&k, 0, sizeof(k));
        const BoxGeom g(rad);
        if (tma::encode_planes_f32(&k.tm, in, W, H, nplanes, g.TS, g.THh, 1) == cudaSuccess) {
            k.out = out;
            k.H = H;
            k.W = W;
            k.rad = rad;
            k.nplanes = nplanes;
            k.status = status;
            return rad == 8 ? launch_box_sum_tma<8>(k, st) : launch_box_sum_tma<-1>(k, st);
        }
    }
    const size_t smem = sizeof(float) * ((size_t)(kBH + 2 * rad) * (kBW + 2 * rad + 1) + (size_t)(kBH + 2 * rad) * (kBW + 1));
    cudaError_t e = cudaFuncSetAttribute(box_sum_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((W + kBW - 1) / kBW, (H + kBH - 1) / kBH, nplanes);
    box_sum_kernel<<<grid, kBThreads, smem, st>>>(in, out, H, W, rad);
    return cudaGetLastError();
}

cudaError_t launch_bwd_contract(int q, const BwdArgs &a, cudaStream_t st)
{
    auto al = [](const void *p) { return ((uintptr_t)p & 15) == 0; };
    if ((a.W & 3) == 0 && al(a.guide) && al(a.rad) && al(a.g) && al(a.BS) && al(a.BA) && al(a.grad_guide) &&
        al(a.grad_map) && al(a.grad_rad)) {
        const int grid4 = (int)(((size_t)a.H * a.W / 4 + 255) / 256);  // one thread per four pixels
        switch (q) {
        case 1: bwd_contract4_kernel<1><<<grid4, 256, 0, st>>>(a); break;
        case 2: bwd_contract4_kernel<2><<<grid4, 256, 0, st>>>(a); break;
        case 3: bwd_contract4_kernel<3><<<grid4, 256, 0, st>>>(a); break;
        case 4: bwd_contract4_kernel<4><<<grid4, 256, 0, st>>>(a); break;
        case 5: bwd_contract4_kernel<5><<<grid4, 256, 0, st>>>(a); break;
        case 6: bwd_contract4_kernel<6><<<grid4, 256, 0, st>>>(a); break;
        case 7: bwd_contract4_kernel<7><<<grid4, 256, 0, st>>>(a); break;
        case 8: bwd_contract4_kernel<8><<<grid4, 256, 0, st>>>(a); break;
        default: return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }
    const int grid = (int)(((size_t)a.H * a.W + 255) / 256);  // one thread per pixel
    switch (q) {
    case 1: bwd_contract_kernel<1><<<grid, 256, 0, st>>>(a); break;
    case 2: bwd_contract_kernel<2><<<grid, 256, 0, st>>>(a); break;
    case 3: bwd_contract_kernel<3><<<grid, 256, 0, st>>>(a); break;
    case 4: bwd_contract_kernel<4><<<grid, 256, 0, st>>>(a); break;
    case 5: bwd_contract_kernel<5><<<grid, 256, 0, st>>>(a); break;
    case 6: bwd_contract_kernel<6><<<grid, 256, 0, st>>>(a); break;
    case 7: bwd_contract_kernel<7><<<grid, 256, 0, st>>>(a); break;
    case 8: bwd_contract_kernel<8><<<grid, 256, 0, st>>>(a); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace flr
