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
#include "flr_internal.cuh"

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

template <int Q>
__global__ void bwd_contract_kernel(const BwdArgs a)
{
    using C = Chan<Q>;
    const int H = a.H, W = a.W;
    const size_t plane = (size_t)H * W;
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < plane; p += (size_t)gridDim.x * blockDim.x) {
        const int y = (int)(p / W), x = (int)(p % W);
        float xs[Q], ys[3];
#pragma unroll
        for (int i = 0; i < Q; ++i) xs[i] = a.guide[i * plane + p] - a.shift[i];
#pragma unroll
        for (int c = 0; c < 3; ++c) ys[c] = a.rad[c * plane + p] - a.shift[Q + c];
        const float *BS = a.BS;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            float d = BS[(C::X0 + i) * plane + p];
#pragma unroll
            for (int j = 0; j < Q; ++j) {
                const int ch = i <= j ? C::xx(i, j) : C::xx(j, i);
                d = fmaf(2.f * BS[ch * plane + p], xs[j], d);
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) d = fmaf(BS[C::xy(i, c) * plane + p], ys[c], d);
            // the applied guide: dz_i = sum_c Abar[i][c] g_c
            float inv_m = 1.f;
            if (a.rc > 0) {
                const float ny = (float)(min(y + a.rc, H - 1) - max(y - a.rc, 0) + 1);
                const float nx = (float)(min(x + a.rc, W - 1) - max(x - a.rc, 0) + 1);
                inv_m = 1.0f / (ny * nx);
            }
            float dz = 0.f;
#pragma unroll
            for (int c = 0; c < 3; ++c) dz = fmaf(a.BA[(3 * (i + 1) + c) * plane + p], a.g[c * plane + p], dz);
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
            float d = BS[(C::Y0 + c) * plane + p];
#pragma unroll
            for (int i = 0; i < Q; ++i) d = fmaf(BS[C::xy(i, c) * plane + p], xs[i], d);
            a.grad_rad[c * plane + p] = d;
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

cudaError_t launch_box_sum(const float *in, float *out, int nplanes, int H, int W, int rad, cudaStream_t st)
{
    const size_t smem = sizeof(float) * ((size_t)(kBH + 2 * rad) * (kBW + 2 * rad + 1) + (size_t)(kBH + 2 * rad) * (kBW + 1));
    cudaError_t e = cudaFuncSetAttribute(box_sum_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((W + kBW - 1) / kBW, (H + kBH - 1) / kBH, nplanes);
    box_sum_kernel<<<grid, kBThreads, smem, st>>>(in, out, H, W, rad);
    return cudaGetLastError();
}

cudaError_t launch_bwd_contract(int q, const BwdArgs &a, cudaStream_t st)
{
    const int grid = elem_grid((size_t)a.H * a.W);
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
