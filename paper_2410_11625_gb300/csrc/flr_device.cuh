// flr_device.cuh -- device helpers shared by the FLR kernels (per-pixel and fast paths):
// the reference-shift sampler and the register Cholesky solve of the centred ridge model.
#pragma once

#include "flr_internal.cuh"

namespace flr {
namespace dev {

// Mean of the inputs over a kShiftSamples^2 grid of pixel centres of [ya,yb) x [xa,xb),
// computed by one warp in a fixed order (identical in every CTA for the same region).
template <int Q>
__device__ void sample_mean(float *dst, const float *__restrict__ guide,
                            const float *__restrict__ rad, int H, int W, int ya, int yb, int xa,
                            int xb, int lane)
{
    constexpr int NS = kShiftSamples;
    const size_t plane = (size_t)H * W;
    float acc[Q + 3];
#pragma unroll
    for (int k = 0; k < Q + 3; ++k) acc[k] = 0.f;
    for (int s = lane; s < NS * NS; s += 32) {
        const int iy = s / NS, ix = s % NS;
        const int y = ya + (int)(((long long)(2 * iy + 1) * (yb - ya)) / (2 * NS));
        const int x = xa + (int)(((long long)(2 * ix + 1) * (xb - xa)) / (2 * NS));
        const size_t off = (size_t)y * W + x;
#pragma unroll
        for (int k = 0; k < Q; ++k) acc[k] += __ldg(guide + k * plane + off);
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[Q + c] += __ldg(rad + c * plane + off);
    }
#pragma unroll
    for (int k = 0; k < Q + 3; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
    }
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < Q + 3; ++k) dst[k] = acc[k] * (1.0f / (NS * NS));
    }
}

__device__ __forceinline__ constexpr int tri(int i, int j) { return i * (i + 1) / 2 + j; }  // i >= j

// X = M^{-1} B for the factor M = L L^T (packed lower triangle, 1/L_jj in inv_d), 3 RHS.
template <int Q>
__device__ __forceinline__ void chol_solve3(const float (&L)[Q * (Q + 1) / 2], const float (&inv_d)[Q],
                                            const float (&B)[Q][3], float (&X)[Q][3])
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float z[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            float t = B[i][c];
#pragma unroll
            for (int k = 0; k < Q; ++k)
                if (k < i) t = fmaf(-L[tri(i, k)], z[k], t);
            z[i] = t * inv_d[i];
        }
#pragma unroll
        for (int ii = 0; ii < Q; ++ii) {
            const int i = Q - 1 - ii;
            float t = z[i];
#pragma unroll
            for (int k = 0; k < Q; ++k)
                if (k > i) t = fmaf(-L[tri(k, i)], X[k][c], t);
            X[i][c] = t * inv_d[i];
        }
    }
}

// In-place left-looking Cholesky M = L L^T of the packed lower triangle, keeping 1 / L_jj.
// Returns whether a pivot fell to tau M_jj or below; pivots are floored at `floor` (every
// exact pivot of M is at least that).  Inner loops run to Q with a predicate so that every
// loop unrolls completely and L stays in registers.
template <int Q>
__device__ __forceinline__ bool chol_factor(float (&L)[Q * (Q + 1) / 2], float floor, float tau, float (&inv_d)[Q])
{
    bool low = false;
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        const float mjj = L[tri(j, j)];
        float d = mjj;
#pragma unroll
        for (int k = 0; k < Q; ++k)
            if (k < j) d = fmaf(-L[tri(j, k)], L[tri(j, k)], d);
        low |= !(d > tau * mjj);
        d = fmaxf(d, floor);
        const float il = rsqrtf(d);
        inv_d[j] = il;
        L[tri(j, j)] = d * il;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            if (i > j) {
                float t = L[tri(i, j)];
#pragma unroll
                for (int k = 0; k < Q; ++k)
                    if (k < j) t = fmaf(-L[tri(i, k)], L[tri(j, k)], t);
                L[tri(i, j)] = t * il;
            }
        }
    }
    return low;
}

// Centred ridge solve of one pixel from its window sums S(ch) = Sp[ch * VS].
// Returns the model (a, b) in the CTA-shifted coordinates and whether a pivot fell low.
template <int Q>
__device__ __forceinline__ bool solve_pixel(const float *Sp, int VS, float n, float eps,
                                            float tau, float (&A)[Q][3], float (&bv)[3],
                                            float (&mu)[Q], float (&muy)[3],
                                            float (&L)[Q * (Q + 1) / 2], float (&inv_d)[Q])
{
    using C = Chan<Q>;
    // A one-pixel window (n = 1) has centred moments exactly zero.  Dividing the guide
    // moments by infinity there (inv_nx = 0) makes mu = 0, M = eps I and D = 0 exactly,
    // so a = 0 and b = mu_y, instead of leaving x x - x x to a rounding that 1/eps would
    // amplify.
    const float inv_n = 1.0f / n;
    const float inv_nx = n > 1.5f ? inv_n : 0.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) mu[i] = Sp[(C::X0 + i) * VS] * inv_nx;
#pragma unroll
    for (int c = 0; c < 3; ++c) muy[c] = Sp[(C::Y0 + c) * VS] * inv_n;
    // M = S/n - mu mu^T + eps I (lower triangle), D = XY/n - mu muy^T
#pragma unroll
    for (int i = 0; i < Q; ++i)
#pragma unroll
        for (int j = 0; j < Q; ++j) {
            if (j <= i) {
                float m = fmaf(-mu[i], mu[j], Sp[C::xx(j, i) * VS] * inv_nx);
                if (i == j) m += eps;
                L[tri(i, j)] = m;
            }
        }
    float D[Q][3];
#pragma unroll
    for (int i = 0; i < Q; ++i)
#pragma unroll
        for (int c = 0; c < 3; ++c) D[i][c] = fmaf(-mu[i], muy[c], Sp[C::xy(i, c) * VS] * inv_nx);

    const bool low = chol_factor<Q>(L, eps > 0.f ? eps : 1e-30f, tau, inv_d);  // every exact pivot is >= eps
    // L z = D, then L^T a = z
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float z[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            float t = D[i][c];
#pragma unroll
            for (int k = 0; k < Q; ++k)
                if (k < i) t = fmaf(-L[tri(i, k)], z[k], t);
            z[i] = t * inv_d[i];
        }
#pragma unroll
        for (int ii = 0; ii < Q; ++ii) {
            const int i = Q - 1 - ii;
            float t = z[i];
#pragma unroll
            for (int k = 0; k < Q; ++k)
                if (k > i) t = fmaf(-L[tri(k, i)], A[k][c], t);
            A[i][c] = t * inv_d[i];
        }
        float b = muy[c];
#pragma unroll
        for (int i = 0; i < Q; ++i) b = fmaf(-A[i][c], mu[i], b);
        bv[c] = b;
    }
    return low;
}

}  // namespace dev
}  // namespace flr
