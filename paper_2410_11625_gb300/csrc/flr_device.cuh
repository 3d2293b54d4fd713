// flr_device.cuh -- device helpers shared by the FLR kernels (per-pixel and fast paths):
// the reference-shift sampler, the register Cholesky solve of the centred ridge model and
// the horizontal window sums of a shared-memory row.
#pragma once

#include "flr_internal.cuh"

namespace flr {
namespace dev {

// Mean of the inputs over a kShiftSamples^2 grid of pixel centres of [ya,yb) x [xa,xb),
// computed by one warp in a fixed order (identical in every CTA for the same region): lane l
// adds samples l, l + 32, ... in turn, then a shuffle tree.  The sample loop has a fixed
// trip count and is unrolled, so all of a lane's loads can be in flight at once.
template <int Q>
__device__ void sample_mean(float *dst, const float *__restrict__ guide,
                            const float *__restrict__ rad, int H, int W, int ya, int yb, int xa,
                            int xb, int lane)
{
    constexpr int NS = kShiftSamples;
    static_assert(NS * NS % 32 == 0, "every lane takes the same number of samples");
    const size_t plane = (size_t)H * W;
    float acc[Q + 3];
#pragma unroll
    for (int k = 0; k < Q + 3; ++k) acc[k] = 0.f;
#pragma unroll
    for (int it = 0; it < NS * NS / 32; ++it) {
        const int s = lane + 32 * it;
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

// ---- horizontal sums of one buffer row -------------------------------------------------
// out[x] = sum_{j=0}^{2K} in[x + j] for x in [x0, x0 + N) (x0 and the rows 16-byte aligned).
// The run's N + 2K input values are read from shared memory once, with 16-byte loads, into
// registers before anything is written (so in == out sums the row in place).  The first
// output is a direct (2K + 1)-term sum; the others add the differences
// d(x) = in[x + 2K] - in[x - 1], four per step as prefix sums of the step's differences, so
// the dependent chain is one add per four outputs.
template <int K, int N>
__device__ __forceinline__ void hsum_run(const float *in, float *out, int x0)
{
    constexpr int NV = N + 2 * K;
    float v[NV];
#pragma unroll
    for (int j = 0; j < NV; j += 4) {
        if (j + 3 < NV) {
            const float4 t = *reinterpret_cast<const float4 *>(in + x0 + j);
            v[j] = t.x, v[j + 1] = t.y, v[j + 2] = t.z, v[j + 3] = t.w;
        } else {
#pragma unroll
            for (int i = j; i < NV; ++i) v[i] = in[x0 + i];
        }
    }
    float S;
    {
        float t[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int j = 0; j <= 2 * K; ++j) t[j & 3] += v[j];
        S = (t[0] + t[1]) + (t[2] + t[3]);
    }
#pragma unroll
    for (int x = 0; x < N; x += 4) {
        float d[4], o[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int xo = x + k;
            d[k] = (xo > 0 && xo < N) ? v[xo + 2 * K] - v[xo - 1] : 0.f;
        }
        const float p1 = d[0], p2 = p1 + d[1], p3 = p2 + d[2], p4 = p3 + d[3];
        o[0] = S + p1;
        o[1] = S + p2;
        o[2] = S + p3;
        o[3] = S + p4;
        S = o[3];
        if (x + 3 < N) {
            *reinterpret_cast<float4 *>(out + x0 + x) = make_float4(o[0], o[1], o[2], o[3]);
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (x + k < N) out[x0 + x + k] = o[k];
        }
    }
}

}  // namespace dev
}  // namespace flr
