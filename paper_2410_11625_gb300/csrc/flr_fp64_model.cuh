// flr_fp64_model.cuh -- FP64 model of one pixel's window, computed by one warp from the
// float32 inputs (used by the FP64 re-solve kernels of the per-pixel path).
//
// What it computes (Sec. 3.1-3.2 and the Appendix): the window sums over the clipped radius-r
// window of the pixel, in double precision directly from the inputs (products of two floats
// are exact in double), centred on the pixel's own input values, then the centred ridge
// model M = S/n - mu mu^T + eps I, a = M^{-1} (X^T Y / n - mu mu_y^T), b = mu_y - a^T mu by FP64
// Cholesky.  The bias is returned relative to a reference shift s: the model maps a guide
// vector z to s_y + b + a^T (z - s).
#pragma once

#include <utility>

#include "flr_internal.cuh"

namespace flr {
namespace dev {

template <int Q, int CH>
__device__ __forceinline__ void fp64_accumulate_one(double &acc, const double (&v)[Q + 3])
{
    constexpr int u = Chan<Q>::slot_u(CH), w = Chan<Q>::slot_v(CH);
    if constexpr (w < 0) acc += v[u];
    else acc += v[u] * v[w];
}

// S[ch] += the product that defines moment channel ch, for every channel.
template <int Q, int... I>
__device__ __forceinline__ void fp64_accumulate(double (&S)[Chan<Q>::NCH], const double (&v)[Q + 3],
                                                std::integer_sequence<int, I...>)
{
    (fp64_accumulate_one<Q, I>(S[I], v), ...);
}

// The model of pixel idx = y * W + x.  Every lane of the warp must call it; the result is
// valid on lane 0.  s: the reference shift (Q guides then 3 radiance channels).
template <int Q>
__device__ void fp64_model(const float *__restrict__ guide, const float *__restrict__ rad, int H, int W, int r,
                           double eps, int idx, int lane, const float *s, double (&A)[Q][3], double (&bv)[3])
{
    using C = Chan<Q>;
    const size_t plane = (size_t)H * W;
    const int y = idx / W, x = idx % W;
    const int ylo = max(0, y - r), yhi = min(H - 1, y + r);
    const int xlo = max(0, x - r), xhi = min(W - 1, x + r);
    const int ww = xhi - xlo + 1, npx = (yhi - ylo + 1) * ww;
    double cen[Q + 3];
#pragma unroll
    for (int k = 0; k < Q; ++k) cen[k] = (double)guide[k * plane + idx];
#pragma unroll
    for (int c = 0; c < 3; ++c) cen[Q + c] = (double)rad[c * plane + idx];
    double S[C::NCH];
#pragma unroll
    for (int ch = 0; ch < C::NCH; ++ch) S[ch] = 0.0;
    for (int p = lane; p < npx; p += 32) {
        const size_t off = (size_t)(ylo + p / ww) * W + (xlo + p % ww);
        double v[Q + 3];
#pragma unroll
        for (int k = 0; k < Q; ++k) v[k] = (double)guide[k * plane + off] - cen[k];
#pragma unroll
        for (int c = 0; c < 3; ++c) v[Q + c] = (double)rad[c * plane + off] - cen[Q + c];
        fp64_accumulate<Q>(S, v, std::make_integer_sequence<int, C::NCH>{});
    }
#pragma unroll
    for (int ch = 0; ch < C::NCH; ++ch)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) S[ch] += __shfl_xor_sync(0xffffffffu, S[ch], o);
    if (lane != 0) return;

    const double inv_n = 1.0 / (double)npx;
    double mu[Q], muy[3], L[Q][Q], D[Q][3];
#pragma unroll
    for (int i = 0; i < Q; ++i) mu[i] = S[C::X0 + i] * inv_n;
#pragma unroll
    for (int c = 0; c < 3; ++c) muy[c] = S[C::Y0 + c] * inv_n;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
#pragma unroll
        for (int j = 0; j <= i; ++j) L[i][j] = S[C::xx(j, i)] * inv_n - mu[i] * mu[j] + (i == j ? eps : 0.0);
#pragma unroll
        for (int c = 0; c < 3; ++c) D[i][c] = S[C::xy(i, c)] * inv_n - mu[i] * muy[c];
    }
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        double d = L[j][j];
#pragma unroll
        for (int k = 0; k < j; ++k) d -= L[j][k] * L[j][k];
        d = sqrt(d > eps ? d : (eps > 0.0 ? eps : 1e-300));  // every exact pivot is >= eps
        L[j][j] = d;
#pragma unroll
        for (int i = j + 1; i < Q; ++i) {
            double t = L[i][j];
#pragma unroll
            for (int k = 0; k < j; ++k) t -= L[i][k] * L[j][k];
            L[i][j] = t / d;
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        double z[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            double t = D[i][c];
#pragma unroll
            for (int k = 0; k < i; ++k) t -= L[i][k] * z[k];
            z[i] = t / L[i][i];
        }
#pragma unroll
        for (int i = Q - 1; i >= 0; --i) {
            double t = z[i];
#pragma unroll
            for (int k = i + 1; k < Q; ++k) t -= L[k][i] * A[k][c];
            A[i][c] = t / L[i][i];
        }
    }
    // bias relative to s: b = mu_y + cen_y - s_y - a^T (mu + cen - s)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        double b = muy[c] + (cen[Q + c] - (double)s[Q + c]);
#pragma unroll
        for (int i = 0; i < Q; ++i) b -= A[i][c] * (mu[i] + (cen[i] - (double)s[i]));
        bv[c] = b;
    }
}

}  // namespace dev
}  // namespace flr
