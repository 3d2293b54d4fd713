// flr_fp64.cu -- FP64 re-solve of the pixels the FP32 forward kernel flagged (sm_103a).
//
// The FP32 Cholesky loses about u * M_jj / d_j of relative precision at pivot j.  Pixels
// whose pivot ratio d_j / M_jj fell to the threshold tau or below are listed by the
// forward kernel; this kernel recomputes each one's window sums in FP64 directly from
// the float32 inputs (products of two floats are exact in double), centred on the pixel's
// own input values, and solves the same centred ridge system (Appendix, multiplicative
// term zero) by FP64 Cholesky.  The model then replaces the FP32 one: in the coefficient
// planes when coefficient averaging follows, or directly in the output otherwise.
// One warp per flagged pixel: lanes split the window's pixels, then a shuffle tree
// reduces the sums.  Rarely run, so it is written for clarity rather than speed.
#include <utility>

#include "flr_internal.cuh"

namespace flr {
namespace {

constexpr int kDThreads = 128;

template <int Q, int CH>
__device__ __forceinline__ void accumulate_one(double &acc, const double (&v)[Q + 3])
{
    constexpr int u = Chan<Q>::slot_u(CH), w = Chan<Q>::slot_v(CH);
    if constexpr (w < 0) acc += v[u];
    else acc += v[u] * v[w];
}

// S[ch] += the product that defines moment channel ch, for every channel.
template <int Q, int... I>
__device__ __forceinline__ void accumulate_moments(double (&S)[Chan<Q>::NCH], const double (&v)[Q + 3],
                                                   std::integer_sequence<int, I...>)
{
    (accumulate_one<Q, I>(S[I], v), ...);
}

template <int Q>
__global__ void __launch_bounds__(kDThreads) flr_fp64_kernel(const Fp64Args a)
{
    using C = Chan<Q>;
    const int lane = threadIdx.x & 31;
    const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nw = (int)((gridDim.x * blockDim.x) >> 5);
    const unsigned long long cnt = *a.flag_count;
    const int n = (int)(cnt < (unsigned long long)a.flag_cap ? cnt : (unsigned long long)a.flag_cap);
    const unsigned long long st0 = a.flag_start ? *a.flag_start : 0ull;
    const int start = (int)(st0 < (unsigned long long)n ? st0 : (unsigned long long)n);
    const int H = a.H, W = a.W, r = a.r;
    const size_t plane = (size_t)H * W;
    for (int e = start + gw; e < n; e += nw) {
        const int idx = a.flag_list[e];
        const int y = idx / W, x = idx % W;
        const int ylo = max(0, y - r), yhi = min(H - 1, y + r);
        const int xlo = max(0, x - r), xhi = min(W - 1, x + r);
        const int ww = xhi - xlo + 1, npx = (yhi - ylo + 1) * ww;
        double cen[Q + 3];
#pragma unroll
        for (int k = 0; k < Q; ++k) cen[k] = (double)a.guide[k * plane + idx];
#pragma unroll
        for (int c = 0; c < 3; ++c) cen[Q + c] = (double)a.rad[c * plane + idx];
        double S[C::NCH];
#pragma unroll
        for (int ch = 0; ch < C::NCH; ++ch) S[ch] = 0.0;
        for (int p = lane; p < npx; p += 32) {
            const size_t off = (size_t)(ylo + p / ww) * W + (xlo + p % ww);
            double v[Q + 3];
#pragma unroll
            for (int k = 0; k < Q; ++k) v[k] = (double)a.guide[k * plane + off] - cen[k];
#pragma unroll
            for (int c = 0; c < 3; ++c) v[Q + c] = (double)a.rad[c * plane + off] - cen[Q + c];
            accumulate_moments<Q>(S, v, std::make_integer_sequence<int, C::NCH>{});
        }
#pragma unroll
        for (int ch = 0; ch < C::NCH; ++ch)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) S[ch] += __shfl_xor_sync(0xffffffffu, S[ch], o);
        if (lane != 0) continue;

        const double inv_n = 1.0 / (double)npx;
        double mu[Q], muy[3], L[Q][Q], D[Q][3], A[Q][3];
#pragma unroll
        for (int i = 0; i < Q; ++i) mu[i] = S[C::X0 + i] * inv_n;
#pragma unroll
        for (int c = 0; c < 3; ++c) muy[c] = S[C::Y0 + c] * inv_n;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
#pragma unroll
            for (int j = 0; j <= i; ++j)
                L[i][j] = S[C::xx(j, i)] * inv_n - mu[i] * mu[j] + (i == j ? a.eps : 0.0);
#pragma unroll
            for (int c = 0; c < 3; ++c) D[i][c] = S[C::xy(i, c)] * inv_n - mu[i] * muy[c];
        }
#pragma unroll
        for (int j = 0; j < Q; ++j) {
            double d = L[j][j];
#pragma unroll
            for (int k = 0; k < j; ++k) d -= L[j][k] * L[j][k];
            d = sqrt(d > a.eps ? d : (a.eps > 0.0 ? a.eps : 1e-300));  // every exact pivot is >= eps
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
        // bias relative to the frame reference shift s: b = mu_y + cen_y - s_y - a^T (mu + cen - s)
        const float *s = a.shift;
        double bv[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            double b = muy[c] + (cen[Q + c] - (double)s[Q + c]);
#pragma unroll
            for (int i = 0; i < Q; ++i) b -= A[i][c] * (mu[i] + (cen[i] - (double)s[i]));
            bv[c] = b;
        }
        if (a.rc == 0 && !a.force_coef) {
            const float *zg = a.map_guide ? a.map_guide : a.guide;
            int bad = 0;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                double o = bv[c];
#pragma unroll
                for (int i = 0; i < Q; ++i) o += A[i][c] * ((double)zg[i * plane + idx] - (double)s[i]);
                const float of = (float)(o + (double)s[Q + c]);
                a.out[c * plane + idx] = of;
                bad += !isfinite(of);
            }
            if (bad && a.nonfinite && lane == 0) atomicAdd(a.nonfinite, (unsigned long long)bad);
        } else {
#pragma unroll
            for (int c = 0; c < 3; ++c) a.coef[c * plane + idx] = (float)bv[c];
#pragma unroll
            for (int i = 0; i < Q; ++i)
#pragma unroll
                for (int c = 0; c < 3; ++c) a.coef[(3 * (i + 1) + c) * plane + idx] = (float)A[i][c];
        }
    }
}

template <int Q>
cudaError_t launch_fp64_q(const Fp64Args &a, int n_sm, cudaStream_t st)
{
    flr_fp64_kernel<Q><<<2 * n_sm, kDThreads, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_fp64(int q, const Fp64Args &a, int n_sm, cudaStream_t st)
{
    switch (q) {
    case 1: return launch_fp64_q<1>(a, n_sm, st);
    case 2: return launch_fp64_q<2>(a, n_sm, st);
    case 3: return launch_fp64_q<3>(a, n_sm, st);
    case 4: return launch_fp64_q<4>(a, n_sm, st);
    case 5: return launch_fp64_q<5>(a, n_sm, st);
    case 6: return launch_fp64_q<6>(a, n_sm, st);
    case 7: return launch_fp64_q<7>(a, n_sm, st);
    case 8: return launch_fp64_q<8>(a, n_sm, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace flr
