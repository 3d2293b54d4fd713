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
#include "flr_fp64_model.cuh"
#include "flr_internal.cuh"

namespace flr {
namespace {

constexpr int kDThreads = 128;

template <int Q>
__global__ void __launch_bounds__(kDThreads) flr_fp64_kernel(const Fp64Args a)
{
    const int lane = threadIdx.x & 31;
    const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nw = (int)((gridDim.x * blockDim.x) >> 5);
    const unsigned long long cnt = *a.flag_count;
    const int n = (int)(cnt < (unsigned long long)a.flag_cap ? cnt : (unsigned long long)a.flag_cap);
    const unsigned long long st0 = a.flag_start ? *a.flag_start : 0ull;
    const int start = (int)(st0 < (unsigned long long)n ? st0 : (unsigned long long)n);
    const size_t plane = (size_t)a.H * a.W;
    const float *s = a.shift;  // frame reference shift
    for (int e = start + gw; e < n; e += nw) {
        const int idx = a.flag_list[e];
        double A[Q][3], bv[3];
        dev::fp64_model<Q>(a.guide, a.rad, a.H, a.W, a.r, a.eps, idx, lane, s, A, bv);
        if (lane != 0) continue;
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
            if (bad && a.nonfinite) atomicAdd(a.nonfinite, (unsigned long long)bad);
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
