// flr_fast_stages.cuh -- the four stages of the paper's fast FLR (Sec. 3.2, 3.2.1) as device
// functions, shared by the one-kernel-per-stage path (flr_fast.cu) and the persistent
// batched kernel (flr_batch.cu).
#pragma once

#include <utility>

#include "flr_device.cuh"
#include "flr_internal.cuh"

namespace flr {
namespace fast {

constexpr int kMaxTaps = 8;

// acc += the product that defines moment channel CH (slots fixed at compile time)
template <int Q, int CH>
__device__ __forceinline__ void moment_one(float &acc, const float (&v)[Q + 3])
{
    constexpr int u = Chan<Q>::slot_u(CH), w = Chan<Q>::slot_v(CH);
    if constexpr (w < 0) acc += v[u];
    else acc = fmaf(v[u], v[w], acc);
}

template <int Q, int... I>
__device__ __forceinline__ void moments_all(float (&acc)[Chan<Q>::NCH], const float (&v)[Q + 3],
                                            std::integer_sequence<int, I...>)
{
    (moment_one<Q, I>(acc[I], v), ...);
}

// L2 eviction priorities for the full-resolution planes.  The moment stage reads the guide
// planes with evict_last so that they are still in L2 when the apply stage reads them again
// as the map guide (66 MB at 1080p, half of L2); the radiance, read once, and the apply's own
// reads take evict_first, so they do not push the guides out.
__device__ __forceinline__ uint64_t l2_policy_keep()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;\n" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t l2_policy_stream()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(p));
    return p;
}
// 8-byte read-only load with an L2 eviction policy
__device__ __forceinline__ float2 ld_f2_hint(const float *p, uint64_t pol)
{
    float2 v;
    asm volatile("ld.global.nc.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;\n"
                 : "=f"(v.x), "=f"(v.y)
                 : "l"(p), "l"(pol));
    return v;
}

struct FastArgs {
    const float *guide, *rad, *map_guide;  // model inputs [q|3][Hi][Wi], map guide [q][Ho][Wo]
    float *out;                            // [3][Ho][Wo]
    float *blk;   // [NCH + Q+3][Hb][Wb]: block sums relative to the block's reference, then that reference
    float *tmp;   // [NCH + 1][Hb][Wb]: horizontally blurred sums (same reference), weighted count
    float *coef;  // [(Q+1)*3][Hb][Wb]: block models relative to the frame reference
    float *tmp2;  // parameter gradients: [NCH + 1][Hb][Wb] horizontal blur with the weights' sigma-derivative
    float *dcoef; // parameter gradients: [3][(Q+1)*3][Hb][Wb] model tangents (sigma, eps, eps_mul)
    float *shift;                          // frame reference shift, Q + 3 floats
    unsigned long long *flag_count;
    int Hi, Wi, Ho, Wo, Hb, Wb, F, s, taps;
    float eps, tau;
    int appendix;   // 1: the Appendix's regularised normalised solve (additive eps, multiplicative eps_mul)
    float eps_mul;
    float w[2 * kMaxTaps + 1];             // Gaussian weights
    float wd[2 * kMaxTaps + 1];            // their derivatives with respect to sigma (parameter gradients)
    int *status = nullptr;                 // set to 1 if a bounded device wait ran out (may be NULL)
};

// 1. block moments.  Block (i, j) covers input rows [iF, iF+F) and columns [jF, jF+F).
// Work item (by, cx): block row by, input columns [512 cx, 512 cx + 512); 256 threads, each
// summing two adjacent columns over the F rows (one 8-byte load per plane and row when the
// rows are 8-byte aligned), then a shuffle tree over the F / 2 lanes of a block.
template <int Q, int F>
__device__ __forceinline__ void stage_moments(const FastArgs &a, int by, int cx)
{
    using C = Chan<Q>;
    constexpr int NS = Q + 3, LPB = F / 2;  // lanes per block
    static_assert(F >= 2 && 32 % F == 0, "block width");
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (by == 0 && cx == 0 && warp == 0) {
        // the frame reference the models are expressed in (used by the solve and apply)
        __shared__ float s_ref[NS];
        dev::sample_mean<Q>(s_ref, a.guide, a.rad, a.Hi, a.Wi, 0, a.Hi, 0, a.Wi, lane);
        __syncwarp();
        if (lane < NS) a.shift[lane] = s_ref[lane];
    }
    const int x = cx * 512 + 2 * tid;  // this thread's columns x, x + 1
    const size_t plane = (size_t)a.Hi * a.Wi;
    const int y0 = by * F, y1 = min(y0 + F, a.Hi);
    // the block's reference: its top-left input pixel (column x of lane (lane & ~(LPB-1)))
    float ref[NS];
    {
        const size_t off0 = (size_t)y0 * a.Wi + min(x, a.Wi - 1);
#pragma unroll
        for (int k = 0; k < Q; ++k) ref[k] = __ldg(a.guide + k * plane + off0);
#pragma unroll
        for (int c = 0; c < 3; ++c) ref[Q + c] = __ldg(a.rad + c * plane + off0);
#pragma unroll
        for (int k = 0; k < NS; ++k) ref[k] = __shfl_sync(0xffffffffu, ref[k], lane & ~(LPB - 1));
    }
    float acc[C::NCH];
#pragma unroll
    for (int c = 0; c < C::NCH; ++c) acc[c] = 0.f;
    if (x < a.Wi) {
        // with an even width, x + 1 < Wi and the 8-byte loads are aligned (x even, planes
        // 16-byte aligned)
        const bool vec = (a.Wi & 1) == 0;
        const bool two = x + 1 < a.Wi;
        const uint64_t pol_keep = l2_policy_keep(), pol_stream = l2_policy_stream();
#pragma unroll
        for (int yy = 0; yy < F; ++yy) {
            const int y = y0 + yy;
            if (y >= y1) break;
            const size_t off = (size_t)y * a.Wi + x;
            float v0[NS], v1[NS];
            if (vec) {
#pragma unroll
                for (int k = 0; k < Q; ++k) {
                    const float2 g = ld_f2_hint(a.guide + k * plane + off, pol_keep);
                    v0[k] = g.x - ref[k];
                    v1[k] = g.y - ref[k];
                }
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float2 g = ld_f2_hint(a.rad + c * plane + off, pol_stream);
                    v0[Q + c] = g.x - ref[Q + c];
                    v1[Q + c] = g.y - ref[Q + c];
                }
            } else {
#pragma unroll
                for (int k = 0; k < Q; ++k) {
                    v0[k] = __ldg(a.guide + k * plane + off) - ref[k];
                    v1[k] = two ? __ldg(a.guide + k * plane + off + 1) - ref[k] : 0.f;
                }
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    v0[Q + c] = __ldg(a.rad + c * plane + off) - ref[Q + c];
                    v1[Q + c] = two ? __ldg(a.rad + c * plane + off + 1) - ref[Q + c] : 0.f;
                }
            }
            moments_all<Q>(acc, v0, std::make_integer_sequence<int, C::NCH>{});
            moments_all<Q>(acc, v1, std::make_integer_sequence<int, C::NCH>{});
        }
    }
    // reduce over the LPB lanes of each block (blocks never straddle a warp: 32 % LPB == 0)
#pragma unroll
    for (int ch = 0; ch < C::NCH; ++ch)
#pragma unroll
        for (int o = 1; o < LPB; o <<= 1) acc[ch] += __shfl_xor_sync(0xffffffffu, acc[ch], o);
    if ((lane & (LPB - 1)) == 0 && x < a.Wi) {
        const int bx = x / F;
        const size_t bplane = (size_t)a.Hb * a.Wb;
        const size_t boff = (size_t)by * a.Wb + bx;
#pragma unroll
        for (int ch = 0; ch < C::NCH; ++ch) a.blk[ch * bplane + boff] = acc[ch];
#pragma unroll
        for (int k = 0; k < NS; ++k) a.blk[(C::NCH + k) * bplane + boff] = ref[k];
    }
}

// Input pixels of block index b along an axis of n pixels split into blocks of F.
__device__ __forceinline__ float block_len(int b, int F, int n) { return (float)min(F, n - b * F); }

// acc += w * (sums of block b re-expressed relative to another reference), given
// d = ref_b - ref_target for the Q + 3 input slots and the block's pixel count nb:
//   sum (v + d) = L + nb d,   sum (v + d)(v' + d') = S + L d' + d L' + nb d d'.
template <int Q>
__device__ __forceinline__ void accumulate_shifted(float (&acc)[Chan<Q>::NCH], const float *src, size_t stride,
                                                   const float (&d)[Q + 3], float nb, float w)
{
    using C = Chan<Q>;
    float L[Q + 3];
#pragma unroll
    for (int k = 0; k < Q + 3; ++k) L[k] = src[(C::X0 + k) * stride];  // X0..Y0+2 are the linear sums
#pragma unroll
    for (int k = 0; k < Q + 3; ++k) acc[C::X0 + k] = fmaf(w, fmaf(nb, d[k], L[k]), acc[C::X0 + k]);
#pragma unroll
    for (int i = 0; i < Q; ++i)
#pragma unroll
        for (int j = 0; j < Q; ++j)
            if (j >= i) {
                const int ch = C::xx(i, j);
                const float t = fmaf(nb * d[i], d[j], fmaf(L[i], d[j], fmaf(d[i], L[j], src[ch * stride])));
                acc[ch] = fmaf(w, t, acc[ch]);
            }
#pragma unroll
    for (int i = 0; i < Q; ++i)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int ch = C::xy(i, c);
            const float t = fmaf(nb * d[i], d[Q + c], fmaf(L[i], d[Q + c], fmaf(d[i], L[Q + c], src[ch * stride])));
            acc[ch] = fmaf(w, t, acc[ch]);
        }
}

// 2. horizontal Gaussian over the block grid, clipped: every neighbour's sums re-expressed
// relative to the target block's reference before weighting; also the weighted count.
template <int Q>
__device__ __forceinline__ void stage_blur_h(const FastArgs &a, size_t k)
{
    using C = Chan<Q>;
    constexpr int NS = Q + 3;
    const size_t bplane = (size_t)a.Hb * a.Wb;
    if (k >= bplane) return;
    const int by = (int)(k / a.Wb), bx = (int)(k % a.Wb);
    float rk[NS];
#pragma unroll
    for (int q = 0; q < NS; ++q) rk[q] = a.blk[(C::NCH + q) * bplane + k];
    float acc[C::NCH];
#pragma unroll
    for (int c = 0; c < C::NCH; ++c) acc[c] = 0.f;
    float n = 0.f;
    const float rows = block_len(by, a.F, a.Hi);
    for (int dd = -a.taps; dd <= a.taps; ++dd) {
        const int xx = bx + dd;
        if (xx < 0 || xx >= a.Wb) continue;
        const size_t kb = (size_t)by * a.Wb + xx;
        float d[NS];
#pragma unroll
        for (int q = 0; q < NS; ++q) d[q] = a.blk[(C::NCH + q) * bplane + kb] - rk[q];
        const float nb = rows * block_len(xx, a.F, a.Wi);
        const float w = a.w[dd + a.taps];
        accumulate_shifted<Q>(acc, a.blk + kb, bplane, d, nb, w);
        n = fmaf(w, nb, n);
    }
#pragma unroll
    for (int c = 0; c < C::NCH; ++c) a.tmp[c * bplane + k] = acc[c];
    a.tmp[C::NCH * bplane + k] = n;
}

// The Appendix's regularised normalised solve of one block (additive term eps, multiplicative
// term eps_mul), in an equivalent un-normalised form.  With D_s = diag(sigma^),
// C^ + eps I = D_s^-1 (W^ + eps D_s^2) D_s^-1 and B^ = D_s^-1 D, so the model
// ((x - mu) / sigma^) A^ has guide coefficients a = A^ / sigma^ = (W^ + eps diag(W^))^-1 D:
// one Cholesky solve of W^ with its diagonal scaled by (1 + eps), no divisions by sigma^.
// W^ = W + eps_mul (mu mu^T + diag(mu^2)) + eps I takes the block's absolute guide means,
// ref + (mean of the sums taken relative to ref); W and D are shift-invariant.  Returns the
// model in the block-shifted coordinates, as solve_pixel, with the factor of M, and whether
// a pivot fell low.
template <int Q>
__device__ __forceinline__ bool solve_appendix(const float *Sp, int VS, float n, float eps, float eps_mul,
                                               float tau, const float *ref, float (&A)[Q][3], float (&bv)[3],
                                               float (&mu)[Q], float (&muy)[3], float (&L)[Q * (Q + 1) / 2],
                                               float (&inv_d)[Q])
{
    using C = Chan<Q>;
    // a one-pixel block: the guide moments drop out (a = 0, b = mu_y), as in solve_pixel
    const float inv_n = 1.0f / n;
    const float inv_nx = n > 1.5f ? inv_n : 0.f;
    float ma[Q], D[Q][3];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        mu[i] = Sp[(C::X0 + i) * VS] * inv_nx;
        ma[i] = ref[i] + mu[i];
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) muy[c] = Sp[(C::Y0 + c) * VS] * inv_n;
    const float grow = 1.f + eps;
#pragma unroll
    for (int i = 0; i < Q; ++i)
#pragma unroll
        for (int j = 0; j < Q; ++j) {
            if (j <= i) {
                float m = fmaf(-mu[i], mu[j], Sp[C::xx(j, i) * VS] * inv_nx);
                m = fmaf(eps_mul * ma[i], ma[j], m);
                if (i == j) m = (fmaf(eps_mul * ma[i], ma[i], m) + eps) * grow;
                L[dev::tri(i, j)] = m;
            }
        }
#pragma unroll
    for (int i = 0; i < Q; ++i)
#pragma unroll
        for (int c = 0; c < 3; ++c) D[i][c] = fmaf(-mu[i], muy[c], Sp[C::xy(i, c) * VS] * inv_nx);
    const bool low = dev::chol_factor<Q>(L, eps > 0.f ? eps : 1e-30f, tau, inv_d);  // every exact pivot is >= eps
    dev::chol_solve3<Q>(L, inv_d, D, A);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float b = muy[c];
#pragma unroll
        for (int i = 0; i < Q; ++i) b = fmaf(-A[i][c], mu[i], b);
        bv[c] = b;
    }
    return low;
}

// 3. vertical Gaussian + per-block solve; S: this thread's column of a [NCH][stride] buffer
template <int Q>
__device__ __forceinline__ void stage_blur_v_solve(const FastArgs &a, size_t k, float *S, int stride)
{
    using C = Chan<Q>;
    const size_t bplane = (size_t)a.Hb * a.Wb;
    if (k >= bplane) return;
    const int by = (int)(k / a.Wb), bx = (int)(k % a.Wb);
    constexpr int NS = Q + 3;
    float rk[NS];
#pragma unroll
    for (int q = 0; q < NS; ++q) rk[q] = a.blk[(C::NCH + q) * bplane + k];
    float n = 0.f;
    {
        float acc[C::NCH];
#pragma unroll
        for (int c = 0; c < C::NCH; ++c) acc[c] = 0.f;
        for (int dd = -a.taps; dd <= a.taps; ++dd) {
            const int yy = by + dd;
            if (yy < 0 || yy >= a.Hb) continue;
            const size_t kb = (size_t)yy * a.Wb + bx;
            float d[NS];
#pragma unroll
            for (int q = 0; q < NS; ++q) d[q] = a.blk[(C::NCH + q) * bplane + kb] - rk[q];
            const float nb = a.tmp[C::NCH * bplane + kb];  // weighted count of that row's sums
            const float w = a.w[dd + a.taps];
            accumulate_shifted<Q>(acc, a.tmp + kb, bplane, d, nb, w);
            n = fmaf(w, nb, n);
        }
#pragma unroll
        for (int c = 0; c < C::NCH; ++c) S[c * stride] = acc[c];
    }
    float A[Q][3], bv[3], mu[Q], muy[3];
    bool low;
    {
        float L[Q * (Q + 1) / 2], inv_d[Q];
        low = a.appendix ? solve_appendix<Q>(S, stride, n, a.eps, a.eps_mul, a.tau, rk, A, bv, mu, muy, L, inv_d)
                         : dev::solve_pixel<Q>(S, stride, n, a.eps, a.tau, A, bv, mu, muy, L, inv_d);
    }
    if (low && a.tau > 0.f) {
        // FP64 re-solve of this block from the same (FP32) window sums
        atomicAdd(a.flag_count, 1ull);
        const double inv_n = 1.0 / (double)n;
        double dmu[Q], dmuy[3], M[Q][Q], D[Q][3];
#pragma unroll
        for (int i = 0; i < Q; ++i) dmu[i] = (double)S[(C::X0 + i) * stride] * inv_n;
#pragma unroll
        for (int c = 0; c < 3; ++c) dmuy[c] = (double)S[(C::Y0 + c) * stride] * inv_n;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
#pragma unroll
            for (int j = 0; j < Q; ++j)
                if (j <= i) {
                    M[i][j] = (double)S[C::xx(j, i) * stride] * inv_n - dmu[i] * dmu[j] + (i == j ? (double)a.eps : 0.0);
                    if (a.appendix) {  // W^ with its diagonal scaled by (1 + eps), as solve_appendix
                        const double mi = (double)rk[i] + dmu[i], mj = (double)rk[j] + dmu[j];
                        M[i][j] += (double)a.eps_mul * mi * mj;
                        if (i == j) M[i][j] = (M[i][j] + (double)a.eps_mul * mi * mi) * (1.0 + (double)a.eps);
                    }
                }
#pragma unroll
            for (int c = 0; c < 3; ++c) D[i][c] = (double)S[C::xy(i, c) * stride] * inv_n - dmu[i] * dmuy[c];
        }
#pragma unroll
        for (int j = 0; j < Q; ++j) {
            double d = M[j][j];
#pragma unroll
            for (int kk = 0; kk < Q; ++kk)
                if (kk < j) d -= M[j][kk] * M[j][kk];
            // every exact pivot is >= eps; rounding in the FP32 sums must not push it below
            d = sqrt(fmax(d, a.eps > 0.f ? (double)a.eps : 1e-300));
            M[j][j] = d;
#pragma unroll
            for (int i = 0; i < Q; ++i)
                if (i > j) {
                    double t = M[i][j];
#pragma unroll
                    for (int kk = 0; kk < Q; ++kk)
                        if (kk < j) t -= M[i][kk] * M[j][kk];
                    M[i][j] = t / d;
                }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            double z[Q], x[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                double t = D[i][c];
#pragma unroll
                for (int kk = 0; kk < Q; ++kk)
                    if (kk < i) t -= M[i][kk] * z[kk];
                z[i] = t / M[i][i];
            }
#pragma unroll
            for (int ii = 0; ii < Q; ++ii) {
                const int i = Q - 1 - ii;
                double t = z[i];
#pragma unroll
                for (int kk = 0; kk < Q; ++kk)
                    if (kk > i) t -= M[kk][i] * x[kk];
                x[i] = t / M[i][i];
            }
            double b = dmuy[c];
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                A[i][c] = (float)x[i];
                b -= x[i] * dmu[i];
            }
            bv[c] = (float)b;
        }
    }
    // the model was fitted relative to this block's reference; re-express the bias
    // relative to the frame reference the apply step uses
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float bb = bv[c] + (rk[Q + c] - a.shift[Q + c]);
#pragma unroll
        for (int i = 0; i < Q; ++i) bb = fmaf(-A[i][c], rk[i] - a.shift[i], bb);
        a.coef[c * bplane + k] = bb;
    }
#pragma unroll
    for (int i = 0; i < Q; ++i)
#pragma unroll
        for (int c = 0; c < 3; ++c) a.coef[(3 * (i + 1) + c) * bplane + k] = A[i][c];
}

// 3'. Tangents of the block models with respect to the Gaussian's sigma and the
// regularisation terms, for their gradients (Sec. 3.2 learns them by backpropagation).  The
// vertical blur gives the blurred sums S from tmp (the horizontal blur, weights w) and
// dS/dsigma from tmp2 (the horizontal blur with w' = dw/dsigma) and tmp: with the separable
// weights w(dy) w(dx), dS = V H' B + V' H B.  The model solves M a = D (b = mu_y - a^T mu), so
// for each parameter theta
//   da = M^-1 (dD - dM a),   db = dmu_y - da^T mu - a^T dmu,
// using the block's Cholesky factor of M.  For sigma, dmu, dW and dD follow from dS and the
// blurred count's tangent dn; eps (the ridge or the Appendix's additive term) and eps_mul (its
// multiplicative term) enter M only:
//   ridge:    M = W + eps I                          dM/deps = I
//   Appendix: M = W^ + eps diag(W^),  W^ = W + eps_mul (m m^T + diag m^2) + eps I  (m: absolute
//             guide means)   dM/deps = I + diag(W^) + eps I,
//             dM/deps_mul = (m m^T + diag m^2) + 2 eps diag(m^2),
//             and for sigma dW^ = dW + eps_mul (dm m^T + m dm^T + 2 diag(m dm)), dM = dW^ + eps diag(dW^).
// Writes the three tangents of the block model in the coef layout, the bias re-expressed
// relative to the frame reference (db - da^T (ref - frame reference)).  Blocks whose Cholesky
// pivot fell low get tangents from the FP32 factor (no FP64 re-solve).  S, dS: this thread's
// columns of two [NCH][stride] buffers.
template <int Q>
__device__ __forceinline__ void stage_blur_v_tangent(const FastArgs &a, size_t k, float *S, float *dS, int stride)
{
    using C = Chan<Q>;
    constexpr int NS = Q + 3;
    const size_t bplane = (size_t)a.Hb * a.Wb;
    if (k >= bplane) return;
    const int by = (int)(k / a.Wb), bx = (int)(k % a.Wb);
    float rk[NS];
#pragma unroll
    for (int q = 0; q < NS; ++q) rk[q] = a.blk[(C::NCH + q) * bplane + k];
    float n = 0.f, dn = 0.f;
    for (int pass = 0; pass < 2; ++pass) {
        float acc[C::NCH];
#pragma unroll
        for (int c = 0; c < C::NCH; ++c) acc[c] = 0.f;
        for (int dd = -a.taps; dd <= a.taps; ++dd) {
            const int yy = by + dd;
            if (yy < 0 || yy >= a.Hb) continue;
            const size_t kb = (size_t)yy * a.Wb + bx;
            float d[NS];
#pragma unroll
            for (int q = 0; q < NS; ++q) d[q] = a.blk[(C::NCH + q) * bplane + kb] - rk[q];
            const float nb = a.tmp[C::NCH * bplane + kb];
            const float w = a.w[dd + a.taps];
            if (pass == 0) {
                accumulate_shifted<Q>(acc, a.tmp + kb, bplane, d, nb, w);
                n = fmaf(w, nb, n);
            } else {
                const float nb2 = a.tmp2[C::NCH * bplane + kb], wd = a.wd[dd + a.taps];
                accumulate_shifted<Q>(acc, a.tmp2 + kb, bplane, d, nb2, w);
                accumulate_shifted<Q>(acc, a.tmp + kb, bplane, d, nb, wd);
                dn = fmaf(w, nb2, fmaf(wd, nb, dn));
            }
        }
        float *dst = pass == 0 ? S : dS;
#pragma unroll
        for (int c = 0; c < C::NCH; ++c) dst[c * stride] = acc[c];
    }
    float A[Q][3], bv[3], mu[Q], muy[3], L[Q * (Q + 1) / 2], inv_d[Q];
    if (a.appendix)
        solve_appendix<Q>(S, stride, n, a.eps, a.eps_mul, a.tau, rk, A, bv, mu, muy, L, inv_d);
    else
        dev::solve_pixel<Q>(S, stride, n, a.eps, a.tau, A, bv, mu, muy, L, inv_d);
    const float inv_n = 1.0f / n;
    const bool one_px = !(n > 1.5f);  // one-pixel block: a = 0, b = mu_y (see solve_pixel)
    // the Appendix's absolute means and diag(W^)
    float m[Q], whd[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        m[i] = rk[i] + mu[i];
        whd[i] = fmaf(-mu[i], mu[i], S[C::xx(i, i) * stride] * inv_n) + 2.f * a.eps_mul * m[i] * m[i] + a.eps;
    }
    float dmu[Q], dmuy[3];
#pragma unroll
    for (int i = 0; i < Q; ++i) dmu[i] = one_px ? 0.f : (dS[(C::X0 + i) * stride] - mu[i] * dn) * inv_n;
#pragma unroll
    for (int c = 0; c < 3; ++c) dmuy[c] = (dS[(C::Y0 + c) * stride] - muy[c] * dn) * inv_n;
    for (int t = 0; t < 3; ++t) {
        // dM (packed lower triangle) and dD of parameter t: 0 sigma, 1 eps, 2 eps_mul
        float dM[Q * (Q + 1) / 2], R[Q][3], da[Q][3];
#pragma unroll
        for (int i = 0; i < Q; ++i)
#pragma unroll
            for (int j = 0; j < Q; ++j) {
                if (j > i) continue;
                float v = 0.f;
                if (t == 0 && !one_px) {
                    const float sxx = S[C::xx(j, i) * stride] * inv_n;
                    v = (dS[C::xx(j, i) * stride] - sxx * dn) * inv_n - dmu[i] * mu[j] - mu[i] * dmu[j];
                    if (a.appendix) v = fmaf(a.eps_mul, dmu[i] * m[j] + m[i] * dmu[j] + (i == j ? 2.f * m[i] * dmu[i] : 0.f), v);
                } else if (t == 1) {
                    v = i == j ? 1.f : 0.f;
                } else if (t == 2 && a.appendix) {
                    v = m[i] * m[j] + (i == j ? m[i] * m[i] : 0.f);
                }
                dM[dev::tri(i, j)] = v;
            }
        if (a.appendix) {  // M = W^ + eps diag(W^): add eps dW^_ii (and W^_ii for eps itself)
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const int ii = dev::tri(i, i);
                dM[ii] = fmaf(a.eps, dM[ii], dM[ii]) + (t == 1 ? whd[i] : 0.f);
            }
        }
#pragma unroll
        for (int i = 0; i < Q; ++i)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float r = 0.f;
                if (t == 0 && !one_px) {
                    const float sxy = S[C::xy(i, c) * stride] * inv_n;
                    r = (dS[C::xy(i, c) * stride] - sxy * dn) * inv_n - dmu[i] * muy[c] - mu[i] * dmuy[c];
                }
#pragma unroll
                for (int j = 0; j < Q; ++j) r = fmaf(-dM[j <= i ? dev::tri(i, j) : dev::tri(j, i)], A[j][c], r);
                R[i][c] = r;
            }
        dev::chol_solve3<Q>(L, inv_d, R, da);
        float *dc = a.dcoef + (size_t)t * 3 * (Q + 1) * bplane;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float db = t == 0 ? dmuy[c] : 0.f;
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                if (one_px) da[i][c] = 0.f;
                db = fmaf(-da[i][c], mu[i], db);
                if (t == 0) db = fmaf(-A[i][c], dmu[i], db);
                db = fmaf(-da[i][c], rk[i] - a.shift[i], db);  // re-expressed relative to the frame reference
            }
            dc[c * bplane + k] = db;
#pragma unroll
            for (int i = 0; i < Q; ++i) dc[(3 * (i + 1) + c) * bplane + k] = da[i][c];
        }
    }
}

// 4. bilinear interpolation of the block models + apply.  Block centres are P = F s output
// pixels apart, so the P pixels of run r, [P r - P/2, P r + P/2), all interpolate between
// block columns r - 1 and r (clamped at the edges): one thread per (output row, run) loads
// the 4 x (Q+1) x 3 corner coefficients once, interpolates them vertically once, and
// streams the run (vector loads and stores when the run is aligned and inside the image).
template <int Q>
__device__ __forceinline__ void stage_apply(const FastArgs &a, size_t t)
{
    constexpr int NC = 3 * (Q + 1);
    const size_t oplane = (size_t)a.Ho * a.Wo;
    const size_t bplane = (size_t)a.Hb * a.Wb;
    const int P = a.F * a.s, den = 2 * P;
    const int nruns = a.Wo / P + 2;
    const size_t total = (size_t)a.Ho * nruns;
    if (t >= total) return;
    {
        const int yo = (int)(t / nruns), r = (int)(t % nruns);
        const int xs = P * r - P / 2;
        if (xs >= a.Wo) return;
        // rows: i0, i1, fy (exact rational coordinate (2 yo + 1 - P) / (2 P))
        int ny = min(max(2 * yo + 1 - P, 0), (a.Hb - 1) * den);
        const int i0 = min(ny / den, max(a.Hb - 2, 0)), i1 = min(i0 + 1, a.Hb - 1);
        const float fy = (float)(ny - i0 * den) / (float)den;
        const int jl = min(max(r - 1, 0), a.Wb - 1), jr = min(max(r, 0), a.Wb - 1);
        // corner models: left values and right-minus-left differences of the two block rows
        // (interpolated horizontally, then vertically, per pixel: the same order and the same
        // roundings as the TMA apply kernel, so both paths agree bit for bit)
        float l0[NC], d0[NC], l1[NC], d1[NC];
        {
            const size_t bl0 = (size_t)i0 * a.Wb + jl, bl1 = (size_t)i1 * a.Wb + jl;
            const size_t br0 = (size_t)i0 * a.Wb + jr, br1 = (size_t)i1 * a.Wb + jr;
#pragma unroll
            for (int k = 0; k < NC; ++k) {
                const float *pl = a.coef + k * bplane;
                l0[k] = __ldg(pl + bl0);
                l1[k] = __ldg(pl + bl1);
                d0[k] = __ldg(pl + br0) - l0[k];
                d1[k] = __ldg(pl + br1) - l1[k];
            }
        }
        float sh[Q + 3];
#pragma unroll
        for (int k = 0; k < Q + 3; ++k) sh[k] = a.shift[k];
        const size_t row = (size_t)yo * a.Wo;
        const bool vec = (a.Wo & 3) == 0 && (P & 3) == 0 && xs >= 0 && xs + P <= a.Wo;
        for (int x0 = 0; x0 < P; x0 += 4) {
            float o[3][4];
            float z[Q][4];
            const int xb = xs + x0;
            if (vec) {
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    const float4 v = __ldg(reinterpret_cast<const float4 *>(a.map_guide + i * oplane + row + xb));
                    z[i][0] = v.x; z[i][1] = v.y; z[i][2] = v.z; z[i][3] = v.w;
                }
            } else {
#pragma unroll
                for (int i = 0; i < Q; ++i)
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int x = xb + u;
                        z[i][u] = (x >= 0 && x < a.Wo && x0 + u < P) ? __ldg(a.map_guide + i * oplane + row + x) : 0.f;
                    }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int x = xb + u;
                int nx = min(max(2 * x + 1 - P, 0), (a.Wb - 1) * den);
                const float fx = fminf(fmaxf((float)(nx - (r - 1) * den) / (float)den, 0.f), 1.f);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    float top = fmaf(fx, d0[c], l0[c]);
                    float acc = fmaf(fy, fmaf(fx, d1[c], l1[c]) - top, top);
#pragma unroll
                    for (int i = 0; i < Q; ++i) {
                        const int k = 3 * (i + 1) + c;
                        top = fmaf(fx, d0[k], l0[k]);
                        acc = fmaf(fmaf(fy, fmaf(fx, d1[k], l1[k]) - top, top), z[i][u] - sh[i], acc);
                    }
                    o[c][u] = acc + sh[Q + c];
                }
            }
            if (vec) {
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    *reinterpret_cast<float4 *>(a.out + c * oplane + row + xb) = make_float4(o[c][0], o[c][1], o[c][2], o[c][3]);
            } else {
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int x = xb + u;
                    if (x >= 0 && x < a.Wo && x0 + u < P)
#pragma unroll
                        for (int c = 0; c < 3; ++c) a.out[c * oplane + row + x] = o[c][u];
                }
            }
        }
    }
}

// Work-item counts of each stage for one frame (256 threads per item).
__host__ __device__ inline int moment_chunks(int Wi) { return (Wi + 511) / 512; }
inline size_t items_moments(const FastArgs &a) { return (size_t)a.Hb * moment_chunks(a.Wi); }
inline size_t items_blocks(const FastArgs &a) { return ((size_t)a.Hb * a.Wb + 255) / 256; }
inline size_t items_apply(const FastArgs &a) { return ((size_t)a.Ho * (a.Wo / (a.F * a.s) + 2) + 255) / 256; }

}  // namespace fast
}  // namespace flr
