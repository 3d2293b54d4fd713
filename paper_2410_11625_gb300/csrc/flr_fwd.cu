// flr_fwd.cu -- FLR forward kernel: windowed moments and per-pixel solve (sm_103a).
//
// What it computes (arXiv 2410.11625, Sec. 3.1-3.2 and the Appendix): for every pixel k
// the box sums over the clipped radius-r window of the linear moments and of the outer
// products x x^T, x y^T (Sec. 3.2: box-filtering the outer products gives X_k^T X_k and
// X_k^T Y_k exactly), then the centred ridge model of the Appendix with eps on the
// diagonal of W = S/n - mu_X^T mu_X, solved by Cholesky in registers:
//     M = W + eps I,  a = M^{-1} (X^T Y / n - mu_X^T mu_Y),  b = mu_Y - a^T mu_X.
// With rc == 0 the model is applied to the centre pixel at once; otherwise (a, b) goes to
// a coefficient plane set that the averaging kernel (flr_apply.cu) consumes.
//
// Layout of the work.  The path is bound by FP32 ALU issue, not by HBM: per pixel it
// does ~60 products, ~280 window-sum adds and a ~300-FMA solve against 56 bytes of HBM
// traffic.  One CTA owns a strip of kTW output columns and a segment of TH rows and walks
// down it kB rows at a time:
//   1. V-pass: 3 x ceil(Wi/32) warps of "walkers", one per (input column, channel
//      group).  A walker keeps the vertical running sums of its channels in registers;
//      each step adds the products of the row entering the window and subtracts those of
//      the row leaving it, recomputed from the inputs (L1/L2-resident), so no ring of
//      moment rows is stored.  Each step's sums go to shared memory.
//   2. H-pass: one thread per (row, channel) slides a radius-r horizontal sum along the
//      shared-memory row, in place.
//   3. Solve: one thread per pixel of the batch reads its Q + 3 + Q(Q+1)/2 + 3Q window
//      sums and solves the Q x Q system in registers (left-looking Cholesky, 3 RHS).
// Precision: values are shifted by the mean of a 16 x 16 sample grid of the CTA's input
// region before any product, so moments are accumulated relative to a local reference
// (the centred form is invariant to the shift); the model is then re-expressed relative
// to a frame-wide reference (the mean of a 16 x 16 grid over the whole frame), which is
// what the averaging and apply steps use.  A pixel whose Cholesky pivot ratio
// d_j / M_jj falls to tau or below is appended to a flag list for the FP64 re-solve
// (flr_fp64.cu).
#include <utility>

#include "flr_internal.cuh"

namespace flr {
namespace {

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

// Running-sum update of one channel: + product of e, - product of l (slots fixed at
// compile time, so e, l and V stay in registers).
template <int Q, int CH, bool LEAVE>
__device__ __forceinline__ void walker_update_one(float &acc, const float (&e)[Q + 3],
                                                  const float (&l)[Q + 3])
{
    constexpr int u = Chan<Q>::slot_u(CH), v = Chan<Q>::slot_v(CH);
    if constexpr (v < 0) {
        acc += e[u];
        if constexpr (LEAVE) acc -= l[u];
    } else {
        acc = fmaf(e[u], e[v], acc);
        if constexpr (LEAVE) acc = fmaf(-l[u], l[v], acc);
    }
}

template <int Q, int G, bool LEAVE, int... I>
__device__ __forceinline__ void walker_update_seq(float (&V)[Chan<Q>::GMAX], const float (&e)[Q + 3],
                                                  const float (&l)[Q + 3],
                                                  std::integer_sequence<int, I...>)
{
    constexpr int c0 = Chan<Q>::group_begin(G);
    (walker_update_one<Q, c0 + I, LEAVE>(V[I], e, l), ...);
}

template <int Q, int G, bool LEAVE>
__device__ __forceinline__ void walker_update(float (&V)[Chan<Q>::GMAX], const float (&e)[Q + 3],
                                              const float (&l)[Q + 3])
{
    walker_update_seq<Q, G, LEAVE>(V, e, l,
                                   std::make_integer_sequence<int, Chan<Q>::group_size(G)>{});
}

template <int Q, int G>
__device__ __forceinline__ void walker_store(const float (&V)[Chan<Q>::GMAX], float *row0, int VS)
{
    using C = Chan<Q>;
    constexpr int c0 = C::group_begin(G), c1 = C::group_end(G);
#pragma unroll
    for (int ch = c0; ch < c1; ++ch) row0[ch * VS] = V[ch - c0];
}

template <int Q>
__device__ __forceinline__ void walker_store_dispatch(int group, const float (&V)[Chan<Q>::GMAX],
                                                      float *row0, int VS)
{
    if (group == 0) walker_store<Q, 0>(V, row0, VS);
    else if (group == 1) walker_store<Q, 1>(V, row0, VS);
    else walker_store<Q, 2>(V, row0, VS);
}

__device__ __forceinline__ constexpr int tri(int i, int j) { return i * (i + 1) / 2 + j; }  // i >= j

// Centred ridge solve of one pixel from its window sums S(ch) = Sp[ch * VS].
// Returns the model (a, b) in the CTA-shifted coordinates and whether a pivot fell low.
template <int Q>
__device__ __forceinline__ bool solve_pixel(const float *Sp, int VS, float n, float eps,
                                            float tau, float (&A)[Q][3], float (&bv)[3],
                                            float (&mu)[Q])
{
    using C = Chan<Q>;
    const float inv_n = 1.0f / n;
    float muy[3];
#pragma unroll
    for (int i = 0; i < Q; ++i) mu[i] = Sp[(C::X0 + i) * VS] * inv_n;
#pragma unroll
    for (int c = 0; c < 3; ++c) muy[c] = Sp[(C::Y0 + c) * VS] * inv_n;
    // M = S/n - mu mu^T + eps I (lower triangle), D = XY/n - mu muy^T.  A one-pixel
    // window (n = 1) has centred moments exactly zero; they are set so rather than left to
    // the rounding of x x - x x, which 1/eps would amplify.
    const float live = n > 1.5f ? 1.f : 0.f;
    float L[Q * (Q + 1) / 2];
#pragma unroll
    for (int i = 0; i < Q; ++i)
#pragma unroll
        for (int j = 0; j < Q; ++j) {
            if (j <= i) {
                float m = live * fmaf(-mu[i], mu[j], Sp[C::xx(j, i) * VS] * inv_n);
                if (i == j) m += eps;
                L[tri(i, j)] = m;
            }
        }
    float D[Q][3];
#pragma unroll
    for (int i = 0; i < Q; ++i)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            D[i][c] = live * fmaf(-mu[i], muy[c], Sp[C::xy(i, c) * VS] * inv_n);

    // left-looking Cholesky M = L L^T, keeping 1 / L_jj.  Inner loops run to Q with a
    // predicate so that every loop unrolls completely and L stays in registers.
    bool low = false;
    float inv_d[Q];
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        const float mjj = L[tri(j, j)];
        float d = mjj;
#pragma unroll
        for (int k = 0; k < Q; ++k)
            if (k < j) d = fmaf(-L[tri(j, k)], L[tri(j, k)], d);
        low |= !(d > tau * mjj);
        d = fmaxf(d, 1e-30f);
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

// Asynchronous 4-byte global->shared copy; src_size 0 writes a zero (no global read).
__device__ __forceinline__ void cp_async4(float *dst, const float *src, bool valid)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src),
                 "r"(valid ? 4 : 0));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::); }

// Stage the input rows a batch of kB walker steps needs: for step b, row yv + b + r
// enters the window and row yv + b - r - 1 leaves it.  Layout [2][kB][Q+3][WS] (0 =
// entering, 1 = leaving); rows outside the image or not yet summed are zero-filled.
template <int Q>
__device__ __forceinline__ void stage_batch(float *stage, int WS, const FwdArgs &a, int yv,
                                            int first_row, int xg0, int Wi, int warp, int lane)
{
    constexpr int NS = Q + 3;
    const size_t plane = (size_t)a.H * a.W;
    for (int row = warp; row < 2 * kB * NS; row += kThreads / 32) {
        const int el = row / (kB * NS), rem = row % (kB * NS);
        const int b = rem / NS, k = rem % NS;
        const int y = el == 0 ? yv + b + a.r : yv + b - a.r - 1;
        const bool row_ok = y >= 0 && y < a.H && (el == 0 || y >= first_row);
        const float *base = k < Q ? a.guide + (size_t)k * plane : a.rad + (size_t)(k - Q) * plane;
        const float *src_row = base + (size_t)(row_ok ? y : 0) * a.W;
        float *dst = stage + (size_t)row * WS;
        for (int wx = lane; wx < Wi; wx += 32) {
            const int gx = xg0 + wx;
            const bool ok = row_ok && gx >= 0 && gx < a.W;
            cp_async4(dst + wx, ok ? src_row + gx : a.rad, ok);
        }
    }
    cp_async_commit();
}

template <int Q>
__global__ void __launch_bounds__(kThreads, 1) flr_fwd_kernel(const FwdArgs a)
{
    using C = Chan<Q>;
    constexpr int NS = Q + 3;
    extern __shared__ float smem[];
    __shared__ float s_cta[NS], s_ref[NS];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int H = a.H, W = a.W, r = a.r;
    const int x0 = blockIdx.x * kTW;
    const int y0 = blockIdx.y * a.TH;
    const int y1 = min(y0 + a.TH, H);
    const int Wi = kTW + 2 * r;
    const int Wi_pad = (Wi + 31) & ~31;
    const int VS = Wi + 1;  // odd row stride: conflict-free for every access pattern below
    const int nColWarps = Wi_pad >> 5;
    float *Vbuf = smem;                                // [kB][NCH][VS]  window sums
    float *stage = smem + (size_t)kB * C::NCH * VS;    // [2][kB][NS][Wi_pad] input rows

    const int first_row = y0 - r;  // first input row summed by this segment
    const int xg0 = x0 - r;        // global column of walker column 0
    int yv = y0 - 2 * r;           // first virtual row: the walkers start with an empty window
    stage_batch<Q>(stage, Wi_pad, a, yv, first_row, xg0, Wi, warp, lane);

    // reference shifts (overlaps the first copies)
    if (warp == 0) {
        sample_mean<Q>(s_ref, a.guide, a.rad, H, W, 0, H, 0, W, lane);
    } else if (warp == 1) {
        sample_mean<Q>(s_cta, a.guide, a.rad, H, W, max(0, y0 - r), min(H, y1 + r), max(0, x0 - r),
                       min(W, x0 + kTW + r), lane);
    }
    __syncthreads();
    if (blockIdx.x == 0 && blockIdx.y == 0 && tid < NS) a.shift_out[tid] = s_ref[tid];

    // walker identity: warp -> (channel group, 32-column block)
    const int group = warp / nColWarps;
    const int wx = (warp % nColWarps) * 32 + lane;
    const bool walker = group < 3 && wx < Wi;
    const bool col_in = walker && xg0 + wx >= 0 && xg0 + wx < W;
    float sh[NS];
#pragma unroll
    for (int k = 0; k < NS; ++k) sh[k] = s_cta[k];

    float V[C::GMAX];
#pragma unroll
    for (int k = 0; k < C::GMAX; ++k) V[k] = 0.f;

    const float tau = a.tau;
    const float eps = a.eps;
    for (; yv < y1; yv += kB) {
        // 1. V-pass over the staged rows
        cp_async_wait_all();
        __syncthreads();
        if (walker) {
#pragma unroll 1
            for (int b = 0; b < kB; ++b) {
                const int yc = yv + b;
                if (yc < y1) {
                    const bool ein_ok = yc + r >= 0 && yc + r < H;
                    const bool lout_ok = yc - r - 1 >= first_row && yc - r - 1 >= 0;
                    const float *se = stage + (size_t)(b * NS) * Wi_pad + wx;
                    const float *sl = stage + (size_t)((kB + b) * NS) * Wi_pad + wx;
                    float e[NS], l[NS];
#pragma unroll
                    for (int k = 0; k < NS; ++k) {
                        e[k] = (col_in && ein_ok) ? se[k * Wi_pad] - sh[k] : 0.f;
                        l[k] = (col_in && lout_ok) ? sl[k * Wi_pad] - sh[k] : 0.f;
                    }
                    if (group == 0) walker_update<Q, 0, true>(V, e, l);
                    else if (group == 1) walker_update<Q, 1, true>(V, e, l);
                    else walker_update<Q, 2, true>(V, e, l);
                }
                walker_store_dispatch<Q>(group, V, Vbuf + (size_t)b * C::NCH * VS + wx, VS);
            }
        }
        __syncthreads();
        // prefetch the next batch's rows while this one is summed and solved
        if (yv + kB < y1) stage_batch<Q>(stage, Wi_pad, a, yv + kB, first_row, xg0, Wi, warp, lane);
        if (yv + kB - 1 < y0) continue;  // warm-up batch: nothing to solve yet

        // 2. H-pass, one thread per (row, channel), in place: slot xo <- sum V[xo..xo+2r].
        //    Chunks of 8 outputs load all their operands before writing any slot.
        for (int row = tid; row < kB * C::NCH; row += kThreads) {
            float *p = Vbuf + (size_t)row * VS;
            float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
            int k = 0;
            for (; k + 4 <= 2 * r + 1; k += 4) {
                s0 += p[k];
                s1 += p[k + 1];
                s2 += p[k + 2];
                s3 += p[k + 3];
            }
            for (; k <= 2 * r; ++k) s0 += p[k];
            float s = (s0 + s1) + (s2 + s3);
            float vprev = 0.f;
#pragma unroll 1
            for (int xo = 0; xo < kTW; xo += 8) {
                float add[8], old[8];
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    add[t] = p[xo + t + 2 * r];
                    old[t] = p[xo + t];
                }
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    if (xo + t > 0) s += add[t] - vprev;
                    vprev = old[t];
                    p[xo + t] = s;
                }
            }
        }
        __syncthreads();
        // 3. solve, one thread per pixel of the batch
        {
            const int b = tid / kTW, xo = tid % kTW;
            const int yc = yv + b, xc = x0 + xo;
            if (yc >= y0 && yc < y1 && xc < W) {
                const float ny = (float)(min(yc + r, H - 1) - max(yc - r, 0) + 1);
                const float nx = (float)(min(xc + r, W - 1) - max(xc - r, 0) + 1);
                float A[Q][3], bv[3], mu[Q];
                const bool low = solve_pixel<Q>(Vbuf + (size_t)b * C::NCH * VS + xo, VS, ny * nx,
                                                eps, tau, A, bv, mu);
                // re-express the bias relative to the frame reference shift
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    float bb = bv[c] + (s_cta[Q + c] - s_ref[Q + c]);
#pragma unroll
                    for (int i = 0; i < Q; ++i) bb = fmaf(-A[i][c], s_cta[i] - s_ref[i], bb);
                    bv[c] = bb;
                }
                const size_t plane = (size_t)H * W;
                const size_t off = (size_t)yc * W + xc;
                if (a.rc == 0) {
                    const float *zg = a.map_guide ? a.map_guide : a.guide;
                    float z[Q];
#pragma unroll
                    for (int i = 0; i < Q; ++i) z[i] = __ldg(zg + i * plane + off) - s_ref[i];
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        float o = bv[c];
#pragma unroll
                        for (int i = 0; i < Q; ++i) o = fmaf(A[i][c], z[i], o);
                        a.out[c * plane + off] = o + s_ref[Q + c];
                    }
                } else {
#pragma unroll
                    for (int c = 0; c < 3; ++c) a.coef[c * plane + off] = bv[c];
#pragma unroll
                    for (int i = 0; i < Q; ++i)
#pragma unroll
                        for (int c = 0; c < 3; ++c) a.coef[(3 * (i + 1) + c) * plane + off] = A[i][c];
                }
                if (low && tau > 0.f) {
                    const unsigned long long slot = atomicAdd(a.flag_count, 1ull);
                    if (slot < (unsigned long long)a.flag_cap) a.flag_list[slot] = (int)off;
                }
            }
        }
        __syncthreads();
    }
    cp_async_wait_all();
}

template <int Q>
cudaError_t launch_fwd_q(const FwdArgs &a, dim3 grid, size_t smem, cudaStream_t st)
{
    flr_fwd_kernel<Q><<<grid, kThreads, smem, st>>>(a);
    return cudaGetLastError();
}

template <int Q>
cudaError_t prepare_q(size_t smem)
{
    return cudaFuncSetAttribute(flr_fwd_kernel<Q>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem);
}

template <int Q>
size_t smem_q(int r)
{
    const int Wi = kTW + 2 * r;
    const int Wi_pad = (Wi + 31) & ~31;
    return sizeof(float) * ((size_t)kB * Chan<Q>::NCH * (Wi + 1) + (size_t)2 * kB * (Q + 3) * Wi_pad);
}

}  // namespace

#define FLR_Q_DISPATCH(q, CALL)  \
    switch (q) {                 \
    case 1: { constexpr int QQ = 1; CALL; } \
    case 2: { constexpr int QQ = 2; CALL; } \
    case 3: { constexpr int QQ = 3; CALL; } \
    case 4: { constexpr int QQ = 4; CALL; } \
    case 5: { constexpr int QQ = 5; CALL; } \
    case 6: { constexpr int QQ = 6; CALL; } \
    case 7: { constexpr int QQ = 7; CALL; } \
    case 8: { constexpr int QQ = 8; CALL; } \
    default: break;              \
    }

cudaError_t launch_fwd(int q, const FwdArgs &a, dim3 grid, size_t smem, cudaStream_t st)
{
    FLR_Q_DISPATCH(q, return launch_fwd_q<QQ>(a, grid, smem, st));
    return cudaErrorInvalidValue;
}

size_t fwd_smem_bytes(int q, int r)
{
    FLR_Q_DISPATCH(q, return smem_q<QQ>(r));
    return 0;
}

cudaError_t fwd_prepare(int q, size_t smem)
{
    FLR_Q_DISPATCH(q, return prepare_q<QQ>(smem));
    return cudaErrorInvalidValue;
}

}  // namespace flr
