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
// Staging: when rows are 16-byte aligned, one thread copies each batch's entering and
// leaving input rows with four TMA box copies (guide and radiance planes, zero fill
// outside the image) completing on an mbarrier; otherwise all threads issue asynchronous
// copies.
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
#include <cstring>
#include <mutex>
#include <utility>

#include "flr_device.cuh"
#include "flr_internal.cuh"
#include "flr_tmem.cuh"
#include "tma.cuh"

namespace flr {
namespace {

using dev::sample_mean;
using dev::solve_pixel;
using dev::chol_solve3;
using dev::tri;

// Block accumulators of one channel: acc += the product of the row's shifted values r
// (slots fixed at compile time, so r and the accumulators stay in registers).
template <int Q, int CH>
__device__ __forceinline__ void walker_add_one(float &acc, const float (&r)[Q + 3])
{
    constexpr int u = Chan<Q>::slot_u(CH), v = Chan<Q>::slot_v(CH);
    if constexpr (v < 0) acc += r[u];
    else acc = fmaf(r[u], r[v], acc);
}

template <int Q, int G, int... I>
__device__ __forceinline__ void walker_add_seq(float (&A)[Chan<Q>::GMAX], const float (&r)[Q + 3],
                                               std::integer_sequence<int, I...>)
{
    constexpr int c0 = Chan<Q>::group_begin(G);
    (walker_add_one<Q, c0 + I>(A[I], r), ...);
}

// E += products of the entering row e, Dn += products of the leaving row l (group G)
template <int Q, int G>
__device__ __forceinline__ void walker_update(float (&E)[Chan<Q>::GMAX], float (&Dn)[Chan<Q>::GMAX],
                                              const float (&e)[Q + 3], const float (&l)[Q + 3])
{
    walker_add_seq<Q, G>(E, e, std::make_integer_sequence<int, Chan<Q>::group_size(G)>{});
    walker_add_seq<Q, G>(Dn, l, std::make_integer_sequence<int, Chan<Q>::group_size(G)>{});
}

// the window sums V = E - Dn of group G to the channel rows of the buffer
template <int Q, int G>
__device__ __forceinline__ void walker_store(const float (&E)[Chan<Q>::GMAX], const float (&Dn)[Chan<Q>::GMAX],
                                             float *row0, int VS)
{
    using C = Chan<Q>;
    constexpr int c0 = C::group_begin(G), c1 = C::group_end(G);
#pragma unroll
    for (int ch = c0; ch < c1; ++ch) row0[ch * VS] = E[ch - c0] - Dn[ch - c0];
}

// Tensor-memory columns of the walker accumulators: warp w keeps E and Dn (2 GMAX columns of
// its lane quarter) at slot w / 4, each slot starting at a multiple of its power-of-two width.
template <int Q>
struct WalkerTmem {
    static constexpr int N = 2 * Chan<Q>::GMAX;
    static constexpr int SLOT = N <= 8 ? 8 : (N <= 16 ? 16 : (N <= 32 ? 32 : 64));
    static constexpr int NSLOT = kThreads / 32 / 4;
    static constexpr int USED = SLOT * NSLOT;
    static constexpr uint32_t COLS = USED <= 32 ? 32u : (USED <= 64 ? 64u : (USED <= 128 ? 128u : 256u));
    static_assert(N <= 64 && USED <= 256, "walker accumulators fit the allocation");
};

// Adjoint of one pixel's model (the reverse of bias, solve, regulariser, centring and
// means), given G(b), G(a) relative to the frame reference shift.  Writes the per-pixel
// gradients of the window sums, in moment-channel order, re-expressed so that the
// contraction with (x - s_ref, y - s_ref) gives the input gradients; returns d/d eps.
template <int Q>
__device__ __forceinline__ float adjoint_pixel(const float (&A)[Q][3], const float (&mu)[Q],
                                               const float (&muy)[3], const float (&L)[Q * (Q + 1) / 2],
                                               const float (&inv_d)[Q], float n, const float *gA,
                                               float *gS, size_t plane, size_t off, const float *s_cta,
                                               const float *s_ref)
{
    using C = Chan<Q>;
    float Gb[3], Gap[Q][3], Gmu[Q], Gnu[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) Gb[c] = __ldg(gA + c * plane + off);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const float dl = s_cta[i] - s_ref[i];
        Gmu[i] = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            // b_ref = b + (s_cta_y - s_ref_y) - a^T (s_cta - s_ref), then b = muy - a^T mu
            const float ga = __ldg(gA + (3 * (i + 1) + c) * plane + off) - dl * Gb[c];
            Gap[i][c] = fmaf(-mu[i], Gb[c], ga);
            Gmu[i] = fmaf(-A[i][c], Gb[c], Gmu[i]);
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) Gnu[c] = Gb[c];
    float GD[Q][3];
    chol_solve3<Q>(L, inv_d, Gap, GD);
    const float inv_n = 1.0f / n;
    const float live = n > 1.5f ? inv_n : 0.f;  // one-pixel window: the model path is constant
    float geps = 0.f;
    float Gxx[Q * (Q + 1) / 2];
#pragma unroll
    for (int i = 0; i < Q; ++i)
#pragma unroll
        for (int j = 0; j < Q; ++j) {
            if (j <= i) {
                float t = 0.f;
#pragma unroll
                for (int c = 0; c < 3; ++c) t = fmaf(GD[i][c], A[j][c], fmaf(A[i][c], GD[j][c], t));
                const float gm = -0.5f * t;
                if (i == j) geps += gm;
                Gxx[tri(i, j)] = gm;
                Gmu[i] = fmaf(-2.f * gm, mu[j], Gmu[i]);
                if (j != i) Gmu[j] = fmaf(-2.f * gm, mu[i], Gmu[j]);
            }
        }
#pragma unroll
    for (int i = 0; i < Q; ++i)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            Gmu[i] = fmaf(-GD[i][c], muy[c], Gmu[i]);
            Gnu[c] = fmaf(-GD[i][c], mu[i], Gnu[c]);
        }
    // scale by 1/n and move the linear terms from the CTA shift to the frame shift
    float dl[Q], dly[3];
#pragma unroll
    for (int i = 0; i < Q; ++i) dl[i] = s_cta[i] - s_ref[i];
#pragma unroll
    for (int c = 0; c < 3; ++c) dly[c] = s_cta[Q + c] - s_ref[Q + c];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        float gx = Gmu[i];
#pragma unroll
        for (int j = 0; j < Q; ++j) gx = fmaf(-2.f * Gxx[i >= j ? tri(i, j) : tri(j, i)], dl[j], gx);
#pragma unroll
        for (int c = 0; c < 3; ++c) gx = fmaf(-GD[i][c], dly[c], gx);
        gS[(C::X0 + i) * plane + off] = gx * live;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float gy = Gnu[c];
#pragma unroll
        for (int i = 0; i < Q; ++i) gy = fmaf(-GD[i][c], dl[i], gy);
        // with n = 1 only the mean of y survives: G(nu) = G(b) exactly
        gS[(C::Y0 + c) * plane + off] = (n > 1.5f ? gy : Gb[c]) * inv_n;
    }
#pragma unroll
    for (int i = 0; i < Q; ++i)
#pragma unroll
        for (int j = 0; j < Q; ++j)
            if (j >= i) gS[C::xx(i, j) * plane + off] = Gxx[tri(j, i)] * live;
#pragma unroll
    for (int i = 0; i < Q; ++i)
#pragma unroll
        for (int c = 0; c < 3; ++c) gS[C::xy(i, c) * plane + off] = GD[i][c] * live;
    return geps;
}

// Asynchronous global->shared copies; a src_size of 0 writes zeros without reading.
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
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::); }

// Shared-memory geometry of one CTA for radius r.
struct FwdGeom {
    int Wi;   // walker (input) columns: kTW + 2r
    int RA;   // r rounded up to a multiple of 4: staged rows start at column x0 - RA
    int WSt;  // staged row length: kTW + 2 RA (a multiple of 4)
    int VS;   // row stride of the window-sum buffer
    __host__ __device__ FwdGeom(int r, bool vec_hpass)
    {
        Wi = kTW + 2 * r;
        RA = (r + 3) & ~3;
        WSt = kTW + 2 * RA;
        // vectorised H-pass: 16-byte aligned rows with stride = 4 (mod 8) floats, so the
        // eight lanes of each 128-bit access phase hit distinct banks; scalar H-pass: an
        // odd stride, so 32 lanes on 32 rows hit distinct banks
        VS = vec_hpass ? (((Wi + 3) & ~7) + 4) : (Wi | 1);
    }
};

constexpr unsigned long long kFwdTimeoutNs = 1000000000ull;  // 1 s per wait

// Kernel parameters: TMA maps of the guide [Q][H][W] and radiance [3][H][W] planes (boxes
// of WSt columns x kB rows x all planes; valid when use_tma) and the forward arguments.
struct alignas(128) FwdKArgs {
    CUtensorMap tg, tr;
    FwdArgs a;
    int use_tma;
};

// Stage the input rows of kB walker steps: for step b, row yv + b + r enters the window
// and row yv + b - r - 1 leaves it.  Layout [2][Q+3][kB][WSt] (0 = entering, 1 = leaving;
// then input plane, step); staged column j is global column x0 - RA + j; anything outside
// the image is zero.
template <int Q>
__device__ __forceinline__ void stage_batch(float *stage, const FwdGeom &gm, const FwdKArgs &k, uint64_t *bar,
                                            int r, int yv, int x0, int warp, int lane)
{
    constexpr int NS = Q + 3;
    const FwdArgs &a = k.a;
    const int xs0 = x0 - gm.RA;
    if (k.use_tma) {
        if (threadIdx.x == 0) {
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // earlier reads before the copies
            tma::mbar_expect_tx(bar, (unsigned)(2 * NS * kB * gm.WSt * 4));
            const size_t box = (size_t)kB * gm.WSt;
            tma::load_3d(stage, &k.tg, xs0, yv + r, 0, bar);
            tma::load_3d(stage + Q * box, &k.tr, xs0, yv + r, 0, bar);
            tma::load_3d(stage + NS * box, &k.tg, xs0, yv - r - 1, 0, bar);
            tma::load_3d(stage + (NS + Q) * box, &k.tr, xs0, yv - r - 1, 0, bar);
        }
        return;
    }
    const size_t plane = (size_t)a.H * a.W;
    const bool vec = (a.W & 3) == 0;  // 16-byte rows: every 4-column chunk is all in or all out
    for (int row = warp; row < 2 * kB * NS; row += kThreads / 32) {
        const int el = row / (kB * NS), rem = row - el * (kB * NS);
        const int kk = rem / kB, b = rem - kk * kB;
        const int y = el == 0 ? yv + b + r : yv + b - r - 1;
        const bool row_ok = y >= 0 && y < a.H;
        const float *base = kk < Q ? a.guide + (size_t)kk * plane : a.rad + (size_t)(kk - Q) * plane;
        const float *src_row = base + (size_t)(row_ok ? y : 0) * a.W;
        float *dst = stage + (size_t)row * gm.WSt;
        if (vec) {
            for (int c = lane; c < (gm.WSt >> 2); c += 32) {
                const int gx = xs0 + 4 * c;
                const bool ok = row_ok && gx >= 0 && gx < a.W;
                cp_async16(dst + 4 * c, ok ? src_row + gx : a.rad, ok);
            }
        } else {
            for (int j = lane; j < gm.WSt; j += 32) {
                const int gx = xs0 + j;
                const bool ok = row_ok && gx >= 0 && gx < a.W;
                cp_async4(dst + j, ok ? src_row + gx : a.rad, ok);
            }
        }
    }
    cp_async_commit();
}

// Wait for the rows staged by the n-th stage_batch call (bounded for the TMA path).
__device__ __forceinline__ void stage_wait(const FwdKArgs &k, uint64_t *bar, int n, int *abort_flag)
{
    if (k.use_tma) {
        if (!tma::wait_warp(bar, (uint32_t)(n & 1), kFwdTimeoutNs) && (threadIdx.x & 31) == 0) {
            *abort_flag = 1;
            if (k.a.status) atomicExch(k.a.status, 1);
        }
    } else {
        cp_async_wait_all();
    }
}

// Horizontal radius-r sums of one shared-memory row, in place, for a radius known only at
// run time: slot xo <- sum of p[xo .. xo + 2r] for xo in [0, kTW).  Chunks of 8 outputs load
// every operand before writing, so no slot is overwritten while still needed.  (Radii known
// at compile time use dev::hsum_run: two runs, each seeded by a direct sum.)
__device__ __forceinline__ void hsum_row(float *p, int r)
{
    float s;
    {
        float t0 = 0.f, t1 = 0.f, t2 = 0.f, t3 = 0.f;
        int k = 0;
        for (; k + 4 <= 2 * r + 1; k += 4) {
            t0 += p[k];
            t1 += p[k + 1];
            t2 += p[k + 2];
            t3 += p[k + 3];
        }
        for (; k <= 2 * r; ++k) t0 += p[k];
        s = (t0 + t1) + (t2 + t3);
    }
    float vprev = 0.f;
#pragma unroll 2
    for (int xo = 0; xo < kTW; xo += 8) {
        float add[8], old[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            add[t] = p[xo + t + 2 * r];
            old[t] = p[xo + t];
        }
        float out[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            if (xo + t > 0) s += add[t] - vprev;
            vprev = old[t];
            out[t] = s;
        }
#pragma unroll
        for (int t = 0; t < 8; ++t) p[xo + t] = out[t];
    }
}

template <int Q, int RT, bool ADJ>
__global__ void __launch_bounds__(kThreads, 1) flr_fwd_kernel(const __grid_constant__ FwdKArgs ka)
{
    using C = Chan<Q>;
    constexpr int NS = Q + 3;
    extern __shared__ __align__(16) float smem[];
    __shared__ float s_cta[NS], s_ref[NS];
    __shared__ int s_abort;
    __shared__ uint32_t s_tmem;
    using WT = WalkerTmem<Q>;
    constexpr int GM = C::GMAX;
    const FwdArgs &a = ka.a;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int H = a.H, W = a.W;
    const int r = RT >= 0 ? RT : a.r;
    const FwdGeom gm(r, RT >= 0);
    const int x0 = blockIdx.x * kTW;
    const int row_hi = a.row_hi < 0 ? H : min(a.row_hi, H);
    const int y0 = a.row_lo + blockIdx.y * a.TH;
    const int y1 = min(y0 + a.TH, row_hi);
    const int ref_rows = a.ref_rows > 0 ? min(a.ref_rows, H) : H;
    const int nColWarps = (gm.Wi + 31) >> 5;
    float *base = smem + (((128 - (tma::smem_addr(smem) & 127)) & 127) >> 2);  // 128-byte aligned
    float *Vbuf = base;                                              // [kB][NCH][VS]  window sums
    float *stage = base + ((size_t)kB * C::NCH * gm.VS + 31) / 32 * 32;  // [2][NS][kB][WSt] input rows
    uint64_t *bar = reinterpret_cast<uint64_t *>(stage + (size_t)2 * NS * kB * gm.WSt);
    if (warp == 0) {  // tensor memory for the walkers' accumulators between batches
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(tma::smem_addr(&s_tmem)),
                     "r"(WT::COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid == 0) {
        s_abort = 0;
        if (ka.use_tma) {
            tma::mbar_init(bar, 1);
            tma::mbar_init_fence();
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    // this warp's lane quarter and slot
    const uint32_t tmem = s_tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(WT::SLOT * (warp >> 2));

    const int first_row = y0 - r;  // first input row summed by this segment
    int yv = y0 - 2 * r;           // first virtual row: the walkers start from an empty window
    int nstaged = 0;               // stage_batch calls so far (mbarrier phase)
    stage_batch<Q>(stage, gm, ka, bar, r, yv, x0, warp, lane);
    ++nstaged;

    // reference shifts (overlaps the first copies)
    if (warp == 0) {
        sample_mean<Q>(s_ref, a.guide, a.rad, H, W, 0, ref_rows, 0, W, lane);
    } else if (warp == 1) {
        sample_mean<Q>(s_cta, a.guide, a.rad, H, W, max(0, y0 - r), min(H, y1 + r), max(0, x0 - r),
                       min(W, x0 + kTW + r), lane);
    }
    __syncthreads();
    if (blockIdx.x == 0 && blockIdx.y == 0 && tid < NS) a.shift_out[tid] = s_ref[tid];

    // walker identity: warp -> (channel group, 32-column block); walker column wx is
    // global column x0 - r + wx and staged column wx + (RA - r)
    const int group = warp / nColWarps;
    const int wx = (warp % nColWarps) * 32 + lane;
    const bool walker = group < 3 && wx < gm.Wi;
    const int gxw = x0 - r + wx;
    // outside the image the staged values are zero, so a zero shift keeps them zero
    const bool col_in = gxw >= 0 && gxw < W;
    float shl[NS];
#pragma unroll
    for (int k = 0; k < NS; ++k) shl[k] = col_in ? s_cta[k] : 0.f;
    const int scol = wx + (gm.RA - r);

    // Vertical window sums as block accumulators: E, the products of the rows entered since
    // the last block start, and Dn, the products of the rows left since then minus the
    // previous block's total.  A block is 2r + 1 entered rows, so V = E - Dn is a sum of at
    // most 2(2r + 1) rounded terms and its error does not grow along the segment (a running
    // sum that adds the entering row and subtracts the leaving one drifts).  Between batches
    // E and Dn wait in tensor memory, so they hold no registers during the solve.
    const int v0 = y0 - 2 * r, WR = 2 * r + 1;

    const float tau = a.tau;
    const float eps = a.eps;
    float geps_acc = 0.f;  // adjoint mode: this thread's share of d L / d eps
    for (; yv < y1; yv += kB) {
        // 1. V-pass over the staged rows
        stage_wait(ka, bar, nstaged - 1, &s_abort);
        __syncthreads();
        if (s_abort) break;  // a copy never completed: issue nothing more on this barrier
        {
            float E[GM], Dn[GM];
            if (yv == v0) {
#pragma unroll
                for (int k = 0; k < GM; ++k) E[k] = Dn[k] = 0.f;
            } else {
                uint32_t st[2 * GM];
                tm_ld_n<2 * GM>(tmem, st);
                tm_wait_ld();
#pragma unroll
                for (int k = 0; k < GM; ++k) {
                    E[k] = __uint_as_float(st[k]);
                    Dn[k] = __uint_as_float(st[GM + k]);
                }
            }
            if (walker) {
#pragma unroll 1
                for (int b = 0; b < kB; ++b) {
                    const int yc = yv + b;
                    if (yc < y1) {
                        if ((yc - v0) % WR == 0) {  // block start: Dn = -(previous block total), E = 0
#pragma unroll
                            for (int k = 0; k < GM; ++k) {
                                Dn[k] = -E[k];
                                E[k] = 0.f;
                            }
                        }
                        const bool ein_ok = yc + r >= 0 && yc + r < H;
                        const bool lout_ok = yc - r - 1 >= first_row && yc - r - 1 >= 0;
                        const float *se = stage + (size_t)b * gm.WSt + scol;
                        const float *sl = stage + (size_t)(NS * kB + b) * gm.WSt + scol;
                        float e[NS], l[NS];
#pragma unroll
                        for (int k = 0; k < NS; ++k) {
                            e[k] = 0.f;
                            l[k] = 0.f;
                        }
                        if (ein_ok) {
#pragma unroll
                            for (int k = 0; k < NS; ++k) e[k] = se[(size_t)k * kB * gm.WSt] - shl[k];
                        }
                        if (lout_ok) {
#pragma unroll
                            for (int k = 0; k < NS; ++k) l[k] = sl[(size_t)k * kB * gm.WSt] - shl[k];
                        }
                        if (group == 0) walker_update<Q, 0>(E, Dn, e, l);
                        else if (group == 1) walker_update<Q, 1>(E, Dn, e, l);
                        else walker_update<Q, 2>(E, Dn, e, l);
                    }
                    float *row0 = Vbuf + (size_t)b * C::NCH * gm.VS + wx;
                    if (group == 0) walker_store<Q, 0>(E, Dn, row0, gm.VS);
                    else if (group == 1) walker_store<Q, 1>(E, Dn, row0, gm.VS);
                    else walker_store<Q, 2>(E, Dn, row0, gm.VS);
                }
            }
            __syncwarp();  // the walkers' branches rejoin before the warp-wide tensor-memory store
            uint32_t st[2 * GM];
#pragma unroll
            for (int k = 0; k < GM; ++k) {
                st[k] = __float_as_uint(E[k]);
                st[GM + k] = __float_as_uint(Dn[k]);
            }
            tm_st_n<2 * GM>(tmem, st);
            tm_wait_st();
        }
        __syncthreads();
        // prefetch the next batch's rows while this one is summed and solved
        if (yv + kB < y1) {
            stage_batch<Q>(stage, gm, ka, bar, r, yv + kB, x0, warp, lane);
            ++nstaged;
        }
        if (yv + kB - 1 < y0) continue;  // warm-up batch: nothing to solve yet

        // 2. H-pass, one thread per (row, channel); with the radius known at compile time two
        //    runs of kTW / 2 outputs, each seeded by a direct (2r + 1)-term sum
        for (int row = tid; row < kB * C::NCH; row += kThreads) {
            float *p = Vbuf + (size_t)row * gm.VS;
            if constexpr (RT >= 0) {
                dev::hsum_run<RT, kTW / 2>(p, p, 0);
                dev::hsum_run<RT, kTW / 2>(p, p, kTW / 2);
            } else {
                hsum_row(p, r);
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
                float A[Q][3], bv[3], mu[Q], muy[3], L[Q * (Q + 1) / 2], inv_d[Q];
                const bool low = solve_pixel<Q>(Vbuf + (size_t)b * C::NCH * gm.VS + xo, gm.VS, ny * nx,
                                                eps, tau, A, bv, mu, muy, L, inv_d);
                const size_t plane = (size_t)H * W;
                const size_t off = (size_t)yc * W + xc;
                if constexpr (ADJ) {
                    geps_acc += adjoint_pixel<Q>(A, mu, muy, L, inv_d, ny * nx, a.gA, a.gS, plane, off,
                                                 s_cta, s_ref);
                    if (a.coef) {  // the model itself (for the backward's averaged models)
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            float bb = bv[c] + (s_cta[Q + c] - s_ref[Q + c]);
#pragma unroll
                            for (int i = 0; i < Q; ++i) bb = fmaf(-A[i][c], s_cta[i] - s_ref[i], bb);
                            a.coef[c * plane + off] = bb;
                        }
#pragma unroll
                        for (int i = 0; i < Q; ++i)
#pragma unroll
                            for (int c = 0; c < 3; ++c) a.coef[(3 * (i + 1) + c) * plane + off] = A[i][c];
                    }
                } else {
                    // re-express the bias relative to the frame reference shift
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        float bb = bv[c] + (s_cta[Q + c] - s_ref[Q + c]);
#pragma unroll
                        for (int i = 0; i < Q; ++i) bb = fmaf(-A[i][c], s_cta[i] - s_ref[i], bb);
                        bv[c] = bb;
                    }
                    if (a.rc == 0 && !a.force_coef) {
                        const float *zg = a.map_guide ? a.map_guide : a.guide;
                        float z[Q];
#pragma unroll
                        for (int i = 0; i < Q; ++i) z[i] = __ldg(zg + i * plane + off) - s_ref[i];
                        int bad = 0;
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            float o = bv[c];
#pragma unroll
                            for (int i = 0; i < Q; ++i) o = fmaf(A[i][c], z[i], o);
                            o += s_ref[Q + c];
                            a.out[c * plane + off] = o;
                            bad += !isfinite(o);
                        }
                        // a flagged pixel's value is replaced by the FP64 re-solve, which counts it
                        if (bad && a.nonfinite && !(low && tau > 0.f)) atomicAdd(a.nonfinite, (unsigned long long)bad);
                    } else {
#pragma unroll
                        for (int c = 0; c < 3; ++c) a.coef[c * plane + off] = bv[c];
#pragma unroll
                        for (int i = 0; i < Q; ++i)
#pragma unroll
                            for (int c = 0; c < 3; ++c) a.coef[(3 * (i + 1) + c) * plane + off] = A[i][c];
                    }
                }
                if ((!ADJ || a.coef) && low && tau > 0.f) {
                    const unsigned long long slot = atomicAdd(a.flag_count, 1ull);
                    if (slot < (unsigned long long)a.flag_cap) a.flag_list[slot] = (int)off;
                }
            }
        }
        __syncthreads();
    }
    if (!ka.use_tma) cp_async_wait_all();
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(s_tmem), "r"(WT::COLS));
    }
    if constexpr (ADJ) {
        double g = (double)geps_acc;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) g += __shfl_xor_sync(0xffffffffu, g, o);
        if (lane == 0 && g != 0.0) atomicAdd(a.geps, g);
    }
}

// The frame reference shift alone (the forward kernel's s_ref: the same sample of rows
// [0, ref_rows)), for a pass that needs it before any forward-kernel launch.
template <int Q>
__global__ void frame_shift_kernel(const float *guide, const float *rad, int H, int W, int ref_rows, float *shift_out)
{
    __shared__ float s[Q + 3];
    sample_mean<Q>(s, guide, rad, H, W, 0, ref_rows > 0 ? min(ref_rows, H) : H, 0, W, threadIdx.x & 31);
    __syncwarp();
    if (threadIdx.x < Q + 3) shift_out[threadIdx.x] = s[threadIdx.x];
}

// Radii with a compile-time specialisation (the radii of the 256x256 and 1080p workloads);
// every other radius runs the generic kernel.
__host__ __device__ constexpr bool specialised(int q, int r) { return q == 8 && (r == 5 || r == 8); }

template <int Q, int RT, bool ADJ>
cudaError_t launch_fwd_qr(const FwdArgs &a, dim3 grid, size_t smem, cudaStream_t st)
{
    FwdKArgs ka;
    std::memset(&ka, 0, sizeof(ka));
    ka.a = a;
    const FwdGeom gm(a.r, RT >= 0);
    const bool aligned = (a.W & 3) == 0 && ((uintptr_t)a.guide & 15) == 0 && ((uintptr_t)a.rad & 15) == 0;
    // boxes of all guide planes and all radiance planes: together the 2 * (Q + 3) * kB * WSt
    // * 4 bytes per batch that stage_batch announces
    ka.use_tma = aligned && tma::encode_planes_f32(&ka.tg, a.guide, a.W, a.H, Q, gm.WSt, kB, Q) == cudaSuccess &&
                         tma::encode_planes_f32(&ka.tr, a.rad, a.W, a.H, 3, gm.WSt, kB, 3) == cudaSuccess
                     ? 1
                     : 0;
    flr_fwd_kernel<Q, RT, ADJ><<<grid, kThreads, smem, st>>>(ka);
    return cudaGetLastError();
}

// The dynamic shared memory a kernel instance may use is a per-device attribute shared by
// every handle (the generic instance serves every radius): it is only ever raised, to the
// largest size requested so far on that device, so a later request for less never takes
// memory from an instance already configured for more.
template <int Q, int RT, bool ADJ>
cudaError_t prepare_qr(size_t smem)
{
    static std::mutex mu;
    static size_t granted[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (smem <= granted[dev]) return cudaSuccess;
    e = cudaFuncSetAttribute(flr_fwd_kernel<Q, RT, ADJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) granted[dev] = smem;
    return e;
}

template <int Q, bool ADJ>
cudaError_t launch_fwd_q(const FwdArgs &a, dim3 grid, size_t smem, cudaStream_t st)
{
    if constexpr (Q == 8) {
        if (a.r == 8) return launch_fwd_qr<8, 8, ADJ>(a, grid, smem, st);
        if (a.r == 5) return launch_fwd_qr<8, 5, ADJ>(a, grid, smem, st);
    }
    return launch_fwd_qr<Q, -1, ADJ>(a, grid, smem, st);
}

template <int Q, bool ADJ>
cudaError_t prepare_q(int r, size_t smem)
{
    if constexpr (Q == 8) {
        if (r == 8) return prepare_qr<8, 8, ADJ>(smem);
        if (r == 5) return prepare_qr<8, 5, ADJ>(smem);
    }
    return prepare_qr<Q, -1, ADJ>(smem);
}

template <int Q>
size_t smem_q(int r, bool adj)
{
    const FwdGeom gm(r, specialised(Q, r));
    // alignment slack, window sums (rounded to 128 bytes), staged rows, mbarrier
    return 128 + sizeof(float) * (((size_t)kB * Chan<Q>::NCH * gm.VS + 31) / 32 * 32 + (size_t)2 * kB * (Q + 3) * gm.WSt) + 16;
}

}  // namespace

#define FLR_Q_DISPATCH(q, ...)  \
    switch (q) {                 \
    case 1: { constexpr int QQ = 1; __VA_ARGS__; } \
    case 2: { constexpr int QQ = 2; __VA_ARGS__; } \
    case 3: { constexpr int QQ = 3; __VA_ARGS__; } \
    case 4: { constexpr int QQ = 4; __VA_ARGS__; } \
    case 5: { constexpr int QQ = 5; __VA_ARGS__; } \
    case 6: { constexpr int QQ = 6; __VA_ARGS__; } \
    case 7: { constexpr int QQ = 7; __VA_ARGS__; } \
    case 8: { constexpr int QQ = 8; __VA_ARGS__; } \
    default: break;              \
    }

cudaError_t launch_fwd(int q, const FwdArgs &a, dim3 grid, size_t smem, cudaStream_t st)
{
    FLR_Q_DISPATCH(q, return launch_fwd_q<QQ, false>(a, grid, smem, st));
    return cudaErrorInvalidValue;
}

cudaError_t launch_adj(int q, const FwdArgs &a, dim3 grid, size_t smem, cudaStream_t st)
{
    FLR_Q_DISPATCH(q, return launch_fwd_q<QQ, true>(a, grid, smem, st));
    return cudaErrorInvalidValue;
}

cudaError_t launch_frame_shift(int q, const float *guide, const float *rad, int H, int W, int ref_rows, float *shift_out,
                               cudaStream_t st)
{
    FLR_Q_DISPATCH(q, frame_shift_kernel<QQ><<<1, 32, 0, st>>>(guide, rad, H, W, ref_rows, shift_out);
                   return cudaGetLastError());
    return cudaErrorInvalidValue;
}

size_t fwd_smem_bytes(int q, int r)
{
    FLR_Q_DISPATCH(q, return smem_q<QQ>(r, false));
    return 0;
}

size_t adj_smem_bytes(int q, int r)
{
    FLR_Q_DISPATCH(q, return smem_q<QQ>(r, true));
    return 0;
}

cudaError_t fwd_prepare(int q, int r, size_t smem)
{
    FLR_Q_DISPATCH(q, return prepare_q<QQ, false>(r, smem));
    return cudaErrorInvalidValue;
}

cudaError_t adj_prepare(int q, int r, size_t smem)
{
    FLR_Q_DISPATCH(q, return prepare_q<QQ, true>(r, smem));
    return cudaErrorInvalidValue;
}

}  // namespace flr
