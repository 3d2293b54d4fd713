// flr_fused.cu -- the whole FLR forward pass in one kernel (sm_103a): windowed moments,
// per-pixel centred ridge solve, coefficient averaging and apply.
//
// What it computes (arXiv 2410.11625, Sec. 3.1-3.2 and the Appendix): for every pixel k, the
// box sums over the clipped radius-r window of the linear moments and of the outer products
// x x^T, x y^T (box-filtering the outer products gives X_k^T X_k and X_k^T Y_k exactly), the
// centred ridge model a_k = (W_k + eps I)^{-1} (X^T Y / n - mu_X mu_Y^T), b_k = mu_Y - a_k^T mu_X
// (the Appendix's decomposition with eps on the diagonal of W), then the mean of the models
// over the clipped radius-rc window around each output pixel i, applied to its map-guide
// vector: I_i = mean_k b_k + (mean_k a_k)^T z_i.  With rc = 0 the pixel's own model is
// applied (Sec. 3.1, I_k = x_k A_k).
//
// Work layout.  One CTA owns a strip of TW output columns and a segment of output rows and
// walks down it kB rows per batch.  It solves TS = TW + 2 rc columns (the models its averaging
// window needs) over the rows [y0 - rc, y1 + rc), and sums moments over TM = TS + 2 r columns.
// Per batch, separated by CTA barriers:
//   1. V-pass: 12 warps of walkers, one thread per (walker column, third of the channel pairs),
//      keep vertical window sums of their channels as two accumulators per channel: E, the
//      products of the rows entered since the last block start, and Dn, the products of the
//      rows left since then minus the previous block's total.  A block is 2r + 1 rows, so
//      V = E - Dn is always a sum of at most 2(2r + 1) rounded terms: the error does not grow
//      along the strip.  Products are recomputed from TMA-staged entering and leaving rows and
//      accumulated two channels at a time with packed FP32 FMAs (fma.rn.f32x2).  Between
//      batches a walker's accumulators wait in tensor memory (tcgen05.st / tcgen05.ld), not in
//      registers, so the solve has the register file to itself.
//   2. H-pass: the horizontal radius-r sums of every channel pair, in place, two chunks per
//      row, each chunk re-seeded by a direct (2r + 1)-term sum (bounded drift).
//   3. Solve: one thread per pixel: centred, unnormalised moments (n M = S - L mu^T + n eps I),
//      left-looking Cholesky in registers, three right-hand sides.  A pixel whose pivot ratio
//      falls to tau or below is listed for an FP64 re-solve and left out of the average (its
//      FP64 model is added by flr_fused_fix_kernel).
//   4. Coefficient H-pass: horizontal radius-rc sums of the 3(Q+1) model coefficients.
//   5. Coefficient V-pass and apply: one thread per (output column, colour) keeps the vertical
//      radius-rc sums of its Q + 1 coefficients with the same block accumulators; the rows
//      that leave its window come from a ring of 2rc + 1 rows kept in tensor memory (the
//      256 KB tensor memory of the SM holds the ring and the walkers' accumulators).
// Values are shifted by the mean of a 16 x 16 sample grid of the CTA's input region before
// any product (the centred form is shift-invariant), and the models are applied in the same
// shifted coordinates, so no frame-wide reference is needed.
#include <cstring>
#include <mutex>
#include <utility>

#include "flr_device.cuh"
#include "flr_fp64_model.cuh"
#include "flr_internal.cuh"
#include "flr_tmem.cuh"
#include "tma.cuh"

namespace flr {
namespace fused {

constexpr int kB = 4;                     // rows per batch
constexpr int kThreads = 384;             // 12 warps
constexpr int kWarps = kThreads / 32;
constexpr int kTS = kThreads / kB;        // solve columns: one solver thread per batch pixel
constexpr unsigned long long kTimeoutNs = 1000000000ull;  // 1 s per bounded wait

__host__ __device__ constexpr int tile_width(int rc) { return (kTS - 2 * rc) & ~3; }

// ---- walker groups -------------------------------------------------------------------
// The NCH moment channels (numbered as in Chan) fall into rows that share their left factor:
// the linear moments (left factor 1: x_0..x_{Q-1}, y_0..y_2) and, for each guide u, the
// products x_u x_v (v = u..Q-1) and x_u y_c, whose right factors are the input slots u..Q+2.
// A walker thread keeps the vertical sums of one group of rows for a pair of adjacent columns,
// so the packed FMAs (fma.rn.f32x2) take their operands straight from 8-byte shared loads of
// the staged rows.  Six groups of at most 13 channels: the linear row, row 0, row 1, and the
// row pairs {2, 7}, {3, 6}, {4, 5}; a group reads the slots from its smallest left factor up.
template <int Q>
struct Groups {
    static_assert(Q == 8, "the walker groups are laid out for eight guides");
    static constexpr int NG = 6, MAXG = 13;
    __host__ __device__ static constexpr int row_a(int g) { return g == 0 ? -1 : g - 1; }
    __host__ __device__ static constexpr int row_b(int g) { return g >= 3 ? Q + 2 - g : -2; }  // -2: none
    __host__ __device__ static constexpr int row_len(int u) { return u < 0 ? Q + 3 : Q + 3 - u; }
    __host__ __device__ static constexpr int size(int g)
    {
        return row_len(row_a(g)) + (row_b(g) >= -1 ? row_len(row_b(g)) : 0);
    }
    // the i-th channel of group g
    __host__ __device__ static constexpr int ch(int g, int i)
    {
        const int ua = row_a(g), na = row_len(ua);
        const int u = i < na ? ua : row_b(g);
        const int k = i < na ? i : i - na;
        if (u < 0) return k < Q ? Chan<Q>::X0 + k : Chan<Q>::Y0 + (k - Q);
        const int v = u + k;
        return v < Q ? Chan<Q>::xx(u, v) : Chan<Q>::xy(u, v - Q);
    }
    __host__ __device__ static constexpr int s0(int g) { return row_a(g) < 0 ? 0 : row_a(g); }
};

// Compile-time geometry of one instantiation.
template <int Q, int R, int RC>
struct Geo {
    static constexpr int NS = Q + 3;
    static constexpr int NCH = Chan<Q>::NCH;
    static constexpr int NCF = 3 * (Q + 1);       // model coefficients per pixel
    static constexpr int NCHB = NCH > 2 * NCF ? NCH : 2 * NCF;  // channel rows of the buffer
    static constexpr int TW = tile_width(RC);     // output columns
    static constexpr int TS = TW + 2 * RC;        // solve columns
    static constexpr int TM = TS + 2 * R;         // walker columns
    static constexpr int NCP = TM / 2;            // walker column pairs
    static constexpr int RA = (R + RC + 3) & ~3;  // staged rows start at column x0 - RA
    // staged row length: covers TW + 2 RA columns, and kB rows of it are a multiple of 128
    // bytes, so every TMA box of the staging buffer starts 128-byte aligned
    static constexpr int WSt = (TW + 2 * RA + 7) & ~7;
    static constexpr int SOFF = RA - R - RC;      // staged column of walker column 0
    static constexpr int VS = TM + ((12 - TM % 8) % 8);  // row stride >= TM, = 4 (mod 8)
    static constexpr int WR = 2 * R + 1, WC = 2 * RC + 1;
    static constexpr int CH = (TS / 2 + 3) & ~3;  // H-pass: runs [0, CH) and [CH, TS)
    static constexpr int CL = (TW / 2 + 3) & ~3;  // coefficient H-pass: runs [0, CL), [CL, TW)
    static constexpr int COLOUR_WARPS = (3 * TW + 31) / 32;
    static constexpr size_t VBUF_FLOATS = ((size_t)kB * NCHB * VS + 31) / 32 * 32;
    static constexpr size_t STAGE_FLOATS = (size_t)2 * NS * kB * WSt;
    // map-guide rows of a batch's output rows (the apply reads them), double-buffered
    static constexpr size_t ZBUF_FLOATS = RC > 0 ? ((size_t)Q * kB * TW + 31) / 32 * 32 : 0;
    static constexpr unsigned ZBYTES = (unsigned)(Q * kB * TW * 4);
    static constexpr size_t SMEM = 128 + 4 * (VBUF_FLOATS + STAGE_FLOATS + 2 * ZBUF_FLOATS) + 16;
    static_assert(TS <= kTS && TM <= 112 && WSt <= 112, "strip geometry");
    static_assert((kB * WSt * 4) % 128 == 0 && (VBUF_FLOATS * 4) % 128 == 0, "TMA boxes 128-byte aligned");
    static_assert(SOFF + TM <= WSt, "walker columns inside the staged rows");
    static_assert((R + RC) % 2 == 0 && SOFF % 2 == 0, "column pairs start at even columns");
    static_assert(NCP <= 64, "two warps of walkers per group");
    static_assert(CH > 2 * R && CH < TS && CL < TW, "H-pass runs");
    static_assert(RC == 0 || (WC <= 17 && COLOUR_WARPS <= 8 && WC >= 4), "coefficient ring");
    static_assert(Q + 1 <= 9, "colour state: 18 tensor-memory columns");
};

// Tensor-memory columns (per lane; 512 allocated, every access aligned to its width).
// Walker warp w (k = w / 4) keeps its 52 accumulators at 32 k (x32), 96 + 16 k (x16) and
// 144 + 4 k (x4); colour warp w (k = w / 4 < 2) keeps its ring slot s at 160 + 136 k + 8 s
// (x8) and 432 + 17 k + s (x1), and its 18 accumulators at 480 + 16 k (x16), 156 + 2 k (x2).
constexpr uint32_t kTmemCols = 512;
__device__ __forceinline__ uint32_t col_w32(int k) { return 32u * k; }
__device__ __forceinline__ uint32_t col_w16(int k) { return 96u + 16u * k; }
__device__ __forceinline__ uint32_t col_w4(int k) { return 144u + 4u * k; }
__device__ __forceinline__ uint32_t col_c2(int k) { return 156u + 2u * k; }
__device__ __forceinline__ uint32_t col_ring8(int k, int s) { return 160u + 136u * k + 8u * s; }
__device__ __forceinline__ uint32_t col_ring1(int k, int s) { return 432u + 17u * k + s; }
__device__ __forceinline__ uint32_t col_c16(int k) { return 480u + 16u * k; }

// ---- V-pass: one group of channels, two columns ---------------------------------------
// E += left(e) * right(e), Dn += left(l) * right(l), V = E - Dn for every channel of group G;
// e and l: the shifted values of the entering and the leaving row at the two columns.
template <int Q, int G, int I>
__device__ __forceinline__ void walk_enter(float2 (&E)[13], const float2 (&e)[Q + 3])
{
    constexpr int c = Groups<Q>::ch(G, I);
    constexpr int u = Chan<Q>::slot_u(c), v = Chan<Q>::slot_v(c);
    if constexpr (v < 0) E[I] = __fadd2_rn(E[I], e[u]);
    else E[I] = __ffma2_rn(e[u], e[v], E[I]);
}
template <int Q, int G, int I>
__device__ __forceinline__ void walk_store(const float2 (&E)[13], const float2 (&Dn)[13], float *vcol, int VS)
{
    constexpr int c = Groups<Q>::ch(G, I);
    *reinterpret_cast<float2 *>(vcol + (size_t)c * VS) = __ffma2_rn(Dn[I], make_float2(-1.f, -1.f), E[I]);
}
// se: the staged entering row of this batch row at the walker's first column; planes are
// kB * WST floats apart, the leaving rows NS planes further on.
template <int Q, int G, int WST, int... I>
__device__ __forceinline__ void walk_rows(float2 (&E)[13], float2 (&Dn)[13], float *vcol, int VS, const float *se,
                                         const float2 (&nsh)[Q + 3], bool ein, bool lout,
                                         std::integer_sequence<int, I...>)
{
    constexpr int NS = Q + 3, S0 = Groups<Q>::s0(G);
    constexpr size_t PL = (size_t)kB * WST;
    if (ein) {
        float2 e[NS];
#pragma unroll
        for (int k = S0; k < NS; ++k) e[k] = __fadd2_rn(*reinterpret_cast<const float2 *>(se + k * PL), nsh[k]);
        (walk_enter<Q, G, I>(E, e), ...);
    }
    if (lout) {
        const float *sl = se + NS * PL;
        float2 l[NS];
#pragma unroll
        for (int k = S0; k < NS; ++k) l[k] = __fadd2_rn(*reinterpret_cast<const float2 *>(sl + k * PL), nsh[k]);
        (walk_enter<Q, G, I>(Dn, l), ...);
    }
    (walk_store<Q, G, I>(E, Dn, vcol, VS), ...);
}

// ---- solve ---------------------------------------------------------------------------------
// Centred ridge model of one pixel from its window sums S (moment channels, Chan order), in
// the unnormalised form n M = S - L mu^T + n eps I, n D = XY - L_y mu^T (the same a as
// M^{-1} D).  Returns whether a Cholesky pivot ratio d_j / (n M)_jj fell to tau or below.
template <int Q>
__device__ __forceinline__ bool solve_px(const float (&S)[Chan<Q>::NCH], float n, float eps, float tau,
                                         float (&A)[Q][3], float (&bv)[3])
{
    using C = Chan<Q>;
    using dev::tri;
    const float inv_n = 1.0f / n;
    float mu[Q], muy[3];
#pragma unroll
    for (int i = 0; i < Q; ++i) mu[i] = S[C::X0 + i] * inv_n;
#pragma unroll
    for (int c = 0; c < 3; ++c) muy[c] = S[C::Y0 + c] * inv_n;
    const float ne = n * eps;
    float L[Q * (Q + 1) / 2], inv_d[Q], Z[Q][3];
#pragma unroll
    for (int i = 0; i < Q; ++i)
#pragma unroll
        for (int j = 0; j < Q; ++j)
            if (j <= i) L[tri(i, j)] = fmaf(-mu[i], S[C::X0 + j], S[C::xx(j, i)]) + (i == j ? ne : 0.f);
#pragma unroll
    for (int i = 0; i < Q; ++i)
#pragma unroll
        for (int c = 0; c < 3; ++c) Z[i][c] = fmaf(-mu[i], S[C::Y0 + c], S[C::xy(i, c)]);
    bool low = false;
    const float dmin = ne > 0.f ? ne : 1e-30f;  // every exact pivot is >= n eps
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        const float mjj = L[tri(j, j)];
        float d = mjj;
#pragma unroll
        for (int k = 0; k < Q; ++k)
            if (k < j) d = fmaf(-L[tri(j, k)], L[tri(j, k)], d);
        low |= !(d > tau * mjj);
        d = fmaxf(d, dmin);
        const float il = rsqrtf(d);
        inv_d[j] = il;
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
        // forward substitution of the three right-hand sides, row j
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float t = Z[j][c];
#pragma unroll
            for (int k = 0; k < Q; ++k)
                if (k < j) t = fmaf(-L[tri(j, k)], Z[k][c], t);
            Z[j][c] = t * il;
        }
    }
    // back substitution L^T a = z
#pragma unroll
    for (int c = 0; c < 3; ++c) {
#pragma unroll
        for (int ii = 0; ii < Q; ++ii) {
            const int i = Q - 1 - ii;
            float t = Z[i][c];
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

// Kernel parameters: TMA maps of the guide [Q][H][W] and radiance [3][H][W] planes (boxes of
// WSt columns x kB rows x all planes) and the arguments.
struct alignas(128) KArgs {
    CUtensorMap tg, tr, tz;  // tz: the map guide, boxes of TW columns x kB rows x Q planes
    FusedArgs a;
};

template <int Q, int R, int RC>
__global__ void __launch_bounds__(kThreads, 1) flr_fused_kernel(const __grid_constant__ KArgs ka)
{
    using C = Chan<Q>;
    using G = Geo<Q, R, RC>;
    constexpr int NS = G::NS, NCH = G::NCH, NCF = G::NCF, NCHB = G::NCHB;
    constexpr int TW = G::TW, TS = G::TS, WSt = G::WSt, VS = G::VS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ float s_sh[NS];
    __shared__ int s_abort, s_nlist, s_wcnt[kWarps];
    __shared__ uint32_t s_tmem;
    const FusedArgs &a = ka.a;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int H = a.H, W = a.W;
    const size_t plane = (size_t)H * W;
    const int x0 = blockIdx.x * TW;
    const int row_hi = a.row_hi < 0 ? H : min(a.row_hi, H);
    const int y0 = a.row_lo + blockIdx.y * a.TH;
    const int y1 = min(y0 + a.TH, row_hi);
    const int cta = blockIdx.y * gridDim.x + blockIdx.x;
    if (y0 >= y1) {  // a segment past the last row (not produced by the host plan)
        if (tid == 0) a.list_count[cta] = 0;
        return;
    }
    const int m_lo = y0 - RC, m_hi = y1 + RC;  // solve rows
    const int v0 = m_lo - 2 * R;               // first walker row: the window starts empty
    int *list = a.list + (size_t)cta * a.list_cap;

    unsigned char *base = smem_raw + ((128 - (tma::smem_addr(smem_raw) & 127)) & 127);
    float *Vbuf = reinterpret_cast<float *>(base);  // [kB][NCHB][VS]: channel rows
    float *stage = Vbuf + G::VBUF_FLOATS;            // [2][NS][kB][WSt]: entering, leaving rows
    float *zbuf = stage + G::STAGE_FLOATS;           // [2][Q][kB][TW]: map-guide rows of the outputs
    uint64_t *bar = reinterpret_cast<uint64_t *>(zbuf + 2 * G::ZBUF_FLOATS);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(tma::smem_addr(&s_tmem)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid == 0) {
        s_abort = 0;
        s_nlist = 0;
        tma::mbar_init(bar, 1);
        tma::mbar_init_fence();
    }
    // the CTA's reference shift: mean of a 16 x 16 sample grid of its input region
    if (warp == 1)
        dev::sample_mean<Q>(s_sh, a.guide, a.rad, H, W, max(0, m_lo - R), min(H, m_hi + R), max(0, x0 - RC - R),
                            min(W, x0 + TW + RC + R), lane);
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = s_tmem + ((uint32_t)(32 * (warp & 3)) << 16);  // this warp's lane quarter
    const int slot_k = warp >> 2;

    // stage the entering (vb + R) and leaving (vb - R - 1) input rows of batch v
    // and, with averaging, the map-guide rows of its output rows v - RC .. into zbuf[batch & 1]
    auto stage_batch = [&](int v) {
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // earlier reads before the copies
        tma::mbar_expect_tx(bar, (unsigned)(2 * NS * kB * WSt * 4) + (RC > 0 ? G::ZBYTES : 0u));
        const size_t box = (size_t)kB * WSt;
        tma::load_3d(stage, &ka.tg, x0 - G::RA, v + R, 0, bar);
        tma::load_3d(stage + Q * box, &ka.tr, x0 - G::RA, v + R, 0, bar);
        tma::load_3d(stage + NS * box, &ka.tg, x0 - G::RA, v - R - 1, 0, bar);
        tma::load_3d(stage + (NS + Q) * box, &ka.tr, x0 - G::RA, v - R - 1, 0, bar);
        if constexpr (RC > 0) tma::load_3d(zbuf + ((v - v0) / kB & 1) * G::ZBUF_FLOATS, &ka.tz, x0, v - RC, 0, bar);
    };
    if (tid == 0) stage_batch(v0);
    int nstaged = 1, nconsumed = 0;

    // walker identity: two warps per channel group, one thread per column pair; walker
    // column 2 cp is global column x0 - RC - R + 2 cp and staged column 2 cp + SOFF
    const int group = warp >> 1;
    const int wcp = ((warp & 1) << 5) + lane;
    const bool walker = wcp < G::NCP;
    const int gxw = x0 - RC - R + 2 * wcp;
    const bool wcol_in = gxw >= 0 && gxw < W;  // W is even and gxw even: both columns or neither
    // solver identity
    const int sb = tid / kTS, sxs = tid % kTS;
    const int sgx = x0 - RC + sxs;
    // colour-thread identity (coefficient V-pass and apply)
    const int cc = tid / TW, cx = tid % TW;
    const bool colour = tid < 3 * TW;
    const int cgx = x0 + cx;
    const float *zg = a.map_guide ? a.map_guide : a.guide;
    unsigned bad = 0;  // non-finite outputs written by this thread

    const float tau = a.tau, eps = a.eps;
    for (int v = v0; v < m_hi; v += kB) {
        if (!tma::wait_warp(bar, (uint32_t)(nconsumed & 1), kTimeoutNs) && lane == 0) {
            s_abort = 1;
            if (a.status) atomicExch(a.status, 1);
        }
        ++nconsumed;
        __syncthreads();
        if (s_abort) break;

        // 1. V-pass
        {
            float2 E[13], Dn[13];
            if (v == v0) {
#pragma unroll
                for (int i = 0; i < 13; ++i) E[i] = Dn[i] = make_float2(0.f, 0.f);
            } else {
                uint32_t st[52];
                tm_ld32(tmem + col_w32(slot_k), st);
                tm_ld16(tmem + col_w16(slot_k), st + 32);
                tm_ld4(tmem + col_w4(slot_k), st + 48);
                tm_wait_ld();
#pragma unroll
                for (int i = 0; i < 13; ++i) {
                    E[i] = make_float2(__uint_as_float(st[2 * i]), __uint_as_float(st[2 * i + 1]));
                    Dn[i] = make_float2(__uint_as_float(st[26 + 2 * i]), __uint_as_float(st[27 + 2 * i]));
                }
            }
            if (walker) {
                float2 nsh[NS];  // minus the shift, both columns (zero outside the image)
#pragma unroll
                for (int k = 0; k < NS; ++k) {
                    const float t = wcol_in ? -s_sh[k] : 0.f;
                    nsh[k] = make_float2(t, t);
                }
#pragma unroll 1
                for (int b = 0; b < kB; ++b) {
                    const int vb = v + b;
                    if (vb >= m_hi) break;
                    const int t = vb - v0;
                    if (t % G::WR == 0) {  // block start: Dn = -(previous block total), E = 0
#pragma unroll
                        for (int i = 0; i < 13; ++i) {
                            Dn[i] = __fmul2_rn(E[i], make_float2(-1.f, -1.f));
                            E[i] = make_float2(0.f, 0.f);
                        }
                    }
                    const bool ein = vb + R >= 0 && vb + R < H;
                    const bool lout = t >= G::WR && vb - R - 1 >= 0 && vb - R - 1 < H;
                    const float *se = stage + (size_t)b * WSt + 2 * wcp + G::SOFF;
                    float *vcol = Vbuf + (size_t)b * NCHB * VS + 2 * wcp;
                    switch (group) {
                    case 0: walk_rows<Q, 0, WSt>(E, Dn, vcol, VS, se, nsh, ein, lout, std::make_integer_sequence<int, Groups<Q>::size(0)>{}); break;
                    case 1: walk_rows<Q, 1, WSt>(E, Dn, vcol, VS, se, nsh, ein, lout, std::make_integer_sequence<int, Groups<Q>::size(1)>{}); break;
                    case 2: walk_rows<Q, 2, WSt>(E, Dn, vcol, VS, se, nsh, ein, lout, std::make_integer_sequence<int, Groups<Q>::size(2)>{}); break;
                    case 3: walk_rows<Q, 3, WSt>(E, Dn, vcol, VS, se, nsh, ein, lout, std::make_integer_sequence<int, Groups<Q>::size(3)>{}); break;
                    case 4: walk_rows<Q, 4, WSt>(E, Dn, vcol, VS, se, nsh, ein, lout, std::make_integer_sequence<int, Groups<Q>::size(4)>{}); break;
                    default: walk_rows<Q, 5, WSt>(E, Dn, vcol, VS, se, nsh, ein, lout, std::make_integer_sequence<int, Groups<Q>::size(5)>{}); break;
                    }
                }
            }
            __syncwarp();  // the walkers' branches rejoin before the warp-wide tensor-memory store
            uint32_t st[52];
#pragma unroll
            for (int i = 0; i < 13; ++i) {
                st[2 * i] = __float_as_uint(E[i].x);
                st[2 * i + 1] = __float_as_uint(E[i].y);
                st[26 + 2 * i] = __float_as_uint(Dn[i].x);
                st[27 + 2 * i] = __float_as_uint(Dn[i].y);
            }
            tm_st32(tmem + col_w32(slot_k), st);
            tm_st16(tmem + col_w16(slot_k), st + 32);
            tm_st4(tmem + col_w4(slot_k), st + 48);
            tm_wait_st();
        }
        __syncthreads();
        // prefetch the next batch's rows while this one is summed, solved and applied
        if (v + kB < m_hi) {
            if (tid == 0) stage_batch(v + kB);
            ++nstaged;
        }
        if (v + kB <= m_lo) continue;  // every row of this batch is a warm-up row

        // 2. H-pass: one thread per (row b, channel), in place, seeded at 0 and CH
        {
            const int hb = tid / NCH, hch = tid % NCH;
            if (tid < kB * NCH && v + hb >= m_lo && v + hb < m_hi) {
                float *row = Vbuf + ((size_t)hb * NCHB + hch) * VS;
                dev::hsum_run<R, G::CH>(row, row, 0);
                dev::hsum_run<R, TS - G::CH>(row, row, G::CH);
            }
        }
        __syncthreads();

        // 3. solve: one thread per pixel of the batch
        bool flag = false;
        {
            const int m = v + sb;
            if (sxs < TS && m >= m_lo && m < m_hi) {
                const bool live = m >= 0 && m < H && sgx >= 0 && sgx < W;
                float *col = Vbuf + (size_t)sb * NCHB * VS + sxs;
                float A[Q][3], bv[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    bv[c] = 0.f;
#pragma unroll
                    for (int i = 0; i < Q; ++i) A[i][c] = 0.f;
                }
                if (live) {
                    float S[NCH];
#pragma unroll
                    for (int ch = 0; ch < NCH; ++ch) S[ch] = col[(size_t)ch * VS];
                    const float ny = (float)(min(m + R, H - 1) - max(m - R, 0) + 1);
                    const float nx = (float)(min(sgx + R, W - 1) - max(sgx - R, 0) + 1);
                    const bool low = solve_px<Q>(S, ny * nx, eps, tau, A, bv);
                    flag = low && tau > 0.f;
                }
                if constexpr (RC > 0) {
                    // model coefficients (relative to the CTA shift) into channel rows [0, NCF)
                    // of this pixel, colour-major; a flagged pixel contributes zero here and its
                    // FP64 model later
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        col[(size_t)(c * (Q + 1)) * VS] = flag ? 0.f : bv[c];
#pragma unroll
                        for (int i = 0; i < Q; ++i) col[(size_t)(c * (Q + 1) + 1 + i) * VS] = flag ? 0.f : A[i][c];
                    }
                } else {
                    if (live && !flag) {
                        const size_t off = (size_t)m * W + sgx;
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            float o = bv[c];
#pragma unroll
                            for (int i = 0; i < Q; ++i) o = fmaf(A[i][c], __ldg(zg + i * plane + off) - s_sh[i], o);
                            o += s_sh[Q + c];
                            a.out[c * plane + off] = o;
                            bad += !isfinite(o);
                        }
                    }
                }
            }
        }
        const int any_flag = __syncthreads_or(flag);
        if (any_flag) {  // append the flagged pixels in (row, column) order
            const unsigned bal = __ballot_sync(0xffffffffu, flag);
            if (lane == 0) s_wcnt[warp] = __popc(bal);
            __syncthreads();
            int at = s_nlist;
            for (int w = 0; w < warp; ++w) at += s_wcnt[w];
            if (flag) list[at + __popc(bal & ((1u << lane) - 1u))] = (v + sb) * W + sgx;
            __syncthreads();
            if (tid == 0) {
                int tot = 0;
                for (int w = 0; w < kWarps; ++w) tot += s_wcnt[w];
                s_nlist += tot;
            }
        }
        if constexpr (RC > 0) {
            // 4. coefficient H-pass: unit (row b, coefficient k, half h): row k -> row NCF + k
            {
                const int uk = tid % NCF, uh = (tid / NCF) & 1, ub = tid / (2 * NCF);
                if (tid < kB * NCF * 2 && v + ub >= m_lo && v + ub < m_hi) {
                    const float *in = Vbuf + ((size_t)ub * NCHB + uk) * VS;
                    float *outp = Vbuf + ((size_t)ub * NCHB + NCF + uk) * VS;
                    if (uh == 0) dev::hsum_run<RC, G::CL>(in, outp, 0);
                    else dev::hsum_run<RC, TW - G::CL>(in, outp, G::CL);
                }
            }
            __syncthreads();
            // 5. coefficient V-pass and apply: thread (colour cc, column cx)
            if (warp < G::COLOUR_WARPS) {
                // map-guide values of this batch's output rows, loaded first so that their
                // latency overlaps the tensor-memory traffic below
                const float *zb = zbuf + ((v - v0) / kB & 1) * G::ZBUF_FLOATS + (colour ? cx : 0);
                float Ec[Q + 1], Dc[Q + 1];
                if (v <= m_lo) {
#pragma unroll
                    for (int j = 0; j <= Q; ++j) Ec[j] = Dc[j] = 0.f;
                } else {
                    uint32_t st[18];
                    tm_ld16(tmem + col_c16(slot_k), st);
                    tm_ld2(tmem + col_c2(slot_k), st + 16);
                    tm_wait_ld();
#pragma unroll
                    for (int j = 0; j <= Q; ++j) {
                        Ec[j] = __uint_as_float(st[j]);
                        Dc[j] = __uint_as_float(st[9 + j]);
                    }
                }
                // the rows leaving the window, from the ring
                uint32_t lv[kB][9];
#pragma unroll
                for (int b = 0; b < kB; ++b) {
                    const int tcm = v + b - m_lo;
                    if (tcm >= G::WC && v + b < m_hi) {
                        tm_ld8(tmem + col_ring8(slot_k, tcm % G::WC), lv[b]);
                        lv[b][8] = tm_ld1(tmem + col_ring1(slot_k, tcm % G::WC));
                    }
                }
                tm_wait_ld();
                const float *hcol = Vbuf + (size_t)(NCF + (colour ? cc : 0) * (Q + 1)) * VS + cx;
                const float mx = (float)(min(cgx + RC, W - 1) - max(cgx - RC, 0) + 1);
                const float inv_mx = 1.0f / mx;
#pragma unroll
                for (int b = 0; b < kB; ++b) {
                    const int m = v + b, tcm = m - m_lo;
                    if (tcm < 0 || m >= m_hi) continue;
                    if (tcm % G::WC == 0) {
#pragma unroll
                        for (int j = 0; j <= Q; ++j) {
                            Dc[j] = -Ec[j];
                            Ec[j] = 0.f;
                        }
                    }
                    if (tcm >= G::WC) {
#pragma unroll
                        for (int j = 0; j <= Q; ++j) Dc[j] += __uint_as_float(lv[b][j]);
                    }
                    uint32_t ent[9];
#pragma unroll
                    for (int j = 0; j <= Q; ++j) {
                        const float hv = colour ? hcol[(size_t)(b * NCHB + j) * VS] : 0.f;
                        Ec[j] += hv;
                        ent[j] = __float_as_uint(hv);
                    }
#pragma unroll
                    for (int j = Q + 1; j < 9; ++j) ent[j] = 0u;
                    __syncwarp();
                    tm_st8(tmem + col_ring8(slot_k, tcm % G::WC), ent);
                    tm_st1(tmem + col_ring1(slot_k, tcm % G::WC), ent[8]);
                    const int y = m - RC;
                    if (colour && y >= y0 && y < y1 && cgx < W) {
                        const float my = (float)(min(y + RC, H - 1) - max(y - RC, 0) + 1);
                        float o = Ec[0] - Dc[0];
#pragma unroll
                        for (int i = 0; i < Q; ++i)
                            o = fmaf(Ec[1 + i] - Dc[1 + i], zb[(i * kB + b) * TW] - s_sh[i], o);
                        o = fmaf(o, inv_mx / my, s_sh[Q + cc]);
                        a.out[cc * plane + (size_t)y * W + cgx] = o;
                        bad += !isfinite(o);
                    }
                }
                __syncwarp();
                uint32_t st[18];
#pragma unroll
                for (int j = 0; j < 9; ++j) {
                    st[j] = __float_as_uint(j <= Q ? Ec[j] : 0.f);
                    st[9 + j] = __float_as_uint(j <= Q ? Dc[j] : 0.f);
                }
                tm_st16(tmem + col_c16(slot_k), st);
                tm_st2(tmem + col_c2(slot_k), st + 16);
                tm_wait_st();
            }
        }
    }
    // after a wait ran out: give the copy it waited for one more bounded wait to land before
    // the CTA exits (no further copy was issued)
    if (s_abort && tid < 32) tma::wait_warp(bar, (uint32_t)((nconsumed - 1) & 1), kTimeoutNs);
    if (bad && a.nonfinite) atomicAdd(a.nonfinite, (unsigned long long)bad);
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(s_tmem), "r"(kTmemCols));
    }
    if (tid == 0) a.list_count[cta] = s_nlist;
    if (tid < NS) a.cta_shift[(size_t)cta * NS + tid] = s_sh[tid];
}

// ---- FP64 correction of flagged pixels ----------------------------------------------------
// One CTA per CTA of the fused launch.  Its flagged pixels (in row, column order) get FP64
// models (one warp each, window sums recomputed in FP64 from the inputs), relative to the
// fused CTA's shift.  With rc = 0 the model's result is written to the pixel; with rc > 0 each
// model's share, (b + a^T (z_i - s)) / m_i, is added to every output i of this CTA whose
// averaging window holds the pixel, one flagged pixel after the other (a fixed order, so the
// result is deterministic).  Adds the number of flagged pixels that this CTA owns (outputs of
// its strip segment) to flag_count.
constexpr int kFixThreads = 256, kFixWarps = kFixThreads / 32;

template <int Q>
__global__ void __launch_bounds__(kFixThreads) flr_fused_fix_kernel(const FusedArgs a)
{
    constexpr int NS = Q + 3, NCF = 3 * (Q + 1);
    __shared__ double s_model[kFixWarps][NCF];
    __shared__ float s_sh[NS];
    __shared__ unsigned long long s_cnt[2];
    const int cta = blockIdx.y * gridDim.x + blockIdx.x;
    const int n = a.list_count[cta];
    if (n == 0) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int H = a.H, W = a.W, rc = a.rc;
    const size_t plane = (size_t)H * W;
    const int TW = tile_width(rc);
    const int x0 = blockIdx.x * TW;
    const int row_hi = a.row_hi < 0 ? H : min(a.row_hi, H);
    const int y0 = a.row_lo + blockIdx.y * a.TH;
    const int y1 = min(y0 + a.TH, row_hi);
    const int x1 = min(x0 + TW, W);
    const int *list = a.list + (size_t)cta * a.list_cap;
    const float *zg = a.map_guide ? a.map_guide : a.guide;
    if (tid < NS) s_sh[tid] = a.cta_shift[(size_t)cta * NS + tid];
    if (tid < 2) s_cnt[tid] = 0ull;
    __syncthreads();
    unsigned own = 0;
    for (int e = tid; e < n; e += kFixThreads) {
        const int idx = list[e], py = idx / W, px = idx % W;
        own += py >= y0 && py < y1 && px >= x0 && px < x1;
    }
    long long dbad = 0;  // change in the number of non-finite output values
    for (int e0 = 0; e0 < n; e0 += kFixWarps) {
        if (e0 + warp < n) {
            double A[Q][3], bv[3];
            dev::fp64_model<Q>(a.guide, a.rad, H, W, a.r, (double)a.eps, list[e0 + warp], lane, s_sh, A, bv);
            if (lane == 0) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    s_model[warp][c * (Q + 1)] = bv[c];
#pragma unroll
                    for (int i = 0; i < Q; ++i) s_model[warp][c * (Q + 1) + 1 + i] = A[i][c];
                }
            }
        }
        __syncthreads();
        const int ne = min(kFixWarps, n - e0);
        for (int k = 0; k < ne; ++k) {
            const int idx = list[e0 + k], py = idx / W, px = idx % W;
            const double *md = s_model[k];
            if (rc == 0) {
                if (tid < 3 && py >= y0 && py < y1 && px >= x0 && px < x1) {
                    double o = md[tid * (Q + 1)];
                    for (int i = 0; i < Q; ++i) o += md[tid * (Q + 1) + 1 + i] * ((double)zg[i * plane + idx] - (double)s_sh[i]);
                    const float of = (float)(o + (double)s_sh[Q + tid]);
                    a.out[tid * plane + idx] = of;
                    dbad += !isfinite(of);
                }
            } else {
                const int wd = 2 * rc + 1;
                for (int t = tid; t < wd * wd; t += kFixThreads) {
                    const int yy = py - rc + t / wd, xx = px - rc + t % wd;
                    if (yy < y0 || yy >= y1 || xx < x0 || xx >= x1) continue;
                    const size_t off = (size_t)yy * W + xx;
                    const float my = (float)(min(yy + rc, H - 1) - max(yy - rc, 0) + 1);
                    const float mx = (float)(min(xx + rc, W - 1) - max(xx - rc, 0) + 1);
                    double zz[Q];
                    for (int i = 0; i < Q; ++i) zz[i] = (double)__ldg(zg + i * plane + off) - (double)s_sh[i];
                    for (int c = 0; c < 3; ++c) {
                        double o = md[c * (Q + 1)];
                        for (int i = 0; i < Q; ++i) o += md[c * (Q + 1) + 1 + i] * zz[i];
                        const float old = a.out[c * plane + off];
                        const float nw = (float)((double)old + o / ((double)my * (double)mx));
                        a.out[c * plane + off] = nw;
                        dbad += (long long)!isfinite(nw) - (long long)!isfinite(old);
                    }
                }
            }
            __syncthreads();
        }
    }
    atomicAdd(&s_cnt[0], (unsigned long long)own);
    if (dbad != 0) atomicAdd(&s_cnt[1], (unsigned long long)dbad);  // two's complement sum
    __syncthreads();
    if (tid == 0) {
        if (a.flag_count) atomicAdd(a.flag_count, s_cnt[0]);
        if (a.nonfinite && s_cnt[1]) atomicAdd(a.nonfinite, s_cnt[1]);
    }
}

// ---- host side -------------------------------------------------------------------------
template <int Q, int R, int RC>
cudaError_t prepare_qr()
{
    return cudaFuncSetAttribute(flr_fused_kernel<Q, R, RC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)Geo<Q, R, RC>::SMEM);
}

template <int Q, int R, int RC>
cudaError_t launch_qr(const FusedArgs &a, dim3 grid, cudaStream_t st)
{
    using G = Geo<Q, R, RC>;
    static std::mutex mu;
    static bool ready[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (!ready[dev]) {  // this kernel instance always asks for the same shared memory
            e = prepare_qr<Q, R, RC>();
            if (e != cudaSuccess) return e;
            ready[dev] = true;
        }
    }
    KArgs ka;
    std::memset(&ka, 0, sizeof(ka));
    ka.a = a;
    if (tma::encode_planes_f32(&ka.tg, a.guide, a.W, a.H, Q, G::WSt, kB, Q) != cudaSuccess ||
        tma::encode_planes_f32(&ka.tr, a.rad, a.W, a.H, 3, G::WSt, kB, 3) != cudaSuccess ||
        tma::encode_planes_f32(&ka.tz, a.map_guide ? a.map_guide : a.guide, a.W, a.H, Q, G::TW, kB, Q) !=
            cudaSuccess)
        return cudaErrorInvalidValue;
    flr_fused_kernel<Q, R, RC><<<grid, kThreads, G::SMEM, st>>>(ka);
    return cudaGetLastError();
}

}  // namespace fused

// Radii of the fused kernel (compile-time instances): the 1080p workload (r = rc = 8), the
// 256 x 256 workload (r = rc = 5) and r = 8 without averaging; Q = 8.
bool fused_supported(int q, int r, int rc)
{
    return q == 8 && ((r == 8 && (rc == 8 || rc == 0)) || (r == 5 && rc == 5));
}

int fused_tile_width(int rc) { return fused::tile_width(rc); }

cudaError_t launch_fused(int q, const FusedArgs &a, dim3 grid, cudaStream_t st)
{
    if (q == 8) {
        if (a.r == 8 && a.rc == 8) return fused::launch_qr<8, 8, 8>(a, grid, st);
        if (a.r == 8 && a.rc == 0) return fused::launch_qr<8, 8, 0>(a, grid, st);
        if (a.r == 5 && a.rc == 5) return fused::launch_qr<8, 5, 5>(a, grid, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_fused_fix(int q, const FusedArgs &a, dim3 grid, cudaStream_t st)
{
    if (q != 8) return cudaErrorInvalidValue;
    fused::flr_fused_fix_kernel<8><<<grid, fused::kFixThreads, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace flr
