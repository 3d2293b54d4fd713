// flnr.cu -- the FLNR guide network (Sec. 3.3) on sm_103a: BF16 implicit-GEMM convolutions
// with FP32 accumulation on the fifth-generation tensor cores (tcgen05, accumulators in
// tensor memory) for the forward pass and for training -- input gradients as convolutions
// with rotated, transposed weights on the forward's TMA-staged kernel, weight gradients as
// one GEMM over pixels per layer with the operands transposed on chip -- Adam on FP32
// master weights, and the flnr_* entry points of include/flr.h.
//
// Network (weights and order as oracle/flnr_ref.py): 11 inputs (8 guides + noisy RGB)
//   in0 3x3 11->16 ReLU, in1 1x1 16->16 ReLU                                   f0 (H)
//   e1a 3x3 16->32 ReLU, e1b 3x3 32->32 stride 2 ReLU                          f1 (H/2)
//   e2a 3x3 32->64 ReLU, e2b 3x3 64->64 stride 2 ReLU                          f2 (H/4)
//   up(f2) ++ f1, d1a 3x3 96->32 ReLU, d1b 3x3 32->32 ReLU                     d1 (H/2)
//   up(d1) ++ f0, d0a 3x3 48->16 ReLU, d0b 3x3 16->16 ReLU                     d0 (H)
//   o0 3x3 16->16 ReLU, o1 1x1 16->8, sigmoid                                  X' (8 ch)
// Activations are NHWC BF16 (channels innermost; the 11 inputs padded to 16, the 8 outputs
// of o1 computed as 16 with zero weights); the enhanced guides leave as planar FP32 for FLR.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "flr.h"

namespace flnr {
namespace {

typedef __nv_bfloat16 bf16;

constexpr int kNL = 12;
struct LayerDef {
    int cin, cout, k, relu;  // true sizes (o1's cout is 8)
};
constexpr LayerDef kLayers[kNL] = {
    {11, 16, 3, 1}, {16, 16, 1, 1}, {16, 32, 3, 1}, {32, 32, 3, 1}, {32, 64, 3, 1}, {64, 64, 3, 1},
    {96, 32, 3, 1}, {32, 32, 3, 1}, {48, 16, 3, 1}, {16, 16, 3, 1}, {16, 16, 3, 1}, {16, 8, 1, 0}};
__host__ __device__ constexpr int pad16(int c) { return (c + 15) / 16 * 16; }

// ---------------------------------------------------------------------------------------
// Asynchronous 16-byte global -> shared copies (zero fill when !valid).
__device__ __forceinline__ void cp_async16(void *dst, const void *src, bool valid)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 16 : 0));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// Arguments of the convolution kernels (stride 1, zero padding KS/2, implicit GEMM on the
// tensor cores).  x [N][H][W][CIN] bf16, w [taps][COUT][CIN] bf16, bias [COUT] fp32.  The
// kernels' template parameters select the epilogue:
//   OUTM 0 -> y [N][H][W][ystride] bf16 at channel offset 0 (ACT 1 = ReLU);
//   OUTM 1 -> yf planar fp32 [N][8][H][W], sigmoid of channels 0..7;
//   MASK   -> the result times (mask > 0), mask [N][H][W][COUT] bf16 (the ReLU of the
//             layer input, for input gradients);
// The decoder kernel reads x as the half-resolution map [N][H/2][W/2][CA] and x2 as the
// skip [N][H][W][CIN-CA] of the concatenated input up2(x) ++ x2.
struct ConvArgs {
    const bf16 *x, *w, *mask;
    const float *bias;
    bf16 *y;
    float *yf;
    int N, H, W, ystride;
    int nbias;  // valid bias entries (the true output channels); 0 without bias
    const bf16 *x2;
    int *status;  // tensor-core path: set to FLNR_STATUS_TIMEOUT if a completion wait ran out
};

// ---------------------------------------------------------------------------------------
// The same convolution on the fifth-generation tensor cores (tcgen05): BF16 operands in shared
// memory, FP32 accumulators in tensor memory (TMEM).
//
// A tile is 16 rows x 8 pixels = the M = 128 rows of one UMMA.  The input tile (with halo) is
// staged as [channel chunk c8][row][col][8 channels], so 8 consecutive pixels of one row and
// one 8-channel chunk form a contiguous 128-byte core matrix.  For tap (ky, kx) the operand A
// (128 output pixels x 16 channels) is then the no-swizzle K-major layout starting at pixel
// (ky, kx) of chunk 2kk: 8-row groups (output rows) SW * 16 bytes apart, the two K halves
// (chunks 2kk, 2kk + 1) SH * SW * 16 bytes apart.  No im2col copy is made.  The weights are
// staged once per CTA as [tap][c8][COUT][8]: operand B (COUT x 16, K-major) has 8-row groups
// 128 bytes apart and K halves COUT * 16 bytes apart.  One thread issues the taps x CIN/16
// MMAs of a tile and commits them to an mbarrier; four warps then read the accumulator rows of
// their TMEM lane quarter (one output pixel per thread) and run the epilogue, while the next
// tiles' inputs are already loading.  Every wait is bounded by the global timer.
#define FLNR_STATUS_TIMEOUT 1
constexpr unsigned long long kTcTimeoutNs = 1000000000ull;  // 1 s per wait

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// shared-memory matrix descriptor: no swizzle, K-major; LBO = distance between the two K
// halves of a core-matrix pair, SBO = distance between 8-row groups
__device__ __forceinline__ uint64_t umma_sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor, kind::f16: D FP32, A and B BF16, both K-major, M = 128, N = n
__host__ __device__ constexpr uint32_t umma_idesc(int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// bounded wait for the mbarrier phase with the given parity, polled by lane 0 of the warp
// (try_wait suspends the thread for up to 20 us per call); false if it ran out
__device__ __forceinline__ bool mbar_wait_warp(uint32_t mbar, uint32_t parity)
{
    uint32_t ok = 1;
    if ((threadIdx.x & 31) == 0) {
        const unsigned long long t0 = global_ns();
        for (;;) {
            uint32_t done;
            asm volatile(
                "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, 20000;\nselp.u32 %0, 1, 0, p;\n}\n"
                : "=r"(done)
                : "r"(mbar), "r"(parity)
                : "memory");
            if (done) break;
            if (global_ns() - t0 > kTcTimeoutNs) {
                ok = 0;
                break;
            }
        }
    }
    return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

template <int N>
constexpr int tmem_cols()
{
    return N <= 32 ? 32 : N <= 64 ? 64 : N <= 128 ? 128 : 256;
}

// Kernel parameters: the tensor map (4-D: channels, W, H, N) of the operand that TMA stages
// (x, or the skip x2 of a decoder layer) and the convolution arguments.
struct alignas(128) TcArgs {
    CUtensorMap tm;
    ConvArgs c;
};

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *tm, int c0, int c1, int c2, int c3,
                                            uint32_t mbar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];\n" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(mbar)
        : "memory");
}

// single-thread bounded wait on an mbarrier phase (the TMA issuer)
__device__ __forceinline__ bool mbar_wait_thread(uint32_t mbar, uint32_t parity)
{
    const unsigned long long t0 = global_ns();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, 20000;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
        if (global_ns() - t0 > kTcTimeoutNs) return false;
    }
}

// Epilogue pieces shared by the tensor-core kernels.  tc_load_acc: one accumulator row (an
// output pixel) from the warp's TMEM lane quarter, COUT columns from `taddr` on.
template <int COUT>
__device__ __forceinline__ void tc_load_acc(uint32_t taddr, float (&v)[COUT])
{
#pragma unroll
    for (int c0 = 0; c0 < COUT; c0 += 16) {
        float q[16];
        tmem_ld16(taddr + (uint32_t)c0, q);
#pragma unroll
        for (int i = 0; i < 16; ++i) v[c0 + i] = q[i];
    }
    asm volatile("tcgen05.wait::ld.sync.aligned;\n");
    asm volatile("tcgen05.fence::before_thread_sync;\n");
}

// tc_store: bias, activation, optional ReLU mask, then bf16 NHWC stores, or sigmoid into
// planar fp32 (OUTM 1).  (n, yy, xx): the output pixel of an [N][a.H][a.W] map.
template <int COUT, int ACT, int OUTM, bool MASK>
__device__ __forceinline__ void tc_store(const ConvArgs &a, float (&v)[COUT], const float (&bias)[COUT], int n,
                                         int yy, int xx)
{
    const bool in = yy < a.H && xx < a.W;
    const size_t pix = ((size_t)n * a.H + yy) * a.W + xx;
#pragma unroll
    for (int c = 0; c < COUT; ++c) {
        v[c] += bias[c];
        if (ACT == 1) v[c] = fmaxf(v[c], 0.f);
    }
    if (MASK && in) {
#pragma unroll
        for (int c8 = 0; c8 < COUT / 8; ++c8) {
            const uint4 m = *reinterpret_cast<const uint4 *>(a.mask + pix * COUT + c8 * 8);
            const __nv_bfloat162 *mh = reinterpret_cast<const __nv_bfloat162 *>(&m);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if (!(__bfloat162float(mh[i].x) > 0.f)) v[c8 * 8 + 2 * i] = 0.f;
                if (!(__bfloat162float(mh[i].y) > 0.f)) v[c8 * 8 + 2 * i + 1] = 0.f;
            }
        }
    }
    if (OUTM == 0) {
#pragma unroll
        for (int c8 = 0; c8 < COUT / 8; ++c8) {
            uint4 o;
            __nv_bfloat162 *oh = reinterpret_cast<__nv_bfloat162 *>(&o);
#pragma unroll
            for (int i = 0; i < 4; ++i) oh[i] = __floats2bfloat162_rn(v[c8 * 8 + 2 * i], v[c8 * 8 + 2 * i + 1]);
            if (in) *reinterpret_cast<uint4 *>(a.y + pix * a.ystride + c8 * 8) = o;
        }
    } else if (in) {
        const size_t hw = (size_t)a.H * a.W, off = (size_t)yy * a.W + xx;
#pragma unroll
        for (int c = 0; c < COUT; ++c)  // a.nbias planes: the head's true outputs
            if (c < a.nbias) a.yf[((size_t)n * a.nbias + c) * hw + off] = 1.f / (1.f + expf(-v[c]));
    }
}

// ---------------------------------------------------------------------------------------
// Warp-specialised tensor-core convolution (layers whose input is one tensor): no CTA-wide
// barrier in the main loop.  Warp 4 (one lane) is the producer: it loads tile j into ring
// stage j % NBUF with one TMA box copy per channel chunk once the MMAs of tile j - NBUF have
// released the stage.  Warp 5 (one lane) issues tile j's MMAs into accumulator j & 1 once the
// stage has landed and the epilogue has drained that accumulator, then commits them to the
// stage's "empty" barrier and the accumulator's "full" barrier.  Warps 0-3 read the
// accumulator rows of their TMEM lane quarter, release the accumulator, and run the epilogue.
// The tile geometry and operand layouts are those described above.  Every wait is bounded.
template <int CIN, int COUT, int KS>
struct WsGeom {
    static constexpr int TH = 16, TW = 8, P = KS / 2, SH = TH + 2 * P, SW = TW + 2 * P, C8 = CIN / 8;
    static constexpr int NBUF = 4;
    static constexpr int PS = (SH * SW * 16 + 127) / 128 * 128;
    static constexpr int XBYTES = C8 * PS;
    static constexpr int WBYTES = (KS * KS * C8 * COUT * 16 + 127) / 128 * 128;
    static constexpr int TMA_BYTES = C8 * SH * SW * 16;
    static constexpr int NBAR = 2 * NBUF + 4;  // full[NBUF], empty[NBUF], accf[2], acce[2]
    static constexpr int SMEM = 128 + WBYTES + NBUF * XBYTES + NBAR * 8 + 16;
    static constexpr int COLS = tmem_cols<2 * COUT>();
};
constexpr int kWsThreads = 192;

template <int CIN, int COUT, int KS, int ACT, int OUTM, bool MASK = false>
__global__ void __launch_bounds__(kWsThreads) conv_ws_kernel(const __grid_constant__ TcArgs args)
{
    using G = WsGeom<CIN, COUT, KS>;
    constexpr int TH = G::TH, TW = G::TW, P = G::P, SW = G::SW, C8 = G::C8, NBUF = G::NBUF, PS = G::PS;
    static_assert(CIN % 16 == 0 && COUT % 16 == 0 && 2 * COUT <= 256, "UMMA shape");
    const ConvArgs &a = args.c;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *base = smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);
    unsigned char *sw = base;
    unsigned char *sx0 = base + G::WBYTES;
    uint64_t *full = reinterpret_cast<uint64_t *>(sx0 + NBUF * G::XBYTES);
    uint64_t *empty = full + NBUF, *accf = empty + NBUF, *acce = accf + 2;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(acce + 2);
    __shared__ int s_issued, s_consumed;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tiles_x = (a.W + TW - 1) / TW, tiles_y = (a.H + TH - 1) / TH;
    const int per_img = tiles_x * tiles_y, ntiles = a.N * per_img;
    const int mine = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                     "r"(G::COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid == 0) {
        for (int i = 0; i < NBUF; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(full + i)));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(empty + i)));
        }
        for (int i = 0; i < 2; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(accf + i)));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;\n" ::"r"(smem_u32(acce + i)));  // 4 epilogue warps
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n");
        asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&args.tm)) : "memory");
        s_issued = 0;
        s_consumed = 0;
    }
    for (int i = tid; i < KS * KS * COUT * C8; i += kWsThreads) {
        const int c8 = i % C8, row = i / C8, tap = row / COUT, co = row % COUT;
        cp_async16(sw + ((tap * C8 + c8) * COUT + co) * 16, a.w + (size_t)row * CIN + c8 * 8, true);
    }
    cp_async_commit();
    cp_async_wait<0>();
    asm volatile("fence.proxy.async.shared::cta;\n");  // weights visible to the tensor core
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    const uint32_t tmem = *tslot;
    auto fail = [&]() {
        if (a.status) atomicExch(a.status, FLNR_STATUS_TIMEOUT);
    };
    auto origin = [&](int j, int &n, int &ty0, int &tx0) {
        const int t = blockIdx.x + j * gridDim.x;
        n = t / per_img;
        const int r = t % per_img;
        ty0 = (r / tiles_x) * TH;
        tx0 = (r % tiles_x) * TW;
    };

    if (warp == 4) {
        if (lane == 0) {  // producer
            for (int j = 0; j < mine; ++j) {
                const int st = j % NBUF;
                if (j >= NBUF && !mbar_wait_thread(smem_u32(empty + st), (uint32_t)((j / NBUF - 1) & 1))) {
                    fail();
                    break;
                }
                int n, ty0, tx0;
                origin(j, n, ty0, tx0);
                const uint32_t bar = smem_u32(full + st);
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(G::TMA_BYTES) : "memory");
                const uint32_t dst = smem_u32(sx0 + st * G::XBYTES);
#pragma unroll
                for (int k = 0; k < C8; ++k) tma_load_4d(dst + k * PS, &args.tm, k * 8, tx0 - P, ty0 - P, n, bar);
                s_issued = j + 1;
            }
        }
    } else if (warp == 5) {
        if (lane == 0) {  // MMA issuer
            constexpr uint32_t idesc = umma_idesc(COUT);
            const uint64_t adesc0 = umma_sdesc(smem_u32(sx0), PS, SW * 16);
            const uint64_t bdesc0 = umma_sdesc(smem_u32(sw), COUT * 16, 128);
            for (int j = 0; j < mine; ++j) {
                const int st = j % NBUF, acc = j & 1;
                if (!mbar_wait_thread(smem_u32(full + st), (uint32_t)((j / NBUF) & 1))) {
                    fail();
                    break;
                }
                s_consumed = j + 1;
                if (j >= 2 && !mbar_wait_thread(smem_u32(acce + acc), (uint32_t)((j / 2 - 1) & 1))) {
                    fail();
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;\n");
                const uint64_t ab = adesc0 + (uint64_t)((st * G::XBYTES) >> 4);
                const uint32_t d = tmem + (uint32_t)(acc * COUT);
#pragma unroll
                for (int tap = 0; tap < KS * KS; ++tap) {
#pragma unroll
                    for (int kk = 0; kk < C8 / 2; ++kk) {
                        const uint32_t aoff = (uint32_t)((2 * kk * PS + ((tap / KS) * SW + tap % KS) * 16) >> 4);
                        const uint32_t boff = (uint32_t)(((tap * C8 + 2 * kk) * COUT * 16) >> 4);
                        umma_bf16(d, ab + aoff, bdesc0 + boff, idesc, (tap | kk) ? 1u : 0u);
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                    smem_u32(empty + st)));
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                    smem_u32(accf + acc)));
            }
        }
    } else {  // epilogue warps 0-3: TMEM lane quarter = warp
        float bias[COUT];
#pragma unroll
        for (int c = 0; c < COUT; ++c) bias[c] = c < a.nbias ? a.bias[c] : 0.f;
        for (int j = 0; j < mine; ++j) {
            const int acc = j & 1;
            if (!mbar_wait_warp(smem_u32(accf + acc), (uint32_t)((j / 2) & 1))) {
                if (lane == 0) fail();
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;\n");
            float v[COUT];
            tc_load_acc<COUT>(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(acc * COUT), v);
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(acce + acc)) : "memory");
            int n, ty0, tx0;
            origin(j, n, ty0, tx0);
            tc_store<COUT, ACT, OUTM, MASK>(a, v, bias, n, ty0 + 4 * warp + (lane >> 3), tx0 + (lane & 7));
        }
    }
    __syncwarp();  // the single-lane roles rejoin their warps before the CTA barrier
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    if (tid == 4 * 32) {  // after a failure: let copies still in flight land before the CTA exits
        for (int j = s_consumed; j < s_issued; ++j) mbar_wait_thread(smem_u32(full + j % NBUF), (uint32_t)((j / NBUF) & 1));
    }
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(G::COLS));
    }
}

// ---------------------------------------------------------------------------------------
// Two layers in one pass: a KS x KS convolution (ReLU) followed by a 1x1 convolution of its
// output (in1 after in0, o1 after o0).  The first layer's tile never reaches HBM: the
// epilogue warps write its bias + ReLU + bfloat16 values into shared memory as the K-major
// A operand of the 1x1 MMA ([chunk][128 pixels][8 channels]), the MMA lane issues that one
// MMA into a second pair of accumulators, and the epilogue warps finish the tile from it
// (ReLU and BF16 for in1, sigmoid into planar FP32 for o1).  Roles as
// conv_ws_kernel; the MMA lane issues tile j's convolution, then tile j - 1's 1x1.
// Barriers: full/empty per input stage, accf/acce per first accumulator, a2full (the A
// operand of the 1x1 written, four epilogue warps), acc2f (1x1 committed) and acc2e (its
// accumulator drained, four warps), all per accumulator slot j & 1.
struct alignas(128) TailArgs {
    CUtensorMap tm;
    ConvArgs c;   // first layer: x, w, bias, nbias, N, H, W, status; y (may be NULL), ystride
    ConvArgs c2;  // 1x1 layer: w, bias, nbias, N, H, W and the outputs (y, ystride / yf)
};

template <int CIN, int COUT, int KS, int COUT2>
struct TailGeom {
    using G1 = WsGeom<CIN, COUT, KS>;
    static constexpr int NBUF = G1::NBUF;
    static constexpr int A2BYTES = (COUT / 8) * 128 * 16;             // one 1x1 A operand
    static constexpr int W2BYTES = ((COUT / 8) * COUT2 * 16 + 127) / 128 * 128;
    static constexpr int NBAR = 2 * NBUF + 10;  // full, empty, accf, acce, a2full, acc2f, acc2e
    static constexpr int SMEM = 128 + G1::WBYTES + W2BYTES + NBUF * G1::XBYTES + 2 * A2BYTES + NBAR * 8 + 16;
    static constexpr int COLS = tmem_cols<2 * COUT + 2 * COUT2>();
};

template <int CIN, int COUT, int KS, int COUT2, int ACT2, int OUTM2>
__global__ void __launch_bounds__(kWsThreads) conv_tail_kernel(const __grid_constant__ TailArgs args)
{
    using T = TailGeom<CIN, COUT, KS, COUT2>;
    using G = typename T::G1;
    constexpr int TH = G::TH, TW = G::TW, P = G::P, SW = G::SW, C8 = G::C8, NBUF = G::NBUF, PS = G::PS;
    static_assert(CIN % 16 == 0 && COUT % 16 == 0 && COUT2 % 16 == 0 && 2 * COUT + 2 * COUT2 <= 256, "UMMA shape");
    const ConvArgs &a = args.c;
    const ConvArgs &a2 = args.c2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *base = smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);
    unsigned char *sw = base;
    unsigned char *sw2 = sw + G::WBYTES;
    unsigned char *sa2 = sw2 + T::W2BYTES;                   // [2][COUT/8][128][8] 1x1 A operands
    unsigned char *sx0 = sa2 + 2 * T::A2BYTES;
    uint64_t *full = reinterpret_cast<uint64_t *>(sx0 + NBUF * G::XBYTES);
    uint64_t *empty = full + NBUF, *accf = empty + NBUF, *acce = accf + 2;
    uint64_t *a2full = acce + 2, *acc2f = a2full + 2, *acc2e = acc2f + 2;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(acc2e + 2);
    __shared__ int s_issued, s_consumed;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tiles_x = (a.W + TW - 1) / TW, tiles_y = (a.H + TH - 1) / TH;
    const int per_img = tiles_x * tiles_y, ntiles = a.N * per_img;
    const int mine = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                     "r"(T::COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid == 0) {
        for (int i = 0; i < NBUF; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(full + i)));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(empty + i)));
        }
        for (int i = 0; i < 2; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(accf + i)));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;\n" ::"r"(smem_u32(acce + i)));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;\n" ::"r"(smem_u32(a2full + i)));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(acc2f + i)));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;\n" ::"r"(smem_u32(acc2e + i)));
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n");
        asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&args.tm)) : "memory");
        s_issued = 0;
        s_consumed = 0;
    }
    for (int i = tid; i < KS * KS * COUT * C8; i += kWsThreads) {
        const int c8 = i % C8, row = i / C8, tap = row / COUT, co = row % COUT;
        cp_async16(sw + ((tap * C8 + c8) * COUT + co) * 16, a.w + (size_t)row * CIN + c8 * 8, true);
    }
    for (int i = tid; i < COUT2 * (COUT / 8); i += kWsThreads) {  // 1x1 weights [COUT2][COUT] -> [c8][COUT2][8]
        const int c8 = i % (COUT / 8), co = i / (COUT / 8);
        cp_async16(sw2 + (c8 * COUT2 + co) * 16, a2.w + (size_t)co * COUT + c8 * 8, true);
    }
    cp_async_commit();
    cp_async_wait<0>();
    asm volatile("fence.proxy.async.shared::cta;\n");  // weights visible to the tensor core
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    const uint32_t tmem = *tslot;
    const uint32_t tmem2 = tmem + (uint32_t)(2 * COUT);  // the 1x1 accumulators
    auto fail = [&]() {
        if (a.status) atomicExch(a.status, FLNR_STATUS_TIMEOUT);
    };
    auto origin = [&](int j, int &n, int &ty0, int &tx0) {
        const int t = blockIdx.x + j * gridDim.x;
        n = t / per_img;
        const int r = t % per_img;
        ty0 = (r / tiles_x) * TH;
        tx0 = (r % tiles_x) * TW;
    };

    if (warp == 4) {
        if (lane == 0) {  // producer
            for (int j = 0; j < mine; ++j) {
                const int st = j % NBUF;
                if (j >= NBUF && !mbar_wait_thread(smem_u32(empty + st), (uint32_t)((j / NBUF - 1) & 1))) {
                    fail();
                    break;
                }
                int n, ty0, tx0;
                origin(j, n, ty0, tx0);
                const uint32_t bar = smem_u32(full + st);
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(G::TMA_BYTES) : "memory");
                const uint32_t dst = smem_u32(sx0 + st * G::XBYTES);
#pragma unroll
                for (int k = 0; k < C8; ++k) tma_load_4d(dst + k * PS, &args.tm, k * 8, tx0 - P, ty0 - P, n, bar);
                s_issued = j + 1;
            }
        }
    } else if (warp == 5) {
        if (lane == 0) {  // MMA issuer
            constexpr uint32_t idesc = umma_idesc(COUT), idesc2 = umma_idesc(COUT2);
            const uint64_t adesc0 = umma_sdesc(smem_u32(sx0), PS, SW * 16);
            const uint64_t bdesc0 = umma_sdesc(smem_u32(sw), COUT * 16, 128);
            const uint64_t a2desc0 = umma_sdesc(smem_u32(sa2), 128 * 16, 128);
            const uint64_t b2desc0 = umma_sdesc(smem_u32(sw2), COUT2 * 16, 128);
            // the 1x1 of tile t: its A operand written, its accumulator slot drained
            auto tail = [&](int t) -> bool {
                const int sl = t & 1;
                if (!mbar_wait_thread(smem_u32(a2full + sl), (uint32_t)((t >> 1) & 1))) return false;
                if (t >= 2 && !mbar_wait_thread(smem_u32(acc2e + sl), (uint32_t)(((t >> 1) - 1) & 1))) return false;
                asm volatile("tcgen05.fence::after_thread_sync;\n");
                const uint32_t d = tmem2 + (uint32_t)(sl * COUT2);
                const uint64_t ab = a2desc0 + (uint64_t)((sl * T::A2BYTES) >> 4);
#pragma unroll
                for (int kk = 0; kk < COUT / 16; ++kk)
                    umma_bf16(d, ab + (uint64_t)((2 * kk * 128 * 16) >> 4), b2desc0 + (uint64_t)((2 * kk * COUT2 * 16) >> 4),
                              idesc2, kk ? 1u : 0u);
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                    smem_u32(acc2f + sl)));
                return true;
            };
            bool ok = true;
            for (int j = 0; j < mine && ok; ++j) {
                const int st = j % NBUF, acc = j & 1;
                if (!mbar_wait_thread(smem_u32(full + st), (uint32_t)((j / NBUF) & 1))) {
                    ok = false;
                    break;
                }
                s_consumed = j + 1;
                if (j >= 2 && !mbar_wait_thread(smem_u32(acce + acc), (uint32_t)((j / 2 - 1) & 1))) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;\n");
                const uint64_t ab = adesc0 + (uint64_t)((st * G::XBYTES) >> 4);
                const uint32_t d = tmem + (uint32_t)(acc * COUT);
#pragma unroll
                for (int tap = 0; tap < KS * KS; ++tap) {
#pragma unroll
                    for (int kk = 0; kk < C8 / 2; ++kk) {
                        const uint32_t aoff = (uint32_t)((2 * kk * PS + ((tap / KS) * SW + tap % KS) * 16) >> 4);
                        const uint32_t boff = (uint32_t)(((tap * C8 + 2 * kk) * COUT * 16) >> 4);
                        umma_bf16(d, ab + aoff, bdesc0 + boff, idesc, (tap | kk) ? 1u : 0u);
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                    smem_u32(empty + st)));
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                    smem_u32(accf + acc)));
                if (j >= 1) ok = tail(j - 1);
            }
            if (ok && mine > 0) ok = tail(mine - 1);
            if (!ok) fail();
        }
    } else {  // epilogue warps 0-3: TMEM lane quarter = warp; row 32w + l = pixel (4w + l/8, l%8)
        float bias[COUT], bias2[COUT2];
#pragma unroll
        for (int c = 0; c < COUT; ++c) bias[c] = c < a.nbias ? a.bias[c] : 0.f;
#pragma unroll
        for (int c = 0; c < COUT2; ++c) bias2[c] = c < a2.nbias ? a2.bias[c] : 0.f;
        const int m = 32 * warp + lane;
        for (int j = 0; j < mine; ++j) {
            const int acc = j & 1;
            if (!mbar_wait_warp(smem_u32(accf + acc), (uint32_t)((j / 2) & 1))) {
                if (lane == 0) fail();
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;\n");
            float v[COUT];
            tc_load_acc<COUT>(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(acc * COUT), v);
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(acce + acc)) : "memory");
            int n, ty0, tx0;
            origin(j, n, ty0, tx0);
            const int yy = ty0 + 4 * warp + (lane >> 3), xx = tx0 + (lane & 7);
            const bool in = yy < a.H && xx < a.W;
            const size_t pix = ((size_t)n * a.H + yy) * a.W + xx;
            // first layer's bias + ReLU, rounded to bfloat16: the 1x1's A operand row m, and
            // (when a.y is set) the first layer's stored output, which the backward pass reads
            unsigned char *arow = sa2 + acc * T::A2BYTES + m * 16;
#pragma unroll
            for (int c8 = 0; c8 < COUT / 8; ++c8) {
                uint4 o;
                __nv_bfloat162 *oh = reinterpret_cast<__nv_bfloat162 *>(&o);
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    oh[i] = __floats2bfloat162_rn(fmaxf(v[c8 * 8 + 2 * i] + bias[c8 * 8 + 2 * i], 0.f),
                                                  fmaxf(v[c8 * 8 + 2 * i + 1] + bias[c8 * 8 + 2 * i + 1], 0.f));
                *reinterpret_cast<uint4 *>(arow + c8 * 128 * 16) = o;
                if (a.y && in) *reinterpret_cast<uint4 *>(a.y + pix * a.ystride + c8 * 8) = o;
            }
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // visible to the tensor core
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(a2full + acc)) : "memory");
            if (!mbar_wait_warp(smem_u32(acc2f + acc), (uint32_t)((j / 2) & 1))) {
                if (lane == 0) fail();
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;\n");
            float v2[COUT2];
            tc_load_acc<COUT2>(tmem2 + ((uint32_t)(32 * warp) << 16) + (uint32_t)(acc * COUT2), v2);
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(acc2e + acc)) : "memory");
            tc_store<COUT2, ACT2, OUTM2, false>(a2, v2, bias2, n, yy, xx);
        }
    }
    __syncwarp();  // the single-lane roles rejoin their warps before the CTA barrier
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    if (tid == 4 * 32) {  // after a failure: let copies still in flight land before the CTA exits
        for (int j = s_consumed; j < s_issued; ++j) mbar_wait_thread(smem_u32(full + j % NBUF), (uint32_t)((j / NBUF) & 1));
    }
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(T::COLS));
    }
}

// ---------------------------------------------------------------------------------------
// Decoder convolution (3x3, ReLU) on up2(lo) ++ skip without forming the upsampled map.
// A stage covers 32 x 16 output pixels: a 16 x 8 block of low-resolution positions (i0 + g,
// j0 + r) and its four parity classes (a, b), output pixel (2(i0 + g) + a, 2(j0 + r) + b),
// one 128-row accumulator per class (row 8g + r).  For tap (dy, dx), t = a + dy - 1 and
// u = b + dx - 1, every pixel of class (a, b) reads the low-resolution map at
// (i0 + g + t/2, j0 + r + u/2) (floor division) and the skip at full-resolution pixel
// (2(i0 + g + t/2) + (t mod 2), 2(j0 + r + u/2) + (u mod 2)).  Rows of a class step by one
// low-resolution position in both operands, so both are plain K-major tiles:
//   lo    CA/8 planes [18][10][8] (rows i0 - 1 .. i0 + 16, columns j0 - 1 .. j0 + 8), one TMA
//         box copy each;
//   skip  its four parity planes (a', b') x CB/8 chunks [18][10][8] (rows i0 - 1 .. i0 + 16
//         of row parity a', columns j0 - 1 .. j0 + 8 of column parity b'), one TMA box copy
//         each from a 5-D view (channels of a column pair, column pairs, row parity, row
//         pairs, images) in which the start channel b' * CB + 8k selects the column parity.
// The products are those of the convolution on the concatenated map; only their order of
// accumulation differs.  Roles and waits as conv_ws_kernel; the MMA lane issues the four
// classes of a stage into one of two accumulator sets (4 * COUT columns each).
template <int CA, int CB, int COUT, int NBUF>
struct UpGeom {
    static constexpr int SH = 18, SW = 10;                       // staged rows and columns
    static constexpr int PS = (SH * SW * 16 + 127) / 128 * 128;  // one chunk plane [SH][SW][8]
    static constexpr int CA8 = CA / 8, CB8 = CB / 8, C8 = CA8 + CB8;
    static constexpr int PLANES = CA8 + 4 * CB8;                 // lo chunks, then skip (a', b', chunk)
    static constexpr int XBYTES = PLANES * PS;
    static constexpr int TMA_BYTES = PLANES * SH * SW * 16;
    static constexpr int WBYTES = (9 * C8 * COUT * 16 + 127) / 128 * 128;
    static constexpr int NBAR = 2 * NBUF + 4;
    static constexpr int SMEM = 128 + WBYTES + NBUF * XBYTES + NBAR * 8 + 16;
    static constexpr int COLS = tmem_cols<8 * COUT>();          // two sets of four class accumulators
};

struct alignas(128) UpArgs {
    CUtensorMap tlo, tskip;
    ConvArgs c;  // x = lo [N][H/2][W/2][CA], x2 = skip [N][H][W][CB], H and W even
};

__device__ __forceinline__ void tma_load_5d(uint32_t dst, const CUtensorMap *tm, int c0, int c1, int c2, int c3,
                                            int c4, uint32_t mbar)
{
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, %6}], [%7];\n" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(mbar)
        : "memory");
}

template <int CA, int CB, int COUT, int NBUF>
__global__ void __launch_bounds__(kWsThreads) conv_up_kernel(const __grid_constant__ UpArgs args)
{
    using G = UpGeom<CA, CB, COUT, NBUF>;
    constexpr int PS = G::PS, SW = G::SW, CA8 = G::CA8, CB8 = G::CB8, C8 = G::C8;
    static_assert(CA % 16 == 0 && CB % 16 == 0 && COUT % 16 == 0 && 8 * COUT <= 256, "UMMA shape");
    const ConvArgs &a = args.c;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *base = smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);
    unsigned char *sw = base;
    unsigned char *sx0 = base + G::WBYTES;
    uint64_t *full = reinterpret_cast<uint64_t *>(sx0 + NBUF * G::XBYTES);
    uint64_t *empty = full + NBUF, *accf = empty + NBUF, *acce = accf + 2;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(acce + 2);
    __shared__ int s_issued, s_consumed;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int HL = a.H / 2, WL = a.W / 2;
    const int tiles_x = (WL + 7) / 8, tiles_y = (HL + 15) / 16;
    const int per_img = tiles_x * tiles_y, ntiles = a.N * per_img;
    const int mine = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                     "r"(G::COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid == 0) {
        for (int i = 0; i < NBUF; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(full + i)));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(empty + i)));
        }
        for (int i = 0; i < 2; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(accf + i)));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;\n" ::"r"(smem_u32(acce + i)));  // 4 epilogue warps
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n");
        asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&args.tlo)) : "memory");
        asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&args.tskip)) : "memory");
        s_issued = 0;
        s_consumed = 0;
    }
    // weights: global [tap][COUT][CA + CB] -> shared [tap][c8][COUT][8] (lo chunks first)
    for (int i = tid; i < 9 * COUT * C8; i += kWsThreads) {
        const int c8 = i % C8, row = i / C8, tap = row / COUT, co = row % COUT;
        cp_async16(sw + ((tap * C8 + c8) * COUT + co) * 16, a.w + (size_t)row * (CA + CB) + c8 * 8, true);
    }
    cp_async_commit();
    cp_async_wait<0>();
    asm volatile("fence.proxy.async.shared::cta;\n");  // weights visible to the tensor core
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    const uint32_t tmem = *tslot;
    auto fail = [&]() {
        if (a.status) atomicExch(a.status, FLNR_STATUS_TIMEOUT);
    };
    auto origin = [&](int j, int &n, int &i0, int &j0) {
        const int t = blockIdx.x + j * gridDim.x;
        n = t / per_img;
        const int r = t % per_img;
        i0 = (r / tiles_x) * 16;
        j0 = (r % tiles_x) * 8;
    };

    if (warp == 4) {
        if (lane == 0) {  // producer
            for (int j = 0; j < mine; ++j) {
                const int st = j % NBUF;
                if (j >= NBUF && !mbar_wait_thread(smem_u32(empty + st), (uint32_t)((j / NBUF - 1) & 1))) {
                    fail();
                    break;
                }
                int n, i0, j0;
                origin(j, n, i0, j0);
                const uint32_t bar = smem_u32(full + st);
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(G::TMA_BYTES) : "memory");
                const uint32_t dst = smem_u32(sx0 + st * G::XBYTES);
#pragma unroll
                for (int k = 0; k < CA8; ++k) tma_load_4d(dst + k * PS, &args.tlo, 8 * k, j0 - 1, i0 - 1, n, bar);
#pragma unroll
                for (int pp = 0; pp < 4; ++pp) {
#pragma unroll
                    for (int k = 0; k < CB8; ++k)
                        tma_load_5d(dst + (CA8 + pp * CB8 + k) * PS, &args.tskip, (pp & 1) * CB + 8 * k, j0 - 1, pp >> 1,
                                    i0 - 1, n, bar);
                }
                s_issued = j + 1;
            }
        }
    } else if (warp == 5) {
        if (lane == 0) {  // MMA issuer
            constexpr uint32_t idesc = umma_idesc(COUT);
            const uint64_t adesc0 = umma_sdesc(smem_u32(sx0), PS, SW * 16);
            const uint64_t bdesc0 = umma_sdesc(smem_u32(sw), COUT * 16, 128);
            for (int j = 0; j < mine; ++j) {
                const int st = j % NBUF, acc = j & 1;
                if (!mbar_wait_thread(smem_u32(full + st), (uint32_t)((j / NBUF) & 1))) {
                    fail();
                    break;
                }
                s_consumed = j + 1;
                if (j >= 2 && !mbar_wait_thread(smem_u32(acce + acc), (uint32_t)((j / 2 - 1) & 1))) {
                    fail();
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;\n");
                const uint64_t ab = adesc0 + (uint64_t)((st * G::XBYTES) >> 4);
#pragma unroll
                for (int cls = 0; cls < 4; ++cls) {
                    const uint32_t d = tmem + (uint32_t)((acc * 4 + cls) * COUT);
#pragma unroll
                    for (int tap = 0; tap < 9; ++tap) {
                        const int t = (cls >> 1) + tap / 3 - 1, u = (cls & 1) + tap % 3 - 1;  // -1 .. 2
                        const int oy = t >> 1, ox = u >> 1, pp = (t & 1) * 2 + (u & 1);
                        const int pos = ((oy + 1) * SW + (ox + 1)) * 16;
#pragma unroll
                        for (int kk = 0; kk < CA8 / 2; ++kk) {
                            const uint32_t aoff = (uint32_t)((2 * kk * PS + pos) >> 4);
                            const uint32_t boff = (uint32_t)(((tap * C8 + 2 * kk) * COUT * 16) >> 4);
                            umma_bf16(d, ab + aoff, bdesc0 + boff, idesc, (tap | kk) ? 1u : 0u);
                        }
#pragma unroll
                        for (int kk = 0; kk < CB8 / 2; ++kk) {
                            const uint32_t aoff = (uint32_t)(((CA8 + pp * CB8 + 2 * kk) * PS + pos) >> 4);
                            const uint32_t boff = (uint32_t)(((tap * C8 + CA8 + 2 * kk) * COUT * 16) >> 4);
                            umma_bf16(d, ab + aoff, bdesc0 + boff, idesc, 1u);
                        }
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                    smem_u32(empty + st)));
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                    smem_u32(accf + acc)));
            }
        }
    } else {  // epilogue warps 0-3: TMEM lane quarter = warp; row 32w + l = position (4w + l/8, l%8)
        float bias[COUT];
#pragma unroll
        for (int c = 0; c < COUT; ++c) bias[c] = c < a.nbias ? a.bias[c] : 0.f;
        const int g = 4 * warp + (lane >> 3), r = lane & 7;
        for (int j = 0; j < mine; ++j) {
            const int acc = j & 1;
            if (!mbar_wait_warp(smem_u32(accf + acc), (uint32_t)((j / 2) & 1))) {
                if (lane == 0) fail();
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;\n");
            int n, i0, j0;
            origin(j, n, i0, j0);
#pragma unroll 1
            for (int cls = 0; cls < 4; ++cls) {
                float v[COUT];
                tc_load_acc<COUT>(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)((acc * 4 + cls) * COUT), v);
                if (cls == 3) {
                    __syncwarp();
                    if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(acce + acc)) : "memory");
                }
                tc_store<COUT, 1, 0, false>(a, v, bias, n, 2 * (i0 + g) + (cls >> 1), 2 * (j0 + r) + (cls & 1));
            }
        }
    }
    __syncwarp();  // the single-lane roles rejoin their warps before the CTA barrier
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    if (tid == 4 * 32) {  // after a failure: let copies still in flight land before the CTA exits
        for (int j = s_consumed; j < s_issued; ++j) mbar_wait_thread(smem_u32(full + j % NBUF), (uint32_t)((j / NBUF) & 1));
    }
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(G::COLS));
    }
}

// ---------------------------------------------------------------------------------------
// Stride-2 3x3 convolution (the second convolution of an encoder block, Sec. 3.3; ReLU):
// output pixel (oy, ox) of the [N][H/2][W/2] map reads input pixels (2oy + u - 1,
// 2ox + v - 1) of the [N][H][W] input (H, W even), so only the kept outputs are computed.
// A tile is 16 x 8 output pixels (oy0 + g, ox0 + r), accumulator row 8g + r.  Its input is
// staged per 8-channel chunk as four parity planes: rows 2i + pr for row pairs
// i = oy0 - 1 .. oy0 + 15, and columns 2j + pc for column pairs j = ox0 .. ox0 + 7 (even
// columns, pc = 0, planes [17][8][8]) or j = ox0 - 1 .. ox0 + 7 (odd columns, pc = 1, planes
// [17][9][8]).  Tap u reads row parity pr = (u != 1) at row offset (u != 0); tap v reads
// column parity pc = (v != 1) at column offset (v == 2) of its plane.  Consecutive output
// pixels step by one pair, so every tap's operand is a plain K-major tile of the staged
// planes: 9 taps x CIN/16 MMAs per tile, no products for the dropped positions.  The planes
// come from two 5-D views of the NHWC input (channels of a column pair, column pairs, row
// parity, row pairs, images), boxes 8 and 9 pairs wide; the start channel pc * CIN + 8k
// selects the column parity.  Roles, waits and epilogue as conv_ws_kernel.
template <int CIN, int COUT, int NBUF_>
struct S2Geom {
    static constexpr int TH = 16, TW = 8, SH = TH + 1, WE = TW, WO = TW + 1, C8 = CIN / 8, NBUF = NBUF_;
    static constexpr int PSE = (SH * WE * 16 + 127) / 128 * 128;  // even-column plane [SH][WE][8]
    static constexpr int PSO = (SH * WO * 16 + 127) / 128 * 128;  // odd-column plane [SH][WO][8]
    static constexpr int ROWP = C8 * (PSE + PSO);                  // one row parity: even chunks, odd chunks
    static constexpr int XBYTES = 2 * ROWP;
    static constexpr int TMA_BYTES = 2 * C8 * SH * (WE + WO) * 16;
    static constexpr int WBYTES = (9 * C8 * COUT * 16 + 127) / 128 * 128;
    static constexpr int NBAR = 2 * NBUF + 4;
    static constexpr int SMEM = 128 + WBYTES + NBUF * XBYTES + NBAR * 8 + 16;
    static constexpr int COLS = tmem_cols<2 * COUT>();
    static_assert(PSE % 128 == 0 && PSO % 128 == 0, "TMA destinations 128-byte aligned");
};

struct alignas(128) S2Args {
    CUtensorMap te, to;  // even-column and odd-column views of the input
    ConvArgs c;          // x [N][H][W][CIN] (H, W: the input's size), y [N][H/2][W/2][ystride]
};

template <int CIN, int COUT, int NBUF>
__global__ void __launch_bounds__(kWsThreads) conv_s2_kernel(const __grid_constant__ S2Args args)
{
    using G = S2Geom<CIN, COUT, NBUF>;
    constexpr int TH = G::TH, TW = G::TW, C8 = G::C8, PSE = G::PSE, PSO = G::PSO, ROWP = G::ROWP;
    static_assert(CIN % 16 == 0 && COUT % 16 == 0 && 2 * COUT <= 256, "UMMA shape");
    const ConvArgs &a = args.c;
    ConvArgs ao = a;  // the output map
    ao.H = a.H / 2;
    ao.W = a.W / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *base = smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);
    unsigned char *sw = base;
    unsigned char *sx0 = base + G::WBYTES;
    uint64_t *full = reinterpret_cast<uint64_t *>(sx0 + NBUF * G::XBYTES);
    uint64_t *empty = full + NBUF, *accf = empty + NBUF, *acce = accf + 2;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(acce + 2);
    __shared__ int s_issued, s_consumed;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tiles_x = (ao.W + TW - 1) / TW, tiles_y = (ao.H + TH - 1) / TH;
    const int per_img = tiles_x * tiles_y, ntiles = a.N * per_img;
    const int mine = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                     "r"(G::COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid == 0) {
        for (int i = 0; i < NBUF; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(full + i)));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(empty + i)));
        }
        for (int i = 0; i < 2; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(accf + i)));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;\n" ::"r"(smem_u32(acce + i)));  // 4 epilogue warps
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n");
        asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&args.te)) : "memory");
        asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&args.to)) : "memory");
        s_issued = 0;
        s_consumed = 0;
    }
    for (int i = tid; i < 9 * COUT * C8; i += kWsThreads) {
        const int c8 = i % C8, row = i / C8, tap = row / COUT, co = row % COUT;
        cp_async16(sw + ((tap * C8 + c8) * COUT + co) * 16, a.w + (size_t)row * CIN + c8 * 8, true);
    }
    cp_async_commit();
    cp_async_wait<0>();
    asm volatile("fence.proxy.async.shared::cta;\n");  // weights visible to the tensor core
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    const uint32_t tmem = *tslot;
    auto fail = [&]() {
        if (a.status) atomicExch(a.status, FLNR_STATUS_TIMEOUT);
    };
    auto origin = [&](int j, int &n, int &oy0, int &ox0) {
        const int t = blockIdx.x + j * gridDim.x;
        n = t / per_img;
        const int r = t % per_img;
        oy0 = (r / tiles_x) * TH;
        ox0 = (r % tiles_x) * TW;
    };

    if (warp == 4) {
        if (lane == 0) {  // producer
            for (int j = 0; j < mine; ++j) {
                const int st = j % NBUF;
                if (j >= NBUF && !mbar_wait_thread(smem_u32(empty + st), (uint32_t)((j / NBUF - 1) & 1))) {
                    fail();
                    break;
                }
                int n, oy0, ox0;
                origin(j, n, oy0, ox0);
                const uint32_t bar = smem_u32(full + st);
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(G::TMA_BYTES) : "memory");
                const uint32_t dst = smem_u32(sx0 + st * G::XBYTES);
#pragma unroll
                for (int pr = 0; pr < 2; ++pr) {
#pragma unroll
                    for (int k = 0; k < C8; ++k)
                        tma_load_5d(dst + pr * ROWP + k * PSE, &args.te, 8 * k, ox0, pr, oy0 - 1, n, bar);
#pragma unroll
                    for (int k = 0; k < C8; ++k)
                        tma_load_5d(dst + pr * ROWP + C8 * PSE + k * PSO, &args.to, CIN + 8 * k, ox0 - 1, pr, oy0 - 1, n, bar);
                }
                s_issued = j + 1;
            }
        }
    } else if (warp == 5) {
        if (lane == 0) {  // MMA issuer
            constexpr uint32_t idesc = umma_idesc(COUT);
            const uint64_t adesc_e = umma_sdesc(smem_u32(sx0), PSE, G::WE * 16);
            const uint64_t adesc_o = umma_sdesc(smem_u32(sx0), PSO, G::WO * 16);
            const uint64_t bdesc0 = umma_sdesc(smem_u32(sw), COUT * 16, 128);
            for (int j = 0; j < mine; ++j) {
                const int st = j % NBUF, acc = j & 1;
                if (!mbar_wait_thread(smem_u32(full + st), (uint32_t)((j / NBUF) & 1))) {
                    fail();
                    break;
                }
                s_consumed = j + 1;
                if (j >= 2 && !mbar_wait_thread(smem_u32(acce + acc), (uint32_t)((j / 2 - 1) & 1))) {
                    fail();
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;\n");
                const uint32_t sbase = (uint32_t)(st * G::XBYTES);
                const uint32_t d = tmem + (uint32_t)(acc * COUT);
#pragma unroll
                for (int tap = 0; tap < 9; ++tap) {
                    const int u = tap / 3, v = tap % 3;
                    const int pr = u != 1, pc = v != 1, ro = u != 0, co = v == 2;
#pragma unroll
                    for (int kk = 0; kk < C8 / 2; ++kk) {
                        const uint32_t off = pc ? sbase + pr * ROWP + C8 * PSE + 2 * kk * PSO + (ro * G::WO + co) * 16
                                                : sbase + pr * ROWP + 2 * kk * PSE + ro * G::WE * 16;
                        const uint64_t ad = (pc ? adesc_o : adesc_e) + (uint64_t)(off >> 4);
                        const uint32_t boff = (uint32_t)(((tap * C8 + 2 * kk) * COUT * 16) >> 4);
                        umma_bf16(d, ad, bdesc0 + boff, idesc, (tap | kk) ? 1u : 0u);
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                    smem_u32(empty + st)));
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                    smem_u32(accf + acc)));
            }
        }
    } else {  // epilogue warps 0-3: TMEM lane quarter = warp
        float bias[COUT];
#pragma unroll
        for (int c = 0; c < COUT; ++c) bias[c] = c < a.nbias ? a.bias[c] : 0.f;
        for (int j = 0; j < mine; ++j) {
            const int acc = j & 1;
            if (!mbar_wait_warp(smem_u32(accf + acc), (uint32_t)((j / 2) & 1))) {
                if (lane == 0) fail();
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;\n");
            float v[COUT];
            tc_load_acc<COUT>(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(acc * COUT), v);
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(acce + acc)) : "memory");
            int n, oy0, ox0;
            origin(j, n, oy0, ox0);
            tc_store<COUT, 1, 0, false>(ao, v, bias, n, oy0 + 4 * warp + (lane >> 3), ox0 + (lane & 7));
        }
    }
    __syncwarp();  // the single-lane roles rejoin their warps before the CTA barrier
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    if (tid == 4 * 32) {  // after a failure: let copies still in flight land before the CTA exits
        for (int j = s_consumed; j < s_issued; ++j) mbar_wait_thread(smem_u32(full + j % NBUF), (uint32_t)((j / NBUF) & 1));
    }
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(G::COLS));
    }
}

// ---------------------------------------------------------------------------------------
// Weight gradient on the tensor cores (tcgen05): for every tap and channel pair
//   dW[o][i][tap] = sum_p dz[p][o] x[p + off(tap)][i],
// one GEMM D[(tap, i)][o] = sum_p A[(tap, i)][p] B[o][p] with the pixels as K: A is the
// im2col of x (M = KS^2 * CIN rows, split into MT accumulators of 128 rows), B = dz^T
// (N = COUT).  A CTA walks a contiguous range of 8 x 8 pixel tiles (K = 64 per tile) and keeps
// its MT accumulators in tensor memory across the whole range:
//   1. x (with a KS/2 halo, zero outside the image) and dz of the tile land in shared memory
//      by cp.async as 16-byte pixel rows [chunk][row][col][8 channels], double-buffered;
//   2. the four warps build the K-major operands from them with ldmatrix.trans: an 8 x 8
//      block of (8 pixels of one tile row) x (8 channels) becomes one 128-byte core matrix
//      (8 channels x 8 pixels); the tap's offset is applied in the ldmatrix row addresses;
//   3. one thread issues MT x 4 MMAs (K = 16 each) and commits them to an mbarrier, which
//      the warps wait on (bounded) before they overwrite the operands with the next tile.
// Operand layouts (no swizzle): A tile mt at mt * 16 KB, core matrix (row group rg, pixel
// row kg) at (16 kg + rg) * 128 (LBO 2048 between K groups, SBO 128 between row groups);
// B core matrix (channel group og, kg) at (kg * COUT/8 + og) * 128 (LBO COUT * 16, SBO 128).
// Rows of A past KS^2 * CIN are never written and their accumulator rows are discarded.
// At the end each thread writes its accumulator row (one (tap, i)) to the CTA's slot of a
// partials buffer; wgrad_reduce_kernel then adds the CTAs' partials in CTA order to the FP32
// master gradient [Cout][Cin][k][k] (padding channels skipped), so the result does not depend
// on the order in which CTAs finish.
struct WgradArgs {
    const bf16 *x, *dz;
    float *gw;    // master layout
    float *part;  // per-CTA partial products [grid][KS^2 CIN][COUT]
    int N, H, W, cin_true, cout_true, tiles_per_cta;
    int *status;
};

// gw[o][i][tap] += sum over the CTAs, in CTA order, of their partial (tap CIN + i, o): the
// weight gradient without atomics, the same every run.  Thread f takes element f of the
// partials' own layout ((tap CIN + i) COUT + o), so that the threads of a warp read
// consecutive addresses of each CTA's partial; the loads of several CTAs are in flight at once
// while the additions keep CTA order.
template <int CIN, int COUT, int KS>
__global__ void __launch_bounds__(32) wgrad_reduce_kernel(const float *part, int nctas, float *gw, int cin_true,
                                                          int cout_true)
{
    constexpr int M = KS * KS * CIN, NB = 64;
    for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < M * COUT; f += gridDim.x * blockDim.x) {
        const int o = f % COUT, row = f / COUT, i = row % CIN, tap = row / CIN;
        if (i >= cin_true || o >= cout_true) continue;
        const float *p = part + f;
        // the partials in CTA order; each batch's loads are issued (in order, as volatile loads)
        // before any of its additions, so a thread has NB of them in flight
        float s = 0.f;
        int b = 0;
        for (; b + NB <= nctas; b += NB) {
            float v[NB];
#pragma unroll
            for (int u = 0; u < NB; ++u)
                asm volatile("ld.global.nc.f32 %0, [%1];" : "=f"(v[u]) : "l"(p + (size_t)(b + u) * M * COUT));
#pragma unroll
            for (int u = 0; u < NB; ++u) s += v[u];
        }
        for (; b < nctas; ++b) s += p[(size_t)b * M * COUT];
        gw[((size_t)o * cin_true + i) * (KS * KS) + tap] += s;
    }
}

template <int CIN, int COUT, int KS>
struct WgGeom {
    static constexpr int P = KS / 2, SH = 8 + 2 * P, SW = 8 + 2 * P, C8 = CIN / 8, O8 = COUT / 8;
    static constexpr int M = KS * KS * CIN, MT = (M + 127) / 128;
    static constexpr int XP = (SH * SW * 16 + 127) / 128 * 128;  // one staged x chunk plane
    static constexpr int STAGE = C8 * XP + O8 * 1024;            // x planes, then dz planes [8][8][8]
    static constexpr int ABYTES = MT * 16384, BBYTES = O8 * 1024;
    static constexpr int SMEM = 128 + 2 * STAGE + ABYTES + BBYTES + 16;
    static constexpr int COLS = tmem_cols<MT * COUT>();
    static constexpr int NU = KS * KS * C8 * 8;  // A core matrices per tile (tap, chunk, pixel row)
    static_assert(MT * COUT <= 512, "accumulators exceed tensor memory");
};

__device__ __forceinline__ void ldsm_x4_trans(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

template <int CIN, int COUT, int KS>
__global__ void __launch_bounds__(128) wgrad_tc_kernel(const WgradArgs a)
{
    using G = WgGeom<CIN, COUT, KS>;
    constexpr int P = G::P, SW = G::SW, C8 = G::C8, O8 = G::O8, XP = G::XP, MT = G::MT;
    static_assert(CIN % 16 == 0 && COUT % 16 == 0, "UMMA shape");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *base = smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);
    unsigned char *stage0 = base;
    unsigned char *opA = base + 2 * G::STAGE;
    unsigned char *opB = opA + G::ABYTES;
    uint64_t *done = reinterpret_cast<uint64_t *>(opB + G::BBYTES);
    __shared__ uint32_t s_tmem;
    __shared__ int s_fail;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tiles_x = (a.W + 7) / 8, tiles_y = (a.H + 7) / 8;
    const long long ntiles = (long long)a.N * tiles_x * tiles_y;
    const long long t0 = (long long)blockIdx.x * a.tiles_per_cta;
    const long long t1 = t0 + a.tiles_per_cta < ntiles ? t0 + a.tiles_per_cta : ntiles;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&s_tmem)),
                     "r"(G::COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(done)));
        asm volatile("fence.mbarrier_init.release.cluster;\n");
        s_fail = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    const uint32_t tmem = s_tmem;

    auto stage = [&](long long t, unsigned char *sb) {
        const int n = (int)(t / ((long long)tiles_x * tiles_y));
        const int r = (int)(t % ((long long)tiles_x * tiles_y));
        const int ty0 = (r / tiles_x) * 8, tx0 = (r % tiles_x) * 8;
        for (int e = tid; e < C8 * G::SH * SW; e += 128) {
            const int c8 = e / (G::SH * SW), pix = e % (G::SH * SW);
            const int yy = ty0 - P + pix / SW, xx = tx0 - P + pix % SW;
            const bool in = yy >= 0 && yy < a.H && xx >= 0 && xx < a.W;
            const bf16 *src = in ? a.x + (((size_t)n * a.H + yy) * a.W + xx) * CIN + c8 * 8 : a.x;
            cp_async16(sb + c8 * XP + pix * 16, src, in);
        }
        unsigned char *sd = sb + C8 * XP;
        for (int e = tid; e < O8 * 64; e += 128) {
            const int o8 = e / 64, pix = e % 64;
            const int yy = ty0 + pix / 8, xx = tx0 + pix % 8;
            const bool in = yy < a.H && xx < a.W;
            const bf16 *src = in ? a.dz + (((size_t)n * a.H + yy) * a.W + xx) * COUT + o8 * 8 : a.dz;
            cp_async16(sd + o8 * 1024 + pix * 16, src, in);
        }
    };

    constexpr uint32_t idesc = umma_idesc(COUT);
    int it = 0;
    if (t0 < t1) stage(t0, stage0);
    cp_async_commit();
    for (long long t = t0; t < t1; ++t, ++it) {
        unsigned char *sb = stage0 + (it & 1) * G::STAGE;
        if (t + 1 < t1) stage(t + 1, stage0 + ((it + 1) & 1) * G::STAGE);
        cp_async_commit();
        cp_async_wait<1>();
        // the MMAs of the previous tile must have read the operands before they are rebuilt
        if (it > 0 && !mbar_wait_warp(smem_u32(done), (uint32_t)((it - 1) & 1))) {
            if (lane == 0) s_fail = 1;
        }
        __syncthreads();
        if (s_fail) break;
        // A: unit q = (tap, chunk, pixel row ty); lanes 8j..8j+7 address unit q + j, row tx
        const uint32_t xs = smem_u32(sb), as = smem_u32(opA);
        for (int q = 4 * warp; q < G::NU; q += 16) {
            const int u = q + (lane >> 3), tx = lane & 7;
            const int ty = u % 8, c8 = (u / 8) % C8, tap = u / (8 * C8);
            const int dy = tap / KS, dx = tap % KS;
            uint32_t v[4];
            ldsm_x4_trans(xs + c8 * XP + ((ty + dy) * SW + tx + dx) * 16, v[0], v[1], v[2], v[3]);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int uj = q + j, tyj = uj % 8, m0 = (uj / (8 * C8)) * CIN + ((uj / 8) % C8) * 8;
                const uint32_t dst = as + (m0 / 128) * 16384 + (tyj * 16 + (m0 % 128) / 8) * 128 + lane * 4;
                asm volatile("st.shared.b32 [%0], %1;\n" ::"r"(dst), "r"(v[j]) : "memory");
            }
        }
        // B: unit q = (channel group og, pixel row ty)
        const uint32_t ds = xs + C8 * XP, bs = smem_u32(opB);
        for (int q = 4 * warp; q < O8 * 8; q += 16) {
            const int u = q + (lane >> 3), tx = lane & 7;
            const int ty = u % 8, og = u / 8;
            uint32_t v[4];
            ldsm_x4_trans(ds + og * 1024 + (ty * 8 + tx) * 16, v[0], v[1], v[2], v[3]);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int uj = q + j;
                const uint32_t dst = bs + ((uj % 8) * O8 + uj / 8) * 128 + lane * 4;
                asm volatile("st.shared.b32 [%0], %1;\n" ::"r"(dst), "r"(v[j]) : "memory");
            }
        }
        asm volatile("fence.proxy.async.shared::cta;\n");  // operands visible to the tensor core
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n");
            const uint64_t ad0 = umma_sdesc(as, 2048, 128), bd0 = umma_sdesc(bs, O8 * 128, 128);
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                const uint64_t bd = bd0 + (uint64_t)((2 * s * O8 * 128) >> 4);
#pragma unroll
                for (int mt = 0; mt < MT; ++mt) {
                    const uint64_t ad = ad0 + (uint64_t)((mt * 16384 + 2 * s * 2048) >> 4);
                    umma_bf16(tmem + (uint32_t)(mt * COUT), ad, bd, idesc, (it > 0 || s > 0) ? 1u : 0u);
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                smem_u32(done)));
        }
    }
    cp_async_wait<0>();
    bool ok = !s_fail;
    if (ok && it > 0 && !mbar_wait_warp(smem_u32(done), (uint32_t)((it - 1) & 1))) {
        ok = false;
        if (lane == 0) s_fail = 1;
    }
    __syncthreads();
    if (s_fail) {
        if (tid == 0 && a.status) atomicExch(a.status, FLNR_STATUS_TIMEOUT);
    } else if (it > 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n");
        const int r = 32 * warp + lane;
#pragma unroll 1
        for (int mt = 0; mt < MT; ++mt) {
            const int m = mt * 128 + r;
#pragma unroll
            for (int o0 = 0; o0 < COUT; o0 += 16) {
                float v[16];
                tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(mt * COUT + o0), v);
                asm volatile("tcgen05.wait::ld.sync.aligned;\n");
                if (m < G::M) {  // this CTA's partial row, summed in a fixed order by wgrad_reduce_kernel
                    float4 *dst = reinterpret_cast<float4 *>(a.part + ((size_t)blockIdx.x * G::M + m) * COUT + o0);
#pragma unroll
                    for (int j = 0; j < 4; ++j) dst[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(G::COLS));
    }
}

// ---------------------------------------------------------------------------------------
// Elementwise and layout kernels
// planar fp32 [N][11][H][W] -> NHWC bf16 with 16 channels (11 used); the radiance channels
// enter the network as log(1 + max(Y, 0)), which keeps fireflies from dominating the features
__global__ void pack_input_kernel(const float *in, bf16 *x, int N, int H, int W)
{
    const size_t hw = (size_t)H * W, total = (size_t)N * hw;
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < total; p += (size_t)gridDim.x * blockDim.x) {
        const size_t n = p / hw, o = p % hw;
        alignas(16) bf16 v[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            float u = 0.f;
            if (c < 8) u = in[(n * 11 + c) * hw + o];
            else if (c < 11) u = log1pf(fmaxf(in[(n * 11 + c) * hw + o], 0.f));  // radiance: log(1 + max(Y, 0))
            v[c] = __float2bfloat16(u);
        }
        *reinterpret_cast<uint4 *>(x + p * 16) = *reinterpret_cast<uint4 *>(v);
        *reinterpret_cast<uint4 *>(x + p * 16 + 8) = *reinterpret_cast<uint4 *>(v + 8);
    }
}

// gradient with respect to the network's planar input [N][11][H][W] from the gradient dx
// [N][H][W][16] with respect to the packed input x: the guides pass through; a radiance
// channel was read as L = log(1 + max(Y, 0)), whose derivative is 1 / (1 + Y) = exp(-L) for
// Y > 0 and 0 for Y < 0 (L is the stored bfloat16 value, so Y > 0 exactly when L > 0)
__global__ void unpack_grad_kernel(const bf16 *dx, const bf16 *x, float *g, int N, int H, int W)
{
    const size_t hw = (size_t)H * W, total = (size_t)N * hw;
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < total; p += (size_t)gridDim.x * blockDim.x) {
        const size_t n = p / hw, o = p % hw;
#pragma unroll
        for (int c = 0; c < 11; ++c) {
            float d = __bfloat162float(dx[p * 16 + c]);
            if (c >= 8) {
                const float L = __bfloat162float(x[p * 16 + c]);
                d = L > 0.f ? d * expf(-L) : 0.f;
            }
            g[(n * 11 + c) * hw + o] = d;
        }
    }
}

// nearest 2x upsampling of lo [N][H/2][W/2][Ca] concatenated with skip [N][H][W][Cb] (the
// input of a decoder level, materialised for its weight gradient)
__global__ void upcat_kernel(const bf16 *lo, const bf16 *skip, bf16 *y, int N, int H, int W, int Ca, int Cb)
{
    // one thread per (pixel, 8-channel group) of y [N][H][W][Ca + Cb]: 16-byte copies
    const int C8 = (Ca + Cb) / 8, A8 = Ca / 8;
    const long long total = (long long)N * H * W * C8;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const int c8 = (int)(e % C8);
        const long long p = e / C8;
        const uint4 *src;
        if (c8 < A8) {
            const int x = (int)(p % W);
            const long long rowp = p / W;  // n * H + y
            const int yy = (int)(rowp % H);
            const long long n = rowp / H;
            src = reinterpret_cast<const uint4 *>(lo + ((n * (H / 2) + yy / 2) * (W / 2) + x / 2) * Ca + c8 * 8);
        } else {
            src = reinterpret_cast<const uint4 *>(skip + p * Cb + (c8 - A8) * 8);
        }
        reinterpret_cast<uint4 *>(y)[e] = *src;
    }
}

// gradient of the sigmoid output head (nout planar outputs): dz[p][c] = g * s (1 - s) for
// c < nout, 0 for the pads of the 16 channels
__global__ void sigmoid_bwd_kernel(const float *g, const float *s, bf16 *dz, int N, int H, int W, int nout)
{
    const size_t hw = (size_t)H * W, total = (size_t)N * hw;
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < total; p += (size_t)gridDim.x * blockDim.x) {
        const size_t n = p / hw, o = p % hw;
        alignas(16) bf16 v[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            float d = 0.f;
            if (c < nout) {
                const float sv = s[(n * nout + c) * hw + o];
                d = g[(n * nout + c) * hw + o] * sv * (1.f - sv);
            }
            v[c] = __float2bfloat16(d);
        }
        *reinterpret_cast<uint4 *>(dz + p * 16) = *reinterpret_cast<uint4 *>(v);
        *reinterpret_cast<uint4 *>(dz + p * 16 + 8) = *reinterpret_cast<uint4 *>(v + 8);
    }
}

// backward of up ++ skip: g_lo[q][c] = mask(lo) * sum_{2x2} gy[p][c] (c < Ca);
// g_skip[p][c] = gy[p][Ca + c] (unmasked, the caller masks where the skip is consumed)
__global__ void upcat_bwd_kernel(const bf16 *gy, const bf16 *lo, bf16 *g_lo, float *g_skip, int N, int H, int W,
                                 int Ca, int Cb)
{
    // eight channels of one pixel per thread (Ca and Cb are multiples of 8): 16-byte loads and
    // stores, the index arithmetic once per eight values
    const int C = Ca + Cb, Hl = H / 2, Wl = W / 2;
    const size_t tl = (size_t)N * Hl * Wl * Ca / 8, ts = (size_t)N * H * W * Cb / 8;
    for (size_t e8 = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e8 < tl + ts; e8 += (size_t)gridDim.x * blockDim.x) {
        if (e8 < tl) {
            const size_t e = 8 * e8;
            const int c = (int)(e % Ca);
            const size_t q = e / Ca;
            const int xl = (int)(q % Wl), yl = (int)((q / Wl) % Hl), n = (int)(q / ((size_t)Wl * Hl));
            const size_t b = (((size_t)n * H + 2 * yl) * W + 2 * xl) * C + c;
            const uint4 r0 = *reinterpret_cast<const uint4 *>(gy + b), r1 = *reinterpret_cast<const uint4 *>(gy + b + C);
            const uint4 r2 = *reinterpret_cast<const uint4 *>(gy + b + (size_t)W * C);
            const uint4 r3 = *reinterpret_cast<const uint4 *>(gy + b + (size_t)W * C + C);
            const uint4 l = *reinterpret_cast<const uint4 *>(lo + e);
            const bf16 *g0 = reinterpret_cast<const bf16 *>(&r0), *g1 = reinterpret_cast<const bf16 *>(&r1);
            const bf16 *g2 = reinterpret_cast<const bf16 *>(&r2), *g3 = reinterpret_cast<const bf16 *>(&r3);
            const bf16 *lv = reinterpret_cast<const bf16 *>(&l);
            uint4 o;
            bf16 *ov = reinterpret_cast<bf16 *>(&o);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const float sum = __bfloat162float(g0[i]) + __bfloat162float(g1[i]) + __bfloat162float(g2[i]) +
                                  __bfloat162float(g3[i]);
                ov[i] = __float2bfloat16(__bfloat162float(lv[i]) > 0.f ? sum : 0.f);
            }
            *reinterpret_cast<uint4 *>(g_lo + e) = o;
        } else {
            const size_t f = 8 * (e8 - tl);
            const int c = (int)(f % Cb);
            const uint4 r = *reinterpret_cast<const uint4 *>(gy + (f / Cb) * C + Ca + c);
            const bf16 *rv = reinterpret_cast<const bf16 *>(&r);
            float4 v0, v1;
            v0.x = __bfloat162float(rv[0]); v0.y = __bfloat162float(rv[1]);
            v0.z = __bfloat162float(rv[2]); v0.w = __bfloat162float(rv[3]);
            v1.x = __bfloat162float(rv[4]); v1.y = __bfloat162float(rv[5]);
            v1.z = __bfloat162float(rv[6]); v1.w = __bfloat162float(rv[7]);
            *reinterpret_cast<float4 *>(g_skip + f) = v0;
            *reinterpret_cast<float4 *>(g_skip + f + 4) = v1;
        }
    }
}

// Gradient with respect to the pre-activation of a layer whose ReLU output f [N][Ho][Wo][C]
// feeds the next encoder convolution (gradient g_path, bf16) and, when g_skip is given, a
// decoder skip (fp32): dz = mask(f) * (g_skip + g_path); no mask when f is NULL.  S = 2 (the
// layer strides by 2): dz is written zero-upsampled onto the layer's input grid
// [N][2Ho][2Wo][C], nonzero only at even rows and columns, so that the stride-1 input- and
// weight-gradient kernels at the input's size give the stride-2 layer's gradients.
template <int S>
__global__ void join_bwd_kernel(const float *g_skip, const bf16 *g_path, const bf16 *f, bf16 *dz, int N, int Ho, int Wo,
                                int C)
{
    // eight channels of one pixel per thread (C a multiple of 8): 16-byte loads and stores
    const int H = S * Ho, W = S * Wo;
    const size_t total8 = (size_t)N * H * W * C / 8;
    for (size_t e8 = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e8 < total8; e8 += (size_t)gridDim.x * blockDim.x) {
        const size_t e = 8 * e8;
        const int c = (int)(e % C);
        const size_t p = e / C;
        const int x = (int)(p % W), y = (int)((p / W) % H), n = (int)(p / ((size_t)W * H));
        uint4 o = make_uint4(0u, 0u, 0u, 0u);  // bfloat16 +0
        if (S == 1 || ((x | y) & 1) == 0) {
            const size_t q = (((size_t)n * Ho + y / S) * Wo + x / S) * C + c;
            const uint4 gp = *reinterpret_cast<const uint4 *>(g_path + q);
            const bf16 *gv = reinterpret_cast<const bf16 *>(&gp);
            float sk[8];
            if (g_skip) {
                const float4 s0 = *reinterpret_cast<const float4 *>(g_skip + q);
                const float4 s1 = *reinterpret_cast<const float4 *>(g_skip + q + 4);
                sk[0] = s0.x; sk[1] = s0.y; sk[2] = s0.z; sk[3] = s0.w;
                sk[4] = s1.x; sk[5] = s1.y; sk[6] = s1.z; sk[7] = s1.w;
            }
            uint4 fm = make_uint4(0u, 0u, 0u, 0u);
            if (f) fm = *reinterpret_cast<const uint4 *>(f + q);
            const bf16 *fv = reinterpret_cast<const bf16 *>(&fm);
            bf16 *ov = reinterpret_cast<bf16 *>(&o);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                float v = __bfloat162float(gv[i]) + (g_skip ? sk[i] : 0.f);
                if (f && !(__bfloat162float(fv[i]) > 0.f)) v = 0.f;
                ov[i] = __float2bfloat16(v);
            }
        }
        *reinterpret_cast<uint4 *>(dz + e) = o;
    }
}

// Bias gradients gb[c] += sum over the pixels of dz[p][c], without atomics and in a fixed
// order, in two passes: thread (t, c) of bias_part_kernel sums dz[p][c] over the pixels
// p = t, t + 256, t + 512, ... in turn (consecutive threads take consecutive channels, so a
// warp reads consecutive values; one warp per CTA, so the 256 C threads spread over 8 C SMs),
// and bias_tree_kernel, one CTA per channel, adds the 256 partial sums by halving.  These are
// the partial sums and the tree of one 256-thread CTA per channel walking the pixels, only
// spread so that the loads are coalesced and many are in flight.
__device__ __forceinline__ unsigned short ld_b16(const bf16 *p)
{
    unsigned short v;
    asm volatile("ld.global.nc.b16 %0, [%1];" : "=h"(v) : "l"(p));
    return v;
}

__global__ void __launch_bounds__(32) bias_part_kernel(const bf16 *dz, float *part, long long P, int C)
{
    constexpr int NB = 128;  // loads issued ahead of their additions
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= 256 * C) return;
    const int t = g / C, c = g % C;
    // the pixels in turn; each batch's loads are issued (in order, as volatile loads) before
    // any of its additions, so a thread has NB of them in flight
    float s = 0.f;
    long long p = t;
    for (; p + (NB - 1) * 256LL < P; p += NB * 256LL) {
        unsigned short v[NB];
#pragma unroll
        for (int u = 0; u < NB; ++u) v[u] = ld_b16(dz + (p + (long long)u * 256) * C + c);
#pragma unroll
        for (int u = 0; u < NB; ++u) s += __bfloat162float(__ushort_as_bfloat16(v[u]));
    }
    for (; p < P; p += 256) s += __bfloat162float(dz[p * C + c]);
    part[(size_t)t * C + c] = s;
}

__global__ void __launch_bounds__(256) bias_tree_kernel(const float *part, float *gb, int C)
{
    __shared__ float red[256];
    const int c = blockIdx.x, t = threadIdx.x;
    red[t] = part[(size_t)t * C + c];
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (t < o) red[t] += red[t + o];
        __syncthreads();
    }
    if (t == 0) gb[c] += red[0];
}

// master fp32 [Cout][Cin][k][k] -> forward bf16 [tap][CoutP][CinP] and dgrad bf16
// [tap'][CinP][CoutP] with tap' = taps - 1 - tap (rotated by 180 degrees), zero pads
__global__ void weights_kernel(const float *w, bf16 *wf, bf16 *wd, int cin, int cout, int cinp, int coutp, int k)
{
    const int taps = k * k;
    const int total = taps * coutp * cinp;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const int i = e % cinp, o = (e / cinp) % coutp, tap = e / (cinp * coutp);
        const float v = (i < cin && o < cout) ? w[((size_t)o * cin + i) * taps + tap] : 0.f;
        wf[e] = __float2bfloat16(v);
        wd[((size_t)(taps - 1 - tap) * cinp + i) * coutp + o] = __float2bfloat16(v);
    }
}

__global__ void adam_kernel(float *w, const float *g, float *m, float *v, size_t n, float lr, float b1, float b2,
                            float eps, float c1, float c2)
{
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const float gr = g[e];
        const float mm = b1 * m[e] + (1.f - b1) * gr;
        const float vv = b2 * v[e] + (1.f - b2) * gr * gr;
        m[e] = mm;
        v[e] = vv;
        w[e] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
    }
}

// L1 loss between prediction and reference (planar fp32, n values): writes d/dpred = sign / n
// and accumulates the mean absolute error into *loss
// SMAPE of pred against ref (Sec. 3.3 trains FLNR on it): loss += mean |p - r| / D with
// D = |p| + |r| + eps, and d/dp = (sign(p - r) / D - |p - r| sign(p) / D^2) / n
__global__ void smape_kernel(const float *pred, const float *ref, float *grad, float *loss, size_t n, float eps)
{
    __shared__ float part[256];
    float s = 0.f;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const float p = pred[e], d = p - ref[e], a = fabsf(d);
        const float inv = 1.f / (fabsf(p) + fabsf(ref[e]) + eps);
        const float sd = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f), sp = p > 0.f ? 1.f : (p < 0.f ? -1.f : 0.f);
        grad[e] = (sd - a * sp * inv) * inv / (float)n;
        s += a * inv;
    }
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, part[0] / (float)n);
}

__global__ void l1_kernel(const float *pred, const float *ref, float *grad, float *loss, size_t n)
{
    __shared__ float part[256];
    float s = 0.f;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const float d = pred[e] - ref[e];
        grad[e] = (d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f)) / (float)n;
        s += fabsf(d);
    }
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, part[0] / (float)n);
}

int egrid(size_t n) { return (int)((n + 255) / 256 < 8192 ? (n + 255) / 256 : 8192); }

// ---------------------------------------------------------------------------------------
// Launch helpers for the template instantiations the network uses.
// cuTensorMapEncodeTiled through the runtime's driver entry point (no link to libcuda)
PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// 4-D map of an NHWC bf16 tensor [N][H][W][C]: box (8 channels, bw, bh, 1), zero fill outside
cudaError_t make_tmap(CUtensorMap *m, const void *base, int C, int W, int H, int N, int bw, int bh)
{
    PFN_cuTensorMapEncodeTiled_v12000 fn = tmap_encoder();
    if (!fn) return cudaErrorNotSupported;
    const cuuint64_t dims[4] = {(cuuint64_t)C, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)N};
    const cuuint64_t strides[3] = {(cuuint64_t)C * 2, (cuuint64_t)W * C * 2, (cuuint64_t)H * W * C * 2};
    const cuuint32_t box[4] = {8, (cuuint32_t)bw, (cuuint32_t)bh, 1};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void *>(base), dims, strides, box, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// 5-D map of an NHWC bf16 tensor [N][H][W][C] (H, W even) that stages one parity plane per
// box: dims (2C channels of a column pair, W/2 column pairs, 2 row parities, H/2 row pairs,
// N); box (8, bw, 1, bh, 1).  The start channel b * C + 8k selects column parity b, chunk k.
cudaError_t make_tmap_parity(CUtensorMap *m, const void *base, int C, int W, int H, int N, int bw, int bh)
{
    PFN_cuTensorMapEncodeTiled_v12000 fn = tmap_encoder();
    if (!fn) return cudaErrorNotSupported;
    const cuuint64_t dims[5] = {(cuuint64_t)2 * C, (cuuint64_t)W / 2, 2, (cuuint64_t)H / 2, (cuuint64_t)N};
    const cuuint64_t strides[4] = {(cuuint64_t)C * 4, (cuuint64_t)W * C * 2, (cuuint64_t)W * C * 4,
                                   (cuuint64_t)H * W * C * 2};
    const cuuint32_t box[5] = {8, (cuuint32_t)bw, 1, (cuuint32_t)bh, 1};
    const cuuint32_t es[5] = {1, 1, 1, 1, 1};
    const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void *>(base), dims, strides, box, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Launch of the warp-specialised convolution.  The occupancy API reports one CTA per SM for
// kernels that allocate tensor memory, so the resident count is computed here from the
// kernel's registers, shared memory and threads, and capped at 512 / (TMEM columns per CTA);
// where threads alone would allow more CTAs than TMEM can hold, the shared-memory request is
// raised so that no more can be resident (an allocation never has to wait for another CTA).
template <int CIN, int COUT, int KS, int ACT, int OUTM, bool MASK = false>
cudaError_t conv_ws_launch(const ConvArgs &a, cudaStream_t st)
{
    using G = WsGeom<CIN, COUT, KS>;
    constexpr int kSmemPerSm = 228 * 1024, kReservedPerCta = 1024, kThreadsPerSm = 2048;
    constexpr int tmem_cap = 512 / G::COLS;
    constexpr int min_smem = tmem_cap < kThreadsPerSm / kWsThreads ? kSmemPerSm / tmem_cap - kReservedPerCta - 256 : 0;
    constexpr size_t smem = (size_t)(G::SMEM > min_smem ? G::SMEM : min_smem);
    static_assert(smem <= 227 * 1024, "warp-specialised conv tile does not fit in shared memory");
    auto kern = conv_ws_kernel<CIN, COUT, KS, ACT, OUTM, MASK>;
    static int per_sm = 0, n_sm = 0;
    if (per_sm == 0) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
        cudaFuncAttributes fa;
        if ((e = cudaFuncGetAttributes(&fa, kern)) != cudaSuccess) return e;
        int dev = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        // registers are split over the SM's four sub-partitions: warps per sub-partition first
        const int regs_per_warp = (fa.numRegs * 32 + 255) / 256 * 256;
        const int by_regs = (4 * (16384 / regs_per_warp)) / (kWsThreads / 32);
        const int by_smem = kSmemPerSm / ((int)smem + (int)fa.sharedSizeBytes + kReservedPerCta);
        int r = kThreadsPerSm / kWsThreads;
        r = r < by_regs ? r : by_regs;
        r = r < by_smem ? r : by_smem;
        r = r < tmem_cap ? r : tmem_cap;
        if (r < 1) return cudaErrorInvalidConfiguration;
        per_sm = r;
    }
    const long long ntiles = (long long)a.N * ((a.H + G::TH - 1) / G::TH) * ((a.W + G::TW - 1) / G::TW);
    if (ntiles <= 0) return cudaSuccess;
    TcArgs ta;
    std::memset(&ta, 0, sizeof(ta));
    ta.c = a;
    cudaError_t e = make_tmap(&ta.tm, a.x, CIN, a.W, a.H, a.N, G::SW, G::SH);
    if (e != cudaSuccess) return e;
    const long long cap = (long long)per_sm * n_sm;
    kern<<<(int)(ntiles < cap ? ntiles : cap), kWsThreads, smem, st>>>(ta);
    return cudaGetLastError();
}

// Input gradient of a layer on the tensor cores: the stride-1 convolution of dz with the
// layer's weights rotated by 180 degrees and transposed ([tap][CinP][CoutP]), no bias, no
// activation, times (mask > 0) when MASK (the ReLU of the layer input).  a: x = dz
// [N][H][W][CIN], w, mask [N][H][W][COUT], y [N][H][W][ystride].
template <int CIN, int COUT, int KS, bool MASK>
cudaError_t dgrad_launch(ConvArgs a, int *status, cudaStream_t st)
{
    a.bias = nullptr;
    a.nbias = 0;
    a.status = status;
    return conv_ws_launch<CIN, COUT, KS, 0, 0, MASK>(a, st);
}

// Launch of the fused KS x KS + 1x1 pair (c: first layer, c2: the 1x1 layer); residency
// computed as for conv_ws_launch.
template <int CIN, int COUT, int KS, int COUT2, int ACT2, int OUTM2>
cudaError_t conv_tail_launch(const ConvArgs &c, const ConvArgs &c2, cudaStream_t st)
{
    using T = TailGeom<CIN, COUT, KS, COUT2>;
    using G = typename T::G1;
    constexpr int kSmemPerSm = 228 * 1024, kReservedPerCta = 1024, kThreadsPerSm = 2048;
    constexpr int tmem_cap = 512 / T::COLS;
    constexpr int min_smem = tmem_cap < kThreadsPerSm / kWsThreads ? kSmemPerSm / tmem_cap - kReservedPerCta - 256 : 0;
    constexpr size_t smem = (size_t)(T::SMEM > min_smem ? T::SMEM : min_smem);
    static_assert(smem <= 227 * 1024, "fused conv stage does not fit in shared memory");
    auto kern = conv_tail_kernel<CIN, COUT, KS, COUT2, ACT2, OUTM2>;
    static int per_sm = 0, n_sm = 0;
    if (per_sm == 0) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
        cudaFuncAttributes fa;
        if ((e = cudaFuncGetAttributes(&fa, kern)) != cudaSuccess) return e;
        int dev = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        const int regs_per_warp = (fa.numRegs * 32 + 255) / 256 * 256;
        const int by_regs = (4 * (16384 / regs_per_warp)) / (kWsThreads / 32);
        const int by_smem = kSmemPerSm / ((int)smem + (int)fa.sharedSizeBytes + kReservedPerCta);
        int r = kThreadsPerSm / kWsThreads;
        r = r < by_regs ? r : by_regs;
        r = r < by_smem ? r : by_smem;
        r = r < tmem_cap ? r : tmem_cap;
        if (r < 1) return cudaErrorInvalidConfiguration;
        per_sm = r;
    }
    const long long ntiles = (long long)c.N * ((c.H + G::TH - 1) / G::TH) * ((c.W + G::TW - 1) / G::TW);
    if (ntiles <= 0) return cudaSuccess;
    TailArgs ta;
    std::memset(&ta, 0, sizeof(ta));
    ta.c = c;
    ta.c2 = c2;
    cudaError_t e = make_tmap(&ta.tm, c.x, CIN, c.W, c.H, c.N, G::SW, G::SH);
    if (e != cudaSuccess) return e;
    const long long cap = (long long)per_sm * n_sm;
    kern<<<(int)(ntiles < cap ? ntiles : cap), kWsThreads, smem, st>>>(ta);
    return cudaGetLastError();
}

// Launch of the parity-class decoder convolution (a.x = lo, a.x2 = skip; H, W even);
// residency computed as for conv_ws_launch.
template <int CA, int CB, int COUT, int NBUF>
cudaError_t conv_up_launch(const ConvArgs &a, cudaStream_t st)
{
    using G = UpGeom<CA, CB, COUT, NBUF>;
    constexpr int kSmemPerSm = 228 * 1024, kReservedPerCta = 1024, kThreadsPerSm = 2048;
    constexpr int tmem_cap = 512 / G::COLS;
    constexpr int min_smem = tmem_cap < kThreadsPerSm / kWsThreads ? kSmemPerSm / tmem_cap - kReservedPerCta - 256 : 0;
    constexpr size_t smem = (size_t)(G::SMEM > min_smem ? G::SMEM : min_smem);
    static_assert(smem <= 227 * 1024, "decoder conv stage does not fit in shared memory");
    auto kern = conv_up_kernel<CA, CB, COUT, NBUF>;
    static int per_sm = 0, n_sm = 0;
    if (per_sm == 0) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
        cudaFuncAttributes fa;
        if ((e = cudaFuncGetAttributes(&fa, kern)) != cudaSuccess) return e;
        int dev = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        const int regs_per_warp = (fa.numRegs * 32 + 255) / 256 * 256;
        const int by_regs = (4 * (16384 / regs_per_warp)) / (kWsThreads / 32);
        const int by_smem = kSmemPerSm / ((int)smem + (int)fa.sharedSizeBytes + kReservedPerCta);
        int r = kThreadsPerSm / kWsThreads;
        r = r < by_regs ? r : by_regs;
        r = r < by_smem ? r : by_smem;
        r = r < tmem_cap ? r : tmem_cap;
        if (r < 1) return cudaErrorInvalidConfiguration;
        per_sm = r;
    }
    if ((a.H | a.W) & 1) return cudaErrorInvalidValue;
    const long long ntiles = (long long)a.N * ((a.H / 2 + 15) / 16) * ((a.W / 2 + 7) / 8);
    if (ntiles <= 0) return cudaSuccess;
    UpArgs ua;
    std::memset(&ua, 0, sizeof(ua));
    ua.c = a;
    cudaError_t e = make_tmap(&ua.tlo, a.x, CA, a.W / 2, a.H / 2, a.N, G::SW, G::SH);
    if (e != cudaSuccess) return e;
    if ((e = make_tmap_parity(&ua.tskip, a.x2, CB, a.W, a.H, a.N, G::SW, G::SH)) != cudaSuccess) return e;
    const long long cap = (long long)per_sm * n_sm;
    kern<<<(int)(ntiles < cap ? ntiles : cap), kWsThreads, smem, st>>>(ua);
    return cudaGetLastError();
}

// Launch of the stride-2 convolution (a.H, a.W: the input's size, both even; output at half
// size); residency computed as for conv_ws_launch.
template <int CIN, int COUT, int NBUF>
cudaError_t conv_s2_launch(const ConvArgs &a, cudaStream_t st)
{
    using G = S2Geom<CIN, COUT, NBUF>;
    constexpr int kSmemPerSm = 228 * 1024, kReservedPerCta = 1024, kThreadsPerSm = 2048;
    constexpr int tmem_cap = 512 / G::COLS;
    constexpr int min_smem = tmem_cap < kThreadsPerSm / kWsThreads ? kSmemPerSm / tmem_cap - kReservedPerCta - 256 : 0;
    constexpr size_t smem = (size_t)(G::SMEM > min_smem ? G::SMEM : min_smem);
    static_assert(smem <= 227 * 1024, "stride-2 conv stage does not fit in shared memory");
    auto kern = conv_s2_kernel<CIN, COUT, NBUF>;
    static int per_sm = 0, n_sm = 0;
    if (per_sm == 0) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
        cudaFuncAttributes fa;
        if ((e = cudaFuncGetAttributes(&fa, kern)) != cudaSuccess) return e;
        int dev = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        const int regs_per_warp = (fa.numRegs * 32 + 255) / 256 * 256;
        const int by_regs = (4 * (16384 / regs_per_warp)) / (kWsThreads / 32);
        const int by_smem = kSmemPerSm / ((int)smem + (int)fa.sharedSizeBytes + kReservedPerCta);
        int r = kThreadsPerSm / kWsThreads;
        r = r < by_regs ? r : by_regs;
        r = r < by_smem ? r : by_smem;
        r = r < tmem_cap ? r : tmem_cap;
        if (r < 1) return cudaErrorInvalidConfiguration;
        per_sm = r;
    }
    if ((a.H | a.W) & 1) return cudaErrorInvalidValue;
    const long long ntiles = (long long)a.N * ((a.H / 2 + G::TH - 1) / G::TH) * ((a.W / 2 + G::TW - 1) / G::TW);
    if (ntiles <= 0) return cudaSuccess;
    S2Args sa;
    std::memset(&sa, 0, sizeof(sa));
    sa.c = a;
    cudaError_t e = make_tmap_parity(&sa.te, a.x, CIN, a.W, a.H, a.N, G::WE, G::SH);
    if (e != cudaSuccess) return e;
    if ((e = make_tmap_parity(&sa.to, a.x, CIN, a.W, a.H, a.N, G::WO, G::SH)) != cudaSuccess) return e;
    const long long cap = (long long)per_sm * n_sm;
    kern<<<(int)(ntiles < cap ? ntiles : cap), kWsThreads, smem, st>>>(sa);
    return cudaGetLastError();
}

// Launch of the tensor-core weight gradient: one CTA per resident slot, each over a
// contiguous range of 8 x 8 pixel tiles.  Residency as for conv_ws_launch: the shared-memory
// request is raised where needed so that no more CTAs than tensor memory can hold share an SM.
template <int CIN, int COUT, int KS>
cudaError_t wgrad_launch(const bf16 *x, const bf16 *dz, float *gw, int N, int H, int W, int cin_true, int cout_true,
                         float *part, size_t part_floats, int *status, cudaStream_t st)
{
    using G = WgGeom<CIN, COUT, KS>;
    constexpr int kSmemPerSm = 228 * 1024, kReservedPerCta = 1024, kThreads = 128, kThreadsPerSm = 2048;
    constexpr int tmem_cap = 512 / G::COLS;
    constexpr int min_smem = tmem_cap < kThreadsPerSm / kThreads ? kSmemPerSm / tmem_cap - kReservedPerCta - 256 : 0;
    constexpr size_t smem = (size_t)(G::SMEM > min_smem ? G::SMEM : min_smem);
    static_assert(smem <= 227 * 1024, "weight-gradient tile does not fit in shared memory");
    auto kern = wgrad_tc_kernel<CIN, COUT, KS>;
    static int per_sm = 0, n_sm = 0;
    if (per_sm == 0) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
        cudaFuncAttributes fa;
        if ((e = cudaFuncGetAttributes(&fa, kern)) != cudaSuccess) return e;
        int dev = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        const int regs_per_warp = (fa.numRegs * 32 + 255) / 256 * 256;
        const int by_regs = (4 * (16384 / regs_per_warp)) / (kThreads / 32);
        const int by_smem = kSmemPerSm / ((int)smem + (int)fa.sharedSizeBytes + kReservedPerCta);
        int r = kThreadsPerSm / kThreads;
        r = r < by_regs ? r : by_regs;
        r = r < by_smem ? r : by_smem;
        r = r < tmem_cap ? r : tmem_cap;
        if (r < 1) return cudaErrorInvalidConfiguration;
        per_sm = r;
    }
    const long long ntiles = (long long)N * ((H + 7) / 8) * ((W + 7) / 8);
    if (ntiles <= 0) return cudaSuccess;
    long long slots = (long long)per_sm * n_sm;
    const long long fit = (long long)(part_floats / ((size_t)G::M * COUT));  // partial slots the buffer holds
    if (slots > fit) slots = fit;
    if (slots < 1) return cudaErrorInvalidValue;
    const long long ctas = ntiles < slots ? ntiles : slots;
    WgradArgs a{x, dz, gw, part, N, H, W, cin_true, cout_true, (int)((ntiles + ctas - 1) / ctas), status};
    const long long grid = (ntiles + a.tiles_per_cta - 1) / a.tiles_per_cta;
    kern<<<(int)grid, kThreads, smem, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // one warp per CTA: the M COUT chains of additions spread over as many SMs as they fill
    wgrad_reduce_kernel<CIN, COUT, KS><<<(KS * KS * CIN * COUT + 31) / 32, 32, 0, st>>>(part, (int)grid, gw, cin_true,
                                                                                       cout_true);
    return cudaGetLastError();
}

}  // namespace
}  // namespace flnr

// =========================================================================================
// The network object behind flnr_*.

struct flnr_net {
    int max_pix = 0;  // N * H * W the activation buffers hold
    int n_sm = 0;
    int nout = 8;     // output channels of the head o1: 8, or 16 (model and map guide sets)
    size_t nparam = 0;
    size_t poff[flnr::kNL][2];  // offsets of each layer's weights and bias in the flat arrays
    float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;  // master fp32, grads, Adam moments
    __nv_bfloat16 *wf[flnr::kNL] = {}, *wd[flnr::kNL] = {};          // bf16 forward / dgrad weights
    std::vector<void *> bufs;
    // activations (bf16 NHWC) and gradients
    __nv_bfloat16 *x0, *a0, *f0, *a1, *f1, *a2, *f2, *c1, *a3, *d1, *c0, *a4, *d0, *a5;
    __nv_bfloat16 *gA, *gB, *gC, *gLo;  // gradient scratch (largest: 48 channels at full res)
    float *gskip0, *gskip1;             // skip gradients (fp32)
    float *wpart = nullptr;             // per-CTA partial weight gradients (fixed-order reduction)
    size_t wpart_floats = 0;
    float *out = nullptr;               // last forward output, planar fp32 [N][8][H][W]
    int *status = nullptr;              // device status word of the tensor-core kernels
    int N = 0, H = 0, W = 0;            // shape of the last forward
    bool weights_fresh = false;
};

namespace {

template <typename T>
int nalloc(flnr_net *n, T **p, size_t count)
{
    void *q = nullptr;
    if (cudaMalloc(&q, count * sizeof(T)) != cudaSuccess) return FLR_ERR_NOMEM;
    n->bufs.push_back(q);
    *p = (T *)q;
    return FLR_OK;
}

// layer l's true sizes in a network with `nout` head outputs
flnr::LayerDef layer_def(int nout, int l)
{
    flnr::LayerDef d = flnr::kLayers[l];
    if (l == flnr::kNL - 1) d.cout = nout;
    return d;
}

cudaError_t refresh_weights(flnr_net *n, cudaStream_t st)
{
    for (int l = 0; l < flnr::kNL; ++l) {
        const auto d = layer_def(n->nout, l);
        const int cinp = flnr::pad16(d.cin), coutp = flnr::pad16(d.cout);
        const int total = d.k * d.k * cinp * coutp;
        flnr::weights_kernel<<<(total + 255) / 256, 256, 0, st>>>(n->w + n->poff[l][0], n->wf[l], n->wd[l], d.cin,
                                                                   d.cout, cinp, coutp, d.k);
    }
    n->weights_fresh = true;
    return cudaGetLastError();
}

}  // namespace

extern "C" {

size_t flnr_param_count(int outputs)
{
    if (outputs != 8 && outputs != 16) return 0;
    size_t s = 0;
    for (int l = 0; l < flnr::kNL; ++l) {
        const auto d = layer_def(outputs, l);
        s += (size_t)d.cout * d.cin * d.k * d.k + d.cout;
    }
    return s;
}

int flnr_create(int max_pixels, int outputs, flnr_net **out)
{
    if (!out || max_pixels <= 0 || (outputs != 8 && outputs != 16)) return FLR_ERR_ARG;
    *out = nullptr;
    flnr_net *n = new (std::nothrow) flnr_net();
    if (!n) return FLR_ERR_NOMEM;
    n->max_pix = max_pixels;
    n->nout = outputs;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n->n_sm, cudaDevAttrMultiProcessorCount, dev);
    size_t off = 0;
    for (int l = 0; l < flnr::kNL; ++l) {
        const auto d = layer_def(outputs, l);
        n->poff[l][0] = off;
        off += (size_t)d.cout * d.cin * d.k * d.k;
        n->poff[l][1] = off;
        off += d.cout;
    }
    n->nparam = off;
    const size_t P = (size_t)max_pixels, P2 = P / 4 + 1, P4 = P / 16 + 1;
    int st = FLR_OK;
    st |= nalloc(n, &n->w, off) | nalloc(n, &n->g, off) | nalloc(n, &n->m, off) | nalloc(n, &n->v, off);
    for (int l = 0; l < flnr::kNL && st == FLR_OK; ++l) {
        const auto &d = flnr::kLayers[l];
        const size_t e = (size_t)d.k * d.k * flnr::pad16(d.cin) * flnr::pad16(d.cout);
        st |= nalloc(n, &n->wf[l], e) | nalloc(n, &n->wd[l], e);
    }
    st |= nalloc(n, &n->x0, P * 16) | nalloc(n, &n->a0, P * 16) | nalloc(n, &n->f0, P * 16);
    st |= nalloc(n, &n->a1, P * 32) | nalloc(n, &n->f1, P2 * 32);
    st |= nalloc(n, &n->a2, P2 * 64) | nalloc(n, &n->f2, P4 * 64) | nalloc(n, &n->c1, P2 * 96);
    st |= nalloc(n, &n->a3, P2 * 32) | nalloc(n, &n->d1, P2 * 32) | nalloc(n, &n->c0, P * 48);
    st |= nalloc(n, &n->a4, P * 16) | nalloc(n, &n->d0, P * 16) | nalloc(n, &n->a5, P * 16);
    st |= nalloc(n, &n->gA, P * 48) | nalloc(n, &n->gB, P * 48) | nalloc(n, &n->gC, P * 48) | nalloc(n, &n->gLo, P * 16);
    st |= nalloc(n, &n->gskip0, P * 16) | nalloc(n, &n->gskip1, P2 * 32) | nalloc(n, &n->out, P * 16);
    st |= nalloc(n, &n->status, 1);
    // partial weight gradients: two CTAs per SM of the largest layer (e2b, 9 * 64 x 64)
    n->wpart_floats = 2 * (size_t)n->n_sm * 9 * 64 * 64;
    st |= nalloc(n, &n->wpart, n->wpart_floats);
    if (st != FLR_OK) {
        flnr_destroy(n);
        return FLR_ERR_NOMEM;
    }
    cudaMemset(n->status, 0, sizeof(int));
    cudaMemset(n->g, 0, off * sizeof(float));
    cudaMemset(n->m, 0, off * sizeof(float));
    cudaMemset(n->v, 0, off * sizeof(float));
    *out = n;
    return FLR_OK;
}

int flnr_destroy(flnr_net *n)
{
    if (!n) return FLR_OK;
    cudaDeviceSynchronize();
    for (void *p : n->bufs) cudaFree(p);
    delete n;
    return FLR_OK;
}

int flnr_set_weights(flnr_net *n, const float *host, size_t count)
{
    if (!n || !host || count != n->nparam) return FLR_ERR_ARG;
    if (cudaMemcpy(n->w, host, count * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) return FLR_ERR_CUDA;
    if (cudaMemset(n->m, 0, count * sizeof(float)) != cudaSuccess || cudaMemset(n->v, 0, count * sizeof(float)) != cudaSuccess)
        return FLR_ERR_CUDA;
    if (refresh_weights(n, nullptr) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) return FLR_ERR_CUDA;
    return FLR_OK;
}

int flnr_get_weights(flnr_net *n, float *host, size_t count)
{
    if (!n || !host || count != n->nparam) return FLR_ERR_ARG;
    return cudaMemcpy(host, n->w, count * sizeof(float), cudaMemcpyDeviceToHost) == cudaSuccess ? FLR_OK : FLR_ERR_CUDA;
}

int flnr_get_state(flnr_net *n, float *host, size_t count)
{
    if (!n || !host || count != 3 * n->nparam) return FLR_ERR_ARG;
    const size_t b = n->nparam * sizeof(float);
    if (cudaMemcpy(host, n->w, b, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(host + n->nparam, n->m, b, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(host + 2 * n->nparam, n->v, b, cudaMemcpyDeviceToHost) != cudaSuccess)
        return FLR_ERR_CUDA;
    return FLR_OK;
}

int flnr_set_state(flnr_net *n, const float *host, size_t count)
{
    if (!n || !host || count != 3 * n->nparam) return FLR_ERR_ARG;
    const size_t b = n->nparam * sizeof(float);
    if (cudaMemcpy(n->w, host, b, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(n->m, host + n->nparam, b, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(n->v, host + 2 * n->nparam, b, cudaMemcpyHostToDevice) != cudaSuccess)
        return FLR_ERR_CUDA;
    if (refresh_weights(n, nullptr) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) return FLR_ERR_CUDA;
    return FLR_OK;
}

int flnr_get_grads(flnr_net *n, float *host, size_t count)
{
    if (!n || !host || count != n->nparam) return FLR_ERR_ARG;
    return cudaMemcpy(host, n->g, count * sizeof(float), cudaMemcpyDeviceToHost) == cudaSuccess ? FLR_OK : FLR_ERR_CUDA;
}

int flnr_zero_grads(flnr_net *n, void *stream)
{
    if (!n) return FLR_ERR_ARG;
    return cudaMemsetAsync(n->g, 0, n->nparam * sizeof(float), (cudaStream_t)stream) == cudaSuccess ? FLR_OK : FLR_ERR_CUDA;
}

#define FLNR_TRY(x)                                 \
    do {                                            \
        if ((x) != cudaSuccess) return FLR_ERR_CUDA; \
    } while (0)

int flnr_guide_forward(flnr_net *n, const float *in, float *guide_out, int N, int H, int W, void *stream)
{
    using namespace flnr;
    if (!n || !in || N <= 0 || H <= 0 || W <= 0 || (H % 4) || (W % 4)) return FLR_ERR_ARG;
    if ((long long)N * H * W > n->max_pix) return FLR_ERR_UNSUPPORTED;
    if (!n->weights_fresh) return FLR_ERR_ARG;  // flnr_set_weights first
    cudaStream_t st = (cudaStream_t)stream;
    n->N = N;
    n->H = H;
    n->W = W;
    const size_t P = (size_t)N * H * W;
    const int H2 = H / 2, W2 = W / 2;
    auto bias = [&](int l) { return n->w + n->poff[l][1]; };
    pack_input_kernel<<<egrid(P), 256, 0, st>>>(in, n->x0, N, H, W);
    FLNR_TRY(cudaGetLastError());
    const ConvArgs z{};
    auto conv = [&](const __nv_bfloat16 *x, int l, __nv_bfloat16 *y, int h, int w) {
        ConvArgs c = z;
        c.x = x; c.w = n->wf[l]; c.bias = bias(l); c.y = y; c.N = N; c.H = h; c.W = w;
        c.ystride = pad16(kLayers[l].cout); c.nbias = layer_def(n->nout, l).cout; c.status = n->status;
        return c;
    };
    ConvArgs c;
    // in0 and in1 in one pass (a0, which the backward pass reads, is still stored)
    FLNR_TRY((conv_tail_launch<16, 16, 3, 16, 1, 0>(conv(n->x0, 0, n->a0, H, W), conv(n->a0, 1, n->f0, H, W), st)));
    // encoder blocks: a 3x3 convolution, then a stride-2 one (sizes passed: the input's)
    FLNR_TRY((conv_ws_launch<16, 32, 3, 1, 0>(conv(n->f0, 2, n->a1, H, W), st)));
    FLNR_TRY((conv_s2_launch<32, 32, 2>(conv(n->a1, 3, n->f1, H, W), st)));
    FLNR_TRY((conv_ws_launch<32, 64, 3, 1, 0>(conv(n->f1, 4, n->a2, H2, W2), st)));
    FLNR_TRY((conv_s2_launch<64, 64, 2>(conv(n->a2, 5, n->f2, H2, W2), st)));
    c = conv(n->f2, 6, n->a3, H2, W2);  // input up(f2) ++ f1, formed while staging
    c.x2 = n->f1;
    FLNR_TRY((conv_up_launch<64, 32, 32, 2>(c, st)));
    FLNR_TRY((conv_ws_launch<32, 32, 3, 1, 0>(conv(n->a3, 7, n->d1, H2, W2), st)));
    c = conv(n->d1, 8, n->a4, H, W);  // input up(d1) ++ f0
    c.x2 = n->f0;
    FLNR_TRY((conv_up_launch<32, 16, 16, 2>(c, st)));
    FLNR_TRY((conv_ws_launch<16, 16, 3, 1, 0>(conv(n->a4, 9, n->d0, H, W), st)));
    float *yf = guide_out ? guide_out : n->out;
    c = conv(n->a5, 11, nullptr, H, W);
    c.yf = yf;
    // o0 and the head o1 (sigmoid into planar FP32) in one pass; a5 is still stored
    FLNR_TRY((conv_tail_launch<16, 16, 3, 16, 2, 1>(conv(n->d0, 10, n->a5, H, W), c, st)));
    if (guide_out)
        FLNR_TRY(cudaMemcpyAsync(n->out, guide_out, P * n->nout * sizeof(float), cudaMemcpyDeviceToDevice, st));
    return FLR_OK;
}

int flnr_guide_backward(flnr_net *n, const float *grad_out, float *grad_in, void *stream)
{
    using namespace flnr;
    if (!n || !grad_out || n->N <= 0) return FLR_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int N = n->N, H = n->H, W = n->W, H2 = H / 2, W2 = W / 2, H4 = H / 4, W4 = W / 4;
    const size_t P = (size_t)N * H * W;
    auto gw = [&](int l) { return n->g + n->poff[l][0]; };
    auto gb = [&](int l) { return n->g + n->poff[l][1]; };
    auto bgrad = [&](const __nv_bfloat16 *dz, long long pix, int C, int ctrue, int l) {
        bias_part_kernel<<<8 * C, 32, 0, st>>>(dz, n->wpart, pix, C);  // 256 C threads; wpart is free between layers
        bias_tree_kernel<<<ctrue, 256, 0, st>>>(n->wpart, gb(l), C);
    };
    // output head: sigmoid, o1 (1x1, 16 -> 8 padded to 16), o0
    sigmoid_bwd_kernel<<<egrid(P), 256, 0, st>>>(grad_out, n->out, n->gA, N, H, W, n->nout);
    FLNR_TRY((wgrad_launch<16, 16, 1>(n->a5, n->gA, gw(11), N, H, W, 16, n->nout, n->wpart, n->wpart_floats, n->status, st)));
    bgrad(n->gA, (long long)P, 16, n->nout, 11);
    FLNR_TRY((dgrad_launch<16, 16, 1, true>({n->gA, n->wd[11], n->a5, nullptr, n->gB, nullptr, N, H, W, 16}, n->status, st)));
    FLNR_TRY((wgrad_launch<16, 16, 3>(n->d0, n->gB, gw(10), N, H, W, 16, 16, n->wpart, n->wpart_floats, n->status, st)));
    bgrad(n->gB, (long long)P, 16, 16, 10);
    FLNR_TRY((dgrad_launch<16, 16, 3, true>({n->gB, n->wd[10], n->d0, nullptr, n->gA, nullptr, N, H, W, 16}, n->status, st)));
    // decoder level 0
    FLNR_TRY((wgrad_launch<16, 16, 3>(n->a4, n->gA, gw(9), N, H, W, 16, 16, n->wpart, n->wpart_floats, n->status, st)));
    bgrad(n->gA, (long long)P, 16, 16, 9);
    FLNR_TRY((dgrad_launch<16, 16, 3, true>({n->gA, n->wd[9], n->a4, nullptr, n->gB, nullptr, N, H, W, 16}, n->status, st)));
    upcat_kernel<<<egrid(P * 6), 256, 0, st>>>(n->d1, n->f0, n->c0, N, H, W, 32, 16);  // d0a's input
    FLNR_TRY(cudaGetLastError());
    FLNR_TRY((wgrad_launch<48, 16, 3>(n->c0, n->gB, gw(8), N, H, W, 48, 16, n->wpart, n->wpart_floats, n->status, st)));
    bgrad(n->gB, (long long)P, 16, 16, 8);
    FLNR_TRY((dgrad_launch<16, 48, 3, false>({n->gB, n->wd[8], nullptr, nullptr, n->gC, nullptr, N, H, W, 48}, n->status, st)));
    upcat_bwd_kernel<<<egrid(P * 48 / 8), 256, 0, st>>>(n->gC, n->d1, n->gLo, n->gskip0, N, H, W, 32, 16);  // gLo = dz(d1b)
    // decoder level 1 (H/2)
    const size_t P2 = P / 4;
    FLNR_TRY((wgrad_launch<32, 32, 3>(n->a3, n->gLo, gw(7), N, H2, W2, 32, 32, n->wpart, n->wpart_floats, n->status, st)));
    bgrad(n->gLo, (long long)P2, 32, 32, 7);
    FLNR_TRY((dgrad_launch<32, 32, 3, true>({n->gLo, n->wd[7], n->a3, nullptr, n->gA, nullptr, N, H2, W2, 32}, n->status, st)));
    upcat_kernel<<<egrid(P2 * 12), 256, 0, st>>>(n->f2, n->f1, n->c1, N, H2, W2, 64, 32);  // d1a's input
    FLNR_TRY(cudaGetLastError());
    FLNR_TRY((wgrad_launch<96, 32, 3>(n->c1, n->gA, gw(6), N, H2, W2, 96, 32, n->wpart, n->wpart_floats, n->status, st)));
    bgrad(n->gA, (long long)P2, 32, 32, 6);
    FLNR_TRY((dgrad_launch<32, 96, 3, false>({n->gA, n->wd[6], nullptr, nullptr, n->gC, nullptr, N, H2, W2, 96}, n->status, st)));
    upcat_bwd_kernel<<<egrid(P2 * 96 / 8), 256, 0, st>>>(n->gC, n->f2, n->gLo, n->gskip1, N, H2, W2, 64, 32);  // gLo = dz(e2b)
    // encoder level 2: e2b (stride 2, H/2 -> H/4), then e2a (H/2).  A stride-2 layer's
    // gradients are those of the stride-1 kernels at its input's size on dz zero-upsampled
    // onto that grid.
    const size_t P4 = P / 16;
    bgrad(n->gLo, (long long)P4, 64, 64, 5);
    join_bwd_kernel<2><<<egrid(P2 * 64 / 8), 256, 0, st>>>(nullptr, n->gLo, nullptr, n->gB, N, H4, W4, 64);
    FLNR_TRY(cudaGetLastError());
    FLNR_TRY((wgrad_launch<64, 64, 3>(n->a2, n->gB, gw(5), N, H2, W2, 64, 64, n->wpart, n->wpart_floats, n->status, st)));
    FLNR_TRY((dgrad_launch<64, 64, 3, true>({n->gB, n->wd[5], n->a2, nullptr, n->gA, nullptr, N, H2, W2, 64}, n->status, st)));
    FLNR_TRY((wgrad_launch<32, 64, 3>(n->f1, n->gA, gw(4), N, H2, W2, 32, 64, n->wpart, n->wpart_floats, n->status, st)));
    bgrad(n->gA, (long long)P2, 64, 64, 4);
    FLNR_TRY((dgrad_launch<64, 32, 3, false>({n->gA, n->wd[4], nullptr, nullptr, n->gB, nullptr, N, H2, W2, 32}, n->status, st)));
    // encoder level 1: e1b (stride 2, H -> H/2; f1 also feeds the d1a skip), then e1a (H)
    join_bwd_kernel<2><<<egrid(P * 32 / 8), 256, 0, st>>>(n->gskip1, n->gB, n->f1, n->gC, N, H2, W2, 32);
    FLNR_TRY(cudaGetLastError());
    FLNR_TRY((wgrad_launch<32, 32, 3>(n->a1, n->gC, gw(3), N, H, W, 32, 32, n->wpart, n->wpart_floats, n->status, st)));
    bgrad(n->gC, (long long)P, 32, 32, 3);
    FLNR_TRY((dgrad_launch<32, 32, 3, true>({n->gC, n->wd[3], n->a1, nullptr, n->gA, nullptr, N, H, W, 32}, n->status, st)));
    FLNR_TRY((wgrad_launch<16, 32, 3>(n->f0, n->gA, gw(2), N, H, W, 16, 32, n->wpart, n->wpart_floats, n->status, st)));
    bgrad(n->gA, (long long)P, 32, 32, 2);
    FLNR_TRY((dgrad_launch<32, 16, 3, false>({n->gA, n->wd[2], nullptr, nullptr, n->gB, nullptr, N, H, W, 16}, n->status, st)));
    join_bwd_kernel<1><<<egrid(P * 16 / 8), 256, 0, st>>>(n->gskip0, n->gB, n->f0, n->gLo, N, H, W, 16);  // dz(in1)
    // input projection (H)
    FLNR_TRY((wgrad_launch<16, 16, 1>(n->a0, n->gLo, gw(1), N, H, W, 16, 16, n->wpart, n->wpart_floats, n->status, st)));
    bgrad(n->gLo, (long long)P, 16, 16, 1);
    FLNR_TRY((dgrad_launch<16, 16, 1, true>({n->gLo, n->wd[1], n->a0, nullptr, n->gA, nullptr, N, H, W, 16}, n->status, st)));
    FLNR_TRY((wgrad_launch<16, 16, 3>(n->x0, n->gA, gw(0), N, H, W, 11, 16, n->wpart, n->wpart_floats, n->status, st)));
    bgrad(n->gA, (long long)P, 16, 16, 0);
    if (grad_in) {  // through in0 to the packed input, then through the input transform
        FLNR_TRY((dgrad_launch<16, 16, 3, false>({n->gA, n->wd[0], nullptr, nullptr, n->gB, nullptr, N, H, W, 16}, n->status, st)));
        unpack_grad_kernel<<<egrid(P), 256, 0, st>>>(n->gB, n->x0, grad_in, N, H, W);
    }
    return cudaGetLastError() == cudaSuccess ? FLR_OK : FLR_ERR_CUDA;
}

}  // extern "C"

namespace {

// One layer's kernels by themselves (flnr_layer): CI / CO are the padded channel counts, CA
// the upsampled part of a decoder input, S2 whether the layer strides by 2 (N, H, W: the
// layer's input size).
template <int CI, int CO, int KS, int CA, bool S2, bool HEAD = false>
int layer_ops(flnr_net *n, int l, int op, const void *a, const void *b, const void *mask, void *out, int N, int H,
              int W, cudaStream_t st)
{
    using namespace flnr;
    using bf = __nv_bfloat16;
    const auto d = layer_def(n->nout, l);
    const long long P = (long long)N * H * W;
    if (op == FLNR_OP_FORWARD) {
        ConvArgs c{};
        c.x = (const bf *)a;
        c.w = n->wf[l];
        c.bias = n->w + n->poff[l][1];
        c.N = N;
        c.H = H;
        c.W = W;
        c.ystride = CO;
        c.nbias = d.cout;
        c.status = n->status;
        if constexpr (HEAD) {
            c.yf = (float *)out;
            FLNR_TRY((conv_ws_launch<CI, CO, KS, 2, 1>(c, st)));
        } else {
            c.y = (bf *)out;
            if constexpr (CA > 0) {
                if (b) {
                    if ((H | W) & 1) return FLR_ERR_ARG;
                    c.x2 = (const bf *)b;
                    FLNR_TRY((conv_up_launch<CA, CI - CA, CO, 2>(c, st)));
                    return FLR_OK;
                }
            }
            if constexpr (S2) {
                if ((H | W) & 1) return FLR_ERR_ARG;
                FLNR_TRY((conv_s2_launch<CI, CO, 2>(c, st)));
            } else {
                FLNR_TRY((conv_ws_launch<CI, CO, KS, 1, 0>(c, st)));
            }
        }
        return FLR_OK;
    }
    const bf *dz = (const bf *)(op == FLNR_OP_DGRAD ? a : b);
    if constexpr (S2) {  // dz [N][H/2][W/2][CO], zero-upsampled onto the input grid in scratch
        if ((H | W) & 1) return FLR_ERR_ARG;
        if (P * CO > (long long)n->max_pix * 48) return FLR_ERR_UNSUPPORTED;
        join_bwd_kernel<2><<<egrid((size_t)P * CO / 8), 256, 0, st>>>(nullptr, dz, nullptr, n->gC, N, H / 2, W / 2, CO);
        FLNR_TRY(cudaGetLastError());
        dz = n->gC;
    }
    if (op == FLNR_OP_DGRAD) {
        if (mask)
            FLNR_TRY((dgrad_launch<CO, CI, KS, true>({dz, n->wd[l], (const bf *)mask, nullptr, (bf *)out, nullptr, N, H, W, CI}, n->status, st)));
        else
            FLNR_TRY((dgrad_launch<CO, CI, KS, false>({dz, n->wd[l], nullptr, nullptr, (bf *)out, nullptr, N, H, W, CI}, n->status, st)));
    } else {
        FLNR_TRY((wgrad_launch<CI, CO, KS>((const bf *)a, dz, n->g + n->poff[l][0], N, H, W, d.cin, d.cout, n->wpart, n->wpart_floats, n->status, st)));
        bias_part_kernel<<<8 * CO, 32, 0, st>>>(dz, n->wpart, P, CO);
        bias_tree_kernel<<<d.cout, 256, 0, st>>>(n->wpart, n->g + n->poff[l][1], CO);
        FLNR_TRY(cudaGetLastError());
    }
    return FLR_OK;
}

}  // namespace

extern "C" {

int flnr_layer(flnr_net *n, int layer, int op, const void *a, const void *b, const void *mask, void *out, int N,
               int H, int W, void *stream)
{
    if (!n || layer < 0 || layer >= flnr::kNL || op < FLNR_OP_FORWARD || op > FLNR_OP_WGRAD || !a || N <= 0 ||
        H <= 0 || W <= 0)
        return FLR_ERR_ARG;
    if ((op == FLNR_OP_WGRAD && !b) || (op != FLNR_OP_WGRAD && !out)) return FLR_ERR_ARG;
    if ((long long)N * H * W > 0x7fffffffLL) return FLR_ERR_ARG;
    if (!n->weights_fresh) return FLR_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    switch (layer) {
    case 0: return layer_ops<16, 16, 3, 0, false>(n, 0, op, a, b, mask, out, N, H, W, st);
    case 1: return layer_ops<16, 16, 1, 0, false>(n, 1, op, a, b, mask, out, N, H, W, st);
    case 2: return layer_ops<16, 32, 3, 0, false>(n, 2, op, a, b, mask, out, N, H, W, st);
    case 3: return layer_ops<32, 32, 3, 0, true>(n, 3, op, a, b, mask, out, N, H, W, st);
    case 4: return layer_ops<32, 64, 3, 0, false>(n, 4, op, a, b, mask, out, N, H, W, st);
    case 5: return layer_ops<64, 64, 3, 0, true>(n, 5, op, a, b, mask, out, N, H, W, st);
    case 6: return layer_ops<96, 32, 3, 64, false>(n, 6, op, a, b, mask, out, N, H, W, st);
    case 7: return layer_ops<32, 32, 3, 0, false>(n, 7, op, a, b, mask, out, N, H, W, st);
    case 8: return layer_ops<48, 16, 3, 32, false>(n, 8, op, a, b, mask, out, N, H, W, st);
    case 9: return layer_ops<16, 16, 3, 0, false>(n, 9, op, a, b, mask, out, N, H, W, st);
    case 10: return layer_ops<16, 16, 3, 0, false>(n, 10, op, a, b, mask, out, N, H, W, st);
    default: return layer_ops<16, 16, 1, 0, false, true>(n, 11, op, a, b, mask, out, N, H, W, st);
    }
}

int flnr_status(flnr_net *n)
{
    if (!n) return FLR_ERR_ARG;
    int h = 0;
    if (cudaDeviceSynchronize() != cudaSuccess) return FLR_ERR_CUDA;
    if (cudaMemcpy(&h, n->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return FLR_ERR_CUDA;
    if (h != 0 && cudaMemset(n->status, 0, sizeof(int)) != cudaSuccess) return FLR_ERR_CUDA;
    return h ? FLR_ERR_TIMEOUT : FLR_OK;
}

int flnr_adam_step(flnr_net *n, float lr, float beta1, float beta2, float eps, int step, void *stream)
{
    if (!n || step < 1 || !(lr >= 0.f)) return FLR_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
    flnr::adam_kernel<<<flnr::egrid(n->nparam), 256, 0, st>>>(n->w, n->g, n->m, n->v, n->nparam, lr, beta1, beta2, eps, c1, c2);
    FLNR_TRY(cudaGetLastError());
    FLNR_TRY(refresh_weights(n, st));
    return FLR_OK;
}

int flnr_l1_loss(const float *pred, const float *ref, float *grad, float *loss, size_t count, void *stream)
{
    if (!pred || !ref || !grad || !loss || count == 0) return FLR_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    FLNR_TRY(cudaMemsetAsync(loss, 0, sizeof(float), st));
    flnr::l1_kernel<<<flnr::egrid(count) < 1024 ? flnr::egrid(count) : 1024, 256, 0, st>>>(pred, ref, grad, loss, count);
    return cudaGetLastError() == cudaSuccess ? FLR_OK : FLR_ERR_CUDA;
}

int flnr_smape_loss(const float *pred, const float *ref, float *grad, float *loss, size_t count, float eps, void *stream)
{
    if (!pred || !ref || !grad || !loss || count == 0 || !(eps > 0.f)) return FLR_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    FLNR_TRY(cudaMemsetAsync(loss, 0, sizeof(float), st));
    flnr::smape_kernel<<<flnr::egrid(count) < 1024 ? flnr::egrid(count) : 1024, 256, 0, st>>>(pred, ref, grad, loss, count,
                                                                                                 eps);
    return cudaGetLastError() == cudaSuccess ? FLR_OK : FLR_ERR_CUDA;
}

}  // extern "C"
