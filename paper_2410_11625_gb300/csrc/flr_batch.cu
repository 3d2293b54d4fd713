// flr_batch.cu -- batched fast FLR / joint denoising and upsampling (Sec. 3.2, 3.2.1) in
// one persistent cooperative launch, and the batched per-pixel entry point.
//
// A serving step denoises several frames of mixed sizes at once.  Instead of four launches
// per frame, one persistent kernel (one CTA per SM, co-resident by cooperative launch)
// walks the work items of every frame stage by stage: block moments, horizontal blur,
// vertical blur + solve, interpolation + apply, with a grid barrier between stages.  The
// frame table travels in the kernel parameters, so a captured CUDA graph replays the whole
// batch with one kernel node.  Every barrier wait is bounded in time: a wait that runs out
// records FLR_BATCH_TIMEOUT in a status word and the kernel carries on to its end, so the
// device never hangs and flr_fast_batch_status reports the failure.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <vector>

#include "flr.h"
#include "flr_fast_stages.cuh"

namespace flr {
namespace {

using fast::FastArgs;

constexpr int kMaxBatch = FLR_MAX_BATCH;
constexpr int kBatchThreads = 256;
constexpr unsigned long long kBarrierTimeoutNs = 2000000000ull;  // 2 s per barrier

struct BatchArgs {
    FastArgs f[kMaxBatch];
    int n;
    unsigned long long off[4][kMaxBatch + 1];  // prefix sums of each stage's work items
    unsigned *bar_count, *bar_gen;
    int *status;
    unsigned long long timeout_ns;
};

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier for co-resident CTAs, bounded in time.  Returns false (and records the
// timeout in *status) if the other CTAs did not all arrive within timeout_ns.
__device__ bool grid_barrier(unsigned *count, unsigned *gen, unsigned nblocks, int *status,
                             unsigned long long timeout_ns)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        const unsigned g = *(volatile unsigned *)gen;
        __threadfence();
        if (atomicAdd(count, 1u) == nblocks - 1) {
            atomicExch(count, 0u);
            __threadfence();
            atomicAdd(gen, 1u);
        } else {
            const unsigned long long t0 = global_ns();
            while (*(volatile unsigned *)gen == g) {
                if (global_ns() - t0 > timeout_ns) {
                    atomicExch(status, FLR_BATCH_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(256);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

__device__ __forceinline__ int frame_of(const unsigned long long *off, int n, unsigned long long item)
{
    int f = 0;
    while (f + 1 < n && item >= off[f + 1]) ++f;
    return f;
}

template <int Q, int F>
__global__ void __launch_bounds__(kBatchThreads, 1) flr_batch_kernel(const __grid_constant__ BatchArgs b)
{
    extern __shared__ float sS[];  // [NCH][kBatchThreads] for the solve stage
    const unsigned nblocks = gridDim.x;
    // stage 1: block moments; item -> (frame, block row, 512-column chunk)
    for (unsigned long long it = blockIdx.x; it < b.off[0][b.n]; it += gridDim.x) {
        const int f = frame_of(b.off[0], b.n, it);
        const FastArgs &a = b.f[f];
        const int chunks = fast::moment_chunks(a.Wi);
        const int local = (int)(it - b.off[0][f]);
        fast::stage_moments<Q, F>(a, local / chunks, local % chunks);
    }
    grid_barrier(b.bar_count, b.bar_gen, nblocks, b.status, b.timeout_ns);
    // stage 2: horizontal blur; item -> 256 blocks
    for (unsigned long long it = blockIdx.x; it < b.off[1][b.n]; it += gridDim.x) {
        const int f = frame_of(b.off[1], b.n, it);
        fast::stage_blur_h<Q>(b.f[f], (size_t)(it - b.off[1][f]) * kBatchThreads + threadIdx.x);
    }
    grid_barrier(b.bar_count, b.bar_gen, nblocks, b.status, b.timeout_ns);
    // stage 3: vertical blur + solve
    for (unsigned long long it = blockIdx.x; it < b.off[2][b.n]; it += gridDim.x) {
        const int f = frame_of(b.off[2], b.n, it);
        fast::stage_blur_v_solve<Q>(b.f[f], (size_t)(it - b.off[2][f]) * kBatchThreads + threadIdx.x,
                                    sS + threadIdx.x, kBatchThreads);
    }
    grid_barrier(b.bar_count, b.bar_gen, nblocks, b.status, b.timeout_ns);
    // stage 4: interpolation + apply; item -> 256 runs
    for (unsigned long long it = blockIdx.x; it < b.off[3][b.n]; it += gridDim.x) {
        const int f = frame_of(b.off[3], b.n, it);
        fast::stage_apply<Q>(b.f[f], (size_t)(it - b.off[3][f]) * kBatchThreads + threadIdx.x);
    }
}

// A barrier that waits for more CTAs than exist: every wait runs out.  Tests the bounded
// wait and the status path without any fault.
__global__ void barrier_selftest_kernel(unsigned *count, unsigned *gen, unsigned expected, int *status,
                                        unsigned long long timeout_ns)
{
    grid_barrier(count, gen, expected, status, timeout_ns);
}

template <int Q, int F>
cudaError_t launch_batch_qf(const BatchArgs &b, int grid, size_t smem, cudaStream_t st)
{
    cudaError_t e = cudaFuncSetAttribute(flr_batch_kernel<Q, F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kBatchThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, flr_batch_kernel<Q, F>, b);
}

template <int Q, int F>
cudaError_t batch_grid_qf(size_t smem, int *grid)
{
    cudaError_t e = cudaFuncSetAttribute(flr_batch_kernel<Q, F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0, dev = 0, n_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, flr_batch_kernel<Q, F>, kBatchThreads, smem)) != cudaSuccess)
        return e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    *grid = per_sm * n_sm;
    return *grid > 0 ? cudaSuccess : cudaErrorInvalidConfiguration;
}

#define FLR_QF_DISPATCH(q, F, ...)                                                  \
    switch ((q) * 16 + (F)) {                                                       \
    case 1 * 16 + 2: { constexpr int QQ = 1, FF = 2; __VA_ARGS__; }                 \
    case 1 * 16 + 4: { constexpr int QQ = 1, FF = 4; __VA_ARGS__; }                 \
    case 1 * 16 + 8: { constexpr int QQ = 1, FF = 8; __VA_ARGS__; }                 \
    case 4 * 16 + 2: { constexpr int QQ = 4, FF = 2; __VA_ARGS__; }                 \
    case 4 * 16 + 4: { constexpr int QQ = 4, FF = 4; __VA_ARGS__; }                 \
    case 4 * 16 + 8: { constexpr int QQ = 4, FF = 8; __VA_ARGS__; }                 \
    case 8 * 16 + 2: { constexpr int QQ = 8, FF = 2; __VA_ARGS__; }                 \
    case 8 * 16 + 4: { constexpr int QQ = 8, FF = 4; __VA_ARGS__; }                 \
    case 8 * 16 + 8: { constexpr int QQ = 8, FF = 8; __VA_ARGS__; }                 \
    default: break;                                                                 \
    }

}  // namespace

bool batch_supported(int q, int F)
{
    return (q == 1 || q == 4 || q == 8) && (F == 2 || F == 4 || F == 8);
}

cudaError_t launch_batch(int q, int F, const void *args, cudaStream_t st)
{
    const BatchArgs &b = *(const BatchArgs *)args;
    const size_t smem = sizeof(float) * (size_t)(q + 3 + q * (q + 1) / 2 + 3 * q) * kBatchThreads;
    int grid = 0;
    cudaError_t e = cudaErrorInvalidValue;
    FLR_QF_DISPATCH(q, F, e = batch_grid_qf<QQ, FF>(smem, &grid); if (e != cudaSuccess) return e;
                    return launch_batch_qf<QQ, FF>(b, grid, smem, st));
    return e;
}

size_t batch_args_size() { return sizeof(BatchArgs); }

cudaError_t launch_barrier_selftest(unsigned *count, unsigned *gen, unsigned expected, int *status,
                                    unsigned long long timeout_ns, int grid, cudaStream_t st)
{
    barrier_selftest_kernel<<<grid, 32, 0, st>>>(count, gen, expected, status, timeout_ns);
    return cudaGetLastError();
}

void fill_batch_args(void *args, int n, const fast::FastArgs *frames, unsigned *count, unsigned *gen, int *status)
{
    BatchArgs &b = *(BatchArgs *)args;
    std::memset(&b, 0, sizeof(b));
    b.n = n;
    for (int i = 0; i < n; ++i) b.f[i] = frames[i];
    for (int s = 0; s < 4; ++s) b.off[s][0] = 0;
    for (int i = 0; i < n; ++i) {
        b.off[0][i + 1] = b.off[0][i] + fast::items_moments(frames[i]);
        b.off[1][i + 1] = b.off[1][i] + fast::items_blocks(frames[i]);
        b.off[2][i + 1] = b.off[2][i] + fast::items_blocks(frames[i]);
        b.off[3][i + 1] = b.off[3][i] + fast::items_apply(frames[i]);
    }
    b.bar_count = count;
    b.bar_gen = gen;
    b.status = status;
    b.timeout_ns = kBarrierTimeoutNs;
}

}  // namespace flr
