// flr_tmem.cuh -- tensor-memory loads and stores of the FLR kernels (sm_103a): a warp moves
// 32 lanes x N 32-bit columns of its own lane quarter (tcgen05.ld / tcgen05.st, shape
// 32x32b), one lane per thread.  The kernels use tensor memory, which the tensor cores use
// for accumulators, as per-thread storage that survives between the phases of a batch.
#pragma once

#include <cstdint>

namespace flr {

// ---- tensor-memory access (32 lanes x 32 bits per warp, one lane per thread) ----------
#define FLR_TM_R4(i) "r"(v[i]), "r"(v[i + 1]), "r"(v[i + 2]), "r"(v[i + 3])
#define FLR_TM_W4(i) "=r"(v[i]), "=r"(v[i + 1]), "=r"(v[i + 2]), "=r"(v[i + 3])
__device__ __forceinline__ void tm_st32(uint32_t ta, const uint32_t *v)
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
        "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};\n" ::"r"(ta),
        FLR_TM_R4(0), FLR_TM_R4(4), FLR_TM_R4(8), FLR_TM_R4(12), FLR_TM_R4(16), FLR_TM_R4(20), FLR_TM_R4(24),
        FLR_TM_R4(28)
        : "memory");
}
__device__ __forceinline__ void tm_st16(uint32_t ta, const uint32_t *v)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};\n" ::"r"(
                     ta),
                 FLR_TM_R4(0), FLR_TM_R4(4), FLR_TM_R4(8), FLR_TM_R4(12)
                 : "memory");
}
__device__ __forceinline__ void tm_st8(uint32_t ta, const uint32_t *v)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};\n" ::"r"(ta), FLR_TM_R4(0),
                 FLR_TM_R4(4)
                 : "memory");
}
__device__ __forceinline__ void tm_st2(uint32_t ta, const uint32_t *v)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1,%2};\n" ::"r"(ta), "r"(v[0]), "r"(v[1]) : "memory");
}
__device__ __forceinline__ void tm_st1(uint32_t ta, uint32_t v0)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x1.b32 [%0], {%1};\n" ::"r"(ta), "r"(v0) : "memory");
}
__device__ __forceinline__ void tm_ld32(uint32_t ta, uint32_t *v)
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
        "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : FLR_TM_W4(0), FLR_TM_W4(4), FLR_TM_W4(8), FLR_TM_W4(12), FLR_TM_W4(16), FLR_TM_W4(20), FLR_TM_W4(24),
          FLR_TM_W4(28)
        : "r"(ta)
        : "memory");
}
__device__ __forceinline__ void tm_ld16(uint32_t ta, uint32_t *v)
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
                 : FLR_TM_W4(0), FLR_TM_W4(4), FLR_TM_W4(8), FLR_TM_W4(12)
                 : "r"(ta)
                 : "memory");
}
__device__ __forceinline__ void tm_ld8(uint32_t ta, uint32_t *v)
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                 : FLR_TM_W4(0), FLR_TM_W4(4)
                 : "r"(ta)
                 : "memory");
}
__device__ __forceinline__ void tm_ld2(uint32_t ta, uint32_t *v)
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%2];\n" : "=r"(v[0]), "=r"(v[1]) : "r"(ta) : "memory");
}
__device__ __forceinline__ uint32_t tm_ld1(uint32_t ta)
{
    uint32_t v0;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];\n" : "=r"(v0) : "r"(ta) : "memory");
    return v0;
}
#undef FLR_TM_R4
#undef FLR_TM_W4
__device__ __forceinline__ void tm_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }
__device__ __forceinline__ void tm_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory"); }

__device__ __forceinline__ void tm_st4(uint32_t ta, const uint32_t *v)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};\n" ::"r"(ta), "r"(v[0]), "r"(v[1]),
                 "r"(v[2]), "r"(v[3])
                 : "memory");
}
__device__ __forceinline__ void tm_ld4(uint32_t ta, uint32_t *v)
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3])
                 : "r"(ta)
                 : "memory");
}

// N columns from ta (N <= 64, ta aligned to the largest power of two in N): the largest
// shapes first, so every access starts at a multiple of its own width.
template <int N>
__device__ __forceinline__ void tm_st_n(uint32_t ta, const uint32_t *v)
{
    if constexpr (N >= 32) {
        tm_st32(ta, v);
        tm_st_n<N - 32>(ta + 32, v + 32);
    } else if constexpr (N >= 16) {
        tm_st16(ta, v);
        tm_st_n<N - 16>(ta + 16, v + 16);
    } else if constexpr (N >= 8) {
        tm_st8(ta, v);
        tm_st_n<N - 8>(ta + 8, v + 8);
    } else if constexpr (N >= 4) {
        tm_st4(ta, v);
        tm_st_n<N - 4>(ta + 4, v + 4);
    } else if constexpr (N >= 2) {
        tm_st2(ta, v);
        tm_st_n<N - 2>(ta + 2, v + 2);
    } else if constexpr (N == 1) {
        tm_st1(ta, v[0]);
    }
}
template <int N>
__device__ __forceinline__ void tm_ld_n(uint32_t ta, uint32_t *v)
{
    if constexpr (N >= 32) {
        tm_ld32(ta, v);
        tm_ld_n<N - 32>(ta + 32, v + 32);
    } else if constexpr (N >= 16) {
        tm_ld16(ta, v);
        tm_ld_n<N - 16>(ta + 16, v + 16);
    } else if constexpr (N >= 8) {
        tm_ld8(ta, v);
        tm_ld_n<N - 8>(ta + 8, v + 8);
    } else if constexpr (N >= 4) {
        tm_ld4(ta, v);
        tm_ld_n<N - 4>(ta + 4, v + 4);
    } else if constexpr (N >= 2) {
        tm_ld2(ta, v);
        tm_ld_n<N - 2>(ta + 2, v + 2);
    } else if constexpr (N == 1) {
        v[0] = tm_ld1(ta);
    }
}

}  // namespace flr
