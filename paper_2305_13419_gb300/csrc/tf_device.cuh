// tf_device.cuh -- device helpers shared by the fused step kernels
// (tf_step.cu: one step per pass; tf_step2.cu: two steps per pass):
// mbarrier / TMA wrappers in inline PTX and the packed FP32x2 arithmetic on
// x-adjacent point pairs.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>

#include "tf_internal.cuh"

namespace tf {
namespace dev {

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// bounded wait for phase `phase` of a barrier: at most `polls` polls, false
// if the phase has not completed by then
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned phase, long long polls = kSpinLimit) {
    for (long long it = 0; it < polls; ++it) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(phase)
            : "memory");
        if (done) return true;
    }
    return false;
}
__device__ __forceinline__ void tma_load_box(void* dst, const CUtensorMap* map, int x, int y, int z, int f,
                                             unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(smem_u32(dst)),
        "l"((unsigned long long)map), "r"(x), "r"(y), "r"(z), "r"(f), "r"(smem_u32(bar))
        : "memory");
}

// Two horizontally adjacent points travel together: a 64-bit register holds
// the pair (low: x, high: x + 1) and the sm_100-family packed FP32 pipe
// (add / sub / mul / fma .f32x2) updates both at once.
typedef unsigned long long f2;

__device__ __forceinline__ f2 pk(float a, float b) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "r"(__float_as_uint(a)), "r"(__float_as_uint(b)));
    return r;
}
__device__ __forceinline__ float lo(f2 v) { return __uint_as_float((unsigned)(v & 0xffffffffull)); }
__device__ __forceinline__ float hi(f2 v) { return __uint_as_float((unsigned)(v >> 32)); }
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
// 8-byte aligned pair in shared or global memory.  A global pair whose high
// point lies past the grid's x end reads and writes the spare column every
// row has there (the row pitch is at least N0 + 1); nothing reads it back.
__device__ __forceinline__ f2 ld2(const float* p) { return *reinterpret_cast<const f2*>(p); }
__device__ __forceinline__ void st2(float* p, f2 v) { *reinterpret_cast<f2*>(p) = v; }
// store the points whose bit is set in m (bit 0: low, bit 1: high)
__device__ __forceinline__ void st2m(float* p, f2 v, unsigned m) {
    if (m == 3u)
        st2(p, v);
    else if (m == 1u)
        p[0] = lo(v);
    else if (m == 2u)
        p[1] = hi(v);
}

// per point: m bit set -> new value, else old value (a bitwise select, no branch)
__device__ __forceinline__ f2 sel2(f2 nv, f2 ov, unsigned m2) {
    const f2 M = (f2)(0u - (m2 & 1u)) | (f2)(0u - (m2 >> 1 & 1u)) << 32;
    return (nv & M) | (ov & ~M);
}

}  // namespace dev
}  // namespace tf
