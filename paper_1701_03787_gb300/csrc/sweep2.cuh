// Building blocks of the on-chip float-float sweeps (kernels_df2.cu): Tensor Memory used as
// per-thread storage, and float-float row updates with one renormalisation per row.
//
// Tensor Memory (TMEM, 128 lanes x 512 columns of 32 bits per SM) is addressed as
// (lane << 16) | column.  With the 32x32b shape each thread of a warp reads or writes its
// own lane: warp w of a CTA reaches lanes 32 (w % 4) .. 32 (w % 4) + 31.  The kernels here
// use it as a second on-chip store, beside shared memory, for the forward sweep's result.
#pragma once
#include <cstdint>

#include "df.cuh"

namespace shen {
namespace sw2 {

using df::F2;

// ------------------------------------------------------------------ Tensor Memory

// Allocate ncols columns (a power of two, 32..512) for this CTA; one whole warp calls it.
// The TMEM address is written to *smem_dst.
__device__ __forceinline__ void tmem_alloc(uint32_t *smem_dst, uint32_t ncols) {
    const uint32_t dst = (uint32_t)__cvta_generic_to_shared(smem_dst);
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tmem_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// 8 consecutive 32-bit columns of this thread's lane, from column `taddr`.
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const float (&v)[8]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
        "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
        "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
        "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7]))
        : "memory");
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Issue a load of 8 columns; the registers are valid only after tmem_wait_ld(v).
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&v)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                   "=r"(v[7])
                 : "r"(taddr)
                 : "memory");
}

// Wait for this thread's outstanding TMEM loads.  The registers of the last load pass
// through the statement, so no use of them can be scheduled before it.
__device__ __forceinline__ void tmem_wait_ld(uint32_t (&v)[8]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]),
                   "+r"(v[7])
                 :
                 : "memory");
}

// ------------------------------------------------------------------ float-float rows

// Running sum of one row: a float-float value kept as an exact float32 head (hi, chained
// through TwoSum) and a float32 tail (lo) that collects the rounding errors of the head
// additions and the low-order parts of the products; renormalised once at the end.
struct Acc {
    float hi, lo;
};

__device__ __forceinline__ Acc acc_start(F2 x) { return {x.hi, x.lo}; }

// acc -= a * b (a, b float-float): the head takes the exact product head via TwoSum, the
// tail takes the product's rounding error, the cross terms and the TwoSum error.
__device__ __forceinline__ void acc_sub_mul(Acc &acc, F2 a, F2 b) {
    const float p = __fmul_rn(a.hi, b.hi);
    const float e = __fmaf_rn(a.hi, b.hi, -p);            // a.hi b.hi = p + e exactly
    float t = __fmaf_rn(a.hi, b.lo, e);
    t = __fmaf_rn(a.lo, b.hi, t);
    const float s = __fsub_rn(acc.hi, p);                 // TwoSum(acc.hi, -p)
    const float bb = __fsub_rn(s, acc.hi);
    const float err = __fadd_rn(__fsub_rn(acc.hi, __fsub_rn(s, bb)), __fsub_rn(-p, bb));
    acc.hi = s;
    acc.lo = __fsub_rn(__fadd_rn(acc.lo, err), t);
}

// acc += a * b
__device__ __forceinline__ void acc_add_mul(Acc &acc, F2 a, F2 b) { acc_sub_mul(acc, F2{-a.hi, -a.lo}, b); }

__device__ __forceinline__ F2 acc_done(Acc acc) { return df::fast_two_sum(acc.hi, acc.lo); }

// a * b renormalised
__device__ __forceinline__ F2 mul_n(F2 a, F2 b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return df::fast_two_sum(p, e);
}

// x + a * b renormalised (a running sum)
__device__ __forceinline__ F2 add_mul(F2 x, F2 a, F2 b) {
    Acc acc = acc_start(x);
    acc_add_mul(acc, a, b);
    return acc_done(acc);
}

// float64 -> float-float (hi = the float64 truncated to 24 significant bits, lo = the next
// 23), integer instructions only.  Finite inputs with 2^-126 <= |d| < 2^128 keep ~47 bits;
// smaller magnitudes (zero included) give 0, larger ones +-inf.
__device__ __forceinline__ F2 from_f64(double d) { return df::from_f64(d); }

// float-float -> float64 (exact widening of both parts, one float64 addition)
__device__ __forceinline__ double to_f64(F2 x) { return df::to_f64(x); }

}  // namespace sw2
}  // namespace shen
