// Column groups: a few warps working together on one mode column held in shared memory
// (the wall-normal transforms).  The group's barrier, complex float-float values and their
// shared-memory slots, warp shuffles, and the prefix sums over the group's threads that
// the column algorithms build on.
#pragma once

#include <cstdint>

#include "df.cuh"

namespace shen {
namespace colg {

using df::F2;

struct Z {   // complex float-float
    F2 re, im;
};

constexpr Z kZero{F2{0.f, 0.f}, F2{0.f, 0.f}};

__device__ __forceinline__ Z ldz(const float4 *A, int i) {
    const float4 v = A[i];
    return Z{F2{v.x, v.y}, F2{v.z, v.w}};
}
__device__ __forceinline__ void stz(float4 *A, int i, Z v) { A[i] = make_float4(v.re.hi, v.re.lo, v.im.hi, v.im.lo); }
__device__ __forceinline__ F2 dneg(F2 a) { return F2{-a.hi, -a.lo}; }
__device__ __forceinline__ F2 nrm(F2 a) { return df::fast_two_sum(a.hi, a.lo); }
__device__ __forceinline__ Z zadd(Z a, Z b) { return Z{df::add(a.re, b.re), df::add(a.im, b.im)}; }
__device__ __forceinline__ Z zsub(Z a, Z b) { return Z{df::add(a.re, dneg(b.re)), df::add(a.im, dneg(b.im))}; }
__device__ __forceinline__ Z zneg(Z a) { return Z{dneg(a.re), dneg(a.im)}; }
__device__ __forceinline__ Z zhalf(Z a) {
    return Z{F2{0.5f * a.re.hi, 0.5f * a.re.lo}, F2{0.5f * a.im.hi, 0.5f * a.im.lo}};
}
__device__ __forceinline__ Z zscale(Z a, F2 s) { return Z{nrm(df::mul(a.re, s)), nrm(df::mul(a.im, s))}; }
__device__ __forceinline__ Z zmulf(Z v, float b) { return Z{nrm(df::mul(v.re, b)), nrm(df::mul(v.im, b))}; }
__device__ __forceinline__ Z zfma(F2 s, Z a, Z b) {  // b + s a
    return Z{df::add(b.re, df::mul(a.re, s)), df::add(b.im, df::mul(a.im, s))};
}
// v - c f (c complex, f real float-float)
__device__ __forceinline__ Z zsubmul(Z v, Z c, F2 f) {
    return Z{df::add(v.re, dneg(df::mul(c.re, f))), df::add(v.im, dneg(df::mul(c.im, f)))};
}
// v - c f and v + c f for a float32 f (one product term fewer than with a pair)
__device__ __forceinline__ Z zsubmulf(Z v, Z c, float f) {
    return Z{df::add(v.re, dneg(df::mul(c.re, f))), df::add(v.im, dneg(df::mul(c.im, f)))};
}
__device__ __forceinline__ Z zaddmulf(Z v, Z c, float f) {
    return Z{df::add(v.re, df::mul(c.re, f)), df::add(v.im, df::mul(c.im, f))};
}
__device__ __forceinline__ Z zfromf64(double2 v) { return Z{df::from_f64(v.x), df::from_f64(v.y)}; }
__device__ __forceinline__ double2 ztof64(Z v) { return make_double2(df::to_f64(v.re), df::to_f64(v.im)); }

__device__ __forceinline__ Z zshfl_xor(Z v, int o) {
    return Z{F2{__shfl_xor_sync(0xffffffffu, v.re.hi, o), __shfl_xor_sync(0xffffffffu, v.re.lo, o)},
             F2{__shfl_xor_sync(0xffffffffu, v.im.hi, o), __shfl_xor_sync(0xffffffffu, v.im.lo, o)}};
}
__device__ __forceinline__ Z zshfl_up(Z v, int o) {
    return Z{F2{__shfl_up_sync(0xffffffffu, v.re.hi, o), __shfl_up_sync(0xffffffffu, v.re.lo, o)},
             F2{__shfl_up_sync(0xffffffffu, v.im.hi, o), __shfl_up_sync(0xffffffffu, v.im.lo, o)}};
}

// Thread group of one mode column: G warps (32 G threads) synchronised by the named
// barrier `id` (ids 1 .. 15; 0 is __syncthreads).
struct Group {
    int t, nt, id;   // thread index in the group, group size, barrier id
    __device__ __forceinline__ void sync() const {
        if (nt == 32)
            __syncwarp();
        else
            asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nt) : "memory");
    }
    // AND of v over the group (also a barrier)
    __device__ __forceinline__ bool all(bool v) const {
        uint32_t r;
        asm volatile(
            "{\n .reg .pred pi, po;\n setp.ne.u32 pi, %1, 0;\n bar.red.and.pred po, %2, %3, pi;\n"
            " selp.u32 %0, 1, 0, po;\n}\n"
            : "=r"(r)
            : "r"((uint32_t)v), "r"(id), "r"(nt)
            : "memory");
        return r != 0;
    }
};

// Inclusive prefix sums over the warp's lanes of two values (one per parity), lane order.
__device__ __forceinline__ void warp_inclusive_scan(int lane, Z &i0, Z &i1) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const Z u0 = zshfl_up(i0, o), u1 = zshfl_up(i1, o);
        if (lane >= o) {
            i0 = zadd(u0, i0);
            i1 = zadd(u1, i1);
        }
    }
}

// Over the group's threads, of two per-thread values t0, t1: the exclusive prefix sums in
// thread order replace them, and s0, s1 receive the totals.  `area` holds 2 float4 per
// warp.  Summation order fixed (within a warp by shuffles, then the warps' totals in warp
// order), so every thread sees the same totals.
__device__ __forceinline__ void group_prefix(const Group &g, float4 *area, Z &t0, Z &t1, Z &s0, Z &s1) {
    const int lane = g.t & 31, warp = g.t >> 5, nw = g.nt >> 5;
    Z i0 = t0, i1 = t1;
    warp_inclusive_scan(lane, i0, i1);
    Z e0 = zshfl_up(i0, 1), e1 = zshfl_up(i1, 1);
    if (lane == 0) e0 = e1 = kZero;
    if (lane == 31) {
        stz(area, 2 * warp, i0);
        stz(area, 2 * warp + 1, i1);
    }
    g.sync();
    Z w0 = kZero, w1 = kZero;
    s0 = s1 = kZero;
    for (int w = 0; w < nw; w++) {
        if (w == warp) {
            w0 = s0;
            w1 = s1;
        }
        s0 = zadd(s0, ldz(area, 2 * w));
        s1 = zadd(s1, ldz(area, 2 * w + 1));
    }
    t0 = zadd(w0, e0);
    t1 = zadd(w1, e1);
}

}  // namespace colg
}  // namespace shen
