// Wall-normal Shen transforms (Sec. 2, Eqs. ifft, sst1, sst2, fstB; Algorithms fst and
// ifst of the appendix) for every Fourier mode of a plan, Chebyshev-Gauss points
// x_i = cos((2i+1) pi / (2N)), i = 0 .. N-1, weights pi / N:
//
//   inverse   u(x_i) = sum_l uhat_l phi_l(x_i)                   (Eq. ifft, S^{-1})
//   scalar    S_l = (u, phi_l)_sigma = (pi/N) sum_i u(x_i) phi_l(x_i)     (Eq. sst1)
//   forward   uhat = B^{-1} S, B = (phi_q, phi_l)_sigma           (Eqs. sst2, fstB)
//
// for the spaces T_k (Eq. Tk), phi_k = T_k - T_{k+2} (Eq. phiD) and
// psi_k = T_k - 2(k+2)/(k+3) T_{k+2} + (k+1)/(k+3) T_{k+4} (Eq. phiN).
//
// Both cosine sums go through one complex FFT of length N per column (Makhoul's
// reordering, IEEE Trans. ASSP 28, 1980), which handles the real and imaginary parts of
// a complex column together:
//   DCT-II   C_k = sum_n x_n cos(pi k (2n+1) / (2N)):  v = (x_0, x_2, ..., x_3, x_1),
//            V = FFT(v),  C_k = (w_k V_k + conj(w_k) V_{N-k}) / 2,  w_k = e^{-i pi k/(2N)};
//            for 0 < k < N/2 the pair (k, N-k) comes from P = w_k V_k, Q = conj(w_k) V_{N-k}
//            as C_k = (P + Q)/2, C_{N-k} = i (P - Q)/2.
//   DCT-III  u_n = sum_k t_k cos(pi k (2n+1) / (2N)):  V_0 = t_0,
//            V_k = e^{i pi k/(2N)} (t_k - i t_{N-k}) / 2,  v = sum_k V_k e^{2 pi i k n/N},
//            u_{2n} = v_n, u_{2n+1} = v_{N-1-n}.
// The FFT is an in-place decimation-in-frequency radix-4 (and one radix-2) pass sequence
// in shared memory; its output sits in digit-reversed positions, which the post-processing
// reads through dpos().  The mass solve B uhat = S (tridiagonal per parity for phi,
// pentadiagonal per parity for psi, the same for every mode) runs as chunked scans: 16
// lanes per parity chain each solve a contiguous chunk with zero carries, a shuffle scan
// composes the chunks' affine carry maps, and a fix-up adds the carried part through the
// precomputed homogeneous solutions of each chunk (per-N tables from the float64 LU of B).
//
// One warp per mode column, persistent blocks; float-float arithmetic (pairs of float32,
// df.cuh), float64 (complex128) in and out.  Power-of-two N only.
#include <algorithm>
#include <cmath>
#include <vector>

#include "df.cuh"
#include "shen_internal.h"

namespace shen {
namespace {

using df::F2;

struct Z {   // complex float-float
    F2 re, im;
};

__device__ __forceinline__ Z ldz(const float4 *A, int i) {
    const float4 v = A[i];
    return Z{F2{v.x, v.y}, F2{v.z, v.w}};
}
__device__ __forceinline__ void stz(float4 *A, int i, Z v) { A[i] = make_float4(v.re.hi, v.re.lo, v.im.hi, v.im.lo); }
__device__ __forceinline__ F2 dneg(F2 a) { return F2{-a.hi, -a.lo}; }
__device__ __forceinline__ F2 nrm(F2 a) { return df::fast_two_sum(a.hi, a.lo); }
__device__ __forceinline__ Z zadd(Z a, Z b) { return Z{df::add(a.re, b.re), df::add(a.im, b.im)}; }
// Sum without the final renormalisation: hi carries the float32 sum, lo the exact error of
// it plus the low parts.  Only fed into a normalising add (never into a product).
__device__ __forceinline__ F2 add_raw(F2 x, F2 y) {
    const F2 s = df::two_sum(x.hi, y.hi);
    return F2{s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo))};
}
__device__ __forceinline__ Z zadd_raw(Z a, Z b) { return Z{add_raw(a.re, b.re), add_raw(a.im, b.im)}; }
__device__ __forceinline__ Z zsub_raw(Z a, Z b) {
    return Z{add_raw(a.re, F2{-b.re.hi, -b.re.lo}), add_raw(a.im, F2{-b.im.hi, -b.im.lo})};
}
__device__ __forceinline__ Z zsub(Z a, Z b) { return Z{df::add(a.re, dneg(b.re)), df::add(a.im, dneg(b.im))}; }
__device__ __forceinline__ Z zmul(Z a, Z w) {        // a w
    return Z{df::add(df::mul(a.re, w.re), dneg(df::mul(a.im, w.im))),
             df::add(df::mul(a.re, w.im), df::mul(a.im, w.re))};
}
__device__ __forceinline__ Z zmulc(Z a, Z w) {       // a conj(w)
    return Z{df::add(df::mul(a.re, w.re), df::mul(a.im, w.im)),
             df::add(df::mul(a.im, w.re), dneg(df::mul(a.re, w.im)))};
}
__device__ __forceinline__ Z zi(Z a) { return Z{dneg(a.im), a.re}; }      // i a
__device__ __forceinline__ Z zmi(Z a) { return Z{a.im, dneg(a.re)}; }     // -i a
__device__ __forceinline__ Z zhalf(Z a) {
    return Z{F2{0.5f * a.re.hi, 0.5f * a.re.lo}, F2{0.5f * a.im.hi, 0.5f * a.im.lo}};
}
__device__ __forceinline__ Z zpow2(Z a, float s) {   // a s, s a power of two (exact)
    return Z{F2{s * a.re.hi, s * a.re.lo}, F2{s * a.im.hi, s * a.im.lo}};
}
__device__ __forceinline__ Z zscale(Z a, F2 s) { return Z{nrm(df::mul(a.re, s)), nrm(df::mul(a.im, s))}; }
__device__ __forceinline__ Z zfma(F2 s, Z a, Z b) {  // b + s a
    return Z{df::add(b.re, df::mul(a.re, s)), df::add(b.im, df::mul(a.im, s))};
}
__device__ __forceinline__ Z zld(const float4 *p) {
    const float4 v = __ldg(p);
    return Z{F2{v.x, v.y}, F2{v.z, v.w}};
}
__device__ __forceinline__ Z zfromf64(double2 v) { return Z{df::from_f64(v.x), df::from_f64(v.y)}; }
__device__ __forceinline__ double2 ztof64(Z v) { return make_double2(df::to_f64(v.re), df::to_f64(v.im)); }

constexpr Z kZero{F2{0.f, 0.f}, F2{0.f, 0.f}};
constexpr F2 kOne{1.f, 0.f};
constexpr F2 kNil{0.f, 0.f};

// Position of frequency k after the in-place DIF passes (radix 4 first, then one radix 2
// when log2 N is odd): the first pass puts k mod 4 in quarter (k mod 4), and so on, so
// the base-4 digits of k come out reversed (times 2, plus the radix-2 digit, for odd lg).
__device__ __forceinline__ uint32_t rev4(uint32_t x, int nd) {   // reverse nd base-4 digits
    if (nd == 0) return 0u;
    uint32_t r = __brev(x) >> (32 - 2 * nd);
    return ((r & 0x55555555u) << 1) | ((r >> 1) & 0x55555555u);
}
__device__ __forceinline__ int dpos(int k, int lg) {
    const int nd = lg >> 1;
    if ((lg & 1) == 0) return (int)rev4((uint32_t)k, nd);
    const uint32_t low = (uint32_t)k & ((1u << (lg - 1)) - 1u);
    return (int)(2u * rev4(low, nd) + ((uint32_t)k >> (lg - 1)));
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

// In-place FFT of the group's column A[0 .. N): forward e^{-2 pi i jk/N}, or (INV) e^{+...},
// unnormalised, output in dpos() order.  tw: per radix-4 pass p (span L = N / 4^p,
// Q = L/4), entries [3 j + m - 1] = e^{-2 pi i m j 4^p / N}, j < Q, m = 1, 2, 3, passes
// stored one after the other, so a pass reads its twiddles contiguously.
template <bool INV>
__device__ void fft_dif(float4 *A, int lg, const float4 *tw, const Group &g) {
    const int N = 1 << lg, half = N >> 1;
    int lgL = lg;
    const float4 *twp = tw;
    for (; lgL >= 2; lgL -= 2) {
        const int lgQ = lgL - 2, Q = 1 << lgQ;
#pragma unroll 2
        for (int b = g.t; b < (N >> 2); b += g.nt) {
            const int j = b & (Q - 1);
            const int base = ((b >> lgQ) << lgL) + j;
            const Z a = ldz(A, base), bb = ldz(A, base + Q), c = ldz(A, base + 2 * Q), d = ldz(A, base + 3 * Q);
            const Z s0 = zadd_raw(a, c), s1 = zsub_raw(a, c), s2 = zadd_raw(bb, d), s3 = zsub_raw(bb, d);
            Z y0 = zadd(s0, s2), y2 = zsub(s0, s2);
            Z y1 = INV ? zadd(s1, zi(s3)) : zadd(s1, zmi(s3));
            Z y3 = INV ? zadd(s1, zmi(s3)) : zadd(s1, zi(s3));
            if (j != 0) {
                Z w1 = ldz(twp, 3 * j), w2 = ldz(twp, 3 * j + 1), w3 = ldz(twp, 3 * j + 2);
                if (INV) {
                    y1 = zmulc(y1, w1);
                    y2 = zmulc(y2, w2);
                    y3 = zmulc(y3, w3);
                } else {
                    y1 = zmul(y1, w1);
                    y2 = zmul(y2, w2);
                    y3 = zmul(y3, w3);
                }
            }
            stz(A, base, y0);
            stz(A, base + Q, y1);
            stz(A, base + 2 * Q, y2);
            stz(A, base + 3 * Q, y3);
        }
        twp += 3 * Q;
        g.sync();
    }
    if (lgL == 1) {
        for (int b = g.t; b < half; b += g.nt) {
            const Z a = ldz(A, 2 * b), c = ldz(A, 2 * b + 1);
            stz(A, 2 * b, zadd(a, c));
            stz(A, 2 * b + 1, zsub(a, c));
        }
        g.sync();
    }
}

// ------------------------------------------------------------------ mass solve

// Shuffles of float-float / complex values within segments of `w` lanes (16 or 32).
__device__ __forceinline__ F2 shup(F2 v, int d, int w) {
    return F2{__shfl_up_sync(0xffffffffu, v.hi, d, w), __shfl_up_sync(0xffffffffu, v.lo, d, w)};
}
__device__ __forceinline__ F2 shdn(F2 v, int d, int w) {
    return F2{__shfl_down_sync(0xffffffffu, v.hi, d, w), __shfl_down_sync(0xffffffffu, v.lo, d, w)};
}
__device__ __forceinline__ Z shup(Z v, int d, int w) { return Z{shup(v.re, d, w), shup(v.im, d, w)}; }
__device__ __forceinline__ Z shdn(Z v, int d, int w) { return Z{shdn(v.re, d, w), shdn(v.im, d, w)}; }
__device__ __forceinline__ F2 dmul(F2 a, F2 b) { return nrm(df::mul(a, b)); }
__device__ __forceinline__ F2 dfma2(F2 a, F2 b, F2 c, F2 d) {   // a b + c d
    return df::add(df::mul(a, b), df::mul(c, d));
}
__device__ __forceinline__ F2 lo2(float4 v) { return F2{v.x, v.y}; }
__device__ __forceinline__ F2 hi2(float4 v) { return F2{v.z, v.w}; }
__device__ __forceinline__ Z znrm(Z v) { return Z{nrm(v.re), nrm(v.im)}; }

// Affine carry map of a chunk on the state (s0, s1) (BW = 2) or s0 (BW = 1):
//   state -> M state + c.
struct CarryMap {
    F2 m00, m01, m10, m11;
    Z c0, c1;
};

// (M, c) o (M', c'):  x -> M (M' x + c') + c
template <int BW>
__device__ __forceinline__ CarryMap compose(const CarryMap &a, const CarryMap &b) {
    CarryMap r;
    if (BW == 1) {
        r.m00 = dmul(a.m00, b.m00);
        r.c0 = zfma(a.m00, b.c0, a.c0);
        r.m01 = r.m10 = r.m11 = kNil;
        r.c1 = kZero;
    } else {
        r.m00 = dfma2(a.m00, b.m00, a.m01, b.m10);
        r.m01 = dfma2(a.m00, b.m01, a.m01, b.m11);
        r.m10 = dfma2(a.m10, b.m00, a.m11, b.m10);
        r.m11 = dfma2(a.m10, b.m01, a.m11, b.m11);
        r.c0 = zfma(a.m01, b.c1, zfma(a.m00, b.c0, a.c0));
        r.c1 = zfma(a.m11, b.c1, zfma(a.m10, b.c0, a.c1));
    }
    return r;
}

template <int BW, bool UP>
__device__ __forceinline__ CarryMap shuffle_map(const CarryMap &m, int d, int w) {
    CarryMap r;
    auto sh = [&](F2 v) { return UP ? shup(v, d, w) : shdn(v, d, w); };
    auto shz = [&](Z v) { return UP ? shup(v, d, w) : shdn(v, d, w); };
    r.m00 = sh(m.m00);
    r.c0 = shz(m.c0);
    if (BW == 2) {
        r.m01 = sh(m.m01); r.m10 = sh(m.m10); r.m11 = sh(m.m11); r.c1 = shz(m.c1);
    } else {
        r.m01 = r.m10 = r.m11 = kNil; r.c1 = kZero;
    }
    return r;
}

// Per-N mass-solve tables, five planes of float4 (float-float pairs), plane f, parity h,
// row i at [(2 f + h) RM + i]:
//   f = 0 (l1, l2)   L_{i,i-1}, L_{i,i-2} of B's LU (unit lower)
//   f = 1 (G1, G2)   chunk-local homogeneous forward solutions for the carries
//                    (y_{s-1}, y_{s-2}) = (1, 0), (0, 1)
//   f = 2 (1/d, f1)  1/U_ii and U_{i,i+1} / U_ii
//   f = 3 (f2, 0)    U_{i,i+2} / U_ii
//   f = 4 (H1, H2)   chunk-local homogeneous backward solutions for (x_{e+1}, x_{e+2})
// Solve B x = S for the column: S in X (padded positions), x written back to X; W is
// scratch.  LP lanes per parity chain (16: lanes 0-15 / 16-31 of one warp; 32: warp 0 of
// the caller for parity 0, warp 1 for parity 1); chunk length K, padding shift psh.
// Table rows of the serial passes are fetched in blocks of PB ahead of their use.
// x -> M x + c applied to the state (t0, t1)
template <int BW>
__device__ __forceinline__ void apply_map(const CarryMap &m, Z t0, Z t1, Z &r0, Z &r1) {
    r0 = zfma(m.m00, t0, m.c0);
    if (BW == 2) {
        r0 = zfma(m.m01, t1, r0);
        r1 = zfma(m.m11, t1, zfma(m.m10, t0, m.c1));
    } else {
        r1 = kZero;
    }
}

// LP = 64: each parity chain spans two warps (chunks 0-31 and 32-63); the warps' scans are
// joined through two float4 slots per direction in the spare tail of X and W and a group
// barrier, so every thread of the (four-warp) group must call.
template <int BW>
__device__ void mass_solve(float4 *X, float4 *W, int n, int K, int psh, const float4 *T, int RM, int h, int j,
                           int LP, const Group &grp, int stride) {
    constexpr int PB = 4;
    const int R = (n - h + 1) / 2;
    const int s = j * K, e = min(R, s + K) - 1;
    const bool act = s < R;
    auto P = [&](int i) {
        const int k = 2 * i + h;
        return k + (k >> psh);
    };
    const float4 *TL = T + (long)(0 + h) * RM, *TG = T + (long)(2 + h) * RM, *TB = T + (long)(4 + h) * RM;
    const float4 *TF = T + (long)(6 + h) * RM, *TH = T + (long)(8 + h) * RM;

    // forward elimination, chunk-local with zero carries: p_i = S_i - l1 p_{i-1} - l2 p_{i-2}
    Z p1 = kZero, p2 = kZero;
    CarryMap mp{kOne, kNil, kNil, kOne, kZero, kZero};
    if (act) {
        float4 la[PB], lb[PB];
        auto load = [&](float4 (&l)[PB], int i0) {
#pragma unroll
            for (int q = 0; q < PB; q++) l[q] = __ldg(TL + min(i0 + q, e));
        };
        auto run = [&](const float4 (&l)[PB], int i0) {
#pragma unroll
            for (int q = 0; q < PB; q++) {
                const int i = i0 + q;
                if (i <= e) {
                    Z y = zfma(dneg(lo2(l[q])), p1, ldz(X, P(i)));
                    if (BW == 2) y = zfma(dneg(hi2(l[q])), p2, y);
                    y = znrm(y);
                    stz(W, P(i), y);
                    p2 = p1;
                    p1 = y;
                }
            }
        };
        load(la, s);
        for (int i0 = s; i0 <= e; i0 += 2 * PB) {
            load(lb, i0 + PB);
            run(la, i0);
            load(la, i0 + 2 * PB);
            run(lb, i0 + PB);
        }
        const float4 ge = __ldg(TG + e);
        mp.m00 = lo2(ge);
        mp.c0 = p1;
        if (BW == 2) {
            mp.m01 = hi2(ge);
            if (e - 1 >= s) {
                const float4 g1 = __ldg(TG + e - 1);
                mp.m10 = lo2(g1);
                mp.m11 = hi2(g1);
                mp.c1 = p2;
            } else {                       // one-row chunk: y_{e-1} = y_{s-1} is the carry itself
                mp.m10 = kOne;
                mp.m11 = kNil;
            }
        }
    }
    if (BW == 1) mp.m01 = mp.m10 = mp.m11 = kNil;
    // inclusive scan of the chunk maps within each warp segment, chunk 0 first
    const int SW = min(LP, 32), jw = j % SW, seg = j / SW;
    for (int d = 1; d < SW; d <<= 1) {
        const CarryMap o = shuffle_map<BW, true>(mp, d, SW);
        if (jw >= d) mp = compose<BW>(mp, o);
    }
    Z Y1, Y2;
    {
        CarryMap ex = shuffle_map<BW, true>(mp, 1, SW);         // exclusive prefix: lane jw - 1
        if (jw == 0) ex = CarryMap{kOne, kNil, kNil, kOne, kZero, kZero};
        Z t0 = kZero, t1 = kZero;                                // state entering the segment
        if (LP == 64) {
            float4 *xf = X + stride - 4 + 2 * h;
            if (seg == 0 && jw == SW - 1) {
                stz(xf, 0, mp.c0);
                stz(xf, 1, mp.c1);
            }
            grp.sync();
            if (seg == 1) {
                t0 = ldz(xf, 0);
                t1 = ldz(xf, 1);
            }
        }
        apply_map<BW>(ex, t0, t1, Y1, Y2);
    }
    if (act) {
#pragma unroll 4
        for (int i = s; i <= e; i++) {
            const float4 gv = __ldg(TG + i);
            Z y = zfma(lo2(gv), Y1, ldz(W, P(i)));
            if (BW == 2) y = zfma(hi2(gv), Y2, y);
            stz(W, P(i), znrm(y));
        }
    }
    // back substitution, chunk-local: q_i = y_i / d_i - f1 q_{i+1} - f2 q_{i+2}
    Z q1 = kZero, q2 = kZero;
    CarryMap mq{kOne, kNil, kNil, kOne, kZero, kZero};
    if (act) {
        float4 ba[PB], bb[PB], fa[PB], fb[PB];
        auto load = [&](float4 (&b)[PB], float4 (&f)[PB], int i0) {
#pragma unroll
            for (int q = 0; q < PB; q++) {
                const int i = max(i0 - q, s);
                b[q] = __ldg(TB + i);
                if (BW == 2) f[q] = __ldg(TF + i);
            }
        };
        auto run = [&](const float4 (&b)[PB], const float4 (&f)[PB], int i0) {
#pragma unroll
            for (int q = 0; q < PB; q++) {
                const int i = i0 - q;
                if (i >= s) {
                    Z x = zscale(ldz(W, P(i)), lo2(b[q]));
                    x = zfma(dneg(hi2(b[q])), q1, x);
                    if (BW == 2) x = zfma(dneg(lo2(f[q])), q2, x);
                    x = znrm(x);
                    stz(W, P(i), x);
                    q2 = q1;
                    q1 = x;
                }
            }
        };
        load(ba, fa, e);
        for (int i0 = e; i0 >= s; i0 -= 2 * PB) {
            load(bb, fb, i0 - PB);
            run(ba, fa, i0);
            load(ba, fa, i0 - 2 * PB);
            run(bb, fb, i0 - PB);
        }
        const float4 hs = __ldg(TH + s);
        mq.m00 = lo2(hs);
        mq.c0 = q1;
        if (BW == 2) {
            mq.m01 = hi2(hs);
            if (s + 1 <= e) {
                const float4 h1 = __ldg(TH + s + 1);
                mq.m10 = lo2(h1);
                mq.m11 = hi2(h1);
                mq.c1 = q2;
            } else {                       // one-row chunk: x_{s+1} = x_{e+1} is the carry itself
                mq.m10 = kOne;
                mq.m11 = kNil;
            }
        }
    }
    if (BW == 1) mq.m01 = mq.m10 = mq.m11 = kNil;
    // inclusive scan from the last chunk down, within each warp segment
    for (int d = 1; d < SW; d <<= 1) {
        const CarryMap o = shuffle_map<BW, false>(mq, d, SW);
        if (jw + d < SW) mq = compose<BW>(mq, o);
    }
    Z X1, X2;
    {
        CarryMap ex = shuffle_map<BW, false>(mq, 1, SW);        // exclusive: lane jw + 1
        if (jw == SW - 1) ex = CarryMap{kOne, kNil, kNil, kOne, kZero, kZero};
        Z t0 = kZero, t1 = kZero;
        if (LP == 64) {
            float4 *xb = W + stride - 4 + 2 * h;
            if (seg == 1 && jw == 0) {
                stz(xb, 0, mq.c0);
                stz(xb, 1, mq.c1);
            }
            grp.sync();
            if (seg == 0) {
                t0 = ldz(xb, 0);
                t1 = ldz(xb, 1);
            }
        }
        apply_map<BW>(ex, t0, t1, X1, X2);
    }
    if (act) {
#pragma unroll 4
        for (int i = s; i <= e; i++) {
            const float4 hv = __ldg(TH + i);
            Z x = zfma(lo2(hv), X1, ldz(W, P(i)));
            if (BW == 2) x = zfma(hi2(hv), X2, x);
            stz(X, P(i), znrm(x));
        }
    }
}

// ------------------------------------------------------------------ kernel

// One-dimensional bulk copies (TMA, cp.async.bulk) of a whole column from global to
// shared memory, completed on a per-warp mbarrier.
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for the phase `parity` of the warp's barrier (each try_wait suspends for a
// bounded time): false after the limit.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    for (uint32_t it = 0; it < (1u << 22); it++)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

struct TrArgs {
    int N, lg;               // Chebyshev modes; log2 of the FFT length (N, or 2 (N - 1) on Gauss-Lobatto points)
    int G, n_groups;         // warps per mode group, groups per block
    long n_modes;
    int stride;              // float4 per buffer
    int n_tw;                // float4 of the per-pass twiddle table (copied to shared memory)
    int K, psh, RM;          // mass solve: chunk length, padding shift, rows per parity stride
    const float4 *tw;        // per-pass twiddles
    const float4 *mk;        // e^{-i pi k/(2N)}, k = 0 .. N/2
    const float4 *coef;      // per k: (g1i_k, g2i_k), (g1_k, g2_k)
    const float4 *mass;      // mass-solve rows of the space
    int *err;                // set to 1 if a column copy did not complete
    F2 pi_over_N;
};

// Buffers of a mode group: 2 (inverse, scalar products, forward in T_k) or 3 (forward in
// phi, psi) of `stride` float4.  The column copy lands in R; the next mode's copy is
// issued as soon as R is free, so it overlaps the current mode's FFT.
constexpr int nbuf_of(int kind, int space) { return (kind == 2 && space != 0) ? 3 : 2; }

// KIND: 0 inverse, 1 scalar product, 2 forward.  SPACE: 0 T_k, 1 phi_k, 2 psi_k.  GL:
// Gauss-Lobatto points (a compile-time choice, so the Gauss kernels carry none of its code).
template <int KIND, int SPACE, bool GL>
__global__ void __launch_bounds__(KIND == 2 && SPACE != 0 ? 512 : 768)
    transform_kernel(TrArgs a, const double *in, double *out) {
    extern __shared__ float4 sm[];
    const int N = a.N, lg = a.lg, half = N >> 1, M = N - 1;
    const float4 *tw = sm;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + a.n_tw);
    for (int t = threadIdx.x; t < a.n_tw; t += blockDim.x) sm[t] = __ldg(a.tw + t);
    const int gsize = 32 * a.G, gi = threadIdx.x / gsize;
    const Group g{(int)threadIdx.x - gi * gsize, gsize, 1 + gi};
    constexpr int NB = nbuf_of(KIND, SPACE);
    float4 *A = sm + a.n_tw + 8 + (long)gi * NB * a.stride;
    float4 *Bf = A + a.stride;
    float4 *R = NB == 3 ? Bf + a.stride : Bf;
    uint64_t *bar = bars + gi;
    const int n = SPACE == 0 ? N : (SPACE == 1 ? N - 2 : N - 4);
    const long groups_total = (long)gridDim.x * a.n_groups;
    const uint32_t col_bytes = (uint32_t)N * 16u;
    long mode = (long)blockIdx.x * a.n_groups + gi;
    if (g.t == 0) {
        mbar_init(bar);
        fence_mbar_init();
        fence_async_smem();
        if (mode < a.n_modes) bulk_load(R, in + 2 * mode * (long)N, col_bytes, bar);
    }
    __syncthreads();
    uint32_t parity = 0;
    auto prefetch_next = [&](long next) {   // R is free: every thread's last access to it is done
        fence_async_smem();
        g.sync();
        if (g.t == 0 && next < a.n_modes) bulk_load(R, in + 2 * next * (long)N, col_bytes, bar);
    };
    auto mkz = [&](int k) { return zld(a.mk + k); };
    for (; mode < a.n_modes; mode += groups_total) {
        const long next = mode + groups_total;
        if (!g.all(mbar_wait(bar, parity))) {
            // the copy did not land: flag it, give it time to finish, stop (group-uniform)
            if (g.t == 0) atomicExch(a.err, 1);
            mbar_wait(bar, parity);
            return;
        }
        parity ^= 1u;
        double2 *y = reinterpret_cast<double2 *>(out) + mode * N;
        const double2 *xs = reinterpret_cast<const double2 *>(R);
        if (KIND == 0) {
            // coefficients (zero beyond the space) converted in place in R (= B), natural order
            for (int k = g.t; k < N; k += g.nt) {
                const double2 v = xs[k];
                stz(Bf, k, k < n ? zfromf64(v) : kZero);
            }
            g.sync();
            auto tk = [&](int k) -> Z {
                if (k >= N) return kZero;
                Z t = ldz(Bf, k);
                if (SPACE == 1 && k >= 2) t = zsub(t, ldz(Bf, k - 2));
                if (SPACE == 2 && k >= 2) {
                    const float4 c = __ldg(a.coef + 2 * k);
                    t = zfma(dneg(F2{c.x, c.y}), ldz(Bf, k - 2), t);
                    if (k >= 4) t = zfma(F2{c.z, c.w}, ldz(Bf, k - 4), t);
                }
                return t;
            };
            if (GL) {
                // Gauss-Lobatto points x_i = cos(i pi / M): u_i = sum_k t_k cos(pi k i / M), a
                // DCT-I, from the FFT Y of the even extension (t_0 .. t_M, t_{M-1} .. t_1):
                // u_i = (Y_i + t_0 + (-1)^i t_M) / 2
                const Z t0 = tk(0), tM = tk(M);
                for (int k = g.t; k <= M; k += g.nt) {
                    const Z t = tk(k);
                    stz(A, k, t);
                    if (k >= 1 && k < M) stz(A, 2 * M - k, t);
                }
                prefetch_next(next);
                fft_dif<false>(A, lg, tw, g);
                for (int i = g.t; i < N; i += g.nt) {
                    const Z e = zadd(t0, (i & 1) ? Z{dneg(tM.re), dneg(tM.im)} : tM);
                    y[i] = ztof64(zhalf(zadd(ldz(A, dpos(i, lg)), e)));
                }
                g.sync();
                continue;
            }
            // pairs (k, N-k), 0 < k <= N/2, with w = e^{-i pi k/(2N)} = mk[k]:
            //   V_k     = conj(w) (t_k - i t_{N-k}) / 2
            //   V_{N-k} = i w (t_{N-k} - i t_k) / 2      (e^{i pi (N-k)/(2N)} = i w)
            for (int k = g.t; k <= half; k += g.nt) {
                if (k == 0) {
                    stz(A, 0, tk(0));
                    continue;
                }
                const Z t1 = tk(k), t2 = tk(N - k), w = mkz(k);
                stz(A, k, zhalf(zmulc(zadd(t1, zmi(t2)), w)));
                if (k != half) stz(A, N - k, zhalf(zi(zmul(zadd(t2, zmi(t1)), w))));
            }
            prefetch_next(next);
            fft_dif<true>(A, lg, tw, g);
            for (int m = g.t; m < N; m += g.nt) {
                const int src = (m & 1) ? N - 1 - (m >> 1) : (m >> 1);
                y[m] = ztof64(ldz(A, dpos(src, lg)));
            }
        } else {
            if (GL) {
                // Gauss-Lobatto: the even extension (u_0 .. u_M, u_{M-1} .. u_1); its FFT gives
                // Y_k = u_0 + (-1)^k u_M + 2 sum_interior u_i cos(pi k i / M), so that
                // (u, T_k)_sigma = pi / (2M) Y_k with the GL weights (pi / M, half at the ends)
                for (int m = g.t; m < N; m += g.nt) {
                    const Z v = zfromf64(xs[m]);
                    stz(A, m, v);
                    if (m >= 1 && m < M) stz(A, 2 * M - m, v);
                }
                prefetch_next(next);
                fft_dif<false>(A, lg, tw, g);
            } else {
            // values -> Makhoul order in A; R free for the next column
            for (int m = g.t; m < N; m += g.nt) {
                const int dst = (m & 1) ? N - 1 - (m >> 1) : (m >> 1);
                stz(A, dst, zfromf64(xs[m]));
            }
            prefetch_next(next);
            fft_dif<false>(A, lg, tw, g);
            // C_k (DCT-II) in place: the pair (k, N-k) is read and written by one thread at
            // positions dpos(k), dpos(N-k)
            for (int k = g.t; k <= half; k += g.nt) {
                if (k == 0) continue;                                  // C_0 = V_0
                const int pk = dpos(k, lg), pn = dpos(N - k, lg);
                const Z w = mkz(k);
                const Z P = zmul(ldz(A, pk), w);
                const Z Q = zmulc(ldz(A, pn), w);
                stz(A, pk, zhalf(zadd(P, Q)));
                if (k != half) stz(A, pn, zhalf(zi(zsub(P, Q))));
            }
            }
            g.sync();
            auto C = [&](int k) { return ldz(A, dpos(k, lg)); };
            if (KIND == 2 && SPACE == 0) {
                // uhat_k = S_k / (pi c_k / 2): Gauss: C_k 2 / (N c_k) (c_0 = 2);
                // Gauss-Lobatto: Y_k / (M c_k) (c_0 = c_M = 2); N, M powers of two
                if (GL) {
                    const float sc = 1.0f / (float)M;
                    for (int k = g.t; k < N; k += g.nt)
                        y[k] = ztof64(zpow2(C(k), (k == 0 || k == M) ? 0.5f * sc : sc));
                } else {
                    const float sc = 2.0f / (float)N;
                    for (int k = g.t; k < N; k += g.nt) y[k] = ztof64(zpow2(C(k), k == 0 ? 0.5f * sc : sc));
                }
            } else {
                // scalar products S_l (Algorithm fst, forwardScalar)
                auto S = [&](int l) -> Z {
                    if (l >= n) return kZero;
                    Z v = C(l);
                    if (SPACE == 1) v = zsub(v, C(l + 2));
                    if (SPACE == 2) {
                        const float4 c = __ldg(a.coef + 2 * l + 1);
                        v = zfma(dneg(F2{c.x, c.y}), C(l + 2), v);
                        v = zfma(F2{c.z, c.w}, C(l + 4), v);
                    }
                    return zscale(v, a.pi_over_N);
                };
                if (KIND == 1) {
                    for (int l = g.t; l < N; l += g.nt) y[l] = ztof64(S(l));
                } else {
                    for (int l = g.t; l < N; l += g.nt) stz(Bf, l + (l >> a.psh), S(l));
                    g.sync();
                    // lanes per parity: two warps each in a four-warp group, one warp each in a
                    // two-warp group, half a warp in a one-warp group
                    const int LP = g.nt >= 128 ? 64 : (g.nt >= 64 ? 32 : 16);
                    if (g.t < 2 * LP)
                        mass_solve<SPACE == 1 ? 1 : 2>(Bf, A, n, a.K, a.psh, a.mass, a.RM, g.t / LP, g.t % LP, LP, g,
                                                       a.stride);
                    g.sync();
                    for (int k = g.t; k < N; k += g.nt)
                        y[k] = k < n ? ztof64(ldz(Bf, k + (k >> a.psh))) : make_double2(0.0, 0.0);
                }
            }
        }
        g.sync();
    }
}

template <int KIND, int SPACE, bool GL>
const void *kernel_ptr() {
    return reinterpret_cast<const void *>(&transform_kernel<KIND, SPACE, GL>);
}

const void *kernel_of(int kind, int space, bool gl) {
    static const void *const k[2][3][3] = {
        {{kernel_ptr<0, 0, false>(), kernel_ptr<0, 1, false>(), kernel_ptr<0, 2, false>()},
         {kernel_ptr<1, 0, false>(), kernel_ptr<1, 1, false>(), kernel_ptr<1, 2, false>()},
         {kernel_ptr<2, 0, false>(), kernel_ptr<2, 1, false>(), kernel_ptr<2, 2, false>()}},
        {{kernel_ptr<0, 0, true>(), kernel_ptr<0, 1, true>(), kernel_ptr<0, 2, true>()},
         {kernel_ptr<1, 0, true>(), kernel_ptr<1, 1, true>(), kernel_ptr<1, 2, true>()},
         {kernel_ptr<2, 0, true>(), kernel_ptr<2, 1, true>(), kernel_ptr<2, 2, true>()}},
    };
    return k[gl ? 1 : 0][kind][space];
}

inline float4 pair4(long double a, long double b) {
    const float ah = (float)a, bh = (float)b;
    return make_float4(ah, (float)(a - (long double)ah), bh, (float)(b - (long double)bh));
}

int ilog2(int v) {
    int l = 0;
    while ((1 << l) < v) l++;
    return l;
}

// Chunk length of the mass solve for n unknowns and LP lanes per parity chain: a power of
// two >= 2 with LP chunks covering the longer parity chain.
int chunk_len(int n, int LP) {
    const int R0 = (n + 1) / 2;
    int K = 2;
    while (LP * K < R0) K <<= 1;
    return K;
}

// Warps per mode group of an N-mode plan (more threads per column for larger N), and the
// mass solve's lanes per parity chain that go with it.
int group_warps(int N) { return std::max(1, std::min(4, N / 256)); }
int lanes_per_parity(int N) { return group_warps(N) >= 4 ? 64 : (group_warps(N) >= 2 ? 32 : 16); }

// Mass-solve tables of one space in the five planes mass_solve reads (B rows: diagonal,
// +1, +2 per parity chain), from the unpivoted LU of each parity chain of B in long double
// arithmetic, rounded to float-float pairs.
void mass_rows(int N, int space, int K, int RM, std::vector<float4> &T, bool gl) {
    const long double pi = 3.141592653589793238462643383279502884L;
    const int n = space == 1 ? N - 2 : N - 4;
    T.assign((size_t)2 * RM * 5, make_float4(0.f, 0.f, 0.f, 0.f));
    for (int h = 0; h < 2; h++) {
        const int R = (n - h + 1) / 2;
        std::vector<long double> dg(R), s1(R, 0.0L), s2(R, 0.0L);
        for (int i = 0; i < R; i++) {
            const long double k = 2 * i + h, ck = (2 * i + h == 0) ? 2.0L : 1.0L;
            // Gauss-Lobatto: c_{N-1} = 2 in the highest row (Table tab:matrices)
            const long double ck2 = (gl && 2 * i + h + 2 == N - 1) ? 2.0L : 1.0L;
            const long double ck4 = (gl && 2 * i + h + 4 == N - 1) ? 2.0L : 1.0L;
            if (space == 1) {
                dg[i] = pi / 2 * (ck + ck2);
                if (i + 1 < R) s1[i] = -pi / 2;
            } else {
                const long double r2 = (k + 2) / (k + 3), r1 = (k + 1) / (k + 3);
                dg[i] = pi / 2 * (ck + 4 * r2 * r2 + ck4 * r1 * r1);
                if (i + 1 < R) s1[i] = -pi * (r2 + (k + 4) * (k + 1) / ((k + 5) * (k + 3)));
                if (i + 2 < R) s2[i] = pi / 2 * r1;
            }
        }
        // unpivoted banded LU: B = L U, L unit lower (l1, l2), U (d, e1, e2); B symmetric
        std::vector<long double> l1(R, 0.0L), l2(R, 0.0L), d(R), e1(R), e2(R);
        for (int i = 0; i < R; i++) {
            if (i >= 2) l2[i] = s2[i - 2] / d[i - 2];
            if (i >= 1) l1[i] = (s1[i - 1] - (i >= 2 ? l2[i] * e1[i - 2] : 0.0L)) / d[i - 1];
            d[i] = dg[i] - (i >= 1 ? l1[i] * e1[i - 1] : 0.0L) - (i >= 2 ? l2[i] * e2[i - 2] : 0.0L);
            e1[i] = s1[i] - (i >= 1 ? l1[i] * e2[i - 1] : 0.0L);
            e2[i] = s2[i];
        }
        auto at = [&](int f, int i) -> float4 & { return T[(size_t)(2 * f + h) * RM + i]; };
        for (int s = 0; s < R; s += K) {
            const int e = std::min(R, s + K) - 1;
            long double a1 = 1, a2 = 0, b1 = 0, b2 = 1;       // (G1, G2) at rows i-1, i-2
            for (int i = s; i <= e; i++) {
                const long double g1 = -l1[i] * a1 - l2[i] * b1, g2 = -l1[i] * a2 - l2[i] * b2;
                at(1, i) = pair4(g1, g2);
                b1 = a1; b2 = a2; a1 = g1; a2 = g2;
            }
            a1 = 1; a2 = 0; b1 = 0; b2 = 1;                    // (H1, H2) at rows i+1, i+2
            for (int i = e; i >= s; i--) {
                const long double f1 = e1[i] / d[i], f2 = e2[i] / d[i];
                const long double x1 = -f1 * a1 - f2 * b1, x2 = -f1 * a2 - f2 * b2;
                at(4, i) = pair4(x1, x2);
                b1 = a1; b2 = a2; a1 = x1; a2 = x2;
            }
        }
        for (int i = 0; i < R; i++) {
            at(0, i) = pair4(l1[i], l2[i]);
            at(2, i) = pair4(1.0L / d[i], e1[i] / d[i]);
            at(3, i) = pair4(e2[i] / d[i], 0.0L);
        }
    }
}

}  // namespace

// Gauss points: N a power of two (FFT length N); Gauss-Lobatto points: N - 1 a power of two
// (FFT length 2 (N - 1)).
bool transform_supported(const Plan &p) {
    const int L = p.gl ? p.N - 1 : p.N;
    return p.N >= 8 && L >= 8 && (L & (L - 1)) == 0;
}

namespace {
int fft_length(const Plan &p) { return p.gl ? 2 * (p.N - 1) : p.N; }
}  // namespace

// Number of float4 of the per-pass twiddle table: 3 Q per radix-4 pass.
int twiddle_count(int N) {
    int c = 0;
    for (int lgL = ilog2(N); lgL >= 2; lgL -= 2) c += 3 * (1 << (lgL - 2));
    return c;
}

// Tables of the transforms of an N-mode plan (float4 units, float-float pairs):
//   [0, ntw)                per-pass twiddles of fft_dif
//   [ntw, ntw + N/2 + 1)    mk[k] = e^{-i pi k/(2N)}, k = 0 .. N/2
//   then 2 N: per k, (2k/(k+1), (k-3)/(k-1)) (psi -> T coefficients, k >= 2 / 4) and
//                    (2(k+2)/(k+3), (k+1)/(k+3)) (Eq. phiN weights, k < N-4)
//   then the mass-solve rows of phi (2 RMd 5) and of psi (2 RMb 5).
cudaError_t transform_setup(Plan &p, long long &bytes, cudaStream_t s) {
    if (!transform_supported(p)) return cudaSuccess;
    const int N = p.N, NF = fft_length(p), lg = ilog2(NF);
    const long double pi = 3.141592653589793238462643383279502884L;
    const int LP = lanes_per_parity(N);
    const int Kd = chunk_len(N - 2, LP), Kb = chunk_len(N - 4, LP);
    const int RMd = (N - 2 + 1) / 2, RMb = (N - 4 + 1) / 2;
    const int ntw = twiddle_count(NF), nmk = N / 2 + 1;
    std::vector<float4> tab;
    tab.reserve((size_t)ntw + nmk + 2 * N);
    for (int lgL = lg, sh = 0; lgL >= 2; lgL -= 2, sh += 2) {
        const int Q = 1 << (lgL - 2);
        for (int j = 0; j < Q; j++)
            for (int m = 1; m <= 3; m++) {
                const long t = ((long)m * j) << sh;                    // < 3N/4
                const long double ang = -2 * pi * (long double)t / NF;
                tab.push_back(pair4(cosl(ang), sinl(ang)));
            }
    }
    for (int k = 0; k < nmk; k++) {
        const long double ang = -pi * k / (2 * (long double)N);
        tab.push_back(pair4(cosl(ang), sinl(ang)));
    }
    for (int k = 0; k < N; k++) {
        const long double K = k;
        const long double gi1 = k >= 2 ? 2 * K / (K + 1) : 0.0L, gi2 = k >= 4 ? (K - 3) / (K - 1) : 0.0L;
        const long double g1 = k < N - 4 ? 2 * (K + 2) / (K + 3) : 0.0L, g2 = k < N - 4 ? (K + 1) / (K + 3) : 0.0L;
        tab.push_back(pair4(gi1, gi2));
        tab.push_back(pair4(g1, g2));
    }
    std::vector<float4> md, mb;
    mass_rows(N, 1, Kd, RMd, md, p.gl);
    mass_rows(N, 2, Kb, RMb, mb, p.gl);
    p.tr_off_mass = (int)tab.size();
    tab.insert(tab.end(), md.begin(), md.end());
    tab.insert(tab.end(), mb.begin(), mb.end());
    p.tr_ntw = ntw;
    bytes += (long long)(tab.size() * sizeof(float4));
    cudaError_t e = cudaMalloc((void **)&p.d_tr, tab.size() * sizeof(float4));
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(p.d_tr, tab.data(), tab.size() * sizeof(float4), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    // launch shape per (kind, space): G warps per mode group (more threads per column for
    // larger N), groups per block from the shared memory budget (twiddles, barriers,
    // nbuf buffers per group) and the kernel's 768-thread bound; persistent grid from the
    // occupancy.  A (kind, space) whose buffers do not fit gets no shape (unsupported).
    int dev = 0, smem_max = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess)
        return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int psh = std::min(ilog2(2 * Kd), ilog2(2 * Kb));
    const int stride = std::max(NF, N + (N >> psh)) + 4;
    p.tr_stride = stride;
    p.tr_psh = psh;
    const int G = group_warps(N);
    const long fixed = (long)(ntw + 8) * sizeof(float4);
    for (int kind = 0; kind < 3; kind++)
        for (int space = 0; space < 3; space++) {
            const long per_group = (long)nbuf_of(kind, space) * stride * sizeof(float4);
            const int max_threads = nbuf_of(kind, space) == 3 ? 512 : 768;   // the kernel's bound
            const int groups = (int)std::min<long>(std::min(8, max_threads / (32 * G)), (smem_max - fixed) / per_group);
            p.tr_groups[kind][space] = 0;
            if (groups < 1) continue;
            const int smem = (int)(fixed + groups * per_group);
            const void *k = kernel_of(kind, space, p.gl);
            if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess)
                return e;
            const int carve = (int)std::min<long>(100, (smem * 100L + smem_max - 1) / smem_max + 1);
            if ((e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, carve)) != cudaSuccess)
                return e;
            int per_sm = 0;
            if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 32 * G * groups, smem)) != cudaSuccess)
                return e;
            if (per_sm < 1) continue;
            const long need = (p.n_modes + groups - 1) / groups;
            p.tr_groups[kind][space] = groups;
            p.tr_G = G;
            p.tr_smem[kind][space] = smem;
            p.tr_grid[kind][space] = (int)std::max<long>(1, std::min<long>((long)per_sm * sms, need));
        }
    return cudaSuccess;
}

bool transform_shape_ok(const Plan &p, int kind, int space) { return p.d_tr && p.tr_groups[kind][space] > 0; }

cudaError_t launch_transform(const Plan &p, int kind, int space, long count, const double *in, double *out,
                             cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    const int N = p.N;
    TrArgs a;
    a.N = N;
    a.lg = ilog2(fft_length(p));
    a.G = p.tr_G;
    a.n_groups = p.tr_groups[kind][space];
    a.n_modes = count;
    a.stride = p.tr_stride;
    a.n_tw = p.tr_ntw;
    a.psh = p.tr_psh;
    const int RMd = (N - 2 + 1) / 2, RMb = (N - 4 + 1) / 2;
    a.K = space == 1 ? chunk_len(N - 2, lanes_per_parity(N)) : chunk_len(N - 4, lanes_per_parity(N));
    a.RM = space == 1 ? RMd : RMb;
    a.tw = p.d_tr;
    a.mk = p.d_tr + p.tr_ntw;
    a.coef = a.mk + (N / 2 + 1);
    const float4 *mass = p.d_tr + p.tr_off_mass;
    a.mass = space == 1 ? mass : mass + (size_t)2 * RMd * 5;
    const double pn = p.gl ? kPi / (2.0 * (N - 1)) : kPi / N;   // weight of the point sum
    const float ph = (float)pn;
    a.pi_over_N = F2{ph, (float)(pn - (double)ph)};
    a.err = p.d_err + 3;
    const long need = (count + a.n_groups - 1) / a.n_groups;
    const dim3 grid((unsigned)std::max<long>(1, std::min<long>(p.tr_grid[kind][space], need))),
        block((unsigned)(32 * a.G * a.n_groups));
    void *args[] = {&a, &in, &out};
    return cudaLaunchKernel(kernel_of(kind, space, p.gl), grid, block, args, (size_t)p.tr_smem[kind][space], s);
}

}  // namespace shen
