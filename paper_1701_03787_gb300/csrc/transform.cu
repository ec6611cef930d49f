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
// On Gauss-Lobatto points (x_i = cos(i pi / M), M = N - 1) the cosine sums are DCT-I: one
// FFT of length 2M of the even extension (x_0 .. x_M, x_{M-1} .. x_1).
// The FFT is an in-place decimation-in-frequency radix-4 (and one radix-2) pass sequence
// in shared memory; its output sits in digit-reversed positions, which the post-processing
// reads through dpos().  The forward transforms in phi and psi solve B uhat = S in the same
// kernel, from the column's Chebyshev coefficients in shared memory: B = P W P^T makes
// uhat a weighted least-squares fit whose triangular part inverts as prefix sums
// (forward_ls), so no banded sweep runs.
//
// One group of warps per mode column, persistent blocks; float-float arithmetic (pairs of
// float32, df.cuh), float64 (complex128) in and out.  FFT length N (Gauss) or 2 (N - 1)
// (Gauss-Lobatto), a power of two or three times one.
#include <algorithm>
#include <cmath>
#include <vector>

#include "chains.cuh"
#include "colgroup.cuh"
#include "df.cuh"
#include "shen_internal.h"

namespace shen {
namespace {

using df::F2;
using namespace colg;

// Sum without the final renormalisation: hi carries the float32 sum, lo the exact error of
// it plus the low parts, so hi + lo is the float-float sum.  lo may exceed half an ulp of
// hi (after cancellation), but the absolute error stays that of float32 arithmetic on lo,
// about 2^-24 |lo| <= 2^-48 times the inputs' magnitude, and a later product or add of
// such a pair keeps that absolute bound (a product drops only lo_x lo_y).  The FFT's
// error is norm-wise (relative to the column's magnitude), so its passes run on raw pairs
// (twice the error of renormalised sums in a float32 emulation, far inside the bound).
__device__ __forceinline__ F2 add_raw(F2 x, F2 y) {
    const F2 s = df::two_sum(x.hi, y.hi);
    return F2{s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo))};
}
__device__ __forceinline__ Z zadd_raw(Z a, Z b) { return Z{add_raw(a.re, b.re), add_raw(a.im, b.im)}; }
__device__ __forceinline__ Z zsub_raw(Z a, Z b) {
    return Z{add_raw(a.re, F2{-b.re.hi, -b.re.lo}), add_raw(a.im, F2{-b.im.hi, -b.im.lo})};
}
__device__ __forceinline__ Z zmul_raw(Z a, Z w) {    // a w, raw sums
    return Z{add_raw(df::mul(a.re, w.re), dneg(df::mul(a.im, w.im))), add_raw(df::mul(a.re, w.im), df::mul(a.im, w.re))};
}
__device__ __forceinline__ Z zmulc_raw(Z a, Z w) {   // a conj(w), raw sums
    return Z{add_raw(df::mul(a.re, w.re), df::mul(a.im, w.im)), add_raw(df::mul(a.im, w.re), dneg(df::mul(a.re, w.im)))};
}
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
__device__ __forceinline__ Z zpow2(Z a, float s) {   // a s, s a power of two (exact)
    return Z{F2{s * a.re.hi, s * a.re.lo}, F2{s * a.im.hi, s * a.im.lo}};
}
__device__ __forceinline__ Z zfma_raw(F2 s, Z a, Z b) {  // b + s a, raw sum
    return Z{add_raw(b.re, df::mul(a.re, s)), add_raw(b.im, df::mul(a.im, s))};
}
__device__ __forceinline__ Z zld(const float4 *p) {
    const float4 v = __ldg(p);
    return Z{F2{v.x, v.y}, F2{v.z, v.w}};
}


// n / d as a float-float, for integers 0 < n, d < 2^13 held exactly in float32: hi from an
// approximate quotient, the remainder n - hi d exactly by one FMA (a multiple of hi's ulp,
// at most a few of them), lo = remainder / d with one correction step.  Relative error of
// hi + lo below 2^-46 (checked for every ratio the transforms use, with the reciprocal off
// by up to 2 ulp).  The psi coefficients are formed this way in registers: read from a
// table they missed L1 (which holds ~28 KB beside the kernels' shared memory) and their
// L2 latency sat on every thread's dependent chain (inverse psi 13.1 -> 11.0 ms).
__device__ __forceinline__ F2 ratio(float n, float d) {
    const float r = __fdividef(1.0f, d);
    const float hi = n * r;
    const float rem = __fmaf_rn(-hi, d, n);
    const float lo = rem * r;
    return F2{hi, __fmaf_rn(__fmaf_rn(-lo, d, rem), r, lo)};
}

// Raw (unrenormalised) sums in the FFT passes of the scalar products and forward transforms
// too.  The inverse transform always uses them.  The Makhoul pair step and the basis
// combination stay renormalised: with the earlier banded mass solve, which amplified the
// scalar products' error by the conditioning of B, raw sums there raised the forward
// transform's error on smooth spectra 15- to 300-fold.
constexpr bool kRawForward = true;

// Position of frequency k after the in-place DIF passes (radix 4 first, then one radix 2
// when log2 N is odd): the first pass puts k mod 4 in quarter (k mod 4), and so on, so
// the base-4 digits of k come out reversed (times 2, plus the radix-2 digit, for odd lg).
__device__ __forceinline__ uint32_t rev4(uint32_t x, int nd) {   // reverse nd base-4 digits
    if (nd == 0) return 0u;
    uint32_t r = __brev(x) >> (32 - 2 * nd);
    return ((r & 0x55555555u) << 1) | ((r >> 1) & 0x55555555u);
}
__device__ __forceinline__ int dpos2(int k, int lg) {
    const int nd = lg >> 1;
    if ((lg & 1) == 0) return (int)rev4((uint32_t)k, nd);
    const uint32_t low = (uint32_t)k & ((1u << (lg - 1)) - 1u);
    return (int)(2u * rev4(low, nd) + ((uint32_t)k >> (lg - 1)));
}
// FFT length f3 2^lg (f3 = 1 or 3): with a leading radix-3 pass frequency k = 3 k' + m sits
// in third m of the array, at the power-of-two position of k' there.
__device__ __forceinline__ int dpos(int k, int lg, int f3) {
    if (f3 == 1) return dpos2(k, lg);
    const int m = k % 3;
    return (m << lg) + dpos2(k / 3, lg);
}

__device__ __forceinline__ F2 lo2(float4 v) { return F2{v.x, v.y}; }
__device__ __forceinline__ F2 hi2(float4 v) { return F2{v.z, v.w}; }


// Physical slot of FFT position p in a group's column buffer A.  After the DIF passes
// frequency k sits at dpos(k), whose top bits come from k's low bits, so eight consecutive
// frequencies read by the eight lanes of a 16-byte access phase would share one bank group
// (8-way conflicts).  XORing position bits lg-1, lg-2 and lg-4 (filled from k's bits 0, 1,
// 2; lg the power-of-two part of the FFT length) into the low three bits spreads them over
// all eight (the XOR only permutes inside aligned blocks of eight).  The layout changes at
// the FFT's last pass: the pre-processing and the FFT passes use natural slots, the last
// pass stores position p at slot swz(p), and every access after the FFT goes through swz.
// s = lg - 4 >= 3, or 0: no swizzle (short columns).
__device__ __forceinline__ int swz(int p, int s) {
    return s ? p ^ (((p >> (s + 2)) & 3) | (((p >> s) & 1) << 2)) : p;
}

// In-place FFT of the group's column A[0 .. NF), NF = f3 2^lg (f3 = 1 or 3): forward
// e^{-2 pi i jk/NF}, or (INV) e^{+...}, unnormalised, output in dpos() order.
// f3 = 3: a radix-3 decimation-in-frequency pass first (tw[0] = e^{-2 pi i/3}; tw[1 + 2 n],
// tw[2 + 2 n] = e^{-2 pi i n/NF}, e^{-2 pi i 2n/NF}, n < Q = NF/3) splits the column into
// three transforms of length 2^lg, which the radix-4 passes then run side by side.
// tw (after the radix-3 part): per radix-4 pass p (span L = 2^lg / 4^p, Q = L/4), entries
// [3 j + m - 1] = e^{-2 pi i m j 4^p / 2^lg}, j < Q, m = 1, 2, 3, passes stored one after the
// other, so a pass reads its twiddles contiguously.
template <bool INV, bool RAW>
__device__ void fft_dif(float4 *A, int lg, int f3, const float4 *tw, const Group &g, int sw) {
    const int N = f3 << lg, half = N >> 1;
    int lgL = lg;
    const float4 *twp = tw;
    if (f3 == 3) {
        const int Q = 1 << lg;
        const float4 om = tw[0];
        const F2 c = lo2(om), sn = INV ? dneg(hi2(om)) : hi2(om);    // cos, sin of -+2 pi/3
        for (int b = g.t; b < Q; b += g.nt) {
            const Z a0 = ldz(A, b), a1 = ldz(A, b + Q), a2 = ldz(A, b + 2 * Q);
            const Z t1 = zadd(a1, a2), t2 = zsub(a1, a2);
            // a0 + w a1 + w^2 a2 and a0 + w^2 a1 + w a2 (w = c + i sn, w^2 = conj(w)):
            // m + i sn t2 and m - i sn t2, m = a0 + c t1
            const Z m = zfma(c, t1, a0);
            const Z s = zi(Z{df::mul(t2.re, sn), df::mul(t2.im, sn)});
            Z y1 = zadd(m, s), y2 = zsub(m, s);
            const Z y0 = zadd(a0, t1);
            if (b != 0) {
                const Z w1 = ldz(tw, 1 + 2 * b), w2 = ldz(tw, 2 + 2 * b);
                y1 = INV ? zmulc(y1, w1) : zmul(y1, w1);
                y2 = INV ? zmulc(y2, w2) : zmul(y2, w2);
            }
            stz(A, b, y0);
            stz(A, b + Q, y1);
            stz(A, b + 2 * Q, y2);
        }
        twp += 1 + 2 * Q;
        g.sync();
    }
    auto bfly4 = [&](Z a, Z bb, Z c, Z d, Z &y0, Z &y1, Z &y2, Z &y3) {   // untwiddled outputs
        const Z s0 = zadd_raw(a, c), s1 = zsub_raw(a, c), s2 = zadd_raw(bb, d), s3 = zsub_raw(bb, d);
        auto sum = [](Z u, Z v) { return RAW ? zadd_raw(u, v) : zadd(u, v); };
        y0 = sum(s0, s2);
        y2 = sum(s0, zneg(s2));
        y1 = sum(s1, INV ? zi(s3) : zmi(s3));
        y3 = sum(s1, INV ? zmi(s3) : zi(s3));
    };
    for (; lgL >= 2; lgL -= 2) {
        const int lgQ = lgL - 2, Q = 1 << lgQ;
        if (lgL == 2 && sw) {
            // last pass (no radix-2 follows), stores to the swizzled slots: the slots of
            // butterflies b and b ^ 1 (one aligned block of eight, two lanes of one warp) mix,
            // so every lane of the warp loads before any stores (uniform trip count)
            const int nb = N >> 2;
            for (int b0 = 0; b0 < nb; b0 += g.nt) {
                const int b = b0 + g.t, base = b << 2;
                Z y0 = kZero, y1 = kZero, y2 = kZero, y3 = kZero;
                if (b < nb)
                    bfly4(ldz(A, base), ldz(A, base + 1), ldz(A, base + 2), ldz(A, base + 3), y0, y1, y2, y3);
                __syncwarp();
                if (b < nb) {
                    stz(A, swz(base, sw), y0);
                    stz(A, swz(base + 1, sw), y1);
                    stz(A, swz(base + 2, sw), y2);
                    stz(A, swz(base + 3, sw), y3);
                }
                __syncwarp();
            }
            g.sync();
            continue;
        }
#pragma unroll 2
        for (int b = g.t; b < (N >> 2); b += g.nt) {
            const int j = b & (Q - 1);
            const int base = ((b >> lgQ) << lgL) + j;
            Z y0, y1, y2, y3;
            bfly4(ldz(A, base), ldz(A, base + Q), ldz(A, base + 2 * Q), ldz(A, base + 3 * Q), y0, y1, y2, y3);
            if (j != 0) {
                Z w1 = ldz(twp, 3 * j), w2 = ldz(twp, 3 * j + 1), w3 = ldz(twp, 3 * j + 2);
                if (INV) {
                    y1 = RAW ? zmulc_raw(y1, w1) : zmulc(y1, w1);
                    y2 = RAW ? zmulc_raw(y2, w2) : zmulc(y2, w2);
                    y3 = RAW ? zmulc_raw(y3, w3) : zmulc(y3, w3);
                } else {
                    y1 = RAW ? zmul_raw(y1, w1) : zmul(y1, w1);
                    y2 = RAW ? zmul_raw(y2, w2) : zmul(y2, w2);
                    y3 = RAW ? zmul_raw(y3, w3) : zmul(y3, w3);
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
        // last pass: as above, the four lanes of an aligned block of eight load before any
        // of them stores to the swizzled slots
        for (int b0 = 0; b0 < half; b0 += g.nt) {
            const int b = b0 + g.t;
            Z y0 = kZero, y1 = kZero;
            if (b < half) {
                const Z a = ldz(A, 2 * b), c = ldz(A, 2 * b + 1);
                y0 = zadd(a, c);
                y1 = zsub(a, c);
            }
            __syncwarp();
            if (b < half) {
                stz(A, swz(2 * b, sw), y0);
                stz(A, swz(2 * b + 1, sw), y1);
            }
            __syncwarp();
        }
        g.sync();
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
    int N, lg, f3;           // Chebyshev modes; FFT length (N, or 2 (N - 1) on Gauss-Lobatto points) = f3 2^lg
    int G, n_groups;         // warps per mode group, groups per block
    long n_modes;
    int stride;              // float4 per buffer
    int n_tw;                // float4 of the per-pass twiddle table (copied to shared memory)
    const float4 *tw;        // per-pass twiddles
    const float4 *mk;        // e^{-i pi k/(2N)}, k = 0 .. N/2
    int *err;                // set to 1 if a column copy did not complete
    F2 pi_over_N;
    // forward transforms in phi / psi, per parity h: ls[h] = (rho_h, kappa_h, tau_h) of the
    // least-squares correction (forward_ls)
    F2 ls[2][3];
};

// Two buffers of `stride` float4 per mode group, A and R (= B).  The column copy lands in
// R; the next mode's copy is issued as soon as R is free, so it overlaps the current
// mode's FFT.
constexpr int kBuffers = 2;

// float4 of per-group shared scratch of the forward transforms in phi / psi (warp totals
// of their sums, up to 4 warps): [0, 8) and [16, 24) scans, [8, 16) sums.
constexpr int kScratch = 24;



// Forward transform in phi (SPACE 1) or psi (SPACE 2), uhat = B^{-1} S (Eqs. sst2, fstB),
// from the column's Chebyshev coefficients chat (chat_K = (u, T_K)_sigma / w_K, w_K =
// pi c_K / 2) without a banded solve.  The discrete norms make B = P^T W P, with W =
// diag(w_K) and P the basis combination (phi_l = sum_K P_Kl T_K, Eqs. phiD, phiN), and
// S = P^T W chat, so uhat is the W-weighted least-squares solution of P uhat = chat.  Per
// parity (K = 2 i + h over the Chebyshev indices K < N of that parity):
//   phi: (P uhat)_K = uhat_i - uhat_{i-1};
//   psi: P = (I - Shift)(I - b Shift), b_i = (K - 1) / (K + 1), since 1 + b_i = 2K / (K + 1)
//        and b_{i-1} = (K - 3) / (K - 1) are the combination's coefficients of Eq. phiN at
//        row K.
// The residual chat - P uhat of the least-squares solution is W^{-1} times a vector of the
// null space of P^T (phi: constants; psi: constants and K^2, orthogonalised in the weight
// omega_K = 1 / c_K as q_K = K^2 - kappa), fixed by asking chat - r to lie in the range of P:
//   r_K = omega_K (cr + cq q_K),  cr = rho sum_K chat_K,  cq = tau sum_K q_K chat_K,
//   rho = 1 / sum omega, kappa = sum omega K^2 / sum omega, tau = 1 / sum omega q^2
// (cq for psi only; rho, kappa, tau per parity from the plan).  The triangular part of P
// then inverts as prefix sums over the parity, and the prefix sums of r have closed forms
// (Omega_K = sum_{m <= K} omega_m = (K + 1) / 2, sum_{m <= K} omega_m m^2 = K (K+1) (K+2) / 6
// for either parity), so with P_K = sum_{m <= K} chat_m:
//   phi: uhat_K = P_K - cr Omega_K;
//   psi: v_K = P_K - cr Omega_K - cq Q_K,  Q_K = K (K+1) (K+2) / 6 - kappa Omega_K,
//        uhat_K = (K + 1)^-1 sum_{m <= K} (m + 1) v_m
// (the last from uhat_i = v_i + b_i uhat_{i-1}: the products of b telescope).
// Every thread of the group owns a run of cpt = 2^lc >= 8 natural indices (from t cpt) and
// keeps its running sums there; the sums across runs go through warp shuffles and the
// group's scratch `scr` (2 float4 per warp and quantity).  The first pass reads the
// Chebyshev coefficients from the FFT's digit-reversed positions in A; the later ones work
// in W (the group's free staging buffer) at k ^ (t & 7): the eight lanes of a 16-byte access
// phase then fall on distinct bank groups (W is not swizzled by swz).
template <int SPACE, bool GL, class ChatFn>
__device__ __forceinline__ void forward_ls(const TrArgs &a, float4 *W, float4 *scr, const Group &g, ChatFn chat,
                                           int n, double2 *y) {
    const int N = a.N;
    const int lane = g.t & 31, warp = g.t >> 5, nw = g.nt >> 5;
    int lc = 3;
    while ((g.nt << lc) < N) lc++;
    const int k0 = min(N, g.t << lc), k1 = min(N, k0 + (1 << lc)), kn = min(k1, n), rx = g.t & 7;
    // pass 1: prefix sums of chat within the run (per parity); psi: sums of K^2 chat (the
    // sums of q chat = K^2 chat - kappa chat follow from them and the totals of chat)
    Z t0 = kZero, t1 = kZero, q[2] = {kZero, kZero};
    for (int k = k0; k < k1; k++) {
        const Z c = chat(k);
        const float kk = (float)k * (float)k;          // exact: k < 4096
        if (k & 1) {
            t1 = zadd(t1, c);
            stz(W, k ^ rx, t1);
            if (SPACE == 2) q[1] = zaddmulf(q[1], c, kk);
        } else {
            t0 = zadd(t0, c);
            stz(W, k ^ rx, t0);
            if (SPACE == 2) q[0] = zaddmulf(q[0], c, kk);
        }
    }
    if (SPACE == 2) {                                // warp sums of K^2 chat, beside the scan's
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            q[0] = zadd(q[0], zshfl_xor(q[0], o));
            q[1] = zadd(q[1], zshfl_xor(q[1], o));
        }
        if (lane == 0) {
            stz(scr + 8, 2 * warp, q[0]);
            stz(scr + 8, 2 * warp + 1, q[1]);
        }
    }
    Z s0, s1;
    group_prefix(g, scr, t0, t1, s0, s1);               // its barrier also covers the sums above
    if (SPACE == 2) {
        q[0] = ldz(scr + 8, 0);
        q[1] = ldz(scr + 8, 1);
        for (int w = 1; w < nw; w++) {
            q[0] = zadd(q[0], ldz(scr + 8, 2 * w));
            q[1] = zadd(q[1], ldz(scr + 8, 2 * w + 1));
        }
    }
    const Z cr0 = zscale(s0, a.ls[0][0]), cr1 = zscale(s1, a.ls[1][0]);
    if (SPACE == 1) {
        for (int k = k0; k < kn; k++) {
            const bool odd = k & 1;
            stz(W, k ^ rx, zsubmulf(zadd(ldz(W, k ^ rx), odd ? t1 : t0), odd ? cr1 : cr0, 0.5f * (float)(k + 1)));
        }
    } else {
        const Z cq0 = zscale(zsubmul(q[0], s0, a.ls[0][1]), a.ls[0][2]);      // tau (sum K^2 chat - kappa sum chat)
        const Z cq1 = zscale(zsubmul(q[1], s1, a.ls[1][1]), a.ls[1][2]);
        const F2 sixth = ratio(1.0f, 6.0f);
        // pass 2: v, then the prefix sums of (K + 1) v within the run
        Z z0 = kZero, z1 = kZero;
        for (int k = k0; k < kn; k++) {
            const bool odd = k & 1;
            const float kf = (float)k, om = 0.5f * (kf + 1.0f);
            const F2 s2 = nrm(df::mul(nrm(df::mul(df::two_prod(kf, kf + 1.0f), kf + 2.0f)), sixth));
            const F2 Q = df::add(s2, dneg(df::mul(a.ls[k & 1][1], om)));
            Z v = zsubmulf(zadd(ldz(W, k ^ rx), odd ? t1 : t0), odd ? cr1 : cr0, om);
            v = zsubmul(v, odd ? cq1 : cq0, Q);
            if (odd) {
                z1 = zaddmulf(z1, v, kf + 1.0f);
                stz(W, k ^ rx, z1);
            } else {
                z0 = zaddmulf(z0, v, kf + 1.0f);
                stz(W, k ^ rx, z0);
            }
        }
        Z u0, u1;
        group_prefix(g, scr + 16, z0, z1, u0, u1);
        for (int k = k0; k < kn; k++)
            stz(W, k ^ rx, zscale(zadd(ldz(W, k ^ rx), (k & 1) ? z1 : z0), ratio(1.0f, (float)(k + 1))));
    }
    g.sync();
    for (int k = g.t; k < N; k += g.nt) y[k] = k < n ? ztof64(ldz(W, k ^ ((k >> lc) & 7))) : make_double2(0.0, 0.0);
}

// KIND: 0 inverse, 1 scalar products, 2 forward (phi, psi: forward_ls on the Chebyshev
// coefficients).  SPACE: 0 T_k, 1 phi_k, 2 psi_k.  GL: Gauss-Lobatto points (a compile-time choice, so the Gauss kernels carry none
// of its code).
template <int KIND, int SPACE, bool GL>
__global__ void __launch_bounds__(768) transform_kernel(TrArgs a, const double *in, double *out) {
    extern __shared__ float4 sm[];
    const int N = a.N, lg = a.lg, f3 = a.f3, half = N >> 1, M = N - 1;
    // slot swizzle of A (swz) for the scalar products and forward transforms, whose
    // post-processing reads the digit-reversed positions two to four times per point; the
    // inverse reads them once, where the swizzle's own instructions cost more than it saves
    const int sw = (KIND != 0 && lg >= 7) ? lg - 4 : 0;
    const float4 *tw = sm;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + a.n_tw);
    for (int t = threadIdx.x; t < a.n_tw; t += blockDim.x) sm[t] = __ldg(a.tw + t);
    const int gsize = 32 * a.G, gi = threadIdx.x / gsize;
    const Group g{(int)threadIdx.x - gi * gsize, gsize, 1 + gi};
    float4 *A = sm + a.n_tw + 8 + (long)gi * kBuffers * a.stride;
    float4 *Bf = A + a.stride;
    float4 *R = Bf;
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
    constexpr bool kLs = KIND == 2 && SPACE != 0;   // forward phi / psi (forward_ls)
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
                if (SPACE == 1 && k >= 2) t = zsub_raw(t, ldz(Bf, k - 2));
                if (SPACE == 2 && k >= 2) {
                    // psi_j = T_j - 2(j+2)/(j+3) T_{j+2} + (j+1)/(j+3) T_{j+4}, so t_k takes
                    // -2k/(k+1) c_{k-2} + (k-3)/(k-1) c_{k-4}
                    const float kf = (float)k;
                    t = zfma_raw(dneg(ratio(2.0f * kf, kf + 1.0f)), ldz(Bf, k - 2), t);
                    if (k >= 4) t = zfma_raw(ratio(kf - 3.0f, kf - 1.0f), ldz(Bf, k - 4), t);
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
                fft_dif<false, kRawForward>(A, lg, f3, tw, g, sw);
                for (int i = g.t; i < N; i += g.nt) {
                    const Z e = zadd(t0, (i & 1) ? Z{dneg(tM.re), dneg(tM.im)} : tM);
                    y[i] = ztof64(zhalf(zadd(ldz(A, swz(dpos(i, lg, f3), sw)), e)));
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
                stz(A, k, zhalf(zmulc_raw(zadd_raw(t1, zmi(t2)), w)));
                if (k != half) stz(A, N - k, zhalf(zi(zmul_raw(zadd_raw(t2, zmi(t1)), w))));
            }
            prefetch_next(next);
            fft_dif<true, true>(A, lg, f3, tw, g, sw);
            for (int m = g.t; m < N; m += g.nt) {
                const int src = (m & 1) ? N - 1 - (m >> 1) : (m >> 1);
                y[m] = ztof64(ldz(A, swz(dpos(src, lg, f3), sw)));
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
                if (kLs)
                    g.sync();                  // A written by every thread before the FFT reads it
                else
                    prefetch_next(next);       // (its barrier orders A's writes the same way)
                fft_dif<false, kRawForward>(A, lg, f3, tw, g, sw);
            } else {
            // values -> Makhoul order in A; R free for the next column (the forward phi / psi
            // kernels use R as forward_ls's work buffer and load the next column after it)
            for (int m = g.t; m < N; m += g.nt) {
                const int dst = (m & 1) ? N - 1 - (m >> 1) : (m >> 1);
                stz(A, dst, zfromf64(xs[m]));
            }
            if (kLs)
                g.sync();
            else
                prefetch_next(next);
            fft_dif<false, kRawForward>(A, lg, f3, tw, g, sw);
            // C_k (DCT-II) in place: the pair (k, N-k) is read and written by one thread at
            // positions dpos(k), dpos(N-k)
            for (int k = g.t; k <= half; k += g.nt) {
                if (k == 0) continue;                                  // C_0 = V_0
                const int pk = dpos(k, lg, f3), pn = dpos(N - k, lg, f3);
                const Z w = mkz(k);
                const Z P = zmul(ldz(A, swz(pk, sw)), w);
                const Z Q = zmulc(ldz(A, swz(pn, sw)), w);
                stz(A, swz(pk, sw), zhalf(zadd(P, Q)));
                if (k != half) stz(A, swz(pn, sw), zhalf(zi(zsub(P, Q))));
            }
            }
            g.sync();
            auto C = [&](int k) { return ldz(A, swz(dpos(k, lg, f3), sw)); };
            if (KIND == 2) {
                // Chebyshev coefficients chat_k = S_k / (pi c_k / 2): Gauss: C_k 2 / (N c_k)
                // (c_0 = 2); Gauss-Lobatto: Y_k / (M c_k) (c_0 = c_M = 2).  2 / N or 1 / M is a
                // power of two for power-of-two lengths; with a factor 3 it is applied as a
                // float-float quotient.
                const float sc = GL ? 1.0f / (float)M : 2.0f / (float)N;
                const F2 scd = GL ? ratio(1.0f, (float)M) : ratio(2.0f, (float)N);
                auto chat = [&](int k) -> Z {
                    const float h = (k == 0 || (GL && k == M)) ? 0.5f : 1.0f;
                    return f3 == 1 ? zpow2(C(k), h * sc) : zpow2(zscale(C(k), scd), h);
                };
                if (SPACE == 0) {
                    for (int k = g.t; k < N; k += g.nt) y[k] = ztof64(chat(k));
                } else {
                    forward_ls<SPACE, GL>(a, R, sm + a.n_tw + 8 + (long)a.n_groups * kBuffers * a.stride +
                                                     (long)gi * kScratch,
                                          g, chat, n, y);
                    prefetch_next(next);
                }
            } else {
                // scalar products S_l (Algorithm fst, forwardScalar)
                auto S = [&](int l) -> Z {
                    if (l >= n) return kZero;
                    Z v = C(l);
                    if (SPACE == 1) v = zsub(v, C(l + 2));
                    if (SPACE == 2) {
                        // Eq. phiN: psi_l = T_l - 2(l+2)/(l+3) T_{l+2} + (l+1)/(l+3) T_{l+4}
                        const float lf = (float)l;
                        v = zfma(dneg(ratio(2.0f * lf + 4.0f, lf + 3.0f)), C(l + 2), v);
                        v = zfma(ratio(lf + 1.0f, lf + 3.0f), C(l + 4), v);
                    }
                    return zscale(v, a.pi_over_N);
                };
                for (int l = g.t; l < N; l += g.nt) y[l] = ztof64(S(l));
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

// Warps per mode group of an N-mode plan (more threads per column for larger N).
int group_warps(int N) { return std::max(1, std::min(4, N / 256)); }

}  // namespace

namespace {
bool pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }
}  // namespace

// Gauss points: N a power of two or three times one (FFT length N); Gauss-Lobatto points:
// N - 1 such a number (FFT length 2 (N - 1)).
bool transform_supported(const Plan &p) {
    const int L = p.gl ? p.N - 1 : p.N;
    return p.N >= 8 && L >= 8 && (pow2(L) || (L % 3 == 0 && pow2(L / 3)));
}

namespace {
int fft_length(const Plan &p) { return p.gl ? 2 * (p.N - 1) : p.N; }
int fft_f3(int NF) { return pow2(NF) ? 1 : 3; }
}  // namespace

// Number of float4 of the per-pass twiddle table: 1 + 2 Q for a radix-3 pass (NF = 3 Q),
// then 3 Q per radix-4 pass.
int twiddle_count(int NF) {
    const int f3 = fft_f3(NF);
    int c = f3 == 3 ? 1 + 2 * (NF / 3) : 0;
    for (int lgL = ilog2(NF / f3); lgL >= 2; lgL -= 2) c += 3 * (1 << (lgL - 2));
    return c;
}

// Tables of the transforms of an N-mode plan (float4 units, float-float pairs):
//   [0, ntw)                per-pass twiddles of fft_dif
//   [ntw, ntw + N/2 + 1)    mk[k] = e^{-i pi k/(2N)}, k = 0 .. N/2
// and the constants of the forward transforms' least-squares correction (forward_ls).
cudaError_t transform_setup(Plan &p, long long &bytes, cudaStream_t s) {
    if (!transform_supported(p)) return cudaSuccess;
    const int N = p.N, NF = fft_length(p), f3 = fft_f3(NF), L2 = NF / f3, lg = ilog2(L2);
    const long double pi = 3.141592653589793238462643383279502884L;
    // per parity h over the Chebyshev indices K = h, h + 2, .. < N with omega_K = 1 / c_K
    // (1/2 at K = 0, and at K = N - 1 on Gauss-Lobatto points):
    // rho = 1 / sum omega, kappa = sum omega K^2 / sum omega, tau = 1 / sum omega (K^2 - kappa)^2
    for (int h = 0; h < 2; h++) {
        long double so = 0.0L, sk = 0.0L;
        for (int K = h; K < N; K += 2) {
            const long double om = (K == 0 || (p.gl && K == N - 1)) ? 0.5L : 1.0L;
            so += om;
            sk += om * (long double)K * K;
        }
        const long double kap = sk / so;
        long double sq = 0.0L;
        for (int K = h; K < N; K += 2) {
            const long double om = (K == 0 || (p.gl && K == N - 1)) ? 0.5L : 1.0L, q = (long double)K * K - kap;
            sq += om * q * q;
        }
        const long double c[3] = {1.0L / so, kap, 1.0L / sq};
        for (int j = 0; j < 3; j++) {
            const float hi = (float)c[j];
            p.tr_ls[h][j][0] = hi;
            p.tr_ls[h][j][1] = (float)(c[j] - (long double)hi);
        }
    }
    const int ntw = twiddle_count(NF), nmk = N / 2 + 1;
    std::vector<float4> tab;
    tab.reserve((size_t)ntw + nmk);
    if (f3 == 3) {                                                     // radix-3 pass
        tab.push_back(pair4(cosl(-2 * pi / 3), sinl(-2 * pi / 3)));
        for (int n = 0; n < L2; n++)
            for (int m = 1; m <= 2; m++) {
                const long double ang = -2 * pi * (long double)(m * n) / NF;
                tab.push_back(pair4(cosl(ang), sinl(ang)));
            }
    }
    for (int lgL = lg, sh = 0; lgL >= 2; lgL -= 2, sh += 2) {           // radix-4 passes on 2^lg
        const int Q = 1 << (lgL - 2);
        for (int j = 0; j < Q; j++)
            for (int m = 1; m <= 3; m++) {
                const long t = ((long)m * j) << sh;                    // < 3 L2 / 4
                const long double ang = -2 * pi * (long double)t / L2;
                tab.push_back(pair4(cosl(ang), sinl(ang)));
            }
    }
    for (int k = 0; k < nmk; k++) {
        const long double ang = -pi * k / (2 * (long double)N);
        tab.push_back(pair4(cosl(ang), sinl(ang)));
    }
    p.tr_ntw = ntw;
    bytes += (long long)(tab.size() * sizeof(float4));
    cudaError_t e = cudaMalloc((void **)&p.d_tr, tab.size() * sizeof(float4));
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(p.d_tr, tab.data(), tab.size() * sizeof(float4), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    // launch shape per (kind, space): G warps per mode group (more threads per column for
    // larger N), groups per block from the shared memory budget (twiddles, barriers,
    // nbuf buffers per group, and the forward phi / psi kernels' scratch) and the kernel's
    // 768-thread bound; persistent grid from the occupancy.  A (kind, space) whose buffers
    // do not fit gets no shape (unsupported).
    int dev = 0, smem_max = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess)
        return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int stride = NF + 4;
    p.tr_stride = stride;
    const int G = group_warps(N);
    const long fixed = (long)(ntw + 8) * sizeof(float4);
    for (int kind = 0; kind < 3; kind++)
        for (int space = 0; space < 3; space++) {
            const long per_group = ((long)kBuffers * stride + (kind == 2 && space != 0 ? kScratch : 0)) *
                                   (long)sizeof(float4);
            const int max_threads = 768;                 // the kernel's bound
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
    const int N = p.N, k = kind;
    TrArgs a;
    a.N = N;
    a.f3 = fft_f3(fft_length(p));
    a.lg = ilog2(fft_length(p) / a.f3);
    a.G = p.tr_G;
    a.n_groups = p.tr_groups[k][space];
    a.n_modes = count;
    a.stride = p.tr_stride;
    a.n_tw = p.tr_ntw;
    a.tw = p.d_tr;
    a.mk = p.d_tr + p.tr_ntw;
    const double pn = p.gl ? kPi / (2.0 * (N - 1)) : kPi / N;   // weight of the point sum
    const float ph = (float)pn;
    a.pi_over_N = F2{ph, (float)(pn - (double)ph)};
    a.err = p.d_err + 3;
    for (int h = 0; h < 2; h++)
        for (int j = 0; j < 3; j++) a.ls[h][j] = F2{p.tr_ls[h][j][0], p.tr_ls[h][j][1]};
    const long need = (count + a.n_groups - 1) / a.n_groups;
    const dim3 grid((unsigned)std::max<long>(1, std::min<long>(p.tr_grid[k][space], need))),
        block((unsigned)(32 * a.G * a.n_groups));
    void *args[] = {&a, &in, &out};
    const cudaError_t e = cudaLaunchKernel(kernel_of(k, space, p.gl), grid, block, args, (size_t)p.tr_smem[k][space], s);
    return e;
}

}  // namespace shen
