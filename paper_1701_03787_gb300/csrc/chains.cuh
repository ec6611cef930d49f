// Per-chain bodies of the thread-per-chain kernels, shared by the single-channel and
// the batched (many instances, uneven N) launches.  A chain is one parity (k = 2 i + par)
// of one mode's column; the real and imaginary parts run side by side.
//
// Source: Mortensen, arXiv:1701.03787, Sec. 4 (Helmholtz odd/even LU; Algorithms
// LUbiharmonic, ReduceAB, LUSolveBiharmonic with the Eq. ab tail).
#pragma once
#include "df.cuh"
#include "shen_internal.h"

namespace shen {
namespace chains {

// err[0]: any bad pivot; err[1]: smallest class with one; err[2]: number of chains with one
__device__ __forceinline__ void flag_error(int *err, long cls) {
    atomicExch(err, 1);
    atomicMin(err + 1, (int)cls);
}
__device__ __forceinline__ bool bad_pivot(double v) { return !(fabs(v) > 0.0) || !isfinite(v); }
__device__ __forceinline__ double2 ld2(const double *p, long idx) {
    return reinterpret_cast<const double2 *>(p)[idx];
}
__device__ __forceinline__ void st2(double *p, long idx, double2 v) {
    reinterpret_cast<double2 *>(p)[idx] = v;
}

// ---------------------------------------------------------------- factorisation

// Helmholtz, per parity chain:  M = alpha B - A restricted to k = 2i + p:
//   M_{i,i-1} = -h (h = alpha pi/2),  M_ii = alpha B_kk - A_kk,
//   M_{i,i+1} = -h + t_i,  M_{i,j>=i+2} = t_i  with t_i = -A_tail(k) = 4 pi (k+1).
// Doolittle without pivoting: l_i = M_{i,i-1}/U0_{i-1}; U_i* = M_i* - l_i U_{i-1,*};
// the tail and the superdiagonal stay constant-offset: U1_i = U2_i - h.
// F: rows_max rows of kHelmF64 doubles (1/U0, U2, l, 0); rows past the chain are zeroed.
__device__ inline void factor_helm_chain(const RowTables &T, int N, double z2, double c, int par, double *F,
                                         int rows_max, int *err, long cls) {
    const int n = N - 2;
    const int rows = (n - par + 1) / 2;
    const double alpha = z2 + c;
    const double h = alpha * kPi / 2;
    double U0 = 0, U2 = 0;
    bool bad = false;
    for (int i = 0; i < rows; i++) {
        const int k = 2 * i + par;
        const double t = -T.adt[k];
        const double Mii = alpha * T.bd0[k] - T.ad0[k];
        double l = 0.0;
        if (i == 0) {
            U0 = Mii;
            U2 = t;
        } else {
            l = -h / U0;
            const double U1prev = U2 - h;
            U0 = Mii - l * U1prev;
            U2 = t - l * U2;
        }
        if (bad_pivot(U0)) {
            flag_error(err, cls);
            bad = true;
        }
        F[i * kHelmF64 + 0] = 1.0 / U0;
        F[i * kHelmF64 + 1] = U2;
        F[i * kHelmF64 + 2] = l;
        F[i * kHelmF64 + 3] = 0.0;
    }
    for (int i = rows; i < rows_max; i++)
        for (int v = 0; v < kHelmF64; v++) F[i * kHelmF64 + v] = 0.0;
    if (bad) atomicAdd(err + 2, 1);
}

// Biharmonic, per parity chain (k = 2i + p), H = Q + ca A + cb B:
//   H_{i,i-2} = cb B_{k,k-4}; H_{i,i-1} = ca A_{k,k-2} + cb B_{k,k-2};
//   H_ii = Q_kk + ca A_kk + cb B_kk; H_{i,i+1} = Q_{k,k+2} + ca A_{k,k+2} + cb B_{k,k+2};
//   H_{i,i+2} = Q_{k,k+4} + cb B_{k,k+4};  H_{i,j>=i+3} = p_k q_j + r_k s_j.
// Algorithm LUbiharmonic row update, with rows i-1, i-2 beyond their three stored
// values taken from Eq. ab (tail T_m(j) = ta_m q_j + tb_m s_j), and ReduceAB for ta, tb.
// F: rows_max rows of kBiF64 doubles (L1, L2, 1/U0, U1, U2, ta, tb, 0).
__device__ inline void factor_bih_chain(const RowTables &T, int N, double z2, double c, int par, double *F,
                                        int rows_max, int *err, long cls) {
    const int n = N - 4;
    const int rows = (n - par + 1) / 2;
    const double ca = -(2.0 * z2 + c);
    const double cb = z2 * (z2 + c);
    // state of rows i-1 (suffix 1) and i-2 (suffix 2)
    double U0_1 = 0, U1_1 = 0, U2_1 = 0, ta_1 = 0, tb_1 = 0;
    double U0_2 = 0, U1_2 = 0, U2_2 = 0, ta_2 = 0, tb_2 = 0;
    bool bad = false;
    for (int i = 0; i < rows; i++) {
        const int k = 2 * i + par;
        auto q = [&](int kk) { return T.qk[kk]; };
        auto s = [&](int kk) { return T.sk[kk]; };
        double L2 = 0.0, L1 = 0.0;
        if (i >= 2) L2 = cb * T.bb4[k - 4] / U0_2;
        if (i >= 1) {
            double t = ca * T.abm[k] + cb * T.bb2[k - 2];
            if (i >= 2) t -= L2 * U1_2;               // U_{i-2,i-1}
            L1 = t / U0_1;
        }
        double U0 = T.qb0[k] + ca * T.ab0[k] + cb * T.bb0[k];
        if (i >= 2) U0 -= L2 * U2_2;                   // U_{i-2,i}
        if (i >= 1) U0 -= L1 * U1_1;                   // U_{i-1,i}
        double U1 = 0.0, U2 = 0.0;
        if (i + 1 < rows) {
            const int k1 = k + 2;
            U1 = T.pk[k] * q(k1) + T.rk[k] * s(k1) + ca * T.abp[k] + cb * T.bb2[k];
            if (i >= 2) U1 -= L2 * (ta_2 * q(k1) + tb_2 * s(k1));   // U_{i-2,i+1}: tail
            if (i >= 1) U1 -= L1 * U2_1;                              // U_{i-1,i+1}
        }
        if (i + 2 < rows) {
            const int k2 = k + 4;
            U2 = T.pk[k] * q(k2) + T.rk[k] * s(k2) + cb * T.bb4[k];
            if (i >= 2) U2 -= L2 * (ta_2 * q(k2) + tb_2 * s(k2));   // U_{i-2,i+2}: tail
            if (i >= 1) U2 -= L1 * (ta_1 * q(k2) + tb_1 * s(k2));   // U_{i-1,i+2}: tail
        }
        double ta = T.pk[k], tb = T.rk[k];
        if (i >= 1) { ta -= L1 * ta_1; tb -= L1 * tb_1; }
        if (i >= 2) { ta -= L2 * ta_2; tb -= L2 * tb_2; }
        if (bad_pivot(U0)) {
            flag_error(err, cls);
            bad = true;
        }
        double *row = F + i * kBiF64;
        row[0] = L1; row[1] = L2; row[2] = 1.0 / U0; row[3] = U1;
        row[4] = U2; row[5] = (i + 3 < rows) ? ta : 0.0; row[6] = (i + 3 < rows) ? tb : 0.0; row[7] = 0.0;
        U0_2 = U0_1; U1_2 = U1_1; U2_2 = U2_1; ta_2 = ta_1; tb_2 = tb_1;
        U0_1 = U0; U1_1 = U1; U2_1 = U2; ta_1 = ta; tb_1 = tb;
    }
    for (int i = rows; i < rows_max; i++)
        for (int v = 0; v < kBiF64; v++) F[i * kBiF64 + v] = 0.0;
    if (bad) atomicAdd(err + 2, 1);
}

// ------------------------------------------------------------- float64 sweeps

// f, u: the column's first complex element (u may equal f).  F: the chain's factors.
// rs: complex elements between consecutive Chebyshev indices of the column (1 for the
// mode-major layout, the plan's mode count for the wall-index-first one).
__device__ inline void solve_helm_fp64_chain(int N, int par, const double *f, double *u, const double *F,
                                             double h, long rs = 1) {
    const int n = N - 2;
    const int rows = (n - par + 1) / 2;
    const long base = 0;
    // forward elimination: y_i = f_i - l_i y_{i-1}.  Rows are loaded PB at a time ahead of
    // the stores (which may alias f when u == f) so that the loads overlap.
    constexpr int PB = 8;
    double2 y = make_double2(0.0, 0.0);
    for (int i0 = 0; i0 < rows; i0 += PB) {
        double2 fb[PB];
        double lb[PB];
#pragma unroll
        for (int q = 0; q < PB; q++) {
            const int i = min(i0 + q, rows - 1);
            fb[q] = ld2(f, base + (2 * i + par) * rs);
            lb[q] = F[i * kHelmF64 + 2];
        }
#pragma unroll
        for (int q = 0; q < PB; q++) {
            if (i0 + q < rows) {
                y.x = fma(-lb[q], y.x, fb[q].x);
                y.y = fma(-lb[q], y.y, fb[q].y);
                st2(u, base + (2 * (i0 + q) + par) * rs, y);
            }
        }
    }
    // back substitution: u_i = (y_i + h u_{i+1} - U2_i S_{i+1}) / U0_i, S_{i+1} = sum_{j>i} u_j
    double2 un = make_double2(0.0, 0.0), S = make_double2(0.0, 0.0);
    for (int i0 = rows - 1; i0 >= 0; i0 -= PB) {
        double2 yb[PB], ab[PB];
#pragma unroll
        for (int q = 0; q < PB; q++) {
            const int i = max(i0 - q, 0);
            yb[q] = ld2(u, base + (2 * i + par) * rs);
            ab[q] = *reinterpret_cast<const double2 *>(F + i * kHelmF64);   // (1/U0, U2), 32-byte rows
        }
#pragma unroll
        for (int q = 0; q < PB; q++) {
            if (i0 - q >= 0) {
                double2 t;
                t.x = fma(-ab[q].y, S.x, fma(h, un.x, yb[q].x));
                t.y = fma(-ab[q].y, S.y, fma(h, un.y, yb[q].y));
                un.x = ab[q].x * t.x;
                un.y = ab[q].x * t.y;
                S.x += un.x;
                S.y += un.y;
                st2(u, base + (2 * (i0 - q) + par) * rs, un);
            }
        }
    }
    if (par == 0) {
        st2(u, n * rs, make_double2(0.0, 0.0));
        st2(u, (n + 1) * rs, make_double2(0.0, 0.0));
    }
}

__device__ inline void solve_bih_fp64_chain(int N, int par, const double *f, double *u, const double *F,
                                            const double *qk, const double *sk, long rs = 1) {
    const int n = N - 4;
    const int rows = (n - par + 1) / 2;
    const long base = 0;
    constexpr int PB = 4;
    // forward elimination: y_i = f_i - L1_i y_{i-1} - L2_i y_{i-2} (loads PB rows ahead)
    double2 y1 = make_double2(0.0, 0.0), y2 = make_double2(0.0, 0.0);
    for (int i0 = 0; i0 < rows; i0 += PB) {
        double2 fb[PB], lb[PB];
#pragma unroll
        for (int q = 0; q < PB; q++) {
            const int i = min(i0 + q, rows - 1);
            fb[q] = ld2(f, base + (2 * i + par) * rs);
            lb[q] = *reinterpret_cast<const double2 *>(F + i * kBiF64);
        }
#pragma unroll
        for (int q = 0; q < PB; q++) {
            if (i0 + q < rows) {
                double2 y;
                y.x = fma(-lb[q].y, y2.x, fma(-lb[q].x, y1.x, fb[q].x));
                y.y = fma(-lb[q].y, y2.y, fma(-lb[q].x, y1.y, fb[q].y));
                st2(u, base + (2 * (i0 + q) + par) * rs, y);
                y2 = y1;
                y1 = y;
            }
        }
    }
    // back substitution (Algorithm LUSolveBiharmonic):
    //   u_i = (y_i - U1_i u_{i+1} - U2_i u_{i+2} - ta_i Sq - tb_i Ss) / U0_i,
    //   Sq = sum_{j>=i+3} q_j u_j, Ss = sum_{j>=i+3} s_j u_j (running sums per parity)
    double2 u1 = make_double2(0.0, 0.0), u2 = u1, u3 = u1, Sq = u1, Ss = u1;
    for (int i0 = rows - 1; i0 >= 0; i0 -= PB) {
        double2 yb[PB], b1[PB], b2[PB];
        double tbb[PB], qv[PB], sv[PB];
#pragma unroll
        for (int q = 0; q < PB; q++) {
            const int i = max(i0 - q, 0);
            yb[q] = ld2(u, base + (2 * i + par) * rs);
            b1[q] = *reinterpret_cast<const double2 *>(F + i * kBiF64 + 2);   // 1/U0, U1
            b2[q] = *reinterpret_cast<const double2 *>(F + i * kBiF64 + 4);   // U2, ta
            tbb[q] = F[i * kBiF64 + 6];
            const int k3 = min(2 * (i + 3) + par, n - 1);
            qv[q] = qk[k3];
            sv[q] = sk[k3];
        }
#pragma unroll
        for (int q = 0; q < PB; q++) {
            const int i = i0 - q;
            if (i >= 0) {
                if (i + 3 < rows) {
                    Sq.x = fma(qv[q], u3.x, Sq.x); Sq.y = fma(qv[q], u3.y, Sq.y);
                    Ss.x = fma(sv[q], u3.x, Ss.x); Ss.y = fma(sv[q], u3.y, Ss.y);
                }
                double2 t;
                t.x = yb[q].x - b1[q].y * u1.x - b2[q].x * u2.x - b2[q].y * Sq.x - tbb[q] * Ss.x;
                t.y = yb[q].y - b1[q].y * u1.y - b2[q].x * u2.y - b2[q].y * Sq.y - tbb[q] * Ss.y;
                const double2 ui = make_double2(b1[q].x * t.x, b1[q].x * t.y);
                st2(u, base + (2 * i + par) * rs, ui);
                u3 = u2;
                u2 = u1;
                u1 = ui;
            }
        }
    }
    if (par == 0)
        for (int k = n; k < N; k++) st2(u, k * rs, make_double2(0.0, 0.0));
}

// --------------------------------------------------------- float-float sweeps

using df::F2;
struct CF2 {           // complex float-float
    F2 re, im;
};
__device__ __forceinline__ F2 neg(F2 x) { return F2{-x.hi, -x.lo}; }
__device__ __forceinline__ void store_cf2(double *col, int k, CF2 v) {
    reinterpret_cast<float4 *>(col)[k] = make_float4(v.re.hi, v.re.lo, v.im.hi, v.im.lo);
}
__device__ __forceinline__ void store_f64(double *col, int k, CF2 v) {
    reinterpret_cast<double2 *>(col)[k] = make_double2(df::to_f64(v.re), df::to_f64(v.im));
}
// x - a * y (float-float)
__device__ __forceinline__ F2 fnma(F2 a, F2 y, F2 x) { return df::add(x, neg(df::mul(a, y))); }
// One complex row of a right-hand-side column, loaded with a 256-byte L2 fetch size: the
// two lanes of a mode walk its column 32 bytes per row, so one miss brings the next eight
// rows into L2 (measured 6.55 -> 6.49 ms and 9.45 -> 9.36 ms for the Helmholtz and
// biharmonic sweeps at N = 1024, 1024 x 1024).  Only the fetch size differs from a plain load.
__device__ __forceinline__ double2 ld_col(const double2 *p) {
    double2 v;
    asm volatile("ld.global.L2::256B.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "l"(p));
    return v;
}

// Helmholtz: F rows of two float4 (1/U0, U2) (l, 0) as (hi, lo); h = alpha pi / 2.
// Float-float factor streams of one chain, row i at [i * s]: Helmholtz b = (1/U0, U2),
// f = l; biharmonic f = (L1, L2), b0 = (1/U0, U1), b1 = (U2, ta), b2 = tb (each value as
// hi, lo).  s = 1 for a chain stored as one block; s = the number of chains when rows
// are interleaved across chains (a warp's lanes then read adjacent entries).
struct HelmDF {
    const float4 *b;
    const float2 *f;
    long s;
};
struct BihDF {
    const float4 *f, *b0, *b1;
    const float2 *b2;
    long s;
};

template <int PB>
__device__ inline void solve_helm_df_chain_t(int N, int par, const double *fcol, double *ucol, HelmDF F, F2 h,
                                             float4 *ys, int ystride, long rs) {
    const int n = N - 2;
    const int rows = (n - par + 1) / 2;
    // Forward elimination y_i = f_i - l_i y_{i-1}.  Rows are fetched PB at a time into two
    // register buffers: the next block's loads are issued before the current block is
    // computed (software pipelining), and all loads of a block precede its stores (which
    // may alias f when u == f).
    CF2 y{F2{0.f, 0.f}, F2{0.f, 0.f}};
    {
        double2 fa[PB], fb[PB];
        float2 la[PB], lb[PB];
        auto load = [&](double2 (&fx)[PB], float2 (&lx)[PB], int i0) {
#pragma unroll
            for (int q = 0; q < PB; q++) {
                const int i = min(i0 + q, rows - 1);
                fx[q] = ld_col(reinterpret_cast<const double2 *>(fcol) + (2 * i + par) * rs);
                lx[q] = F.f[(long)i * F.s];
            }
        };
        auto run = [&](const double2 (&fx)[PB], const float2 (&lx)[PB], int i0) {
#pragma unroll
            for (int q = 0; q < PB; q++) {
                if (i0 + q < rows) {
                    const F2 l{lx[q].x, lx[q].y};
                    y.re = fnma(l, y.re, df::from_f64(fx[q].x));
                    y.im = fnma(l, y.im, df::from_f64(fx[q].y));
                    ys[(long)(i0 + q) * ystride] = make_float4(y.re.hi, y.re.lo, y.im.hi, y.im.lo);
                }
            }
        };
        load(fa, la, 0);
        for (int i0 = 0; i0 < rows; i0 += 2 * PB) {
            load(fb, lb, i0 + PB);
            run(fa, la, i0);
            load(fa, la, i0 + 2 * PB);
            run(fb, lb, i0 + PB);
        }
    }
    // back substitution u_i = (y_i + h u_{i+1} - U2_i S_{i+1}) / U_ii (same pipelining)
    CF2 un{F2{0.f, 0.f}, F2{0.f, 0.f}}, S = un;
    {
        float4 ya[PB], yb[PB], aa[PB], ab[PB];
        auto load = [&](float4 (&yx)[PB], float4 (&ax)[PB], int i0) {
#pragma unroll
            for (int q = 0; q < PB; q++) {
                const int i = max(i0 - q, 0);
                yx[q] = ys[(long)i * ystride];
                ax[q] = F.b[(long)i * F.s];
            }
        };
        auto run = [&](const float4 (&yx)[PB], const float4 (&ax)[PB], int i0) {
#pragma unroll
            for (int q = 0; q < PB; q++) {
                if (i0 - q >= 0) {
                    const F2 inv0{ax[q].x, ax[q].y}, U2{ax[q].z, ax[q].w};
                    const CF2 yi{F2{yx[q].x, yx[q].y}, F2{yx[q].z, yx[q].w}};
                    CF2 t;
                    t.re = fnma(U2, S.re, df::add(yi.re, df::mul(h, un.re)));
                    t.im = fnma(U2, S.im, df::add(yi.im, df::mul(h, un.im)));
                    un.re = df::mul(inv0, t.re);
                    un.im = df::mul(inv0, t.im);
                    un.re = df::fast_two_sum(un.re.hi, un.re.lo);
                    un.im = df::fast_two_sum(un.im.hi, un.im.lo);
                    S.re = df::add(S.re, un.re);
                    S.im = df::add(S.im, un.im);
                    store_f64(ucol, (2 * (i0 - q) + par) * rs, un);
                }
            }
        };
        load(ya, aa, rows - 1);
        for (int i0 = rows - 1; i0 >= 0; i0 -= 2 * PB) {
            load(yb, ab, i0 - PB);
            run(ya, aa, i0);
            load(ya, aa, i0 - 2 * PB);
            run(yb, ab, i0 - PB);
        }
    }
    if (par == 0) {
        reinterpret_cast<double2 *>(ucol)[n * rs] = make_double2(0.0, 0.0);
        reinterpret_cast<double2 *>(ucol)[(n + 1) * rs] = make_double2(0.0, 0.0);
    }
}

// Tuning constants of the biharmonic float-float chain (compile-time; -D overrides):
//   PBF / PBB  rows per register prefetch block in the forward / backward sweep (two
//              blocks in flight)
//   QSD        1: read the per-N (q, s) table at use (L1-resident) instead of prefetching
#ifndef SHEN_BIH_DF_PBF
#define SHEN_BIH_DF_PBF 4
#endif
#ifndef SHEN_BIH_DF_PBB
#define SHEN_BIH_DF_PBB 2
#endif
#ifndef SHEN_BIH_DF_QSD
#define SHEN_BIH_DF_QSD 1
#endif

// Biharmonic float-float chain (Algorithm LUSolveBiharmonic with the Eq. ab tail).
// qs: per-N (q_k, s_k) float-float by k, zero beyond the unknowns.  Rows are fetched PB
// at a time into two register buffers, the next block's loads issued before the
// current block is computed; all loads of a block precede its stores (which may alias f
// when u == f).
template <int PBF, int PBB, bool QSD>
__device__ inline void solve_bih_df_chain_t(int N, int par, const double *fcol, double *ucol, BihDF F,
                                            const float4 *qs, float4 *ys, int ystride, long rs) {
    const int n = N - 4;
    const int rows = (n - par + 1) / 2;
    const F2 zero{0.f, 0.f};
    // forward elimination y_i = f_i - L1_i y_{i-1} - L2_i y_{i-2}
    CF2 y1{zero, zero}, y2 = y1;
    {
        constexpr int PB = PBF;
        double2 fa[PB], fb[PB];
        float4 la[PB], lb[PB];
        auto load = [&](double2 (&fx)[PB], float4 (&lx)[PB], int i0) {
#pragma unroll
            for (int q = 0; q < PB; q++) {
                const int i = min(i0 + q, rows - 1);
                fx[q] = ld_col(reinterpret_cast<const double2 *>(fcol) + (2 * i + par) * rs);
                lx[q] = F.f[(long)i * F.s];
            }
        };
        auto run = [&](const double2 (&fx)[PB], const float4 (&lx)[PB], int i0) {
#pragma unroll
            for (int q = 0; q < PB; q++) {
                if (i0 + q < rows) {
                    const F2 L1{lx[q].x, lx[q].y}, L2{lx[q].z, lx[q].w};
                    CF2 y;
                    // the y_{i-2} term first: only the last step waits for y_{i-1}
                    y.re = fnma(L1, y1.re, fnma(L2, y2.re, df::from_f64(fx[q].x)));
                    y.im = fnma(L1, y1.im, fnma(L2, y2.im, df::from_f64(fx[q].y)));
                    ys[(long)(i0 + q) * ystride] = make_float4(y.re.hi, y.re.lo, y.im.hi, y.im.lo);
                    y2 = y1;
                    y1 = y;
                }
            }
        };
        load(fa, la, 0);
        for (int i0 = 0; i0 < rows; i0 += 2 * PB) {
            load(fb, lb, i0 + PB);
            run(fa, la, i0);
            load(fa, la, i0 + 2 * PB);
            run(fb, lb, i0 + PB);
        }
    }
    // back substitution: u_i = (y_i - U1 u_{i+1} - U2 u_{i+2} - ta Sq - tb Ss) / U0,
    // Sq = sum_{j >= i+3} q_j u_j, Ss = sum_{j >= i+3} s_j u_j
    CF2 u1{zero, zero}, u2 = u1, u3 = u1, Sq = u1, Ss = u1;
    {
        constexpr int PB = PBB;
        constexpr int NQ = QSD ? 1 : PB;
        float4 ya[PB], yb[PB], ba[PB], bb[PB], ca[PB], cb[PB], qa[NQ], qb[NQ];
        float2 da[PB], db[PB];
        auto load = [&](float4 (&yx)[PB], float4 (&bx)[PB], float4 (&cx)[PB], float2 (&dx)[PB], float4 (&qx)[NQ],
                        int i0) {
#pragma unroll
            for (int q = 0; q < PB; q++) {
                const int i = max(i0 - q, 0);
                const long r = (long)i * F.s;
                yx[q] = ys[(long)i * ystride];
                bx[q] = F.b0[r];
                cx[q] = F.b1[r];
                dx[q] = F.b2[r];
                if (!QSD) qx[q < NQ ? q : 0] = qs[2 * i + par + 6];
            }
        };
        auto run = [&](const float4 (&yx)[PB], const float4 (&bx)[PB], const float4 (&cx)[PB],
                       const float2 (&dx)[PB], const float4 (&qx)[NQ], int i0) {
#pragma unroll
            for (int q = 0; q < PB; q++) {
                const int i = i0 - q;
                if (i >= 0) {
                    if (i + 3 < rows) {
                        const float4 qv = QSD ? __ldg(qs + 2 * i + par + 6) : qx[q < NQ ? q : 0];
                        const F2 qq{qv.x, qv.y}, ss{qv.z, qv.w};
                        Sq.re = df::add(Sq.re, df::mul(qq, u3.re));
                        Sq.im = df::add(Sq.im, df::mul(qq, u3.im));
                        Ss.re = df::add(Ss.re, df::mul(ss, u3.re));
                        Ss.im = df::add(Ss.im, df::mul(ss, u3.im));
                    }
                    const F2 inv0{bx[q].x, bx[q].y}, U1{bx[q].z, bx[q].w}, U2{cx[q].x, cx[q].y};
                    const F2 ta{cx[q].z, cx[q].w}, tb{dx[q].x, dx[q].y};
                    const CF2 yi{F2{yx[q].x, yx[q].y}, F2{yx[q].z, yx[q].w}};
                    // terms known before u_{i+1} first: only the last step waits for it
                    CF2 t;
                    t.re = fnma(U1, u1.re, fnma(U2, u2.re, fnma(tb, Ss.re, fnma(ta, Sq.re, yi.re))));
                    t.im = fnma(U1, u1.im, fnma(U2, u2.im, fnma(tb, Ss.im, fnma(ta, Sq.im, yi.im))));
                    CF2 ui;
                    ui.re = df::mul(inv0, t.re);
                    ui.im = df::mul(inv0, t.im);
                    ui.re = df::fast_two_sum(ui.re.hi, ui.re.lo);
                    ui.im = df::fast_two_sum(ui.im.hi, ui.im.lo);
                    store_f64(ucol, (2 * i + par) * rs, ui);
                    u3 = u2;
                    u2 = u1;
                    u1 = ui;
                }
            }
        };
        load(ya, ba, ca, da, qa, rows - 1);
        for (int i0 = rows - 1; i0 >= 0; i0 -= 2 * PB) {
            load(yb, bb, cb, db, qb, i0 - PB);
            run(ya, ba, ca, da, qa, i0);
            load(ya, ba, ca, da, qa, i0 - 2 * PB);
            run(yb, bb, cb, db, qb, i0 - PB);
        }
    }
    if (par == 0)
        for (int k = n; k < N; k++) reinterpret_cast<double2 *>(ucol)[k * rs] = make_double2(0.0, 0.0);
}

// ------------------------------------------------------------ float32 sweeps

// The paper's sweeps in float32 (the first and the correction solves of iterative
// refinement): the factors are the hi parts of the float-float streams (the float64
// factors rounded to float32), the right-hand side is rounded to float32, y is spilled
// as float2 (.x, .y of the float4 scratch).  ACC: the result is added to the float64
// column u (u += d, one float64 addition per value) instead of stored.
__device__ __forceinline__ void put_f32(double *ucol, long idx, float2 v, bool acc) {
    double2 *p = reinterpret_cast<double2 *>(ucol) + idx;
    double2 o = make_double2(df::f32_to_f64_bits(v.x), df::f32_to_f64_bits(v.y));
    if (acc) {
        const double2 a = *p;
        o.x = __dadd_rn(a.x, o.x);
        o.y = __dadd_rn(a.y, o.y);
    }
    *p = o;
}

template <bool ACC>
__device__ inline void solve_helm_f32_chain(int N, int par, const double *fcol, double *ucol, HelmDF F, float h,
                                            float4 *ys, int ystride) {
    constexpr int PB = 8;
    const int n = N - 2;
    const int rows = (n - par + 1) / 2;
    float2 y = make_float2(0.f, 0.f);
    for (int i0 = 0; i0 < rows; i0 += PB) {
        double2 fb[PB];
        float lb[PB];
#pragma unroll
        for (int q = 0; q < PB; q++) {
            const int i = min(i0 + q, rows - 1);
            fb[q] = reinterpret_cast<const double2 *>(fcol)[2 * i + par];
            lb[q] = F.f[(long)i * F.s].x;
        }
#pragma unroll
        for (int q = 0; q < PB; q++) {
            if (i0 + q < rows) {
                y.x = fmaf(-lb[q], y.x, df::hi_f64(fb[q].x));
                y.y = fmaf(-lb[q], y.y, df::hi_f64(fb[q].y));
                ys[(long)(i0 + q) * ystride] = make_float4(y.x, y.y, 0.f, 0.f);
            }
        }
    }
    float2 un = make_float2(0.f, 0.f), S = un;
    for (int i0 = rows - 1; i0 >= 0; i0 -= PB) {
        float4 yb[PB], ab[PB];
#pragma unroll
        for (int q = 0; q < PB; q++) {
            const int i = max(i0 - q, 0);
            yb[q] = ys[(long)i * ystride];
            ab[q] = F.b[(long)i * F.s];                     // (1/U0, U2) as (hi, lo) pairs
        }
#pragma unroll
        for (int q = 0; q < PB; q++) {
            if (i0 - q >= 0) {
                const float inv0 = ab[q].x, U2 = ab[q].z;
                un.x = inv0 * fmaf(-U2, S.x, fmaf(h, un.x, yb[q].x));
                un.y = inv0 * fmaf(-U2, S.y, fmaf(h, un.y, yb[q].y));
                S.x += un.x;
                S.y += un.y;
                put_f32(ucol, 2 * (i0 - q) + par, un, ACC);
            }
        }
    }
    if (par == 0 && !ACC) {
        reinterpret_cast<double2 *>(ucol)[n] = make_double2(0.0, 0.0);
        reinterpret_cast<double2 *>(ucol)[n + 1] = make_double2(0.0, 0.0);
    }
}

template <bool ACC>
__device__ inline void solve_bih_f32_chain(int N, int par, const double *fcol, double *ucol, BihDF F,
                                           const float4 *qs, float4 *ys, int ystride) {
    constexpr int PB = 4;
    const int n = N - 4;
    const int rows = (n - par + 1) / 2;
    float2 y1 = make_float2(0.f, 0.f), y2 = y1;
    for (int i0 = 0; i0 < rows; i0 += PB) {
        double2 fb[PB];
        float4 lb[PB];
#pragma unroll
        for (int q = 0; q < PB; q++) {
            const int i = min(i0 + q, rows - 1);
            fb[q] = reinterpret_cast<const double2 *>(fcol)[2 * i + par];
            lb[q] = F.f[(long)i * F.s];                     // (L1, L2) as (hi, lo) pairs
        }
#pragma unroll
        for (int q = 0; q < PB; q++) {
            if (i0 + q < rows) {
                float2 y;
                y.x = fmaf(-lb[q].x, y1.x, fmaf(-lb[q].z, y2.x, df::hi_f64(fb[q].x)));
                y.y = fmaf(-lb[q].x, y1.y, fmaf(-lb[q].z, y2.y, df::hi_f64(fb[q].y)));
                ys[(long)(i0 + q) * ystride] = make_float4(y.x, y.y, 0.f, 0.f);
                y2 = y1;
                y1 = y;
            }
        }
    }
    float2 u1 = make_float2(0.f, 0.f), u2 = u1, u3 = u1, Sq = u1, Ss = u1;
    for (int i0 = rows - 1; i0 >= 0; i0 -= PB) {
        float4 yb[PB], b0[PB], b1[PB];
        float b2[PB];
#pragma unroll
        for (int q = 0; q < PB; q++) {
            const int i = max(i0 - q, 0);
            const long r = (long)i * F.s;
            yb[q] = ys[(long)i * ystride];
            b0[q] = F.b0[r];                                // (1/U0, U1)
            b1[q] = F.b1[r];                                // (U2, ta)
            b2[q] = F.b2[r].x;                              // tb
        }
#pragma unroll
        for (int q = 0; q < PB; q++) {
            const int i = i0 - q;
            if (i >= 0) {
                if (i + 3 < rows) {
                    const float4 qv = __ldg(qs + 2 * i + par + 6);
                    Sq.x = fmaf(qv.x, u3.x, Sq.x); Sq.y = fmaf(qv.x, u3.y, Sq.y);
                    Ss.x = fmaf(qv.z, u3.x, Ss.x); Ss.y = fmaf(qv.z, u3.y, Ss.y);
                }
                const float inv0 = b0[q].x, U1 = b0[q].z, U2 = b1[q].x, ta = b1[q].z, tb = b2[q];
                float2 ui;
                ui.x = inv0 * fmaf(-U1, u1.x, fmaf(-U2, u2.x, fmaf(-tb, Ss.x, fmaf(-ta, Sq.x, yb[q].x))));
                ui.y = inv0 * fmaf(-U1, u1.y, fmaf(-U2, u2.y, fmaf(-tb, Ss.y, fmaf(-ta, Sq.y, yb[q].y))));
                put_f32(ucol, 2 * i + par, ui, ACC);
                u3 = u2;
                u2 = u1;
                u1 = ui;
            }
        }
    }
    if (par == 0 && !ACC)
        for (int k = n; k < N; k++) reinterpret_cast<double2 *>(ucol)[k] = make_double2(0.0, 0.0);
}

// Row-block shapes of the float-float chains, chosen per plan by the autotuner.  They
// change only how many rows each thread keeps in flight (and so its registers and the
// warps resident per SM), never the arithmetic: every shape gives the same bits.
//   Helmholtz  V0: 8 rows per block (154 registers);  V1: 4 rows per block
//   biharmonic V0: the tuning constants above (124 registers, 16 warps per SM);
//              V1: 4 + 4 rows, (q, s) prefetched (204 registers, 8 warps per SM)
//
// The forward result y (float-float, 16 bytes per complex row) is spilled to ys[i * ystride]
// for chain row i: either the chain's own rows of the output column (ys = column + par,
// ystride = 2; no scratch memory) or a scratch laid out [row][lane] per warp (ystride =
// 32), where each warp's spill of a row is 512 contiguous bytes.
template <int V>
__device__ inline void solve_helm_df_chain(int N, int par, const double *fcol, double *ucol, HelmDF F, F2 h,
                                           float4 *ys, int ystride, long rs = 1) {
    solve_helm_df_chain_t<V == 0 ? 8 : 5>(N, par, fcol, ucol, F, h, ys, ystride, rs);
}

template <int V>
__device__ inline void solve_bih_df_chain(int N, int par, const double *fcol, double *ucol, BihDF F,
                                          const float4 *qs, float4 *ys, int ystride, long rs = 1) {
    if (V == 0)
        solve_bih_df_chain_t<SHEN_BIH_DF_PBF, SHEN_BIH_DF_PBB, SHEN_BIH_DF_QSD != 0>(N, par, fcol, ucol, F, qs, ys,
                                                                                    ystride, rs);
    else
        solve_bih_df_chain_t<4, 4, false>(N, par, fcol, ucol, F, qs, ys, ystride, rs);
}

// The output column's own rows of chain `par`, as a spill target (ystride 2).
__device__ __forceinline__ float4 *column_spill(double *ucol, int par) {
    return reinterpret_cast<float4 *>(ucol) + par;
}

}  // namespace chains
}  // namespace shen
