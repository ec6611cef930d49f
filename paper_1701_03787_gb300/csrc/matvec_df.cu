// Right-hand-side operators of the Crank-Nicolson step (Eqs. gfin, ufin) in float-float
// arithmetic:
//   Helmholtz   (R_h x)_k = g (B_{k,k-2} x_{k-2} + B_kk x_k + B_{k,k+2} x_{k+2}) + A_kk x_k
//                           + A_tail(k) sum_{j = k+2, k+4, ...} x_j,            g = c - z2
//   biharmonic  (R_b x)_k = Q_kk x_k + p_k sum_{j >= k+2} q_j x_j + r_k sum_{j >= k+2} s_j x_j
//                           + ga (A_{k,k-2} x_{k-2} + A_kk x_k + A_{k,k+2} x_{k+2})
//                           + gb (B_{k-4,k} x_{k-4} + B_{k-2,k} x_{k-2} + B_kk x_k
//                                 + B_{k,k+2} x_{k+2} + B_{k,k+4} x_{k+4}),
//                           ga = c - 2 z2, gb = z2 (z2 - c)
// (sums over the same parity; entries beyond the unknowns are zero), then out = R x + beta y.
//
// MODE 2 evaluates the mass matrix alone (B_D or B_B): out = B x + beta y; MODE 3 the
// negated operator, out = -R x + beta y (the biharmonic Crank-Nicolson step in the
// scaled form of the solve, see shen_linear_step).
// The same kernels also evaluate the system operators of the solves (MODE 1):
//   H_h = (z2 + c) B - A      and      H_b = Q - (2 z2 + c) A + z2 (z2 + c) B,
// i.e. the RHS structure with other scalars, for the a posteriori residual
// ||f - H u|| / ||f|| of each mode (no vector written, only the per-mode norms).
//
// One thread per (mode, parity) chain walks its rows from the top down, carrying the
// running sums of the upper-triangular parts (the suffix sums of Sec. 4) and a window
// of five neighbouring x values in registers; x is read once, y once, out written once.
// Each row's terms are accumulated as one float-float sum (error-free products and
// TwoSum, renormalised once per row); the final + beta y is one float64 fused
// multiply-add.  The per-N row coefficients come from float-float tables built at plan
// creation (csrc/plan.cu: build_row_tables in float64, split into hi + lo here).
#include <algorithm>

#include "chains.cuh"

namespace shen {
namespace {

using chains::CF2;
using df::F2;

// sum = hi + lo, not renormalised between terms
struct Acc {
    float hi, lo;
};

__device__ __forceinline__ Acc acc_of(F2 x) { return Acc{x.hi, x.lo}; }

// acc += a * b (float-float times float-float)
__device__ __forceinline__ void acc_mad(Acc &acc, F2 a, F2 b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    const F2 s = df::two_sum(acc.hi, p);
    acc.hi = s.hi;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(s.lo, e));
}

__device__ __forceinline__ F2 acc_done(Acc acc) { return df::fast_two_sum(acc.hi, acc.lo); }

__device__ __forceinline__ F2 ff(float4 v, int half) { return half ? F2{v.z, v.w} : F2{v.x, v.y}; }

__device__ __forceinline__ CF2 ld_cf2(const double *col, long k) {
    const double2 v = reinterpret_cast<const double2 *>(col)[k];
    return CF2{df::from_f64(v.x), df::from_f64(v.y)};
}

__device__ __forceinline__ void st_out(double *out, const double *y, double beta, long k, CF2 r) {
    double2 v = make_double2(df::to_f64(r.re), df::to_f64(r.im));
    if (y) {
        const double2 yi = reinterpret_cast<const double2 *>(y)[k];
        v.x = fma(beta, yi.x, v.x);
        v.y = fma(beta, yi.y, v.y);
    }
    reinterpret_cast<double2 *>(out)[k] = v;
}

struct Chain {
    long col;        // offset of element 0 of the mode's column (doubles)
    long rs;         // complex elements between consecutive Chebyshev indices: 1 for
                     // mode-major fields, n_modes for wall-index-first ones
    long mode;
    int par;
    double z2;
};

__device__ __forceinline__ bool chain_of(const Plan &p, long tid, Chain &c) {
    if (tid >= 2 * p.n_modes) return false;
    const long mode = tid >> 1;
    c.par = (int)(tid & 1);
    c.col = p.wall_first ? 2 * mode : 2 * mode * p.N;
    c.rs = p.wall_first ? p.n_modes : 1;
    c.mode = mode;
    c.z2 = p.d_class_z2[p.d_mode_class[mode]];
    return true;
}

// Residual accumulation of one chain: sum |f_k - (H u)_k|^2 and sum |f_k|^2 over its rows
// (float64); the two chains of a mode (adjacent lanes) are combined at the end.
struct Res {
    double rr = 0.0, ff = 0.0;
    __device__ __forceinline__ void add(const double *f, long k, CF2 hu) {
        const double2 fk = reinterpret_cast<const double2 *>(f)[k];
        const double dr = fk.x - df::to_f64(hu.re), di = fk.y - df::to_f64(hu.im);
        rr = fma(dr, dr, fma(di, di, rr));
        ff = fma(fk.x, fk.x, fma(fk.y, fk.y, ff));
    }
    // lane pair (2j, 2j + 1) = both chains of one mode; both are always active together
    __device__ __forceinline__ void finish(const Plan &p, const Chain &c, double *rel) {
        const unsigned pair = 3u << ((threadIdx.x & 31) & ~1u);
        const double r2 = rr + __shfl_xor_sync(pair, rr, 1);
        const double f2 = ff + __shfl_xor_sync(pair, ff, 1);
        if (c.par == 0) {
            const double q = f2 > 0.0 ? sqrt(r2 / f2) : (r2 > 0.0 ? INFINITY : 0.0);
            if (rel) rel[c.mode] = q;
            // non-negative doubles order like their bit patterns
            atomicMax(p.d_resmax, (unsigned long long)__double_as_longlong(q));
        }
    }
};

// Helmholtz table row k: T[2k] = (B_kk, A_kk), T[2k + 1] = (A_tail(k), 0), each (hi, lo).
template <int MODE>
__global__ void __launch_bounds__(128) matvec_helmholtz_df_kernel(Plan p, const float4 *T, const double *x,
                                                                  const double *y, double beta, double *out,
                                                                  double *rel) {
    Chain c;
    if (!chain_of(p, blockIdx.x * (long)blockDim.x + threadIdx.x, c)) return;
    const int N = p.N, n = N - 2, par = c.par;
    const int rows = (n - par + 1) / 2;
    const long rs = c.rs;
    const double *xc_ = x + c.col;
    const double *yc_ = y ? y + c.col : nullptr;
    constexpr int OP = MODE == 3 ? 0 : MODE;                    // operator: R_h, H_h or B
    double *oc = MODE != 1 ? out + c.col : nullptr;
    const double gd = OP == 0 ? p.c - c.z2 : (OP == 1 ? p.c + c.z2 : 1.0);   // coefficient of B
    const F2 g = df::from_f64(gd);
    const F2 gm = df::from_f64(-gd * (kPi / 2));                 // g B_{k,k+-2}
    Res res;
    const F2 zero{0.f, 0.f};
    CF2 S{zero, zero};                                           // sum_{j >= i+1} x_j (chain rows)
    CF2 xn{zero, zero};                                          // x_{i+1}
    CF2 xc = rows > 0 ? ld_cf2(xc_, (2 * (rows - 1) + par) * rs) : xn;  // x_i
    for (int i = rows - 1; i >= 0; i--) {
        const int k = 2 * i + par;
        S.re = df::add(S.re, xn.re);
        S.im = df::add(S.im, xn.im);
        const CF2 xp = i > 0 ? ld_cf2(xc_, (k - 2) * rs) : CF2{zero, zero};
        const float4 t0 = T[2 * k], t1 = T[2 * k + 1];
        // coefficient of x_k: g B_kk +- A_kk (+ for R_h, - for H_h, none for B)
        const F2 zero2{0.f, 0.f};
        Acc a0 = acc_of(OP == 0 ? ff(t0, 1) : (OP == 1 ? chains::neg(ff(t0, 1)) : zero2));
        acc_mad(a0, g, ff(t0, 0));
        const F2 c0 = acc_done(a0);
        const F2 at = OP == 0 ? ff(t1, 0) : (OP == 1 ? chains::neg(ff(t1, 0)) : zero2);
        CF2 r;
        Acc ar{0.f, 0.f}, ai{0.f, 0.f};
        acc_mad(ar, at, S.re);
        acc_mad(ai, at, S.im);
        acc_mad(ar, gm, xp.re);
        acc_mad(ai, gm, xp.im);
        acc_mad(ar, gm, xn.re);
        acc_mad(ai, gm, xn.im);
        acc_mad(ar, c0, xc.re);
        acc_mad(ai, c0, xc.im);
        r.re = acc_done(ar);
        r.im = acc_done(ai);
        if (MODE == 3) r = CF2{chains::neg(r.re), chains::neg(r.im)};
        if (MODE != 1) st_out(oc, yc_, beta, k * rs, r);
        else res.add(yc_, k * rs, r);
        xn = xc;
        xc = xp;
    }
    if (MODE == 1) {
        res.finish(p, c, rel);
    } else if (par == 0) {
        reinterpret_cast<double2 *>(oc)[n * rs] = make_double2(0.0, 0.0);
        reinterpret_cast<double2 *>(oc)[(n + 1) * rs] = make_double2(0.0, 0.0);
    }
}

// Biharmonic table row k (6 float4): (Q_kk, p_k) (r_k, A_kk) (A_{k,k+2}, A_{k,k-2})
// (B_kk, B_{k,k+2}) (B_{k,k+4}, q_{k+2}) (s_{k+2}, 0).
// The right-hand-side operators (MODE 0, 3) are held to 64 registers so that 8 blocks (32
// warps) fit on an SM: measured 9.28 against 9.50 ms at N = 1024, 1024 x 1024.
template <int MODE>
__global__ void __launch_bounds__(128, (MODE == 0 || MODE == 3) ? 8 : 0) matvec_biharmonic_df_kernel(
    Plan p, const float4 *T, const double *x, const double *y, double beta, double *out, double *rel) {
    Chain c;
    if (!chain_of(p, blockIdx.x * (long)blockDim.x + threadIdx.x, c)) return;
    const int N = p.N, n = N - 4, par = c.par;
    const int rows = (n - par + 1) / 2;
    const long rs = c.rs;
    const double *xc_ = x + c.col;
    const double *yc_ = y ? y + c.col : nullptr;
    constexpr int OP = MODE == 3 ? 0 : MODE;                    // operator: R_b, H_b or B
    double *oc = MODE != 1 ? out + c.col : nullptr;
    // coefficients of A and B: R_b (c - 2 z2, z2 (z2 - c)), H_b (-(2 z2 + c), z2 (z2 + c)),
    // or the mass matrix alone (0, 1, and no Q)
    const F2 ga = df::from_f64(OP == 0 ? p.c - 2.0 * c.z2 : (OP == 1 ? -(2.0 * c.z2 + p.c) : 0.0));
    const F2 gb = df::from_f64(OP == 0 ? c.z2 * (c.z2 - p.c) : (OP == 1 ? c.z2 * (c.z2 + p.c) : 1.0));
    Res res;
    const F2 zero{0.f, 0.f};
    const CF2 z{zero, zero};
    auto X = [&](int i) { return (i >= 0 && i < rows) ? ld_cf2(xc_, (2 * i + par) * rs) : z; };
    CF2 Sq = z, Ss = z;                                          // sums over chain rows >= i+1
    CF2 xm2 = X(rows - 3), xm1 = X(rows - 2), xc = X(rows - 1), xp1 = z, xp2 = z;
    for (int i = rows - 1; i >= 0; i--) {
        const int k = 2 * i + par;
        const float4 t0 = T[6 * k], t1 = T[6 * k + 1], t2 = T[6 * k + 2], t3 = T[6 * k + 3], t4 = T[6 * k + 4],
                     t5 = T[6 * k + 5];
        if (i + 1 < rows) {                                      // add q_{k+2} x_{k+2}, s_{k+2} x_{k+2}
            const F2 q = ff(t4, 1), s = ff(t5, 0);
            Acc a = acc_of(Sq.re);
            acc_mad(a, q, xp1.re);
            Sq.re = acc_done(a);
            a = acc_of(Sq.im);
            acc_mad(a, q, xp1.im);
            Sq.im = acc_done(a);
            a = acc_of(Ss.re);
            acc_mad(a, s, xp1.re);
            Ss.re = acc_done(a);
            a = acc_of(Ss.im);
            acc_mad(a, s, xp1.im);
            Ss.im = acc_done(a);
        }
        // row coefficients of x_{k-4} .. x_{k+4}
        const F2 bm4 = i >= 2 ? ff(T[6 * (k - 4) + 4], 0) : zero;      // B_{k-4,k}
        const F2 bm2 = i >= 1 ? ff(T[6 * (k - 2) + 3], 1) : zero;      // B_{k-2,k}
        const F2 am = i >= 1 ? ff(t2, 1) : zero;
        Acc a = acc_of(OP == 2 ? zero : ff(t0, 0));                      // Q_kk + ga A_kk + gb B_kk
        acc_mad(a, ga, ff(t1, 1));
        acc_mad(a, gb, ff(t3, 0));
        const F2 c0 = acc_done(a);
        a = Acc{0.f, 0.f};
        acc_mad(a, ga, am);
        acc_mad(a, gb, bm2);
        const F2 cm2 = acc_done(a);
        a = Acc{0.f, 0.f};
        acc_mad(a, ga, ff(t2, 0));
        acc_mad(a, gb, ff(t3, 1));
        const F2 cp2 = acc_done(a);
        a = Acc{0.f, 0.f};
        acc_mad(a, gb, bm4);
        const F2 cm4 = acc_done(a);
        a = Acc{0.f, 0.f};
        acc_mad(a, gb, ff(t4, 0));
        const F2 cp4 = acc_done(a);
        const F2 pk = OP == 2 ? zero : ff(t0, 1), rk = OP == 2 ? zero : ff(t1, 0);
        CF2 r;
        Acc ar{0.f, 0.f}, ai{0.f, 0.f};
        acc_mad(ar, pk, Sq.re);
        acc_mad(ai, pk, Sq.im);
        acc_mad(ar, rk, Ss.re);
        acc_mad(ai, rk, Ss.im);
        acc_mad(ar, cm4, xm2.re);
        acc_mad(ai, cm4, xm2.im);
        acc_mad(ar, cp4, xp2.re);
        acc_mad(ai, cp4, xp2.im);
        acc_mad(ar, cm2, xm1.re);
        acc_mad(ai, cm2, xm1.im);
        acc_mad(ar, cp2, xp1.re);
        acc_mad(ai, cp2, xp1.im);
        acc_mad(ar, c0, xc.re);
        acc_mad(ai, c0, xc.im);
        r.re = acc_done(ar);
        r.im = acc_done(ai);
        if (MODE == 3) r = CF2{chains::neg(r.re), chains::neg(r.im)};
        if (MODE != 1) st_out(oc, yc_, beta, k * rs, r);
        else res.add(yc_, k * rs, r);
        xp2 = xp1;
        xp1 = xc;
        xc = xm1;
        xm1 = xm2;
        xm2 = X(i - 3);
    }
    if (MODE == 1) {
        res.finish(p, c, rel);
    } else if (par == 0) {
        for (int k = n; k < N; k++) reinterpret_cast<double2 *>(oc)[k * rs] = make_double2(0.0, 0.0);
    }
}

__device__ __forceinline__ float4 pair4(double a, double b) {
    const float ah = (float)a, bh = (float)b;
    return make_float4(ah, (float)(a - (double)ah), bh, (float)(b - (double)bh));
}

// Float-float matvec tables from the float64 row tables: Helmholtz 2 N float4, then
// biharmonic 6 N float4 (entries beyond the unknowns are zero in the float64 tables or
// never read).
__global__ void pack_matvec_df_kernel(Plan p, float4 *T) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int N = p.N;
    if (k >= N) return;
    const RowTables &t = p.tab;
    T[2 * k] = pair4(t.bd0[k], t.ad0[k]);
    T[2 * k + 1] = pair4(t.adt[k], 0.0);
    float4 *B = T + 2 * N;
    const double q2 = k + 2 < N ? t.qk[k + 2] : 0.0, s2 = k + 2 < N ? t.sk[k + 2] : 0.0;
    B[6 * k] = pair4(t.qb0[k], t.pk[k]);
    B[6 * k + 1] = pair4(t.rk[k], t.ab0[k]);
    B[6 * k + 2] = pair4(t.abp[k], t.abm[k]);
    B[6 * k + 3] = pair4(t.bb0[k], t.bb2[k]);
    B[6 * k + 4] = pair4(t.bb4[k], q2);
    B[6 * k + 5] = pair4(s2, 0.0);
}

inline unsigned nblk(long threads, int bs) { return (unsigned)((threads + bs - 1) / bs); }

}  // namespace

size_t matvec_df_floats(const Plan &p) { return (size_t)8 * p.N * 4; }

cudaError_t pack_matvec_df(const Plan &p, float *T, cudaStream_t s) {
    pack_matvec_df_kernel<<<nblk(p.N, 128), 128, 0, s>>>(p, reinterpret_cast<float4 *>(T));
    return cudaGetLastError();
}

cudaError_t launch_matvec_df(const Plan &p, int problem, const double *x, const double *y, double beta,
                             double *out, cudaStream_t s) {
    if (p.n_modes <= 0) return cudaSuccess;
    const float4 *T = reinterpret_cast<const float4 *>(p.d_mv_df);
    if (problem == SHEN_HELMHOLTZ)
        matvec_helmholtz_df_kernel<0><<<nblk(2 * p.n_modes, 128), 128, 0, s>>>(p, T, x, y, beta, out, nullptr);
    else
        matvec_biharmonic_df_kernel<0><<<nblk(2 * p.n_modes, 128), 128, 0, s>>>(p, T + 2 * p.N, x, y, beta, out,
                                                                                nullptr);
    return cudaGetLastError();
}

cudaError_t launch_matvec_neg_df(const Plan &p, int problem, const double *x, const double *y, double beta,
                                 double *out, cudaStream_t s) {
    if (p.n_modes <= 0) return cudaSuccess;
    const float4 *T = reinterpret_cast<const float4 *>(p.d_mv_df);
    if (problem == SHEN_HELMHOLTZ)
        matvec_helmholtz_df_kernel<3><<<nblk(2 * p.n_modes, 128), 128, 0, s>>>(p, T, x, y, beta, out, nullptr);
    else
        matvec_biharmonic_df_kernel<3><<<nblk(2 * p.n_modes, 128), 128, 0, s>>>(p, T + 2 * p.N, x, y, beta, out,
                                                                                nullptr);
    return cudaGetLastError();
}

cudaError_t launch_mass_df(const Plan &p, int problem, const double *x, const double *y, double beta, double *out,
                           cudaStream_t s) {
    if (p.n_modes <= 0) return cudaSuccess;
    const float4 *T = reinterpret_cast<const float4 *>(p.d_mv_df);
    if (problem == SHEN_HELMHOLTZ)
        matvec_helmholtz_df_kernel<2><<<nblk(2 * p.n_modes, 128), 128, 0, s>>>(p, T, x, y, beta, out, nullptr);
    else
        matvec_biharmonic_df_kernel<2><<<nblk(2 * p.n_modes, 128), 128, 0, s>>>(p, T + 2 * p.N, x, y, beta, out,
                                                                                nullptr);
    return cudaGetLastError();
}

cudaError_t launch_residual_df(const Plan &p, int problem, const double *f, const double *u, double *rel,
                               cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(p.d_resmax, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess || p.n_modes <= 0) return e;
    const float4 *T = reinterpret_cast<const float4 *>(p.d_mv_df);
    if (problem == SHEN_HELMHOLTZ)
        matvec_helmholtz_df_kernel<1><<<nblk(2 * p.n_modes, 128), 128, 0, s>>>(p, T, u, f, 0.0, nullptr, rel);
    else
        matvec_biharmonic_df_kernel<1><<<nblk(2 * p.n_modes, 128), 128, 0, s>>>(p, T + 2 * p.N, u, f, 0.0,
                                                                                nullptr, rel);
    return cudaGetLastError();
}

}  // namespace shen
