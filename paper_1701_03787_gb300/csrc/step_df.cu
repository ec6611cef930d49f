// The Crank-Nicolson step of the wall-normal velocity and vorticity (Eqs. ufin, gfin) with
// the right-hand-side operator fused into the solve's forward sweep.
//
// In the scaled forms of this library the right-hand-side matrices are the system matrices
// plus banded parts (Eqs. ufin, gfin; Biharmonic_matrix, Helmholtz_matrix):
//   Helmholtz   R_h = (c - z2) B + A        = 2 c B - H_h
//   biharmonic  R_b = Q + (c - 2 z2) A + z2 (z2 - c) B = H_b + 2 c (A - z2 B)
// so that the steps  H_h g_new = R_h g_old + s load_g  and  H_b u_new = -R_b u_old - s load_u
// (s = 2 / nu) read
//   g_new = -g_old + H_h^-1 (2 c B g_old + s load_g)
//   u_new = -u_old + H_b^-1 (-2 c (A - z2 B) u_old - s load_u).
// The banded operators need no suffix sums (Q, the only full upper triangle, cancels), so
// their rows are formed top down inside the forward elimination: one pass reads u_old and
// the load and writes y, the back substitution writes u_new = d - u_old (re-reading u_old).
// That replaces an operator pass (read x and the load, write the right-hand side) and the
// solve's read of it.  |d| ~ 2 |u_old| for small time steps, so the difference loses no
// digits.
//
// Work decomposition, spill scratch, class order and float-float arithmetic as in the
// thread-per-chain solves (kernels_df.cu): one thread per (mode, parity) chain.
#include <algorithm>

#include "chains.cuh"
#include "sweep2.cuh"

namespace shen {
namespace {

using chains::CF2;
using df::F2;
using sw2::Acc;

__device__ __forceinline__ CF2 ldc(const double *col, long k) {
    const double2 v = reinterpret_cast<const double2 *>(col)[k];
    return CF2{df::from_f64(v.x), df::from_f64(v.y)};
}
__device__ __forceinline__ F2 ff(float4 v, int h) { return h ? F2{v.z, v.w} : F2{v.x, v.y}; }

// acc += a * x for the real and imaginary parts
__device__ __forceinline__ void cmad(Acc &re, Acc &im, F2 a, const CF2 &x) {
    sw2::acc_add_mul(re, a, x.re);
    sw2::acc_add_mul(im, a, x.im);
}

constexpr int kPB = 4;   // rows per prefetch block

// Helmholtz chain: w_i = 2 c (B g_old)_k + s load_k, y = L^-1 w, d = U^-1 y, g_new = d - g_old.
// Th: the Helmholtz operator table (row k: (B_kk, A_kk), (A_tail, 0)); B_{k,k+-2} = -pi/2.
__device__ void step_helm_chain(const Plan &p, int par, double z2, const double *xcol, const double *lcol,
                                double *ucol, chains::HelmDF F, const float4 *Th, float4 *ys) {
    const int N = p.N, n = N - 2;
    const int rows = (n - par + 1) / 2;
    const F2 zero{0.f, 0.f};
    const CF2 z{zero, zero};
    const F2 twoc = df::from_f64(2.0 * p.c), s = df::from_f64(2.0 / p.nu);
    const F2 boff = df::from_f64(-kPi / 2);
    const F2 h = df::from_f64((z2 + p.c) * (kPi / 2));
    auto X = [&](int i) { return (i >= 0 && i < rows) ? ldc(xcol, 2 * i + par) : z; };
    // forward: window x_{i-1}, x_i, x_{i+1}
    CF2 xm = z, x0 = X(0), xp = X(1);
    CF2 y = z;
    for (int i0 = 0; i0 < rows; i0 += kPB) {
        CF2 xn[kPB], ld[kPB];
        float2 lf[kPB];
        float4 tb[kPB];
#pragma unroll
        for (int q = 0; q < kPB; q++) {
            const int i = i0 + q;
            const bool ok = i < rows;
            xn[q] = ok ? X(i + 2) : z;
            ld[q] = (ok && lcol) ? ldc(lcol, 2 * i + par) : z;
            lf[q] = ok ? F.f[(long)i * F.s] : make_float2(0.f, 0.f);
            tb[q] = __ldg(Th + 2 * min(2 * i + par, n - 1));
        }
#pragma unroll
        for (int q = 0; q < kPB; q++) {
            const int i = i0 + q;
            if (i >= rows) break;
            // (B x)_k = B_kk x_k - pi/2 (x_{k-2} + x_{k+2})
            Acc br{0.f, 0.f}, bi{0.f, 0.f};
            cmad(br, bi, ff(tb[q], 0), x0);
            cmad(br, bi, boff, xm);
            cmad(br, bi, boff, xp);
            const CF2 Bx{sw2::acc_done(br), sw2::acc_done(bi)};
            Acc wr{0.f, 0.f}, wi{0.f, 0.f};
            cmad(wr, wi, twoc, Bx);
            cmad(wr, wi, s, ld[q]);
            // y_i = w_i - l_i y_{i-1}
            const F2 l{lf[q].x, lf[q].y};
            sw2::acc_sub_mul(wr, l, y.re);
            sw2::acc_sub_mul(wi, l, y.im);
            y = CF2{sw2::acc_done(wr), sw2::acc_done(wi)};
            ys[(long)i * 32] = make_float4(y.re.hi, y.re.lo, y.im.hi, y.im.lo);
            xm = x0;
            x0 = xp;
            xp = xn[q];
        }
    }
    // back: d_i = (y_i + h d_{i+1} - U2_i S) / U0_i, S = sum_{j > i} d_j; g_new_i = d_i - g_old_i
    CF2 dn = z, S = z;
    for (int i0 = rows - 1; i0 >= 0; i0 -= kPB) {
        float4 yb[kPB], bb[kPB];
        CF2 xo[kPB];
#pragma unroll
        for (int q = 0; q < kPB; q++) {
            const int i = max(i0 - q, 0);
            yb[q] = ys[(long)i * 32];
            bb[q] = F.b[(long)i * F.s];
            xo[q] = ldc(xcol, 2 * i + par);
        }
#pragma unroll
        for (int q = 0; q < kPB; q++) {
            const int i = i0 - q;
            if (i < 0) break;
            const F2 inv0{bb[q].x, bb[q].y}, U2{bb[q].z, bb[q].w};
            Acc ar = sw2::acc_start(F2{yb[q].x, yb[q].y}), ai = sw2::acc_start(F2{yb[q].z, yb[q].w});
            sw2::acc_sub_mul(ar, U2, S.re);
            sw2::acc_sub_mul(ai, U2, S.im);
            sw2::acc_add_mul(ar, h, dn.re);
            sw2::acc_add_mul(ai, h, dn.im);
            const CF2 d{sw2::mul_n(inv0, sw2::acc_done(ar)), sw2::mul_n(inv0, sw2::acc_done(ai))};
            S = CF2{df::add(S.re, d.re), df::add(S.im, d.im)};
            dn = d;
            const CF2 g{df::add(d.re, chains::neg(xo[q].re)), df::add(d.im, chains::neg(xo[q].im))};
            chains::store_f64(ucol, 2 * i + par, g);
        }
    }
    if (par == 0) {
        reinterpret_cast<double2 *>(ucol)[n] = make_double2(0.0, 0.0);
        reinterpret_cast<double2 *>(ucol)[n + 1] = make_double2(0.0, 0.0);
    }
}

// Biharmonic chain: w_i = -2 c ((A - z2 B) u_old)_k - s load_k, y = L^-1 w, back substitution
// of Algorithm LUSolveBiharmonic for d, u_new = d - u_old.  Tb: the biharmonic operator table
// (row k, 6 float4: (Q_kk, p_k) (r_k, A_kk) (A_{k,k+2}, A_{k,k-2}) (B_kk, B_{k,k+2})
// (B_{k,k+4}, q_{k+2}) (s_{k+2}, 0)); B is symmetric, so B_{k,k-2}, B_{k,k-4} are rows k-2, k-4's
// B_{k-2,k}, B_{k-4,k}.
__device__ void step_bih_chain(const Plan &p, int par, double z2, const double *xcol, const double *lcol,
                               double *ucol, chains::BihDF F, const float4 *Tb, const float4 *qs, float4 *ys) {
    const int N = p.N, n = N - 4;
    const int rows = (n - par + 1) / 2;
    const F2 zero{0.f, 0.f};
    const CF2 z{zero, zero};
    const F2 m2c = df::from_f64(-2.0 * p.c), ms = df::from_f64(-2.0 / p.nu), mz2 = df::from_f64(-z2);
    auto X = [&](int i) { return (i >= 0 && i < rows) ? ldc(xcol, 2 * i + par) : z; };
    CF2 xm2 = z, xm1 = z, x0 = X(0), xp1 = X(1), xp2 = X(2);
    F2 bm2 = zero, bm4a = zero, bm4b = zero;   // B_{k-2,k}; B_{k-4,k} and B_{k-2,k+2} carried
    CF2 y1 = z, y2 = z;
    for (int i0 = 0; i0 < rows; i0 += kPB) {
        CF2 xn[kPB], ld[kPB];
        float4 lf[kPB];
#pragma unroll
        for (int q = 0; q < kPB; q++) {
            const int i = i0 + q;
            const bool ok = i < rows;
            xn[q] = ok ? X(i + 3) : z;
            ld[q] = (ok && lcol) ? ldc(lcol, 2 * i + par) : z;
            lf[q] = ok ? F.f[(long)i * F.s] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int q = 0; q < kPB; q++) {
            const int i = i0 + q;
            if (i >= rows) break;
            // the per-N rows (the same for every mode: L1 / L2 resident)
            const int k = 2 * i + par;
            const float4 t1 = __ldg(Tb + 6 * k + 1), t2 = __ldg(Tb + 6 * k + 2), t3 = __ldg(Tb + 6 * k + 3),
                         t4 = __ldg(Tb + 6 * k + 4);
            // (B x)_k and (A x)_k over the same parity
            Acc br{0.f, 0.f}, bi{0.f, 0.f};
            cmad(br, bi, bm4a, xm2);
            cmad(br, bi, bm2, xm1);
            cmad(br, bi, ff(t3, 0), x0);
            cmad(br, bi, ff(t3, 1), xp1);
            cmad(br, bi, ff(t4, 0), xp2);
            const CF2 Bx{sw2::acc_done(br), sw2::acc_done(bi)};
            Acc ar{0.f, 0.f}, ai{0.f, 0.f};
            cmad(ar, ai, ff(t2, 1), xm1);
            cmad(ar, ai, ff(t1, 1), x0);
            cmad(ar, ai, ff(t2, 0), xp1);
            cmad(ar, ai, mz2, Bx);                                     // (A - z2 B) x
            const CF2 W{sw2::acc_done(ar), sw2::acc_done(ai)};
            Acc wr{0.f, 0.f}, wi{0.f, 0.f};
            cmad(wr, wi, m2c, W);
            cmad(wr, wi, ms, ld[q]);
            // y_i = w_i - L2 y_{i-2} - L1 y_{i-1}
            const F2 L1{lf[q].x, lf[q].y}, L2{lf[q].z, lf[q].w};
            sw2::acc_sub_mul(wr, L2, y2.re);
            sw2::acc_sub_mul(wi, L2, y2.im);
            sw2::acc_sub_mul(wr, L1, y1.re);
            sw2::acc_sub_mul(wi, L1, y1.im);
            const CF2 y{sw2::acc_done(wr), sw2::acc_done(wi)};
            ys[(long)i * 32] = make_float4(y.re.hi, y.re.lo, y.im.hi, y.im.lo);
            y2 = y1;
            y1 = y;
            xm2 = xm1;
            xm1 = x0;
            x0 = xp1;
            xp1 = xp2;
            xp2 = xn[q];
            // the next row's B_{k,k-2} is this row's B_{k,k+2}; its B_{k,k-4} the previous row's B_{k,k+4}
            bm4a = bm4b;
            bm4b = ff(t4, 0);
            bm2 = ff(t3, 1);
        }
    }
    // back substitution for d (Algorithm LUSolveBiharmonic), u_new = d - u_old
    CF2 d1 = z, d2 = z, d3 = z, Sq = z, Ss = z;
    for (int i0 = rows - 1; i0 >= 0; i0 -= kPB) {
        float4 yb[kPB], b0[kPB], b1[kPB];
        float2 b2[kPB];
        CF2 xo[kPB];
#pragma unroll
        for (int q = 0; q < kPB; q++) {
            const int i = max(i0 - q, 0);
            const long r = (long)i * F.s;
            yb[q] = ys[(long)i * 32];
            b0[q] = F.b0[r];
            b1[q] = F.b1[r];
            b2[q] = F.b2[r];
            xo[q] = ldc(xcol, 2 * i + par);
        }
#pragma unroll
        for (int q = 0; q < kPB; q++) {
            const int i = i0 - q;
            if (i < 0) break;
            if (i + 3 < rows) {
                const float4 qv = __ldg(qs + 2 * i + par + 6);
                Sq = CF2{sw2::add_mul(Sq.re, F2{qv.x, qv.y}, d3.re), sw2::add_mul(Sq.im, F2{qv.x, qv.y}, d3.im)};
                Ss = CF2{sw2::add_mul(Ss.re, F2{qv.z, qv.w}, d3.re), sw2::add_mul(Ss.im, F2{qv.z, qv.w}, d3.im)};
            }
            const F2 inv0{b0[q].x, b0[q].y}, U1{b0[q].z, b0[q].w}, U2{b1[q].x, b1[q].y}, ta{b1[q].z, b1[q].w};
            const F2 tb{b2[q].x, b2[q].y};
            Acc ar = sw2::acc_start(F2{yb[q].x, yb[q].y}), ai = sw2::acc_start(F2{yb[q].z, yb[q].w});
            sw2::acc_sub_mul(ar, ta, Sq.re);
            sw2::acc_sub_mul(ai, ta, Sq.im);
            sw2::acc_sub_mul(ar, tb, Ss.re);
            sw2::acc_sub_mul(ai, tb, Ss.im);
            sw2::acc_sub_mul(ar, U2, d2.re);
            sw2::acc_sub_mul(ai, U2, d2.im);
            sw2::acc_sub_mul(ar, U1, d1.re);
            sw2::acc_sub_mul(ai, U1, d1.im);
            const CF2 d{sw2::mul_n(inv0, sw2::acc_done(ar)), sw2::mul_n(inv0, sw2::acc_done(ai))};
            const CF2 u{df::add(d.re, chains::neg(xo[q].re)), df::add(d.im, chains::neg(xo[q].im))};
            chains::store_f64(ucol, 2 * i + par, u);
            d3 = d2;
            d2 = d1;
            d1 = d;
        }
    }
    if (par == 0)
        for (int k = n; k < N; k++) reinterpret_cast<double2 *>(ucol)[k] = make_double2(0.0, 0.0);
}

// Fixed grid of resident blocks, warp slots striding over the warp-sized groups of chains in
// the class order, each slot with its [row][lane] slice of the problem's spill scratch (as
// the float-float solves).
template <int PROBLEM>
__global__ void __launch_bounds__(128, 3) step_df_kernel(Plan p, const double *x, const double *load, double *u,
                                                      float4 *scr) {
    const int lane = threadIdx.x & 31;
    const long slot = (blockIdx.x * (long)blockDim.x + threadIdx.x) >> 5;
    const long nslots = ((long)gridDim.x * blockDim.x) >> 5;
    const int rows = PROBLEM == SHEN_HELMHOLTZ ? p.rows_h : p.rows_b;
    float4 *ys = scr + slot * (long)rows * 32 + lane;
    const float4 *T = reinterpret_cast<const float4 *>(p.d_mv_df);
    const long nch = 2 * p.n_classes;
    for (long t0 = slot * 32; t0 < 2 * p.n_modes; t0 += nslots * 32) {
        const long t = t0 + lane;
        if (t >= 2 * p.n_modes) continue;
        const long mode = p.d_order[t >> 1];
        const int par = (int)(t & 1);
        const int cls = p.d_mode_class[mode];
        const long off = 2 * mode * (long)p.N, ch = 2L * cls + par;
        const double z2 = p.d_class_z2[cls];
        if (PROBLEM == SHEN_HELMHOLTZ)
            step_helm_chain(p, par, z2, x + off, load ? load + off : nullptr, u + off,
                            chains::HelmDF{p.df_hb + ch, p.df_hf + ch, nch}, T, ys);
        else
            step_bih_chain(p, par, z2, x + off, load ? load + off : nullptr, u + off,
                           chains::BihDF{p.df_bf + ch, p.df_bb0 + ch, p.df_bb1 + ch, p.df_bb2 + ch, nch},
                           T + 2 * p.N, p.df_qs, ys);
    }
}

}  // namespace

// Resident grid of the step kernels (within the warp slots of the problem's spill scratch).
cudaError_t step_setup(Plan &p) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const void *ks[2] = {(const void *)step_df_kernel<SHEN_HELMHOLTZ>, (const void *)step_df_kernel<SHEN_BIHARMONIC>};
    for (int pb = 0; pb < 2; pb++) {
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ks[pb], 128, 0);
        if (e != cudaSuccess) return e;
        const long slots = std::max(p.df_grid[pb][0], p.df_grid[pb][1]);
        p.step_grid[pb] = (int)std::max(1L, std::min<long>((long)std::max(1, per_sm) * sms, slots));
    }
    return cudaSuccess;
}

// One Crank-Nicolson step of `problem` for every mode (mode-major fields):
//   Helmholtz  u = -x + H_h^-1 (2 c B x + (2/nu) load)      (H_h u = R_h x + (2/nu) load)
//   biharmonic u = -x + H_b^-1 (-2 c (A - z2 B) x - (2/nu) load)   (H_b u = -R_b x - (2/nu) load)
// load may be null.  Uses the problem's float-float spill scratch (the solves' rule on overlap).
cudaError_t launch_step_df(const Plan &p, int problem, const double *x, const double *load, double *u,
                           cudaStream_t s) {
    if (p.n_modes <= 0) return cudaSuccess;
    const int pb = problem == SHEN_HELMHOLTZ ? 0 : 1;
    const long blocks = std::min<long>((2 * p.n_modes + 127) / 128, p.step_grid[pb]);
    if (problem == SHEN_HELMHOLTZ)
        step_df_kernel<SHEN_HELMHOLTZ><<<(unsigned)blocks, 128, 0, s>>>(p, x, load, u, p.d_ys[0]);
    else
        step_df_kernel<SHEN_BIHARMONIC><<<(unsigned)blocks, 128, 0, s>>>(p, x, load, u, p.d_ys[1]);
    return cudaGetLastError();
}

}  // namespace shen
