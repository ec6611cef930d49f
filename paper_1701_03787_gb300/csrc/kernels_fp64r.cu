// float64 sweeps followed by one step of iterative refinement whose residual is formed in
// double-double arithmetic (precision SHEN_FP64_R1).
//
// At high wavenumbers the unpivoted O(N) algorithm of Sec. 4 loses a few digits (the
// systems' componentwise condition reaches ~1e5 at N = 1024, z = 1145, which is where
// Table tab:roundoff shows the roundoff growing), and a residual formed in float64 has a
// floor of the same order.  Here the residual r = f - H u is formed with every matrix
// entry and every product and sum carried as an unevaluated pair of float64 (Dekker's
// TwoProd with a fused multiply-add, Knuth's TwoSum; Dekker 1971, Knuth TAOCP vol. 2,
// 4.2.2), so r is resolved far below the float64 rounding of u.  One float64 solve of
// H d = r and u += d then leave only the float64 rounding of the result.
//
// Matrix structure per parity chain (Sec. 3, Table tab:matrices, Eqs. N_Q, pk, rk;
// stiffness with the + sign under which Eqs. ufin, gfin discretise the PDEs):
//   Dirichlet  (B u)_k = B_kk u_k - pi/2 (u_{k-2} + u_{k+2}),
//              (A u)_k = A_kk u_k + A_tail(k) sum_{j = k+2, k+4, ...} u_j
//   biharmonic (B u)_k = B_{k,k-4} u_{k-4} + B_{k,k-2} u_{k-2} + B_kk u_k + B_{k,k+2} u_{k+2}
//                        + B_{k,k+4} u_{k+4} (B symmetric),
//              (A u)_k = A_{k,k-2} u_{k-2} + A_kk u_k + A_{k,k+2} u_{k+2},
//              (Q u)_k = Q_kk u_k + p_k sum_{j >= k+2} q_j u_j + r_k sum_{j >= k+2} s_j u_j.
// Each entry is a rational multiple of pi (or a rational): it is formed on the host from
// exact integers by a double-double division and a product with pi as a double-double.
//
// Work decomposition: one thread per (mode, parity) chain, as in the float64 kernels.
// Each chain first copies its right-hand side into its slot of the plan's spill scratch
// ([warp slot][row][lane], 16 bytes per row), so u may alias f.  The residual overwrites
// that copy row by row from the bottom up (the suffix sums run in that direction), the
// correction's forward sweep runs in place on it and the back substitution adds d to u.
#include <algorithm>
#include <cmath>
#include <vector>

#include "chains.cuh"

namespace shen {

// ------------------------------------------------------------------ host tables

namespace {

struct HDD {      // host double-double, value = hi + lo
    double hi, lo;
};

HDD h_fast_two_sum(double a, double b) {
    const double s = a + b;
    return {s, b - (s - a)};
}

HDD h_two_prod(double a, double b) {
    const double p = a * b;
    return {p, std::fma(a, b, -p)};
}

HDD h_mul(HDD x, HDD y) {
    const double p = x.hi * y.hi;
    double e = std::fma(x.hi, y.hi, -p);
    e = std::fma(x.hi, y.lo, e);
    e = std::fma(x.lo, y.hi, e);
    return h_fast_two_sum(p, e);
}

// (a * b) / den exactly rounded to double-double; a, b, den integers below 2^53 with
// a * b below 2^106 (the product is formed exactly by TwoProd).
HDD h_ratio(double a, double b, double den) {
    const HDD num = h_two_prod(a, b);
    const double q1 = num.hi / den;
    const HDD pq = h_two_prod(q1, den);
    const double r = ((num.hi - pq.hi) - pq.lo) + num.lo;
    return h_fast_two_sum(q1, r / den);
}

// pi as a double-double: the float64 nearest pi and the float64 nearest the rest.
const HDD kPiDD = {3.141592653589793116, 1.2246467991473532e-16};

HDD h_pi_ratio(double a, double b, double den) { return h_mul(h_ratio(a, b, den), kPiDD); }

}  // namespace

// Entry k of each table at [t * (N + 8) + k], as (hi, lo); rows beyond the unknowns are 0.
void build_dd_tables(int N, bool gl, std::vector<double2> &T) {
    const int S = N + 8;
    T.assign((size_t)kDdTables * S, make_double2(0.0, 0.0));
    auto put = [&](int t, int k, HDD v) { T[(size_t)t * S + k] = make_double2(v.hi, v.lo); };
    auto c = [&](int k) { return (k == 0 || (gl && k == N - 1)) ? 2.0 : 1.0; };
    put(kDdHboff, 0, h_pi_ratio(-1, 1, 2));
    for (int k = 0; k < N - 2; k++) {
        const double K = k;
        put(kDdHb0, k, h_pi_ratio(c(k) + c(k + 2), 1, 2));
        put(kDdHa0, k, h_pi_ratio(-2 * (K + 1), K + 2, 1));
        put(kDdHat, k, h_pi_ratio(-4 * (K + 1), 1, 1));
    }
    for (int k = 0; k < N - 4; k++) {
        const double K = k, K3 = K + 3;
        put(kDdBb0, k, h_pi_ratio(c(k) * K3 * K3 + 4 * (K + 2) * (K + 2) + c(k + 4) * (K + 1) * (K + 1), 1,
                                  2 * K3 * K3));
        put(kDdBb2, k, h_pi_ratio(-((K + 2) * (K + 5) + (K + 1) * (K + 4)), 1, K3 * (K + 5)));
        put(kDdBb4, k, h_pi_ratio(K + 1, 1, 2 * K3));
        put(kDdBa0, k, h_pi_ratio(-4 * (K + 1) * (K + 2), K + 2, K3));
        put(kDdBap, k, h_pi_ratio(2 * (K + 1), K + 2, 1));
        put(kDdBam, k, h_pi_ratio(2 * (K - 1), K + 2, 1));
        put(kDdBq0, k, h_pi_ratio(8 * (K + 1) * (K + 1), (K + 2) * (K + 4), 1));
        put(kDdBp, k, h_pi_ratio(8 * K * (K + 1), (K + 2) * (K + 4), 1));
        put(kDdBr, k, h_pi_ratio(24 * (K + 1), K + 2, 1));
        put(kDdBq, k, h_ratio(1, 1, K3));
        put(kDdBs, k, h_ratio(K + 2, K + 2, K3));
    }
}

namespace {

// ---------------------------------------------------------------- device arithmetic

struct DD {
    double hi, lo;
};

__device__ __forceinline__ DD two_sum(double a, double b) {
    const double s = __dadd_rn(a, b);
    const double bb = __dsub_rn(s, a);
    return {s, __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb))};
}

__device__ __forceinline__ DD fast_two_sum(double a, double b) {
    const double s = __dadd_rn(a, b);
    return {s, __dsub_rn(b, __dsub_rn(s, a))};
}

__device__ __forceinline__ DD add(DD x, DD y) {
    const DD s = two_sum(x.hi, y.hi);
    return fast_two_sum(s.hi, __dadd_rn(s.lo, __dadd_rn(x.lo, y.lo)));
}

__device__ __forceinline__ DD neg(DD x) { return {-x.hi, -x.lo}; }

__device__ __forceinline__ DD mul(DD x, double y) {          // y exact
    const double p = __dmul_rn(x.hi, y);
    double e = __fma_rn(x.hi, y, -p);
    e = __fma_rn(x.lo, y, e);
    return fast_two_sum(p, e);
}

__device__ __forceinline__ DD mul(DD x, DD y) {
    const double p = __dmul_rn(x.hi, y.hi);
    double e = __fma_rn(x.hi, y.hi, -p);
    e = __fma_rn(x.hi, y.lo, e);
    e = __fma_rn(x.lo, y.hi, e);
    return fast_two_sum(p, e);
}

__device__ __forceinline__ DD ldd(const double2 *t, int k) {
    const double2 v = t[k];
    return {v.x, v.y};
}

struct CDD {      // complex double-double
    DD re, im;
};
__device__ __forceinline__ CDD cmul(DD a, double2 u) { return {mul(a, u.x), mul(a, u.y)}; }
__device__ __forceinline__ CDD cmul(DD a, CDD v) { return {mul(a, v.re), mul(a, v.im)}; }
__device__ __forceinline__ CDD cadd(CDD a, CDD b) { return {add(a.re, b.re), add(a.im, b.im)}; }

// Spill scratch row i of this thread's slot ([row][lane], 32 lanes of 16 bytes per row).
__device__ __forceinline__ double2 &srow(double2 *ys, int i) { return ys[(long)i * 32]; }

struct Item {
    long col;
    int cls, par;
};

__device__ __forceinline__ bool item_of(const Plan &p, const int *order, long m0, long count, long tid, Item &w) {
    if (tid >= 2 * count) return false;
    const long it = tid >> 1;
    w.par = (int)(tid & 1);
    const long mode = order ? (long)order[it] : m0 + it;
    w.col = mode - m0;
    w.cls = p.d_mode_class[mode];
    return true;
}

// ------------------------------------------------------------------ Helmholtz

__device__ void helm_fp64r_chain(const Plan &p, int par, double z2, const double *fcol, double *ucol,
                                 const double *F, double2 *ys) {
    const int N = p.N, n = N - 2;
    const int rows = (n - par + 1) / 2;
    const double h = (z2 + p.c) * kPi / 2;
    const double2 *f2 = reinterpret_cast<const double2 *>(fcol);
    double2 *u2 = reinterpret_cast<double2 *>(ucol);
    for (int i = 0; i < rows; i++) srow(ys, i) = f2[2 * i + par];      // keep f (u may alias it)
    chains::solve_helm_fp64_chain(N, par, fcol, ucol, F, h, 1);
    // residual r = f - alpha B u + A u, bottom up (S = sum_{j > i} u_j)
    const DD alpha = two_sum(z2, p.c);
    const double2 *T = p.d_dd;
    const int Ts = N + 8;
    const DD boff = ldd(T + kDdHboff * Ts, 0);
    CDD S{{0, 0}, {0, 0}};
    double2 un = make_double2(0.0, 0.0);                               // u_{i+1}
    double2 uc = rows > 0 ? u2[2 * (rows - 1) + par] : un;            // u_i
    for (int i = rows - 1; i >= 0; i--) {
        const int k = 2 * i + par;
        const double2 up = i > 0 ? u2[k - 2] : make_double2(0.0, 0.0);   // u_{i-1}
        const DD b0 = ldd(T + kDdHb0 * Ts, k), a0 = ldd(T + kDdHa0 * Ts, k), at = ldd(T + kDdHat * Ts, k);
        const double2 fi = srow(ys, i);
        // (B u) and (A u) of row k, re and im
        const CDD Bu = cadd(cmul(b0, uc), cadd(cmul(boff, up), cmul(boff, un)));
        const CDD Au = cadd(cmul(a0, uc), cmul(at, S));
        const CDD aBu = cmul(alpha, Bu);
        const DD rre = add(add(DD{fi.x, 0.0}, neg(aBu.re)), Au.re);
        const DD rim = add(add(DD{fi.y, 0.0}, neg(aBu.im)), Au.im);
        srow(ys, i) = make_double2(rre.hi, rim.hi);
        S.re = add(S.re, DD{uc.x, 0.0});
        S.im = add(S.im, DD{uc.y, 0.0});
        un = uc;
        uc = up;
    }
    // correction: forward y = f - l y_{i-1} in place, back d_i = (y_i + h d_{i+1} - U2_i Sd_{i+1}) / U0,
    // u_i += d_i
    double2 y = make_double2(0.0, 0.0);
    for (int i = 0; i < rows; i++) {
        const double l = F[i * kHelmF64 + 2];
        const double2 r = srow(ys, i);
        y.x = fma(-l, y.x, r.x);
        y.y = fma(-l, y.y, r.y);
        srow(ys, i) = y;
    }
    double2 dn = make_double2(0.0, 0.0), Sd = dn;
    for (int i = rows - 1; i >= 0; i--) {
        const double inv0 = F[i * kHelmF64 + 0], U2 = F[i * kHelmF64 + 1];
        const double2 yi = srow(ys, i);
        double2 t;
        t.x = fma(-U2, Sd.x, fma(h, dn.x, yi.x));
        t.y = fma(-U2, Sd.y, fma(h, dn.y, yi.y));
        dn = make_double2(inv0 * t.x, inv0 * t.y);
        Sd.x += dn.x;
        Sd.y += dn.y;
        double2 ui = u2[2 * i + par];
        ui.x += dn.x;
        ui.y += dn.y;
        u2[2 * i + par] = ui;
    }
}

// ------------------------------------------------------------------ biharmonic

__device__ void bih_fp64r_chain(const Plan &p, int par, double z2, const double *fcol, double *ucol,
                                const double *F, double2 *ys) {
    const int N = p.N, n = N - 4;
    const int rows = (n - par + 1) / 2;
    const double2 *f2 = reinterpret_cast<const double2 *>(fcol);
    double2 *u2 = reinterpret_cast<double2 *>(ucol);
    for (int i = 0; i < rows; i++) srow(ys, i) = f2[2 * i + par];
    chains::solve_bih_fp64_chain(N, par, fcol, ucol, F, p.tab.qk, p.tab.sk, 1);
    // residual r = f - Q u - a A u - b B u, bottom up (Sq, Ss = sums over j > i of q_j u_j, s_j u_j)
    const DD zc = two_sum(z2, p.c);
    const DD a = neg(two_sum(2.0 * z2, p.c));                         // -(2 z2 + c)
    const DD b = mul(zc, z2);                                         // z2 (z2 + c)
    const double2 *T = p.d_dd;
    const int Ts = N + 8;
    auto tab = [&](int t, int k) { return ldd(T + t * Ts, k); };
    const double2 zero = make_double2(0.0, 0.0);
    CDD Sq{{0, 0}, {0, 0}}, Ss = Sq;
    // window u_{i-2} .. u_{i+2}
    double2 up2 = zero, up1 = zero;
    double2 u0 = rows > 0 ? u2[2 * (rows - 1) + par] : zero;
    double2 um1 = rows > 1 ? u2[2 * (rows - 2) + par] : zero;
    double2 um2 = rows > 2 ? u2[2 * (rows - 3) + par] : zero;
    for (int i = rows - 1; i >= 0; i--) {
        const int k = 2 * i + par;
        const int km2 = max(k - 2, 0), km4 = max(k - 4, 0);
        CDD Bu = cmul(tab(kDdBb0, k), u0);
        Bu = cadd(Bu, cmul(tab(kDdBb2, k), up1));
        Bu = cadd(Bu, cmul(tab(kDdBb4, k), up2));
        Bu = cadd(Bu, cmul(tab(kDdBb2, km2), um1));
        Bu = cadd(Bu, cmul(tab(kDdBb4, km4), um2));
        CDD Au = cmul(tab(kDdBa0, k), u0);
        Au = cadd(Au, cmul(tab(kDdBap, k), up1));
        Au = cadd(Au, cmul(tab(kDdBam, k), um1));
        CDD Qu = cmul(tab(kDdBq0, k), u0);
        Qu = cadd(Qu, cmul(tab(kDdBp, k), Sq));
        Qu = cadd(Qu, cmul(tab(kDdBr, k), Ss));
        const CDD H = cadd(Qu, cadd(cmul(a, Au), cmul(b, Bu)));
        const double2 fi = srow(ys, i);
        const DD rre = add(DD{fi.x, 0.0}, neg(H.re));
        const DD rim = add(DD{fi.y, 0.0}, neg(H.im));
        srow(ys, i) = make_double2(rre.hi, rim.hi);
        Sq = cadd(Sq, cmul(tab(kDdBq, k), u0));
        Ss = cadd(Ss, cmul(tab(kDdBs, k), u0));
        up2 = up1;
        up1 = u0;
        u0 = um1;
        um1 = um2;
        um2 = i >= 3 ? u2[2 * (i - 3) + par] : zero;
    }
    // correction: forward y_i = r_i - L1 y_{i-1} - L2 y_{i-2} in place; back substitution of
    // Algorithm LUSolveBiharmonic for d, u_i += d_i
    double2 y1 = zero, y2 = zero;
    for (int i = 0; i < rows; i++) {
        const double L1 = F[i * kBiF64 + 0], L2 = F[i * kBiF64 + 1];
        const double2 r = srow(ys, i);
        double2 y;
        y.x = fma(-L2, y2.x, fma(-L1, y1.x, r.x));
        y.y = fma(-L2, y2.y, fma(-L1, y1.y, r.y));
        srow(ys, i) = y;
        y2 = y1;
        y1 = y;
    }
    double2 d1 = zero, d2 = zero, d3 = zero, Dq = zero, Dsum = zero;
    for (int i = rows - 1; i >= 0; i--) {
        if (i + 3 < rows) {
            const int k3 = 2 * (i + 3) + par;
            const double q = p.tab.qk[k3], s = p.tab.sk[k3];
            Dq.x = fma(q, d3.x, Dq.x);
            Dq.y = fma(q, d3.y, Dq.y);
            Dsum.x = fma(s, d3.x, Dsum.x);
            Dsum.y = fma(s, d3.y, Dsum.y);
        }
        const double *row = F + i * kBiF64;
        const double inv0 = row[2], U1 = row[3], U2 = row[4], ta = row[5], tb = row[6];
        const double2 yi = srow(ys, i);
        double2 t;
        t.x = yi.x - U1 * d1.x - U2 * d2.x - ta * Dq.x - tb * Dsum.x;
        t.y = yi.y - U1 * d1.y - U2 * d2.y - ta * Dq.y - tb * Dsum.y;
        const double2 di = make_double2(inv0 * t.x, inv0 * t.y);
        double2 ui = u2[2 * i + par];
        ui.x += di.x;
        ui.y += di.y;
        u2[2 * i + par] = ui;
        d3 = d2;
        d2 = d1;
        d1 = di;
    }
}

// Fixed grid of resident blocks; warp slot w takes the warp-sized groups of chains w, w + W, ...
// and uses its own [row][lane] slice of the plan's scratch.
__global__ void __launch_bounds__(128) fp64r_kernel(Plan p, int problem, const int *order, long m0, long count,
                                                    const double *f, double *u, float4 *scr) {
    const int lane = threadIdx.x & 31;
    const long slot = (blockIdx.x * (long)blockDim.x + threadIdx.x) >> 5;
    const long nslots = ((long)gridDim.x * blockDim.x) >> 5;
    const int rows = problem == SHEN_HELMHOLTZ ? p.rows_h : p.rows_b;
    double2 *ys = reinterpret_cast<double2 *>(scr + slot * (long)rows * 32 + lane);
    for (long t0 = slot * 32; t0 < 2 * count; t0 += nslots * 32) {
        Item w;
        if (!item_of(p, order, m0, count, t0 + lane, w)) continue;
        const long off = 2 * w.col * (long)p.N;
        const double z2 = p.d_class_z2[w.cls];
        const long ch = (long)w.cls * 2 + w.par;
        if (problem == SHEN_HELMHOLTZ)
            helm_fp64r_chain(p, w.par, z2, f + off, u + off, p.d_fac_h + ch * p.rows_h * kHelmF64, ys);
        else
            bih_fp64r_chain(p, w.par, z2, f + off, u + off, p.d_fac_b + ch * p.rows_b * kBiF64, ys);
    }
}

}  // namespace

cudaError_t launch_solve_fp64r(const Plan &p, int problem, long m0, long count, const double *f, double *u,
                               cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    const int pb = problem == SHEN_HELMHOLTZ ? 0 : 1;
    const int *order = (m0 == 0 && count == p.n_modes) ? p.d_order : nullptr;
    // the scratch holds max(df_grid[pb]) blocks of 4 warp slots
    const long slots_blocks = std::max(p.df_grid[pb][0], p.df_grid[pb][1]);
    const unsigned g = (unsigned)std::max(1L, std::min<long>((2 * count + 127) / 128, slots_blocks));
    fp64r_kernel<<<g, 128, 0, s>>>(p, problem, order, m0, count, f, u, p.d_ys[pb]);
    return cudaGetLastError();
}

}  // namespace shen
