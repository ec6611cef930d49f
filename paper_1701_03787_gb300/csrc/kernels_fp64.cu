// float64 kernels: plan-time LU factorisation of every distinct z2, the float64
// sweeps (forward elimination + back substitution) and the right-hand-side operators.
//
// Source: Mortensen, arXiv:1701.03787.  Helmholtz: Sec. 4 (odd/even decoupling,
// upper-Hessenberg LU without pivoting, three values per U row).  Biharmonic:
// Algorithms LUbiharmonic, ReduceAB and LUSolveBiharmonic with the tail of Eq. ab.
// Right-hand sides: Eqs. gfin and ufin.
//
// Work decomposition: one thread per (mode, parity) chain; the real and imaginary
// parts share the factors and run side by side in the thread.  The forward sweep
// writes y into the output column, the backward sweep reads it back in reverse and
// overwrites it with u, so no scratch memory is needed and u == f works.
#include "chains.cuh"

namespace shen {
namespace {

using chains::ld2;
using chains::st2;

__global__ void factor_helmholtz_kernel(Plan p) {
    const long tid = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (tid >= 2 * p.n_classes) return;
    const long cls = tid >> 1;
    const int par = (int)(tid & 1);
    chains::factor_helm_chain(p.tab, p.N, p.d_class_z2[cls], p.c, par,
                              p.d_fac_h + ((cls * 2 + par) * (long)p.rows_h) * kHelmF64, p.rows_h, p.d_err, cls);
}

__global__ void factor_biharmonic_kernel(Plan p) {
    const long tid = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (tid >= 2 * p.n_classes) return;
    const long cls = tid >> 1;
    const int par = (int)(tid & 1);
    chains::factor_bih_chain(p.tab, p.N, p.d_class_z2[cls], p.c, par,
                             p.d_fac_b + ((cls * 2 + par) * (long)p.rows_b) * kBiF64, p.rows_b, p.d_err, cls);
}

struct WorkItem {
    long mode;   // global mode index
    long col;    // column offset relative to the field pointer
    int cls;
    int par;
};

__device__ __forceinline__ bool work_item(const Plan &p, const int *order, long m0, long count,
                                          WorkItem &w) {
    long tid = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (tid >= 2 * count) return false;
    long item = tid >> 1;
    w.par = (int)(tid & 1);
    w.mode = order ? (long)order[item] : m0 + item;
    w.col = w.mode - m0;
    w.cls = p.d_mode_class[w.mode];
    return true;
}

__global__ void __launch_bounds__(128) solve_helmholtz_fp64_kernel(Plan p, const int *order, long m0,
                                                                   long count, const double *f, double *u) {
    WorkItem w;
    if (!work_item(p, order, m0, count, w)) return;
    const double h = (p.d_class_z2[w.cls] + p.c) * kPi / 2;
    const long off = 2 * w.col * (p.wall_first ? 1L : (long)p.N), rs = p.wall_first ? p.n_modes : 1L;
    chains::solve_helm_fp64_chain(p.N, w.par, f + off, u + off,
                                  p.d_fac_h + ((long)(w.cls * 2 + w.par) * p.rows_h) * kHelmF64, h, rs);
}

__global__ void __launch_bounds__(128) solve_biharmonic_fp64_kernel(Plan p, const int *order, long m0,
                                                                    long count, const double *f, double *u) {
    WorkItem w;
    if (!work_item(p, order, m0, count, w)) return;
    const long off = 2 * w.col * (p.wall_first ? 1L : (long)p.N), rs = p.wall_first ? p.n_modes : 1L;
    chains::solve_bih_fp64_chain(p.N, w.par, f + off, u + off,
                                 p.d_fac_b + ((long)(w.cls * 2 + w.par) * p.rows_b) * kBiF64, p.tab.qk, p.tab.sk, rs);
}

// ------------------------------------------------------------ RHS operators

// Helmholtz R_h = (c - z2) B + A:
//   (R x)_k = g (B_{k,k-2} x_{k-2} + B_kk x_k + B_{k,k+2} x_{k+2}) + A_kk x_k
//             + A_tail(k) sum_{j = k+2, k+4, ...} x_j,   g = c - z2, B_{k,k+-2} = -pi/2.
__global__ void __launch_bounds__(128) matvec_helmholtz_fp64_kernel(Plan p, const double *x, const double *y,
                                                                    double beta, double *out, double sign) {
    WorkItem w;
    if (!work_item(p, nullptr, 0, p.n_modes, w)) return;
    const int N = p.N, n = N - 2, par = w.par;
    const int rows = (n - par + 1) / 2;
    // element k at complex index base + k rs (mode-major: rs = 1; wall-index-first: rs = n_modes)
    const long base = p.wall_first ? w.col : w.col * N, rs = p.wall_first ? p.n_modes : 1L;
    const double g = p.c - p.d_class_z2[w.cls];
    const double off = -kPi / 2;
    double2 S = make_double2(0.0, 0.0);                 // sum_{j >= i+1} x_j
    double2 xn = make_double2(0.0, 0.0);                // x_{i+1}
    double2 xc = rows > 0 ? ld2(x, base + (2 * (rows - 1) + par) * rs) : xn;   // x_i
    for (int i = rows - 1; i >= 0; i--) {
        const int k = 2 * i + par;
        S.x += xn.x; S.y += xn.y;
        const double2 xp = i > 0 ? ld2(x, base + (k - 2) * rs) : make_double2(0.0, 0.0);
        const double b0 = p.tab.bd0[k], a0 = p.tab.ad0[k], at = p.tab.adt[k];
        double2 r;
        r.x = g * (off * (xp.x + xn.x) + b0 * xc.x) + a0 * xc.x + at * S.x;
        r.y = g * (off * (xp.y + xn.y) + b0 * xc.y) + a0 * xc.y + at * S.y;
        r.x *= sign;
        r.y *= sign;
        if (y) {
            const double2 yi = ld2(y, base + k * rs);
            r.x = fma(beta, yi.x, r.x);
            r.y = fma(beta, yi.y, r.y);
        }
        st2(out, base + k * rs, r);
        xn = xc;
        xc = xp;
    }
    if (par == 0) {
        st2(out, base + n * rs, make_double2(0.0, 0.0));
        st2(out, base + (n + 1) * rs, make_double2(0.0, 0.0));
    }
}

// Biharmonic R_b = Q + (c - 2 z2) A + z2 (z2 - c) B:
//   (Q x)_k = Q_kk x_k + p_k sum_{j>=k+2} q_j x_j + r_k sum_{j>=k+2} s_j x_j
//   (A x)_k = A_{k,k-2} x_{k-2} + A_kk x_k + A_{k,k+2} x_{k+2}
//   (B x)_k = B_{k-4,k} x_{k-4} + B_{k-2,k} x_{k-2} + B_kk x_k + B_{k,k+2} x_{k+2} + B_{k,k+4} x_{k+4}
__global__ void __launch_bounds__(128) matvec_biharmonic_fp64_kernel(Plan p, const double *x, const double *y,
                                                                     double beta, double *out, double sign) {
    WorkItem w;
    if (!work_item(p, nullptr, 0, p.n_modes, w)) return;
    const int N = p.N, n = N - 4, par = w.par;
    const int rows = (n - par + 1) / 2;
    // element k at complex index base + k rs (mode-major: rs = 1; wall-index-first: rs = n_modes)
    const long base = p.wall_first ? w.col : w.col * N, rs = p.wall_first ? p.n_modes : 1L;
    const double z2 = p.d_class_z2[w.cls];
    const double ga = p.c - 2.0 * z2, gb = z2 * (z2 - p.c);
    const RowTables &T = p.tab;
    const double2 zero = make_double2(0.0, 0.0);
    auto X = [&](int i) { return (i >= 0 && i < rows) ? ld2(x, base + (2 * i + par) * rs) : zero; };
    double2 Sq = zero, Ss = zero;                      // sums over j >= i+1
    double2 xm2 = X(rows - 3), xm1 = X(rows - 2), xc = X(rows - 1), xp1 = zero, xp2 = zero;
    for (int i = rows - 1; i >= 0; i--) {
        const int k = 2 * i + par;
        if (i + 1 < rows) {
            const double q = T.qk[k + 2], s = T.sk[k + 2];
            Sq.x = fma(q, xp1.x, Sq.x); Sq.y = fma(q, xp1.y, Sq.y);
            Ss.x = fma(s, xp1.x, Ss.x); Ss.y = fma(s, xp1.y, Ss.y);
        }
        const double bm4 = i >= 2 ? T.bb4[k - 4] : 0.0, bm2 = i >= 1 ? T.bb2[k - 2] : 0.0;
        const double bp2 = T.bb2[k], bp4 = T.bb4[k];
        const double am = i >= 1 ? T.abm[k] : 0.0, ap = T.abp[k];
        double2 r;
        r.x = T.qb0[k] * xc.x + T.pk[k] * Sq.x + T.rk[k] * Ss.x
            + ga * (am * xm1.x + T.ab0[k] * xc.x + ap * xp1.x)
            + gb * (bm4 * xm2.x + bm2 * xm1.x + T.bb0[k] * xc.x + bp2 * xp1.x + bp4 * xp2.x);
        r.y = T.qb0[k] * xc.y + T.pk[k] * Sq.y + T.rk[k] * Ss.y
            + ga * (am * xm1.y + T.ab0[k] * xc.y + ap * xp1.y)
            + gb * (bm4 * xm2.y + bm2 * xm1.y + T.bb0[k] * xc.y + bp2 * xp1.y + bp4 * xp2.y);
        r.x *= sign;
        r.y *= sign;
        if (y) {
            const double2 yi = ld2(y, base + k * rs);
            r.x = fma(beta, yi.x, r.x);
            r.y = fma(beta, yi.y, r.y);
        }
        st2(out, base + k * rs, r);
        xp2 = xp1; xp1 = xc; xc = xm1; xm1 = xm2; xm2 = X(i - 3);
    }
    if (par == 0)
        for (int k = n; k < N; k++) st2(out, base + k * rs, zero);
}

inline unsigned blocks_for(long threads, int bs) { return (unsigned)((threads + bs - 1) / bs); }

}  // namespace

cudaError_t launch_factor_helmholtz(const Plan &p, cudaStream_t s) {
    factor_helmholtz_kernel<<<blocks_for(2 * p.n_classes, 128), 128, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_factor_biharmonic(const Plan &p, cudaStream_t s) {
    factor_biharmonic_kernel<<<blocks_for(2 * p.n_classes, 128), 128, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_solve_fp64(const Plan &p, int problem, long m0, long count, const double *f, double *u,
                              cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    // wall-index-first fields: modes in their own order, so that a warp's rows are contiguous
    const int *order = (m0 == 0 && count == p.n_modes && !p.wall_first) ? p.d_order : nullptr;
    if (problem == SHEN_HELMHOLTZ)
        solve_helmholtz_fp64_kernel<<<blocks_for(2 * count, 128), 128, 0, s>>>(p, order, m0, count, f, u);
    else
        solve_biharmonic_fp64_kernel<<<blocks_for(2 * count, 128), 128, 0, s>>>(p, order, m0, count, f, u);
    return cudaGetLastError();
}

cudaError_t launch_matvec_fp64(const Plan &p, int problem, const double *x, const double *y, double beta,
                               double *out, cudaStream_t s, double sign) {
    if (p.n_modes <= 0) return cudaSuccess;
    if (problem == SHEN_HELMHOLTZ)
        matvec_helmholtz_fp64_kernel<<<blocks_for(2 * p.n_modes, 128), 128, 0, s>>>(p, x, y, beta, out, sign);
    else
        matvec_biharmonic_fp64_kernel<<<blocks_for(2 * p.n_modes, 128), 128, 0, s>>>(p, x, y, beta, out, sign);
    return cudaGetLastError();
}

}  // namespace shen
