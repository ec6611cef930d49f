// Velocity recovery of the linear step (Sec. 3): with the wall-normal velocity u
// (biharmonic coefficients) and g (Dirichlet coefficients) of the new time level,
//   f = -du/dx projected on the Dirichlet space:  B_D f = -C u,  C_kj = (psi_j', phi_k)
//   (Eq. ffin with the sign of Eq. f), and, for every mode except m = n = 0,
//   v = i (n g - m f) / z2,   w = -i (n f + m g) / z2        (Eqs. f3, g3 solved).
//
// C has three diagonals (Table tab:matrices): C_{k,k-3} = pi (k-2)(k+1)/k,
// C_{k,k-1} = -2 pi (k+1)^2/(k+2), C_{k,k+1} = pi (k+1), coupling opposite parities;
// B_D is tridiagonal per parity (B_kk = pi/2 (c_k + c_{k+2}), B_{k,k+-2} = -pi/2) and the
// same for every mode, so its LU factors are one per-N table.
//
// One thread per (mode, parity of f), on a fixed grid of resident blocks whose warp slots
// stride over the chains: the forward sweep forms the right-hand side -C u from a
// rolling window of u rows of the other parity and eliminates with the table's l; it
// spills y (float-float) to the plan's [warp slot][row][lane] scratch (512 contiguous
// bytes per warp and row).  The back substitution finishes f row by row and turns
// (f, g) into (v, w) at once, so f is never stored unless the caller asks for it.
// Float-float arithmetic; float64 in and out.
#include <algorithm>
#include <cmath>
#include <vector>

#include "chains.cuh"

namespace shen {
namespace {

using chains::CF2;
using df::F2;

// Element k of a u or g column, with the sweeps' 256-byte L2 fetch size (chains::ld_col:
// 10.72 -> 10.58 ms at N = 1024, 1024 x 1024).  The outputs never overlap u or g.
__device__ __forceinline__ CF2 ld_cf2(const double *col, long k) {
    const double2 v = chains::ld_col(reinterpret_cast<const double2 *>(col) + k);
    return CF2{df::from_f64(v.x), df::from_f64(v.y)};
}

__device__ __forceinline__ F2 nrm(F2 x) { return df::fast_two_sum(x.hi, x.lo); }

// a * x + b * y for float-float scalars a, b and complex float-float x, y
__device__ __forceinline__ CF2 lin2(F2 a, CF2 x, F2 b, CF2 y) {
    return CF2{nrm(df::add(df::mul(a, x.re), df::mul(b, y.re))), nrm(df::add(df::mul(a, x.im), df::mul(b, y.im)))};
}

// Table row k (3 float4): (l_k, 1/U0_k) of B_D's LU on k's parity chain,
// (-C_{k,k-3}, -C_{k,k-1}), (-C_{k,k+1}, 0); entries outside the matrices are zero.
__device__ void velocity_chain(const Plan &p, const float4 *T, const double *u, const double *g, double *v,
                               double *w, double *fo, long tid, float4 *ys) {
    const long mode = tid >> 1;
    const int par = (int)(tid & 1);
    const int N = p.N, n = N - 2, nu_ = N - 4;
    const int rows = (n - par + 1) / 2;
    // wavenumbers of the mode (grid layout ix * Nz + iz, FFT order in iz)
    const long ix = mode / p.grid_Nz, iz = mode % p.grid_Nz;
    const long kz = iz < p.grid_Nz / 2 ? iz : iz - p.grid_Nz;
    const double m = 2.0 * kPi * (double)ix / p.grid_Lx, nn = 2.0 * kPi * (double)kz / p.grid_Lz;
    const double z2 = m * m + nn * nn;
    if (!(z2 > 0.0)) return;                      // m = n = 0: mean flow (Eqs. v00, w00), not here
    const F2 a = df::from_f64(nn / z2), b = df::from_f64(m / z2);
    // element k of the mode's columns at complex index k rs from col (mode-major: rs = 1;
    // wall-index-first: rs = n_modes)
    const long col = p.wall_first ? 2 * mode : 2 * mode * N;
    const long rs = p.wall_first ? p.n_modes : 1L;
    const double *uc = u + col, *gc = g + col;
    double *vc = v + col, *wc = w + col;
    double *fc = fo ? fo + col : nullptr;
    const F2 zero{0.f, 0.f};
    const CF2 z{zero, zero};
    auto U = [&](int j) { return (j >= 0 && j < nu_) ? ld_cf2(uc, j * rs) : z; };
    // forward: y_i = r_i - l_i y_{i-1}, r_i = -(C u)_k, k = 2 i + par.  (Register prefetch of
    // the rows, as in the solves, made this kernel slower: its long float-float body runs
    // best in these plain rolled loops.)
    CF2 um3 = U(par - 3), um1 = U(par - 1), up1 = U(par + 1);
    CF2 y{zero, zero};
    for (int i = 0; i < rows; i++) {
        const int k = 2 * i + par;
        const float4 t0 = T[3 * k], t1 = T[3 * k + 1], t2 = T[3 * k + 2];
        const F2 l{t0.x, t0.y}, c3{t1.x, t1.y}, c1{t1.z, t1.w}, cp{t2.x, t2.y};
        CF2 r;
        r.re = nrm(df::add(df::add(df::mul(c3, um3.re), df::mul(c1, um1.re)), df::mul(cp, up1.re)));
        r.im = nrm(df::add(df::add(df::mul(c3, um3.im), df::mul(c1, um1.im)), df::mul(cp, up1.im)));
        y.re = chains::fnma(l, y.re, r.re);
        y.im = chains::fnma(l, y.im, r.im);
        ys[(long)i * 32] = make_float4(y.re.hi, y.re.lo, y.im.hi, y.im.lo);
        um3 = um1;
        um1 = up1;
        up1 = U(k + 3);
    }
    // back substitution f_i = (y_i + (pi/2) f_{i+1}) / U0_i, then v, w of row k
    const F2 half_pi = df::from_f64(kPi / 2);
    CF2 fn = z;
    for (int i = rows - 1; i >= 0; i--) {
        const int k = 2 * i + par;
        const float4 yv = ys[(long)i * 32];
        const F2 inv{T[3 * k].z, T[3 * k].w};
        CF2 f;
        f.re = nrm(df::mul(inv, df::add(F2{yv.x, yv.y}, df::mul(half_pi, fn.re))));
        f.im = nrm(df::mul(inv, df::add(F2{yv.z, yv.w}, df::mul(half_pi, fn.im))));
        const CF2 gk = ld_cf2(gc, k * rs);
        // v = i (a g - b f), w = -i (a f + b g);  i (x + i y) = -y + i x
        const CF2 t = lin2(a, gk, chains::neg(b), f);
        const CF2 sm = lin2(a, f, b, gk);
        reinterpret_cast<double2 *>(vc)[k * rs] = make_double2(-df::to_f64(t.im), df::to_f64(t.re));
        reinterpret_cast<double2 *>(wc)[k * rs] = make_double2(df::to_f64(sm.im), -df::to_f64(sm.re));
        if (fc) reinterpret_cast<double2 *>(fc)[k * rs] = make_double2(df::to_f64(f.re), df::to_f64(f.im));
        fn = f;
    }
    if (par == 0)
        for (int k = n; k < N; k++) {
            reinterpret_cast<double2 *>(vc)[k * rs] = make_double2(0.0, 0.0);
            reinterpret_cast<double2 *>(wc)[k * rs] = make_double2(0.0, 0.0);
            if (fc) reinterpret_cast<double2 *>(fc)[k * rs] = make_double2(0.0, 0.0);
        }
}

__global__ void __launch_bounds__(128) velocity_df_kernel(Plan p, const float4 *T, const double *u,
                                                          const double *g, double *v, double *w, double *fo,
                                                          float4 *scr) {
    const int lane = threadIdx.x & 31;
    const long slot = (blockIdx.x * (long)blockDim.x + threadIdx.x) >> 5;
    const long nslots = ((long)gridDim.x * blockDim.x) >> 5;
    float4 *ys = scr + slot * (long)((p.N - 2 + 1) / 2) * 32 + lane;
    for (long t0 = slot * 32; t0 < 2 * p.n_modes; t0 += nslots * 32)
        if (t0 + lane < 2 * p.n_modes) velocity_chain(p, T, u, g, v, w, fo, t0 + lane, ys);
}

inline float4 pair4(double a, double b) {
    const float ah = (float)a, bh = (float)b;
    return make_float4(ah, (float)(a - (double)ah), bh, (float)(b - (double)bh));
}

}  // namespace

// Per-N table of velocity_df_kernel, built on the host in float64 and split into
// float-float pairs: 3 N float4 (gl: Chebyshev-Gauss-Lobatto B_D, c_{N-1} = 2).
void build_velocity_table(int N, std::vector<float4> &T, bool gl) {
    const double pi = kPi;
    T.assign((size_t)3 * N, make_float4(0.f, 0.f, 0.f, 0.f));
    const int n = N - 2, nu = N - 4;
    double U0prev[2] = {0.0, 0.0};
    const double off = -pi / 2;
    for (int k = 0; k < n; k++) {
        const int par = k & 1;
        const double d = pi / 2 * ((k == 0 ? 2.0 : 1.0) + ((gl && k + 2 == N - 1) ? 2.0 : 1.0));
        double l = 0.0, U0 = d;
        if (k >= 2) {
            l = off / U0prev[par];
            U0 = d - l * off;
        }
        U0prev[par] = U0;
        const double K = k;
        const double cm3 = (k - 3 >= 0 && k - 3 < nu) ? pi * (K - 2) * (K + 1) / K : 0.0;
        const double cm1 = (k - 1 >= 0 && k - 1 < nu) ? -2 * pi * (K + 1) * (K + 1) / (K + 2) : 0.0;
        const double cp1 = (k + 1 < nu) ? pi * (K + 1) : 0.0;
        T[3 * k] = pair4(l, 1.0 / U0);
        T[3 * k + 1] = pair4(-cm3, -cm1);
        T[3 * k + 2] = pair4(-cp1, 0.0);
    }
}

cudaError_t launch_velocity_df(const Plan &p, const double *u, const double *g, double *v, double *w, double *f,
                               cudaStream_t s) {
    if (p.n_modes <= 0) return cudaSuccess;
    velocity_df_kernel<<<(unsigned)p.vel_grid, 128, 0, s>>>(p, reinterpret_cast<const float4 *>(p.d_vel_df), u, g,
                                                            v, w, f, p.d_vel_ys);
    return cudaGetLastError();
}

cudaError_t velocity_setup(Plan &p, long long &bytes) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, velocity_df_kernel, 128, 0);
    if (e != cudaSuccess) return e;
    const long needed = (2 * p.n_modes + 127) / 128;
    p.vel_grid = (int)std::max<long>(1, std::min<long>((long)std::max(1, per_sm) * sms, needed));
    const size_t n = (size_t)p.vel_grid * 4 * ((p.N - 2 + 1) / 2) * 32;        // float4
    bytes += (long long)(n * sizeof(float4));
    return cudaMalloc((void **)&p.d_vel_ys, n * sizeof(float4));
}

}  // namespace shen
