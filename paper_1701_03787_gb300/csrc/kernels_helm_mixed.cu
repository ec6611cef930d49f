// Helmholtz solve with float32 sweeps and one step of iterative refinement
// (Sec. 4 algorithm; the refinement is this library's precision scheme).
//
//   u0 = H^-1 f     float32 forward elimination + back substitution with the float64
//                   LU factors rounded to float32
//   r  = f - H u0   residual: float-float (DF variant) or float64 (F64 variant)
//   d  = H^-1 r     float32 sweeps again
//   u  = u0 + d     float-float / float64, written as float64
//
// Work decomposition: one warp per mode.  Lane l owns Chebyshev indices
// [2 R l, 2 R (l+1)) of the column, i.e. rows l R .. l R + R - 1 of both parity
// chains (k = 2 i + parity), held in registers.  The sweeps are linear recurrences
// along each chain; every lane runs its R rows with a zero carry, the warp combines
// the lane maps with a shuffle scan (affine maps: scalar for the forward sweep, 2x2
// for the back substitution whose state is (u_i, sum_{j >= i} u_j)), and each lane
// then adds the carried part.
//
// Helmholtz system per parity (k = 2i + p, alpha = z2 + c, h = alpha pi / 2):
//   H_{i,i-1} = -h,  H_ii = pi (alpha delta_k + 2 (k+1)(k+2)),  H_{i,j>i} = pi 4 (k+1) - h [j = i+1]
//   with delta_k = (c_k + 1) / 2.  LU: y_i = f_i + g_i y_{i-1} (g_i = h / U_{i-1,i-1}),
//   u_i = (y_i + h u_{i+1} - U2_i S_{i+1}) / U_ii,  S_{i+1} = sum_{j > i} u_j.
#include "df.cuh"
#include "shen_internal.h"

namespace shen {
namespace {

constexpr float kPiHi = 3.14159274101257324f;           // float(pi)
constexpr float kPiLo = -8.74227765734758577e-08f;      // pi - float(pi)

template <int R>
struct HelmCol {
    float2 w[2][R];     // working column (re, im) per parity and row-in-lane
};

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// Forward elimination y_i = f_i + g_i y_{i-1} across the warp, in place in w.
// gs (shared, [parity][j][lane]) holds g for row lane*R + j (0 for the chain's first
// row and for padding rows).  Both parity chains advance in the same loop (ILP).
template <int R>
__device__ __forceinline__ void forward_sweep(float2 (&w)[2][R], const float *gs, int lane) {
    float2 y[2] = {f2(0.f, 0.f), f2(0.f, 0.f)};
    float G[2] = {1.f, 1.f};
#pragma unroll
    for (int j = 0; j < R; j++)
#pragma unroll
        for (int p = 0; p < 2; p++) {
            const float g = gs[(p * R + j) * 32 + lane];
            y[p].x = fmaf(g, y[p].x, w[p][j].x);
            y[p].y = fmaf(g, y[p].y, w[p][j].y);
            w[p][j] = y[p];
            G[p] *= g;
        }
    // inclusive scan of the lane maps carry -> Y + G carry over lanes 0..31
#pragma unroll
    for (int d = 1; d < 32; d <<= 1)
#pragma unroll
        for (int p = 0; p < 2; p++) {
            const float Gu = __shfl_up_sync(0xffffffffu, G[p], d);
            const float Yx = __shfl_up_sync(0xffffffffu, y[p].x, d);
            const float Yy = __shfl_up_sync(0xffffffffu, y[p].y, d);
            if (lane >= d) {
                y[p].x = fmaf(G[p], Yx, y[p].x);
                y[p].y = fmaf(G[p], Yy, y[p].y);
                G[p] *= Gu;
            }
        }
    float2 c[2];
#pragma unroll
    for (int p = 0; p < 2; p++) {
        c[p].x = __shfl_up_sync(0xffffffffu, y[p].x, 1);
        c[p].y = __shfl_up_sync(0xffffffffu, y[p].y, 1);
        if (lane == 0) c[p] = f2(0.f, 0.f);
    }
    float P[2] = {1.f, 1.f};
#pragma unroll
    for (int j = 0; j < R; j++)
#pragma unroll
        for (int p = 0; p < 2; p++) {
            P[p] *= gs[(p * R + j) * 32 + lane];
            w[p][j].x = fmaf(P[p], c[p].x, w[p][j].x);
            w[p][j].y = fmaf(P[p], c[p].y, w[p][j].y);
        }
}

// Back substitution across the warp, in place in w (y in, u out).
// Per row: a = h inv0, c = U2 inv0;  u_i = a u_{i+1} - c S_{i+1} + inv0 y_i,  S_i = S_{i+1} + u_i.
// m0 (shared, [parity][j][lane]) receives row 0 of the lane-local transfer matrices
// (the response of u_i to the carried state) for the carried part.
template <int R>
__device__ __forceinline__ void backward_sweep(float2 (&w)[2][R], const float2 *fac, int lane, float h,
                                               float2 *m0) {
    float2 u[2] = {f2(0.f, 0.f), f2(0.f, 0.f)}, S[2] = {f2(0.f, 0.f), f2(0.f, 0.f)};
    float t00[2] = {1.f, 1.f}, t01[2] = {0.f, 0.f}, t10[2] = {0.f, 0.f}, t11[2] = {1.f, 1.f};
#pragma unroll
    for (int j = R - 1; j >= 0; j--)
#pragma unroll
        for (int p = 0; p < 2; p++) {
            const float2 fu = fac[(p * R + j) * 32 + lane];   // (inv0, U2)
            const float a = h * fu.x, c = fu.y * fu.x;
            float2 un;
            un.x = fmaf(a, u[p].x, fmaf(-c, S[p].x, fu.x * w[p][j].x));
            un.y = fmaf(a, u[p].y, fmaf(-c, S[p].y, fu.x * w[p][j].y));
            S[p].x += un.x;
            S[p].y += un.y;
            u[p] = un;
            w[p][j] = un;
            const float n00 = fmaf(a, t00[p], -c * t10[p]), n01 = fmaf(a, t01[p], -c * t11[p]);
            t10[p] += n00;
            t11[p] += n01;
            t00[p] = n00;
            t01[p] = n01;
            m0[(p * R + j) * 32 + lane] = f2(n00, n01);
        }
    // suffix scan over lanes of the affine maps x -> T x + v, state v = (u, S)
#pragma unroll
    for (int d = 1; d < 32; d <<= 1)
#pragma unroll
        for (int p = 0; p < 2; p++) {
            const float b00 = __shfl_down_sync(0xffffffffu, t00[p], d), b01 = __shfl_down_sync(0xffffffffu, t01[p], d);
            const float b10 = __shfl_down_sync(0xffffffffu, t10[p], d), b11 = __shfl_down_sync(0xffffffffu, t11[p], d);
            const float wux = __shfl_down_sync(0xffffffffu, u[p].x, d), wuy = __shfl_down_sync(0xffffffffu, u[p].y, d);
            const float wSx = __shfl_down_sync(0xffffffffu, S[p].x, d), wSy = __shfl_down_sync(0xffffffffu, S[p].y, d);
            if (lane + d < 32) {
                u[p].x = fmaf(t00[p], wux, fmaf(t01[p], wSx, u[p].x));
                u[p].y = fmaf(t00[p], wuy, fmaf(t01[p], wSy, u[p].y));
                S[p].x = fmaf(t10[p], wux, fmaf(t11[p], wSx, S[p].x));
                S[p].y = fmaf(t10[p], wuy, fmaf(t11[p], wSy, S[p].y));
                const float n00 = fmaf(t00[p], b00, t01[p] * b10), n01 = fmaf(t00[p], b01, t01[p] * b11);
                const float n10 = fmaf(t10[p], b00, t11[p] * b10), n11 = fmaf(t10[p], b01, t11[p] * b11);
                t00[p] = n00; t01[p] = n01; t10[p] = n10; t11[p] = n11;
            }
        }
    float2 cu[2], cS[2];
#pragma unroll
    for (int p = 0; p < 2; p++) {
        cu[p].x = __shfl_down_sync(0xffffffffu, u[p].x, 1);
        cu[p].y = __shfl_down_sync(0xffffffffu, u[p].y, 1);
        cS[p].x = __shfl_down_sync(0xffffffffu, S[p].x, 1);
        cS[p].y = __shfl_down_sync(0xffffffffu, S[p].y, 1);
        if (lane == 31) cu[p] = cS[p] = f2(0.f, 0.f);
    }
#pragma unroll
    for (int j = 0; j < R; j++)
#pragma unroll
        for (int p = 0; p < 2; p++) {
            const float2 m = m0[(p * R + j) * 32 + lane];
            w[p][j].x = fmaf(m.x, cu[p].x, fmaf(m.y, cS[p].x, w[p][j].x));
            w[p][j].y = fmaf(m.x, cu[p].y, fmaf(m.y, cS[p].y, w[p][j].y));
        }
}

}  // namespace
}  // namespace shen

namespace shen {
namespace {

// Residual r = f - H u0 for the lane's rows, written (rounded to float32) into w.
// u0c: the lane's u0 values (exact float32 numbers).  Float-float (DF = true) or
// float64 (DF = false) arithmetic.  H / pi row i (chain parity p, k = 2i + p):
//   E_i = alpha (delta_k u_i - (u_{i-1} + u_{i+1}) / 2) + 2(k+1)(k+2) u_i + 4(k+1) sum_{j>i} u_j
//   r_i = f_i - pi E_i.
template <int R, bool DF>
__device__ __forceinline__ void residual(float2 (&w)[2][R], const float2 *u0s, const double *fcol,
                                         int lane, int n, double alpha) {
#define U0(pp, jj) u0s[((pp) * R + (jj)) * 32 + lane]
    const df::F2 a_df = df::from_f64(alpha);
    const df::F2 pi_df = {kPiHi, kPiLo};
#pragma unroll
    for (int p = 0; p < 2; p++) {
        // lane totals of u0 (for the sum over rows above the lane), then a suffix scan
        float tre = 0.f, tim = 0.f, ere = 0.f, eim = 0.f;
        double dre = 0.0, dim = 0.0;
#pragma unroll
        for (int j = 0; j < R; j++) {
            if (DF) {
                const float2 uv = U0(p, j);
                df::F2 s = df::two_sum(tre, uv.x); tre = s.hi; ere += s.lo;
                s = df::two_sum(tim, uv.y); tim = s.hi; eim += s.lo;
            } else {
                const float2 uv = U0(p, j);
                dre += (double)uv.x;
                dim += (double)uv.y;
            }
        }
        // inclusive suffix scan of the lane totals
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            if (DF) {
                const float a0 = __shfl_down_sync(0xffffffffu, tre, d), a1 = __shfl_down_sync(0xffffffffu, ere, d);
                const float b0 = __shfl_down_sync(0xffffffffu, tim, d), b1 = __shfl_down_sync(0xffffffffu, eim, d);
                if (lane + d < 32) {
                    df::F2 s = df::add(df::F2{tre, ere}, df::F2{a0, a1}); tre = s.hi; ere = s.lo;
                    s = df::add(df::F2{tim, eim}, df::F2{b0, b1}); tim = s.hi; eim = s.lo;
                }
            } else {
                const double a0 = __shfl_down_sync(0xffffffffu, dre, d), b0 = __shfl_down_sync(0xffffffffu, dim, d);
                if (lane + d < 32) { dre += a0; dim += b0; }
            }
        }
        // exclusive: sum over lanes above
        df::F2 Tre, Tim;
        double Dre, Dim;
        {
            float a0 = __shfl_down_sync(0xffffffffu, tre, 1), a1 = __shfl_down_sync(0xffffffffu, ere, 1);
            float b0 = __shfl_down_sync(0xffffffffu, tim, 1), b1 = __shfl_down_sync(0xffffffffu, eim, 1);
            double da = __shfl_down_sync(0xffffffffu, dre, 1), db = __shfl_down_sync(0xffffffffu, dim, 1);
            if (lane == 31) { a0 = a1 = b0 = b1 = 0.f; da = db = 0.0; }
            Tre = df::fast_two_sum(a0, a1);
            Tim = df::fast_two_sum(b0, b1);
            Dre = da; Dim = db;
        }
        // neighbours across lane boundaries
        const float2 top = U0(p, R - 1), bot = U0(p, 0);
        float2 below = make_float2(__shfl_up_sync(0xffffffffu, top.x, 1), __shfl_up_sync(0xffffffffu, top.y, 1));
        float2 above = make_float2(__shfl_down_sync(0xffffffffu, bot.x, 1), __shfl_down_sync(0xffffffffu, bot.y, 1));
        if (lane == 0) below = make_float2(0.f, 0.f);
        if (lane == 31) above = make_float2(0.f, 0.f);
#pragma unroll
        for (int j = R - 1; j >= 0; j--) {
            const int i = lane * R + j;
            const int k = 2 * i + p;
            const float2 um = j > 0 ? U0(p, j - 1) : below;
            const float2 uc = U0(p, j);
            const float2 up = j < R - 1 ? U0(p, j + 1) : above;
            if (k < n) {
                const double2 fk = reinterpret_cast<const double2 *>(fcol)[k];
                const float delta = k == 0 ? 1.5f : 1.0f;
                const float e = 2.0f * (float)((k + 1) * (k + 2));
                const float t = 4.0f * (float)(k + 1);
                float2 r;
                if (DF) {
#pragma unroll
                    for (int c = 0; c < 2; c++) {
                        const float vm = c ? um.y : um.x, vc = c ? uc.y : uc.x, vp = c ? up.y : up.x;
                        const df::F2 T = c ? Tim : Tre;
                        const double fv = c ? fk.y : fk.x;
                        // b = delta u_i - (u_{i-1} + u_{i+1}) / 2
                        const df::F2 s = df::two_sum(vm, vp);
                        const df::F2 q = df::two_prod(delta, vc);
                        df::F2 b = df::two_sum(q.hi, -0.5f * s.hi);
                        b.lo = __fadd_rn(b.lo, __fsub_rn(q.lo, 0.5f * s.lo));
                        df::F2 E = df::mul(a_df, b);                           // alpha b
                        E = df::add(E, df::two_prod(e, vc));                   // + e u_i
                        E = df::add(E, df::mul(T, t));                         // + t sum_{j>i} u_j
                        const df::F2 piE = df::mul(pi_df, E);
                        const df::F2 fd = df::from_f64(fv);
                        const df::F2 d0 = df::two_sum(fd.hi, -piE.hi);
                        const float rv = __fadd_rn(d0.hi, __fadd_rn(d0.lo, __fsub_rn(fd.lo, piE.lo)));
                        if (c) r.y = rv; else r.x = rv;
                    }
                } else {
#pragma unroll
                    for (int c = 0; c < 2; c++) {
                        const double vm = c ? um.y : um.x, vc = c ? uc.y : uc.x, vp = c ? up.y : up.x;
                        const double T = c ? Dim : Dre;
                        const double fv = c ? fk.y : fk.x;
                        const double b = (double)delta * vc - 0.5 * (vm + vp);
                        const double E = fma(alpha, b, fma((double)e, vc, (double)t * T));
                        const float rv = (float)fma(-kPi, E, fv);
                        if (c) r.y = rv; else r.x = rv;
                    }
                }
                w[p][j] = r;
            } else {
                w[p][j] = make_float2(0.f, 0.f);
            }
            // sum over rows > i-1 for the next (lower) row
            if (DF) {
                Tre = df::add(Tre, uc.x);
                Tim = df::add(Tim, uc.y);
            } else {
                Dre += (double)uc.x;
                Dim += (double)uc.y;
            }
        }
    }
#undef U0
}

// One warp per work item.  fac: float32 factors [class][parity][j][lane] = (inv0, U2).
template <int R, bool DF>
__global__ void __launch_bounds__(128) helm_mixed_kernel(Plan p, const int *order, long m0, long count,
                                                         const double *f, double *u, const float2 *fac) {
    extern __shared__ float2 smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long item = (long)blockIdx.x * (blockDim.x >> 5) + warp;
    if (item >= count) return;                          // whole warp exits together
    const long mode = order ? (long)order[item] : m0 + item;
    const long col = mode - m0;
    const int cls = p.d_mode_class[mode];
    const int N = p.N, n = N - 2;
    const double alpha = p.d_class_z2[cls] + p.c;
    const float h = (float)(alpha * kPi / 2);
    float2 *m0buf = smem + (size_t)warp * (5 * R * 32);     // [2][R][32] transfer rows
    float2 *u0buf = m0buf + 2 * R * 32;                      // [2][R][32] u0
    float *gbuf = reinterpret_cast<float *>(u0buf + 2 * R * 32);   // [2][R][32] g
    const double *fcol = f + 2 * col * N;
    double *ucol = u + 2 * col * N;
    const float2 *F = fac + (size_t)cls * 2 * R * 32;

    float2 w[2][R];
#pragma unroll
    for (int j = 0; j < R; j++)
#pragma unroll
        for (int pp = 0; pp < 2; pp++) {
            const int i = lane * R + j, k = 2 * i + pp;
            if (k < n) {
                const double2 fk = reinterpret_cast<const double2 *>(fcol)[k];
                if (DF) w[pp][j] = make_float2(df::from_f64(fk.x).hi, df::from_f64(fk.y).hi);
                else w[pp][j] = make_float2((float)fk.x, (float)fk.y);
            } else {
                w[pp][j] = make_float2(0.f, 0.f);
            }
            float prev = 0.f;                          // 1/U of row i-1
            if (i > 0) prev = j > 0 ? F[(pp * R + j - 1) * 32 + lane].x : F[(pp * R + R - 1) * 32 + lane - 1].x;
            gbuf[(pp * R + j) * 32 + lane] = h * prev;
        }
    __syncwarp();
    // solve 1
    forward_sweep<R>(w, gbuf, lane);
    backward_sweep<R>(w, F, lane, h, m0buf);
#pragma unroll
    for (int pp = 0; pp < 2; pp++)
#pragma unroll
        for (int j = 0; j < R; j++) u0buf[(pp * R + j) * 32 + lane] = w[pp][j];
    __syncwarp();
    // residual and solve 2
    residual<R, DF>(w, u0buf, fcol, lane, n, alpha);
    forward_sweep<R>(w, gbuf, lane);
    backward_sweep<R>(w, F, lane, h, m0buf);
    // u = u0 + d
#pragma unroll
    for (int j = 0; j < R; j++)
#pragma unroll
        for (int pp = 0; pp < 2; pp++) {
            const int i = lane * R + j, k = 2 * i + pp;
            if (k < N) {
                double2 out = make_double2(0.0, 0.0);
                if (k < n) {
                    const float2 a = u0buf[(pp * R + j) * 32 + lane];
                    if (DF) {
                        out.x = df::to_f64(df::two_sum(a.x, w[pp][j].x));
                        out.y = df::to_f64(df::two_sum(a.y, w[pp][j].y));
                    } else {
                        out.x = (double)a.x + (double)w[pp][j].x;
                        out.y = (double)a.y + (double)w[pp][j].y;
                    }
                }
                reinterpret_cast<double2 *>(ucol)[k] = out;
            }
        }
    // trailing entries beyond the lanes' reach (at most 2: N - 2 unknowns <= 64 R)
    if (lane == 0)
        for (int k = max(n, 64 * R); k < N; k++) reinterpret_cast<double2 *>(ucol)[k] = make_double2(0.0, 0.0);
}

// float64 factors -> float32 table in the lane layout: row i = lane R + j of chain
// (class, parity) goes to [class][parity][j][lane].
__global__ void pack_helm_f32_kernel(Plan p, int R, float2 *out) {
    const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    const long total = p.n_classes * 2 * (long)R * 32;
    if (t >= total) return;
    const int lane = (int)(t % 32);
    const int j = (int)((t / 32) % R);
    const long chain = t / (32L * R);                  // class * 2 + parity
    const int i = lane * R + j;
    float2 v = make_float2(0.f, 0.f);
    if (i < p.rows_h) {
        const double *row = p.d_fac_h + (chain * p.rows_h + i) * kHelmF64;
        v = make_float2((float)row[0], (float)row[1]);   // 1/U_ii, U2
        if (row[0] == 0.0) v = make_float2(0.f, 0.f);
    }
    out[t] = v;
}

template <int R, bool DF>
cudaError_t launch_helm_mixed_R(const Plan &p, const int *order, long m0, long count, const double *f, double *u,
                                const float2 *fac, cudaStream_t s) {
    const int warps = 4;
    const size_t smem = (size_t)warps * 5 * R * 32 * sizeof(float2);
    auto kern = helm_mixed_kernel<R, DF>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const unsigned blocks = (unsigned)((count + warps - 1) / warps);
    kern<<<blocks, warps * 32, smem, s>>>(p, order, m0, count, f, u, fac);
    return cudaGetLastError();
}

}  // namespace

int helm_mixed_R(int N) {
    const int rows = (N - 2 + 1) / 2;
    const int R = (rows + 31) / 32;
    if (R <= 1) return 1;
    if (R <= 2) return 2;
    if (R <= 4) return 4;
    if (R <= 8) return 8;
    if (R <= 16) return 16;
    if (R <= 24) return 24;
    if (R <= 32) return 32;
    return 0;
}

cudaError_t pack_helm_f32(const Plan &p, int R, float2 *out, cudaStream_t s) {
    const long total = p.n_classes * 2 * (long)R * 32;
    pack_helm_f32_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(p, R, out);
    return cudaGetLastError();
}

cudaError_t launch_helm_mixed(const Plan &p, bool dfres, long m0, long count, const double *f, double *u,
                              cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    const int *order = (m0 == 0 && count == p.n_modes) ? p.d_order : nullptr;
    const float2 *fac = reinterpret_cast<const float2 *>(p.d_fac_h32);
    const int R = p.R_h;
#define SHEN_CASE(RR)                                                                         \
    case RR:                                                                                  \
        return dfres ? launch_helm_mixed_R<RR, true>(p, order, m0, count, f, u, fac, s)       \
                     : launch_helm_mixed_R<RR, false>(p, order, m0, count, f, u, fac, s);
    switch (R) {
        SHEN_CASE(1) SHEN_CASE(2) SHEN_CASE(4) SHEN_CASE(8) SHEN_CASE(16) SHEN_CASE(24) SHEN_CASE(32)
    default: return cudaErrorInvalidValue;
    }
#undef SHEN_CASE
}

}  // namespace shen
