// Helmholtz solve with float32 sweeps and one step of iterative refinement
// (Sec. 4 algorithm of arXiv:1701.03787; the refinement is this library's precision
// scheme):
//
//   u0 = H^-1 f     float32 forward elimination + back substitution with the float64
//                   LU factors rounded to float32
//   r  = f - H u0   residual: float-float (DF variant) or float64 (F64 variant)
//   d  = H^-1 r     float32 sweeps again
//   u  = u0 + d     float-float / float64, written as float64
//
// Work decomposition: L lanes per parity chain (k = 2 i + parity).  L = 16: one warp per
// mode, lanes 0-15 on the even chain and 16-31 on the odd one; L = 32: one warp per
// (mode, parity), the two warps of a block on the two parities of one mode.  Lane s of a
// chain owns rows s R .. s R + R - 1 of it, held in registers.  The sweeps are linear
// recurrences along each chain: every lane runs its R rows with a zero carry, the L
// lanes of a chain combine their maps with a shuffle scan (scalar affine maps for the forward sweep, 2x2 maps
// for the back substitution whose state is (u_i, sum_{j >= i} u_j)), and each lane
// then adds the carried part.
//
// Helmholtz system per parity (k = 2i + p, alpha = z2 + c, h = alpha pi / 2):
//   H_{i,i-1} = -h,  H_ii = pi (alpha delta_k + 2 (k+1)(k+2)),
//   H_{i,i+1} = -h + 4 pi (k+1),  H_{i,j>i+1} = 4 pi (k+1),  delta_k = (c_k + c_{k+2}) / 2.
//   LU: y_i = f_i + g_i y_{i-1} (g_i = h / U_{i-1,i-1}),
//   u_i = (y_i + h u_{i+1} - U2_i S_{i+1}) / U_ii,  S_{i+1} = sum_{j > i} u_j.
#include "df.cuh"
#include "shen_internal.h"

namespace shen {
namespace {

constexpr float kPiHi = 3.14159274101257324f;           // float(pi)
constexpr float kPiLo = -8.74227765734758577e-08f;      // pi - float(pi)
constexpr unsigned kFull = 0xffffffffu;

// One complex row of f with a 256-byte L2 fetch size: a lane reads its segment of the
// column row by row, so one miss brings its next rows into L2 (9.39 -> 9.25 ms for the
// float-float-residual kernel at N = 1024, 1024 x 1024).  u is written only after the
// warp's last read of f; with 32 lanes per chain the two warps of a mode (one per parity)
// touch disjoint rows.
__device__ __forceinline__ double2 ld_f(const double2 *p) {
    double2 v;
    asm volatile("ld.global.L2::256B.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "l"(p));
    return v;
}
// chains of at least this many rows per lane at 16 lanes run on 32 lanes
#ifndef SHEN_MIXED_L32_MIN
#define SHEN_MIXED_L32_MIN 16
#endif
constexpr int kMixedL32Min = SHEN_MIXED_L32_MIN;

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// Forward elimination y_i = f_i + g_i y_{i-1}, in place in w.  gs: [j][lane] shared.
template <int R, int L>
__device__ __forceinline__ void forward_sweep(float2 (&w)[R], const float *gs, int lane, int s) {
    float2 y = f2(0.f, 0.f);
    float G = 1.f;
#pragma unroll
    for (int j = 0; j < R; j++) {
        const float g = gs[j * 32 + lane];
        y.x = fmaf(g, y.x, w[j].x);
        y.y = fmaf(g, y.y, w[j].y);
        w[j] = y;
        G *= g;
    }
#pragma unroll
    for (int d = 1; d < L; d <<= 1) {
        const float Gu = __shfl_up_sync(kFull, G, d, L);
        const float Yx = __shfl_up_sync(kFull, y.x, d, L);
        const float Yy = __shfl_up_sync(kFull, y.y, d, L);
        if (s >= d) {
            y.x = fmaf(G, Yx, y.x);
            y.y = fmaf(G, Yy, y.y);
            G *= Gu;
        }
    }
    float cx = __shfl_up_sync(kFull, y.x, 1, L), cy = __shfl_up_sync(kFull, y.y, 1, L);
    if (s == 0) cx = cy = 0.f;
    float P = 1.f;
#pragma unroll
    for (int j = 0; j < R; j++) {
        P *= gs[j * 32 + lane];
        w[j].x = fmaf(P, cx, w[j].x);
        w[j].y = fmaf(P, cy, w[j].y);
    }
}

// Back substitution, in place in w (y in, u out).  Per row a = h inv0, c = U2 inv0:
//   u_i = a u_{i+1} - c S_{i+1} + inv0 y_i,  S_i = S_{i+1} + u_i.
// With FIRST, m0 ([j][lane] shared) receives row 0 of the lane-local transfer matrices
// (response of u_i to the carried state); otherwise the stored rows are reused.
template <int R, int L, bool FIRST>
__device__ __forceinline__ void backward_sweep(float2 (&w)[R], const float2 *fac, int lane, int s, float h,
                                               float2 *m0) {
    float2 u = f2(0.f, 0.f), S = f2(0.f, 0.f);
    float t00 = 1.f, t01 = 0.f, t10 = 0.f, t11 = 1.f;
#pragma unroll
    for (int j = R - 1; j >= 0; j--) {
        const float2 fu = fac[j * L];                   // (inv0, U2) of row s R + j
        const float a = h * fu.x, c = fu.y * fu.x;
        float2 un;
        un.x = fmaf(a, u.x, fmaf(-c, S.x, fu.x * w[j].x));
        un.y = fmaf(a, u.y, fmaf(-c, S.y, fu.x * w[j].y));
        S.x += un.x;
        S.y += un.y;
        u = un;
        w[j] = un;
        const float n00 = fmaf(a, t00, -c * t10), n01 = fmaf(a, t01, -c * t11);
        t10 += n00;
        t11 += n01;
        t00 = n00;
        t01 = n01;
        if (FIRST) m0[j * 32 + lane] = f2(n00, n01);
    }
    // suffix scan over the L lanes of the chain of the maps x -> T x + v, v = (u, S)
#pragma unroll
    for (int d = 1; d < L; d <<= 1) {
        const float b00 = __shfl_down_sync(kFull, t00, d, L), b01 = __shfl_down_sync(kFull, t01, d, L);
        const float b10 = __shfl_down_sync(kFull, t10, d, L), b11 = __shfl_down_sync(kFull, t11, d, L);
        const float wux = __shfl_down_sync(kFull, u.x, d, L), wuy = __shfl_down_sync(kFull, u.y, d, L);
        const float wSx = __shfl_down_sync(kFull, S.x, d, L), wSy = __shfl_down_sync(kFull, S.y, d, L);
        if (s + d < L) {
            u.x = fmaf(t00, wux, fmaf(t01, wSx, u.x));
            u.y = fmaf(t00, wuy, fmaf(t01, wSy, u.y));
            S.x = fmaf(t10, wux, fmaf(t11, wSx, S.x));
            S.y = fmaf(t10, wuy, fmaf(t11, wSy, S.y));
            const float n00 = fmaf(t00, b00, t01 * b10), n01 = fmaf(t00, b01, t01 * b11);
            const float n10 = fmaf(t10, b00, t11 * b10), n11 = fmaf(t10, b01, t11 * b11);
            t00 = n00; t01 = n01; t10 = n10; t11 = n11;
        }
    }
    float cux = __shfl_down_sync(kFull, u.x, 1, L), cuy = __shfl_down_sync(kFull, u.y, 1, L);
    float cSx = __shfl_down_sync(kFull, S.x, 1, L), cSy = __shfl_down_sync(kFull, S.y, 1, L);
    if (s == L - 1) cux = cuy = cSx = cSy = 0.f;
#pragma unroll
    for (int j = 0; j < R; j++) {
        const float2 m = m0[j * 32 + lane];
        w[j].x = fmaf(m.x, cux, fmaf(m.y, cSx, w[j].x));
        w[j].y = fmaf(m.x, cuy, fmaf(m.y, cSy, w[j].y));
    }
}

// Residual r = f - H u0 for the lane's rows, rounded to float32 into rs ([j][lane]
// shared).  u0s ([j][lane] shared) holds u0 (exact float32 values).  H / pi, row i:
//   E_i = alpha (delta_k u_i - (u_{i-1} + u_{i+1}) / 2) + 2(k+1)(k+2) u_i + 4(k+1) sum_{j>i} u_j
//   r_i = f_i - pi E_i.
// The row loop is kept rolled (its body is long) so the kernel stays small.
template <int R, int L, bool DF>
__device__ __forceinline__ void residual(float2 *rs, const float2 *u0s, const double *fcol, int lane, int s,
                                         int p, int n, double alpha, int k_gl) {
    const df::F2 a_df = df::from_f64(alpha);
    const df::F2 pi_df = {kPiHi, kPiLo};
    // lane totals of u0, then the sum over the lanes above (rows with larger i)
    float tre = 0.f, tim = 0.f, ere = 0.f, eim = 0.f;
    double dre = 0.0, dim = 0.0;
#pragma unroll 4
    for (int j = 0; j < R; j++) {
        const float2 uv = u0s[j * 32 + lane];
        if (DF) {
            df::F2 q = df::two_sum(tre, uv.x); tre = q.hi; ere += q.lo;
            q = df::two_sum(tim, uv.y); tim = q.hi; eim += q.lo;
        } else {
            dre += (double)uv.x;
            dim += (double)uv.y;
        }
    }
#pragma unroll
    for (int d = 1; d < L; d <<= 1) {
        if (DF) {
            const float a0 = __shfl_down_sync(kFull, tre, d, L), a1 = __shfl_down_sync(kFull, ere, d, L);
            const float b0 = __shfl_down_sync(kFull, tim, d, L), b1 = __shfl_down_sync(kFull, eim, d, L);
            if (s + d < L) {
                df::F2 q = df::add(df::F2{tre, ere}, df::F2{a0, a1}); tre = q.hi; ere = q.lo;
                q = df::add(df::F2{tim, eim}, df::F2{b0, b1}); tim = q.hi; eim = q.lo;
            }
        } else {
            const double a0 = __shfl_down_sync(kFull, dre, d, L), b0 = __shfl_down_sync(kFull, dim, d, L);
            if (s + d < L) { dre += a0; dim += b0; }
        }
    }
    // running sums over rows above the current row: (hi, unnormalised error)
    float Tre, Tim, Ere, Eim;
    double Dre, Dim;
    {
        float a0 = __shfl_down_sync(kFull, tre, 1, L), a1 = __shfl_down_sync(kFull, ere, 1, L);
        float b0 = __shfl_down_sync(kFull, tim, 1, L), b1 = __shfl_down_sync(kFull, eim, 1, L);
        double da = __shfl_down_sync(kFull, dre, 1, L), db = __shfl_down_sync(kFull, dim, 1, L);
        if (s == L - 1) { a0 = a1 = b0 = b1 = 0.f; da = db = 0.0; }
        Tre = a0; Ere = a1; Tim = b0; Eim = b1;
        Dre = da; Dim = db;
    }
    const float2 top = u0s[(R - 1) * 32 + lane], bot = u0s[lane];
    float2 below = f2(__shfl_up_sync(kFull, top.x, 1, L), __shfl_up_sync(kFull, top.y, 1, L));
    float2 above = f2(__shfl_down_sync(kFull, bot.x, 1, L), __shfl_down_sync(kFull, bot.y, 1, L));
    if (s == 0) below = f2(0.f, 0.f);
    if (s == L - 1) above = f2(0.f, 0.f);
    float2 up = above;
    float2 uc = top;
    // per-class constants: pi alpha / 2 (float-float)
    const df::F2 pih = df::mul(pi_df, df::F2{0.5f * a_df.hi, 0.5f * a_df.lo});
    const int k_top = 2 * (s * R + R - 1) + p;
    double2 fnext = k_top < n ? ld_f(reinterpret_cast<const double2 *>(fcol) + k_top) : make_double2(0.0, 0.0);
#pragma unroll 1
    for (int j = R - 1; j >= 0; j--) {
        const int k = 2 * (s * R + j) + p;
        const double2 fk = fnext;
        if (j > 0 && k - 2 < n) fnext = ld_f(reinterpret_cast<const double2 *>(fcol) + k - 2);   // prefetch
        const float2 um = j > 0 ? u0s[(j - 1) * 32 + lane] : below;
        float2 r = f2(0.f, 0.f);
        if (k < n) {
            // row coefficients times pi (float-float): pi (alpha delta_k + 2(k+1)(k+2)), 4 pi (k+1)
            // delta_k = (c_k + c_{k+2}) / 2; c_{k+2} = c_{N-1} = 2 at Gauss-Lobatto points (k = k_gl)
            const float delta = (k == 0 ? 1.5f : 1.0f) + (k == k_gl ? 0.5f : 0.0f);
            const float e = 2.0f * (float)((k + 1) * (k + 2));
            const float t = 4.0f * (float)(k + 1);
            float rv[2];
            if (DF) {
                const df::F2 D = df::mul(pi_df, df::add(df::mul(a_df, delta), df::two_prod(e, 1.0f)));
                const df::F2 piT = df::two_prod(kPiHi, t);
                const float piTlo = kPiLo * t;
#pragma unroll
                for (int c = 0; c < 2; c++) {
                    const float vm = c ? um.y : um.x, vc = c ? uc.y : uc.x, vp = c ? up.y : up.x;
                    const double fv = c ? fk.y : fk.x;
                    const df::F2 T = df::fast_two_sum(c ? Tim : Tre, c ? Eim : Ere);
                    const df::F2 nb = df::two_sum(vm, vp);                 // u_{i-1} + u_{i+1}
                    const df::F2 p1 = df::mul(D, vc);                      // pi H_ii u_i
                    const df::F2 p2 = df::mul(pih, nb);                    // pi alpha/2 (u_{i-1} + u_{i+1})
                    df::F2 p3 = df::mul(T, piT.hi);                        // 4 pi (k+1) sum_{j>i} u_j
                    p3.lo = __fmaf_rn(T.hi, __fadd_rn(piT.lo, piTlo), p3.lo);
                    const df::F2 fd = df::from_f64(fv);
                    const df::F2 s1 = df::two_sum(fd.hi, -p1.hi);
                    const df::F2 s2 = df::two_sum(s1.hi, p2.hi);
                    const df::F2 s3 = df::two_sum(s2.hi, -p3.hi);
                    const float lo = __fadd_rn(__fadd_rn(__fsub_rn(fd.lo, p1.lo), __fsub_rn(p2.lo, p3.lo)),
                                               __fadd_rn(__fadd_rn(s1.lo, s2.lo), s3.lo));
                    rv[c] = __fadd_rn(s3.hi, lo);
                }
            } else {
#pragma unroll
                for (int c = 0; c < 2; c++) {
                    const float vm = c ? um.y : um.x, vc = c ? uc.y : uc.x, vp = c ? up.y : up.x;
                    const double fv = c ? fk.y : fk.x;
                    const double T = c ? Dim : Dre;
                    const double b = (double)delta * vc - 0.5 * ((double)vm + (double)vp);
                    const double E = fma(alpha, b, fma((double)e, (double)vc, (double)t * T));
                    rv[c] = (float)fma(-kPi, E, fv);
                }
            }
            r = f2(rv[0], rv[1]);
        }
        rs[j * 32 + lane] = r;
        if (DF) {
            df::F2 q = df::two_sum(Tre, uc.x); Tre = q.hi; Ere = __fadd_rn(Ere, q.lo);
            q = df::two_sum(Tim, uc.y); Tim = q.hi; Eim = __fadd_rn(Eim, q.lo);
        } else {
            Dre += (double)uc.x;
            Dim += (double)uc.y;
        }
        up = uc;
        uc = um;
    }
}

// Blocks of two warps.  L = 16: a warp per mode (work item); L = 32: a warp per parity
// chain, the block's two warps on one mode.  fac: float32 factors [class][parity][j][s] =
// (inv0, U2), s < L.
template <int R, int L, bool DF>
__global__ void __launch_bounds__(64) helm_mixed_kernel(Plan p, const int *order, long m0, long count,
                                                         const double *f, double *u, const float2 *fac) {
    static_assert(L == 16 || L == 32, "16 or 32 lanes per chain");
    extern __shared__ float2 smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int s = lane & (L - 1);
    const long wid = (long)blockIdx.x * (blockDim.x >> 5) + warp;
    const long item = L == 16 ? wid : wid >> 1;
    const int par = L == 16 ? lane >> 4 : (int)(wid & 1);
    if (item >= count) return;                          // the whole warp leaves together
    const long mode = order ? (long)order[item] : m0 + item;
    const long col = mode - m0;
    const int cls = p.d_mode_class[mode];
    const int N = p.N, n = N - 2;
    const double alpha = p.d_class_z2[cls] + p.c;
    const float h = (float)(alpha * kPi / 2);
    float2 *m0buf = smem + (size_t)warp * (5 * R * 16);            // [R][32] transfer rows / r
    float2 *u0buf = m0buf + R * 32;                                 // [R][32] u0
    float *gbuf = reinterpret_cast<float *>(u0buf + R * 32);        // [R][32] g
    const double *fcol = f + 2 * col * N;
    double *ucol = u + 2 * col * N;
    const float2 *F = fac + ((size_t)cls * 2 + par) * R * L + s;   // row s R + j at F[j * L]

    float2 w[R];
#pragma unroll
    for (int j = 0; j < R; j++) {
        const int i = s * R + j, k = 2 * i + par;
        if (k < n) {
            const double2 fk = ld_f(reinterpret_cast<const double2 *>(fcol) + k);
            if (DF) w[j] = f2(df::hi_f64(fk.x), df::hi_f64(fk.y));
            else w[j] = f2((float)fk.x, (float)fk.y);
        } else {
            w[j] = f2(0.f, 0.f);
        }
        float prev = 0.f;                               // 1/U of row i-1
        if (i > 0) prev = j > 0 ? F[(j - 1) * L].x : F[(R - 1) * L - 1].x;
        gbuf[j * 32 + lane] = h * prev;
    }
    __syncwarp();
    forward_sweep<R, L>(w, gbuf, lane, s);
    backward_sweep<R, L, true>(w, F, lane, s, h, m0buf);
#pragma unroll
    for (int j = 0; j < R; j++) u0buf[j * 32 + lane] = w[j];
    __syncwarp();
    residual<R, L, DF>(m0buf, u0buf, fcol, lane, s, par, n, alpha, p.gl ? n - 1 : -1);
    __syncwarp();
#pragma unroll
    for (int j = 0; j < R; j++) w[j] = m0buf[j * 32 + lane];
    __syncwarp();
    forward_sweep<R, L>(w, gbuf, lane, s);
    backward_sweep<R, L, true>(w, F, lane, s, h, m0buf);
#pragma unroll
    for (int j = 0; j < R; j++) {
        const int k = 2 * (s * R + j) + par;
        if (k < N) {
            double2 out = make_double2(0.0, 0.0);
            if (k < n) {
                const float2 a = u0buf[j * 32 + lane];
                if (DF) {   // exact widening of both terms, one float64 add (correctly rounded)
                    out.x = __dadd_rn(df::f32_to_f64_bits(a.x), df::f32_to_f64_bits(w[j].x));
                    out.y = __dadd_rn(df::f32_to_f64_bits(a.y), df::f32_to_f64_bits(w[j].y));
                } else {
                    out.x = (double)a.x + (double)w[j].x;
                    out.y = (double)a.y + (double)w[j].y;
                }
            }
            reinterpret_cast<double2 *>(ucol)[k] = out;
        }
    }
    // trailing entries beyond the lanes' reach (at most 2, since N - 2 <= 2 L R)
    if (s == 0 && par == 0)
        for (int k = max(n, 2 * L * R); k < N; k++) reinterpret_cast<double2 *>(ucol)[k] = make_double2(0.0, 0.0);
}

// float64 factors -> float32 table in the lane layout: row i = s R + j of chain
// (class, parity) goes to [class][parity][j][s], s < L.
__global__ void pack_helm_f32_kernel(Plan p, int R, int L, float2 *out) {
    const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    const long total = p.n_classes * 2 * (long)R * L;
    if (t >= total) return;
    const int s = (int)(t % L);
    const int j = (int)((t / L) % R);
    const long chain = t / ((long)L * R);              // class * 2 + parity
    const int i = s * R + j;
    float2 v = make_float2(0.f, 0.f);
    if (i < p.rows_h) {
        const double *row = p.d_fac_h + (chain * p.rows_h + i) * kHelmF64;
        v = make_float2((float)row[0], (float)row[1]);   // 1/U_ii, U2
    }
    out[t] = v;
}

template <int R, int L, bool DF>
cudaError_t launch_helm_mixed_R(const Plan &p, const int *order, long m0, long count, const double *f, double *u,
                                const float2 *fac, cudaStream_t st) {
    const int warps = 2;
    // per warp: transfer rows and u0 ([R][32] float2 each) and g ([R][32] float)
    const size_t smem = (size_t)warps * 5 * R * 16 * sizeof(float2);
    auto kern = helm_mixed_kernel<R, L, DF>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const long per_block = L == 16 ? warps : 1;          // modes per block
    const unsigned blocks = (unsigned)((count + per_block - 1) / per_block);
    kern<<<blocks, warps * 32, smem, st>>>(p, order, m0, count, f, u, fac);
    return cudaGetLastError();
}

}  // namespace

// Rows per lane of the fused Helmholtz refinement kernels, counted at 16 lanes per parity
// chain (R16; chains of more than 128 rows then run on 32 lanes with R16 / 2 rows each).
int helm_mixed_R(int N) {
    const int rows = (N - 2 + 1) / 2;
    const int R = (rows + 15) / 16;
    if (N > 2048) return 0;
    if (R <= 2) return 2;
    if (R <= 4) return 4;
    if (R <= 8) return 8;
    if (R <= 16) return 16;
    if (R <= 24) return 24;
    if (R <= 32) return 32;
    if (R <= 48) return 48;
    if (R <= 64) return 64;
    return 0;
}

// Lanes per chain for R16 rows per lane at 16 lanes: chains of more than 128 rows take a
// whole warp each (R16 / 2 rows per lane), which halves the registers and shared memory a
// warp holds (N = 1024: 168 -> 118 registers, 11.85 -> 9.39 ms for the 1024 x 1024 grid).
static int mixed_lanes(int R16) { return R16 >= kMixedL32Min ? 32 : 16; }

cudaError_t pack_helm_f32(const Plan &p, int R16, float2 *out, cudaStream_t s) {
    const int L = mixed_lanes(R16), R = R16 * 16 / L;
    const long total = p.n_classes * 2 * (long)R * L;
    pack_helm_f32_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(p, R, L, out);
    return cudaGetLastError();
}

cudaError_t launch_helm_mixed(const Plan &p, bool dfres, long m0, long count, const double *f, double *u,
                              cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    const int *order = (m0 == 0 && count == p.n_modes) ? p.d_order : nullptr;
    const float2 *fac = reinterpret_cast<const float2 *>(p.d_fac_h32);
#define SHEN_CASE(RR, LL)                                                                              \
    case RR:                                                                                           \
        return dfres ? launch_helm_mixed_R<RR * 16 / LL, LL, true>(p, order, m0, count, f, u, fac, s)  \
                     : launch_helm_mixed_R<RR * 16 / LL, LL, false>(p, order, m0, count, f, u, fac, s);
    if (mixed_lanes(p.R_h) == 16) {
        switch (p.R_h) {
            SHEN_CASE(2, 16) SHEN_CASE(4, 16) SHEN_CASE(8, 16) SHEN_CASE(16, 16) SHEN_CASE(24, 16)
            SHEN_CASE(32, 16) SHEN_CASE(48, 16) SHEN_CASE(64, 16)
        default: return cudaErrorInvalidValue;
        }
    }
    switch (p.R_h) {
        SHEN_CASE(16, 32) SHEN_CASE(24, 32) SHEN_CASE(32, 32) SHEN_CASE(48, 32) SHEN_CASE(64, 32)
    default: return cudaErrorInvalidValue;
    }
#undef SHEN_CASE
}

}  // namespace shen
