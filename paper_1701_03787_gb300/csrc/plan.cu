// Plan construction and the C ABI of libshensolve.
//
// A plan holds, for one channel (N, Fourier grid, nu, dt): the per-N row tables of
// the Galerkin matrices (Table tab:matrices, Eqs. N_Q, pk, rk of arXiv:1701.03787),
// the grouping of modes by z2 (modes with equal z2 have equal systems), and the
// float64 LU factors of the Helmholtz and biharmonic systems of every distinct z2,
// computed once on the device (Alg. NS: LU decompositions before the time loop).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <utility>
#include <vector>

#include "shen_internal.h"

using namespace shen;

namespace {

#define SHEN_CUDA_TRY(expr)                                \
    do {                                                   \
        cudaError_t e_ = (expr);                           \
        if (e_ != cudaSuccess) {                           \
            (void)cudaGetLastError();                      \
            return e_ == cudaErrorMemoryAllocation ? SHEN_ERR_ALLOC : SHEN_ERR_CUDA; \
        }                                                  \
    } while (0)

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

}  // namespace

namespace shen {
// Row tables of the Galerkin matrices for N Chebyshev modes (Chebyshev-Gauss scalar
// product, so c_0 = 2 and c_k = 1 for k > 0 including k = N - 1).
// gl: Chebyshev-Gauss-Lobatto scalar product, c_{N-1} = 2 in the mass matrices' highest
// rows (Table tab:matrices: the c_{k+2} term of B_D, the c_{k+4} term of B_B).
void build_row_tables(int N, std::vector<double> &h, std::vector<float> &h32, int &stride, bool gl) {
    const double pi = kPi;
    stride = N;
    h.assign((size_t)16 * N, 0.0);
    h32.assign((size_t)2 * N, 0.0f);
    double *bd0 = &h[0 * N], *ad0 = &h[1 * N], *adt = &h[2 * N];
    double *bb0 = &h[3 * N], *bb2 = &h[4 * N], *bb4 = &h[5 * N];
    double *ab0 = &h[6 * N], *abp = &h[7 * N], *abm = &h[8 * N], *qb0 = &h[9 * N];
    double *pk = &h[10 * N], *rk = &h[11 * N], *qk = &h[12 * N], *sk = &h[13 * N];
    for (int k = 0; k < N; k++) {
        const double K = k, ck = (k == 0) ? 2.0 : 1.0;
        const double ck2 = (gl && k + 2 == N - 1) ? 2.0 : 1.0, ck4 = (gl && k + 4 == N - 1) ? 2.0 : 1.0;
        // Dirichlet phi_k = T_k - T_{k+2}: B_kk = pi/2 (c_k + c_{k+2}); A = (phi_j'', phi_k)
        bd0[k] = pi / 2 * (ck + ck2);
        ad0[k] = -2 * pi * (K + 1) * (K + 2);
        adt[k] = -4 * pi * (K + 1);
        // biharmonic psi_k: B (Table tab:matrices), A = (psi_j'', psi_k), Q (Eqs. N_Q, pk, rk)
        const double r2 = (K + 2) / (K + 3), r1 = (K + 1) / (K + 3);
        bb0[k] = pi / 2 * (ck + 4 * r2 * r2 + ck4 * r1 * r1);
        bb2[k] = -pi * (r2 + (K + 4) * (K + 1) / ((K + 5) * (K + 3)));
        bb4[k] = pi / 2 * r1;
        ab0[k] = -4 * pi * (K + 1) * (K + 2) * (K + 2) / (K + 3);
        abp[k] = 2 * pi * (K + 1) * (K + 2);
        abm[k] = 2 * pi * (K - 1) * (K + 2);
        qb0[k] = 8 * pi * (K + 1) * (K + 1) * (K + 2) * (K + 4);
        pk[k] = 8 * pi * K * (K + 1) * (K + 2) * (K + 4);
        rk[k] = 24 * pi * (K + 1) * (K + 2);
        qk[k] = 1.0 / (K + 3);
        sk[k] = (K + 2) * (K + 2) / (K + 3);
        h32[k] = (float)qk[k];
        h32[N + k] = (float)sk[k];
    }
}
}  // namespace shen

namespace {

void free_plan(Plan &p) {
    cudaFree(p.d_class_z2);
    cudaFree(p.d_mode_class);
    cudaFree(p.d_order);
    cudaFree(p.d_tab);
    cudaFree(p.d_tab32);
    cudaFree(p.d_fac_h);
    cudaFree(p.d_fac_b);
    cudaFree(p.d_fac_h32);
    cudaFree(p.d_fac_b32);
    cudaFree(p.d_err);
    cudaFree(p.d_resmax);
    cudaFree(p.d_fac_df);
    cudaFree(p.d_mv_df);
    cudaFree(p.d_vel_df);
    cudaFree(p.d_vel_ys);
    cudaFree(p.d_tr);
    cudaFree(p.d_ys[0]);
    cudaFree(p.d_ys[1]);
    cudaFree((void *)p.d_dd);
    cudaFree(p.d_gsp[0]);
    cudaFree(p.d_gsp[1]);
    cudaFree(p.d_wf_stage);
    p = Plan{};
}

template <class T>
cudaError_t dalloc(T **ptr, size_t count, long long &bytes) {
    bytes += (long long)(count * sizeof(T));
    return cudaMalloc((void **)ptr, count * sizeof(T));
}

shen_status create_from_z2(shen_plan_t *out, int N, long n_modes, const double *z2, double nu, double dt,
                           unsigned flags, void *stream) {
    if (!out) return SHEN_ERR_ARG;
    *out = nullptr;
    if ((flags & ~(SHEN_PLAN_DF_ONLY | SHEN_PLAN_GL | SHEN_PLAN_WALL_FIRST)) != 0 || N < 8 || N > 8192 ||
        n_modes < 1 ||
        n_modes > (1L << 30) || !z2)
        return SHEN_ERR_ARG;
    if (!(nu > 0) || !(dt > 0) || !std::isfinite(nu) || !std::isfinite(dt)) return SHEN_ERR_ARG;
    const double c = 2.0 / (nu * dt);
    if (!std::isfinite(c)) return SHEN_ERR_ARG;
    for (long m = 0; m < n_modes; m++)
        if (!(z2[m] >= 0) || !std::isfinite(z2[m])) return SHEN_ERR_ARG;

    // group modes by z2
    std::vector<std::pair<double, int>> srt((size_t)n_modes);
    for (long m = 0; m < n_modes; m++) srt[m] = {z2[m], (int)m};
    std::sort(srt.begin(), srt.end());
    std::vector<int> order((size_t)n_modes), mode_class((size_t)n_modes);
    std::vector<double> class_z2;
    for (long w = 0; w < n_modes; w++) {
        if (w == 0 || srt[w].first != srt[w - 1].first) class_z2.push_back(srt[w].first);
        order[w] = srt[w].second;
        mode_class[srt[w].second] = (int)class_z2.size() - 1;
    }
    {
        // Number the classes in order of first appearance in the mode order, and visit
        // the modes by class: same-class modes stay side by side (one set of factor rows
        // per warp lane group) while both the field columns and the factor rows are
        // walked nearly in address order.  (Visiting the modes in z2 order instead
        // scatters each warp's columns over the whole field and costs up to 2x in the
        // serial sweeps.)
        const long nc = (long)class_z2.size();
        std::vector<int> renum((size_t)nc, -1), count((size_t)nc + 1, 0);
        int next = 0;
        for (long m = 0; m < n_modes; m++) {
            int &r = renum[mode_class[m]];
            if (r < 0) r = next++;
        }
        std::vector<double> cz((size_t)nc);
        for (long c = 0; c < nc; c++) cz[renum[c]] = class_z2[c];
        class_z2.swap(cz);
        for (long m = 0; m < n_modes; m++) {
            mode_class[m] = renum[mode_class[m]];
            count[mode_class[m] + 1]++;
        }
        for (long c = 0; c < nc; c++) count[c + 1] += count[c];
        for (long m = 0; m < n_modes; m++) order[count[mode_class[m]]++] = (int)m;
    }

    shen_plan_s *plan = new (std::nothrow) shen_plan_s;
    if (!plan) return SHEN_ERR_ALLOC;
    Plan &p = plan->p;
    p.N = N;
    p.n_modes = n_modes;
    p.n_classes = (long)class_z2.size();
    p.nu = nu;
    p.dt = dt;
    p.c = c;
    p.rows_h = (N - 2 + 1) / 2;
    p.rows_b = (N - 4 + 1) / 2;

    std::vector<double> tab;
    std::vector<float> tab32;
    int stride = 0;
    const bool gl = (flags & SHEN_PLAN_GL) != 0;
    p.gl = gl;
    p.wall_first = (flags & SHEN_PLAN_WALL_FIRST) != 0;
    build_row_tables(N, tab, tab32, stride, gl);

    cudaStream_t s = as_stream(stream);
    auto fail = [&](shen_status st) {
        free_plan(p);
        delete plan;
        return st;
    };
#define PLAN_TRY(expr)                                                                   \
    do {                                                                                 \
        cudaError_t e_ = (expr);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            (void)cudaGetLastError();                                                    \
            return fail(e_ == cudaErrorMemoryAllocation ? SHEN_ERR_ALLOC : SHEN_ERR_CUDA); \
        }                                                                                \
    } while (0)
    long long &B = p.device_bytes;
    PLAN_TRY(dalloc(&p.d_class_z2, (size_t)p.n_classes, B));
    PLAN_TRY(dalloc(&p.d_mode_class, (size_t)n_modes, B));
    PLAN_TRY(dalloc(&p.d_order, (size_t)n_modes, B));
    PLAN_TRY(dalloc(&p.d_tab, tab.size(), B));
    PLAN_TRY(dalloc(&p.d_tab32, tab32.size(), B));
    PLAN_TRY(dalloc(&p.d_fac_h, (size_t)p.n_classes * 2 * p.rows_h * kHelmF64, B));
    PLAN_TRY(dalloc(&p.d_fac_b, (size_t)p.n_classes * 2 * p.rows_b * kBiF64, B));
    PLAN_TRY(dalloc(&p.d_err, 4, B));
    PLAN_TRY(dalloc(&p.d_resmax, 1, B));
    PLAN_TRY(cudaMemsetAsync(p.d_resmax, 0, sizeof(unsigned long long), s));

    PLAN_TRY(cudaMemcpyAsync(p.d_class_z2, class_z2.data(), class_z2.size() * sizeof(double),
                             cudaMemcpyHostToDevice, s));
    PLAN_TRY(cudaMemcpyAsync(p.d_mode_class, mode_class.data(), mode_class.size() * sizeof(int),
                             cudaMemcpyHostToDevice, s));
    PLAN_TRY(cudaMemcpyAsync(p.d_order, order.data(), order.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    PLAN_TRY(cudaMemcpyAsync(p.d_tab, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    PLAN_TRY(cudaMemcpyAsync(p.d_tab32, tab32.data(), tab32.size() * sizeof(float), cudaMemcpyHostToDevice, s));
    const int err_init[4] = {0, 0x7fffffff, 0, 0};
    PLAN_TRY(cudaMemcpyAsync(p.d_err, err_init, sizeof(err_init), cudaMemcpyHostToDevice, s));
    const double *t = p.d_tab;
    p.tab.bd0 = t + 0 * stride; p.tab.ad0 = t + 1 * stride; p.tab.adt = t + 2 * stride;
    p.tab.bb0 = t + 3 * stride; p.tab.bb2 = t + 4 * stride; p.tab.bb4 = t + 5 * stride;
    p.tab.ab0 = t + 6 * stride; p.tab.abp = t + 7 * stride; p.tab.abm = t + 8 * stride;
    p.tab.qb0 = t + 9 * stride; p.tab.pk = t + 10 * stride; p.tab.rk = t + 11 * stride;
    p.tab.qk = t + 12 * stride; p.tab.sk = t + 13 * stride;
    p.tab.qk32 = p.d_tab32; p.tab.sk32 = p.d_tab32 + stride;

    PLAN_TRY(launch_factor_helmholtz(p, s));
    PLAN_TRY(launch_factor_biharmonic(p, s));
    // float-float copies of the factors for the float-float sweeps
    PLAN_TRY(dalloc(&p.d_fac_df, df_table_floats(p), B));
    PLAN_TRY(pack_df(p, s));
    PLAN_TRY(df_setup(p, B));
    PLAN_TRY(df2_setup(p, B));
    PLAN_TRY(dalloc(&p.d_mv_df, matvec_df_floats(p), B));
    PLAN_TRY(pack_matvec_df(p, p.d_mv_df, s));
    std::vector<float4> vel;
    build_velocity_table(N, vel, gl);
    PLAN_TRY(dalloc(&p.d_vel_df, vel.size() * 4, B));
    PLAN_TRY(cudaMemcpyAsync(p.d_vel_df, vel.data(), vel.size() * sizeof(float4), cudaMemcpyHostToDevice, s));
    PLAN_TRY(velocity_setup(p, B));
    PLAN_TRY(transform_setup(p, B, s));
    PLAN_TRY(wall_first_setup(p, B));
    {
        std::vector<double2> dd;
        build_dd_tables(N, gl, dd);
        double2 *d = nullptr;
        PLAN_TRY(dalloc(&d, dd.size(), B));
        p.d_dd = d;
        PLAN_TRY(cudaMemcpyAsync(d, dd.data(), dd.size() * sizeof(double2), cudaMemcpyHostToDevice, s));
    }
    // float32 factors in the lane layout of the fused Helmholtz refinement kernels
    p.df_only = (flags & SHEN_PLAN_DF_ONLY) != 0;
    p.R_h = p.df_only ? 0 : helm_mixed_R(N);
    if (p.R_h > 0) {
        PLAN_TRY(dalloc(&p.d_fac_h32, (size_t)p.n_classes * 2 * p.R_h * 16 * 2, B));
        PLAN_TRY(pack_helm_f32(p, p.R_h, reinterpret_cast<float2 *>(p.d_fac_h32), s));
    }

    int err_host[2];
    PLAN_TRY(cudaMemcpyAsync(err_host, p.d_err, sizeof(err_host), cudaMemcpyDeviceToHost, s));
    PLAN_TRY(cudaStreamSynchronize(s));
    if (err_host[0]) return fail(SHEN_ERR_SINGULAR);
    if (p.df_only) {                     // the float-float tables are built: drop the float64 ones
        cudaFree(p.d_fac_h);
        cudaFree(p.d_fac_b);
        p.d_fac_h = p.d_fac_b = nullptr;
        B -= (long long)sizeof(double) * p.n_classes * 2 * ((long long)p.rows_h * kHelmF64 + (long long)p.rows_b * kBiF64);
    }
#undef PLAN_TRY
    *out = plan;
    return SHEN_OK;
}

bool aligned16(const void *ptr) { return (reinterpret_cast<uintptr_t>(ptr) & 15u) == 0; }

// Input and output ranges either coincide (in place) or are disjoint.
bool overlap_ok(const double *a, const double *b, long n_doubles) {
    if (!a || !b || a == b) return true;
    const double *ae = a + n_doubles, *be = b + n_doubles;
    return ae <= b || be <= a;
}

shen_status check_precision(const Plan &p, int problem, int precision) {
    if (precision == SHEN_FP64_R1)        // float64 factors, mode-major fields
        return (p.df_only || p.wall_first) ? SHEN_ERR_UNSUPPORTED : SHEN_OK;
    if (p.df_only && precision != SHEN_DF)
        return precision >= SHEN_FP64 && precision <= SHEN_DF ? SHEN_ERR_UNSUPPORTED : SHEN_ERR_ARG;
    if (p.wall_first && precision != SHEN_DF && precision != SHEN_FP64)   // mixed kernels: mode-major only
        return precision >= SHEN_FP64 && precision <= SHEN_DF ? SHEN_ERR_UNSUPPORTED : SHEN_ERR_ARG;
    if (precision == SHEN_FP64 || precision == SHEN_DF) return SHEN_OK;
    if (precision < SHEN_FP32_R1 || precision > SHEN_DF_R2) return SHEN_ERR_ARG;
    const bool r1 = precision == SHEN_FP32_R1 || precision == SHEN_DF_R1;
    if (problem == SHEN_HELMHOLTZ && r1 && p.R_h > 0) return SHEN_OK;

    return SHEN_ERR_UNSUPPORTED;
}

}  // namespace

namespace shen {
// Enqueue the kernel of (problem, precision) for modes [m0, m0 + count).
cudaError_t launch_solve_range(const Plan &p, int problem, int precision, long m0, long count, const double *f,
                               double *u, cudaStream_t s) {
    if (precision == SHEN_FP64) return launch_solve_fp64(p, problem, m0, count, f, u, s);
    if (precision == SHEN_DF) return launch_solve_df(p, problem, m0, count, f, u, s);
    if (precision == SHEN_FP64_R1) return launch_solve_fp64r(p, problem, m0, count, f, u, s);
    return launch_helm_mixed(p, precision == SHEN_DF_R1, m0, count, f, u, s);
}
}  // namespace shen

namespace {

shen_status solve_range(shen_plan_t plan, int problem, long m0, long count, const double *f, double *u,
                        int precision, void *stream) {
    if (!plan) return SHEN_ERR_ARG;
    const Plan &p = plan->p;
    if (problem != SHEN_HELMHOLTZ && problem != SHEN_BIHARMONIC) return SHEN_ERR_ARG;
    if (m0 < 0 || count < 0 || m0 + count > p.n_modes) return SHEN_ERR_ARG;
    if (precision == SHEN_AUTO) precision = p.auto_prec[problem];
    shen_status ps = check_precision(p, problem, precision);
    if (ps != SHEN_OK) return ps;
    if (count == 0) return SHEN_OK;                          // an empty range: f, u are not read
    if (!f || !u) return SHEN_ERR_ARG;
    if (!aligned16(f) || !aligned16(u)) return SHEN_ERR_ARG;
    if (!overlap_ok(f, u, 2 * count * (long)p.N)) return SHEN_ERR_ARG;
    SHEN_CUDA_TRY(launch_solve_range(p, problem, precision, m0, count, f, u, as_stream(stream)));
    return SHEN_OK;
}

}  // namespace

extern "C" {

shen_status shen_plan_create(shen_plan_t *plan, int N, int Nx, int Nz, double nu, double dt, double Lx,
                             double Lz, unsigned flags, void *stream) {
    if (!plan) return SHEN_ERR_ARG;
    *plan = nullptr;
    if (Nx < 2 || Nz < 2 || (Nx & 1) || (Nz & 1)) return SHEN_ERR_ARG;
    if (!(Lx > 0) || !(Lz > 0) || !std::isfinite(Lx) || !std::isfinite(Lz)) return SHEN_ERR_ARG;
    const long nxh = Nx / 2 + 1;
    const long n_modes = nxh * (long)Nz;
    if (n_modes > (1L << 30)) return SHEN_ERR_ARG;
    std::vector<double> z2((size_t)n_modes);
    for (long ix = 0; ix < nxh; ix++) {
        const double kx = 2 * kPi * (double)ix / Lx;
        for (long iz = 0; iz < Nz; iz++) {
            const long kzi = iz < Nz / 2 ? iz : iz - Nz;
            const double kz = 2 * kPi * (double)kzi / Lz;
            z2[ix * Nz + iz] = kx * kx + kz * kz;
        }
    }
    const shen_status st = create_from_z2(plan, N, n_modes, z2.data(), nu, dt, flags, stream);
    if (st == SHEN_OK) {
        Plan &p = (*plan)->p;
        p.grid_Nx = Nx;
        p.grid_Nz = Nz;
        p.grid_Lx = Lx;
        p.grid_Lz = Lz;
    }
    return st;
}

shen_status shen_plan_create_z2(shen_plan_t *plan, int N, long n_modes, const double *z2_host, double nu,
                                double dt, unsigned flags, void *stream) {
    return create_from_z2(plan, N, n_modes, z2_host, nu, dt, flags, stream);
}

shen_status shen_helmholtz_solve(shen_plan_t plan, const double *f, double *u, int precision, void *stream) {
    if (!plan) return SHEN_ERR_ARG;
    return solve_range(plan, SHEN_HELMHOLTZ, 0, plan->p.n_modes, f, u, precision, stream);
}

shen_status shen_biharmonic_solve(shen_plan_t plan, const double *f, double *u, int precision, void *stream) {
    if (!plan) return SHEN_ERR_ARG;
    return solve_range(plan, SHEN_BIHARMONIC, 0, plan->p.n_modes, f, u, precision, stream);
}

shen_status shen_solve_modes(shen_plan_t plan, int problem, long mode_begin, long mode_count, const double *f,
                             double *u, int precision, void *stream) {
    return solve_range(plan, problem, mode_begin, mode_count, f, u, precision, stream);
}

shen_status shen_rhs_matvec_ex(shen_plan_t plan, int problem, const double *x, const double *y, double beta,
                               double *out, int precision, void *stream) {
    if (precision == SHEN_AUTO) precision = SHEN_DF;
    if (precision != SHEN_FP64 && precision != SHEN_DF)
        return precision >= SHEN_FP32_R1 && precision <= SHEN_DF_R2 ? SHEN_ERR_UNSUPPORTED : SHEN_ERR_ARG;
    if (precision == SHEN_FP64) return shen_rhs_matvec(plan, problem, x, y, beta, out, stream);
    if (!plan || !x || !out) return SHEN_ERR_ARG;
    const Plan &p = plan->p;
    if (problem != SHEN_HELMHOLTZ && problem != SHEN_BIHARMONIC) return SHEN_ERR_ARG;
    if (!aligned16(x) || !aligned16(out) || (y && !aligned16(y))) return SHEN_ERR_ARG;
    const long nd = 2 * p.n_modes * (long)p.N;
    if (x == out || (y && y == out)) return SHEN_ERR_ARG;
    if (!overlap_ok(x, out, nd) || !overlap_ok(y, out, nd)) return SHEN_ERR_ARG;
    if (y && !std::isfinite(beta)) return SHEN_ERR_ARG;
    SHEN_CUDA_TRY(launch_matvec_df(p, problem, x, y, beta, out, as_stream(stream)));
    return SHEN_OK;
}

shen_status shen_velocity(shen_plan_t plan, const double *u, const double *g, double *v, double *w, double *f,
                          int precision, void *stream) {
    if (!plan || !u || !g || !v || !w) return SHEN_ERR_ARG;
    if (precision == SHEN_AUTO) precision = SHEN_DF;
    if (precision != SHEN_DF)
        return precision >= SHEN_FP64 && precision <= SHEN_DF ? SHEN_ERR_UNSUPPORTED : SHEN_ERR_ARG;
    const Plan &p = plan->p;
    if (p.grid_Nz <= 0) return SHEN_ERR_UNSUPPORTED;            // explicit z2 list: no (m, n)
    for (const void *q : {(const void *)u, (const void *)g, (const void *)v, (const void *)w, (const void *)f})
        if (q && !aligned16(q)) return SHEN_ERR_ARG;
    const long nd = 2 * p.n_modes * (long)p.N;
    // outputs disjoint from the inputs and from each other
    const double *outs[3] = {v, w, f};
    for (int a = 0; a < 3; a++) {
        if (!outs[a]) continue;
        for (const double *in : {u, g})
            if (outs[a] == in || !overlap_ok(outs[a], in, nd)) return SHEN_ERR_ARG;
        for (int b = a + 1; b < 3; b++)
            if (outs[b] && (outs[a] == outs[b] || !overlap_ok(outs[a], outs[b], nd))) return SHEN_ERR_ARG;
    }
    SHEN_CUDA_TRY(launch_velocity_df(p, u, g, v, w, f, as_stream(stream)));
    return SHEN_OK;
}

shen_status shen_linear_step(shen_plan_t plan, const double *u_old, const double *g_old, const double *load_u,
                             const double *load_g, double *u_new, double *g_new, double *v, double *w,
                             int precision, void *stream) {
    if (!plan || !u_old || !g_old || !u_new || !g_new || !v || !w) return SHEN_ERR_ARG;
    Plan &p = plan->p;
    if (p.grid_Nz <= 0) return SHEN_ERR_UNSUPPORTED;            // the velocity step needs (m, n)
    const long nd = 2 * p.n_modes * (long)p.N;
    // every output disjoint from every input and from the other outputs
    const double *ins[4] = {u_old, g_old, load_u, load_g};
    double *outs[4] = {u_new, g_new, v, w};
    for (int a = 0; a < 4; a++) {
        if (!aligned16(outs[a])) return SHEN_ERR_ARG;
        for (int b = 0; b < 4; b++)
            if (ins[b] && (!aligned16(ins[b]) || outs[a] == ins[b] || !overlap_ok(outs[a], ins[b], nd)))
                return SHEN_ERR_ARG;
        for (int b = a + 1; b < 4; b++)
            if (outs[a] == outs[b] || !overlap_ok(outs[a], outs[b], nd)) return SHEN_ERR_ARG;
    }
    int ph = precision == SHEN_AUTO ? p.auto_prec[SHEN_HELMHOLTZ] : precision;
    int pb = precision == SHEN_AUTO ? p.auto_prec[SHEN_BIHARMONIC] : precision;
    shen_status st = check_precision(p, SHEN_HELMHOLTZ, ph);
    if (st == SHEN_OK) st = check_precision(p, SHEN_BIHARMONIC, pb);
    if (st != SHEN_OK) return st;
    // Scaled Crank-Nicolson steps (Eqs. gfin, ufin; the solves' H_h = (2/(nu dt)) Hbar,
    // H_b = -(2/(nu dt)) Hchk, the operators' R = (2/(nu dt)) x paper right-hand side):
    //   H_h g_new = R_h g_old + (2/nu) load_g,   H_b u_new = -R_b u_old - (2/nu) load_u
    const double load_scale = 2.0 / p.nu;
    cudaStream_t s = as_stream(stream);
    // right-hand sides into the new fields (float-float operators unless float64 was asked)
    auto rhs = [&](int problem, const double *x, const double *load, double *out) {
        const double sg = problem == SHEN_BIHARMONIC ? -1.0 : 1.0;
        if (precision == SHEN_FP64 || precision == SHEN_FP64_R1)
            return launch_matvec_fp64(p, problem, x, load, sg * load_scale, out, s, sg);
        return sg > 0 ? launch_matvec_df(p, problem, x, load, load_scale, out, s)
                      : launch_matvec_neg_df(p, problem, x, load, -load_scale, out, s);
    };
    SHEN_CUDA_TRY(rhs(SHEN_BIHARMONIC, u_old, load_u, u_new));
    SHEN_CUDA_TRY(launch_solve_range(p, SHEN_BIHARMONIC, pb, 0, p.n_modes, u_new, u_new, s));
    SHEN_CUDA_TRY(rhs(SHEN_HELMHOLTZ, g_old, load_g, g_new));
    SHEN_CUDA_TRY(launch_solve_range(p, SHEN_HELMHOLTZ, ph, 0, p.n_modes, g_new, g_new, s));
    SHEN_CUDA_TRY(launch_velocity_df(p, u_new, g_new, v, w, nullptr, s));
    return SHEN_OK;
}

shen_status shen_mass_matvec(shen_plan_t plan, int problem, const double *x, const double *y, double beta,
                             double *out, void *stream) {
    if (!plan || !x || !out) return SHEN_ERR_ARG;
    const Plan &p = plan->p;
    if (problem != SHEN_HELMHOLTZ && problem != SHEN_BIHARMONIC) return SHEN_ERR_ARG;
    if (!aligned16(x) || !aligned16(out) || (y && !aligned16(y))) return SHEN_ERR_ARG;
    const long nd = 2 * p.n_modes * (long)p.N;
    if (x == out || (y && y == out)) return SHEN_ERR_ARG;
    if (!overlap_ok(x, out, nd) || !overlap_ok(y, out, nd)) return SHEN_ERR_ARG;
    if (y && !std::isfinite(beta)) return SHEN_ERR_ARG;
    SHEN_CUDA_TRY(launch_mass_df(p, problem, x, y, beta, out, as_stream(stream)));
    return SHEN_OK;
}

shen_status shen_transform(shen_plan_t plan, int kind, int space, const double *in, double *out, void *stream) {
    if (!plan || !in || !out) return SHEN_ERR_ARG;
    if (kind < SHEN_TRANSFORM_INVERSE || kind > SHEN_TRANSFORM_FORWARD) return SHEN_ERR_ARG;
    if (space < SHEN_SPACE_CHEBYSHEV || space > SHEN_SPACE_BIHARMONIC) return SHEN_ERR_ARG;
    const Plan &p = plan->p;
    if (!aligned16(in) || !aligned16(out)) return SHEN_ERR_ARG;
    if (!overlap_ok(in, out, 2 * p.n_modes * (long)p.N)) return SHEN_ERR_ARG;
    if (!transform_supported(p) || !transform_shape_ok(p, kind, space)) return SHEN_ERR_UNSUPPORTED;
    if (p.wall_first)
        SHEN_CUDA_TRY(launch_transform_wall_first(p, kind, space, p.n_modes, in, out, as_stream(stream)));
    else
        SHEN_CUDA_TRY(launch_transform(p, kind, space, p.n_modes, in, out, as_stream(stream)));
    return SHEN_OK;
}

shen_status shen_transform_modes(shen_plan_t plan, int kind, int space, long mode_begin, long mode_count,
                                 const double *in, double *out, void *stream) {
    if (!plan) return SHEN_ERR_ARG;
    if (kind < SHEN_TRANSFORM_INVERSE || kind > SHEN_TRANSFORM_FORWARD) return SHEN_ERR_ARG;
    if (space < SHEN_SPACE_CHEBYSHEV || space > SHEN_SPACE_BIHARMONIC) return SHEN_ERR_ARG;
    const Plan &p = plan->p;
    if (mode_begin < 0 || mode_count < 0 || mode_begin + mode_count > p.n_modes) return SHEN_ERR_ARG;
    if (!transform_supported(p) || !transform_shape_ok(p, kind, space)) return SHEN_ERR_UNSUPPORTED;
    if (mode_count == 0) return SHEN_OK;                     // an empty range: in, out are not read
    if (!in || !out) return SHEN_ERR_ARG;
    if (!aligned16(in) || !aligned16(out)) return SHEN_ERR_ARG;
    // the range's elements span (N - 1) n_modes + mode_count complex values on a wall-first
    // plan (in, out point at element (mode_begin, 0)), mode_count N on a mode-major one
    const long span = p.wall_first ? (long)(p.N - 1) * p.n_modes + mode_count : mode_count * (long)p.N;
    if (!overlap_ok(in, out, 2 * span)) return SHEN_ERR_ARG;
    if (p.wall_first)
        SHEN_CUDA_TRY(launch_transform_wall_first(p, kind, space, mode_count, in, out, as_stream(stream)));
    else
        SHEN_CUDA_TRY(launch_transform(p, kind, space, mode_count, in, out, as_stream(stream)));
    return SHEN_OK;
}

shen_status shen_residual(shen_plan_t plan, int problem, const double *f, const double *u, double *rel,
                          void *stream) {
    if (!plan || !f || !u) return SHEN_ERR_ARG;
    if (problem != SHEN_HELMHOLTZ && problem != SHEN_BIHARMONIC) return SHEN_ERR_ARG;
    if (!aligned16(f) || !aligned16(u) || (rel && (reinterpret_cast<uintptr_t>(rel) & 7u))) return SHEN_ERR_ARG;
    SHEN_CUDA_TRY(launch_residual_df(plan->p, problem, f, u, rel, as_stream(stream)));
    return SHEN_OK;
}

shen_status shen_last_error_detail(shen_plan_t plan, double *max_rel_residual, long *n_singular) {
    if (!plan) return SHEN_ERR_ARG;
    int err_host[4];
    unsigned long long bits = 0;
    SHEN_CUDA_TRY(cudaMemcpy(err_host, plan->p.d_err, sizeof(err_host), cudaMemcpyDeviceToHost));
    SHEN_CUDA_TRY(cudaMemcpy(&bits, plan->p.d_resmax, sizeof(bits), cudaMemcpyDeviceToHost));
    if (max_rel_residual) {
        double v;
        std::memcpy(&v, &bits, sizeof(v));
        *max_rel_residual = v;
    }
    if (n_singular) *n_singular = err_host[2];
    return SHEN_OK;
}

shen_status shen_rhs_matvec(shen_plan_t plan, int problem, const double *x, const double *y, double beta,
                            double *out, void *stream) {
    if (!plan || !x || !out) return SHEN_ERR_ARG;
    const Plan &p = plan->p;
    if (problem != SHEN_HELMHOLTZ && problem != SHEN_BIHARMONIC) return SHEN_ERR_ARG;
    if (!aligned16(x) || !aligned16(out) || (y && !aligned16(y))) return SHEN_ERR_ARG;
    const long nd = 2 * p.n_modes * (long)p.N;
    if (x == out || (y && y == out)) return SHEN_ERR_ARG;
    if (!overlap_ok(x, out, nd) || !overlap_ok(y, out, nd)) return SHEN_ERR_ARG;
    if (y && !std::isfinite(beta)) return SHEN_ERR_ARG;
    SHEN_CUDA_TRY(launch_matvec_fp64(p, problem, x, y, beta, out, as_stream(stream)));
    return SHEN_OK;
}

shen_status shen_plan_info(shen_plan_t plan, long *n_modes, long *n_classes, long *N, long long *device_bytes) {
    if (!plan) return SHEN_ERR_ARG;
    if (n_modes) *n_modes = plan->p.n_modes;
    if (n_classes) *n_classes = plan->p.n_classes;
    if (N) *N = plan->p.N;
    if (device_bytes) *device_bytes = plan->p.device_bytes + host_pipe_bytes(plan->host);
    return SHEN_OK;
}

shen_status shen_plan_check(shen_plan_t plan, long *where) {
    if (!plan) return SHEN_ERR_ARG;
    int err_host[4];
    SHEN_CUDA_TRY(cudaMemcpy(err_host, plan->p.d_err, sizeof(err_host), cudaMemcpyDeviceToHost));
    if (where) *where = err_host[0] ? err_host[1] : -1;
    if (err_host[0]) return SHEN_ERR_SINGULAR;
    return err_host[3] ? SHEN_ERR_CUDA : SHEN_OK;
}

void shen_plan_destroy(shen_plan_t plan) {
    if (!plan) return;
    host_pipe_free(plan->host);
    free_plan(plan->p);
    delete plan;
}

shen_status shen_solve_host(shen_plan_t plan, int problem, const double *f_host, double *u_host, int precision,
                            void *stream) {
    if (!plan || !f_host || !u_host) return SHEN_ERR_ARG;
    if (plan->p.wall_first) return SHEN_ERR_UNSUPPORTED;   // mode-major fields only
    if (problem != SHEN_HELMHOLTZ && problem != SHEN_BIHARMONIC) return SHEN_ERR_ARG;
    const long nd = 2 * plan->p.n_modes * (long)plan->p.N;
    if (!overlap_ok(f_host, u_host, nd)) return SHEN_ERR_ARG;
    if (precision == SHEN_AUTO) precision = plan->p.auto_prec[problem];
    const shen_status ps = check_precision(plan->p, problem, precision);
    if (ps != SHEN_OK) return ps;
    SHEN_CUDA_TRY(host_solve(plan->p, plan->host, problem, precision, f_host, u_host, as_stream(stream)));
    return SHEN_OK;
}

shen_status shen_plan_autotune(shen_plan_t plan, int problem, const double *f, double *u, int *chosen, float *ms,
                               void *stream) {
    if (!plan || !f || !u) return SHEN_ERR_ARG;
    if (problem != SHEN_HELMHOLTZ && problem != SHEN_BIHARMONIC) return SHEN_ERR_ARG;
    Plan &p = plan->p;
    const long nd = 2 * p.n_modes * (long)p.N;
    if (!aligned16(f) || !aligned16(u) || f == u || !overlap_ok(f, u, nd)) return SHEN_ERR_ARG;
    struct Cand {
        int prec, variant;
    };
    std::vector<Cand> cands;
    if (!p.wall_first) SHEN_CUDA_TRY(df2_alloc(p));           // shapes 2, 3 are candidates
    for (Cand c : {Cand{SHEN_FP64, 0}, Cand{SHEN_DF, 0}, Cand{SHEN_DF, 1}, Cand{SHEN_DF, 2}, Cand{SHEN_DF, 3},
                   Cand{SHEN_DF_R1, 0}, Cand{SHEN_FP32_R1, 0}})
        if (check_precision(p, problem, c.prec) == SHEN_OK && !(c.variant >= 2 && p.wall_first))
            cands.push_back(c);
    cudaStream_t s = as_stream(stream);
    cudaEvent_t ev[4];
    for (int i = 0; i < 4; i++)
        if (cudaEventCreate(&ev[i]) != cudaSuccess) {
            for (int j = 0; j < i; j++) cudaEventDestroy(ev[j]);
            (void)cudaGetLastError();
            return SHEN_ERR_CUDA;
        }
    const int v0 = p.df_variant[problem];
    float best = 0.f, best_df = 0.f;
    Cand pick{SHEN_DF, v0};
    int pick_df = v0;
    cudaError_t e = cudaSuccess;
    for (const Cand &c : cands) {
        p.df_variant[problem] = c.variant;
        // one untimed solve, then the median of three timed ones
        e = launch_solve_range(p, problem, c.prec, 0, p.n_modes, f, u, s);
        float t[3] = {0.f, 0.f, 0.f};
        for (int r = 0; r < 3 && e == cudaSuccess; r++) {
            e = cudaEventRecord(ev[0], s);
            if (e == cudaSuccess) e = launch_solve_range(p, problem, c.prec, 0, p.n_modes, f, u, s);
            if (e == cudaSuccess) e = cudaEventRecord(ev[1], s);
            if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&t[r], ev[0], ev[1]);
        }
        if (e != cudaSuccess) break;
        std::sort(t, t + 3);
        if (best == 0.f || t[1] < best) {
            best = t[1];
            pick = c;
        }
        if (c.prec == SHEN_DF && (best_df == 0.f || t[1] < best_df)) {
            best_df = t[1];
            pick_df = c.variant;
        }
    }
    for (int i = 0; i < 4; i++) cudaEventDestroy(ev[i]);
    if (e != cudaSuccess) {
        p.df_variant[problem] = v0;
        (void)cudaGetLastError();
        return SHEN_ERR_CUDA;
    }
    // the faster float-float shape serves every float-float solve of this problem
    p.auto_prec[problem] = pick.prec;
    p.df_variant[problem] = pick_df;
    if (chosen) *chosen = pick.prec;
    if (ms) *ms = best;
    return SHEN_OK;
}

shen_status shen_solve_refine(shen_plan_t plan, int problem, const double *f, double *u, double *work, int steps,
                              int residual, void *stream) {
    if (!plan || !f || !u || !work) return SHEN_ERR_ARG;
    if (problem != SHEN_HELMHOLTZ && problem != SHEN_BIHARMONIC) return SHEN_ERR_ARG;
    if (steps < 0 || steps > 2) return SHEN_ERR_ARG;
    if (residual != SHEN_FP64 && residual != SHEN_DF) return SHEN_ERR_ARG;
    const Plan &p = plan->p;
    if (p.wall_first) return SHEN_ERR_UNSUPPORTED;   // mode-major fields only
    for (const void *q : {(const void *)f, (const void *)u, (const void *)work})
        if (!aligned16(q)) return SHEN_ERR_ARG;
    const long nd = 2 * p.n_modes * (long)p.N;
    // f is read at every step: u and work must not overlap it or each other
    if (u == f || work == f || work == u || !overlap_ok(u, f, nd) || !overlap_ok(work, f, nd) ||
        !overlap_ok(work, u, nd))
        return SHEN_ERR_ARG;
    cudaStream_t s = as_stream(stream);
    SHEN_CUDA_TRY(launch_solve_f32(p, problem, false, f, u, s));
    // r = f - H u through the right-hand-side operators with c -> -c:
    // H_h = -R_h(-c) and H_b = R_b(-c) (same matrices, the time-step sign flipped)
    Plan q = p;
    q.c = -p.c;
    for (int step = 0; step < steps; step++) {
        if (residual == SHEN_DF) {
            if (problem == SHEN_HELMHOLTZ) SHEN_CUDA_TRY(launch_matvec_df(q, problem, u, f, 1.0, work, s));
            else SHEN_CUDA_TRY(launch_matvec_neg_df(q, problem, u, f, 1.0, work, s));
        } else {
            SHEN_CUDA_TRY(launch_matvec_fp64(q, problem, u, f, 1.0, work, s, problem == SHEN_HELMHOLTZ ? 1.0 : -1.0));
        }
        SHEN_CUDA_TRY(launch_solve_f32(p, problem, true, work, u, s));
    }
    return SHEN_OK;
}

shen_status shen_plan_set_shape(shen_plan_t plan, int problem, int shape) {
    if (!plan) return SHEN_ERR_ARG;
    if (problem != SHEN_HELMHOLTZ && problem != SHEN_BIHARMONIC) return SHEN_ERR_ARG;
    if (shape < 0 || shape >= kDfShapes) return SHEN_ERR_ARG;
    if (shape >= 2 && plan->p.wall_first) return SHEN_ERR_UNSUPPORTED;   // mode-major fields only
    if (shape >= 2) SHEN_CUDA_TRY(df2_alloc(plan->p));
    plan->p.df_variant[problem] = shape;
    return SHEN_OK;
}

shen_status shen_plan_get_shape(shen_plan_t plan, int problem, int *shape) {
    if (!plan || !shape) return SHEN_ERR_ARG;
    if (problem != SHEN_HELMHOLTZ && problem != SHEN_BIHARMONIC) return SHEN_ERR_ARG;
    *shape = plan->p.df_variant[problem];
    return SHEN_OK;
}

const char *shen_status_string(int status) {
    switch (status) {
    case SHEN_OK: return "ok";
    case SHEN_ERR_ARG: return "invalid argument";
    case SHEN_ERR_ALLOC: return "allocation failed";
    case SHEN_ERR_CUDA: return "CUDA error";
    case SHEN_ERR_SINGULAR: return "zero or non-finite pivot";
    case SHEN_ERR_UNSUPPORTED: return "unsupported request";
    default: return "unknown status";
    }
}

int shen_version(void) { return 100; }

}  // extern "C"
