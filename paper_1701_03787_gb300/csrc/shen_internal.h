// Internal declarations shared by the library's translation units (not installed).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <vector>
#include <cuda_runtime.h>
#include "../../include/shensolve.h"

namespace shen {

constexpr double kPi = 3.14159265358979323846;

// Per-N row tables, indexed by the Chebyshev index k of the basis function
// (Table tab:matrices, Eqs. N_Q, pk, rk; stiffness with the + sign).  Device copies.
struct RowTables {
    // Dirichlet space, k = 0 .. N-3
    const double *bd0;   // B_kk = pi/2 (c_k + 1); B_{k,k+-2} = -pi/2
    const double *ad0;   // A_kk = -2 pi (k+1)(k+2)
    const double *adt;   // A_kj = -4 pi (k+1) for j = k+2, k+4, ...
    // biharmonic space, k = 0 .. N-5 (B symmetric)
    const double *bb0, *bb2, *bb4;   // B_kk, B_{k,k+2}, B_{k,k+4}
    const double *ab0, *abp, *abm;   // A_kk, A_{k,k+2}, A_{k,k-2}
    const double *qb0;               // Q_kk
    const double *pk, *rk, *qk, *sk; // Q_kj = p_k q_j + r_k s_j (j = k+2, k+4, ...)
    // float32 copies for the mixed-precision sweeps
    const float *qk32, *sk32;
};

// Layout of the per-class LU factors (class = one distinct z2).  Chain (class, parity)
// holds rows i = 0 .. rows-1 (Chebyshev index k = 2 i + parity).
//   Helmholtz float64, 4 doubles per row: 1/U_ii, U_i,i+2 tail value (U2), l_i, 0
//       (U_i,i+1 = U2_i - h with h = alpha pi / 2; l_i = L_{i,i-1})
//   biharmonic float64, 8 doubles per row: L1 = L_{i,i-1}, L2 = L_{i,i-2}, 1/U_ii,
//       U1 = U_{i,i+1}, U2 = U_{i,i+2}, ta, tb (tail U_ij = ta_i q_j + tb_i s_j,
//       j >= i+3; Eq. ab), 0
constexpr int kHelmF64 = 4;
constexpr int kDfShapes = 4;   // shapes of the single-plan float-float sweeps (0, 1: thread per
                               // chain; 2, 3: lane per real chain, y on chip, with / without TMEM)
constexpr int kBiF64 = 8;

// Double-double per-N tables of the refinement residual (precision SHEN_FP64_R1), each
// N + 8 entries (hi, lo) indexed by the Chebyshev index k: Dirichlet B_kk, A_kk, A_tail,
// B_{k,k+-2} (entry 0 only); biharmonic B_kk, B_{k,k+2}, B_{k,k+4}, A_kk, A_{k,k+2},
// A_{k,k-2}, Q_kk, p_k, r_k, q_k, s_k.
enum {
    kDdHb0, kDdHa0, kDdHat, kDdHboff,
    kDdBb0, kDdBb2, kDdBb4, kDdBa0, kDdBap, kDdBam, kDdBq0, kDdBp, kDdBr, kDdBq, kDdBs,
    kDdTables
};

struct Plan {
    int N = 0;
    long n_modes = 0, n_classes = 0;
    double nu = 0, dt = 0, c = 0;
    int rows_h = 0, rows_b = 0;           // max rows per parity chain
    // device arrays
    double *d_class_z2 = nullptr;         // [n_classes]
    int *d_mode_class = nullptr;          // [n_modes]
    int *d_order = nullptr;               // [n_modes] modes sorted by class
    double *d_tab = nullptr;              // backing store of RowTables
    float *d_tab32 = nullptr;
    RowTables tab{};
    double *d_fac_h = nullptr;            // Helmholtz factors
    double *d_fac_b = nullptr;            // biharmonic factors
    float *d_fac_h32 = nullptr, *d_fac_b32 = nullptr;
    int *d_err = nullptr;                 // [4]: flag, first bad class, chains with a bad pivot,
                                          //      a transform column copy that did not complete
    unsigned long long *d_resmax = nullptr;   // largest relative residual of the last shen_residual (bits)
    int R_h = 0;                          // rows per lane (at 16 lanes) of the fused Helmholtz kernels
    float *d_fac_df = nullptr;            // backing store of the float-float factor streams below
    // float-float factor streams, row i of chain ch = 2 class + parity at [i * 2 n_classes + ch]
    const float4 *df_hb = nullptr, *df_bf = nullptr, *df_bb0 = nullptr, *df_bb1 = nullptr;
    const float2 *df_hf = nullptr, *df_bb2 = nullptr;
    const float4 *df_qs = nullptr;        // per-N (q_k, s_k), N + 8 entries
    float *d_mv_df = nullptr;             // float-float row tables of the rhs_matvec operators
    float *d_vel_df = nullptr;            // float-float per-N table of the velocity recovery
    float4 *d_vel_ys = nullptr;           // its spill scratch, [warp slot][row][lane]
    int vel_grid = 0;                     // its fixed grid of resident blocks
    // wall-normal transforms (power-of-two N, Gauss points): per-N tables, launch shape
    float4 *d_tr = nullptr;
    int tr_stride = 0, tr_ntw = 0, tr_G = 1;
    float tr_ls[2][3][2] = {};   // forward phi / psi: (rho, kappa, tau) per parity, float-float pairs
    int tr_groups[3][3] = {}, tr_smem[3][3] = {}, tr_grid[3][3] = {};   // per (kind, space)
    // grid of the modes (plans from shen_plan_create; zero for explicit z2 lists)
    int grid_Nx = 0, grid_Nz = 0;
    double grid_Lx = 0, grid_Lz = 0;
    // autotuned choices per problem (SHEN_HELMHOLTZ, SHEN_BIHARMONIC): the path SHEN_AUTO
    // runs, and the row-block shape of the float-float kernels
    bool df_only = false;                 // SHEN_PLAN_DF_ONLY: float64 factors freed after conversion
    bool gl = false;                      // SHEN_PLAN_GL: Gauss-Lobatto scalar product
    bool wall_first = false;              // SHEN_PLAN_WALL_FIRST: fields stored Chebyshev-index-major
    // float-float kernels: fixed grid of resident blocks per [problem][shape], and the
    // per-problem spill scratch of the forward result, [warp slot][chain row][lane]
    int df_grid[2][2] = {{0, 0}, {0, 0}};   // shapes 0 and 1
    int f32_grid[2] = {0, 0};             // float32 sweeps of shen_solve_refine
    float4 *d_ys[2] = {nullptr, nullptr};
    int auto_prec[2] = {5, 5};            // SHEN_DF until tuned
    int df_variant[2] = {0, 0};

    const double2 *d_dd = nullptr;        // double-double residual tables (kDdTables x (N + 8))
    // on-chip float-float sweeps (shapes 2 and 3): one CTA per SM, per-problem global spill of
    // the forward results that do not fit on chip ([warp slot][block][row][lane] float2)
    int df2_grid = 0;
    float2 *d_gsp[2] = {nullptr, nullptr};
    double2 *d_wf_stage = nullptr;        // wall-first plans: staging of the transforms (wallfirst.cu)

    long long device_bytes = 0;
};

// kernels_fp64.cu
cudaError_t launch_factor_helmholtz(const Plan &p, cudaStream_t s);
cudaError_t launch_factor_biharmonic(const Plan &p, cudaStream_t s);
cudaError_t launch_solve_fp64(const Plan &p, int problem, long m0, long count, const double *f,
                              double *u, cudaStream_t s);
cudaError_t launch_matvec_fp64(const Plan &p, int problem, const double *x, const double *y,
                               double beta, double *out, cudaStream_t s, double sign = 1.0);   // sign R x + beta y

// kernels_fp64r.cu
void build_dd_tables(int N, bool gl, std::vector<double2> &T);
cudaError_t launch_solve_fp64r(const Plan &p, int problem, long m0, long count, const double *f, double *u,
                               cudaStream_t s);   // float64 sweeps + one double-double-residual step

// kernels_df2.cu
cudaError_t df2_setup(Plan &p, long long &bytes);
cudaError_t df2_alloc(Plan &p);                 // the spill of shapes 2 and 3 (on first use)
cudaError_t launch_solve_df2(const Plan &p, int problem, bool tmem, long m0, long count, const double *f,
                             double *u, cudaStream_t s);

// kernels_helm_mixed.cu
int helm_mixed_R(int N);                       // rows per lane for N (0: unsupported)
cudaError_t pack_helm_f32(const Plan &p, int R, float2 *out, cudaStream_t s);
cudaError_t launch_helm_mixed(const Plan &p, bool dfres, long m0, long count, const double *f, double *u,
                              cudaStream_t s);

// kernels_df.cu
size_t df_table_floats(const Plan &p);
cudaError_t pack_df(Plan &p, cudaStream_t s);
cudaError_t launch_solve_df(const Plan &p, int problem, long m0, long count, const double *f, double *u,
                            cudaStream_t s);
cudaError_t df_setup(Plan &p, long long &bytes);   // grids and spill scratch of the float-float kernels
cudaError_t launch_solve_f32(const Plan &p, int problem, bool acc, const double *rhs, double *u,
                             cudaStream_t s);   // u = H^-1 rhs, or u += H^-1 rhs (acc), float32 sweeps

// velocity.cu
void build_velocity_table(int N, std::vector<float4> &T, bool gl);
cudaError_t launch_velocity_df(const Plan &p, const double *u, const double *g, double *v, double *w, double *f,
                               cudaStream_t s);
cudaError_t velocity_setup(Plan &p, long long &bytes);   // grid and spill scratch of the velocity kernel

// transform.cu
bool transform_supported(const Plan &p);
bool transform_shape_ok(const Plan &p, int kind, int space);   // the launch fits on this GPU
cudaError_t transform_setup(Plan &p, long long &bytes, cudaStream_t s);   // tables and launch shape
cudaError_t launch_transform(const Plan &p, int kind, int space, long count, const double *in, double *out,
                             cudaStream_t s);   // count columns from in / out

// wallfirst.cu
long wall_first_chunk(const Plan &p);
cudaError_t wall_first_setup(Plan &p, long long &bytes);
cudaError_t launch_transform_wall_first(const Plan &p, int kind, int space, long count, const double *in,
                                        double *out, cudaStream_t s);

// matvec_df.cu
size_t matvec_df_floats(const Plan &p);
cudaError_t pack_matvec_df(const Plan &p, float *T, cudaStream_t s);
cudaError_t launch_matvec_df(const Plan &p, int problem, const double *x, const double *y, double beta,
                             double *out, cudaStream_t s);
cudaError_t launch_matvec_neg_df(const Plan &p, int problem, const double *x, const double *y, double beta,
                                 double *out, cudaStream_t s);   // out = -R x + beta y
cudaError_t launch_mass_df(const Plan &p, int problem, const double *x, const double *y, double beta, double *out,
                           cudaStream_t s);
cudaError_t launch_residual_df(const Plan &p, int problem, const double *f, const double *u, double *rel,
                               cudaStream_t s);

}  // namespace shen

namespace shen {
struct HostPipe;
void host_pipe_free(HostPipe *h);
long long host_pipe_bytes(const HostPipe *h);
cudaError_t host_solve(Plan &p, HostPipe *&h, int problem, int precision, const double *f_host, double *u_host,
                       cudaStream_t user);
}  // namespace shen

struct shen_plan_s {
    shen::Plan p;
    shen::HostPipe *host = nullptr;   // staging for solves on host fields (created on first use)
};
