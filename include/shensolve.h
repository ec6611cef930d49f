/*
 * shensolve -- batched Shen-Galerkin wall-normal solves on NVIDIA GB300 (sm_103a).
 *
 * C ABI.  Every pointer argument is a plain pointer; every size is in elements.
 * Nothing here depends on PyTorch or any other framework.
 *
 * The operations (Mortensen, "A spectral-Galerkin turbulent channel flow solver for
 * large-scale simulations", arXiv:1701.03787):
 *
 *   For every Fourier mode (kx, kz) of a wall-normal resolution of N Chebyshev modes
 *   (N = N_x + 1 in the paper's notation), with z2 = (2 pi kx / Lx)^2 + (2 pi kz / Lz)^2
 *   and c = 2 / (nu dt):
 *
 *   Helmholtz  (Sec. 3, Eqs. gfin, Helmholtz_matrix):  (alpha B - A) u = f,
 *       alpha = z2 + c, Shen Dirichlet basis phi_k = T_k - T_{k+2} (Sec. 2, Eq. phiD),
 *       B = (phi_j, phi_k), A = (phi_j'', phi_k); N - 2 unknowns.  This is the paper's
 *       Hbar scaled by 2 / (nu dt).
 *   Biharmonic (Sec. 3, Eqs. ufin, Biharmonic_matrix):  (Q + a A + b B) u = f,
 *       a = -(2 z2 + c), b = z2 (z2 + c), Shen biharmonic basis (Sec. 2, Eq. phiN),
 *       Q = (psi_j'''', psi_k) (Eqs. N_Q, pk, rk); N - 4 unknowns.  This is the paper's
 *       Hchk scaled by -2 / (nu dt).
 *   Right-hand-side operators (Eqs. gfin, ufin, scaled by 2 / (nu dt)):
 *       Helmholtz  R_h = (c - z2) B + A            (= 2 Bbar - Hbar)
 *       biharmonic R_b = Q + (c - 2 z2) A + z2 (z2 - c) B   (= 2 Achk - 2 z2 Bchk - Hchk)
 *   Scalar products are Chebyshev-Gauss (Sec. 2); stiffness matrices carry the sign
 *   A = +(phi'', phi) under which Eqs. ufin / gfin discretise the PDEs.
 *
 *   The solves use the paper's O(N) direct algorithms (Sec. 4): odd/even decoupling,
 *   LU without pivoting, U rows with three stored values plus the constant tail
 *   (Helmholtz) or the a_k q_j + b_k s_j tail of Eq. ab (biharmonic; Algorithms
 *   LUbiharmonic, ReduceAB, LUSolveBiharmonic).  Factorisation happens once, in
 *   shen_plan_create (the paper's "compute LU decompositions" before the time loop).
 *
 * Data layout ("mode-major"): a field is n_modes columns of N complex values, each
 * complex value two doubles (re, im) interleaved; element (m, k) is at
 * [2 * (m * N + k)].  Mode index m = ix * Nz + iz, ix = 0 .. Nx/2 (kx = ix),
 * iz = 0 .. Nz-1 (kz = iz for iz < Nz/2, else iz - Nz).  Input entries k >= N-2
 * (Helmholtz) or k >= N-4 (biharmonic) are ignored; the same output entries are
 * written as 0.  Field pointers are DEVICE pointers unless a function says HOST,
 * must be 16-byte aligned, and stay owned by the caller.  u == f (in place) is
 * allowed; any other overlap between input and output is an error.
 *
 * Asynchrony: calls enqueue work on `stream` (a cudaStream_t passed as void*;
 * NULL = the legacy default stream) and return once it is enqueued.  The status
 * reports argument and launch errors; device-side conditions (a zero pivot) are
 * recorded in the plan and returned by shen_plan_check after the stream is synced.
 *
 * Errors: no function throws; a failed call leaves the plan valid.
 */
#ifndef SHENSOLVE_H
#define SHENSOLVE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct shen_plan_s *shen_plan_t;

typedef enum {
    SHEN_OK = 0,
    SHEN_ERR_ARG = 1,          /* invalid argument (size, pointer, alignment, overlap) */
    SHEN_ERR_ALLOC = 2,        /* device or host allocation failed */
    SHEN_ERR_CUDA = 3,         /* a CUDA call or kernel launch failed */
    SHEN_ERR_SINGULAR = 4,     /* a zero or non-finite pivot was met in a factorisation */
    SHEN_ERR_UNSUPPORTED = 5   /* valid request the library does not implement */
} shen_status;

typedef enum { SHEN_HELMHOLTZ = 0, SHEN_BIHARMONIC = 1 } shen_problem;

/* Plan creation flags. */
#define SHEN_PLAN_DF_ONLY 1u   /* keep only the float-float factor tables (shen_plan_create) */
#define SHEN_PLAN_GL 2u        /* Chebyshev-Gauss-Lobatto scalar product (Sec. 2): the GL point sum,
                                  i.e. c_{N_x} = 2 in the mass matrices' highest rows (Table
                                  tab:matrices); default Chebyshev-Gauss.  Single and batched plans. */
#define SHEN_PLAN_WALL_FIRST 4u /* fields stored wall-index-first, the paper's uhat(l, m, n) order (Sec. 2):
                                  element (m, k) at complex index k * n_modes + m, so each Chebyshev
                                  index k holds all modes contiguously.  Supported by the solves
                                  (SHEN_FP64, SHEN_DF shapes 0 and 1, SHEN_AUTO resolving to them;
                                  shen_solve_modes with f, u pointing at element (mode_begin, 0) of
                                  the full field), the operators (shen_rhs_matvec, _ex,
                                  shen_mass_matvec, shen_residual), shen_velocity, shen_linear_step
                                  and the transforms (shen_transform, and shen_transform_modes with
                                  in, out pointing at element (mode_begin, 0)): each gives the
                                  transpose of the mode-major result bit for bit.  The transforms
                                  go through a chunked transpose into 128 MB of plan-owned staging.
                                  shen_solve_host, shen_solve_refine, SHEN_FP64_R1 and the
                                  float32-sweep precisions return SHEN_ERR_UNSUPPORTED on such a
                                  plan.  Single plans (shen_plan_create / _z2) only. */

/* Arithmetic of a solve.  All variants read and write float64 (complex128) fields and
 * use the same float64 LU factors (built once per plan); they differ in how the
 * sweeps run:
 *   SHEN_FP64       forward elimination and back substitution in float64 (the
 *                   paper's algorithm as printed).
 *   SHEN_FP32_R1 /  sweeps in float32 with the factors rounded to float32, then
 *   SHEN_FP32_R2    1 / 2 steps of iterative refinement whose residual r = f - H u
 *                   and correction u += d are computed in float64.
 *   SHEN_DF_R1 /    as SHEN_FP32_R*, but the residual and the correction use
 *   SHEN_DF_R2      float-float arithmetic (pairs of float32, error-free
 *                   transformations of Dekker and Knuth) instead of float64.
 *   SHEN_DF         forward elimination and back substitution themselves in
 *                   float-float arithmetic (~48 significant bits) with the factors
 *                   as float-float pairs; no refinement.
 *   SHEN_AUTO       the path recorded for the plan and problem by shen_plan_autotune
 *                   / shen_batch_autotune (SHEN_DF until then).
 *   SHEN_FP64_R1    the float64 sweeps, then one step of iterative refinement whose
 *                   residual r = f - H u is formed in double-double arithmetic (every
 *                   matrix entry, product and sum as an unevaluated pair of float64;
 *                   the entries from exact rationals times pi) and whose correction
 *                   H d = r runs the float64 sweeps again: u += d.  For the systems
 *                   where the unpivoted algorithm's own roundoff reaches ~1e-12
 *                   (Table tab:roundoff: high z, large N) this restores the float64
 *                   solution of the exactly assembled system to ~1e-15.  About 30
 *                   times the cost of SHEN_FP64 on GB300 (float64 runs at 1/64 of the
 *                   float32 rate).  Single-channel plans with their float64 factors
 *                   (not SHEN_PLAN_DF_ONLY) and mode-major fields; u == f allowed.
 * A solve returns SHEN_ERR_UNSUPPORTED for a (problem, precision) pair that is not
 * built: the float32-sweep variants exist for the Helmholtz problem, N <= 2048, one
 * refinement step. */
typedef enum {
    SHEN_FP64 = 0,
    SHEN_FP32_R1 = 1,
    SHEN_FP32_R2 = 2,
    SHEN_DF_R1 = 3,
    SHEN_DF_R2 = 4,
    SHEN_DF = 5,
    SHEN_AUTO = 6,
    SHEN_FP64_R1 = 7
} shen_precision;

/* Create a plan for one channel: N Chebyshev modes (8 <= N <= 8192), Fourier grid
 * Nx x Nz (even, >= 2), viscosity nu > 0, time step dt > 0, box lengths Lx, Lz > 0
 * (the paper's Re_tau = 2000 box is Lx = 2 pi, Lz = pi).  Builds the per-N tables,
 * groups modes by z2 (modes with equal z2 share one factorisation) and computes the
 * float64 LU factors of both systems for every distinct z2 on the device, on
 * `stream`.  Blocks until the plan is ready.  flags: SHEN_PLAN_GL (Gauss-Lobatto
 * points instead of Gauss) and/or SHEN_PLAN_DF_ONLY to keep
 * only the float-float factor tables (about half the device memory: the float64 factors
 * are computed, converted and freed at creation); solves of such a plan accept
 * SHEN_DF and SHEN_AUTO only (others: SHEN_ERR_UNSUPPORTED); shen_rhs_matvec, which
 * uses no factors, is unaffected.
 * Errors: SHEN_ERR_ARG on bad sizes/parameters; SHEN_ERR_ALLOC; SHEN_ERR_CUDA;
 * SHEN_ERR_SINGULAR if a pivot is zero or not finite. */
shen_status shen_plan_create(shen_plan_t *plan, int N, int Nx, int Nz, double nu, double dt,
                             double Lx, double Lz, unsigned flags, void *stream);

/* Same, for an explicit list of n_modes squared wavenumbers z2[] (HOST array,
 * z2 >= 0, finite), in the order the fields store their columns. */
shen_status shen_plan_create_z2(shen_plan_t *plan, int N, long n_modes, const double *z2_host,
                                double nu, double dt, unsigned flags, void *stream);

/* Helmholtz solve (alpha B - A) u = f for every mode of the plan. f, u: DEVICE
 * fields of n_modes * N complex values.
 *
 * Concurrency (all solve entry points of a plan): the float-float sweeps (SHEN_DF, and
 * SHEN_AUTO when it resolves to it) spill their forward results to a scratch the plan
 * holds per problem, so two float-float solves of the SAME problem on one plan must
 * not run at the same time (issue them on one stream, or order the streams).  A
 * Helmholtz and a biharmonic solve may overlap; SHEN_FP64_R1 uses the same scratch (same
 * rule); other precisions use no scratch. */
shen_status shen_helmholtz_solve(shen_plan_t plan, const double *f, double *u, int precision,
                                 void *stream);

/* Biharmonic solve (Q + a A + b B) u = f for every mode of the plan. */
shen_status shen_biharmonic_solve(shen_plan_t plan, const double *f, double *u, int precision,
                                  void *stream);

/* Solve modes [mode_begin, mode_begin + mode_count) only: f and u point at the
 * column of mode_begin (a shard of a larger field).  problem: shen_problem.
 * mode_count = 0 (an empty shard, e.g. more ranks than modes) checks the plan, problem,
 * precision and range, launches nothing and returns SHEN_OK; f and u are not read then
 * and may be NULL. */
shen_status shen_solve_modes(shen_plan_t plan, int problem, long mode_begin, long mode_count,
                             const double *f, double *u, int precision, void *stream);

/* Solve every mode of the plan (problem SHEN_HELMHOLTZ / SHEN_BIHARMONIC) for fields
 * in HOST memory: f_host and u_host hold n_modes * N complex values (u_host == f_host
 * allowed); page-locked (pinned) host memory gives full copy bandwidth, pageable memory
 * works more slowly.  The field is streamed through three plan-owned device staging
 * slots (about 256 MB each, allocated at the first call and counted by
 * shen_plan_info) in chunks of whole modes; copy-in, solve and copy-out of successive
 * chunks overlap on internal streams.  The work starts after what is already queued
 * on `stream`, and `stream` waits for the last copy-out: synchronise `stream` before
 * reading u_host.  Host arrays must stay valid until then.  Successive calls on one
 * plan share the staging slots and internal streams: calls issued on two different
 * caller streams follow each other through the pipeline without draining it between
 * them.  Calls on one plan must come from one host thread at a time.  Errors as the
 * device solves. */
shen_status shen_solve_host(shen_plan_t plan, int problem, const double *f_host, double *u_host, int precision,
                            void *stream);

/* One linear step of the channel-flow solver (Sec. 3, Algorithm NS, its linear part),
 * in the scaled forms of the solves:
 *   u_new = -H_b^-1 (R_b u_old + (2/nu) load_u)       (Eq. ufin; load_u = S(h_v^{k+1/2}))
 *   g_new =  H_h^-1 (R_h g_old + (2/nu) load_g)       (Eq. gfin; load_g = S(h_g^{k+1/2}))
 * The minus sign of the biharmonic step: the solve's H_b is -2/(nu dt) times the
 * paper's Hchk, while R_b is +2/(nu dt) times its right-hand-side matrix.
 *   (v, w) from u_new, g_new as shen_velocity          (Eqs. ffin, f3, g3)
 * load_u / load_g may be NULL (no nonlinear term).  The right-hand sides use the
 * float-float operators (float64 ones when precision is SHEN_FP64); the solves use
 * `precision` (SHEN_AUTO: each problem's autotuned path).  The m = n = 0 mode's v and w
 * are left untouched (mean flow: see shen_mass_matvec).  Composed of the library's
 * kernels on `stream` (two operators, two solves in place in u_new and g_new, the
 * velocity recovery); no scratch memory.  All fields DEVICE, n_modes * N complex; the
 * outputs must not overlap the inputs or each other (SHEN_ERR_ARG).  Plans from an
 * explicit z2 list: SHEN_ERR_UNSUPPORTED.  Float-float solves of a plan must not run
 * concurrently with this call. */
shen_status shen_linear_step(shen_plan_t plan, const double *u_old, const double *g_old, const double *load_u,
                             const double *load_g, double *u_new, double *g_new, double *v, double *w,
                             int precision, void *stream);

/* Mass matrix of the problem's space (B_D for SHEN_HELMHOLTZ, B_B for SHEN_BIHARMONIC;
 * Table tab:matrices): out = B x + beta y for every mode, float-float arithmetic.
 * Arguments and errors as shen_rhs_matvec.  With it, the mean-flow equations of the
 * m = n = 0 mode (Eqs. v00, w00), scaled like the Helmholtz solve, read
 *     H_h v_new = R_h v_old + (2 / nu) (B_D H_y - S(beta)),  S(beta)_k = pi beta [k = 0],
 * which a one-mode plan (shen_plan_create_z2 with z2 = {0}) evaluates with
 * shen_mass_matvec, shen_rhs_matvec and shen_helmholtz_solve. */
shen_status shen_mass_matvec(shen_plan_t plan, int problem, const double *x, const double *y, double beta,
                             double *out, void *stream);

/* Velocity recovery of the linear step (Sec. 3).  From the wall-normal velocity u
 * (biharmonic coefficients, the solution of shen_biharmonic_solve) and g (Dirichlet
 * coefficients, the solution of shen_helmholtz_solve) of every mode:
 *   f = -du/dx projected on the Dirichlet space, B_D f = -C u with
 *       C_kj = (psi_j', phi_k) (Eq. ffin; the sign is that of Eq. f, f + du/dx = 0),
 *   v = i (n g - m f) / z2,  w = -i (n f + m g) / z2  (Eqs. f3, g3 solved for v, w),
 * with m = 2 pi ix / Lx and n = 2 pi kz / Lz the mode's wavenumbers (ix, kz as in the
 * mode layout), z2 = m^2 + n^2.  The mode m = n = 0 is left untouched: its v and w come
 * from the mean-flow Helmholtz solves (Eqs. v00, w00).  Float-float arithmetic
 * (precision SHEN_DF or SHEN_AUTO; others SHEN_ERR_UNSUPPORTED).
 *
 * u, g: DEVICE fields of the plan (u's entries N-4.. and g's N-2.. are ignored);
 * v, w: DEVICE outputs (entries N-2.. written 0); f: DEVICE output or NULL.  Outputs
 * must not overlap the inputs or each other (SHEN_ERR_ARG).  Plans built from an
 * explicit z2 list carry no (m, n): SHEN_ERR_UNSUPPORTED. */
shen_status shen_velocity(shen_plan_t plan, const double *u, const double *g, double *v, double *w, double *f,
                          int precision, void *stream);

/* ---- Wall-normal transforms (Sec. 2, Eqs. ifft, sst1, sst2, fstB; Algorithms fst, ifst) ----
 *
 * For every mode column of the plan, between the values at the N Chebyshev-Gauss points
 * x_i = cos((2i+1) pi / (2N)), i = 0 .. N-1 (weights pi / N) -- or, for SHEN_PLAN_GL plans,
 * the N Chebyshev-Gauss-Lobatto points x_i = cos(i pi / (N-1)) (weights pi / (N-1), half
 * at the two ends) -- and the coefficients of one of three spaces:
 *   SHEN_SPACE_CHEBYSHEV   T_k, k = 0 .. N-1                              (Eq. Tk)
 *   SHEN_SPACE_DIRICHLET   phi_k = T_k - T_{k+2}, k = 0 .. N-3            (Eq. phiD)
 *   SHEN_SPACE_BIHARMONIC  psi_k = T_k - 2(k+2)/(k+3) T_{k+2} + (k+1)/(k+3) T_{k+4},
 *                          k = 0 .. N-5                                     (Eq. phiN)
 * kind:
 *   SHEN_TRANSFORM_INVERSE  out_i = sum_k in_k phi_k(x_i)     (Eq. ifft; inputs beyond
 *                           the space's dimension are ignored)
 *   SHEN_TRANSFORM_SCALAR   out_k = (u, phi_k)_sigma = (pi/N) sum_i in_i phi_k(x_i)
 *                           (Eq. sst1; entries beyond the dimension written 0)
 *   SHEN_TRANSFORM_FORWARD  out = B^{-1} (u, phi)_sigma with the space's mass matrix B
 *                           (Eqs. sst2, fstB; Table tab:matrices), the sigma-orthogonal
 *                           projection of u on the space (entries beyond written 0)
 * Each cosine sum is one complex FFT per column, of length N on Gauss points (Makhoul's
 * reordering, DCT-II / DCT-III) or 2 (N-1) on Gauss-Lobatto points (the even extension,
 * DCT-I), run in float-float arithmetic (about 48 significant bits) in shared memory.  The
 * forward transforms in phi and psi solve with B in the same kernel: since B = P^T W P (P
 * the basis combination, W the discrete norms of the T_k), out is the W-weighted
 * least-squares fit of the Chebyshev coefficients, computed as prefix sums with a rank-1
 * (phi) or rank-2 (psi) correction, without forming B.  Relative errors are of order
 * 1e-14 for the inverse and scalar transforms and for the forward transform in T_k; the
 * forward transforms in phi and psi add the norm of the prefix sums (growing like N for
 * phi, N^2 for psi), well inside the float64 solve of B's own error (whose conditioning
 * is about 1e9 for the biharmonic B at N = 1024).
 *
 * in, out: DEVICE fields of n_modes * N complex values in the plan's layout (in == out
 * allowed; other overlap SHEN_ERR_ARG).  The FFT length must be 2^p or 3 2^p (N on Gauss
 * points, 2 (N - 1) on Gauss-Lobatto points), at least 8; other plans return
 * SHEN_ERR_UNSUPPORTED, as do lengths whose two shared-memory buffers do not fit one block
 * (on GB300: N = 8192 on Gauss points, N = 4097 on Gauss-Lobatto points).  Asynchronous on
 * `stream`.  Mode-major plans use no scratch memory, so calls on one plan may overlap;
 * wall-index-first plans gather each chunk of columns into plan-owned staging, transform it
 * and scatter it back, so their calls on one plan must not overlap.  Each column is staged
 * in shared memory by a bulk asynchronous copy; a copy that does not complete within a
 * bounded wait stops the kernel and is reported by shen_plan_check as SHEN_ERR_CUDA. */
typedef enum {
    SHEN_SPACE_CHEBYSHEV = 0,
    SHEN_SPACE_DIRICHLET = 1,
    SHEN_SPACE_BIHARMONIC = 2
} shen_space;

typedef enum {
    SHEN_TRANSFORM_INVERSE = 0,
    SHEN_TRANSFORM_SCALAR = 1,
    SHEN_TRANSFORM_FORWARD = 2
} shen_transform_kind;

shen_status shen_transform(shen_plan_t plan, int kind, int space, const double *in, double *out, void *stream);

/* The same for modes [mode_begin, mode_begin + mode_count) only: in and out point at the
 * column of mode_begin (a shard of a larger field, as for shen_solve_modes).  The transforms
 * do not depend on the mode, so a shard's columns are the full transform's columns bit for
 * bit.  mode_count = 0 checks the arguments (SHEN_ERR_UNSUPPORTED as above), launches
 * nothing and returns SHEN_OK; in and out may then be NULL. */
shen_status shen_transform_modes(shen_plan_t plan, int kind, int space, long mode_begin, long mode_count,
                                 const double *in, double *out, void *stream);

/* A posteriori check of a solve: for every mode, the relative residual
 * ||f - H u||_2 / ||f||_2 over the unknowns, H the Helmholtz or biharmonic system
 * matrix of the plan (Eqs. Helmholtz_matrix, Biharmonic_matrix in the scaled form of
 * shen_helmholtz_solve / shen_biharmonic_solve).  H u is evaluated in float-float
 * arithmetic, the difference and the norms in float64; relative residuals are resolved
 * down to about 1e-14 (Helmholtz) and 1e-12 (biharmonic, whose Q tail p_k q_j + r_k s_j
 * cancels between its two terms).  f, u: DEVICE fields of the plan; rel: DEVICE array of n_modes
 * doubles, or NULL.  The largest value is also kept by the plan for
 * shen_last_error_detail.  Asynchronous on `stream`. */
shen_status shen_residual(shen_plan_t plan, int problem, const double *f, const double *u, double *rel,
                          void *stream);

/* Synchronous error detail of the plan: *max_rel_residual (may be NULL) = the largest
 * relative residual found by the plan's last shen_residual (0 before any), and
 * *n_singular (may be NULL) = the number of (class, parity) factorisations that met a
 * zero or non-finite pivot when the plan was built (such a plan is refused at creation
 * with SHEN_ERR_SINGULAR, so this is 0 for every plan a caller holds). */
shen_status shen_last_error_detail(shen_plan_t plan, double *max_rel_residual, long *n_singular);

/* Time the candidate paths of `problem` on this plan and record the fastest for
 * SHEN_AUTO.  The candidates are the paths that meet a 1e-10 per-mode relative error
 * bar against the float64 oracle in the library's parity tests:
 *   Helmholtz:  SHEN_FP64, SHEN_DF, SHEN_DF_R1, SHEN_FP32_R1;
 *   biharmonic: SHEN_FP64, SHEN_DF.
 * Each float-float candidate is timed in each of its shapes (see shen_plan_set_shape;
 * shapes 2 and 3 on mode-major plans only).  The chosen shape then
 * serves every float-float solve of the plan and problem.  No candidate changes the
 * method or its accuracy class beyond that bar.
 *
 * f, u: DEVICE fields of the plan (n_modes * N complex values); they are solved in
 * place of a real workload and u is overwritten; u must not overlap f.  Synchronous:
 * returns after the timing (CUDA events on `stream`).  *chosen (may be NULL) receives
 * the chosen shen_precision, *ms (may be NULL) its time per solve in milliseconds.
 * Errors as the solves. */
shen_status shen_plan_autotune(shen_plan_t plan, int problem, const double *f, double *u, int *chosen,
                               float *ms, void *stream);

/* Iterative refinement over float32 sweeps, the precision pattern of the workload this
 * library serves (Sec. 4's algorithms in float32, the residual in higher precision):
 *   u = H^-1 f                      float32 forward elimination and back substitution,
 *                                   the float64 LU factors rounded to float32
 *   repeat `steps` times (0, 1 or 2):
 *     work = f - H u                residual in float64 (residual = SHEN_FP64) or in
 *                                   float-float (SHEN_DF), through the operators of
 *                                   shen_rhs_matvec with c -> -c (H_h = -R_h(-c),
 *                                   H_b = R_b(-c))
 *     u += H^-1 work                float32 sweeps, the sum in float64
 * for every mode of the plan, problem SHEN_HELMHOLTZ or SHEN_BIHARMONIC.  f, u, work:
 * DEVICE fields of the plan; work is the caller's scratch (overwritten); none of the three
 * may overlap another (SHEN_ERR_ARG).  Uses the problem's float-float scratch like
 * SHEN_DF solves (the same concurrency rule).  Measured accuracy against the oracle and
 * time are in the library's tests and benchmark: on GB300 one float64 or float-float
 * pass costs more than the float32 sweep it corrects, so SHEN_DF is the faster path at
 * the same accuracy.  Mode-major plans only. */
shen_status shen_solve_refine(shen_plan_t plan, int problem, const double *f, double *u, double *work, int steps,
                              int residual, void *stream);

/* Shape of the plan's float-float sweeps for `problem` (the choice shen_plan_autotune
 * makes):
 *   0  one thread per (mode, parity) chain, real and imaginary parts together, rows
 *      prefetched in registers, 4 (biharmonic) / 8 (Helmholtz) per block, two blocks in
 *      flight; the forward result spilled to a plan scratch in global memory;
 *   1  the same with 4 + 4 rows (biharmonic) / 5 rows (Helmholtz) per block (same bits
 *      as 0);
 *   2  one lane per real chain (the real or imaginary part of one parity chain), one
 *      CTA of 4 warps per SM, the forward result of each chain kept in Tensor Memory
 *      (its last 256 rows) and shared memory (the 96 rows before them), only the rest
 *      spilled to global memory; each row's float-float sum renormalised once;
 *   3  as 2 without the Tensor Memory part.
 * Shapes 2 and 3 round differently from 0 and 1 (same terms, same order, one
 * renormalisation per row instead of one per term): the results agree to the
 * float-float rounding.  Mode-major plans only (SHEN_ERR_UNSUPPORTED on a
 * SHEN_PLAN_WALL_FIRST plan).  shen_plan_set_shape returns SHEN_ERR_ARG for another
 * shape; the setting lasts until the next call or shen_plan_autotune.  A property of the
 * library, not of the method. */
shen_status shen_plan_set_shape(shen_plan_t plan, int problem, int shape);
shen_status shen_plan_get_shape(shen_plan_t plan, int problem, int *shape);

/* Right-hand-side operator: out = R x + beta * y for every mode (R = R_h or R_b by
 * `problem`).  y may be NULL (then beta is ignored).  x, y, out: DEVICE fields;
 * out must not overlap x or y.  float64 arithmetic.
 * R_h = (c - z2) B_D + A_D = (2/(nu dt)) (2 Bbar - Hbar) and R_b = Q + (c - 2 z2) A_B +
 * z2 (z2 - c) B_B = (2/(nu dt)) (2 Achk - 2 z2 Bchk - Hchk) (Eqs. gfin, ufin).  The
 * Helmholtz system carries the same factor, so the Crank-Nicolson step reads
 * H_h g_new = R_h g_old + (2/nu) S(h_g); the biharmonic system carries the opposite one
 * (H_b = -(2/(nu dt)) Hchk), so that step reads H_b u_new = -R_b u_old - (2/nu) S(h_v)
 * (shen_linear_step applies both). */
shen_status shen_rhs_matvec(shen_plan_t plan, int problem, const double *x, const double *y,
                            double beta, double *out, void *stream);

/* Same operator with a choice of arithmetic: precision SHEN_FP64 (as shen_rhs_matvec)
 * or SHEN_DF (SHEN_AUTO means SHEN_DF): each row's terms summed in float-float
 * arithmetic from float-float row tables, the running sums of the upper-triangular
 * parts carried in float-float, and + beta y as one float64 fused multiply-add.
 * Relative error of order 1e-14 against the float64 operator.  Other precisions:
 * SHEN_ERR_UNSUPPORTED.  Arguments and errors as shen_rhs_matvec. */
shen_status shen_rhs_matvec_ex(shen_plan_t plan, int problem, const double *x, const double *y, double beta,
                               double *out, int precision, void *stream);

/* Plan facts: number of modes, number of distinct z2 (factorisations), device bytes
 * held by the plan.  Any output pointer may be NULL. */
shen_status shen_plan_info(shen_plan_t plan, long *n_modes, long *n_classes, long *N,
                           long long *device_bytes);

/* Device-side error state of the plan after the stream is synchronised: SHEN_OK, or
 * SHEN_ERR_SINGULAR (with the first offending class index in *where if non-NULL), or
 * SHEN_ERR_CUDA if a transform's column copy did not complete (shen_transform). */
shen_status shen_plan_check(shen_plan_t plan, long *where);

/* Free the plan (after any work using it has completed).  NULL is ignored. */
void shen_plan_destroy(shen_plan_t plan);

/* ---- Batched plans: many independent channels with uneven sizes in one launch ----
 *
 * Each instance is a channel as in shen_plan_create (its own N, Fourier grid, nu, dt,
 * box).  The batched field stores instance i's mode-major columns (n_modes_i * N_i
 * complex values) after those of instances 0 .. i-1; shen_batch_offsets returns the
 * complex-element offset of each instance.  The solve is one persistent launch whose
 * warps take chunks of modes from a work queue ordered by decreasing N (one queue
 * counter per problem, plan-owned device memory, reset by an asynchronous memset at
 * every call: a Helmholtz and a biharmonic solve of the same plan may overlap on the
 * GPU, two solves of the same problem on the same plan must not).  The solve enqueues
 * on `stream` only. */
typedef struct shen_batch_s *shen_batch_t;

typedef struct {
    int N;                /* Chebyshev modes, 8 <= N <= 8192 */
    int Nx, Nz;           /* Fourier grid, even, >= 2 */
    double nu, dt;        /* viscosity and time step, > 0 */
    double Lx, Lz;        /* box lengths, > 0 */
} shen_instance_desc;

/* Build a batched plan from n_inst HOST descriptors.  Blocks until ready.  flags: 0 or
 * SHEN_PLAN_GL (every instance on Gauss-Lobatto points).  Errors as shen_plan_create. */
shen_status shen_batch_plan_create(shen_batch_t *batch, int n_inst, const shen_instance_desc *descs,
                                   unsigned flags, void *stream);

/* Total modes, total complex elements of a batched field, distinct (instance, z2)
 * factorisations, device bytes held.  Any output pointer may be NULL. */
shen_status shen_batch_info(shen_batch_t batch, long *n_modes, long *field_elems, long *n_classes,
                            long long *device_bytes);

/* offsets[0 .. n_inst]: complex-element offset of each instance's field in the batched
 * field, and the total (HOST array of n_inst + 1 longs). */
shen_status shen_batch_offsets(shen_batch_t batch, long *offsets);

/* Solve every mode of every instance: problem SHEN_HELMHOLTZ or SHEN_BIHARMONIC,
 * (float-float solves spill their forward results to a scratch the plan holds per
 * problem; like the per-problem work queue, this allows a Helmholtz and a biharmonic
 * solve to overlap, but not two solves of the same problem on one plan) 
 * precision SHEN_FP64, SHEN_DF or SHEN_AUTO (others: SHEN_ERR_UNSUPPORTED).  f, u: DEVICE batched
 * fields (u == f allowed).  Layout and zeroed trailing entries as for single plans. */
shen_status shen_batch_solve(shen_batch_t batch, int problem, const double *f, double *u, int precision,
                             void *stream);

/* Autotuning for batched plans, as shen_plan_autotune: candidates SHEN_FP64 and
 * SHEN_DF, the latter in both row-block shapes, each launched on a persistent grid
 * sized to that kernel's residency.  f, u: DEVICE batched fields (u must not overlap f;
 * u is overwritten).  Synchronous. */
shen_status shen_batch_autotune(shen_batch_t batch, int problem, const double *f, double *u, int *chosen,
                                float *ms, void *stream);

/* Solve every mode of every instance for batched fields in HOST memory, as
 * shen_solve_host does for single plans: f_host and u_host hold the batched field
 * (field_elems complex values, u_host == f_host allowed); page-locked (pinned) host
 * memory gives full copy bandwidth.  The field is cut into chunks of whole modes (at
 * most 256 MB each, contiguous in the field); each chunk is copied into one of three
 * device staging slots, solved there by one persistent launch over its modes (in the
 * batch's decreasing-N order) and copied back, with the copies of neighbouring chunks
 * overlapping the solve on internal streams.  The first call sets up the slots, the
 * chunks' work lists (4 bytes per mode) and the streams, blocking while it copies the
 * work lists; shen_batch_info counts them from then on.  The work starts after what is
 * queued on `stream`, and `stream` waits for the last copy-out: synchronise it before
 * reading u_host.  Calls on one plan share the pipeline (they follow each other chunk by
 * chunk) and must come from one host thread at a time; like shen_batch_solve, a call
 * must not overlap a device solve of the same problem on the same plan.  problem and
 * precision as shen_batch_solve; results equal shen_batch_solve's bit for bit. */
shen_status shen_batch_solve_host(shen_batch_t batch, int problem, const double *f_host, double *u_host,
                                  int precision, void *stream);

/* Device-side error state of the batched plan (SHEN_OK or SHEN_ERR_SINGULAR). */
shen_status shen_batch_check(shen_batch_t batch);

/* Free a batched plan (after its work has completed).  NULL is ignored. */
void shen_batch_destroy(shen_batch_t batch);

/* Same solve as shen_batch_solve, for callers that cannot allocate device memory when
 * they solve -- for example an application whose device memory is carved up in
 * advance by its own pool allocator.  The paper has no counterpart: this
 * is a property of the library, not of the method.
 *
 * It allocates nothing and uses none of the plan's scratch: its work-queue counter
 * lives in a fixed 256-byte device array that the library holds on every GPU it is
 * loaded on until the process exits.  The plan itself (created beforehand) and the
 * fields are the caller's.  Every call looks up that array's address in the current
 * context; the first call on a device also loads the array there, so make that first
 * call before any stream capture.  Every call resets the counter on `stream` before its
 * launch, so calls that overlap on the GPU (on any stream, any plan) race on it: issue
 * them one after the other.  The counter covers every batch a plan can hold
 * (shen_batch_plan_create limits a batch to 2^30 modes).  Errors as shen_batch_solve. */
shen_status shen_batch_solve_noalloc(shen_batch_t batch, int problem, const double *f, double *u,
                                     int precision, void *stream);

/* Static description of a status code. */
const char *shen_status_string(int status);

/* Library version as major * 10000 + minor * 100 + patch. */
int shen_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SHENSOLVE_H */
