/*
 * The paper's O(N) direct solvers, written plainly in C (oracle, test infrastructure).
 *
 * Not part of the product: only the tests and the CPU-baseline legs of bench.py load
 * this file's shared library.  It shares nothing with the CUDA path.
 *
 * Source: Mortensen, arXiv:1701.03787, Sec. 4.
 *  - Helmholtz (Eq. gfin, Sec. 4 prose): the matrix decouples into odd and even
 *    rows, each an upper-Hessenberg system; LU without pivoting gives L with one
 *    subdiagonal and U whose row k holds three distinct values U_kk, U_k,k+2,
 *    U_k,k+4 with U_kj = U_k,k+4 for every j >= k+6 of the same parity.
 *  - Biharmonic (Eq. ufin): Algorithm LUbiharmonic (L with subdiagonals k-2, k-4),
 *    Algorithm ReduceAB (Eq. ab: U_kj = xi0 (a_k q_j + b_k s_j) for j >= k+6),
 *    Algorithm LUSolveBiharmonic (forward elimination, back substitution with the
 *    four running sums q^o, q^e, s^o, s^e).
 *
 * Matrices (Table tab:matrices, Eqs. N_Q, pk, rk; scaled forms with xi0 = 1):
 *   Helmholtz  H = alpha B - A,  B = (phi_j, phi_k), A = (phi_j'', phi_k)
 *   biharmonic H = Q + a A + b B with A = (psi_j'', psi_k), B = (psi_j, psi_k),
 *              Q = (psi_j'''', psi_k)
 * Stiffness closed forms (exact inner products; A taken with the + sign under which
 * Eqs. ufin/gfin are the Crank-Nicolson form of the PDEs):
 *   Dirichlet   A_kk = -2 pi (k+1)(k+2),  A_kj = -4 pi (k+1) for j = k+2, k+4, ...
 *   biharmonic  A_kk = -4 pi (k+1)(k+2)^2/(k+3), A_k,k+2 = 2 pi (k+1)(k+2),
 *               A_k,k-2 = 2 pi (k-1)(k+2)
 *   Q_kk = 8 pi (k+1)^2 (k+2)(k+4) (the printed diagonal of Eq. N_Q is a misprint),
 *   Q_kj = p_k q_j + r_k s_j for j = k+2, k+4, ... (Eqs. pk, rk).
 * In Algorithms 1-3 "N" is read as the index of the last unknown (N_modes - 5).
 *
 * Layout: complex values interleaved (re, im); a mode's column holds N entries,
 * entries beyond the unknowns are ignored on input and written 0 on output.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static const double PI = 3.14159265358979323846;

static double ck(int k) { return k == 0 ? 2.0 : 1.0; }

/* ---------------------------------------------------------------- Helmholtz */

static double hd_entry(int k, int j, double alpha)
{   /* (alpha B - A)_{kj} for same-parity j >= k-2 */
    if (j == k - 2) return -alpha * PI / 2;
    if (j == k) return alpha * PI / 2 * (ck(k) + 1.0) + 2 * PI * (k + 1) * (k + 2);
    if (j == k + 2) return -alpha * PI / 2 + 4 * PI * (k + 1);
    return 4 * PI * (k + 1);               /* j >= k+4 */
}

/* work: 5*n doubles. */
int on_helmholtz_solve(int N, double alpha, const double *f, double *u, double *work)
{
    int n = N - 2;
    if (n < 1) return -1;
    double *L = work, *U0 = work + n, *U1 = work + 2 * n, *U2 = work + 3 * n, *yy = work + 4 * n;
    /* factorisation, each parity chain separately (odd/even decoupling) */
    for (int k = 0; k < n; k++) {
        if (k < 2) {
            L[k] = 0;
            U0[k] = hd_entry(k, k, alpha);
            U1[k] = hd_entry(k, k + 2, alpha);
            U2[k] = hd_entry(k, k + 4, alpha);
        } else {
            L[k] = hd_entry(k, k - 2, alpha) / U0[k - 2];
            U0[k] = hd_entry(k, k, alpha) - L[k] * U1[k - 2];
            U1[k] = hd_entry(k, k + 2, alpha) - L[k] * U2[k - 2];
            U2[k] = hd_entry(k, k + 4, alpha) - L[k] * U2[k - 2];
        }
    }
    for (int c = 0; c < 2; c++) {          /* Re, Im */
        for (int k = 0; k < n; k++) {
            double fk = f[2 * k + c];
            yy[k] = k < 2 ? fk : fk - L[k] * yy[k - 2];
        }
        double sum[2] = {0, 0};            /* sum of u_j, j >= k+4, per parity */
        for (int k = n - 1; k >= 0; k--) {
            int p = k & 1;
            double up2 = k + 2 < n ? u[2 * (k + 2) + c] : 0.0;
            if (k + 4 < n) sum[p] += u[2 * (k + 4) + c];
            u[2 * k + c] = (yy[k] - U1[k] * up2 - U2[k] * sum[p]) / U0[k];
        }
    }
    for (int k = n; k < N; k++) u[2 * k] = u[2 * k + 1] = 0.0;
    return 0;
}

/* --------------------------------------------------------------- Biharmonic */

static double pk(int k) { return 8.0 * k * (k + 1) * (k + 2) * (k + 4) * PI; }
static double rk(int k) { return 24.0 * (k + 1) * (k + 2) * PI; }
static double qj(int j) { return 1.0 / (j + 3); }
static double sj(int j) { return (double)(j + 2) * (j + 2) / (j + 3); }

static double bb_entry(int k, int j)
{   /* B_{kj} = (psi_j, psi_k), symmetric, Table tab:matrices (c_{N_x} = 1, GC) */
    if (j < k) { int t = j; j = k; k = t; }
    double r = (double)(k + 2) / (k + 3), s = (double)(k + 1) / (k + 3);
    if (j == k) return PI / 2 * (ck(k) + 4 * r * r + s * s);
    if (j == k + 2) return -PI * (r + (double)(k + 4) * (k + 1) / ((double)(k + 5) * (k + 3)));
    if (j == k + 4) return PI / 2 * s;
    return 0.0;
}

static double ab_entry(int k, int j)
{   /* A_{kj} = (psi_j'', psi_k) */
    if (j == k) return -4 * PI * (k + 1) * (double)(k + 2) * (k + 2) / (k + 3);
    if (j == k + 2) return 2 * PI * (k + 1) * (k + 2);
    if (j == k - 2) return 2 * PI * (k - 1) * (k + 2);
    return 0.0;
}

static double qb_entry(int k, int j)
{   /* Q_{kj} = (psi_j'''', psi_k) */
    if (j < k || ((j - k) & 1)) return 0.0;
    if (j == k) return 8 * PI * (k + 1) * (double)(k + 1) * (k + 2) * (k + 4);
    return pk(k) * qj(j) + rk(k) * sj(j);
}

static double hb_entry(int k, int j, double a, double b)
{
    return qb_entry(k, j) + a * ab_entry(k, j) + b * bb_entry(k, j);
}

/* Algorithm LUbiharmonic with dense U (as printed), O(n^2) memory: small n only.
 * Lk2[k] = L_{k,k-2}, Lk4[k] = L_{k,k-4}; U is n*n row-major. */
static void lu_biharmonic_dense(int n, double a, double b, double *Lk2, double *Lk4, double *U)
{
    int Nl = n - 1;
    memset(U, 0, sizeof(double) * n * n);
    for (int k = 0; k < n; k++) Lk2[k] = Lk4[k] = 0.0;
    int Me = Nl / 2, Mo = (Nl - 1) / 2;
    for (int j = 0; j <= Me; j++) U[0 * n + 2 * j] = hb_entry(0, 2 * j, a, b);
    for (int j = 0; j <= Mo; j++) U[1 * n + 2 * j + 1] = hb_entry(1, 2 * j + 1, a, b);
    if (Nl >= 2) {
        Lk2[2] = hb_entry(2, 0, a, b) / U[0];
        for (int j = 1; j <= Me; j++) U[2 * n + 2 * j] = hb_entry(2, 2 * j, a, b) - Lk2[2] * U[0 * n + 2 * j];
    }
    if (Nl >= 3) {
        Lk2[3] = hb_entry(3, 1, a, b) / U[1 * n + 1];
        for (int j = 1; j <= Mo; j++) U[3 * n + 2 * j + 1] = hb_entry(3, 2 * j + 1, a, b) - Lk2[3] * U[1 * n + 2 * j + 1];
    }
    for (int k = 4; k <= Nl; k++) {
        int M = (Nl - k) / 2;
        Lk4[k] = hb_entry(k, k - 4, a, b) / U[(k - 4) * n + (k - 4)];
        for (int j = -1; j <= M; j++)
            U[k * n + k + 2 * j] = hb_entry(k, k + 2 * j, a, b) - Lk4[k] * U[(k - 4) * n + k + 2 * j];
        Lk2[k] = U[k * n + k - 2] / U[(k - 2) * n + (k - 2)];
        for (int j = -1; j <= M; j++)
            U[k * n + k + 2 * j] -= Lk2[k] * U[(k - 2) * n + k + 2 * j];
    }
}

/* Algorithm ReduceAB: a_k, b_k for k = 0..n-7 (stored for all k, zero beyond). */
static void reduce_ab(int n, const double *Lk2, const double *Lk4, double *av, double *bv)
{
    int last = n - 7;                      /* N_x - 10 with N_x - 4 = n - 1 */
    for (int k = 0; k < n; k++) av[k] = bv[k] = 0.0;
    for (int k = 0; k <= 1 && k <= last; k++) {
        av[k] = pk(k);
        bv[k] = rk(k);
        if (k + 2 <= last) {
            av[k + 2] = pk(k + 2) - Lk2[k + 2] * av[k];
            bv[k + 2] = rk(k + 2) - Lk2[k + 2] * bv[k];
        }
    }
    for (int k = 4; k <= last; k++) {
        av[k] = pk(k) - Lk2[k] * av[k - 2] - Lk4[k] * av[k - 4];
        bv[k] = rk(k) - Lk2[k] * bv[k - 2] - Lk4[k] * bv[k - 4];
    }
}

/* Algorithm LUSolveBiharmonic for one real right-hand side (stride 2 in f / u). */
static void lu_solve_biharmonic(int n, const double *f, double *u, const double *Lk2, const double *Lk4,
                                const double *Ud0, const double *Ud2, const double *Ud4,
                                const double *av, const double *bv, double *y)
{
    int Nl = n - 1;
    for (int k = 0; k <= 1; k++) {
        y[k] = f[2 * k];
        if (k + 2 <= Nl) y[k + 2] = f[2 * (k + 2)] - Lk2[k + 2] * y[k];
    }
    for (int k = 4; k <= Nl; k++) y[k] = f[2 * k] - Lk2[k] * y[k - 2] - Lk4[k] * y[k - 4];
    for (int k = Nl; k >= Nl - 1; k--) {
        u[2 * k] = y[k] / Ud0[k];
        u[2 * (k - 2)] = (y[k - 2] - Ud2[k - 2] * u[2 * k]) / Ud0[k - 2];
    }
    double qo = 0, qe = 0, so = 0, se = 0;
    for (int k = Nl - 4; k >= 0; k--) {
        double v = y[k] - Ud2[k] * u[2 * (k + 2)] - Ud4[k] * u[2 * (k + 4)];
        if (k < Nl - 5) {
            int j = k + 6;
            if (k & 1) {
                qo += u[2 * j] * qj(j);
                so += u[2 * j] * sj(j);
                v -= qo * av[k] + so * bv[k];
            } else {
                qe += u[2 * j] * qj(j);
                se += u[2 * j] * sj(j);
                v -= qe * av[k] + se * bv[k];
            }
        }
        u[2 * k] = v / Ud0[k];
    }
}

/* Dense-U variant (Algorithm 1 exactly as printed).  work: n*n + 9n doubles. */
int on_biharmonic_solve_dense_lu(int N, double a, double b, const double *f, double *u, double *work)
{
    int n = N - 4;
    if (n < 4) return -1;
    double *U = work, *Lk2 = U + (size_t)n * n, *Lk4 = Lk2 + n, *av = Lk4 + n, *bv = av + n;
    double *Ud0 = bv + n, *Ud2 = Ud0 + n, *Ud4 = Ud2 + n, *y = Ud4 + n;
    lu_biharmonic_dense(n, a, b, Lk2, Lk4, U);
    reduce_ab(n, Lk2, Lk4, av, bv);
    for (int k = 0; k < n; k++) {
        Ud0[k] = U[(size_t)k * n + k];
        Ud2[k] = k + 2 < n ? U[(size_t)k * n + k + 2] : 0.0;
        Ud4[k] = k + 4 < n ? U[(size_t)k * n + k + 4] : 0.0;
    }
    for (int c = 0; c < 2; c++) lu_solve_biharmonic(n, f + c, u + c, Lk2, Lk4, Ud0, Ud2, Ud4, av, bv, y);
    for (int k = n; k < N; k++) u[2 * k] = u[2 * k + 1] = 0.0;
    return 0;
}

/* Compact O(n) factorisation: the same row updates as Algorithm LUbiharmonic, with
 * the entries of rows k-2, k-4 beyond their three stored values taken from Eq. ab
 * (storage < 7N, Sec. 4).  Rows k-2 and k-4 are reached by the update at columns
 * k-2, k, k+2, k+4 (the rest of row k follows Eq. ab through a_k, b_k). */
static void lu_biharmonic_compact(int n, double a, double b, double *Lk2, double *Lk4,
                                  double *Ud0, double *Ud2, double *Ud4, double *av, double *bv)
{
    for (int k = 0; k < n; k++) {
        /* U_{m,j} for a finished row m < k (j same parity as m, j >= m) */
#define UROW(m, j) ((j) == (m) ? Ud0[m] : (j) == (m) + 2 ? Ud2[m] : (j) == (m) + 4 ? Ud4[m] \
                    : (av[m] * qj(j) + bv[m] * sj(j)))
        double l4 = 0.0, l2 = 0.0;
        if (k >= 4) l4 = hb_entry(k, k - 4, a, b) / Ud0[k - 4];
        if (k >= 2) {
            double t = hb_entry(k, k - 2, a, b) - (k >= 4 ? l4 * UROW(k - 4, k - 2) : 0.0);
            l2 = t / Ud0[k - 2];
        }
        Lk4[k] = l4;
        Lk2[k] = l2;
        double v[3];
        for (int s = 0; s < 3; s++) {
            int j = k + 2 * s;
            if (j >= n) { v[s] = 0.0; continue; }
            double h = hb_entry(k, j, a, b);
            if (k >= 4) h -= l4 * UROW(k - 4, j);
            if (k >= 2) h -= l2 * UROW(k - 2, j);
            v[s] = h;
        }
        Ud0[k] = v[0]; Ud2[k] = v[1]; Ud4[k] = v[2];
        /* Algorithm ReduceAB, interleaved: a_k = p_k - L_{k,k-2} a_{k-2} - L_{k,k-4} a_{k-4} */
        /* (only k <= n-7 is ever read: a lookup UROW(m, j) beyond the band has
           j = m+6 or m+8 < n) */
        av[k] = pk(k) - (k >= 2 ? l2 * av[k - 2] : 0.0) - (k >= 4 ? l4 * av[k - 4] : 0.0);
        bv[k] = rk(k) - (k >= 2 ? l2 * bv[k - 2] : 0.0) - (k >= 4 ? l4 * bv[k - 4] : 0.0);
#undef UROW
    }
}

/* work: 9n doubles. */
int on_biharmonic_solve(int N, double a, double b, const double *f, double *u, double *work)
{
    int n = N - 4;
    if (n < 4) return -1;
    double *Lk2 = work, *Lk4 = Lk2 + n, *av = Lk4 + n, *bv = av + n;
    double *Ud0 = bv + n, *Ud2 = Ud0 + n, *Ud4 = Ud2 + n, *y = Ud4 + n;
    lu_biharmonic_compact(n, a, b, Lk2, Lk4, Ud0, Ud2, Ud4, av, bv);
    for (int c = 0; c < 2; c++) lu_solve_biharmonic(n, f + c, u + c, Lk2, Lk4, Ud0, Ud2, Ud4, av, bv, y);
    for (int k = n; k < N; k++) u[2 * k] = u[2 * k + 1] = 0.0;
    return 0;
}

/* ------------------------------------------------------------- mode batches */

int on_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Thread count of the mode batches below (timing the baseline on one core). */
void on_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* f, u: n_modes columns of N complex (2N doubles) each; coef per mode. */
int on_helmholtz_solve_modes(int N, long n_modes, const double *alpha, const double *f, double *u)
{
    int err = 0;
#pragma omp parallel reduction(| : err)
    {
        double *work = (double *)malloc(sizeof(double) * 5 * (size_t)N);
#pragma omp for schedule(static)
        for (long m = 0; m < n_modes; m++)
            err |= on_helmholtz_solve(N, alpha[m], f + 2 * (size_t)N * m, u + 2 * (size_t)N * m, work);
        free(work);
    }
    return err ? -1 : 0;
}

int on_biharmonic_solve_modes(int N, long n_modes, const double *a, const double *b, const double *f, double *u)
{
    int err = 0;
#pragma omp parallel reduction(| : err)
    {
        double *work = (double *)malloc(sizeof(double) * 9 * (size_t)N);
#pragma omp for schedule(static)
        for (long m = 0; m < n_modes; m++)
            err |= on_biharmonic_solve(N, a[m], b[m], f + 2 * (size_t)N * m, u + 2 * (size_t)N * m, work);
        free(work);
    }
    return err ? -1 : 0;
}
