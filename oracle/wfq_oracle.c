/*
 * Plain FP64 CPU oracle for the omega-FQ charge-response solve (arXiv 2103.00438).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares no
 * code, header, table or helper with the CUDA library under
 * paper_2103_00438_gb300/; the two meet only on the seeded inputs produced by
 * paper_2103_00438_gb300/structures.py (positions and parameters, no method
 * arithmetic).
 *
 * Every routine is the paper's definition written out with plain loops (OpenMP
 * only distributes independent rows), in double / double complex, with no
 * blocking, fusion or reordering beyond what the cited equation states.
 *
 * Equation numbers follow the order of the paper's numbered displays:
 *   Eq. 2  external potential         V_i = -E0 (r_i . k)
 *   Eq. 3  charge kernel              D_ij = erf(r_ij / sqrt(w_i^2 + w_j^2)) / r_ij,  D_ii = eta_i
 *   Eq. 4  Gaussian width rule        w_i = sqrt(2/pi) / eta_i
 *   Eq. 6  Fermi damping              f(r) = 1 / (1 + exp[-d (r / (s r0) - 1)])
 *   Eq. 9  real conductance kernel    Kbar_ij = (1 - f(r_ij)) A_ij / r_ij  (i != j)
 *   Eq. 11 A_ij = sum_k Kbar_ik (D_kj - D_ij)
 *   Eq. 12 z(w) = -(w / (2 n0 tau)) (w tau + i)
 *   Eq. 13 R_i = sum_j (V_i - V_j) Kbar_ij
 *   Eq. 14 (A - z I) q = R
 *   Eq. 16/17 P = diag(sum_k Kbar_ik),  A = (Kbar - P) D
 *   Eq. 24 GMRES iterate x_m = x_0 + V_m y_m over K_m(A, r_0)   (Section 3)
 *   Eq. 27 absolute residual || R - (A - zI) q ||_2
 *   Eq. 28 sigma_k = (4 pi w / c) sum_i (k_i / E0) Im q_i  ->  alpha_{k'k} = sum_i q_i r_{i,k'} / E0
 *   Eq. 33 RMSE = || R - (A - zI) q ||_2 / sqrt(N)
 *
 * Readings of the paper taken here:
 *   - Eq. 1 prints "+ i w" inside the sum over j; it is the diagonal term i w q_i,
 *     consistent with Eq. 14's shift -z I.
 *   - Eq. 4 prints eta_j on the right-hand side; the width of atom i uses eta_i,
 *     which is what makes the r -> 0 limit of Eq. 3 equal the diagonal eta_i.
 *   - The effective area A_ij of Eq. 5/9 is one uniform constant.
 *   - Kbar is dense by Eq. 9; for large N the CSR builder keeps the pairs with
 *     1 - f(r) >= cutoff_eps (cutoff_eps = 0 keeps every pair).
 *   - J-symmetric QMR (Section 3) uses the bilinear form u^T D v, no conjugation.
 *
 * Build: gcc -O2 -fopenmp -shared -fPIC (oracle/build.py).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

static const double ORC_PI = 3.14159265358979323846;

/* ------------------------------------------------------------------ */
/* Geometry helpers                                                    */
/* ------------------------------------------------------------------ */

static double dist(const double *xyz, int64_t i, int64_t j)
{
    double dx = xyz[3 * i + 0] - xyz[3 * j + 0];
    double dy = xyz[3 * i + 1] - xyz[3 * j + 1];
    double dz = xyz[3 * i + 2] - xyz[3 * j + 2];
    return sqrt(dx * dx + dy * dy + dz * dz);
}

/* Eq. 4 (reading: index i on both sides). */
void orc_widths(int64_t n, const double *eta, double *width)
{
    for (int64_t i = 0; i < n; ++i)
        width[i] = sqrt(2.0 / ORC_PI) / eta[i];
}

/* One entry of Eq. 3. */
double orc_d_entry(const double *xyz, const double *eta, int64_t i, int64_t j)
{
    if (i == j)
        return eta[i];
    double wi = sqrt(2.0 / ORC_PI) / eta[i];
    double wj = sqrt(2.0 / ORC_PI) / eta[j];
    double r = dist(xyz, i, j);
    return erf(r / sqrt(wi * wi + wj * wj)) / r;
}

/* Dense D (Eq. 3), row-major n x n. */
void orc_d_matrix(int64_t n, const double *xyz, const double *eta, double *D)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j)
            D[i * n + j] = orc_d_entry(xyz, eta, i, j);
}

/* Eq. 6. */
double orc_fermi(double r, double r0, double d_fermi, double s_fermi)
{
    return 1.0 / (1.0 + exp(-d_fermi * (r / (s_fermi * r0) - 1.0)));
}

/* One off-diagonal entry of Kbar (Eq. 9).  1 - f is evaluated as
 * 1 / (1 + exp(+d (x - 1))), the same quantity without the cancellation of 1 - f. */
double orc_kbar_entry(double r, double r0, double d_fermi, double s_fermi, double area)
{
    double one_minus_f = 1.0 / (1.0 + exp(d_fermi * (r / (s_fermi * r0) - 1.0)));
    return one_minus_f * area / r;
}

/* Dense Kbar (Eq. 9), zero diagonal, row-major n x n, every pair kept. */
void orc_kbar_matrix(int64_t n, const double *xyz, double r0, double d_fermi,
                     double s_fermi, double area, double *K)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j)
            K[i * n + j] = (i == j) ? 0.0
                                    : orc_kbar_entry(dist(xyz, i, j), r0, d_fermi, s_fermi, area);
}

/* Kbar as CSR by a brute-force double loop over all pairs: pair (i,j) is kept when
 * 1 - f(r_ij) >= cutoff_eps.  Pass 1 (col == NULL) fills rowptr only; pass 2 fills
 * col / val.  Returns nnz. */
int64_t orc_kbar_csr(int64_t n, const double *xyz, double r0, double d_fermi,
                     double s_fermi, double area, double cutoff_eps,
                     int64_t *rowptr, int64_t *col, double *val)
{
    if (col == NULL) {
#pragma omp parallel for schedule(dynamic, 64)
        for (int64_t i = 0; i < n; ++i) {
            int64_t c = 0;
            for (int64_t j = 0; j < n; ++j) {
                if (j == i) continue;
                double r = dist(xyz, i, j);
                double omf = 1.0 / (1.0 + exp(d_fermi * (r / (s_fermi * r0) - 1.0)));
                if (omf >= cutoff_eps) ++c;
            }
            rowptr[i + 1] = c;
        }
        rowptr[0] = 0;
        for (int64_t i = 0; i < n; ++i) rowptr[i + 1] += rowptr[i];
        return rowptr[n];
    }
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        int64_t p = rowptr[i];
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double r = dist(xyz, i, j);
            double omf = 1.0 / (1.0 + exp(d_fermi * (r / (s_fermi * r0) - 1.0)));
            if (omf >= cutoff_eps) {
                col[p] = j;
                val[p] = omf * area / r;
                ++p;
            }
        }
    }
    return rowptr[n];
}

/* Eq. 12: z = -(w / (2 n0 tau)) (w tau + i). */
void orc_z(double omega, double n0, double tau, double *zr, double *zi)
{
    cplx z = -(omega / (2.0 * n0 * tau)) * (omega * tau + I);
    *zr = creal(z);
    *zi = cimag(z);
}

/* Eq. 2 and Eq. 13 from a CSR Kbar:  R_i = sum_j (V_i - V_j) Kbar_ij,  V_i = -E0 (r_i . k). */
void orc_rhs_csr(int64_t n, const double *xyz, const int64_t *rowptr, const int64_t *col,
                 const double *val, const double *kdir, double E0, double *R)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double Vi = -E0 * (xyz[3 * i] * kdir[0] + xyz[3 * i + 1] * kdir[1] + xyz[3 * i + 2] * kdir[2]);
        double s = 0.0;
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            int64_t j = col[p];
            double Vj = -E0 * (xyz[3 * j] * kdir[0] + xyz[3 * j + 1] * kdir[1] + xyz[3 * j + 2] * kdir[2]);
            s += (Vi - Vj) * val[p];
        }
        R[i] = s;
    }
}

/* Eq. 2 and Eq. 13 from a dense Kbar. */
void orc_rhs_dense(int64_t n, const double *xyz, const double *K, const double *kdir,
                   double E0, double *R)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double Vi = -E0 * (xyz[3 * i] * kdir[0] + xyz[3 * i + 1] * kdir[1] + xyz[3 * i + 2] * kdir[2]);
        double s = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            double Vj = -E0 * (xyz[3 * j] * kdir[0] + xyz[3 * j + 1] * kdir[1] + xyz[3 * j + 2] * kdir[2]);
            s += (Vi - Vj) * K[i * n + j];
        }
        R[i] = s;
    }
}

/* Eq. 11, literally: A_ij = sum_k Kbar_ik (D_kj - D_ij).  O(n^3). */
void orc_a_matrix(int64_t n, const double *D, const double *K, double *A)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j) {
            double s = 0.0;
            for (int64_t k = 0; k < n; ++k)
                s += K[i * n + k] * (D[k * n + j] - D[i * n + j]);
            A[i * n + j] = s;
        }
}

/* ------------------------------------------------------------------ */
/* Operators y = (A - z I) x                                           */
/* ------------------------------------------------------------------ */

/* Kinds of operator representation the solvers accept. */
enum { ORC_OP_DENSE_A = 0, ORC_OP_STORED_D = 1, ORC_OP_OTF_D = 2 };

typedef struct {
    int kind;
    int64_t n;
    const double *A;       /* ORC_OP_DENSE_A: n x n, Eq. 11 */
    const double *D;       /* ORC_OP_STORED_D: n x n, Eq. 3 */
    const double *xyz;     /* ORC_OP_OTF_D: positions for Eq. 3 recomputed per use */
    const double *eta;
    const int64_t *rowptr; /* Kbar CSR (factored kinds) */
    const int64_t *col;
    const double *val;
    cplx z;
} orc_op;

/* u = D x with D either stored or recomputed entry by entry from Eq. 3. */
static void orc_d_apply(const orc_op *op, const cplx *x, cplx *u)
{
    int64_t n = op->n;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        cplx s = 0.0;
        if (op->kind == ORC_OP_STORED_D) {
            for (int64_t j = 0; j < n; ++j) s += op->D[i * n + j] * x[j];
        } else {
            for (int64_t j = 0; j < n; ++j) s += orc_d_entry(op->xyz, op->eta, i, j) * x[j];
        }
        u[i] = s;
    }
}

/* y = (A - z I) x.  Dense kind: A from Eq. 11.  Factored kinds: Eq. 17,
 * y = Kbar u - P u - z x with u = D x and P_ii = sum_k Kbar_ik (Eq. 16). */
static void orc_op_apply(const orc_op *op, const cplx *x, cplx *y)
{
    int64_t n = op->n;
    if (op->kind == ORC_OP_DENSE_A) {
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            cplx s = 0.0;
            for (int64_t j = 0; j < n; ++j) s += op->A[i * n + j] * x[j];
            y[i] = s - op->z * x[i];
        }
        return;
    }
    cplx *u = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    orc_d_apply(op, x, u);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        cplx ku = 0.0;
        double p = 0.0;
        for (int64_t q = op->rowptr[i]; q < op->rowptr[i + 1]; ++q) {
            ku += op->val[q] * u[op->col[q]];
            p += op->val[q];
        }
        y[i] = ku - p * u[i] - op->z * x[i];
    }
    free(u);
}

static void op_init(orc_op *op, int kind, int64_t n, const double *A, const double *D,
                    const double *xyz, const double *eta, const int64_t *rowptr,
                    const int64_t *col, const double *val, double zr, double zi)
{
    op->kind = kind; op->n = n; op->A = A; op->D = D; op->xyz = xyz; op->eta = eta;
    op->rowptr = rowptr; op->col = col; op->val = val; op->z = zr + I * zi;
}

/* Public apply: y = (A - z I) x, complex vectors as interleaved (re, im) doubles. */
void orc_apply(int kind, int64_t n, const double *A, const double *D, const double *xyz,
               const double *eta, const int64_t *rowptr, const int64_t *col,
               const double *val, double zr, double zi, const double *x, double *y)
{
    orc_op op;
    op_init(&op, kind, n, A, D, xyz, eta, rowptr, col, val, zr, zi);
    orc_op_apply(&op, (const cplx *)x, (cplx *)y);
}

/* Plain u = D x (stored or recomputed D), for the J = D products of QMR and for tests. */
void orc_d_matvec(int kind, int64_t n, const double *D, const double *xyz, const double *eta,
                  const double *x, double *u)
{
    orc_op op;
    op_init(&op, kind, n, NULL, D, xyz, eta, NULL, NULL, NULL, 0.0, 0.0);
    orc_d_apply(&op, (const cplx *)x, (cplx *)u);
}

/* ------------------------------------------------------------------ */
/* Direct solve: LU with partial pivoting of the complex matrix A - zI  */
/* ------------------------------------------------------------------ */

/* Solves (A - z I) q = R for one right-hand side.  A real n x n (Eq. 11), R complex.
 * Returns 0, or -1 if a zero pivot is met. */
int orc_lu_solve(int64_t n, const double *A, double zr, double zi, const double *R, double *q)
{
    cplx z = zr + I * zi;
    cplx *M = (cplx *)malloc(sizeof(cplx) * (size_t)n * (size_t)n);
    cplx *b = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t j = 0; j < n; ++j) M[i * n + j] = A[i * n + j];
        M[i * n + i] -= z;
        b[i] = R[2 * i] + I * R[2 * i + 1];
    }
    int status = 0;
    for (int64_t k = 0; k < n; ++k) {
        int64_t piv = k;
        double best = cabs(M[k * n + k]);
        for (int64_t i = k + 1; i < n; ++i)
            if (cabs(M[i * n + k]) > best) { best = cabs(M[i * n + k]); piv = i; }
        if (best == 0.0) { status = -1; break; }
        if (piv != k) {
            for (int64_t j = 0; j < n; ++j) {
                cplx t = M[k * n + j]; M[k * n + j] = M[piv * n + j]; M[piv * n + j] = t;
            }
            cplx t = b[k]; b[k] = b[piv]; b[piv] = t;
        }
#pragma omp parallel for schedule(static)
        for (int64_t i = k + 1; i < n; ++i) {
            cplx l = M[i * n + k] / M[k * n + k];
            M[i * n + k] = l;
            for (int64_t j = k + 1; j < n; ++j) M[i * n + j] -= l * M[k * n + j];
            b[i] -= l * b[k];
        }
    }
    if (status == 0) {
        for (int64_t i = n - 1; i >= 0; --i) {
            cplx s = b[i];
            for (int64_t j = i + 1; j < n; ++j) s -= M[i * n + j] * b[j];
            b[i] = s / M[i * n + i];
        }
        for (int64_t i = 0; i < n; ++i) { q[2 * i] = creal(b[i]); q[2 * i + 1] = cimag(b[i]); }
    }
    free(M);
    free(b);
    return status;
}

/* ------------------------------------------------------------------ */
/* Vector helpers (complex, Euclidean)                                 */
/* ------------------------------------------------------------------ */

static double vnorm(int64_t n, const cplx *x)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += creal(x[i]) * creal(x[i]) + cimag(x[i]) * cimag(x[i]);
    return sqrt(s);
}

/* <u, v> = u^H v */
static cplx vdot(int64_t n, const cplx *u, const cplx *v)
{
    cplx s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += conj(u[i]) * v[i];
    return s;
}

/* u^T v (bilinear, no conjugation) */
static cplx vbil(int64_t n, const cplx *u, const cplx *v)
{
    cplx s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += u[i] * v[i];
    return s;
}

/* ------------------------------------------------------------------ */
/* GMRES (Section 3, Eq. 24): Arnoldi with modified Gram-Schmidt, Givens QR of the
 * Hessenberg matrix, x_m = x_0 + V_m y_m.  restart = 0 means full (unrestarted)
 * GMRES; restart = k gives GMRES(k), restarting from the last iterate.  Start
 * vector x_0 = 0 (Section 4).  Stops when the Givens residual estimate
 * |g_{j+1}| <= rel_tol * ||R||; the true residual of Eq. 27 is recomputed at exit.
 * Returns 0 on convergence, 1 if max_iter was reached.
 * out[0] = iterations (operator applies inside Arnoldi), out[1] = true ||r||/||R||,
 * out[2] = restarts performed.                                                  */
/* ------------------------------------------------------------------ */
int orc_gmres(int kind, int64_t n, const double *A, const double *D, const double *xyz,
              const double *eta, const int64_t *rowptr, const int64_t *col, const double *val,
              double zr, double zi, const double *Rv, int restart, double rel_tol,
              int max_iter, double *qv, double *out)
{
    orc_op op;
    op_init(&op, kind, n, A, D, xyz, eta, rowptr, col, val, zr, zi);
    const cplx *b = (const cplx *)Rv;
    cplx *x = (cplx *)qv;
    int m = (restart > 0) ? restart : max_iter;
    if (m > max_iter) m = max_iter;
    cplx *V = (cplx *)malloc(sizeof(cplx) * (size_t)n * (size_t)(m + 1));
    cplx *H = (cplx *)calloc((size_t)(m + 1) * (size_t)m, sizeof(cplx)); /* H[i*m + j] */
    double *cs = (double *)malloc(sizeof(double) * (size_t)m);
    cplx *sn = (cplx *)malloc(sizeof(cplx) * (size_t)m);
    cplx *g = (cplx *)malloc(sizeof(cplx) * (size_t)(m + 1));
    cplx *y = (cplx *)malloc(sizeof(cplx) * (size_t)m);
    cplx *r = (cplx *)malloc(sizeof(cplx) * (size_t)n);

    for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
    double bnorm = vnorm(n, b);
    int iters = 0, restarts = 0, converged = 0;
    if (bnorm == 0.0) converged = 1;

    while (!converged && iters < max_iter) {
        /* r = b - (A - zI) x */
        orc_op_apply(&op, x, r);
        for (int64_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
        double beta = vnorm(n, r);
        if (beta <= rel_tol * bnorm) { converged = 1; break; }
        for (int64_t i = 0; i < n; ++i) V[i] = r[i] / beta;
        for (int j = 0; j <= m; ++j) g[j] = 0.0;
        g[0] = beta;
        memset(H, 0, sizeof(cplx) * (size_t)(m + 1) * (size_t)m);
        int jdone = 0;
        for (int j = 0; j < m && iters < max_iter; ++j) {
            cplx *w = V + (size_t)(j + 1) * (size_t)n;
            orc_op_apply(&op, V + (size_t)j * (size_t)n, w);
            ++iters;
            for (int i = 0; i <= j; ++i) {
                cplx *vi = V + (size_t)i * (size_t)n;
                cplx h = vdot(n, vi, w);
                H[i * m + j] = h;
                for (int64_t t = 0; t < n; ++t) w[t] -= h * vi[t];
            }
            double hn = vnorm(n, w);
            H[(j + 1) * m + j] = hn;
            if (hn != 0.0)
                for (int64_t t = 0; t < n; ++t) w[t] /= hn;
            /* previous rotations on column j */
            for (int i = 0; i < j; ++i) {
                cplx a = H[i * m + j], c2 = H[(i + 1) * m + j];
                H[i * m + j] = cs[i] * a + sn[i] * c2;
                H[(i + 1) * m + j] = -conj(sn[i]) * a + cs[i] * c2;
            }
            /* new rotation zeroing H[j+1][j] */
            cplx a = H[j * m + j];
            double bb = cabs(H[(j + 1) * m + j]);
            double nu = sqrt(cabs(a) * cabs(a) + bb * bb);
            if (cabs(a) == 0.0) { cs[j] = 0.0; sn[j] = 1.0; }
            else { cs[j] = cabs(a) / nu; sn[j] = (a / cabs(a)) * conj(H[(j + 1) * m + j]) / nu; }
            H[j * m + j] = cs[j] * a + sn[j] * H[(j + 1) * m + j];
            H[(j + 1) * m + j] = 0.0;
            g[j + 1] = -conj(sn[j]) * g[j];
            g[j] = cs[j] * g[j];
            jdone = j + 1;
            if (cabs(g[j + 1]) <= rel_tol * bnorm || hn == 0.0) break;
        }
        /* back substitution H y = g, x += V y */
        for (int i = jdone - 1; i >= 0; --i) {
            cplx s = g[i];
            for (int k = i + 1; k < jdone; ++k) s -= H[i * m + k] * y[k];
            y[i] = s / H[i * m + i];
        }
        for (int i = 0; i < jdone; ++i) {
            const cplx *vi = V + (size_t)i * (size_t)n;
            for (int64_t t = 0; t < n; ++t) x[t] += y[i] * vi[t];
        }
        if (jdone > 0 && cabs(g[jdone]) <= rel_tol * bnorm) {
            /* confirm with the true residual below */
            orc_op_apply(&op, x, r);
            for (int64_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
            if (vnorm(n, r) <= rel_tol * bnorm) converged = 1;
        }
        if (!converged && iters < max_iter) ++restarts;
    }
    orc_op_apply(&op, x, r);
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
    out[0] = iters;
    out[1] = (bnorm > 0.0) ? vnorm(n, r) / bnorm : 0.0;
    out[2] = restarts;
    free(V); free(H); free(cs); free(sn); free(g); free(y); free(r);
    return converged ? 0 : 1;
}

/* ------------------------------------------------------------------ */
/* J-symmetric QMR from BCG without look-ahead (Section 3; J = D by Eq. 18).
 *
 * BCG on M = A - zI with the shadow vectors taken as J r and J p, so that only M
 * products are needed; inner products are the bilinear form [u, v] = u^T D v.
 * The QMR iterate is obtained from the BCG iterates by quasi-minimal-residual
 * smoothing:  1/tau_k^2 = 1/tau_{k-1}^2 + 1/||r_k||^2,
 *             y_k = y_{k-1} + (tau_k^2/||r_k||^2)(x_k - y_{k-1}),
 *             s_k = s_{k-1} + (tau_k^2/||r_k||^2)(r_k - s_{k-1}),
 * where x_k, r_k are the BCG iterate/residual and y_k, s_k the QMR ones.
 * Stops when ||s_k|| <= rel_tol ||R||; returns 0, 1 (max_iter) or 2 (breakdown:
 * rho or sigma exactly zero).  out as for orc_gmres (out[2] = 0).              */
/* ------------------------------------------------------------------ */
int orc_qmr(int kind, int64_t n, const double *D, const double *xyz, const double *eta,
            const int64_t *rowptr, const int64_t *col, const double *val,
            double zr, double zi, const double *Rv, double rel_tol, int max_iter,
            double *qv, double *out)
{
    if (kind == ORC_OP_DENSE_A) return -1;  /* needs D for J */
    orc_op op;
    op_init(&op, kind, n, NULL, D, xyz, eta, rowptr, col, val, zr, zi);
    const cplx *b = (const cplx *)Rv;
    cplx *yq = (cplx *)qv;
    cplx *x = (cplx *)calloc((size_t)n, sizeof(cplx));
    cplx *r = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    cplx *p = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    cplx *s = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    cplx *Mp = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    cplx *Jv = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) { r[i] = b[i]; p[i] = b[i]; s[i] = b[i]; yq[i] = 0.0; }
    double bnorm = vnorm(n, b);
    double tau2 = bnorm * bnorm;
    orc_d_apply(&op, r, Jv);
    cplx rho = vbil(n, r, Jv);
    int iters = 0, status = 1;
    if (bnorm == 0.0) status = 0;
    while (status == 1 && iters < max_iter) {
        orc_op_apply(&op, p, Mp);
        ++iters;
        orc_d_apply(&op, p, Jv);
        cplx sigma = vbil(n, Jv, Mp);
        if (sigma == 0.0 || rho == 0.0) { status = 2; break; }
        cplx alpha = rho / sigma;
        for (int64_t i = 0; i < n; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * Mp[i]; }
        double rn = vnorm(n, r);
        double tau2_new = 1.0 / (1.0 / tau2 + 1.0 / (rn * rn));
        double wgt = tau2_new / (rn * rn);
        for (int64_t i = 0; i < n; ++i) {
            yq[i] += wgt * (x[i] - yq[i]);
            s[i] += wgt * (r[i] - s[i]);
        }
        tau2 = tau2_new;
        if (vnorm(n, s) <= rel_tol * bnorm) { status = 0; break; }
        orc_d_apply(&op, r, Jv);
        cplx rho_new = vbil(n, r, Jv);
        cplx beta = rho_new / rho;
        rho = rho_new;
        for (int64_t i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
    }
    orc_op_apply(&op, yq, Mp);
    for (int64_t i = 0; i < n; ++i) Mp[i] = b[i] - Mp[i];
    out[0] = iters;
    out[1] = (bnorm > 0.0) ? vnorm(n, Mp) / bnorm : 0.0;
    out[2] = 0;
    free(x); free(r); free(p); free(s); free(Mp); free(Jv);
    return status;
}

/* ------------------------------------------------------------------ */
/* Outputs                                                             */
/* ------------------------------------------------------------------ */

/* alpha_{k'} = sum_i q_i r_{i,k'} / E0 for k' = x, y, z (Eq. 28 without the 4 pi w / c
 * prefactor and the imaginary part).  q complex interleaved; alpha[2*k'] re, [2*k'+1] im. */
void orc_alpha(int64_t n, const double *xyz, const double *qv, double E0, double *alpha)
{
    const cplx *q = (const cplx *)qv;
    for (int k = 0; k < 3; ++k) {
        cplx s = 0.0;
        for (int64_t i = 0; i < n; ++i) s += q[i] * xyz[3 * i + k];
        s /= E0;
        alpha[2 * k] = creal(s);
        alpha[2 * k + 1] = cimag(s);
    }
}

/* Eq. 27 residual norm ||R - (A - zI) q||_2 (absolute). */
double orc_residual_norm(int kind, int64_t n, const double *A, const double *D,
                         const double *xyz, const double *eta, const int64_t *rowptr,
                         const int64_t *col, const double *val, double zr, double zi,
                         const double *Rv, const double *qv)
{
    orc_op op;
    op_init(&op, kind, n, A, D, xyz, eta, rowptr, col, val, zr, zi);
    cplx *t = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    orc_op_apply(&op, (const cplx *)qv, t);
    const cplx *b = (const cplx *)Rv;
    for (int64_t i = 0; i < n; ++i) t[i] = b[i] - t[i];
    double r = vnorm(n, t);
    free(t);
    return r;
}

/* Selected rows of y = (A - zI) x for one complex vector x (Eq. 17 with D from Eq. 3
 * recomputed entry by entry): y_i = sum_p Kbar_ip (u_j - u_i) - z x_i with
 * u_j = sum_k D_jk x_k evaluated for i and each neighbour j of i (found by a brute-force
 * scan with the keep rule 1 - f(r) >= cutoff_eps of orc_kbar_csr).  Also returns, per
 * row, bound_i = sum_p Kbar_ip (s_i + s_j) + |z| |x_i| with s = |D| |x| (the scale the
 * tests measure rounding errors against).  For sampled checks at sizes where a full
 * apply is out of reach. */
static void d_row_sums(int64_t n, const double *xyz, const double *eta, int64_t j, const cplx *x, cplx *u,
                       double *sabs)
{
    cplx s = 0.0;
    double a = 0.0;
    for (int64_t k = 0; k < n; ++k) {
        double d = orc_d_entry(xyz, eta, j, k);
        s += d * x[k];
        a += fabs(d) * cabs(x[k]);
    }
    *u = s;
    *sabs = a;
}

void orc_apply_rows(int64_t n, const double *xyz, const double *eta, double r0, double d_fermi, double s_fermi,
                    double area, double cutoff_eps, double zr, double zi, const double *xv, int64_t nrows,
                    const int64_t *rows, double *y, double *bound)
{
    const cplx *x = (const cplx *)xv;
    cplx z = zr + I * zi;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t t = 0; t < nrows; ++t) {
        int64_t i = rows[t];
        cplx ui;
        double si;
        d_row_sums(n, xyz, eta, i, x, &ui, &si);
        cplx acc = 0.0;
        double b = 0.0;
        /* neighbours of i by a brute-force scan with the same keep rule as orc_kbar_csr */
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double r = dist(xyz, i, j);
            double omf = 1.0 / (1.0 + exp(d_fermi * (r / (s_fermi * r0) - 1.0)));
            if (omf < cutoff_eps) continue;
            double kij = omf * area / r;
            cplx uj;
            double sj;
            d_row_sums(n, xyz, eta, j, x, &uj, &sj);
            acc += kij * (uj - ui);
            b += kij * (si + sj);
        }
        cplx yi = acc - z * x[i];
        y[2 * t] = creal(yi);
        y[2 * t + 1] = cimag(yi);
        bound[t] = b + cabs(z) * cabs(x[i]);
    }
}

/* Selected rows of R (Eq. 13 with the potential of Eq. 2), each row's neighbours found by a
 * brute-force scan with the keep rule of orc_kbar_csr: R_i = sum_j Kbar_ij (V_i - V_j),
 * V = -E0 (r . kdir).  For residual audits of structures too large for a CSR of Kbar. */
void orc_rhs_rows(int64_t n, const double *xyz, double r0, double d_fermi, double s_fermi, double area,
                  double cutoff_eps, const double *kdir, double E0, int64_t nrows, const int64_t *rows,
                  double *R)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t t = 0; t < nrows; ++t) {
        int64_t i = rows[t];
        double Vi = -E0 * (xyz[3 * i] * kdir[0] + xyz[3 * i + 1] * kdir[1] + xyz[3 * i + 2] * kdir[2]);
        double s = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double r = dist(xyz, i, j);
            double omf = 1.0 / (1.0 + exp(d_fermi * (r / (s_fermi * r0) - 1.0)));
            if (omf < cutoff_eps) continue;
            double Vj = -E0 * (xyz[3 * j] * kdir[0] + xyz[3 * j + 1] * kdir[1] + xyz[3 * j + 2] * kdir[2]);
            s += (Vi - Vj) * (omf * area / r);
        }
        R[t] = s;
    }
}

/* Complex Euclidean inner product, exported for tests of the Arnoldi basis. */
void orc_vdot(int64_t n, const double *u, const double *v, double *out)
{
    cplx s = vdot(n, (const cplx *)u, (const cplx *)v);
    out[0] = creal(s);
    out[1] = cimag(s);
}
