/*
 * nrs_oracle.c -- plain FP64 CPU oracle of the nearest-neighbour (NEAREST)
 * regularized stokeslet method (Gallagher & Smith, "Passively parallel
 * regularized stokeslets", Sec. 3 and Sec. 4).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * reference that the CUDA library is checked against.  Only the test suite,
 * the package's smoke check and the benchmark's CPU-baseline leg may load it;
 * the product path never calls into it.  It shares no code with the CUDA
 * sources.
 *
 * Everything is double precision.  Build with -ffp-contract=off so that no
 * multiply-add is fused: the nearest-neighbour decision below must be the
 * plain rounded expression ((dx*dx + dy*dy) + dz*dz).  OpenMP only splits
 * independent outer loops (rows m, columns j); it never changes the order
 * of the operations that produce any single value.
 *
 * Layouts: points are rows of 4 doubles (x, y, z, pad-or-weight); matrices
 * are column-major with leading dimension lda (entry (i,j) at A[i + j*lda]).
 * Unknown ordering: 3m+j for force point m and component j, then 6 per free
 * body in body order ([U(3), Omega(3)] as columns, [force(3), moment(3)] as
 * rows).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846

enum { OR_FREE = 0, OR_PRESCRIBED = 1, OR_STATIC = 2 };

int or_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Kernels of Sec. 3                                                         */
/* ------------------------------------------------------------------------ */

/* Regularized stokeslet (Sec. 3, the Cortez blob solution):
 *   S_jk(r) = (delta_jk (|r|^2 + 2 eps^2) + r_j r_k) / (|r|^2 + eps^2)^{3/2},
 * with r = x - y.  S is returned row-major, S[3*j + k]. */
void or_stokeslet(const double *r, double eps, double *S)
{
    double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
    double e2 = eps * eps;
    double rho = r2 + e2;
    double inv = 1.0 / (rho * sqrt(rho));
    for (int j = 0; j < 3; ++j)
        for (int k = 0; k < 3; ++k) {
            double v = r[j] * r[k];
            if (j == k) v += r2 + 2.0 * e2;
            S[3 * j + k] = v * inv;
        }
}

/* Singular stokeslet (Oseen tensor, Sec. 2): delta_jk/|r| + r_j r_k/|r|^3. */
void or_oseen(const double *r, double *S)
{
    double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
    double rr = sqrt(r2);
    for (int j = 0; j < 3; ++j)
        for (int k = 0; k < 3; ++k)
            S[3 * j + k] = (j == k ? 1.0 / rr : 0.0) + r[j] * r[k] / (r2 * rr);
}

/* Blob (Sec. 3): phi_eps(r) = 15 eps^4 / (8 pi (|r|^2 + eps^2)^{7/2}). */
double or_blob(const double *r, double eps)
{
    double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
    double rho = r2 + eps * eps;
    return 15.0 * eps * eps * eps * eps / (8.0 * OR_PI * pow(rho, 3.5));
}

/* Regularized pressure numerator (Sec. 3):
 *   P_k(r) = r_k (2|r|^2 + 5 eps^2) / (|r|^2 + eps^2)^{5/2}. */
void or_pressure(const double *r, double eps, double *P)
{
    double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
    double e2 = eps * eps;
    double rho = r2 + e2;
    double f = (2.0 * r2 + 5.0 * e2) / (rho * rho * sqrt(rho));
    for (int k = 0; k < 3; ++k) P[k] = r[k] * f;
}

/* ------------------------------------------------------------------------ */
/* Nearest-neighbour map nu (Sec. 3, the argmin defining n-hat)              */
/* ------------------------------------------------------------------------ */

/* For each quadrature point q, nn[q] = the force point n minimising
 * d^2 = ((dx*dx + dy*dy) + dz*dz), dx = x_n.x - X_q.x, taken over the force
 * points of q's own body (global == 0) or over all force points
 * (global != 0).  Candidates are visited in ascending n and only a strictly
 * smaller d^2 replaces the incumbent, so exact ties go to the lowest index.
 * Returns 0, or -1 if some quadrature point has no candidate. */
int or_nearest(int nbodies, const int64_t *n_off, const int64_t *q_off,
               const double *x, const double *X, int global, int32_t *nn)
{
    int bad = 0;
    for (int b = 0; b < nbodies; ++b) {
        int64_t n_lo = global ? 0 : n_off[b];
        int64_t n_hi = global ? n_off[nbodies] : n_off[b + 1];
        if (n_hi <= n_lo && q_off[b + 1] > q_off[b]) bad = 1;
#pragma omp parallel for schedule(static)
        for (int64_t q = q_off[b]; q < q_off[b + 1]; ++q) {
            double best = INFINITY;
            int64_t arg = -1;
            for (int64_t n = n_lo; n < n_hi; ++n) {
                double dx = x[4 * n + 0] - X[4 * q + 0];
                double dy = x[4 * n + 1] - X[4 * q + 1];
                double dz = x[4 * n + 2] - X[4 * q + 2];
                double d2 = (dx * dx + dy * dy) + dz * dz;
                if (d2 < best) {
                    best = d2;
                    arg = n;
                }
            }
            nn[q] = (int32_t)arg;
        }
    }
    return bad ? -1 : 0;
}

/* Segments of nu: seg_ptr[n]..seg_ptr[n+1] lists, in ascending q, the
 * quadrature points whose nearest force point is n (stable counting sort).
 * This is the column structure of the sparse Q x N matrix nu (Sec. 3). */
void or_segments(int64_t N, int64_t Q, const int32_t *nn, int32_t *seg_ptr, int32_t *perm)
{
    int64_t *cursor = (int64_t *)calloc((size_t)N + 1, sizeof(int64_t));
    for (int64_t q = 0; q < Q; ++q) cursor[nn[q] + 1]++;
    for (int64_t n = 0; n < N; ++n) cursor[n + 1] += cursor[n];
    for (int64_t n = 0; n <= N; ++n) seg_ptr[n] = (int32_t)cursor[n];
    for (int64_t q = 0; q < Q; ++q) perm[cursor[nn[q]]++] = (int32_t)q;
    free(cursor);
}

/* ------------------------------------------------------------------------ */
/* Kinematics: body frame -> lab frame (Sec. 4, state Y = [X0; B])           */
/* ------------------------------------------------------------------------ */

/* out_i = x0 + B p_i for rows of 4 doubles; column 3 is copied unchanged
 * (pad or quadrature weight).  B is row-major 3x3 (B[3*r + c]); its columns
 * are the body basis vectors in the lab frame. */
void or_rigid_map(int64_t count, const double *p, const double *x0, const double *B, double *out)
{
    for (int64_t i = 0; i < count; ++i) {
        for (int r = 0; r < 3; ++r)
            out[4 * i + r] = x0[r] + (B[3 * r + 0] * p[4 * i + 0] + B[3 * r + 1] * p[4 * i + 1] +
                                      B[3 * r + 2] * p[4 * i + 2]);
        out[4 * i + 3] = p[4 * i + 3];
    }
}

/* ------------------------------------------------------------------------ */
/* Assembly (Sec. 3, eq. nnrsbie; Sec. 4 steps 1 and 2)                      */
/* ------------------------------------------------------------------------ */

/* Stokeslet part A_s of the system (rows/columns 0..3N-1):
 *   A[3m+j, 3n+k] = (1/(8 pi mu)) * sum_q S^eps_jk(x_m - X_q) w_q nu[q,n],
 * i.e. the product of the dense 3N x 3Q stokeslet matrix (weights w_q
 * included) with the 0/1 nearest-neighbour matrix.  Every force point m is
 * paired with every quadrature point q of every body.  The block is first
 * accumulated as sum_q S w_q, then multiplied by 1/(8 pi mu). */
/* Rows 3m..3m+2 of A_s for one force point m, written to dst[j + col*ld]
 * (col = 0..3N-1): zeroed, accumulated over every q in ascending order,
 * then scaled by c = 1/(8 pi mu). */
static void assemble_row(int64_t m, int64_t N, const double *x, int64_t Q, const double *Xw,
                         const int32_t *nn, double eps, double c, double *dst, int64_t ld)
{
    for (int64_t jj = 0; jj < 3 * N; ++jj)
        for (int j = 0; j < 3; ++j) dst[j + jj * ld] = 0.0;
    for (int64_t q = 0; q < Q; ++q) {
        double r[3] = {x[4 * m + 0] - Xw[4 * q + 0], x[4 * m + 1] - Xw[4 * q + 1],
                       x[4 * m + 2] - Xw[4 * q + 2]};
        double S[9];
        or_stokeslet(r, eps, S);
        int64_t n = nn[q];
        double w = Xw[4 * q + 3];
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k) dst[j + (3 * n + k) * ld] += S[3 * j + k] * w;
    }
    for (int64_t jj = 0; jj < 3 * N; ++jj)
        for (int j = 0; j < 3; ++j) dst[j + jj * ld] *= c;
}

void or_assemble_stokeslet(int64_t N, const double *x, int64_t Q, const double *Xw,
                           const int32_t *nn, double eps, double mu, double *A, int64_t lda)
{
    double c = 1.0 / (8.0 * OR_PI * mu);
#pragma omp parallel for schedule(static)
    for (int64_t m = 0; m < N; ++m) assemble_row(m, N, x, Q, Xw, nn, eps, c, A + 3 * m, lda);
}

/* The same rows for a subset of force points: rows[r] = m gives
 * out[(3r+j) + (3n+k)*ldo] = A[3m+j, 3n+k] (ldo >= 3*nrows), the sampled
 * check of a matrix too large to assemble whole. */
void or_assemble_rows(int64_t nrows, const int64_t *rows, int64_t N, const double *x, int64_t Q,
                      const double *Xw, const int32_t *nn, double eps, double mu, double *out,
                      int64_t ldo)
{
    double c = 1.0 / (8.0 * OR_PI * mu);
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < nrows; ++r)
        assemble_row(rows[r], N, x, Q, Xw, nn, eps, c, out + 3 * r, ldo);
}

/* Rigid-body border of the swimming problem (Sec. 2 last paragraph, Sec. 4).
 * For the f-th free body b (base = 3N + 6f) and each of its force points m,
 * with r = x_m - x0_b:
 *   columns U:     A[3m+j, base+j]   = -1        (velocity -U)
 *   columns Omega: A[3m+j, base+3+k] = [r]x_jk   ([r]x Omega = r x Omega = -Omega x r)
 * so that row 3m+j reads  sum A_s f - U - Omega x r = (prescribed velocity).
 * Rows (force and moment balance, quadrature-weighted):
 *   A[base+j,   3n+j] = W_n = sum_q w_q nu[q,n]
 *   A[base+3+j, 3n+k] = [R_n]x_jk, R_n = sum_q w_q nu[q,n] (X_q - x0_b)
 * for every force point n of body b; the 6F x 6F corner is zero.
 * [v]x = [[0,-v3,v2],[v3,0,-v1],[-v2,v1,0]]. */
void or_border(int nbodies, const int64_t *n_off, const int64_t *q_off, const int32_t *kind,
               const double *x, const double *Xw, const int32_t *nn, const double *x0,
               double *A, int64_t lda)
{
    int64_t N = n_off[nbodies];
    int64_t Q = q_off[nbodies];
    int nfree = 0;
    for (int b = 0; b < nbodies; ++b) nfree += (kind[b] == OR_FREE);
    int64_t n = 3 * N + 6 * (int64_t)nfree;
    /* clear border rows and columns */
    for (int64_t i = 3 * N; i < n; ++i)
        for (int64_t j = 0; j < n; ++j) A[i + j * lda] = 0.0;
    for (int64_t j = 3 * N; j < n; ++j)
        for (int64_t i = 0; i < n; ++i) A[i + j * lda] = 0.0;
    double *W = (double *)calloc((size_t)N, sizeof(double));
    double *R = (double *)calloc((size_t)N * 3, sizeof(double));
    int32_t *body_of_n = (int32_t *)malloc(sizeof(int32_t) * (size_t)(N > 0 ? N : 1));
    for (int b = 0; b < nbodies; ++b)
        for (int64_t m = n_off[b]; m < n_off[b + 1]; ++m) body_of_n[m] = b;
    for (int64_t q = 0; q < Q; ++q) {
        int64_t m = nn[q];
        int b = body_of_n[m];
        double w = Xw[4 * q + 3];
        W[m] += w;
        for (int j = 0; j < 3; ++j) R[3 * m + j] += w * (Xw[4 * q + j] - x0[3 * b + j]);
    }
    int f = 0;
    for (int b = 0; b < nbodies; ++b) {
        if (kind[b] != OR_FREE) continue;
        int64_t base = 3 * N + 6 * (int64_t)f;
        for (int64_t m = n_off[b]; m < n_off[b + 1]; ++m) {
            double r[3] = {x[4 * m + 0] - x0[3 * b + 0], x[4 * m + 1] - x0[3 * b + 1],
                           x[4 * m + 2] - x0[3 * b + 2]};
            double cr[9] = {0.0, -r[2], r[1], r[2], 0.0, -r[0], -r[1], r[0], 0.0};
            double cR[9] = {0.0, -R[3 * m + 2], R[3 * m + 1], R[3 * m + 2], 0.0, -R[3 * m + 0],
                            -R[3 * m + 1], R[3 * m + 0], 0.0};
            for (int j = 0; j < 3; ++j) {
                A[(3 * m + j) + (base + j) * lda] = -1.0;
                for (int k = 0; k < 3; ++k) {
                    A[(3 * m + j) + (base + 3 + k) * lda] = cr[3 * j + k];
                    A[(base + 3 + j) + (3 * m + k) * lda] = cR[3 * j + k];
                }
                A[(base + j) + (3 * m + j) * lda] = W[m];
            }
        }
        ++f;
    }
    free(W);
    free(R);
    free(body_of_n);
}

/* Right-hand side: for force point m of body b, v = B_b xidot_m (the
 * prescribed deformation velocity, turned to the lab frame), plus
 * U_b + Omega_b x (x_m - x0_b) for a body with prescribed rigid motion;
 * static bodies give v = 0.  Force/moment rows get the external force and
 * moment on each free body (ext may be NULL for zero).  B is row-major per
 * body (9 doubles). */
void or_rhs(int nbodies, const int64_t *n_off, const int32_t *kind, const double *x,
            const double *x0, const double *B, const double *xidot, const double *U,
            const double *Om, const double *ext, double *b_out)
{
    int64_t N = n_off[nbodies];
    int f = 0;
    for (int b = 0; b < nbodies; ++b) {
        const double *Bb = B + 9 * b;
        for (int64_t m = n_off[b]; m < n_off[b + 1]; ++m) {
            double v[3] = {0.0, 0.0, 0.0};
            if (kind[b] != OR_STATIC)
                for (int r = 0; r < 3; ++r)
                    v[r] = Bb[3 * r + 0] * xidot[4 * m + 0] + Bb[3 * r + 1] * xidot[4 * m + 1] +
                           Bb[3 * r + 2] * xidot[4 * m + 2];
            if (kind[b] == OR_PRESCRIBED) {
                double r[3] = {x[4 * m + 0] - x0[3 * b + 0], x[4 * m + 1] - x0[3 * b + 1],
                               x[4 * m + 2] - x0[3 * b + 2]};
                const double *o = Om + 3 * b;
                double oxr[3] = {o[1] * r[2] - o[2] * r[1], o[2] * r[0] - o[0] * r[2],
                                 o[0] * r[1] - o[1] * r[0]};
                for (int j = 0; j < 3; ++j) v[j] += U[3 * b + j] + oxr[j];
            }
            for (int j = 0; j < 3; ++j) b_out[3 * m + j] = v[j];
        }
        if (kind[b] == OR_FREE) {
            for (int j = 0; j < 6; ++j) b_out[3 * N + 6 * f + j] = ext ? ext[6 * f + j] : 0.0;
            ++f;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Velocity at field points (Sec. 3: the NEAREST boundary integral evaluated  */
/* off the body, as used for particle tracking)                              */
/* ------------------------------------------------------------------------ */

/* u_j(x_p) = (1/(8 pi mu)) sum_q sum_k S^eps_jk(x_p - X_q) w_q f_k(n(q)) for
 * P field points xp (rows of 4 doubles), summed in ascending q; per q the
 * three terms (S_jk w_q) f_k are added in k order before joining the sum.
 * f holds 3 values per force point (the first 3N unknowns of the solution),
 * nn the nearest force point of each quadrature point.  u: rows of 4 doubles
 * (u_x, u_y, u_z, 0). */
void or_velocity(int64_t P, const double *xp, int64_t Q, const double *Xw, const int32_t *nn,
                 const double *f, double eps, double mu, double *u)
{
    double c = 1.0 / (8.0 * OR_PI * mu);
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < P; ++p) {
        double acc[3] = {0.0, 0.0, 0.0};
        for (int64_t q = 0; q < Q; ++q) {
            double r[3] = {xp[4 * p + 0] - Xw[4 * q + 0], xp[4 * p + 1] - Xw[4 * q + 1],
                           xp[4 * p + 2] - Xw[4 * q + 2]};
            double S[9];
            or_stokeslet(r, eps, S);
            double w = Xw[4 * q + 3];
            const double *fq = f + 3 * (int64_t)nn[q];
            for (int j = 0; j < 3; ++j) {
                double v = (S[3 * j + 0] * w) * fq[0] + (S[3 * j + 1] * w) * fq[1] +
                           (S[3 * j + 2] * w) * fq[2];
                acc[j] += v;
            }
        }
        for (int j = 0; j < 3; ++j) u[4 * p + j] = acc[j] * c;
        u[4 * p + 3] = 0.0;
    }
}

/* ------------------------------------------------------------------------ */
/* Dense solve (Sec. 4 step 3: the backslash solve)                          */
/* ------------------------------------------------------------------------ */

/* Right-looking LU with partial pivoting, unblocked (Doolittle, unit L).
 * Pivot = first row of maximal |a_ik| at or below the diagonal.  ipiv[k] is
 * the 0-based row swapped with row k.  Returns 0, or k+1 for the first
 * exactly-zero pivot (the factorisation still completes, as in LAPACK). */
int or_lu(int64_t n, double *A, int64_t lda, int32_t *ipiv)
{
    int info = 0;
    for (int64_t k = 0; k < n; ++k) {
        int64_t p = k;
        double amax = fabs(A[k + k * lda]);
        for (int64_t i = k + 1; i < n; ++i) {
            double a = fabs(A[i + k * lda]);
            if (a > amax) {
                amax = a;
                p = i;
            }
        }
        ipiv[k] = (int32_t)p;
        if (p != k)
            for (int64_t j = 0; j < n; ++j) {
                double t = A[k + j * lda];
                A[k + j * lda] = A[p + j * lda];
                A[p + j * lda] = t;
            }
        double piv = A[k + k * lda];
        if (piv == 0.0) {
            if (!info) info = (int)(k + 1);
            continue;
        }
        for (int64_t i = k + 1; i < n; ++i) A[i + k * lda] /= piv;
#pragma omp parallel for schedule(static)
        for (int64_t j = k + 1; j < n; ++j) {
            double a = A[k + j * lda];
            if (a != 0.0)
                for (int64_t i = k + 1; i < n; ++i) A[i + j * lda] -= A[i + k * lda] * a;
        }
    }
    return info;
}

/* Solve A x = b (trans == 0) or A^T x = b (trans != 0) in place in b from
 * the factors of or_lu. */
void or_lu_solve(int64_t n, const double *LU, int64_t lda, const int32_t *ipiv, double *b, int trans)
{
    if (!trans) {
        for (int64_t k = 0; k < n; ++k)
            if (ipiv[k] != k) {
                double t = b[k];
                b[k] = b[ipiv[k]];
                b[ipiv[k]] = t;
            }
        for (int64_t j = 0; j < n; ++j) {
            double bj = b[j];
            for (int64_t i = j + 1; i < n; ++i) b[i] -= LU[i + j * lda] * bj;
        }
        for (int64_t j = n - 1; j >= 0; --j) {
            b[j] /= LU[j + j * lda];
            double bj = b[j];
            for (int64_t i = 0; i < j; ++i) b[i] -= LU[i + j * lda] * bj;
        }
    } else {
        /* A^T = U^T L^T P: solve U^T y = b, L^T z = y, x = P^T z */
        for (int64_t j = 0; j < n; ++j) {
            double s = b[j];
            for (int64_t i = 0; i < j; ++i) s -= LU[i + j * lda] * b[i];
            b[j] = s / LU[j + j * lda];
        }
        for (int64_t j = n - 1; j >= 0; --j) {
            double s = b[j];
            for (int64_t i = j + 1; i < n; ++i) s -= LU[i + j * lda] * b[i];
            b[j] = s;
        }
        for (int64_t k = n - 1; k >= 0; --k)
            if (ipiv[k] != k) {
                double t = b[k];
                b[k] = b[ipiv[k]];
                b[ipiv[k]] = t;
            }
    }
}

/* Error-free transformations: Knuth's TwoSum and Dekker's TwoProduct with
 * Veltkamp splitting (factor 2^27 + 1); no fused multiply-add is used. */
static inline void two_sum(double a, double b, double *s, double *e)
{
    double t = a + b;
    double bb = t - a;
    *e = (a - (t - bb)) + (b - bb);
    *s = t;
}

static inline void split(double a, double *hi, double *lo)
{
    double c = 134217729.0 * a;
    double h = c - (c - a);
    *hi = h;
    *lo = a - h;
}

static inline void two_prod(double a, double b, double *p, double *e)
{
    double ah, al, bh, bl;
    double t = a * b;
    split(a, &ah, &al);
    split(b, &bh, &bl);
    *e = ((ah * bh - t) + ah * bl + al * bh) + al * bl;
    *p = t;
}

/* r = b - A x with every product and sum carried in double-double
 * (hi + lo), rounded to double at the end. */
void or_residual_dd(int64_t n, const double *A, int64_t lda, const double *x, const double *b,
                    double *r)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double sh = b[i], sl = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            double p, pe, s, se;
            two_prod(A[i + j * lda], x[j], &p, &pe);
            two_sum(sh, -p, &s, &se);
            sl += se - pe;
            sh = s;
        }
        double h, l;
        two_sum(sh, sl, &h, &l);
        r[i] = h;
    }
}

/* Iterative refinement with a double-double residual: x <- x + LU^{-1} r
 * until ||d||_inf <= tol ||x||_inf (or maxit steps).  Returns the number of
 * refinement steps taken. */
int or_refine(int64_t n, const double *A, int64_t lda, const double *LU, const int32_t *ipiv,
              const double *b, double *x, int maxit, double tol)
{
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    int it;
    for (it = 0; it < maxit; ++it) {
        or_residual_dd(n, A, lda, x, b, r);
        or_lu_solve(n, LU, lda, ipiv, r, 0);
        double dn = 0.0, xn = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            x[i] += r[i];
            if (fabs(r[i]) > dn) dn = fabs(r[i]);
            if (fabs(x[i]) > xn) xn = fabs(x[i]);
        }
        if (dn <= tol * xn) {
            ++it;
            break;
        }
    }
    free(r);
    return it;
}

/* 1-norm condition estimate kappa_1(A) = ||A||_1 * est(||A^{-1}||_1) with
 * Hager's algorithm (Hager 1984, as refined by Higham 1988). */
double or_cond1(int64_t n, const double *A, int64_t lda, const double *LU, const int32_t *ipiv)
{
    double anorm = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        double s = 0.0;
        for (int64_t i = 0; i < n; ++i) s += fabs(A[i + j * lda]);
        if (s > anorm) anorm = s;
    }
    double *v = (double *)malloc(sizeof(double) * (size_t)n);
    double *z = (double *)malloc(sizeof(double) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) v[i] = 1.0 / (double)n;
    double est = 0.0;
    int64_t jlast = -1;
    for (int it = 0; it < 5; ++it) {
        or_lu_solve(n, LU, lda, ipiv, v, 0);
        double y1 = 0.0;
        for (int64_t i = 0; i < n; ++i) y1 += fabs(v[i]);
        if (it > 0 && y1 <= est) break;
        est = y1;
        for (int64_t i = 0; i < n; ++i) z[i] = v[i] >= 0.0 ? 1.0 : -1.0;
        or_lu_solve(n, LU, lda, ipiv, z, 1);
        int64_t j = 0;
        for (int64_t i = 1; i < n; ++i)
            if (fabs(z[i]) > fabs(z[j])) j = i;
        if (j == jlast) break;
        jlast = j;
        for (int64_t i = 0; i < n; ++i) v[i] = 0.0;
        v[j] = 1.0;
    }
    free(v);
    free(z);
    return anorm * est;
}
