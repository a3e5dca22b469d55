// solve.cu -- GMRES-based iterative refinement (Carson & Higham 2018) of the
// dense NEAREST system (Gallagher & Smith, Sec. 4 step 3):
//
//   x  = U^{-1} L^{-1} P b                       (or a supplied guess)
//   repeat:  r = b - A x                          (FP64, FP64 matrix)
//            solve A d = r by GMRES on M^{-1} A   (M = the LU factor)
//            x = x + d                            (FP64)
//   until ||d||_inf <= tol ||x||_inf.
//
// The triangular solves with the factor run as one cooperative launch per
// triangle: CTA k owns row block k, subtracts the contributions of earlier
// blocks as soon as their flags are published, solves its diagonal block and
// publishes its own flag (release/acquire at GPU scope).  Every wait is
// bounded; a wait that runs out sets ST_TIMEOUT and the kernel returns.
// All CTAs are co-resident (cooperative launch), and each CTA takes its blocks
// in dependency order, so the waits always end.
#include <math.h>

#include <algorithm>

#include "nrs_internal.cuh"

namespace nrs {

constexpr int TR_NB = 64;

// scalar slots of Ctx::d_scal
enum {
    SC_BETA = 0,
    SC_INNER_DONE = 1,
    SC_DN = 2,
    SC_XN = 3,
    SC_OUTER_DONE = 4,
    SC_RN = 5,
    SC_BN = 6,
    SC_AN = 7,
    SC_RES = 8,
    SC_DNPREV = 10,
    SC_STAG = 11,  // the last correction did not halve
    SC_FXA = 12,   // ||A||_inf and ||x||_inf: the anchor of the exact residual
    SC_FXX = 13,
    SC_COUNT = 16
};

__device__ __forceinline__ int32_t ld_acquire(const int32_t *p)
{
    int32_t v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int32_t *p, int32_t v)
{
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int32_t ld_relaxed(const int32_t *p)
{
    int32_t v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Thread 0 waits (bounded) for flags[j] == epoch; returns false if this or
// another CTA gave up, in which case every thread of the CTA must return.
__device__ __forceinline__ bool wait_flag(const int32_t *flags, int64_t j, int32_t epoch,
                                          int32_t *status, int *s_abort)
{
    if (threadIdx.x == 0) {
        long long spins = 0;
        int ok = 1;
        while (ld_acquire(&flags[j]) != epoch) {
            if (ld_relaxed(status) & ST_TIMEOUT) {
                ok = 0;
                break;
            }
            if (++spins > kSpinLimit) {
                atomicOr(status, ST_TIMEOUT);
                ok = 0;
                break;
            }
            __nanosleep(100);
        }
        *s_abort = !ok;
    }
    __syncthreads();
    return !*s_abort;
}

// y = L^{-1} P b  (L unit lower, P from rowperm), b in FP64, y in T.
template <typename T, int NB>
__global__ void __launch_bounds__(NB)
    k_trsv_lower(int64_t n, const T *__restrict__ LU, int64_t lda, const int32_t *__restrict__ rowperm,
                 const double *__restrict__ b, T *y, int32_t *flags, int32_t epoch, int32_t *status)
{
    __shared__ T ys[NB];
    __shared__ T sacc[NB];
    __shared__ T Ld[NB][NB + 1];
    __shared__ int s_abort;
    const int tid = threadIdx.x;
    const int64_t nblk = ceil_div(n, NB);
    for (int64_t blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
        const int64_t r0 = blk * NB;
        const int rows = (int)min((int64_t)NB, n - r0);
        const bool act = tid < rows;
        // the diagonal block does not depend on other blocks: stage it first
        if (act)
            for (int c = 0; c < rows; ++c) Ld[tid][c] = LU[r0 + tid + (r0 + c) * lda];
        T acc = act ? (T)b[rowperm[r0 + tid]] : T(0);
        for (int64_t j = 0; j < blk; ++j) {
            if (!wait_flag(flags, j, epoch, status, &s_abort)) return;
            ys[tid] = __ldcg(&y[j * NB + tid]);
            __syncthreads();
            if (act) {
                const T *col = LU + r0 + tid + j * NB * lda;
#pragma unroll 8
                for (int c = 0; c < NB; ++c) acc -= col[c * lda] * ys[c];
            }
            __syncthreads();
        }
        sacc[tid] = acc;
        __syncthreads();
        for (int c = 0; c < rows; ++c) {
            const T yc = sacc[c];
            if (act && tid > c) sacc[tid] -= Ld[tid][c] * yc;
            __syncthreads();
        }
        if (act) y[r0 + tid] = sacc[tid];
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            st_release(&flags[blk], epoch);
        }
    }
}

// x = U^{-1} y (U upper with its diagonal); the published blocks of x are
// kept in T (xw) for the other CTAs, and written to x in TO.
template <typename T, int NB, typename TO>
__global__ void __launch_bounds__(NB)
    k_trsv_upper(int64_t n, const T *__restrict__ LU, int64_t lda, const T *__restrict__ y, T *xw,
                 TO *__restrict__ x, int32_t *flags, int32_t epoch, int32_t *status)
{
    __shared__ T xs[NB];
    __shared__ T sacc[NB];
    __shared__ T xout[NB];
    __shared__ T Ud[NB][NB + 1];
    __shared__ int s_abort;
    const int tid = threadIdx.x;
    const int64_t nblk = ceil_div(n, NB);
    for (int64_t i = blockIdx.x; i < nblk; i += gridDim.x) {
        const int64_t blk = nblk - 1 - i;
        const int64_t r0 = blk * NB;
        const int rows = (int)min((int64_t)NB, n - r0);
        const bool act = tid < rows;
        if (act)
            for (int c = 0; c < rows; ++c) Ud[tid][c] = LU[r0 + tid + (r0 + c) * lda];
        T acc = act ? y[r0 + tid] : T(0);
        for (int64_t j = nblk - 1; j > blk; --j) {
            if (!wait_flag(flags, j, epoch, status, &s_abort)) return;
            const int cols = (int)min((int64_t)NB, n - j * NB);
            xs[tid] = tid < cols ? __ldcg(&xw[j * NB + tid]) : T(0);
            __syncthreads();
            if (act) {
                const T *col = LU + r0 + tid + j * NB * lda;
                for (int c = 0; c < cols; ++c) acc -= col[c * lda] * xs[c];
            }
            __syncthreads();
        }
        sacc[tid] = acc;
        __syncthreads();
        for (int c = rows - 1; c >= 0; --c) {
            const T xc = sacc[c] / Ud[c][c];
            if (act && tid < c) sacc[tid] -= Ud[tid][c] * xc;
            if (tid == c) xout[c] = xc;
            __syncthreads();
        }
        if (act) {
            xw[r0 + tid] = xout[tid];
            x[r0 + tid] = (TO)xout[tid];
        }
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            st_release(&flags[blk], epoch);
        }
    }
}

// ---- dense FP64 matrix-vector products --------------------------------------

constexpr int MV_THREADS = 128;

// part[s*n + i] = sum_{j in split s} A[i,j] v[j] (|A[i,j]| when ABS) for the
// FP64 matrix.  Each thread owns two adjacent rows (one 16-byte load per
// column), so a warp reads 512 contiguous bytes per column; rows i+1 >= n read
// the padding rows below n (allocated, results discarded).
template <bool ABS>
__global__ void __launch_bounds__(MV_THREADS)
    k_gemv_part(int64_t n, const double *__restrict__ A, int64_t lda, const double *__restrict__ v,
                double *__restrict__ part, int64_t cols_per_split)
{
    const int64_t i = ((int64_t)blockIdx.x * MV_THREADS + threadIdx.x) * 2;
    const int64_t j0 = (int64_t)blockIdx.y * cols_per_split;
    const int64_t j1 = min(n, j0 + cols_per_split);
    if (i >= n) return;
    double s0 = 0.0, s1 = 0.0;
    const double *a = A + i;
#pragma unroll 8
    for (int64_t j = j0; j < j1; ++j) {
        const double2 x = __ldg(reinterpret_cast<const double2 *>(a + j * lda));
        if (ABS) {
            s0 += fabs(x.x);
            s1 += fabs(x.y);
        } else {
            const double vj = __ldg(&v[j]);
            s0 += x.x * vj;
            s1 += x.y * vj;
        }
    }
    part[blockIdx.y * n + i] = s0;
    if (i + 1 < n) part[blockIdx.y * n + i + 1] = s1;
}

// vf[i] = v[i] as a float pair (the input of k_gemv32_part)
__global__ void k_split_vec(int64_t n, const double *__restrict__ v, float2 *__restrict__ vf)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) vf[i] = df_split(v[i]);
}

// Same with the FP32 explicit inverse of the Gauss-Jordan factor: four rows
// per thread (one 16-byte load per column), the FP64 vector as float pairs
// and double-float products and sums (df_fma), so the preconditioner is
// applied to about 2^-46 of |M| |v|.
__global__ void __launch_bounds__(MV_THREADS)
    k_gemv32_part(int64_t n, const float *__restrict__ M, int64_t lda, const float2 *__restrict__ vf,
                  double *__restrict__ part, int64_t cols_per_split)
{
    const int64_t i = ((int64_t)blockIdx.x * MV_THREADS + threadIdx.x) * 4;
    const int64_t j0 = (int64_t)blockIdx.y * cols_per_split;
    const int64_t j1 = min(n, j0 + cols_per_split);
    if (i >= n) return;
    float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
    float c0 = 0.0f, c1 = 0.0f, c2 = 0.0f, c3 = 0.0f;
    const float *a = M + i;
#pragma unroll 4
    for (int64_t j = j0; j < j1; ++j) {
        const float4 x = __ldg(reinterpret_cast<const float4 *>(a + j * lda));
        const float2 vj = __ldg(&vf[j]);
        df_fma(x.x, vj, s0, c0);
        df_fma(x.y, vj, s1, c1);
        df_fma(x.z, vj, s2, c2);
        df_fma(x.w, vj, s3, c3);
    }
    double *p = part + blockIdx.y * n + i;
    p[0] = (double)s0 + (double)c0;
    if (i + 1 < n) p[1] = (double)s1 + (double)c1;
    if (i + 2 < n) p[2] = (double)s2 + (double)c2;
    if (i + 3 < n) p[3] = (double)s3 + (double)c3;
}

// The residual's product, exact (fx_add): fx[(s*3 + w)*n + i] = word w of
// sum_{j in split s} fl(A[i,j] v[j]) as a 192-bit integer with the anchor of
// ||A||_inf = scal[SC_FXA], ||v||_inf = scal[SC_FXX]; part[s*n + i] = the
// FP64 sum of the products' rounding errors.  Two rows per thread as in
// k_gemv_part.
__global__ void __launch_bounds__(MV_THREADS)
    k_gemv_part_fx(int64_t n, const double *__restrict__ A, int64_t lda,
                   const double *__restrict__ v, const double *__restrict__ scal,
                   unsigned long long *__restrict__ fx, double *__restrict__ part,
                   int64_t cols_per_split)
{
    const int64_t i = ((int64_t)blockIdx.x * MV_THREADS + threadIdx.x) * 2;
    const int64_t j0 = (int64_t)blockIdx.y * cols_per_split;
    const int64_t j1 = min(n, j0 + cols_per_split);
    if (i >= n) return;
    const int c = fx_anchor(scal[SC_FXA], scal[SC_FXX]);
    Fx192 s0{0, 0, 0}, s1{0, 0, 0};
    double e0 = 0.0, e1 = 0.0;
    const double *a = A + i;
#pragma unroll 4
    for (int64_t j = j0; j < j1; ++j) {
        const double2 x = __ldg(reinterpret_cast<const double2 *>(a + j * lda));
        const double vj = __ldg(&v[j]);
        const double p0 = __dmul_rn(x.x, vj), p1 = __dmul_rn(x.y, vj);
        e0 = __dadd_rn(e0, __fma_rn(x.x, vj, -p0));
        e1 = __dadd_rn(e1, __fma_rn(x.y, vj, -p1));
        fx_add(s0, p0, c);
        fx_add(s1, p1, c);
    }
    unsigned long long *f = fx + blockIdx.y * 3 * n;
    f[i] = s0.w0;
    f[n + i] = s0.w1;
    f[2 * n + i] = s0.w2;
    part[blockIdx.y * n + i] = e0;
    if (i + 1 < n) {
        f[i + 1] = s1.w0;
        f[n + i + 1] = s1.w1;
        f[2 * n + i + 1] = s1.w2;
        part[blockIdx.y * n + i + 1] = e1;
    }
}

// out[i] = b[i] - (sum_s fx + sum_s part), the integer sums exact, rounded once
__global__ void k_gemv_finish_fx(int64_t n, const unsigned long long *__restrict__ fx,
                                 const double *__restrict__ part, int splits,
                                 const double *__restrict__ scal, const double *__restrict__ b,
                                 double *__restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = fx_anchor(scal[SC_FXA], scal[SC_FXX]);
    Fx192 S{0, 0, 0};
    double es = 0.0;
    for (int k = 0; k < splits; ++k) {
        const unsigned long long *f = fx + (int64_t)k * 3 * n;
        fx_merge(S, Fx192{f[i], f[n + i], f[2 * n + i]});
        es = __dadd_rn(es, part[k * n + i]);
    }
    out[i] = fx_residual(b[i], S, c, es);
}

// out[i] = b[i] - sum_s part (b != NULL), or sum_s part
__global__ void k_gemv_finish(int64_t n, const double *__restrict__ part, int splits,
                              const double *__restrict__ b, double *__restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = 0.0;
    for (int k = 0; k < splits; ++k) s += part[k * n + i];
    out[i] = b ? b[i] - s : s;
}

// ---- reductions (single block, fixed order => deterministic) --------------

constexpr int RED_THREADS = 1024;

__device__ double block_sum(double v)
{
    __shared__ double sh[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    if (threadIdx.x < 32)
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    return v;  // valid in thread 0
}

__device__ double block_max(double v)
{
    __shared__ double sh[32];
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    if (threadIdx.x < 32)
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    return v;
}

// v <- v / ||v||_2, scal[slot] = ||v||_2 (and g[0] = ||v|| when g != NULL)
__global__ void __launch_bounds__(RED_THREADS)
    k_normalize(int64_t n, double *__restrict__ v, double *__restrict__ scal, int slot,
                double *__restrict__ g, int32_t *status)
{
    __shared__ double s_nrm;
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += RED_THREADS) s += v[i] * v[i];
    s = block_sum(s);
    if (threadIdx.x == 0) {
        s_nrm = sqrt(s);
        scal[slot] = s_nrm;
        if (g) g[0] = s_nrm;
        if (!isfinite(s_nrm)) atomicOr(status, ST_NONFINITE);
    }
    __syncthreads();
    const double inv = s_nrm > 0.0 ? 1.0 / s_nrm : 0.0;
    for (int64_t i = threadIdx.x; i < n; i += RED_THREADS) v[i] *= inv;
}

// h[i] = V_i . w for i < k  (one block per basis vector)
__global__ void __launch_bounds__(RED_THREADS)
    k_dots(int64_t n, const double *__restrict__ V, int64_t ldv, const double *__restrict__ w,
           double *__restrict__ h)
{
    const double *vi = V + blockIdx.x * ldv;
    double s = 0.0;
    for (int64_t e = threadIdx.x; e < n; e += RED_THREADS) s += vi[e] * w[e];
    s = block_sum(s);
    if (threadIdx.x == 0) h[blockIdx.x] = s;
}

// w -= sum_{i<k} h[i] V_i
__global__ void k_project_out(int64_t n, const double *__restrict__ V, int64_t ldv,
                              const double *__restrict__ h, int k, double *__restrict__ w)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    double s = w[e];
    for (int i = 0; i < k; ++i) s -= h[i] * V[i * ldv + e];
    w[e] = s;
}

// Arnoldi bookkeeping and Givens rotations for column j of H ((m+1) x m,
// column-major); h1, h2 are the two classical Gram-Schmidt passes, hn the
// norm of the new vector.  Sets SC_INNER_DONE when |g_{j+1}| <= tol_in beta.
__global__ void k_givens(int j, int ldh, double *__restrict__ H, const double *__restrict__ h1,
                         const double *__restrict__ h2, double *__restrict__ gv, int m,
                         double *__restrict__ scal, double tol_in, int32_t *status)
{
    if (threadIdx.x != 0) return;
    double *col = H + (int64_t)j * ldh;
    for (int i = 0; i <= j; ++i) col[i] = h1[i] + h2[i];
    const double hn = scal[SC_RES + 1];
    col[j + 1] = hn;
    double *cs = gv, *sn = gv + m, *g = gv + 2 * m;
    for (int i = 0; i < j; ++i) {
        const double a = col[i], b = col[i + 1];
        col[i] = cs[i] * a + sn[i] * b;
        col[i + 1] = -sn[i] * a + cs[i] * b;
    }
    const double a = col[j], b = col[j + 1];
    const double r = hypot(a, b);
    const double c = r > 0.0 ? a / r : 1.0, s = r > 0.0 ? b / r : 0.0;
    cs[j] = c;
    sn[j] = s;
    col[j] = r;
    col[j + 1] = 0.0;
    g[j + 1] = -s * g[j];
    g[j] = c * g[j];
    const double res = fabs(g[j + 1]);
    scal[SC_RES] = res;
    if (!isfinite(res)) atomicOr(status, ST_NONFINITE);
    if (res <= tol_in * scal[SC_BETA] || hn == 0.0 || !isfinite(res)) scal[SC_INNER_DONE] = 1.0;
}

// y = R^{-1} g for the k x k leading triangle of H (single thread)
__global__ void k_lsq(int k, int ldh, const double *__restrict__ H, double *__restrict__ gv, int m)
{
    if (threadIdx.x != 0) return;
    const double *g = gv + 2 * m;
    double *y = gv + 3 * m + 1;
    for (int i = k - 1; i >= 0; --i) {
        double s = g[i];
        for (int l = i + 1; l < k; ++l) s -= H[(int64_t)l * ldh + i] * y[l];
        y[i] = s / H[(int64_t)i * ldh + i];
    }
}

// d = V y (first k columns); x += d
__global__ void k_update(int64_t n, const double *__restrict__ V, int64_t ldv,
                         const double *__restrict__ y, int k, double *__restrict__ x,
                         double *__restrict__ d)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    double s = 0.0;
    for (int i = 0; i < k; ++i) s += y[i] * V[i * ldv + e];
    d[e] = s;
    x[e] += s;
}

// SC_DN = ||d||_inf, SC_XN = ||x||_inf, SC_STAG = the correction did not
// halve.  SC_OUTER_DONE when SC_DN <= tol SC_XN,
// when the next correction predicted from the observed rate is far below that,
// or when refinement has stagnated at the accuracy an FP64 residual can
// deliver: the update no longer halves (SC_DN >= SC_DNPREV / 2) and is already
// below floor * SC_XN (the usual stopping rule of iterative refinement; the
// floor, 1e-11, stays an order of magnitude below the 1e-10 accuracy target).
__global__ void __launch_bounds__(RED_THREADS)
    k_outer_check(int64_t n, const double *__restrict__ d, const double *__restrict__ x,
                  double *__restrict__ scal, double tol, double floor, int32_t *status)
{
    double dn = 0.0, xn = 0.0;
    for (int64_t e = threadIdx.x; e < n; e += RED_THREADS) {
        dn = fmax(dn, fabs(d[e]));
        xn = fmax(xn, fabs(x[e]));
    }
    dn = block_max(dn);
    xn = block_max(xn);
    if (threadIdx.x == 0) {
        scal[SC_DN] = dn;
        scal[SC_XN] = xn;
        if (!isfinite(dn) || !isfinite(xn)) {
            atomicOr(status, ST_NONFINITE);
            scal[SC_OUTER_DONE] = 1.0;
        } else if (dn <= tol * xn) {
            scal[SC_OUTER_DONE] = 1.0;
        } else if (scal[SC_DNPREV] > 0.0 && dn * (dn / scal[SC_DNPREV]) <= 1e-3 * tol * xn) {
            // linear convergence at rate dn/dn_prev: the next correction is
            // predicted far below the tolerance
            scal[SC_OUTER_DONE] = 1.0;
        } else if (scal[SC_DNPREV] > 0.0 && dn >= 0.5 * scal[SC_DNPREV] && dn <= floor * xn) {
            scal[SC_OUTER_DONE] = 1.0;
        }
        scal[SC_STAG] = (scal[SC_DNPREV] > 0.0 && dn >= 0.5 * scal[SC_DNPREV]) ? 1.0 : 0.0;
        scal[SC_DNPREV] = dn;
    }
}

// ||v||_inf into scal[slot]
__global__ void __launch_bounds__(RED_THREADS)
    k_nrm_inf(int64_t n, const double *__restrict__ v, double *__restrict__ scal, int slot)
{
    double m = 0.0;
    for (int64_t e = threadIdx.x; e < n; e += RED_THREADS) m = fmax(m, fabs(v[e]));
    m = block_max(m);
    if (threadIdx.x == 0) scal[slot] = m;
}

// scal[slot] = max_i sum_s part[s*n + i] (||A||_inf from k_gemv_part<true>)
__global__ void __launch_bounds__(RED_THREADS)
    k_rowsum_max(int64_t n, const double *__restrict__ part, int splits, double *__restrict__ scal,
                 int slot)
{
    double m = 0.0;
    for (int64_t e = threadIdx.x; e < n; e += RED_THREADS) {
        double s = 0.0;
        for (int k = 0; k < splits; ++k) s += part[k * n + e];
        m = fmax(m, s);
    }
    m = block_max(m);
    if (threadIdx.x == 0) scal[slot] = m;
}

// ---- host side ---------------------------------------------------------------

template <typename K>
static int coop_grid(Ctx &c, K kernel, int threads, int64_t nblk)
{
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0);
    int64_t g = (int64_t)std::max(per_sm, 1) * c.num_sms;
    return (int)std::min<int64_t>(g, nblk);
}

// x (FP64, length n) = M^{-1} v with the factor of the last nrs_factor.
static cudaError_t apply_precond_impl(Ctx &c, const double *v, double *x);

static cudaError_t apply_precond(Ctx &c, const double *v, double *x)
{
    c.tbeg(PH_TRSV);
    cudaError_t e = apply_precond_impl(c, v, x);
    c.tend(PH_TRSV);
    c.launches += c.factored_prec != NRS_FP64 ? 3 : 2;
    return e;
}

static cudaError_t apply_precond_impl(Ctx &c, const double *v, double *x)
{
    const int64_t nblk = ceil_div(c.n, TR_NB);
    cudaError_t e;
    if (c.factored_prec != NRS_FP64) {
        // explicit inverse from the Gauss-Jordan factor: x = M v
        const int64_t cps = ceil_div(c.n, c.splits32);
        dim3 grid((unsigned)ceil_div(c.n, 4 * MV_THREADS), (unsigned)c.splits32);
        k_split_vec<<<(unsigned)ceil_div(c.n, 256), 256, 0, c.stream>>>(c.n, v, c.d_vf);
        k_gemv32_part<<<grid, MV_THREADS, 0, c.stream>>>(c.n, c.d_A32, c.lda, c.d_vf, c.d_part, cps);
        k_gemv_finish<<<(unsigned)ceil_div(c.n, 256), 256, 0, c.stream>>>(c.n, c.d_part, c.splits32,
                                                                          nullptr, x);
        return cudaGetLastError();
    }
    {
        auto kl = k_trsv_lower<double, TR_NB>;
        auto ku = k_trsv_upper<double, TR_NB, double>;
        int epoch = ++c.trsv_epoch;
        int64_t n = c.n, lda = c.lda;
        double *LU = c.d_LU64;
        double *y = c.d_t64;
        void *args_l[] = {&n, &LU, &lda, &c.d_rowperm, &v, &y, &c.d_flags, &epoch, &c.d_status};
        e = cudaLaunchCooperativeKernel((void *)kl, coop_grid(c, kl, TR_NB, nblk), TR_NB, args_l, 0,
                                        c.stream);
        if (e != cudaSuccess) return e;
        int epoch2 = ++c.trsv_epoch;
        double *xw = c.d_t64 + c.lda;  // second half of the FP64 work vector
        void *args_u[] = {&n, &LU, &lda, &y, &xw, &x, &c.d_flags, &epoch2, &c.d_status};
        return cudaLaunchCooperativeKernel((void *)ku, coop_grid(c, ku, TR_NB, nblk), TR_NB, args_u,
                                           0, c.stream);
    }
}

static void gemv(Ctx &c, const double *v, const double *b, double *out)
{
    const int64_t cps = ceil_div(c.n, c.splits64);
    dim3 grid((unsigned)ceil_div(c.n, 2 * MV_THREADS), (unsigned)c.splits64);
    c.tbeg(PH_GEMV);
    k_gemv_part<false><<<grid, MV_THREADS, 0, c.stream>>>(c.n, c.d_A64, c.lda, v, c.d_part, cps);
    k_gemv_finish<<<(unsigned)ceil_div(c.n, 256), 256, 0, c.stream>>>(c.n, c.d_part, c.splits64, b,
                                                                      out);
    c.tend(PH_GEMV);
    c.launches += 2;
}

// r = b - A x with the FP64 matrix: to about u^2 (exact products, fx_add)
// unless the context asks for a plain FP64 residual
static void residual(Ctx &c, const double *x, const double *b, double *r)
{
    if (!c.residual_dd) {
        gemv(c, x, b, r);
        return;
    }
    const int64_t cps = ceil_div(c.n, c.splits64);
    dim3 grid((unsigned)ceil_div(c.n, 2 * MV_THREADS), (unsigned)c.splits64);
    c.tbeg(PH_GEMV);
    // the anchor: ||A||_inf and ||x||_inf
    k_gemv_part<true><<<grid, MV_THREADS, 0, c.stream>>>(c.n, c.d_A64, c.lda, nullptr, c.d_part, cps);
    k_rowsum_max<<<1, RED_THREADS, 0, c.stream>>>(c.n, c.d_part, c.splits64, c.d_scal, SC_FXA);
    k_nrm_inf<<<1, RED_THREADS, 0, c.stream>>>(c.n, x, c.d_scal, SC_FXX);
    k_gemv_part_fx<<<grid, MV_THREADS, 0, c.stream>>>(c.n, c.d_A64, c.lda, x, c.d_scal,
                                                      c.d_part_fx, c.d_part, cps);
    k_gemv_finish_fx<<<(unsigned)ceil_div(c.n, 256), 256, 0, c.stream>>>(
        c.n, c.d_part_fx, c.d_part, c.splits64, c.d_scal, b, r);
    c.tend(PH_GEMV);
    c.launches += 5;
}

void enqueue_residual(Ctx &c, const double *x, const double *b, double *r) { residual(c, x, b, r); }

static double read_scalar(Ctx &c, int slot, cudaError_t *err)
{
    double v = 0.0;
    *err = cudaMemcpyAsync(&v, c.d_scal + slot, sizeof(double), cudaMemcpyDeviceToHost, c.stream);
    if (*err == cudaSuccess) *err = cudaStreamSynchronize(c.stream);
    return v;
}

void enqueue_backward_error(Ctx &c, const double *b, const double *x, double *out3)
{
    residual(c, x, b, c.d_r);
    k_nrm_inf<<<1, RED_THREADS, 0, c.stream>>>(c.n, c.d_r, out3, 0);
    const int64_t cps = ceil_div(c.n, c.splits64);
    dim3 grid((unsigned)ceil_div(c.n, 2 * MV_THREADS), (unsigned)c.splits64);
    k_gemv_part<true><<<grid, MV_THREADS, 0, c.stream>>>(c.n, c.d_A64, c.lda, nullptr, c.d_part, cps);
    k_gemv_finish<<<(unsigned)ceil_div(c.n, 256), 256, 0, c.stream>>>(c.n, c.d_part, c.splits64,
                                                                      nullptr, c.d_w);
    k_nrm_inf<<<1, RED_THREADS, 0, c.stream>>>(c.n, c.d_w, out3, 1);
    k_nrm_inf<<<1, RED_THREADS, 0, c.stream>>>(c.n, b, out3, 2);
    c.launches += 5;
}

cudaError_t choose_start(Ctx &c, const double *b, const double *xp, double *xc, double *x0,
                         double *norms)
{
    join_assembly(c);
    cudaError_t e = apply_precond(c, b, xc);
    if (e != cudaSuccess) return e;
    gemv(c, xp, b, c.d_r);
    c.tbeg(PH_KRYLOV);
    k_nrm_inf<<<1, RED_THREADS, 0, c.stream>>>(c.n, c.d_r, norms, 0);
    c.tend(PH_KRYLOV);
    gemv(c, xc, b, c.d_r);
    c.tbeg(PH_KRYLOV);
    k_nrm_inf<<<1, RED_THREADS, 0, c.stream>>>(c.n, c.d_r, norms, 1);
    pick_start(c, xp, xc, norms, x0);
    c.tend(PH_KRYLOV);
    c.launches += 2;
    return cudaGetLastError();
}

static nrs_status finish_solve(Ctx &c, const double *b, double *x, nrs_solve_report *rep,
                               int *inner_out, int outer, int inner_total, bool converged,
                               const double *dn_xn = nullptr);

static nrs_status run_gmres_ir_device(Ctx &c, const double *b, double *x, const double *x0,
                                      nrs_solve_report *rep, int *inner_out)
{
    cudaError_t e = cudaSuccess;
    if (x0) e = cudaMemcpyAsync(x, x0, sizeof(double) * c.n, cudaMemcpyDeviceToDevice, c.stream);
    if (e == cudaSuccess) e = launch_gmres_persistent(c, b, x, x0 == nullptr, c.d_pg_stats);
    double st[7] = {0, 0, 0, 0, 0, 0, 0};
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(st, c.d_pg_stats, sizeof(st), cudaMemcpyDeviceToHost, c.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    if (e != cudaSuccess) {
        c.err = std::string("CUDA error in solve: ") + cudaGetErrorString(e);
        return NRS_ECUDA;
    }
    c.res_exact_total += (int64_t)st[5];
    c.res_work_total += (int64_t)st[6];
    return finish_solve(c, b, x, rep, inner_out, (int)st[0], (int)st[1], st[2] != 0.0, st + 3);
}

nrs_status run_gmres_ir(Ctx &c, const double *b, double *x, const double *x0, nrs_solve_report *rep,
                        int *inner_out)
{
    join_assembly(c);  // the FP64 matrix of the residuals
    if (c.solve_mode == 0 && pg_supported(c)) return run_gmres_ir_device(c, b, x, x0, rep, inner_out);
    const int64_t n = c.n;
    const int m = c.max_inner;
    const int64_t ldv = c.lda;
    const int ldh = m + 1;
    const double tol_in = c.tol_in;
    cudaError_t e = cudaSuccess;
#define CKE(call)                                                           \
    do {                                                                    \
        e = (call);                                                         \
        if (e != cudaSuccess) {                                             \
            c.err = std::string("CUDA error in solve: ") + cudaGetErrorString(e); \
            return NRS_ECUDA;                                               \
        }                                                                   \
    } while (0)
    CKE(cudaMemsetAsync(c.d_scal, 0, sizeof(double) * SC_COUNT, c.stream));
    if (x0) {
        CKE(cudaMemcpyAsync(x, x0, sizeof(double) * n, cudaMemcpyDeviceToDevice, c.stream));
    } else {
        CKE(apply_precond(c, b, x));
    }
    int outer = 0, inner_total = 0;
    bool converged = false;
    double *h1 = c.d_scal + SC_COUNT;
    double *h2 = h1 + (m + 1);
    bool have_an = false;
    for (outer = 0; outer < c.max_outer; ++outer) {
        residual(c, x, b, c.d_r);  // r = b - A x
        if (outer > 0) {
            // stagnating corrections: stop once the normwise backward error of
            // x is at most 1e-15 (as in gmres_persistent.cu)
            const double stag = read_scalar(c, SC_STAG, &e);
            if (e != cudaSuccess) CKE(e);
            if (stag != 0.0) {
                k_nrm_inf<<<1, RED_THREADS, 0, c.stream>>>(n, c.d_r, c.d_scal, SC_RN);
                k_nrm_inf<<<1, RED_THREADS, 0, c.stream>>>(n, b, c.d_scal, SC_BN);
                c.launches += 2;
                if (!have_an) {
                    const int64_t cps = ceil_div(c.n, c.splits64);
                    dim3 grid((unsigned)ceil_div(c.n, 2 * MV_THREADS), (unsigned)c.splits64);
                    k_gemv_part<true><<<grid, MV_THREADS, 0, c.stream>>>(c.n, c.d_A64, c.lda,
                                                                         nullptr, c.d_part, cps);
                    k_gemv_finish<<<(unsigned)ceil_div(c.n, 256), 256, 0, c.stream>>>(
                        c.n, c.d_part, c.splits64, nullptr, c.d_w);
                    k_nrm_inf<<<1, RED_THREADS, 0, c.stream>>>(n, c.d_w, c.d_scal, SC_AN);
                    c.launches += 3;
                    have_an = true;
                }
                double sc[SC_COUNT];
                CKE(cudaMemcpyAsync(sc, c.d_scal, sizeof(sc), cudaMemcpyDeviceToHost, c.stream));
                CKE(cudaStreamSynchronize(c.stream));
                if (sc[SC_RN] <= 1e-15 * (sc[SC_AN] * sc[SC_XN] + sc[SC_BN])) {
                    converged = true;
                    break;
                }
            }
        }
        double *V0 = c.d_V;
        CKE(apply_precond(c, c.d_r, V0));
        c.tbeg(PH_KRYLOV);
        CKE(cudaMemsetAsync(c.d_gv, 0, sizeof(double) * (4 * m + 2), c.stream));
        CKE(cudaMemsetAsync(c.d_scal + SC_INNER_DONE, 0, sizeof(double), c.stream));
        k_normalize<<<1, RED_THREADS, 0, c.stream>>>(n, V0, c.d_scal, SC_BETA, c.d_gv + 2 * m,
                                                     c.d_status);
        c.tend(PH_KRYLOV);
        c.launches += 1;
        int k = 0;
        for (int j = 0; j < m; ++j) {
            double *Vj = c.d_V + j * ldv;
            double *Vn = c.d_V + (j + 1) * ldv;
            gemv(c, Vj, nullptr, c.d_w);     // w = A v_j
            CKE(apply_precond(c, c.d_w, Vn));  // v_{j+1} = M^{-1} w
            const unsigned ge = (unsigned)ceil_div(n, 256);
            c.tbeg(PH_KRYLOV);
            k_dots<<<j + 1, RED_THREADS, 0, c.stream>>>(n, c.d_V, ldv, Vn, h1);
            k_project_out<<<ge, 256, 0, c.stream>>>(n, c.d_V, ldv, h1, j + 1, Vn);
            k_dots<<<j + 1, RED_THREADS, 0, c.stream>>>(n, c.d_V, ldv, Vn, h2);
            k_project_out<<<ge, 256, 0, c.stream>>>(n, c.d_V, ldv, h2, j + 1, Vn);
            k_normalize<<<1, RED_THREADS, 0, c.stream>>>(n, Vn, c.d_scal, SC_RES + 1, nullptr,
                                                         c.d_status);
            k_givens<<<1, 32, 0, c.stream>>>(j, ldh, c.d_H, h1, h2, c.d_gv, m, c.d_scal, tol_in,
                                             c.d_status);
            c.tend(PH_KRYLOV);
            c.launches += 6;
            k = j + 1;
            ++inner_total;
            double done = read_scalar(c, SC_INNER_DONE, &e);
            if (e != cudaSuccess) CKE(e);
            if (done != 0.0) break;
        }
        c.tbeg(PH_KRYLOV);
        k_lsq<<<1, 32, 0, c.stream>>>(k, ldh, c.d_H, c.d_gv, m);
        k_update<<<(unsigned)ceil_div(n, 256), 256, 0, c.stream>>>(n, c.d_V, ldv, c.d_gv + 3 * m + 1,
                                                                   k, x, c.d_w);
        k_outer_check<<<1, RED_THREADS, 0, c.stream>>>(n, c.d_w, x, c.d_scal, c.tol, 1e-11,
                                                       c.d_status);
        c.tend(PH_KRYLOV);
        c.launches += 3;
        double od = read_scalar(c, SC_OUTER_DONE, &e);
        if (e != cudaSuccess) CKE(e);
        if (od != 0.0) {
            converged = true;
            ++outer;
            break;
        }
    }
#undef CKE
    c.res_exact_total += outer;  // one residual (exact, or FP64) a refinement step
    return finish_solve(c, b, x, rep, inner_out, outer, inner_total, converged);
}

// Status word, statistics and (when asked) the backward error of a finished
// solve; dn_xn (host, or NULL to read them from d_scal) = ||d||_inf, ||x||_inf
// of the last refinement step.
static nrs_status finish_solve(Ctx &c, const double *b, double *x, nrs_solve_report *rep,
                               int *inner_out, int outer, int inner_total, bool converged,
                               const double *dn_xn)
{
    const int64_t n = c.n;
    cudaError_t e = cudaSuccess;
    c.solves += 1;
    c.outer_total += outer;
    c.inner_total += inner_total;
#define CKE(call)                                                           \
    do {                                                                    \
        e = (call);                                                         \
        if (e != cudaSuccess) {                                             \
            c.err = std::string("CUDA error in solve: ") + cudaGetErrorString(e); \
            return NRS_ECUDA;                                               \
        }                                                                   \
    } while (0)
    int32_t st = 0;
    CKE(cudaMemcpyAsync(&st, c.d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, c.stream));
    CKE(cudaStreamSynchronize(c.stream));
    CKE(cudaMemsetAsync(c.d_status, 0, sizeof(int32_t), c.stream));  // reported: clear
    if (inner_out) *inner_out = inner_total;
    if (rep) {
        // backward error ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf)
        residual(c, x, b, c.d_r);
        k_nrm_inf<<<1, RED_THREADS, 0, c.stream>>>(n, c.d_r, c.d_scal, SC_RN);
        k_nrm_inf<<<1, RED_THREADS, 0, c.stream>>>(n, b, c.d_scal, SC_BN);
        {
            const int64_t cps = ceil_div(c.n, c.splits64);
            dim3 grid((unsigned)ceil_div(c.n, 2 * MV_THREADS), (unsigned)c.splits64);
            k_gemv_part<true><<<grid, MV_THREADS, 0, c.stream>>>(c.n, c.d_A64, c.lda, nullptr,
                                                                 c.d_part, cps);
            k_gemv_finish<<<(unsigned)ceil_div(c.n, 256), 256, 0, c.stream>>>(
                c.n, c.d_part, c.splits64, nullptr, c.d_w);
            k_nrm_inf<<<1, RED_THREADS, 0, c.stream>>>(n, c.d_w, c.d_scal, SC_AN);
        }
        double sc[SC_COUNT];
        CKE(cudaMemcpyAsync(sc, c.d_scal, sizeof(sc), cudaMemcpyDeviceToHost, c.stream));
        CKE(cudaStreamSynchronize(c.stream));
        rep->outer = outer;
        rep->inner = inner_total;
        rep->converged = converged ? 1 : 0;
        const double dn = dn_xn ? dn_xn[0] : sc[SC_DN], xn = dn_xn ? dn_xn[1] : sc[SC_XN];
        rep->backward_err = sc[SC_RN] / (sc[SC_AN] * xn + sc[SC_BN]);
        rep->last_update = xn > 0 ? dn / xn : 0.0;
        rep->status = NRS_OK;
    }
#undef CKE
    nrs_status out = NRS_OK;
    if (st & ST_TIMEOUT) out = NRS_ETIMEOUT;
    else if (st & ST_NONFINITE) out = NRS_ENONFINITE;
    else if (!converged) out = NRS_ENOCONV;
    if (rep) rep->status = out;
    if (out != NRS_OK) {
        c.err = out == NRS_ETIMEOUT     ? "a bounded device wait ran out"
                : out == NRS_ENONFINITE ? "non-finite value in the refinement"
                                        : "refinement did not reach the tolerance";
    }
    return out;
}

}  // namespace nrs
