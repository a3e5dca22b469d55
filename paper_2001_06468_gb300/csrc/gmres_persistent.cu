// gmres_persistent.cu -- the GMRES-based iterative refinement of solve.cu
// (Carson & Higham 2018; the solve of Gallagher & Smith, Sec. 4 step 3) as
// ONE cooperative launch per right-hand side, for the factors that leave an
// explicit FP32 inverse M (Gauss-Jordan): the preconditioner is then a
// matrix-vector product, and the whole refinement -- FP64 residuals, Arnoldi
// with classical Gram-Schmidt applied twice, Givens rotations, the FP64
// update and the stopping rule -- runs on the device with no host round trip.
//
// Work split.  Matrix-vector products (A in FP64, M in FP32) are tiled over
// all CTAs as (row chunk, column split) tiles that write partial sums.  The
// length-n vector work (finishing the products, dot products, projections,
// norms, the update) is owned by the first DCH CTAs, CTA d owning elements
// [d*ED, (d+1)*ED): the same CTA that finishes a vector chunk also projects
// and normalises it, so only grid-wide quantities need a grid barrier.  GB300
// runs FP64 at a small fraction of its FP32 rate, so even the dot products
// are spread over many SMs.  Small state (the Hessenberg matrix, the Givens
// rotations, the least-squares solution, the stopping decisions) is kept in
// every CTA's shared memory and computed redundantly in the same order from
// the same values, so all CTAs take the same branches without a broadcast.
// Every reduction has a fixed order: the result is deterministic.
//
// The residual b - A x is computed to about u^2 by default (the
// three-precision form of Carson & Higham, whose solution reaches working
// accuracy for kappa(A) up to about 1/u) -- every product's rounded value
// summed exactly as an integer, its rounding error in FP64 (fx_add) -- or in
// FP64.
//
// Stopping rule: that of k_outer_check (solve.cu), plus one for very
// ill-conditioned systems, where an FP64 residual leaves corrections of about
// kappa(A) u that never shrink: once the corrections stagnate, the iteration
// also stops when the normwise backward error of x is at most 1e-15.
//
// Grid barriers are bounded: a CTA that waits more than kSpinLimit polls sets
// ST_TIMEOUT and returns, and every CTA returns at its next barrier once the
// flag is set.  The launch is cooperative, so all CTAs are co-resident.
#include <math.h>

#include <algorithm>

#include "nrs_internal.cuh"

namespace nrs {

constexpr int PG_THREADS = 256;
constexpr int PG_MAXM = 64;      // largest restart length of this kernel
constexpr int PG_MAXCH = 128;    // most chunk-owner CTAs
constexpr int MV_GROUPS = PG_THREADS / 32;  // column groups inside a product tile
constexpr int MV64_ROWS = 64;   // rows of an FP64 product tile: 32 row pairs x 8 column groups
constexpr int MV32_ROWS = 128;  // rows of an FP32 product tile: 32 row quads x 8 column groups

struct PgArgs {
    int64_t n, lda, ldv;
    const double *A;      // FP64 system matrix, column-major
    const float *M;       // explicit FP32 inverse (the preconditioner), column-major
    const double *b;
    double *x;            // in: starting guess unless cold; out: solution
    double *V;            // Krylov basis, n x (m+1), leading dimension ldv
    double *w;            // n: A v, then the residual
    double *part;         // partial sums of the FP64 products [splits][n]
    double *part32;       // partial sums of the FP32 products [splits][n]
    unsigned long long *part_fx;  // the exact residual's integer partial sums [splits][3][n]
    float2 *vf;           // input of the next preconditioner product as float pairs [n]
    const float2 *Adf;    // float-pair copy of A for the GMRES products, or null (FP64 A)
    float2 *Vf;           // the raw Krylov vector of the next product as float pairs [n]
    int dd;               // residual b - A x to u^2 (1: exact products, mv64fx_partial) or FP64 (0)
    double *dpart;        // reduction partials [3][PG_MAXCH][m+2]
    int32_t *bar;         // grid barrier: [0] arrivals since the launch ([1] unused)
    int32_t *status;
    double *out;          // [0] outer steps, [1] inner iterations, [2] converged,
                          // [3] ||d||_inf, [4] ||x||_inf, [5] exact residuals,
                          // [6] working-precision residuals (kept or not)
    double tol, floor, tol_in;
    int m, max_outer, cold, dch;
    int rc64, s64, rc32, s32;
    int64_t cps64, cps32, ed;
};

__device__ __forceinline__ int32_t pg_ld_acquire(const int32_t *p)
{
    int32_t v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void pg_st_release(int32_t *p, int32_t v)
{
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int32_t pg_ld_relaxed(const int32_t *p)
{
    int32_t v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// L2 prefetch for the matrix-vector products: the products stream each matrix
// once, with 8 to 24 warps an SM (the cooperative launch's occupancy), so
// the loads alone keep too few bytes in flight (3, 10 and 16 columns ahead
// measured slower than 6).  A warp's tile spans 512
// bytes of a column (64 rows of 8 bytes, or 128 rows of 4); lanes 0-3 each
// prefetch one of its four 128-byte lines six of its columns ahead of the
// warp's current one.  Lines whose first row is at or beyond n are skipped
// (such a line could run past the column's lda rows).
constexpr int PF_COLS = 6 * MV_GROUPS;

template <int ELEM>
__device__ __forceinline__ void pf_line(const void *m, int64_t lda, int64_t n, int64_t row0,
                                        int64_t j, int64_t j1, int lane)
{
    constexpr int rows_per_line = 128 / ELEM;
    const int64_t jp = j + PF_COLS, r = row0 + (int64_t)lane * rows_per_line;
    if (lane < 4 && jp < j1 && r < n) {
        const char *p = reinterpret_cast<const char *>(m) + (r + jp * lda) * ELEM;
        asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
    }
}

// Grid-wide barrier (bounded).  Returns false when the solve must stop.  One
// monotonic arrival counter per launch (zeroed before it): barrier number k
// is passed once the counter reaches k * gridDim.x, so the last arrival
// releases everyone with its own atomic (no reset, no second flag); tgt is
// the calling thread's running target.  Busy polling first, then polling
// with short sleeps.
__device__ bool grid_sync(const PgArgs &a, int *s_ok, int32_t &tgt)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        tgt += (int32_t)gridDim.x;
        __threadfence();
        atomicAdd(&a.bar[0], 1);
        long long spins = 0;
        while (pg_ld_acquire(&a.bar[0]) < tgt) {
            ++spins;
            if (spins > kSpinLimit ||
                ((spins & 1023) == 0 && (pg_ld_relaxed(a.status) & ST_TIMEOUT))) {
                atomicOr(a.status, ST_TIMEOUT);
                ok = 0;
                break;
            }
            if (spins > 64) __nanosleep(32);
        }
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

// part[s][i] = scale * sum_{j in split s} A[i, j] v[j] (|A[i, j]| when ABS).  A tile is 64 rows x
// one column split; lane l of warp g takes rows 2l, 2l+1 (one 16-byte load per
// column, 512 contiguous bytes per warp) and columns j0+g, j0+g+8, ...; the 8
// column groups are summed in shared memory in a fixed order.
template <bool ABS>
__device__ void mv64_partial(const PgArgs &a, const double *v, double scale, double *sm)
{
    const int64_t tiles = (int64_t)a.rc64 * a.s64;
    const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const int64_t rc = t % a.rc64, s = t / a.rc64;
        const int64_t i = rc * MV64_ROWS + 2 * lane;
        const int64_t j0 = s * a.cps64, j1 = min(a.n, j0 + a.cps64);
        double s0 = 0.0, s1 = 0.0;
        if (i < a.n) {
            const double *col = a.A + i;
#pragma unroll 8
            for (int64_t j = j0 + grp; j < j1; j += MV_GROUPS) {
                pf_line<8>(a.A, a.lda, a.n, rc * MV64_ROWS, j, j1, lane);
                const double2 x = __ldg(reinterpret_cast<const double2 *>(col + j * a.lda));
                if (ABS) {  // row sums of |A|
                    s0 += fabs(x.x);
                    s1 += fabs(x.y);
                } else {
                    const double vj = __ldcg(v + j);
                    s0 = fma(x.x, vj, s0);
                    s1 = fma(x.y, vj, s1);
                }
            }
        }
        sm[grp * MV64_ROWS + 2 * lane] = s0;
        sm[grp * MV64_ROWS + 2 * lane + 1] = s1;
        __syncthreads();
        if (threadIdx.x < MV64_ROWS) {
            const int64_t r = rc * MV64_ROWS + threadIdx.x;
            double acc = 0.0;
#pragma unroll
            for (int g = 0; g < MV_GROUPS; ++g) acc += sm[g * MV64_ROWS + threadIdx.x];
            if (r < a.n) a.part[s * a.n + r] = acc * scale;
        }
        __syncthreads();
    }
}

// part[s][i] = scale * sum_{j in split s} A[i, j] v[j] from the float-pair copy
// of A (a.Adf: hi + lo per entry, about 48 bits) and the raw Krylov vector as
// float pairs (a.Vf): double-float products and sums on the FP32 pipe (df_fma,
// plus the lo hi term), about 2^-46 of |A| |v|; the tile layout of
// mv64_partial, one 16-byte load per column for the two rows of a lane.
__device__ void mv64df_partial(const PgArgs &a, double scale, double *sm)
{
    const int64_t tiles = (int64_t)a.rc64 * a.s64;
    const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const int64_t rc = t % a.rc64, s = t / a.rc64;
        const int64_t i = rc * MV64_ROWS + 2 * lane;
        const int64_t j0 = s * a.cps64, j1 = min(a.n, j0 + a.cps64);
        float s0 = 0.0f, c0 = 0.0f, s1 = 0.0f, c1 = 0.0f;
        if (i < a.n) {
            const float2 *col = a.Adf + i;
#pragma unroll 4
            for (int64_t j = j0 + grp; j < j1; j += MV_GROUPS) {
                pf_line<8>(a.Adf, a.lda, a.n, rc * MV64_ROWS, j, j1, lane);
                const float4 x = __ldg(reinterpret_cast<const float4 *>(col + j * a.lda));
                const float2 vj = __ldcg(a.Vf + j);
                df_fma(x.x, vj, s0, c0);
                c0 = __fmaf_rn(x.y, vj.x, c0);
                df_fma(x.z, vj, s1, c1);
                c1 = __fmaf_rn(x.w, vj.x, c1);
            }
        }
        sm[grp * MV64_ROWS + 2 * lane] = (double)s0 + (double)c0;
        sm[grp * MV64_ROWS + 2 * lane + 1] = (double)s1 + (double)c1;
        __syncthreads();
        if (threadIdx.x < MV64_ROWS) {
            const int64_t r = rc * MV64_ROWS + threadIdx.x;
            double acc = 0.0;
#pragma unroll
            for (int g = 0; g < MV_GROUPS; ++g) acc += sm[g * MV64_ROWS + threadIdx.x];
            if (r < a.n) a.part[s * a.n + r] = acc * scale;
        }
        __syncthreads();
    }
}

// The residual's product, exact: fx[s][.][i] = sum_{j in split s} fl(A[i, j]
// v[j]) as a 192-bit integer (fx_add, anchor c) and part[s][i] = the FP64 sum
// of the products' rounding errors; the tile layout of mv64_partial.  The 8
// column groups are merged by a tree in shared memory (groups g + h into g,
// h = 4, 2, 1): exact for the integers, a fixed order for the error sums.
__device__ void mv64fx_partial(const PgArgs &a, const double *v, int c, double *sm)
{
    const int64_t tiles = (int64_t)a.rc64 * a.s64;
    const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;
    unsigned long long *su = reinterpret_cast<unsigned long long *>(sm);
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const int64_t rc = t % a.rc64, s = t / a.rc64;
        const int64_t i = rc * MV64_ROWS + 2 * lane;
        const int64_t j0 = s * a.cps64, j1 = min(a.n, j0 + a.cps64);
        Fx192 s0{0, 0, 0}, s1{0, 0, 0};
        double e0 = 0.0, e1 = 0.0;
        if (i < a.n) {
            const double *col = a.A + i;
#pragma unroll 4
            for (int64_t j = j0 + grp; j < j1; j += MV_GROUPS) {
                pf_line<8>(a.A, a.lda, a.n, rc * MV64_ROWS, j, j1, lane);
                const double2 x = __ldg(reinterpret_cast<const double2 *>(col + j * a.lda));
                const double vj = __ldcg(v + j);
                const double p0 = __dmul_rn(x.x, vj), p1 = __dmul_rn(x.y, vj);
                e0 = __dadd_rn(e0, __fma_rn(x.x, vj, -p0));
                e1 = __dadd_rn(e1, __fma_rn(x.y, vj, -p1));
                fx_add(s0, p0, c);
                fx_add(s1, p1, c);
            }
        }
        // tree over the column groups: slot k holds rows 2l, 2l+1 of group
        // h + k as 8 values (3 + 3 integer words, 2 error sums)
        for (int h = MV_GROUPS / 2; h >= 1; h >>= 1) {
            unsigned long long *q = su + ((grp - h) * 32 + lane) * 8;
            if (grp >= h && grp < 2 * h) {
                q[0] = s0.w0;
                q[1] = s0.w1;
                q[2] = s0.w2;
                q[3] = s1.w0;
                q[4] = s1.w1;
                q[5] = s1.w2;
                q[6] = (unsigned long long)__double_as_longlong(e0);
                q[7] = (unsigned long long)__double_as_longlong(e1);
            }
            __syncthreads();
            if (grp < h) {
                const unsigned long long *r = su + (grp * 32 + lane) * 8;
                fx_merge(s0, Fx192{r[0], r[1], r[2]});
                fx_merge(s1, Fx192{r[3], r[4], r[5]});
                e0 = __dadd_rn(e0, __longlong_as_double((long long)r[6]));
                e1 = __dadd_rn(e1, __longlong_as_double((long long)r[7]));
            }
            __syncthreads();
        }
        if (grp == 0 && i < a.n) {
            unsigned long long *f = a.part_fx + s * 3 * a.n;
            f[i] = s0.w0;
            f[a.n + i] = s0.w1;
            f[2 * a.n + i] = s0.w2;
            a.part[s * a.n + i] = e0;
            if (i + 1 < a.n) {
                f[i + 1] = s1.w0;
                f[a.n + i + 1] = s1.w1;
                f[2 * a.n + i + 1] = s1.w2;
                a.part[s * a.n + i + 1] = e1;
            }
        }
    }
}

// b[e] - sum over the column splits of the exact products and their error
// sums (mv64fx_partial), rounded once
__device__ __forceinline__ double residual_fx_at(const PgArgs &a, double be, int64_t e, int c)
{
    Fx192 S{0, 0, 0};
    double es = 0.0;
    for (int k = 0; k < a.s64; ++k) {
        const unsigned long long *f = a.part_fx + (int64_t)k * 3 * a.n;
        fx_merge(S, Fx192{__ldcg(f + e), __ldcg(f + a.n + e), __ldcg(f + 2 * a.n + e)});
        es = __dadd_rn(es, __ldcg(a.part + k * a.n + e));
    }
    return fx_residual(be, S, c, es);
}

// part32[s][i] = sum_{j in split s} M[i, j] v[j] with the FP32 entries of M
// and the FP64 vector v given as float pairs (a.vf): double-float products
// and sums on the FP32 pipe (df_fma), so the preconditioner is applied to
// about 2^-46 of |M| |v| -- a fixed operator for GMRES even where
// kappa(A) u_fp32 >> 1, which FP32 products of a rounded v (2^-24) are not.
// 128 rows per tile, lane l takes rows 4l..4l+3 (one 16-byte load per column);
// the 8 column groups are added in FP64 in a fixed order.
__device__ void mv32_partial(const PgArgs &a, double *sm)
{
    const int64_t tiles = (int64_t)a.rc32 * a.s32;
    const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const int64_t rc = t % a.rc32, s = t / a.rc32;
        const int64_t i = rc * MV32_ROWS + 4 * lane;
        const int64_t j0 = s * a.cps32, j1 = min(a.n, j0 + a.cps32);
        float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
        float c0 = 0.0f, c1 = 0.0f, c2 = 0.0f, c3 = 0.0f;
        if (i < a.n) {
            const float *col = a.M + i;
#pragma unroll 4
            for (int64_t j = j0 + grp; j < j1; j += MV_GROUPS) {
                pf_line<4>(a.M, a.lda, a.n, rc * MV32_ROWS, j, j1, lane);
                const float4 x = __ldg(reinterpret_cast<const float4 *>(col + j * a.lda));
                const float2 vj = __ldcg(a.vf + j);
                df_fma(x.x, vj, s0, c0);
                df_fma(x.y, vj, s1, c1);
                df_fma(x.z, vj, s2, c2);
                df_fma(x.w, vj, s3, c3);
            }
        }
        double *q = sm + grp * MV32_ROWS + 4 * lane;
        q[0] = (double)s0 + (double)c0;
        q[1] = (double)s1 + (double)c1;
        q[2] = (double)s2 + (double)c2;
        q[3] = (double)s3 + (double)c3;
        __syncthreads();
        if (threadIdx.x < MV32_ROWS) {
            const int64_t r = rc * MV32_ROWS + threadIdx.x;
            double acc = 0.0;
#pragma unroll
            for (int g = 0; g < MV_GROUPS; ++g) acc += sm[g * MV32_ROWS + threadIdx.x];
            if (r < a.n) a.part32[s * a.n + r] = acc;
        }
        __syncthreads();
    }
}

__device__ __forceinline__ double sum_parts(const PgArgs &a, int splits, int64_t e)
{
    double s = 0.0;
    for (int k = 0; k < splits; ++k) s += __ldcg(a.part + k * a.n + e);
    return s;
}

__device__ __forceinline__ double sum_parts32(const PgArgs &a, int64_t e)
{
    double s = 0.0;
    for (int k = 0; k < a.s32; ++k) s += __ldcg(a.part32 + k * a.n + e);
    return s;
}

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_max_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Block-wide sum in a fixed order; the result is returned to every thread.
__device__ double block_sum_all(double v, double *sred)
{
    v = warp_sum_d(v);
    if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    for (int i = 0; i < PG_THREADS / 32; ++i) s += sred[i];
    __syncthreads();
    return s;
}

__device__ double block_max_all(double v, double *sred)
{
    v = warp_max_d(v);
    if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    for (int i = 0; i < PG_THREADS / 32; ++i) s = fmax(s, sred[i]);
    __syncthreads();
    return s;
}

// dpart[region][d][i] = V_i . u over this CTA's chunk, for i <= j (one warp per i)
__device__ void chunk_dots(const PgArgs &a, int region, int j, const double *u, int64_t e0,
                           int64_t e1)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double *dp = a.dpart + ((int64_t)region * PG_MAXCH + blockIdx.x) * (a.m + 2);
    for (int i = wid; i <= j; i += PG_THREADS / 32) {
        const double *vi = a.V + (int64_t)i * a.ldv;
        double s = 0.0;
        for (int64_t e = e0 + lane; e < e1; e += 32) s = fma(__ldcg(vi + e), __ldcg(u + e), s);
        s = warp_sum_d(s);
        if (lane == 0) dp[i] = s;
    }
}

// Sum (or maximum) over chunks of dpart[region][d][slot], d < dch <= 256:
// thread d loads chunk d, then a fixed-order block reduction; every thread
// of the CTA gets the value.
__device__ double chunk_total(const PgArgs &a, int region, int slot, bool is_max, double *sred)
{
    double v = 0.0;
    if ((int)threadIdx.x < a.dch)
        v = __ldcg(a.dpart + ((int64_t)region * PG_MAXCH + threadIdx.x) * (a.m + 2) + slot);
    return is_max ? block_max_all(v, sred) : block_sum_all(v, sred);
}

// h[i] = sum over chunks d of dpart[region][d][i], i <= j, into shared memory
// (warp i sums the chunks with its lanes, then a fixed-order warp reduction)
__device__ void sum_dots(const PgArgs &a, int region, int j, double *h)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int i = wid; i <= j; i += PG_THREADS / 32) {
        double s = 0.0;
        for (int d = lane; d < a.dch; d += 32)
            s += __ldcg(a.dpart + ((int64_t)region * PG_MAXCH + d) * (a.m + 2) + i);
        s = warp_sum_d(s);
        if (lane == 0) h[i] = s;
    }
    __syncthreads();
}

// The residual r_e = res(e, b_e) of the CTA's own chunk into a.w and, as
// float pairs, a.vf (the next preconditioner product's input); the chunk's
// ||r||_inf (infinite if any r_e is not finite) and ||b||_inf into dp1[0],
// dp1[1] by its owner.
template <class Res>
__device__ __forceinline__ void store_residual(const PgArgs &a, int64_t e0, int64_t e1, bool owner,
                                               double *dp1, double *sred, Res res)
{
    double rmax = 0.0, bmax = 0.0;
    for (int64_t e = e0 + threadIdx.x; e < e1; e += PG_THREADS) {
        const double be = __ldg(a.b + e);
        const double re = res(e, be);
        a.w[e] = re;
        a.vf[e] = df_split(re);
        rmax = fmax(rmax, fabs(re));
        bmax = fmax(bmax, fabs(be));
        if (!isfinite(re)) rmax = INFINITY;
    }
    rmax = block_max_all(rmax, sred);
    bmax = block_max_all(bmax, sred);
    if (owner && threadIdx.x == 0) {
        dp1[0] = rmax;
        dp1[1] = bmax;
    }
}

// MINB = 3 caps the kernel at 85 registers a thread so that three CTAs share
// an SM (large systems, whose products stream from HBM, and the chains of a
// batch, which run side by side); MINB = 1 leaves the registers free for the
// one-CTA-per-SM grid of a lone system that sits in L2
// working-precision residuals in the refinement: the smallest backward error
// at which one is used, and the expected reduction of the backward error by
// one correction (negative: ten times the inner tolerance)
constexpr double PG_CHEAP_ETA = 1e-8;
constexpr double PG_CHEAP_RED = -1.0;

template <int MINB>
__global__ void __launch_bounds__(PG_THREADS, MINB) k_gmres_ir(PgArgs a)
{
    __shared__ double sH[(PG_MAXM + 1) * PG_MAXM];  // column-major, leading dimension PG_MAXM+1
    __shared__ double scs[PG_MAXM], ssn[PG_MAXM], sg[PG_MAXM + 1], sy[PG_MAXM];
    __shared__ double sh1[PG_MAXM + 1], sh2[PG_MAXM + 1];
    __shared__ double sred[PG_THREADS / 32];
    // product tiles: [0, 512) the FP64 sums; the preconditioner's tile and
    // the exact residual's group tree take all 1024
    __shared__ __align__(16) double smv[2 * MV_GROUPS * MV64_ROWS];
    __shared__ int s_ok;
    int32_t tgt = 0;  // grid barrier target (thread 0)
    static_assert(MV_GROUPS * MV32_ROWS <= 2 * MV_GROUPS * MV64_ROWS, "shared product tile");
    constexpr int LDH = PG_MAXM + 1;
    const int m = a.m;
    const int64_t n = a.n;
    const bool owner = (int)blockIdx.x < a.dch;
    const int64_t e0 = owner ? min(n, (int64_t)blockIdx.x * a.ed) : n;
    const int64_t e1 = owner ? min(n, e0 + a.ed) : n;
    const int nslot = m + 1;  // slot of norms in region 2 / maxima in region 0
    double *dp0 = a.dpart + (0 * PG_MAXCH + (int64_t)blockIdx.x) * (m + 2);
    double *dp1 = a.dpart + (1 * PG_MAXCH + (int64_t)blockIdx.x) * (m + 2);
    double *dp2 = a.dpart + (2 * PG_MAXCH + (int64_t)blockIdx.x) * (m + 2);

    if (a.cold) {  // x = M b
        for (int64_t e = e0 + threadIdx.x; e < e1; e += PG_THREADS) a.vf[e] = df_split(__ldg(a.b + e));
        if (!grid_sync(a, &s_ok, tgt)) return;
        mv32_partial(a, smv);
        if (!grid_sync(a, &s_ok, tgt)) return;
        for (int64_t e = e0 + threadIdx.x; e < e1; e += PG_THREADS) a.x[e] = sum_parts32(a, e);
        if (!grid_sync(a, &s_ok, tgt)) return;
    }
    int outer = 0, inner_total = 0, converged = 0;
    double dn = 0.0, xn = 0.0, dn_prev = 0.0, normA = -1.0;
    bool stagnant = false;
    if (a.dd) {
        // the exact residual's anchor needs ||A||_inf and ||x||_inf up front
        mv64_partial<true>(a, nullptr, 1.0, smv);
        if (!grid_sync(a, &s_ok, tgt)) return;
        double amax = 0.0, xmax = 0.0;
        for (int64_t e = e0 + threadIdx.x; e < e1; e += PG_THREADS) {
            amax = fmax(amax, sum_parts(a, a.s64, e));
            xmax = fmax(xmax, fabs(__ldcg(a.x + e)));
        }
        amax = block_max_all(amax, sred);
        xmax = block_max_all(xmax, sred);
        if (owner && threadIdx.x == 0) {
            dp1[2] = amax;
            dp0[1] = xmax;
        }
        if (!grid_sync(a, &s_ok, tgt)) return;
        normA = chunk_total(a, 1, 2, true, sred);
        xn = chunk_total(a, 0, 1, true, sred);
    }
    double eta_prev = INFINITY;  // backward error of the previous step's residual
    int n_exact = 0, n_work = 0;  // residuals formed: exact (or FP64), working precision
    for (outer = 0; outer < a.max_outer; ++outer) {
        // While the residual is large, a working-precision residual serves the
        // correction as well as the exact one: its error, about 2^-46 (|A| |x|)_i
        // (the float-pair product, or the FP64 one), is at most ~1e-4 of r once
        // the normwise backward error eta = ||r|| / (||A|| ||x|| + ||b||) is at
        // least PG_CHEAP_ETA, below the correction's own tolerance.  It is tried
        // first when the previous residual's eta, times the reduction a
        // correction is expected to bring, is still at least PG_CHEAP_ETA, and
        // kept if its own eta is; otherwise the exact residual is formed.  A
        // step on a working-precision residual never ends the refinement.
        bool cheap = false;
        const double red = PG_CHEAP_RED < 0.0 ? 10.0 * a.tol_in : PG_CHEAP_RED;
        if (a.dd && eta_prev * red >= PG_CHEAP_ETA) {
            if (a.Adf) {
                for (int64_t e = e0 + threadIdx.x; e < e1; e += PG_THREADS)
                    a.Vf[e] = df_split(__ldcg(a.x + e));
                if (!grid_sync(a, &s_ok, tgt)) return;
                mv64df_partial(a, 1.0, smv);
            } else {
                mv64_partial<false>(a, a.x, 1.0, smv);
            }
            if (!grid_sync(a, &s_ok, tgt)) return;
            store_residual(a, e0, e1, owner, dp1, sred,
                           [&](int64_t e, double be) { return be - sum_parts(a, a.s64, e); });
            if (!grid_sync(a, &s_ok, tgt)) return;
            const double rn = chunk_total(a, 1, 0, true, sred);
            const double bn = chunk_total(a, 1, 1, true, sred);
            const double eta = rn / (normA * xn + bn);
            cheap = isfinite(rn) && eta >= PG_CHEAP_ETA;
            eta_prev = eta;
            ++n_work;
        }
        if (!cheap) {
            // r = b - A x (exact products and error sums, or FP64), with
            // ||r||_inf and ||b||_inf per chunk; xn is ||x||_inf of this x
            const int fxc = a.dd ? fx_anchor(normA, xn) : 0;
            ++n_exact;
            if (a.dd)
                mv64fx_partial(a, a.x, fxc, smv);
            else
                mv64_partial<false>(a, a.x, 1.0, smv);
            if (!grid_sync(a, &s_ok, tgt)) return;
            store_residual(a, e0, e1, owner, dp1, sred, [&](int64_t e, double be) {
                return a.dd ? residual_fx_at(a, be, e, fxc) : be - sum_parts(a, a.s64, e);
            });
            if (!grid_sync(a, &s_ok, tgt)) return;
            if (a.dd) {
                const double rn = chunk_total(a, 1, 0, true, sred);
                const double bn = chunk_total(a, 1, 1, true, sred);
                eta_prev = rn / (normA * xn + bn);
            }
        }
        if (stagnant && !cheap) {
            // The corrections stopped shrinking.  If x already solves a nearby
            // system to working precision (normwise backward error
            // ||r|| / (||A|| ||x|| + ||b||) <= 1e-15), further steps only
            // chase rounding noise: stop.  ||A||_inf is computed once (at the start
            // when the residual is exact).
            if (normA < 0.0) {
                mv64_partial<true>(a, nullptr, 1.0, smv);
                if (!grid_sync(a, &s_ok, tgt)) return;
                double amax = 0.0;
                for (int64_t e = e0 + threadIdx.x; e < e1; e += PG_THREADS)
                    amax = fmax(amax, sum_parts(a, a.s64, e));
                amax = block_max_all(amax, sred);
                if (owner && threadIdx.x == 0) dp1[2] = amax;
                if (!grid_sync(a, &s_ok, tgt)) return;
                normA = chunk_total(a, 1, 2, true, sred);
            }
            const double rn = chunk_total(a, 1, 0, true, sred);
            const double bn = chunk_total(a, 1, 1, true, sred);
            if (rn <= 1e-15 * (normA * xn + bn)) {
                converged = 1;
                break;
            }
        }
        // V_0 = M r (raw), beta = ||V_0||
        mv32_partial(a, smv);
        if (!grid_sync(a, &s_ok, tgt)) return;
        {
            double s = 0.0;
            for (int64_t e = e0 + threadIdx.x; e < e1; e += PG_THREADS) {
                const double v = sum_parts32(a, e);
                a.V[e] = v;
                if (a.Adf) a.Vf[e] = df_split(v);
                s = fma(v, v, s);
            }
            s = block_sum_all(s, sred);
            if (owner && threadIdx.x == 0) dp2[nslot] = s;
        }
        if (!grid_sync(a, &s_ok, tgt)) return;
        const double beta = sqrt(chunk_total(a, 2, nslot, false, sred));
        if (!isfinite(beta)) {
            if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(a.status, ST_NONFINITE);
            break;
        }
        for (int i = threadIdx.x; i <= m; i += PG_THREADS) sg[i] = i == 0 ? beta : 0.0;
        __syncthreads();
        double sv = beta > 0.0 ? 1.0 / beta : 0.0;  // scale of the raw V_j
        int k = 0;
        bool bad = false;
        for (int j = 0; j < m; ++j) {
            double *Vj = a.V + (int64_t)j * a.ldv;
            double *u = a.V + (int64_t)(j + 1) * a.ldv;
            // w = A v_j (the FP64 matrix, or its float-pair copy and a.Vf)
            if (a.Adf)
                mv64df_partial(a, sv, smv);
            else
                mv64_partial<false>(a, Vj, sv, smv);
            if (!grid_sync(a, &s_ok, tgt)) return;
            for (int64_t e = e0 + threadIdx.x; e < e1; e += PG_THREADS) {
                Vj[e] = __ldcg(Vj + e) * sv;  // v_j normalised in place (own chunk)
                const double we = sum_parts(a, a.s64, e);
                a.w[e] = we;
                a.vf[e] = df_split(we);
            }
            if (!grid_sync(a, &s_ok, tgt)) return;
            // u = M w, then two classical Gram-Schmidt passes and the norm
            mv32_partial(a, smv);
            if (!grid_sync(a, &s_ok, tgt)) return;
            for (int64_t e = e0 + threadIdx.x; e < e1; e += PG_THREADS) u[e] = sum_parts32(a, e);
            __syncthreads();
            if (owner) chunk_dots(a, 0, j, u, e0, e1);
            if (!grid_sync(a, &s_ok, tgt)) return;
            sum_dots(a, 0, j, sh1);
            for (int64_t e = e0 + threadIdx.x; e < e1; e += PG_THREADS) {
                double s = __ldcg(u + e);
                for (int i = 0; i <= j; ++i) s = fma(-sh1[i], __ldcg(a.V + (int64_t)i * a.ldv + e), s);
                u[e] = s;
            }
            __syncthreads();
            if (owner) chunk_dots(a, 1, j, u, e0, e1);
            if (!grid_sync(a, &s_ok, tgt)) return;
            sum_dots(a, 1, j, sh2);
            {
                double s2 = 0.0;
                for (int64_t e = e0 + threadIdx.x; e < e1; e += PG_THREADS) {
                    double s = __ldcg(u + e);
                    for (int i = 0; i <= j; ++i)
                        s = fma(-sh2[i], __ldcg(a.V + (int64_t)i * a.ldv + e), s);
                    u[e] = s;
                    if (a.Adf) a.Vf[e] = df_split(s);
                    s2 = fma(s, s, s2);
                }
                s2 = block_sum_all(s2, sred);
                if (owner && threadIdx.x == 0) dp2[nslot] = s2;
            }
            if (!grid_sync(a, &s_ok, tgt)) return;
            const double hn = sqrt(chunk_total(a, 2, nslot, false, sred));
            // column j of H, previous rotations, the new rotation (every CTA, same order)
            double res = 0.0;
            if (threadIdx.x == 0) {
                double *col = sH + (int64_t)j * LDH;
                for (int i = 0; i <= j; ++i) col[i] = sh1[i] + sh2[i];
                col[j + 1] = hn;
                for (int i = 0; i < j; ++i) {
                    const double p = col[i], q = col[i + 1];
                    col[i] = scs[i] * p + ssn[i] * q;
                    col[i + 1] = -ssn[i] * p + scs[i] * q;
                }
                const double p = col[j], q = col[j + 1];
                const double r = hypot(p, q);
                const double c = r > 0.0 ? p / r : 1.0, s = r > 0.0 ? q / r : 0.0;
                scs[j] = c;
                ssn[j] = s;
                col[j] = r;
                col[j + 1] = 0.0;
                sg[j + 1] = -s * sg[j];
                sg[j] = c * sg[j];
                sred[0] = fabs(sg[j + 1]);
            }
            __syncthreads();
            res = sred[0];
            __syncthreads();
            k = j + 1;
            ++inner_total;
            if (!isfinite(res) || !isfinite(hn)) {
                bad = true;
                break;
            }
            sv = hn > 0.0 ? 1.0 / hn : 0.0;
            if (res <= a.tol_in * beta || hn == 0.0) break;
        }
        if (bad) {
            if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(a.status, ST_NONFINITE);
            break;
        }
        // y = R^{-1} g (k x k), then x += d = V y on the own chunk
        if (threadIdx.x == 0) {
            for (int i = k - 1; i >= 0; --i) {
                double s = sg[i];
                for (int l = i + 1; l < k; ++l) s -= sH[(int64_t)l * LDH + i] * sy[l];
                sy[i] = s / sH[(int64_t)i * LDH + i];
            }
        }
        __syncthreads();
        {
            double dmax = 0.0, xmax = 0.0;
            for (int64_t e = e0 + threadIdx.x; e < e1; e += PG_THREADS) {
                double s = 0.0;
                for (int i = 0; i < k; ++i) s = fma(sy[i], __ldcg(a.V + (int64_t)i * a.ldv + e), s);
                const double xe = __ldcg(a.x + e) + s;
                a.x[e] = xe;
                dmax = fmax(dmax, fabs(s));
                xmax = fmax(xmax, fabs(xe));
                if (!isfinite(s) || !isfinite(xe)) dmax = INFINITY;
            }
            dmax = block_max_all(dmax, sred);
            xmax = block_max_all(xmax, sred);
            if (owner && threadIdx.x == 0) {
                dp0[0] = dmax;
                dp0[1] = xmax;
            }
        }
        if (!grid_sync(a, &s_ok, tgt)) return;
        dn = chunk_total(a, 0, 0, true, sred);
        xn = chunk_total(a, 0, 1, true, sred);
        // stopping rule of k_outer_check (solve.cu)
        bool done = false;
        if (!isfinite(dn) || !isfinite(xn)) {
            if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(a.status, ST_NONFINITE);
            done = true;
        } else if (cheap) {
            // a correction from a working-precision residual: go on
        } else if (dn <= a.tol * xn) {
            done = true;
        } else if (dn_prev > 0.0 && dn * (dn / dn_prev) <= 1e-3 * a.tol * xn) {
            done = true;
        } else if (dn_prev > 0.0 && dn >= 0.5 * dn_prev && dn <= a.floor * xn) {
            done = true;
        }
        stagnant = dn_prev > 0.0 && dn >= 0.5 * dn_prev;
        dn_prev = dn;
        if (done) {
            converged = 1;
            ++outer;
            break;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.out[0] = outer;
        a.out[1] = inner_total;
        a.out[2] = converged;
        a.out[3] = dn;
        a.out[4] = xn;
        a.out[5] = n_exact;
        a.out[6] = n_work;
    }
}

// ---- host side ---------------------------------------------------------------

bool pg_supported(const Ctx &c) { return c.factored_prec != NRS_FP64 && c.max_inner <= PG_MAXM; }

// systems from this order up stream their matrices from HBM in the products
static constexpr int64_t PG_WIDE_N = 4096;

static const void *pg_kernel(const Ctx &c)
{
    return c.n >= PG_WIDE_N || c.pg_shared ? (const void *)k_gmres_ir<3>
                                           : (const void *)k_gmres_ir<1>;
}

int pg_grid(Ctx &c)
{
    if (c.pg_grid > 0) return c.pg_grid;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pg_kernel(c), PG_THREADS, 0);
    // one CTA per SM while barriers dominate (matrices in L2); three once the
    // products stream the matrices from HBM and need more bytes in flight
    // (measured at n = 27648: 2, 3, 4 CTAs an SM 280, 276, 282 ms per step)
    per_sm = std::max(1, std::min(per_sm, c.n >= PG_WIDE_N ? 3 : 1));
    c.pg_grid = per_sm * c.num_sms;
    return c.pg_grid;
}

int pg_max_coresident(const Ctx &c)
{
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pg_kernel(c), PG_THREADS, 0);
    return std::max(1, per_sm) * c.num_sms;
}

size_t pg_dpart_doubles(int max_inner) { return (size_t)3 * PG_MAXCH * (max_inner + 2); }

// The number of column splits s in [lo, 64] of a product with rc row tiles on a
// grid of G CTAs: the smallest whose rc s tiles fill their last wave to 97 %,
// else the best fill.
static int pick_splits(int64_t rc, int G, int lo)
{
    lo = std::max(1, std::min(lo, 64));
    int best = lo;
    double best_fill = -1.0;
    for (int s = lo; s <= 64; ++s) {
        const int64_t t = rc * s;
        const double fill = (double)t / (double)(ceil_div(t, G) * G);
        if (fill > best_fill + 1e-12) {
            best_fill = fill;
            best = s;
        }
        if (fill >= 0.97) break;
    }
    return best;
}

// One refinement of A x = b on the device.  Fills stats[0..4] (device) as
// described in PgArgs::out.
cudaError_t launch_gmres_persistent(Ctx &c, const double *b, double *x, bool cold, double *stats)
{
    PgArgs a{};
    const int G = pg_grid(c);
    a.n = c.n;
    a.lda = c.lda;
    a.ldv = c.lda;
    a.A = c.d_A64;
    a.M = c.d_A32;
    a.b = b;
    a.x = x;
    a.V = c.d_V;
    a.w = c.d_w;
    a.part = c.d_part;
    a.part32 = c.d_part32;
    a.part_fx = c.d_part_fx;
    a.vf = c.d_vf;
    a.Adf = c.arnoldi_df ? c.d_Adf : nullptr;
    a.Vf = c.d_vf2;
    a.dd = c.residual_dd;
    a.dpart = c.d_dpart;
    a.bar = c.d_bar;
    a.status = c.d_status;
    a.out = stats;
    a.tol = c.tol;
    a.floor = 1e-11;
    a.tol_in = c.tol_in;
    a.m = c.max_inner;
    a.max_outer = c.max_outer;
    a.cold = cold ? 1 : 0;
    a.rc64 = (int)ceil_div(c.n, MV64_ROWS);
    a.rc32 = (int)ceil_div(c.n, MV32_ROWS);
    // column splits: at least one tile per CTA, then the fewest splits whose
    // tiles fill the last wave of the grid to 97 % (at n = 27648: 432 row
    // tiles on 304 CTAs fill 71 % with one split, 99.5 % with seven)
    a.s64 = pick_splits(a.rc64, G, (int)std::max<int64_t>(1, ceil_div(G, a.rc64)));
    // at least 8 column splits for the FP32 product: each partial sum then
    // covers at most n / 8 columns before the splits are added in FP64
    a.s32 = pick_splits(a.rc32, G, (int)std::max<int64_t>(8, ceil_div(G, a.rc32)));
    a.s64 = (int)std::min<int64_t>(a.s64, c.n);
    a.s32 = (int)std::min<int64_t>(a.s32, c.n);
    a.cps64 = ceil_div(c.n, a.s64);
    a.cps32 = ceil_div(c.n, a.s32);
    // chunk owners: at most PG_MAXCH CTAs, about 64 elements each
    a.dch = (int)std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(PG_MAXCH, G),
                                                        ceil_div(c.n, 64)));
    a.ed = ceil_div(c.n, a.dch);
    a.dch = (int)ceil_div(c.n, a.ed);
    cudaError_t e = cudaMemsetAsync(c.d_bar, 0, 2 * sizeof(int32_t), c.stream);
    if (e != cudaSuccess) return e;
    void *args[] = {&a};
    c.tbeg(PH_KRYLOV);
    e = cudaLaunchCooperativeKernel(pg_kernel(c), G, PG_THREADS, args, 0, c.stream);
    c.tend(PH_KRYLOV);
    c.launches += 1;
    return e;
}

}  // namespace nrs
