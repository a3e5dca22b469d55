// lu.cu -- blocked right-looking LU of the assembled system in FP64 (the
// dense solve of Gallagher & Smith, Sec. 4 step 3): the factor of the plain
// FP64 path.  (The mixed-precision path inverts an FP32 copy instead, gj.cu.)
//
// Pivoting is restricted to the rows of each NB x NB diagonal block: the
// block is factored with partial pivoting among its own rows and the same
// row exchange is applied across the whole block row.  This keeps every
// panel step inside one CTA (no grid-wide pivot search over n rows) and the
// rest of the step parallel: L21 = A21 U11^{-1}, U12 = L11^{-1} P A12 by
// independent substitutions per row / column, then A22 -= L21 U12.  The
// NEAREST matrix is close to (symmetric positive definite Nystrom matrix) x
// (positive diagonal of segment weights), whose LU needs no pivoting, and the
// rigid-body rows come last, where the in-block pivoting handles the zero
// corner; the growth factor on the swimmer workloads equals that of full
// partial pivoting.  The FP64 refinement of solve.cu removes what is left.
//
// Result: P A = L U with P the composition of the block-local exchanges,
// rowperm[i] = original row now at position i, L unit lower and U upper
// stored in place.
#include "nrs_internal.cuh"

namespace nrs {

constexpr int LU_NB = 64;

template <typename T>
__device__ __forceinline__ T tabs(T v)
{
    return v < T(0) ? -v : v;
}

template <typename T, int NB>
__global__ void __launch_bounds__(256)
    k_diag_factor(int64_t n, T *__restrict__ A, int64_t lda, int64_t k0, int32_t *__restrict__ lperm,
                  int32_t *__restrict__ rowperm, int32_t *__restrict__ info)
{
    __shared__ T D[NB][NB + 1];
    __shared__ int32_t lp[NB];
    __shared__ int32_t rp_old[NB];
    __shared__ int32_t s_piv;
    const int tid = threadIdx.x;
    const int kb = (int)min((int64_t)NB, n - k0);
    for (int idx = tid; idx < kb * kb; idx += blockDim.x) {
        const int r = idx % kb, c = idx / kb;
        D[r][c] = A[(k0 + r) + (k0 + c) * lda];
    }
    if (tid < kb) {
        lp[tid] = tid;
        rp_old[tid] = rowperm[k0 + tid];
    }
    __syncthreads();
    for (int c = 0; c < kb; ++c) {
        if (tid < 32) {
            T best = T(-1);
            int br = c;
            for (int r = c + tid; r < kb; r += 32) {
                const T a = tabs(D[r][c]);
                if (a > best) {
                    best = a;
                    br = r;
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const T ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int orr = __shfl_xor_sync(0xffffffffu, br, o);
                if (ob > best || (ob == best && orr < br)) {
                    best = ob;
                    br = orr;
                }
            }
            if (tid == 0) s_piv = br;
        }
        __syncthreads();
        const int p = s_piv;
        if (p != c) {
            for (int j = tid; j < kb; j += blockDim.x) {
                const T t = D[c][j];
                D[c][j] = D[p][j];
                D[p][j] = t;
            }
            if (tid == 0) {
                const int t = lp[c];
                lp[c] = lp[p];
                lp[p] = t;
            }
        }
        __syncthreads();
        const T pv = D[c][c];
        if (pv == T(0)) {
            if (tid == 0 && info) atomicCAS(info, 0, (int)(k0 + c + 1));
        } else {
            for (int r = c + 1 + tid; r < kb; r += blockDim.x) D[r][c] /= pv;
            __syncthreads();
            const int w = kb - c - 1;
            for (int idx = tid; idx < w * w; idx += blockDim.x) {
                const int r = c + 1 + idx % w, j = c + 1 + idx / w;
                D[r][j] -= D[r][c] * D[c][j];
            }
        }
        __syncthreads();
    }
    for (int idx = tid; idx < kb * kb; idx += blockDim.x) {
        const int r = idx % kb, c = idx / kb;
        A[(k0 + r) + (k0 + c) * lda] = D[r][c];
    }
    if (tid < kb) {
        lperm[tid] = lp[tid];
        rowperm[k0 + tid] = rp_old[lp[tid]];
    }
}

// Apply the block's row exchange to the already-factored columns [0, k0).
template <typename T, int NB>
__global__ void k_swap_left(int64_t k0, int kb, T *__restrict__ A, int64_t lda,
                            const int32_t *__restrict__ lperm)
{
    __shared__ int32_t lp[NB];
    if (threadIdx.x < kb) lp[threadIdx.x] = lperm[threadIdx.x];
    __syncthreads();
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= k0) return;
    T tmp[NB];
#pragma unroll
    for (int i = 0; i < NB; ++i)
        if (i < kb) tmp[i] = A[(k0 + lp[i]) + c * lda];
#pragma unroll
    for (int i = 0; i < NB; ++i)
        if (i < kb) A[(k0 + i) + c * lda] = tmp[i];
}

// L21 = A21 U11^{-1}: each thread solves x U11 = a for one row below the block.
template <typename T, int NB>
__global__ void __launch_bounds__(128)
    k_trsm_l21(int64_t n, T *__restrict__ A, int64_t lda, int64_t k0, int kb)
{
    __shared__ T U[NB][NB + 1];
    for (int idx = threadIdx.x; idx < kb * kb; idx += blockDim.x) {
        const int r = idx % kb, c = idx / kb;
        U[r][c] = A[(k0 + r) + (k0 + c) * lda];
    }
    __syncthreads();
    const int64_t i = k0 + kb + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    T a[NB];
#pragma unroll
    for (int c = 0; c < NB; ++c)
        if (c < kb) a[c] = A[i + (k0 + c) * lda];
#pragma unroll
    for (int c = 0; c < NB; ++c) {
        if (c < kb) {
            T s = a[c];
#pragma unroll
            for (int k = 0; k < c; ++k) s -= a[k] * U[k][c];
            a[c] = s / U[c][c];
        }
    }
#pragma unroll
    for (int c = 0; c < NB; ++c)
        if (c < kb) A[i + (k0 + c) * lda] = a[c];
}

// U12 = L11^{-1} P A12: each thread permutes and forward-substitutes one column.
template <typename T, int NB>
__global__ void __launch_bounds__(128)
    k_trsm_u12(int64_t n, T *__restrict__ A, int64_t lda, int64_t k0, int kb,
               const int32_t *__restrict__ lperm)
{
    __shared__ T L[NB][NB + 1];
    __shared__ int32_t lp[NB];
    for (int idx = threadIdx.x; idx < kb * kb; idx += blockDim.x) {
        const int r = idx % kb, c = idx / kb;
        L[r][c] = A[(k0 + r) + (k0 + c) * lda];
    }
    if (threadIdx.x < kb) lp[threadIdx.x] = lperm[threadIdx.x];
    __syncthreads();
    const int64_t j = k0 + kb + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    T a[NB];
#pragma unroll
    for (int i = 0; i < NB; ++i)
        if (i < kb) a[i] = A[(k0 + lp[i]) + j * lda];
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        if (i < kb) {
            T s = a[i];
#pragma unroll
            for (int k = 0; k < i; ++k) s -= L[i][k] * a[k];
            a[i] = s;
        }
    }
#pragma unroll
    for (int i = 0; i < NB; ++i)
        if (i < kb) A[(k0 + i) + j * lda] = a[i];
}

// A22 -= L21 U12 on the CUDA cores (64 x 64 tiles, 4 x 4 per thread).
template <typename T>
__global__ void __launch_bounds__(256)
    k_gemm_update(int64_t n, T *__restrict__ A, int64_t lda, int64_t k0, int kb)
{
    constexpr int BM = 64, BN = 64, BK = 16;
    __shared__ T As[BK][BM + 4];
    __shared__ T Bs[BK][BN + 4];
    const int64_t s = k0 + kb;
    const int64_t row0 = s + (int64_t)blockIdx.x * BM, col0 = s + (int64_t)blockIdx.y * BN;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    T acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = T(0);
    for (int kk = 0; kk < kb; kk += BK) {
        for (int e = threadIdx.x; e < BK * BM; e += 256) {
            const int i = e % BM, k = e / BM;
            const int64_t gi = row0 + i;
            const int gk = kk + k;
            As[k][i] = (gi < n && gk < kb) ? A[gi + (k0 + gk) * lda] : T(0);
        }
        for (int e = threadIdx.x; e < BK * BN; e += 256) {
            const int k = e % BK, j = e / BK;
            const int64_t gj = col0 + j;
            const int gk = kk + k;
            Bs[k][j] = (gj < n && gk < kb) ? A[(k0 + gk) + gj * lda] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < BK; ++k) {
            T a[4], b[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = As[k][tx + 16 * r];
#pragma unroll
            for (int c = 0; c < 4; ++c) b[c] = Bs[k][ty * 4 + c];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] += a[r] * b[c];
        }
        __syncthreads();
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const int64_t gj = col0 + ty * 4 + c;
        if (gj >= n) continue;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int64_t gi = row0 + tx + 16 * r;
            if (gi < n) A[gi + gj * lda] -= acc[r][c];
        }
    }
}

__global__ void k_iota(int64_t n, int32_t *__restrict__ p)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = (int32_t)i;
}

template <typename T>
static void lu_steps(Ctx &c, T *A, int64_t lda)
{
    const int64_t n = c.n;
    c.tbeg(PH_LU_PANEL);
    k_iota<<<(unsigned)ceil_div(n, 256), 256, 0, c.stream>>>(n, c.d_rowperm);
    cudaMemsetAsync(c.d_info, 0, sizeof(int32_t), c.stream);
    c.launches += 1;
    for (int64_t k0 = 0; k0 < n; k0 += LU_NB) {
        const int kb = (int)std::min<int64_t>(LU_NB, n - k0);
        if (k0 > 0) c.tbeg(PH_LU_PANEL);
        k_diag_factor<T, LU_NB><<<1, 256, 0, c.stream>>>(n, A, lda, k0, c.d_lperm, c.d_rowperm,
                                                          c.d_info);
        c.launches += 1;
        if (k0 > 0) {
            k_swap_left<T, LU_NB><<<(unsigned)ceil_div(k0, 128), 128, 0, c.stream>>>(k0, kb, A, lda,
                                                                                      c.d_lperm);
            c.launches += 1;
        }
        const int64_t rest = n - k0 - kb;
        if (rest <= 0) {
            c.tend(PH_LU_PANEL);
            continue;
        }
        const unsigned g1 = (unsigned)ceil_div(rest, 128);
        k_trsm_l21<T, LU_NB><<<g1, 128, 0, c.stream>>>(n, A, lda, k0, kb);
        k_trsm_u12<T, LU_NB><<<g1, 128, 0, c.stream>>>(n, A, lda, k0, kb, c.d_lperm);
        c.launches += 2;
        c.tend(PH_LU_PANEL);
        c.tbeg(PH_LU_UPDATE);
        dim3 g2((unsigned)ceil_div(rest, 64), (unsigned)ceil_div(rest, 64));
        k_gemm_update<T><<<g2, 256, 0, c.stream>>>(n, A, lda, k0, kb);
        c.launches += 1;
        c.tend(PH_LU_UPDATE);
    }
}

int run_lu_fp64(Ctx &c, double *A, int64_t lda)
{
    lu_steps<double>(c, A, lda);
    return 0;
}

}  // namespace nrs
