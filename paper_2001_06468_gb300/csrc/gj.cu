// gj.cu -- explicit inverse of the FP32 system matrix by blocked Gauss-Jordan
// elimination, the preconditioner of the mixed-precision refinement (the
// dense solve of Gallagher & Smith, Sec. 4 step 3).
//
// With M the FP32 copy of A, step k (block rows/columns K = [k0, k0+kb)) is
//     D^{-1} = inverse of M[K,K]      (partial pivoting inside the block)
//     R      = D^{-1} M[K,:]          (scaled block row;  R[:,K] := 0)
//     C      = M[:,K]                 (block column;      C[K,:] := 0)
//     M     -= C R                    (rank-kb update of the whole matrix)
//     M[K,:] = R,  M[:,K] = -C D^{-1},  M[K,K] = D^{-1}.
// After the last step M holds A^{-1}.  Pivoting never leaves the diagonal
// block (the same restriction as the blocked LU of lu.cu, with the same
// Schur complements), so no row permutation survives into the inverse.  The
// update is a dense GEMM over the whole matrix every step -- the tensor-core
// kernel of tc_gemm.cu when available -- and applying the preconditioner is
// one bandwidth-bound matrix-vector product instead of a chain of dependent
// triangular solves.
#include "nrs_internal.cuh"

namespace nrs {

constexpr int GJ_NB = 64;

// D^{-1} by Gauss-Jordan on [D | I] with partial pivoting (one CTA).
// Dinv is row-major kb x kb (pitch GJ_NB).  A zero pivot records info.
__global__ void __launch_bounds__(256)
    k_gj_diag(int64_t n, const float *__restrict__ M, int64_t lda, int64_t k0,
              float *__restrict__ Dinv, int32_t *__restrict__ info)
{
    constexpr int NB = GJ_NB;
    __shared__ float W[NB][2 * NB + 1];
    __shared__ float F[NB];
    __shared__ int s_piv;
    const int tid = threadIdx.x;
    const int kb = (int)min((int64_t)NB, n - k0);
    for (int idx = tid; idx < kb * kb; idx += blockDim.x) {
        const int r = idx % kb, c = idx / kb;
        W[r][c] = M[(k0 + r) + (k0 + c) * lda];
        W[r][kb + c] = (r == c) ? 1.0f : 0.0f;
    }
    __syncthreads();
    const int w2 = 2 * kb;
    for (int c = 0; c < kb; ++c) {
        if (tid < 32) {
            float best = -1.0f;
            int br = c;
            for (int r = c + tid; r < kb; r += 32) {
                const float a = fabsf(W[r][c]);
                if (a > best) {
                    best = a;
                    br = r;
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const float ob = __shfl_xor_sync(0xffffffffu, best, o);
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
        if (p != c)
            for (int j = tid; j < w2; j += blockDim.x) {
                const float t = W[c][j];
                W[c][j] = W[p][j];
                W[p][j] = t;
            }
        __syncthreads();
        const float pv = W[c][c];
        if (pv == 0.0f) {
            if (tid == 0 && info) atomicCAS(info, 0, (int)(k0 + c + 1));
            __syncthreads();
            continue;
        }
        const float inv = 1.0f / pv;
        for (int j = tid; j < w2; j += blockDim.x) W[c][j] *= inv;
        if (tid < kb) F[tid] = W[tid][c];
        __syncthreads();
        for (int idx = tid; idx < kb * w2; idx += blockDim.x) {
            const int r = idx / w2, j = idx % w2;
            if (r != c) W[r][j] -= F[r] * W[c][j];
        }
        __syncthreads();
    }
    for (int idx = tid; idx < kb * kb; idx += blockDim.x) {
        const int r = idx / kb, c = idx % kb;
        Dinv[r * NB + c] = W[r][kb + c];
    }
}

// R[:, j] = D^{-1} M[K, j] for one tile of 64 columns (R[:,K] = 0), written
// transposed: Rt[j * NB + r] (column j's kb entries contiguous).  The CTAs of
// the last grid row copy the block column C = M[:, K] into Cb (row-major,
// Cb[i * NB + c], rows of K set to zero).
__global__ void __launch_bounds__(256)
    k_gj_prep(int64_t n, const float *__restrict__ M, int64_t lda, int64_t k0,
              const float *__restrict__ Dinv, float *__restrict__ Rt, float *__restrict__ Cb)
{
    constexpr int NB = GJ_NB;
    __shared__ float Ds[NB][NB + 1];
    __shared__ float Ms[NB][NB + 1];
    const int tid = threadIdx.x;
    const int kb = (int)min((int64_t)NB, n - k0);
    if (blockIdx.y == 1) {
        // block column copy: rows i = blockIdx.x * 256 + tid
        const int64_t i = (int64_t)blockIdx.x * 256 + tid;
        if (i >= n) return;
        const bool in_k = i >= k0 && i < k0 + kb;
        for (int c = 0; c < NB; ++c)
            Cb[i * NB + c] = (c < kb && !in_k) ? M[i + (k0 + c) * lda] : 0.0f;
        return;
    }
    const int64_t j0 = (int64_t)blockIdx.x * NB;
    if (j0 >= n) return;
    const int nj = (int)min((int64_t)NB, n - j0);
    for (int idx = tid; idx < NB * NB; idx += blockDim.x) {
        const int r = idx / NB, c = idx % NB;
        Ds[r][c] = (r < kb && c < kb) ? Dinv[r * NB + c] : 0.0f;
        const int rr = idx % NB, cc = idx / NB;  // coalesced over rows of M
        Ms[rr][cc] = (rr < kb && cc < nj) ? M[(k0 + rr) + (j0 + cc) * lda] : 0.0f;
    }
    __syncthreads();
    const bool tile_is_k = (j0 == k0);
    for (int idx = tid; idx < NB * NB; idx += blockDim.x) {
        const int c = idx / NB, r = idx % NB;  // output Rt[(j0+c)*NB + r]
        if (c >= nj) continue;
        float s = 0.0f;
        if (!tile_is_k && r < kb) {
#pragma unroll 16
            for (int t = 0; t < NB; ++t) s += Ds[r][t] * Ms[t][c];
        }
        Rt[(j0 + c) * NB + r] = s;
    }
}

// M[i, j] -= sum_c Cb[i,c] Rt[j,c] on the CUDA cores (64 x 64 tiles); tiles in
// block row or column K are skipped (their update is zero by construction).
__global__ void __launch_bounds__(256)
    k_gj_update_simt(int64_t n, float *__restrict__ M, int64_t lda, int64_t k0,
                     const float *__restrict__ Cb, const float *__restrict__ Rt)
{
    constexpr int NB = GJ_NB, BM = 64, BN = 64, BK = 16;
    const int64_t row0 = (int64_t)blockIdx.x * BM, col0 = (int64_t)blockIdx.y * BN;
    if (row0 == k0 || col0 == k0) return;
    __shared__ float As[BK][BM + 4];
    __shared__ float Bs[BK][BN + 4];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    float acc[4][4] = {};
    for (int kk = 0; kk < NB; kk += BK) {
        for (int e = threadIdx.x; e < BK * BM; e += 256) {
            const int k = e % BK, i = e / BK;
            const int64_t gi = row0 + i;
            As[k][i] = gi < n ? Cb[gi * NB + kk + k] : 0.0f;
            const int64_t gj = col0 + i;
            Bs[k][i] = gj < n ? Rt[gj * NB + kk + k] : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < BK; ++k) {
            float a[4], b[4];
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
            if (gi < n) M[gi + gj * lda] -= acc[r][c];
        }
    }
}

// Block row K <- R, block column K <- -C D^{-1}, M[K,K] <- D^{-1}.
// Grid x over 256-wide chunks; y = 0: columns j (block row), y = 1: rows i.
__global__ void __launch_bounds__(256)
    k_gj_finish(int64_t n, float *__restrict__ M, int64_t lda, int64_t k0,
                const float *__restrict__ Dinv, const float *__restrict__ Rt,
                const float *__restrict__ Cb)
{
    constexpr int NB = GJ_NB;
    __shared__ float Ds[NB][NB + 1];
    const int tid = threadIdx.x;
    const int kb = (int)min((int64_t)NB, n - k0);
    for (int idx = tid; idx < NB * NB; idx += blockDim.x) {
        const int r = idx / NB, c = idx % NB;
        Ds[r][c] = (r < kb && c < kb) ? Dinv[r * NB + c] : 0.0f;
    }
    __syncthreads();
    const int64_t t = (int64_t)blockIdx.x * 256 + tid;
    if (t >= n) return;
    if (blockIdx.y == 0) {
        const int64_t j = t;  // block row K, column j
        if (j >= k0 && j < k0 + kb) {
            for (int r = 0; r < kb; ++r) M[(k0 + r) + j * lda] = Ds[r][j - k0];
        } else {
            for (int r = 0; r < kb; ++r) M[(k0 + r) + j * lda] = Rt[j * NB + r];
        }
    } else {
        const int64_t i = t;  // block column K, row i
        if (i >= k0 && i < k0 + kb) return;
        float cr[NB];
#pragma unroll
        for (int c = 0; c < NB; ++c) cr[c] = Cb[i * NB + c];
        for (int c = 0; c < kb; ++c) {
            float s = 0.0f;
#pragma unroll
            for (int t2 = 0; t2 < NB; ++t2) s += cr[t2] * Ds[t2][c];
            M[i + (k0 + c) * lda] = -s;
        }
    }
}

// Tensor-core version of the update (tc_gemm.cu); false if not available for
// this precision.
bool launch_tc_gj_update(Ctx &c, float *M, int64_t lda, int64_t k0, const float *Cb,
                         const float *Rt, int prec);

int run_gj_fp32(Ctx &c, float *M, int64_t lda, int prec)
{
    const int64_t n = c.n;
    cudaMemsetAsync(c.d_info, 0, sizeof(int32_t), c.stream);
    const unsigned gcols = (unsigned)ceil_div(n, GJ_NB);
    const unsigned g256 = (unsigned)ceil_div(n, 256);
    for (int64_t k0 = 0; k0 < n; k0 += GJ_NB) {
        c.tbeg(PH_LU_PANEL);
        k_gj_diag<<<1, 256, 0, c.stream>>>(n, M, lda, k0, c.d_gj_dinv, c.d_info);
        k_gj_prep<<<dim3(std::max(gcols, g256), 2), 256, 0, c.stream>>>(n, M, lda, k0, c.d_gj_dinv,
                                                                         c.d_gj_rt, c.d_gj_cb);
        c.tend(PH_LU_PANEL);
        c.tbeg(PH_LU_UPDATE);
        bool done = false;
        if (prec == NRS_TF32 || prec == NRS_BF16)
            done = launch_tc_gj_update(c, M, lda, k0, c.d_gj_cb, c.d_gj_rt, prec);
        if (!done)
            k_gj_update_simt<<<dim3(gcols, gcols), 256, 0, c.stream>>>(n, M, lda, k0, c.d_gj_cb,
                                                                        c.d_gj_rt);
        c.tend(PH_LU_UPDATE);
        c.tbeg(PH_LU_PANEL);
        k_gj_finish<<<dim3(g256, 2), 256, 0, c.stream>>>(n, M, lda, k0, c.d_gj_dinv, c.d_gj_rt,
                                                         c.d_gj_cb);
        c.tend(PH_LU_PANEL);
        c.launches += 4;
    }
    return 0;
}

}  // namespace nrs
