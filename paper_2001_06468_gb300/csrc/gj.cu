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

// D^{-1} by Gauss-Jordan on [D | I] with partial pivoting (one CTA of 256
// threads, two barriers per column).
//  * Thread (r, s) = (tid / 4, tid % 4) keeps row r of the augmented matrix,
//    columns s + 4 i, in registers: the left half in L[16], the right half in
//    Rr[16].  After each group of four columns the finished left columns are
//    shifted out (L[i] <- L[i+1]) so that every register index is static.
//  * Column c is published in colbuf[c & 1] by its owners during step c-1;
//    every warp then finds the pivot on its own with warp reductions: the
//    unused row of largest |value|, lowest row on ties.  Only the pivot row is
//    copied to shared memory for the others.
//  * Rows are never moved or scaled during the sweep: step c subtracts
//    (W[r][c] / W[p][c]) W[p] from every row r != p.  At the end the left half
//    of pivot row p_c is pv_c e_c, so logical row c of D^{-1} is the right
//    half of physical row p_c divided by pv_c.
// Padding rows/columns (kb < 64) are identity.  Dinv is row-major 64 x 64; a
// zero pivot records info.
//
// With Cb and Rt given (the lookahead), the block is first brought up to date,
// D = M[K,K] - C[K,:] R[:,K]: the part of the previous step's rank-64 update
// that the main stream skips.  (Nothing reads M[K,K] afterwards: it is
// overwritten with D^{-1} at the end of the step.)
__global__ void __launch_bounds__(256)
    k_gj_diag(int64_t n, const float *__restrict__ M, int64_t lda, int64_t k0,
              float *__restrict__ Dinv, int32_t *__restrict__ info,
              const float *__restrict__ Cb, const float *__restrict__ Rt)
{
    constexpr int NB = GJ_NB;
    __shared__ float colbuf[2][NB];
    __shared__ float prow[2 * NB];
    __shared__ int pos[NB];
    __shared__ float pivval[NB];
    __shared__ float Cs[NB][NB + 1];
    __shared__ float Rs[NB][NB + 1];
    const int tid = threadIdx.x, lane = tid & 31;
    const int r = tid >> 2, s = tid & 3;
    const int kb = (int)min((int64_t)NB, n - k0);
    float L[16], Rr[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const int j = s + 4 * i;
        L[i] = (r < kb && j < kb) ? M[(k0 + r) + (k0 + j) * lda] : (r == j ? 1.0f : 0.0f);
        Rr[i] = (r == j) ? 1.0f : 0.0f;
    }
    if (Cb) {
        float cv[16], rv[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int idx = tid + 256 * q, a = idx & 63, b = idx >> 6;
            cv[q] = b < kb ? Cb[(k0 + b) * NB + a] : 0.0f;
            rv[q] = b < kb ? Rt[(k0 + b) * NB + a] : 0.0f;
        }
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int idx = tid + 256 * q, a = idx & 63, b = idx >> 6;
            Cs[b][a] = cv[q];
            Rs[b][a] = rv[q];
        }
        __syncthreads();
        // L[i] (row r, column j = s + 4 i) -= sum_t C[r][t] R[j][t]
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int j = s + 4 * i;
            float acc = 0.0f;
#pragma unroll 16
            for (int t = 0; t < NB; ++t) acc += Cs[r][t] * Rs[j][t];
            if (r < kb && j < kb) L[i] -= acc;
        }
    }
    if (s == 0) colbuf[0][r] = L[0];
    unsigned long long used = 0ull;
    __syncthreads();
    for (int cc = 0; cc < NB / 4; ++cc) {
#pragma unroll
        for (int sp = 0; sp < 4; ++sp) {
            const int c = 4 * cc + sp;
            const int buf = sp & 1;
            const float a0 = fabsf(colbuf[buf][lane]), a1 = fabsf(colbuf[buf][lane + 32]);
            const bool u0 = (used >> lane) & 1ull, u1 = (used >> (lane + 32)) & 1ull;
            const unsigned k0v = u0 ? 0u : (0x80000000u | __float_as_uint(a0));
            const unsigned k1v = u1 ? 0u : (0x80000000u | __float_as_uint(a1));
            const unsigned key = k0v >= k1v ? k0v : k1v;
            const int row = k0v >= k1v ? lane : lane + 32;
            const unsigned mx = __reduce_max_sync(0xffffffffu, key);
            const int p = (int)__reduce_min_sync(0xffffffffu, key == mx ? (unsigned)row : 64u);
            used |= 1ull << p;
            const float pv = colbuf[buf][p];
            if (tid == 0) {
                pos[p] = c;
                pivval[c] = pv;
                if (pv == 0.0f && info) atomicCAS(info, 0, (int)(k0 + c + 1));
            }
            if (r == p) {
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    prow[s + 4 * i] = L[i];
                    prow[NB + s + 4 * i] = Rr[i];
                }
            }
            __syncthreads();
            if (r != p) {
                const float g = colbuf[buf][r] / pv;
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    L[i] -= g * prow[s + 4 * i];
                    Rr[i] -= g * prow[NB + s + 4 * i];
                }
            }
            // publish column c + 1 for the next step
            if (s == ((sp + 1) & 3)) colbuf[buf ^ 1][r] = (sp < 3) ? L[0] : L[1];
            __syncthreads();
        }
        // columns 4 cc .. 4 cc + 3 are finished: shift them out of L
#pragma unroll
        for (int i = 0; i < 15; ++i) L[i] = L[i + 1];
        L[15] = 0.0f;
    }
    const int lr = pos[r];
    const float d = 1.0f / pivval[lr];
#pragma unroll
    for (int i = 0; i < 16; ++i) Dinv[lr * NB + s + 4 * i] = Rr[i] * d;
}

// Prep of step K.  grid.y = 0: R[:, j] = D^{-1} M[K, j] for one 64-column tile
// (R[:,K] = 0), stored transposed Rt[j * 64 + r].  grid.y = 1: the block column
// C = M[:, K] for one 64-row tile, stored row-major Cb[i * 64 + c] (rows of K
// zero).  Both through shared memory so every global access is coalesced.
__global__ void __launch_bounds__(256)
    k_gj_prep(int64_t n, const float *__restrict__ M, int64_t lda, int64_t k0,
              const float *__restrict__ Dinv, float *__restrict__ Rt, float *__restrict__ Cb)
{
    constexpr int NB = GJ_NB;
    __shared__ float Ds[NB][NB + 1];
    __shared__ float Ms[NB][NB + 1];
    const int tid = threadIdx.x;
    const int kb = (int)min((int64_t)NB, n - k0);
    const int64_t t0 = (int64_t)blockIdx.x * NB;
    if (t0 >= n) return;
    const int nt = (int)min((int64_t)NB, n - t0);
    if (blockIdx.y == 1) {
        const bool in_k = (t0 == k0);
        float v[16];  // all loads in flight before the first shared store
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int idx = tid + 256 * q, i = idx & 63, c = idx >> 6;
            v[q] = (i < nt && c < kb && !in_k) ? M[(t0 + i) + (k0 + c) * lda] : 0.0f;
        }
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int idx = tid + 256 * q;
            Ms[idx & 63][idx >> 6] = v[q];
        }
        __syncthreads();
        for (int idx = tid; idx < NB * NB; idx += 256) {
            const int c = idx & 63, i = idx >> 6;
            if (i < nt) Cb[(t0 + i) * NB + c] = Ms[i][c];
        }
        return;
    }
    const bool tile_is_k = (t0 == k0);
    {
        float dv[16], mv[16];  // all loads in flight before the first shared store
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int idx = tid + 256 * q, a = idx & 63, b = idx >> 6;
            dv[q] = Dinv[b * NB + a];
            mv[q] = (a < kb && b < nt) ? M[(k0 + a) + (t0 + b) * lda] : 0.0f;
        }
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int idx = tid + 256 * q, a = idx & 63, b = idx >> 6;
            Ds[b][a] = dv[q];
            Ms[a][b] = mv[q];
        }
    }
    __syncthreads();
    // thread computes R[r, t0 + c] for r = tr + 16 rr, c = tc + 16 cc (4 x 4)
    const int tr = tid & 15, tc = tid >> 4;
    float acc[4][4] = {};
#pragma unroll 8
    for (int t = 0; t < NB; ++t) {
        float a[4], b[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) a[q] = Ds[tr + 16 * q][t];
#pragma unroll
        for (int q = 0; q < 4; ++q) b[q] = Ms[t][tc + 16 * q];
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < 4; ++y) acc[x][y] += a[x] * b[y];
    }
#pragma unroll
    for (int y = 0; y < 4; ++y) {
        const int c = tc + 16 * y;
        if (c >= nt) continue;
#pragma unroll
        for (int x = 0; x < 4; ++x) {
            const int rr = tr + 16 * x;
            Rt[(t0 + c) * NB + rr] = (tile_is_k || rr >= kb) ? 0.0f : acc[x][y];
        }
    }
}

// M[i, j] -= sum_c Cb[i,c] Rt[j,c] on the CUDA cores (64 x 64 tiles); tiles in
// block row or column K are skipped (their update is zero by construction),
// and so is the diagonal tile at skip0 (updated separately by the lookahead).
__global__ void __launch_bounds__(256)
    k_gj_update_simt(int64_t n, float *__restrict__ M, int64_t lda, int64_t k0,
                     const float *__restrict__ Cb, const float *__restrict__ Rt, int64_t skip0)
{
    constexpr int NB = GJ_NB, BM = 64, BN = 64, BK = 16;
    const int64_t row0 = (int64_t)blockIdx.x * BM, col0 = (int64_t)blockIdx.y * BN;
    if (row0 == k0 || col0 == k0 || (row0 == skip0 && col0 == skip0)) return;
    __shared__ float As[BK][BM + 4];
    __shared__ float Bs[BK][BN + 4];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    float acc[4][4] = {};
    for (int kk = 0; kk < NB; kk += BK) {
        float av[4], bv[4];  // all loads in flight before the shared stores
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = threadIdx.x + 256 * q, k = e % BK, i = e / BK;
            const int64_t gi = row0 + i, gj = col0 + i;
            av[q] = gi < n ? Cb[gi * NB + kk + k] : 0.0f;
            bv[q] = gj < n ? Rt[gj * NB + kk + k] : 0.0f;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = threadIdx.x + 256 * q, k = e % BK, i = e / BK;
            As[k][i] = av[q];
            Bs[k][i] = bv[q];
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

// Block row K <- R, block column K <- -C D^{-1}, M[K,K] <- D^{-1}, in 64-wide
// tiles.  grid.y = 0: column tile t0 of block row K; grid.y = 1: row tile t0
// of block column K.
__global__ void __launch_bounds__(256)
    k_gj_finish(int64_t n, float *__restrict__ M, int64_t lda, int64_t k0,
                const float *__restrict__ Dinv, const float *__restrict__ Rt,
                const float *__restrict__ Cb)
{
    constexpr int NB = GJ_NB;
    __shared__ float Ds[NB][NB + 1];
    __shared__ float Cs[NB][NB + 1];
    const int tid = threadIdx.x;
    const int kb = (int)min((int64_t)NB, n - k0);
    const int64_t t0 = (int64_t)blockIdx.x * NB;
    if (t0 >= n) return;
    const int nt = (int)min((int64_t)NB, n - t0);
    if (blockIdx.y == 0) {
        const bool tile_is_k = (t0 == k0);
        float v[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int idx = tid + 256 * q, rr = idx & 63, c = idx >> 6;
            const bool in = rr < kb && c < nt;
            v[q] = !in ? 0.0f : (tile_is_k ? Dinv[rr * NB + c] : Rt[(t0 + c) * NB + rr]);
        }
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int idx = tid + 256 * q, rr = idx & 63, c = idx >> 6;
            if (rr < kb && c < nt) M[(k0 + rr) + (t0 + c) * lda] = v[q];
        }
        return;
    }
    if (t0 == k0) return;
    {
        float dv[16], cv[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int idx = tid + 256 * q, a = idx & 63, b = idx >> 6;
            dv[q] = Dinv[b * NB + a];
            cv[q] = b < nt ? Cb[(t0 + b) * NB + a] : 0.0f;
        }
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int idx = tid + 256 * q, a = idx & 63, b = idx >> 6;
            Ds[b][a] = dv[q];
            Cs[b][a] = cv[q];
        }
    }
    __syncthreads();
    // thread computes out[i][c] = -sum_t C[i][t] Dinv[t][c], i = tr + 16 x, c = tc + 16 y
    const int tr = tid & 15, tc = tid >> 4;
    float acc[4][4] = {};
#pragma unroll 8
    for (int t = 0; t < NB; ++t) {
        float a[4], b[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) a[q] = Cs[tr + 16 * q][t];
#pragma unroll
        for (int q = 0; q < 4; ++q) b[q] = Ds[t][tc + 16 * q];
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < 4; ++y) acc[x][y] += a[x] * b[y];
    }
#pragma unroll
    for (int y = 0; y < 4; ++y) {
        const int c = tc + 16 * y;
        if (c >= kb) continue;
#pragma unroll
        for (int x = 0; x < 4; ++x) {
            const int i = tr + 16 * x;
            if (i < nt) M[(t0 + i) + (k0 + c) * lda] = -acc[x][y];
        }
    }
}

// Tensor-core version of the update (tc_gemm.cu); false if not available for
// this precision.
bool launch_tc_gj_update(Ctx &c, float *M, int64_t lda, int64_t k0, const float *Cb,
                         const float *Rt, int prec, int64_t skip0);

void launch_simt_rank64(Ctx &c, float *M, int64_t lda, int64_t n, const float *Cb, const float *Rt)
{
    const unsigned g = (unsigned)ceil_div(n, GJ_NB);
    // k0 = -GJ_NB: no tile is skipped
    k_gj_update_simt<<<dim3(g, g), 256, 0, c.stream>>>(n, M, lda, -GJ_NB, Cb, Rt, -GJ_NB);
    c.launches += 1;
}

// One inversion.  Main stream, step k: prep_k, update_k (all of M but the
// next diagonal block), finish_k.  Side stream, as soon as prep_k is done:
// update of the next diagonal block alone, then its inverse (k_gj_diag into
// the other D^{-1} buffer), which so overlaps update_k and finish_k; prep_{k+1}
// waits for it.
int run_gj_fp32(Ctx &c, float *M, int64_t lda, int prec)
{
    const int64_t n = c.n;
    cudaMemsetAsync(c.d_info, 0, sizeof(int32_t), c.stream);
    const unsigned gcols = (unsigned)ceil_div(n, GJ_NB);
    float *dinv[2] = {c.d_gj_dinv, c.d_gj_dinv + GJ_NB * GJ_NB};
    c.tbeg(PH_LU_DIAG);
    k_gj_diag<<<1, 256, 0, c.stream>>>(n, M, lda, 0, dinv[0], c.d_info, nullptr, nullptr);
    c.tend(PH_LU_DIAG);
    c.launches += 1;
    int kstep = 0;
    for (int64_t k0 = 0; k0 < n; k0 += GJ_NB, ++kstep) {
        float *dk = dinv[kstep & 1];
        const int64_t k1 = k0 + GJ_NB;
        const bool next = k1 < n;
        c.tbeg(PH_LU_PANEL);
        k_gj_prep<<<dim3(gcols, 2), 256, 0, c.stream>>>(n, M, lda, k0, dk, c.d_gj_rt, c.d_gj_cb);
        c.tend(PH_LU_PANEL);
        if (next) {
            cudaEventRecord(c.ev_prep, c.stream);
            cudaStreamWaitEvent(c.stream2, c.ev_prep, 0);
            c.tbeg(PH_LU_DIAG, c.stream2);
            k_gj_diag<<<1, 256, 0, c.stream2>>>(n, M, lda, k1, dinv[(kstep + 1) & 1], c.d_info,
                                                 c.d_gj_cb, c.d_gj_rt);
            c.tend(PH_LU_DIAG, c.stream2);
            cudaEventRecord(c.ev_diag, c.stream2);
            c.launches += 1;
        }
        const int64_t skip0 = next ? k1 : -GJ_NB;
        c.tbeg(PH_LU_UPDATE);
        bool done = false;
        if (prec == NRS_TF32 || prec == NRS_BF16)
            done = launch_tc_gj_update(c, M, lda, k0, c.d_gj_cb, c.d_gj_rt, prec, skip0);
        if (!done)
            k_gj_update_simt<<<dim3(gcols, gcols), 256, 0, c.stream>>>(n, M, lda, k0, c.d_gj_cb,
                                                                        c.d_gj_rt, skip0);
        c.tend(PH_LU_UPDATE);
        c.tbeg(PH_LU_PANEL);
        k_gj_finish<<<dim3(gcols, 2), 256, 0, c.stream>>>(n, M, lda, k0, dk, c.d_gj_rt, c.d_gj_cb);
        c.tend(PH_LU_PANEL);
        if (next) cudaStreamWaitEvent(c.stream, c.ev_diag, 0);
        c.launches += 3;
    }
    return 0;
}

}  // namespace nrs
