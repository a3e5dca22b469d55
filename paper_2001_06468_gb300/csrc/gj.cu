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

// D^{-1} of the 64 x 64 diagonal block by Gauss-Jordan elimination with
// partial pivoting, written for the latency of one pivot step (this kernel is
// the critical path of the factorisation: one launch per block column).
//
// Lookahead (Dprev given, P = the previous block, K = this one): the block is
// first brought up to date by the part of step P's rank-64 update that the
// main stream skips, from the un-finished block row and column P of M:
//     R_PK = Dprev M[P,K],   D = M[K,K] - M[K,P] R_PK,
// both 4 x 4 register-tiled over 256 threads, the same products (and the same
// order of operations) as the prep and finish kernels.  Two tiles of step P's
// finish depend on nothing else and are written here to `stage` instead of M
// (the finish of step P skips them, and the prep of step K reads them from
// there): stage[0..4096) = R_PK (column-major, 64 x 64) is M[P,K] after step
// P, and stage[4096..8192) = -M[K,P] Dprev is M[K,P] after step P; the latter
// is computed by warps 2, 3, 6 and 7 while warps 0 and 1 do the elimination.
// The elimination: two warps, lane l of warp w holding row r = 32 w + l in
// registers T[64]:
//  * exchange (sweep) form, in place: at the step for column c with pivot row
//    p, every other row i gets T_i[j] -= (T_i[c] / T_p[c]) T_p[j] (j != c) and
//    T_i[c] = -T_i[c] / T_p[c]; the pivot row is divided by T_p[c] and gets
//    T_p[c] = 1 / T_p[c].  After the 64 steps row p_c holds row c of D^{-1}
//    with column d standing for original row p_d.
//  * the pivot row's division is deferred: it keeps its values, sets
//    T_p[c] = 1 and records s_p = 1 / T_p[c]; later updates of that row are
//    the same formula on the unscaled values, and s_p is applied at the end;
//  * the registers rotate by one column per step, so the current column is
//    always T[0] (static register indices) and after 64 steps every column
//    is back in place;
//  * pivot: the unused row of largest |T[c]|, lowest row on ties (warp
//    reductions, then the two warps' candidates); each warp's candidate
//    writes its row to a double-buffered shared slot before the one 64-thread
//    barrier of the step, and every lane reads the winner's row from there.
// Padding rows/columns (kb < 64) are identity.  Dinv is row-major 64 x 64; a
// zero pivot records info.
__global__ void __launch_bounds__(256)
    k_gj_diag(int64_t n, const float *__restrict__ M, int64_t lda, int64_t k0,
              float *__restrict__ Dinv, int32_t *__restrict__ info,
              const float *__restrict__ Dprev, float *__restrict__ stage)
{
    constexpr int NB = GJ_NB, LDT = NB + 4;
    // two 64 x 68 buffers: B0 = Dprev^T, then R_PK, then the block D (rows of
    // 65 floats), then the output; B1 = M[P,K], then M[K,P]^T
    __shared__ __align__(16) float sraw[2 * NB * LDT];
    float(*B0)[LDT] = reinterpret_cast<float(*)[LDT]>(sraw);
    float(*B1)[LDT] = reinterpret_cast<float(*)[LDT]>(sraw + NB * LDT);
    float(*sm0)[NB + 1] = reinterpret_cast<float(*)[NB + 1]>(sraw);
    __shared__ __align__(16) float cand[2][2][NB];  // [step parity][warp][column]
    __shared__ unsigned ckey[2][2];
    __shared__ float cpiv[2][2];
    __shared__ int crow[2][2];
    __shared__ int pivrow[NB];
    const int tid = threadIdx.x;
    const int kb = (int)min((int64_t)NB, n - k0);
    const int64_t kp = k0 - NB;
    {
        // thread owns the 4 x 4 tile rows r0..r0+3, columns j0..j0+3
        const int r0 = 4 * (tid >> 4), j0 = 4 * (tid & 15);
        float L[4][4];
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            const int j = j0 + jj;
            if (r0 + 3 < kb && j < kb) {
                const float4 v = *reinterpret_cast<const float4 *>(M + (k0 + r0) + (k0 + j) * lda);
                L[0][jj] = v.x;
                L[1][jj] = v.y;
                L[2][jj] = v.z;
                L[3][jj] = v.w;
            } else {
#pragma unroll
                for (int ii = 0; ii < 4; ++ii) {
                    const int r = r0 + ii;
                    L[ii][jj] = (r < kb && j < kb) ? M[(k0 + r) + (k0 + j) * lda]
                                                   : (r == j ? 1.0f : 0.0f);
                }
            }
        }
        if (Dprev) {
            float dv[16], mv[16], cv[16];  // all loads in flight before the first shared store
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int idx = tid + 256 * q, a = idx & 63, b = idx >> 6;
                dv[q] = Dprev[b * NB + a];                                        // Dprev[b][a]
                mv[q] = b < kb ? M[(kp + a) + (k0 + b) * lda] : 0.0f;            // M[P+a][K+b]
                cv[q] = a < kb ? M[(k0 + a) + (kp + b) * lda] : 0.0f;            // M[K+a][P+b]
            }
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int idx = tid + 256 * q, a = idx & 63, b = idx >> 6;
                B0[a][b] = dv[q];
                B1[a][b] = mv[q];
            }
            __syncthreads();
            // R_PK[s0 + x][t0 + y] = sum_t Dprev[s0 + x][t] M[P+t][K + t0 + y]
            const int s0 = 4 * (tid & 15), c0 = 4 * (tid >> 4);
            float acc[4][4] = {};
#pragma unroll 8
            for (int t = 0; t < NB; ++t) {
                const float4 a4 = *reinterpret_cast<const float4 *>(&B0[t][s0]);
                const float4 b4 = *reinterpret_cast<const float4 *>(&B1[t][c0]);
                const float x4[4] = {a4.x, a4.y, a4.z, a4.w};
                const float y4[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
                for (int x = 0; x < 4; ++x)
#pragma unroll
                    for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(x4[x], y4[y], acc[x][y]);
            }
            __syncthreads();  // B0 and B1 are free
#pragma unroll
            for (int x = 0; x < 4; ++x)
                *reinterpret_cast<float4 *>(&B0[s0 + x][c0]) =
                    make_float4(acc[x][0], acc[x][1], acc[x][2], acc[x][3]);
#pragma unroll
            for (int y = 0; y < 4; ++y)
                *reinterpret_cast<float4 *>(&stage[(s0) + (c0 + y) * NB]) =
                    make_float4(acc[0][y], acc[1][y], acc[2][y], acc[3][y]);
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int idx = tid + 256 * q;
                B1[idx >> 6][idx & 63] = cv[q];  // B1[t][i] = M[K+i][P+t]
            }
            __syncthreads();
            // L -= M[K,P] R_PK on the tile: per t one 16-byte load of each operand
            float acc2[4][4] = {};
#pragma unroll 8
            for (int t = 0; t < NB; ++t) {
                const float4 c4 = *reinterpret_cast<const float4 *>(&B1[t][r0]);
                const float4 r4 = *reinterpret_cast<const float4 *>(&B0[t][j0]);
                const float cc[4] = {c4.x, c4.y, c4.z, c4.w};
                const float rr[4] = {r4.x, r4.y, r4.z, r4.w};
#pragma unroll
                for (int ii = 0; ii < 4; ++ii)
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj) acc2[ii][jj] = fmaf(cc[ii], rr[jj], acc2[ii][jj]);
            }
#pragma unroll
            for (int ii = 0; ii < 4; ++ii)
#pragma unroll
                for (int jj = 0; jj < 4; ++jj)
                    if (r0 + ii < kb && j0 + jj < kb) L[ii][jj] -= acc2[ii][jj];
            __syncthreads();  // everyone is done with R_PK in B0
        }
#pragma unroll
        for (int ii = 0; ii < 4; ++ii)
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) sm0[r0 + ii][j0 + jj] = L[ii][jj];
    }
    __syncthreads();
    if (tid >= 64) {
        // warps 2, 3, 6, 7 (the scheduler partitions that warps 0 and 1 do not
        // use): stage[4096 + i + 64 c] = -sum_t M[K+i][P+t] Dprev[t][c] on a
        // 4 x 8 tile per thread (M[K,P] transposed in B1, Dprev from global)
        const int wq = tid >> 5;
        if (!Dprev || wq == 4 || wq == 5) return;
        const int u = wq < 4 ? tid - 64 : tid - 128, i0 = 4 * (u & 15), c0 = 8 * (u >> 4);
        float acc[4][8] = {};
#pragma unroll 4
        for (int t = 0; t < NB; ++t) {
            const float4 a4 = *reinterpret_cast<const float4 *>(&B1[t][i0]);
            const float4 d0 = __ldg(reinterpret_cast<const float4 *>(Dprev + t * NB + c0));
            const float4 d1 = __ldg(reinterpret_cast<const float4 *>(Dprev + t * NB + c0 + 4));
            const float x4[4] = {a4.x, a4.y, a4.z, a4.w};
            const float y8[8] = {d0.x, d0.y, d0.z, d0.w, d1.x, d1.y, d1.z, d1.w};
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 8; ++y) acc[x][y] = fmaf(x4[x], y8[y], acc[x][y]);
        }
        float *stx = stage + NB * NB;
#pragma unroll
        for (int y = 0; y < 8; ++y)
            *reinterpret_cast<float4 *>(&stx[i0 + (c0 + y) * NB]) =
                make_float4(-acc[0][y], -acc[1][y], -acc[2][y], -acc[3][y]);
        return;
    }
    const int w = tid >> 5, r = tid;
    float T[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) T[j] = sm0[r][j];
    bool used = false;
    float scale = 1.0f;
    int mypos = 0;
    unsigned zero_at = 0xffffffffu;  // step of a zero pivot in this row, if any
#pragma unroll 4
    for (int c = 0; c < NB; ++c) {
        const int b = c & 1;
        const float colv = T[0];
        // the reciprocal is formed before the search, so that the winner can
        // publish it with its row and nobody divides after the barrier
        const float myr = 1.0f / colv;
        const unsigned key = used ? 0u : (0x80000000u | __float_as_uint(fabsf(colv)));
        const unsigned mx = __reduce_max_sync(0xffffffffu, key);
        const int best = (int)__reduce_min_sync(0xffffffffu, key == mx ? (unsigned)r : 255u);
        if (r == best) {
            float4 *dst = reinterpret_cast<float4 *>(&cand[b][w][0]);
#pragma unroll
            for (int q = 0; q < NB / 4; ++q)
                dst[q] = make_float4(T[4 * q], T[4 * q + 1], T[4 * q + 2], T[4 * q + 3]);
            ckey[b][w] = mx;
            cpiv[b][w] = myr;
            crow[b][w] = best;
        }
        asm volatile("bar.sync 1, 64;" ::: "memory");
        const unsigned kw0 = ckey[b][0], kw1 = ckey[b][1];
        const float pv0 = cpiv[b][0], pv1 = cpiv[b][1];
        const int rw0 = crow[b][0], rw1 = crow[b][1];
        const int win = kw0 >= kw1 ? 0 : 1;  // warp 0 (the lower rows) on ties
        const float rpiv = win ? pv1 : pv0;
        const int p = win ? rw1 : rw0;
        const bool is_piv = (r == p);
        if (is_piv) {
            used = true;
            scale = rpiv;
            mypos = c;
            if (colv == 0.0f) zero_at = (unsigned)c;
        }
        const float f = is_piv ? 0.0f : colv * rpiv;
        const float newc = is_piv ? 1.0f : -f;
        const float4 *pr4 = reinterpret_cast<const float4 *>(&cand[b][win][0]);
#pragma unroll
        for (int q = 0; q < NB / 4; ++q) {
            const float4 v = pr4[q];
            if (q > 0) T[4 * q] = fmaf(-f, v.x, T[4 * q]);
            T[4 * q + 1] = fmaf(-f, v.y, T[4 * q + 1]);
            T[4 * q + 2] = fmaf(-f, v.z, T[4 * q + 2]);
            T[4 * q + 3] = fmaf(-f, v.w, T[4 * q + 3]);
        }
#pragma unroll
        for (int j = 0; j < NB - 1; ++j) T[j] = T[j + 1];
        T[NB - 1] = newc;
    }
    // the pivot order (row pivoted at step c) and the first zero pivot, from
    // the rows' own records: no per-step bookkeeping in the loop
    pivrow[mypos] = r;
    zero_at = __reduce_min_sync(0xffffffffu, zero_at);
    if ((tid & 31) == 0) crow[0][w] = (int)zero_at;
    asm volatile("bar.sync 1, 64;" ::: "memory");  // pivrow complete
    if (tid == 0 && info) {
        const unsigned z = min((unsigned)crow[0][0], (unsigned)crow[0][1]);
        if (z != 0xffffffffu) atomicCAS(info, 0, (int)(k0 + z + 1));
    }
    // row mypos of D^{-1}, column pivrow[d] = T[d] * scale: through shared
    // memory (B0, read into the registers before the loop) so that the global
    // stores are coalesced
#pragma unroll
    for (int d = 0; d < NB; ++d) sm0[mypos][pivrow[d]] = T[d] * scale;
    asm volatile("bar.sync 1, 64;" ::: "memory");
    for (int i = 0; i < NB; ++i) Dinv[i * NB + tid] = sm0[i][tid];
}

// Prep of step K.  grid.y = 0: R[:, j] = D^{-1} M[K, j] for one 64-column tile
// (R[:,K] = 0), stored transposed Rt[j * 64 + r].  grid.y = 1: the block column
// C = M[:, K] for one 64-row tile, stored row-major Cb[i * 64 + c] (rows of K
// zero).  Both through shared memory so every global access is coalesced.
// With `stage` given (K > 0), the tiles M[K-1,K] and M[K,K-1] as left by step
// K-1 are read from there (the diagonal inverse of this step wrote them; the
// finish of step K-1 skips them in M).
__global__ void __launch_bounds__(256)
    k_gj_prep(int64_t n, const float *__restrict__ M, int64_t lda, int64_t k0,
              const float *__restrict__ Dinv, float *__restrict__ Rt, float *__restrict__ Cb,
              const float *__restrict__ stage)
{
    constexpr int NB = GJ_NB;
    __shared__ __align__(16) float Ds[NB][NB + 4];
    __shared__ __align__(16) float Ms[NB][NB + 4];
    const int tid = threadIdx.x;
    const int kb = (int)min((int64_t)NB, n - k0);
    const int64_t t0 = (int64_t)blockIdx.x * NB;
    if (t0 >= n) return;
    const int nt = (int)min((int64_t)NB, n - t0);
    const bool staged = stage && t0 == k0 - NB;
    if (blockIdx.y == 1) {
        const bool in_k = (t0 == k0);
        // M[t0 + i][K + c], or column-major 64 x 64 in stage for the tile above
        const float *src = staged ? stage : M + t0 + k0 * lda;
        const int64_t ld = staged ? NB : lda;
        float v[16];  // all loads in flight before the first shared store
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int idx = tid + 256 * q, i = idx & 63, c = idx >> 6;
            v[q] = (i < nt && c < kb && !in_k) ? src[i + c * ld] : 0.0f;
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
    // D^{-1} transposed and the block row, rows of 68 floats (16-byte loads)
    float(*DT)[NB + 4] = reinterpret_cast<float(*)[NB + 4]>(&Ds[0][0]);
    float(*MK)[NB + 4] = reinterpret_cast<float(*)[NB + 4]>(&Ms[0][0]);
    {
        // M[K + a][t0 + b], or column-major 64 x 64 in stage for the tile left of K
        const float *src = staged ? stage + NB * NB : M + k0 + t0 * lda;
        const int64_t ld = staged ? NB : lda;
        float dv[16], mv[16];  // all loads in flight before the first shared store
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int idx = tid + 256 * q, a = idx & 63, b = idx >> 6;
            dv[q] = Dinv[b * NB + a];                               // D^{-1}[b][a]
            mv[q] = (a < kb && b < nt) ? src[a + b * ld] : 0.0f;  // M[K+a][t0+b]
        }
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int idx = tid + 256 * q, a = idx & 63, b = idx >> 6;
            DT[a][b] = dv[q];
            MK[a][b] = mv[q];
        }
    }
    __syncthreads();
    // thread computes R[r0 + x][t0 + c0 + y] for the 4 x 4 tile at (r0, c0)
    const int r0 = 4 * (tid & 15), c0 = 4 * (tid >> 4);
    float acc[4][4] = {};
#pragma unroll 8
    for (int t = 0; t < NB; ++t) {
        const float4 a4 = *reinterpret_cast<const float4 *>(&DT[t][r0]);
        const float4 b4 = *reinterpret_cast<const float4 *>(&MK[t][c0]);
        const float a[4] = {a4.x, a4.y, a4.z, a4.w};
        const float b[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(a[x], b[y], acc[x][y]);
    }
#pragma unroll
    for (int y = 0; y < 4; ++y) {
        const int c = c0 + y;
        if (c >= nt) continue;
        float v[4];
#pragma unroll
        for (int x = 0; x < 4; ++x) v[x] = (tile_is_k || r0 + x >= kb) ? 0.0f : acc[x][y];
        *reinterpret_cast<float4 *>(&Rt[(t0 + c) * NB + r0]) = make_float4(v[0], v[1], v[2], v[3]);
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
// of block column K.  The tiles at skip_t0 (the next block, whose diagonal
// inverse computes them and leaves them for the next prep) are not written.
__global__ void __launch_bounds__(256)
    k_gj_finish(int64_t n, float *__restrict__ M, int64_t lda, int64_t k0,
                const float *__restrict__ Dinv, const float *__restrict__ Rt,
                const float *__restrict__ Cb, int64_t skip_t0)
{
    constexpr int NB = GJ_NB;
    __shared__ __align__(16) float Ds[NB][NB + 4];
    __shared__ __align__(16) float Cs[NB][NB + 4];
    const int tid = threadIdx.x;
    const int kb = (int)min((int64_t)NB, n - k0);
    const int64_t t0 = (int64_t)blockIdx.x * NB;
    if (t0 >= n || t0 == skip_t0) return;
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
    // C transposed and D^{-1}, rows of 68 floats (16-byte loads)
    float(*CT)[NB + 4] = reinterpret_cast<float(*)[NB + 4]>(&Cs[0][0]);
    float(*DD)[NB + 4] = reinterpret_cast<float(*)[NB + 4]>(&Ds[0][0]);
    {
        float dv[16], cv[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int idx = tid + 256 * q, a = idx & 63, b = idx >> 6;
            dv[q] = Dinv[b * NB + a];                             // D^{-1}[b][a]
            cv[q] = b < nt ? Cb[(t0 + b) * NB + a] : 0.0f;       // C[t0+b][a]
        }
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int idx = tid + 256 * q, a = idx & 63, b = idx >> 6;
            DD[b][a] = dv[q];
            CT[a][b] = cv[q];
        }
    }
    __syncthreads();
    // thread computes out[i0 + x][c0 + y] = -sum_t C[i][t] D^{-1}[t][c] on its 4 x 4 tile
    const int i0 = 4 * (tid & 15), c0 = 4 * (tid >> 4);
    float acc[4][4] = {};
#pragma unroll 8
    for (int t = 0; t < NB; ++t) {
        const float4 a4 = *reinterpret_cast<const float4 *>(&CT[t][i0]);
        const float4 b4 = *reinterpret_cast<const float4 *>(&DD[t][c0]);
        const float a[4] = {a4.x, a4.y, a4.z, a4.w};
        const float b[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(a[x], b[y], acc[x][y]);
    }
#pragma unroll
    for (int y = 0; y < 4; ++y) {
        const int c = c0 + y;
        if (c >= kb) continue;
        float *col = M + t0 + (k0 + c) * lda;
        if (i0 + 3 < nt) {
            *reinterpret_cast<float4 *>(col + i0) =
                make_float4(-acc[0][y], -acc[1][y], -acc[2][y], -acc[3][y]);
        } else {
#pragma unroll
            for (int x = 0; x < 4; ++x)
                if (i0 + x < nt) col[i0 + x] = -acc[x][y];
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

// One inversion.  Streams: main (S), lookahead (S2), finish (S4).  Step k
// (block K, next block K+1):
//   S2: (waits the update of step k-1 and the finish of step k-1) the
//       diagonal inverse of K+1 with its lookahead from D_K^{-1} and the
//       un-finished block row and column K; it also leaves the two finished
//       tiles M[K,K+1], M[K+1,K] in stage[k+1 mod 2]              -> ev_diag
//   S : prep_k: the panels R = D_K^{-1} M[K,:], C = M[:,K]    -> ev_fin_ready
//   S4: finish_k: block row K <- R, block column K <- -C D_K^{-1},
//       M[K,K] <- D_K^{-1}, all but the two staged tiles      -> ev_fin[k mod 2]
//   S : (waits finish_{k-1}) update_k, M -= C R over all of M but block row
//       and column K and the block (K+1,K+1)                       -> ev_upd
//   S : waits ev_diag before prep_{k+1}.
// Per block the diagonal chain is one inverse and the update chain one prep
// and one update; finish runs beside the update.  D^{-1}, the panels and the
// staged tiles alternate between two buffers, and every reuse of a buffer
// is ordered after the last reader of its previous contents.
// The diagonal inverse is one latency-bound CTA on the critical path; it asks
// for (and leaves unused) enough dynamic shared memory that no other CTA of
// the factorisation (prep and finish 35 KB, update 66.5 KB) fits beside it on
// its SM, while one CTA of the FP64 assembly (16.5 KB) that may run beside the
// factorisation still does.  Every kernel that runs beside it prefers the
// largest shared-memory carveout, so that an SM running one of them can
// still take the diagonal inverse.
constexpr int GJ_DIAG_EXCL_SMEM = 164 * 1024;

int run_gj_fp32(Ctx &c, float *M, int64_t lda, int prec)
{
    static bool diag_attr = false;
    if (!diag_attr) {
        cudaFuncSetAttribute(k_gj_diag, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             GJ_DIAG_EXCL_SMEM);
        const void *fns[] = {(const void *)k_gj_diag, (const void *)k_gj_prep,
                             (const void *)k_gj_finish, (const void *)k_gj_update_simt};
        for (const void *f : fns)
            cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
        diag_attr = true;
    }
    const int64_t n = c.n;
    cudaMemsetAsync(c.d_info, 0, sizeof(int32_t), c.stream);
    const unsigned gcols = (unsigned)ceil_div(n, GJ_NB);
    float *dinv[2] = {c.d_gj_dinv, c.d_gj_dinv + GJ_NB * GJ_NB};
    float *rt[2] = {c.d_gj_rt, c.d_gj_rt + (size_t)GJ_NB * c.lda};
    float *cb[2] = {c.d_gj_cb, c.d_gj_cb + (size_t)GJ_NB * c.lda};
    float *stg[2] = {c.d_gj_stage, c.d_gj_stage + 2 * GJ_NB * GJ_NB};
    c.tbeg(PH_LU_DIAG);
    k_gj_diag<<<1, 256, GJ_DIAG_EXCL_SMEM, c.stream>>>(n, M, lda, 0, dinv[0], c.d_info, nullptr, nullptr);
    c.tend(PH_LU_DIAG);
    cudaEventRecord(c.ev_upd, c.stream);
    c.launches += 1;
    int kstep = 0;
    for (int64_t k0 = 0; k0 < n; k0 += GJ_NB, ++kstep) {
        const int b = kstep & 1;
        const int64_t k1 = k0 + GJ_NB;
        const bool next = k1 < n;
        if (next) {
            cudaStreamWaitEvent(c.stream2, c.ev_upd, 0);
            if (kstep > 0) cudaStreamWaitEvent(c.stream2, c.ev_fin[b ^ 1], 0);
            c.tbeg(PH_LU_DIAG, c.stream2);
            k_gj_diag<<<1, 256, GJ_DIAG_EXCL_SMEM, c.stream2>>>(n, M, lda, k1, dinv[b ^ 1], c.d_info, dinv[b],
                                                stg[b ^ 1]);
            c.tend(PH_LU_DIAG, c.stream2);
            cudaEventRecord(c.ev_diag, c.stream2);
            c.launches += 1;
        }
        c.tbeg(PH_LU_PANEL);
        k_gj_prep<<<dim3(gcols, 2), 256, 0, c.stream>>>(n, M, lda, k0, dinv[b], rt[b], cb[b],
                                                        kstep > 0 ? stg[b] : nullptr);
        c.tend(PH_LU_PANEL);
        cudaEventRecord(c.ev_fin_ready, c.stream);
        cudaStreamWaitEvent(c.stream4, c.ev_fin_ready, 0);
        c.tbeg(PH_LU_PANEL, c.stream4);
        k_gj_finish<<<dim3(gcols, 2), 256, 0, c.stream4>>>(n, M, lda, k0, dinv[b], rt[b], cb[b],
                                                           next ? k1 : -1);
        c.tend(PH_LU_PANEL, c.stream4);
        cudaEventRecord(c.ev_fin[b], c.stream4);
        if (kstep > 0) cudaStreamWaitEvent(c.stream, c.ev_fin[b ^ 1], 0);
        const int64_t skip0 = next ? k1 : -GJ_NB;
        c.tbeg(PH_LU_UPDATE);
        bool done = false;
        if (prec == NRS_TF32 || prec == NRS_BF16)
            done = launch_tc_gj_update(c, M, lda, k0, cb[b], rt[b], prec, skip0);
        if (!done)
            k_gj_update_simt<<<dim3(gcols, gcols), 256, 0, c.stream>>>(n, M, lda, k0, cb[b], rt[b],
                                                                        skip0);
        c.tend(PH_LU_UPDATE);
        cudaEventRecord(c.ev_upd, c.stream);
        if (next) cudaStreamWaitEvent(c.stream, c.ev_diag, 0);
        else cudaStreamWaitEvent(c.stream, c.ev_fin[b], 0);
        c.launches += 3;
    }
    return 0;
}

}  // namespace nrs
