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

// D^{-1} by Gauss-Jordan on [D | I] with partial pivoting, eight columns at a
// time (one CTA of 256 threads, three barriers per panel of eight columns).
//  * Thread (r, s) = (tid / 4, tid % 4) keeps row r of the augmented matrix in
//    registers: left columns [16 s, 16 s + 16) in Lc, right columns
//    [64 + 16 s, ...) in Rc.  The panel loop is unrolled, so every index is static.
//  * Panel P (columns 8P .. 8P+7): the owners publish the panel columns; warp 0
//    runs partial pivoting on the 64 x 8 panel alone (unused row of largest
//    |value|, lowest row on ties, exactly the choices column-by-column
//    Gauss-Jordan makes) and inverts Pv, the 8 x 8 panel block of the chosen
//    pivot rows, in pivot order.  Then every row is updated at once:
//        pivot rows  W_P <- Pv^{-1} W_P,
//        other rows  W_r <- W_r - (W_r[panel] Pv^{-1}) W_P,
//    which zeroes the panel columns outside the pivot rows and turns the pivot
//    rows' panel block into the identity.
//  * Rows are never moved: at the end the left half of pivot row p_c is e_c,
//    so logical row c of D^{-1} is the right half of physical row p_c.
// Padding rows/columns (kb < 64) are identity.  Dinv is row-major 64 x 64; a
// zero pivot records info.
__global__ void __launch_bounds__(256)
    k_gj_diag(int64_t n, const float *__restrict__ M, int64_t lda, int64_t k0,
              float *__restrict__ Dinv, int32_t *__restrict__ info)
{
    constexpr int NB = GJ_NB, PW = 8, RP = 2 * NB + 4;
    __shared__ float colp[NB][PW + 1];
    __shared__ __align__(16) float prows[PW][RP];
    __shared__ float Pinv[PW][PW];
    __shared__ int piv_s[PW];
    __shared__ int pos[NB];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int r = tid >> 2, s = tid & 3;
    const int kb = (int)min((int64_t)NB, n - k0);
    float Lc[16], Rc[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const int j = 16 * s + i;
        Lc[i] = (r < kb && j < kb) ? M[(k0 + r) + (k0 + j) * lda] : (r == j ? 1.0f : 0.0f);
        Rc[i] = (r == j) ? 1.0f : 0.0f;
    }
    unsigned long long used = 0ull;  // warp 0 only
#pragma unroll
    for (int P = 0; P < NB / PW; ++P) {
        const int slotP = P >> 1, base = (P & 1) * PW;
        __syncwarp();  // this row's readers of colp (previous panel) are done
        if (s == slotP) {
#pragma unroll
            for (int k = 0; k < PW; ++k) colp[r][k] = Lc[base + k];
        }
        __syncthreads();
        if (warp == 0) {
            float va[PW], vb[PW];
#pragma unroll
            for (int k = 0; k < PW; ++k) {
                va[k] = colp[lane][k];
                vb[k] = colp[lane + 32][k];
            }
#pragma unroll
            for (int k = 0; k < PW; ++k) {
                const bool u0 = (used >> lane) & 1ull, u1 = (used >> (lane + 32)) & 1ull;
                const unsigned k0v = u0 ? 0u : (0x80000000u | __float_as_uint(fabsf(va[k])));
                const unsigned k1v = u1 ? 0u : (0x80000000u | __float_as_uint(fabsf(vb[k])));
                const unsigned key = k0v >= k1v ? k0v : k1v;
                const int row = k0v >= k1v ? lane : lane + 32;
                const unsigned mx = __reduce_max_sync(0xffffffffu, key);
                const int p = (int)__reduce_min_sync(0xffffffffu, key == mx ? (unsigned)row : 64u);
                used |= 1ull << p;
                const int owner = p & 31;
                const bool upper = p >= 32;
                float pv[PW];
#pragma unroll
                for (int j = 0; j < PW; ++j)
                    pv[j] = __shfl_sync(0xffffffffu, upper ? vb[j] : va[j], owner);
                const float d = pv[k];
                if (lane == 0) {
                    piv_s[k] = p;
                    pos[p] = PW * P + k;
                    if (d == 0.0f && info) atomicCAS(info, 0, (int)(k0 + PW * P + k + 1));
                }
                if (lane != p) {
                    const float g = va[k] / d;
#pragma unroll
                    for (int j = 0; j < PW; ++j) va[j] -= g * pv[j];
                }
                if (lane + 32 != p) {
                    const float g = vb[k] / d;
#pragma unroll
                    for (int j = 0; j < PW; ++j) vb[j] -= g * pv[j];
                }
            }
            __syncwarp();
            // Pinv = inverse of the pivot rows' original panel block, in pivot
            // order (lane k < 8 holds row k of [Pv | I]; no further pivoting)
            float a[PW], e[PW];
            const int pr = lane < PW ? piv_s[lane] : 0;
#pragma unroll
            for (int j = 0; j < PW; ++j) {
                a[j] = lane < PW ? colp[pr][j] : 0.0f;
                e[j] = (lane == j) ? 1.0f : 0.0f;
            }
#pragma unroll
            for (int k = 0; k < PW; ++k) {
                float bk[2 * PW];
#pragma unroll
                for (int j = 0; j < PW; ++j) {
                    bk[j] = __shfl_sync(0xffffffffu, a[j], k);
                    bk[PW + j] = __shfl_sync(0xffffffffu, e[j], k);
                }
                if (lane != k) {
                    const float f = a[k] / bk[k];
#pragma unroll
                    for (int j = 0; j < PW; ++j) {
                        a[j] -= f * bk[j];
                        e[j] -= f * bk[PW + j];
                    }
                }
            }
            if (lane < PW) {
                float al = 1.0f;  // a[lane] with a static index
#pragma unroll
                for (int j = 0; j < PW; ++j)
                    if (lane == j) al = a[j];
                const float dd = 1.0f / al;
#pragma unroll
                for (int j = 0; j < PW; ++j) Pinv[lane][j] = e[j] * dd;
            }
        }
        __syncthreads();
        // pivot rows publish their (old) rows
        int kr = -1;
#pragma unroll
        for (int k = 0; k < PW; ++k)
            if (piv_s[k] == r) kr = k;
        if (kr >= 0) {
#pragma unroll
            for (int i = 0; i < 16; i += 4) {
                *reinterpret_cast<float4 *>(&prows[kr][16 * s + i]) =
                    make_float4(Lc[i], Lc[i + 1], Lc[i + 2], Lc[i + 3]);
                *reinterpret_cast<float4 *>(&prows[kr][NB + 16 * s + i]) =
                    make_float4(Rc[i], Rc[i + 1], Rc[i + 2], Rc[i + 3]);
            }
        }
        __syncthreads();
        float coef[PW];  // pivot rows: Pinv[kr][k]; others: -(W_r[panel] Pinv)[k]
        if (kr >= 0) {
#pragma unroll
            for (int k = 0; k < PW; ++k) coef[k] = Pinv[kr][k];
        } else {
            float w[PW];
#pragma unroll
            for (int j = 0; j < PW; ++j) w[j] = colp[r][j];
#pragma unroll
            for (int k = 0; k < PW; ++k) {
                float t = 0.0f;
#pragma unroll
                for (int j = 0; j < PW; ++j) t += w[j] * Pinv[j][k];
                coef[k] = -t;
            }
        }
        const float keep = kr >= 0 ? 0.0f : 1.0f;
#pragma unroll
        for (int i = 0; i < 16; i += 4) {
            float4 accl = make_float4(keep * Lc[i], keep * Lc[i + 1], keep * Lc[i + 2], keep * Lc[i + 3]);
            float4 accr = make_float4(keep * Rc[i], keep * Rc[i + 1], keep * Rc[i + 2], keep * Rc[i + 3]);
#pragma unroll
            for (int k = 0; k < PW; ++k) {
                const float4 pl = *reinterpret_cast<const float4 *>(&prows[k][16 * s + i]);
                const float4 pr4 = *reinterpret_cast<const float4 *>(&prows[k][NB + 16 * s + i]);
                accl.x += coef[k] * pl.x;
                accl.y += coef[k] * pl.y;
                accl.z += coef[k] * pl.z;
                accl.w += coef[k] * pl.w;
                accr.x += coef[k] * pr4.x;
                accr.y += coef[k] * pr4.y;
                accr.z += coef[k] * pr4.z;
                accr.w += coef[k] * pr4.w;
            }
            Lc[i] = accl.x;
            Lc[i + 1] = accl.y;
            Lc[i + 2] = accl.z;
            Lc[i + 3] = accl.w;
            Rc[i] = accr.x;
            Rc[i + 1] = accr.y;
            Rc[i + 2] = accr.z;
            Rc[i + 3] = accr.w;
        }
    }
    __syncthreads();
    const int lr = pos[r];
#pragma unroll
    for (int i = 0; i < 16; ++i) Dinv[lr * NB + 16 * s + i] = Rc[i];
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

// Lookahead: the rank-64 update of the next diagonal block only,
// M[K1, K1] -= C[K1, :] R[:, K1] (one CTA), so that its inverse can be taken
// while the rest of the update runs on the main stream.
__global__ void __launch_bounds__(256)
    k_gj_diag_update(int64_t n, float *__restrict__ M, int64_t lda, int64_t k1,
                     const float *__restrict__ Cb, const float *__restrict__ Rt)
{
    constexpr int NB = GJ_NB;
    __shared__ float Cs[NB][NB + 1];
    __shared__ float Rs[NB][NB + 1];
    const int tid = threadIdx.x;
    const int kb = (int)min((int64_t)NB, n - k1);
    {
        float cv[16], rv[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int idx = tid + 256 * q, a = idx & 63, b = idx >> 6;
            cv[q] = b < kb ? Cb[(k1 + b) * NB + a] : 0.0f;
            rv[q] = b < kb ? Rt[(k1 + b) * NB + a] : 0.0f;
        }
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int idx = tid + 256 * q, a = idx & 63, b = idx >> 6;
            Cs[b][a] = cv[q];
            Rs[b][a] = rv[q];
        }
    }
    __syncthreads();
    const int tr = tid & 15, tc = tid >> 4;
    float acc[4][4] = {};
#pragma unroll 8
    for (int t = 0; t < NB; ++t) {
        float a[4], b[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) a[q] = Cs[tr + 16 * q][t];
#pragma unroll
        for (int q = 0; q < 4; ++q) b[q] = Rs[tc + 16 * q][t];
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < 4; ++y) acc[x][y] += a[x] * b[y];
    }
#pragma unroll
    for (int y = 0; y < 4; ++y) {
        const int j = tc + 16 * y;
        if (j >= kb) continue;
#pragma unroll
        for (int x = 0; x < 4; ++x) {
            const int i = tr + 16 * x;
            if (i < kb) M[(k1 + i) + (k1 + j) * lda] -= acc[x][y];
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
    k_gj_diag<<<1, 256, 0, c.stream>>>(n, M, lda, 0, dinv[0], c.d_info);
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
            k_gj_diag_update<<<1, 256, 0, c.stream2>>>(n, M, lda, k1, c.d_gj_cb, c.d_gj_rt);
            k_gj_diag<<<1, 256, 0, c.stream2>>>(n, M, lda, k1, dinv[(kstep + 1) & 1], c.d_info);
            c.tend(PH_LU_DIAG, c.stream2);
            cudaEventRecord(c.ev_diag, c.stream2);
            c.launches += 2;
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
