// gj2.cu -- the explicit FP32 inverse of gj.cu for large systems, by
// Gauss-Jordan elimination blocked on two levels, so that the updates of the
// whole matrix are rank-256 products on the tensor cores rather than rank-64
// ones (which move 8 n^2 bytes of M for only 2 n^2 64 flops: HBM-bound).
//
// Outer step b (block K = [k0, k0 + W), W <= 256 columns):
//   1. the column panel P = M[:, K] is eliminated by four inner Gauss-Jordan
//      steps of 64 columns that touch only P (each: the 64 x 64 diagonal
//      block's inverse with partial pivoting inside the block, k_gj_diag; the
//      scaled block row R = D^{-1} P[Kk, :]; P -= C R, P[Kk, :] = R,
//      P[:, Kk] = -C D^{-1}, P[Kk, Kk] = D^{-1}).  A Gauss-Jordan step acts on
//      a column only through that column's own entries, so these are exactly
//      the inner steps' action on the panel, and P ends as the block column
//      G = E[:, K] of their product E.
//   2. every other column j takes the same four steps at once:
//      M[:, j] <- E M[:, j] = M[:, j] + (G - I_K) M[K, j]
//      (rows K included: they become D_K^{-1} M[K, j]), a rank-W product of
//      the panel G' = G - I_K (n x W) with the old block row T = M[K, :]
//      (W x n), both stored K-major and split into TF32 hi + lo for the
//      split-precision tensor-core product (hi hi + hi lo + lo hi).
// After the last outer step M holds A^{-1}.  Pivoting stays inside 64 x 64
// diagonal blocks, as in gj.cu and lu.cu.
//
// The update (k_tc_gj2_update) is a persistent kernel, one CTA per SM, warp
// specialised: warp 0 loads the operand tiles with TMA (128-byte swizzle)
// into two shared-memory stages, warp 1 issues tcgen05.mma kind::tf32 into
// one of two 128 x 256 FP32 accumulators in tensor memory, warps 2-17 add the
// finished accumulator to M (tcgen05.ld, coalesced column-major
// read-modify-write, four warps per 32 rows) while the next tile's products run.  Every wait is
// bounded: one that runs out sets ST_TIMEOUT, the roles stop, and the CTA
// waits (bounded) for its own copies and products before freeing tensor memory.
#include <cuda.h>
#include <cuda_fp16.h>

#include "tc_prims.cuh"

namespace nrs {

using namespace tcp;

namespace {

constexpr int G2_W = 256;                  // outer block (columns of the panel, K of the product)
constexpr int G2_BM = 128, G2_BN = 256;    // output tile of the update
constexpr int G2_KB = 128;                 // bytes of K per pipeline stage and operand row
constexpr uint32_t G2_A_BYTES = G2_BM * G2_KB;                           // 16 KB
constexpr uint32_t G2_B_BYTES = G2_BN * G2_KB;                           // 32 KB
constexpr uint32_t G2_STAGE_BYTES = 2 * G2_A_BYTES + 2 * G2_B_BYTES;     // 96 KB
constexpr int G2_STAGES = 2;
constexpr int G2_RING = 4;                 // claimed tile indices in flight (producer -> MMA, epilogue)
// SMs the two-level factorisation leaves to the next block's panel elimination
// while the bulk of the current block's update runs
constexpr int GJ2_PANEL_SMS = 24;
constexpr int G2_SMEM = G2_STAGES * G2_STAGE_BYTES + 1024;
constexpr int G2_EPI_WARPS = 16;         // four per accumulator lane quarter, 64 columns each
constexpr int G2_EPI_PARTS = G2_EPI_WARPS / 4;  // column parts of a tile (one warp a lane quarter each)
constexpr int G2_CPW = G2_BN / G2_EPI_PARTS;    // columns of an epilogue warp
static_assert(G2_EPI_WARPS % 4 == 0 && G2_CPW % 32 == 0, "epilogue warps in lane-quarter groups");
constexpr int G2_THREADS = 64 + 32 * G2_EPI_WARPS;
// register budget of about 96 a thread whatever the warp count (the launch
// bound's block count only sets it: one CTA fits an SM), so that the rest of
// the SM's registers stay with the FP64 assembly beside the factorisation
constexpr int G2_MINB = 65536 / (G2_THREADS * 96) > 0 ? 65536 / (G2_THREADS * 96) : 1;
constexpr int G2_TMEM_COLS = 2 * G2_BN;    // two accumulators

__device__ __forceinline__ void g2_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Column tiles of one update launch: [c_lo, c_hi) without [s_lo, s_hi) (an
// empty exclusion has s_lo = s_hi).
struct G2Cols {
    int c_lo, c_hi, s_lo, s_hi;
};

// Output tile t of the update: row tile t % nrt, the (t / nrt)-th column tile
// of the launch's range.
__device__ __forceinline__ void g2_tile(int64_t t, int nrt, const G2Cols &cc, int &rt, int &ct)
{
    rt = (int)(t % nrt);
    ct = cc.c_lo + (int)(t / nrt);
    if (ct >= cc.s_lo) ct += cc.s_hi - cc.s_lo;
}

// L2 prefetch of the lines of M that epilogue warp (lane quarter q, column
// part `part`) of tile t will read: 32 rows x 4 bytes = one 128-byte line per
// column, lane l taking columns l, l + 32, ... of the part's G2_CPW.  Only lines
// whose first row is below n (and so whole inside the column's lda rows).
__device__ __forceinline__ void l2_prefetch_part(const float *M, int64_t lda, int64_t n,
                                                 int64_t t, int nrt, const G2Cols &cc, int q,
                                                 int part, int lane)
{
    int rt, ct;
    g2_tile(t, nrt, cc, rt, ct);
    const int64_t r0 = (int64_t)rt * G2_BM + q * 32;
    if (r0 >= n) return;
#pragma unroll
    for (int k = 0; k < G2_CPW / 32; ++k) {
        const int64_t col = (int64_t)ct * G2_BN + part * G2_CPW + lane + 32 * k;
        if (col < n)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(M + r0 + col * lda) : "memory");
    }
}

// M[i, j] += sum_{c < 256} A[i][c] B[j][c] for all rows i < n and the columns
// j of the 256-wide column tiles `cc`, A = Ah + Al and B = Bh + Bl the
// split panels (row-major, 256 elements a row), products hi hi + hi lo + lo hi.
// F16 = false: TF32 pieces (FP32 storage, kind::tf32, 32 K a stage); true:
// scaled FP16 pieces (kind::f16, 64 K a stage), row i of A and row j of B
// stored times 2^e_i, 2^f_j, undone by sA[i] = 2^-e_i, sB[j] = 2^-f_j here.
template <bool F16>
__global__ void __launch_bounds__(G2_THREADS, G2_MINB)
    k_tc_gj2_update(const __grid_constant__ CUtensorMap tmAh, const __grid_constant__ CUtensorMap tmAl,
                    const __grid_constant__ CUtensorMap tmBh, const __grid_constant__ CUtensorMap tmBl,
                    int64_t n, float *__restrict__ M, int64_t lda, int nrt, G2Cols cc,
                    const float *__restrict__ sA, const float *__restrict__ sB,
                    unsigned long long *__restrict__ claim, int max_tiles, int32_t *status)
{
    constexpr int KC = F16 ? 64 : 32;      // K elements per stage (128 bytes)
    constexpr int NCH = G2_W / KC;         // stages per tile
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t full[G2_STAGES], empty[G2_STAGES], tfull[2], tempty[2], drain;
    __shared__ uint64_t ifull[G2_RING], iempty[G2_RING];  // the ring of claimed tile indices
    __shared__ long long s_tile[G2_RING];
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int s_abort;
    __shared__ float s_scale[G2_EPI_WARPS][G2_CPW];  // FP16 variant: column scales per warp
    uint8_t *base = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t ntiles = (int64_t)nrt * ((cc.c_hi - cc.c_lo) - (cc.s_hi - cc.s_lo));

    if (threadIdx.x == 0) {
        for (int s = 0; s < G2_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&tfull[a], 1);
            mbar_init(&tempty[a], G2_EPI_WARPS);
        }
        for (int r = 0; r < G2_RING; ++r) {
            mbar_init(&ifull[r], 1);
            mbar_init(&iempty[r], 1 + G2_EPI_WARPS);
        }
        mbar_init(&drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_slot)),
                     "r"(G2_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == 0) {
        // ---- producer: claims the next tile from the launch's counter (CTAs
        // that start late, beside other kernels, simply take fewer tiles; at
        // most max_tiles), hands its index to the MMA and epilogue warps
        // through the ring, and loads the four operand tiles of each of its
        // stages by TMA
        if (lane == 0) {
            int64_t it = 0;
            int last_k[G2_STAGES] = {-1, -1};
            for (int64_t lt = 0; !s_abort; ++lt) {
                const int r = (int)(lt % G2_RING), ru = (int)(lt / G2_RING);
                if (!mbar_wait(&iempty[r], (uint32_t)((ru & 1) ^ 1))) {
                    atomicOr(status, ST_TIMEOUT);
                    s_abort = 1;
                    break;
                }
                long long t = -1;
                if (lt < max_tiles) {
                    t = (long long)atomicAdd(claim, 1ULL);
                    if (t >= ntiles) t = -1;
                }
                s_tile[r] = t;
                g2_arrive(&ifull[r]);
                if (t < 0) break;
                int rt, ct;
                g2_tile(t, nrt, cc, rt, ct);
                for (int ch = 0; ch < NCH; ++ch, ++it) {
                    const int s = (int)(it & 1), k = (int)(it >> 1);
                    if (!mbar_wait(&empty[s], (uint32_t)((k & 1) ^ 1))) {
                        atomicOr(status, ST_TIMEOUT);
                        s_abort = 1;
                        break;
                    }
                    uint8_t *st = base + (size_t)s * G2_STAGE_BYTES;
                    mbar_expect_tx(&full[s], G2_STAGE_BYTES);
                    tma_load_2d(st, &tmAh, ch * KC, rt * G2_BM, &full[s]);
                    tma_load_2d(st + G2_A_BYTES, &tmAl, ch * KC, rt * G2_BM, &full[s]);
                    tma_load_2d(st + 2 * G2_A_BYTES, &tmBh, ch * KC, ct * G2_BN, &full[s]);
                    tma_load_2d(st + 2 * G2_A_BYTES + G2_B_BYTES, &tmBl, ch * KC, ct * G2_BN,
                                &full[s]);
                    last_k[s] = k;
                }
            }
            if (s_abort) {
                // the copies already issued land by themselves: wait for them
                for (int s = 0; s < G2_STAGES; ++s)
                    if (last_k[s] >= 0) mbar_wait(&full[s], (uint32_t)(last_k[s] & 1));
            }
        }
    } else if (warp == 1) {
        // ---- MMA issuer: 4 K-steps of 32 bytes (8 TF32 or 16 FP16) x 3 products per stage
        if (lane == 0) {
            constexpr uint32_t idesc = F16 ? idesc_f16(G2_BM, G2_BN) : idesc_tf32(G2_BM, G2_BN);
            int64_t it = 0;
            for (int64_t lt = 0; !s_abort; ++lt) {
                const int r = (int)(lt % G2_RING), ru = (int)(lt / G2_RING);
                if (!mbar_wait(&ifull[r], (uint32_t)(ru & 1))) {
                    atomicOr(status, ST_TIMEOUT);
                    s_abort = 1;
                    break;
                }
                const long long t = s_tile[r];
                g2_arrive(&iempty[r]);
                if (t < 0) break;
                const int a = (int)(lt & 1), u = (int)(lt >> 1);
                if (!mbar_wait(&tempty[a], (uint32_t)((u & 1) ^ 1))) {
                    atomicOr(status, ST_TIMEOUT);
                    s_abort = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(a * G2_BN);
                bool ok = true;
                for (int ch = 0; ch < NCH; ++ch, ++it) {
                    const int s = (int)(it & 1), k = (int)(it >> 1);
                    if (!mbar_wait(&full[s], (uint32_t)(k & 1))) {
                        atomicOr(status, ST_TIMEOUT);
                        s_abort = 1;
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t st = smem_u32(base + (size_t)s * G2_STAGE_BYTES);
#pragma unroll
                    for (int kk = 0; kk < G2_KB / 32; ++kk) {
                        const uint32_t kofs = (uint32_t)kk * 32u;
                        const uint64_t ah = desc_sw128_kmajor(st + kofs);
                        const uint64_t al = desc_sw128_kmajor(st + G2_A_BYTES + kofs);
                        const uint64_t bh = desc_sw128_kmajor(st + 2 * G2_A_BYTES + kofs);
                        const uint64_t bl = desc_sw128_kmajor(st + 2 * G2_A_BYTES + G2_B_BYTES + kofs);
                        if (F16) {
                            mma_f16(d, al, bh, idesc, (ch > 0 || kk > 0) ? 1u : 0u);
                            mma_f16(d, ah, bl, idesc, 1u);
                            mma_f16(d, ah, bh, idesc, 1u);
                        } else {
                            mma_tf32(d, al, bh, idesc, (ch > 0 || kk > 0) ? 1u : 0u);
                            mma_tf32(d, ah, bl, idesc, 1u);
                            mma_tf32(d, ah, bh, idesc, 1u);
                        }
                    }
                    mma_commit(&empty[s]);  // the stage is free once these have read it
                }
                if (!ok) break;
                mma_commit(&tfull[a]);
            }
            // every product issued by this thread is complete before teardown
            mma_commit(&drain);
            mbar_wait(&drain, 0);
        }
    } else {
        // ---- epilogue: warp w reads accumulator lanes 32 (w % 4) .. + 31 (the
        // quarter its rank in the warpgroup may access) and G2_CPW of the 256
        // columns, 16 at a time; the next 16 columns of M (of this tile, or the
        // first ones of the CTA's next tile when its index is already out) are
        // loaded while the current ones are added and stored.  The FP16
        // variant's column scales of the tile are staged once per tile in
        // shared memory.
        constexpr int CW = 16, CPW = G2_CPW, NCHK = CPW / CW;
        const int q = warp & 3, part = (warp - 2) >> 2;
        float *scl = s_scale[warp - 2];
        float *p = nullptr;
        int64_t ncol = 0, row = 0, col0 = 0;
        bool live = false;
        auto setup = [&](int64_t tt) {
            int rt, ct;
            g2_tile(tt, nrt, cc, rt, ct);
            row = (int64_t)rt * G2_BM + q * 32 + lane;
            col0 = (int64_t)ct * G2_BN + part * CPW;
            p = M + row + col0 * lda;
            ncol = n - col0;
            live = row < n;
        };
        float cur[CW], nxt[CW];
        bool prefetched = false;  // cur holds the first columns of the next tile
        for (int64_t lt = 0;; ++lt) {
            const int r = (int)(lt % G2_RING), ru = (int)(lt / G2_RING);
            const bool gi = mbar_wait(&ifull[r], (uint32_t)(ru & 1));
            if (!__all_sync(0xffffffffu, gi) || s_abort) {
                if (lane == 0) {
                    atomicOr(status, ST_TIMEOUT);
                    s_abort = 1;
                }
                break;
            }
            const long long t = s_tile[r];
            __syncwarp();
            if (lane == 0) g2_arrive(&iempty[r]);
            if (t < 0) break;
            if (!prefetched) {
                setup(t);
#pragma unroll
                for (int j = 0; j < CW; ++j)
                    cur[j] = (live && j < ncol) ? __ldcs(p + j * lda) : 0.0f;
            }
            prefetched = false;
            // L2 prefetch of this warp's lines of the tile (one 128-byte line per
            // column: 32 rows of the lane quarter), and of the next tile's when
            // its index is already out, so the loads of M below hit L2 (the
            // FP16 variant, whose products leave the epilogue as the bound;
            // measured slower for the TF32 one)
            if (F16) {
                l2_prefetch_part(M, lda, n, t, nrt, cc, q, part, lane);
                const int r2 = (int)((lt + 1) % G2_RING), ru2 = (int)((lt + 1) / G2_RING);
                if (__all_sync(0xffffffffu, mbar_try_wait(&ifull[r2], (uint32_t)(ru2 & 1)))) {
                    const long long t2 = s_tile[r2];
                    if (t2 >= 0) l2_prefetch_part(M, lda, n, t2, nrt, cc, q, part, lane);
                }
            }
            const int a = (int)(lt & 1), u = (int)(lt >> 1);
            // this tile's geometry (setup() may move on to the next tile below)
            float *const pt = p;
            const int64_t nc = ncol, c0 = col0;
            const bool lv = live;
            const float sa = (F16 && lv) ? __ldg(sA + row) : 1.0f;
            if (F16) {
                for (int c = lane; c < CPW; c += 32) scl[c] = c < nc ? __ldg(sB + c0 + c) : 0.0f;
                __syncwarp();
            }
            const bool got = mbar_wait(&tfull[a], (uint32_t)(u & 1));
            if (!__all_sync(0xffffffffu, got) || s_abort) {
                if (lane == 0) {
                    atomicOr(status, ST_TIMEOUT);
                    s_abort = 1;
                }
                break;
            }
            tc_fence_after();
            const uint32_t tb =
                tmem + (uint32_t)(a * G2_BN + part * CPW) + ((uint32_t)(q * 32) << 16);
            const bool full = lv && nc >= CPW;
#pragma unroll 1
            for (int chunk = 0; chunk < NCHK; ++chunk) {
                uint32_t v[CW];
                tmem_ld_16cols_async(tb + (uint32_t)(chunk * CW), v);
                if (chunk + 1 < NCHK) {
                    const float *pn = pt + (int64_t)(chunk + 1) * CW * lda;
#pragma unroll
                    for (int j = 0; j < CW; ++j)
                        nxt[j] = (lv && (chunk + 1) * CW + j < nc) ? __ldcs(pn + j * lda) : 0.0f;
                } else {
                    // the next tile's first columns, if its index is already out
                    const int r2 = (int)((lt + 1) % G2_RING), ru2 = (int)((lt + 1) / G2_RING);
                    const bool ready =
                        __all_sync(0xffffffffu, mbar_try_wait(&ifull[r2], (uint32_t)(ru2 & 1)));
                    const long long t2 = ready ? s_tile[r2] : -1;
                    if (t2 >= 0) {
                        setup(t2);
#pragma unroll
                        for (int j = 0; j < CW; ++j)
                            nxt[j] = (live && j < ncol) ? __ldcs(p + j * lda) : 0.0f;
                        prefetched = true;
                    }
                }
                tmem_wait_ld();
                float *pc = pt + (int64_t)chunk * CW * lda;
                if (full) {
#pragma unroll
                    for (int j = 0; j < CW; ++j) {
                        float d = __uint_as_float(v[j]);
                        // undo the operands' power-of-two scaling (exact)
                        if (F16) d = (d * sa) * scl[chunk * CW + j];
                        __stcs(pc + j * lda, cur[j] + d);
                    }
                } else if (lv) {
#pragma unroll
                    for (int j = 0; j < CW; ++j) {
                        if (chunk * CW + j >= nc) continue;
                        float d = __uint_as_float(v[j]);
                        if (F16) d = (d * sa) * scl[chunk * CW + j];
                        __stcs(pc + j * lda, cur[j] + d);
                    }
                }
#pragma unroll
                for (int j = 0; j < CW; ++j) cur[j] = nxt[j];
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) g2_arrive(&tempty[a]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(G2_TMEM_COLS)
                     : "memory");
}

// R[a][j] = sum_b Dinv[a][b] M[r0 + b, k0 + j] for the 64 columns
// j in [64 blockIdx.x, +64) of the panel (R[:, own block] = 0), FP32, R
// row-major 64 x 256.  Dinv: row-major 64 x 64 (k_gj_diag).
__global__ void __launch_bounds__(256)
    k_gj2_rpanel(int64_t n, const float *__restrict__ M, int64_t lda, int64_t k0, int W, int64_t r0,
                 const float *__restrict__ Dinv, float *__restrict__ R)
{
    __shared__ float Ds[64][65], Ms[64][65];
    const int tid = threadIdx.x;
    const int j0 = blockIdx.x * 64;
    const int kb = (int)min((int64_t)64, n - r0);
    const int own = (int)(r0 - k0);
    for (int i = tid; i < 64 * 64; i += 256) {
        const int a = i >> 6, b = i & 63;
        Ds[a][b] = Dinv[i];
        // Ms[b][j] = M[r0 + b, k0 + j0 + j] (column j contiguous in b)
        const int jj = i >> 6, bb = i & 63;
        Ms[bb][jj] = (bb < kb && j0 + jj < W) ? __ldcg(M + (r0 + bb) + (k0 + j0 + jj) * lda) : 0.0f;
    }
    __syncthreads();
    const bool own_blk = (j0 == own);
    // thread: rows a0..a0+3, columns jj0..jj0+3
    const int a0 = 4 * (tid >> 4), jj0 = 4 * (tid & 15);
    float acc[4][4] = {};
#pragma unroll 8
    for (int b = 0; b < 64; ++b) {
        float d[4], m[4];
#pragma unroll
        for (int x = 0; x < 4; ++x) {
            d[x] = Ds[a0 + x][b];
            m[x] = Ms[b][jj0 + x];
        }
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(d[x], m[y], acc[x][y]);
    }
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y)
            R[(a0 + x) * G2_W + j0 + jj0 + y] = own_blk ? 0.0f : acc[x][y];
}

// One inner step on the panel, rows [64 blockIdx.x, +64):
//   rows of Kk:      P[Kk, j] = R[:, j] (j outside the own block), P[Kk, Kk] = D^{-1}
//   the other rows:  P[i, j] -= C_i R[:, j],  P[i, Kk] = -C_i D^{-1},  C_i = P[i, Kk]
// FP32 fused multiply-adds in ascending c; P = M[:, k0 .. k0 + W).  A CTA
// computes its 64 rows x all 256 columns at once from shared memory (C^T
// 64 x 64 and the right-hand factor 64 x 256: 80 KB, two CTAs an SM): warp w
// takes rows 8 w .. 8 w + 7, lane l the columns 4 l + {0..3} and 128 + 4 l +
// {0..3}, so each step of c is four 16-byte shared loads (the C ones a
// broadcast, the others conflict-free) for 64 FMAs, and each thread's
// read-modify-write of a column is one 32-byte sector.
constexpr int PU_SMEM = (64 * 64 + 64 * G2_W) * (int)sizeof(float);
static_assert(G2_W == 256, "the panel update's thread layout covers 256 columns");

__global__ void __launch_bounds__(256, 2)
    k_gj2_panel_update(int64_t n, float *__restrict__ M, int64_t lda, int64_t k0, int W, int64_t r0,
                       const float *__restrict__ Dinv, const float *__restrict__ R)
{
    extern __shared__ __align__(16) float pu_smem[];
    float *Cs = pu_smem;            // [c][r] = P[i0 + r, r0 + c]
    float *Rs = pu_smem + 64 * 64;  // [c][j]
    const int tid = threadIdx.x;
    const int64_t i0 = (int64_t)blockIdx.x * 64;
    const int kb = (int)min((int64_t)64, n - r0);
    const int own = (int)(r0 - k0);
    const int rows = (int)min((int64_t)64, n - i0);
    if (i0 == r0) {
        // the diagonal block's rows: R outside the own block, D^{-1} inside
        for (int idx = tid; idx < 64 * W; idx += 256) {
            const int a = idx & 63, j = idx >> 6;
            if (a >= kb) continue;
            const bool in_own = j >= own && j < own + 64;
            const float v = in_own ? (j - own < kb ? Dinv[a * 64 + (j - own)] : 0.0f) : R[a * G2_W + j];
            if (!in_own || j - own < kb) M[(r0 + a) + (k0 + j) * lda] = v;
        }
        return;
    }
    // staging: every load of a thread issued before the first store (16-byte
    // loads, all in flight together), then the stores
    {
        // C^T: four runs of 4 rows of one column each (rows i0 + 4 (t & 15) ..
        // + 3 of column r0 + (t >> 4) + 16 u)
        float4 cv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int idx = tid + 256 * u, r = 4 * (idx & 15), c = idx >> 4;
            const float *src = M + (i0 + r) + (r0 + c) * lda;
            if (c < kb && r + 4 <= rows)
                cv[u] = *reinterpret_cast<const float4 *>(src);
            else
                cv[u] = make_float4(c < kb && r < rows ? src[0] : 0.0f,
                                    c < kb && r + 1 < rows ? src[1] : 0.0f,
                                    c < kb && r + 2 < rows ? src[2] : 0.0f,
                                    c < kb && r + 3 < rows ? src[3] : 0.0f);
        }
        // the right-hand factor: R outside the own block, D^{-1} inside (zero
        // beyond kb rows and W columns), 16 runs of 4 columns of one row
        float4 rv[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int idx = tid + 256 * u, j = 4 * (idx & 63), c = idx >> 6;
            const bool in_own = j >= own && j < own + 64;
            const float *src = in_own ? Dinv + c * 64 + (j - own) : R + c * G2_W + j;
            const int lim = in_own ? own + kb : W;  // columns below lim are live
            if (c < kb && j + 4 <= lim)
                rv[u] = *reinterpret_cast<const float4 *>(src);
            else
                rv[u] = make_float4(c < kb && j < lim ? src[0] : 0.0f,
                                    c < kb && j + 1 < lim ? src[1] : 0.0f,
                                    c < kb && j + 2 < lim ? src[2] : 0.0f,
                                    c < kb && j + 3 < lim ? src[3] : 0.0f);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int idx = tid + 256 * u, r = 4 * (idx & 15), c = idx >> 4;
            *reinterpret_cast<float4 *>(Cs + c * 64 + r) = cv[u];
        }
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int idx = tid + 256 * u, j = 4 * (idx & 63), c = idx >> 6;
            *reinterpret_cast<float4 *>(Rs + c * G2_W + j) = rv[u];
        }
    }
    __syncthreads();
    const int rg = tid >> 5, cg = tid & 31;
    float acc[8][8];
#pragma unroll
    for (int x = 0; x < 8; ++x)
#pragma unroll
        for (int y = 0; y < 8; ++y) acc[x][y] = 0.0f;
#pragma unroll 4
    for (int c = 0; c < 64; ++c) {
        const float4 ca = *reinterpret_cast<const float4 *>(Cs + c * 64 + 8 * rg);
        const float4 cb = *reinterpret_cast<const float4 *>(Cs + c * 64 + 8 * rg + 4);
        const float4 ba = *reinterpret_cast<const float4 *>(Rs + c * G2_W + 4 * cg);
        const float4 bb = *reinterpret_cast<const float4 *>(Rs + c * G2_W + 128 + 4 * cg);
        const float cv[8] = {ca.x, ca.y, ca.z, ca.w, cb.x, cb.y, cb.z, cb.w};
        const float rv[8] = {ba.x, ba.y, ba.z, ba.w, bb.x, bb.y, bb.z, bb.w};
#pragma unroll
        for (int x = 0; x < 8; ++x)
#pragma unroll
            for (int y = 0; y < 8; ++y) acc[x][y] = fmaf(cv[x], rv[y], acc[x][y]);
    }
    const bool full = 8 * rg + 8 <= rows;
#pragma unroll
    for (int y = 0; y < 8; ++y) {
        const int j = (y < 4 ? 4 * cg : 128 + 4 * cg) + (y & 3);
        if (j >= W) continue;
        const bool in_own = j >= own && j < own + 64;
        if (in_own && j - own >= kb) continue;
        float *p = M + (k0 + j) * lda + i0 + 8 * rg;
        if (full) {
            // lda is a multiple of 32 and i0 of 64: 32-byte aligned
            float4 *p4 = reinterpret_cast<float4 *>(p);
            float4 u = in_own ? make_float4(0.f, 0.f, 0.f, 0.f) : p4[0];
            float4 v = in_own ? make_float4(0.f, 0.f, 0.f, 0.f) : p4[1];
            if (in_own) {
                u = make_float4(-acc[0][y], -acc[1][y], -acc[2][y], -acc[3][y]);
                v = make_float4(-acc[4][y], -acc[5][y], -acc[6][y], -acc[7][y]);
            } else {
                u = make_float4(u.x - acc[0][y], u.y - acc[1][y], u.z - acc[2][y], u.w - acc[3][y]);
                v = make_float4(v.x - acc[4][y], v.y - acc[5][y], v.z - acc[6][y], v.w - acc[7][y]);
            }
            p4[0] = u;
            p4[1] = v;
        } else {
#pragma unroll
            for (int x = 0; x < 8; ++x) {
                if (8 * rg + x >= rows) continue;
                p[x] = in_own ? -acc[x][y] : p[x] - acc[x][y];
            }
        }
    }
}

// The product's operands, split into TF32 hi (cvt.rna) and lo = x - hi:
//   bpart = 0: A[i][c] = M[i, k0 + c] - (i == k0 + c) for c < W (0 for c >= W
//              and rows >= n), 64 rows x 64 columns (blockIdx.y) a CTA through
//              shared memory (grid.y = 4);
//   bpart = 1: B[j][c] = M[k0 + c, j] for c < W, j outside [k0, k0 + W)
//              (0 otherwise), 64 columns j a CTA: one contiguous run of M each.
// Both row-major with 256 floats a row, rows up to `rows_pad`.
__global__ void __launch_bounds__(256)
    k_gj2_prep(int64_t n, const float *__restrict__ M, int64_t lda, int64_t k0, int W,
               int64_t rows_pad, int bpart, float *__restrict__ Ah, float *__restrict__ Al,
               float *__restrict__ Bh, float *__restrict__ Bl)
{
    __shared__ float T[64][65];
    const int tid = threadIdx.x;
    const int64_t i0 = (int64_t)blockIdx.x * 64;
    if (i0 >= rows_pad) return;
    if (!bpart) {
        const int c0 = blockIdx.y * 64;
        for (int idx = tid; idx < 64 * 64; idx += 256) {
            const int r = idx & 63, c = idx >> 6;
            const int64_t i = i0 + r;
            float v = 0.0f;
            if (i < n && c0 + c < W) {
                v = M[i + (k0 + c0 + c) * lda];
                if (i == k0 + c0 + c) v -= 1.0f;
            }
            T[r][c] = v;
        }
        __syncthreads();
        for (int idx = tid; idx < 64 * 64; idx += 256) {
            const int c = idx & 63, r = idx >> 6;
            float h, l;
            split_tf32(T[r][c], h, l);
            Ah[(i0 + r) * G2_W + c0 + c] = h;
            Al[(i0 + r) * G2_W + c0 + c] = l;
        }
    } else {
        for (int idx = tid; idx < 64 * G2_W; idx += 256) {
            const int c = idx & (G2_W - 1), jr = idx >> 8;
            const int64_t j = i0 + jr;
            float v = 0.0f;
            if (j < n && c < W && !(j >= k0 && j < k0 + W)) v = M[(k0 + c) + j * lda];
            float h, l;
            split_tf32(v, h, l);
            Bh[j * G2_W + c] = h;
            Bl[j * G2_W + c] = l;
        }
    }
}

// Power of two 2^e bringing the magnitude m > 0 into [2^14, 2^15) (e clamped
// to [-100, 100]; 0 for m = 0), as e.
__device__ __forceinline__ int g2_scale_exp(float m)
{
    if (!(m > 0.0f) || !isfinite(m)) return 0;
    return max(-100, min(100, 14 - ilogbf(m)));
}

__device__ __forceinline__ float g2_pow2(int e) { return __int_as_float((127 + e) << 23); }

// x (already scaled) as hi = fp16(x) and lo = fp16(x - hi): about 22 bits of x,
// the FP16 analogue of split_tf32 (x - hi is exact in FP32).
__device__ __forceinline__ void split_f16(float x, __half &hi, __half &lo)
{
    hi = __float2half_rn(x);
    lo = __float2half_rn(x - __half2float(hi));
}

// The product's operands as scaled FP16 pairs (the FP16 variant of k_gj2_prep):
// row i of A = G - I_K and row j of B (column j of the block row) are each
// multiplied by the power of two 2^e that brings their largest magnitude into
// [2^14, 2^15) -- so no piece overflows FP16 and the low pieces stay above
// its subnormal range except for entries below 2^-24 of their row's maximum --
// then split (split_f16); sA[i] = 2^-e_i, sB[j] = 2^-f_j.
//   bpart = 0: A rows [64 blockIdx.x, +64): the row maxima first (a thread
//              per row and quarter of the 256 columns), then 64 x 64 column
//              chunks transposed through shared memory;
//   bpart = 1: B rows j in [64 blockIdx.x, +64), a warp per 8 of them.
// Both row-major with 256 halves a row, rows up to `rows_pad`.
__global__ void __launch_bounds__(256)
    k_gj2_prep16(int64_t n, const float *__restrict__ M, int64_t lda, int64_t k0, int W,
                 int64_t rows_pad, int bpart, __half *__restrict__ Ah, __half *__restrict__ Al,
                 __half *__restrict__ Bh, __half *__restrict__ Bl, float *__restrict__ sA,
                 float *__restrict__ sB)
{
    __shared__ float T[64][65];
    __shared__ float smax[4][64];
    __shared__ float sscale[64];
    const int tid = threadIdx.x;
    const int64_t i0 = (int64_t)blockIdx.x * 64;
    if (i0 >= rows_pad) return;
    if (!bpart) {
        {
            const int r = tid & 63, qc = tid >> 6;
            const int64_t i = i0 + r;
            float m = 0.0f;
            if (i < n)
                for (int c = qc * 64; c < qc * 64 + 64 && c < W; ++c) {
                    float v = M[i + (k0 + c) * lda];
                    if (i == k0 + c) v -= 1.0f;
                    m = fmaxf(m, fabsf(v));
                }
            smax[qc][r] = m;
        }
        __syncthreads();
        if (tid < 64) {
            const float m = fmaxf(fmaxf(smax[0][tid], smax[1][tid]), fmaxf(smax[2][tid], smax[3][tid]));
            const int e = g2_scale_exp(m);
            sscale[tid] = g2_pow2(e);
            sA[i0 + tid] = g2_pow2(-e);
        }
        for (int c0 = 0; c0 < G2_W; c0 += 64) {
            __syncthreads();
            for (int idx = tid; idx < 64 * 64; idx += 256) {
                const int r = idx & 63, c = idx >> 6;
                const int64_t i = i0 + r;
                float v = 0.0f;
                if (i < n && c0 + c < W) {
                    v = M[i + (k0 + c0 + c) * lda];
                    if (i == k0 + c0 + c) v -= 1.0f;
                }
                T[r][c] = v;
            }
            __syncthreads();
            for (int idx = tid; idx < 64 * 64; idx += 256) {
                const int c = idx & 63, r = idx >> 6;
                __half h, l;
                split_f16(T[r][c] * sscale[r], h, l);
                Ah[(i0 + r) * G2_W + c0 + c] = h;
                Al[(i0 + r) * G2_W + c0 + c] = l;
            }
        }
    } else {
        const int warp = tid >> 5, lane = tid & 31;
        for (int jr = warp; jr < 64; jr += 8) {
            const int64_t j = i0 + jr;
            const bool col_live = j < n && !(j >= k0 && j < k0 + W);
            float v[G2_W / 32];
            float m = 0.0f;
#pragma unroll
            for (int t = 0; t < G2_W / 32; ++t) {
                const int c = lane + 32 * t;
                v[t] = (col_live && c < W) ? M[(k0 + c) + j * lda] : 0.0f;
                m = fmaxf(m, fabsf(v[t]));
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
            const int e = g2_scale_exp(m);
            const float sc = g2_pow2(e);
#pragma unroll
            for (int t = 0; t < G2_W / 32; ++t) {
                __half h, l;
                split_f16(v[t] * sc, h, l);
                Bh[j * G2_W + lane + 32 * t] = h;
                Bl[j * G2_W + lane + 32 * t] = l;
            }
            if (lane == 0) sB[j] = g2_pow2(-e);
        }
    }
}

typedef CUresult (*EncodeTiledFn2)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                   const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                   const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn2 encode_fn2()
{
    static EncodeTiledFn2 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn2>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

// 2-D map over a row-major [rows][256] panel of FP32 (f16 = false) or FP16
// elements, boxes of 128 bytes x box_rows with 128-byte swizzle; rows >=
// `rows` read as zero.
bool make_panel256_map(CUtensorMap *tm, const void *ptr, int64_t rows, int box_rows, bool f16)
{
    EncodeTiledFn2 enc = encode_fn2();
    if (!enc) return false;
    const size_t es = f16 ? 2 : 4;
    cuuint64_t dims[2] = {(cuuint64_t)G2_W, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)G2_W * es};
    cuuint32_t box[2] = {(cuuint32_t)(G2_KB / es), (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    return enc(tm, f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
               const_cast<void *>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool gj2_supported(const Ctx &c)
{
    return tc_available() && encode_fn2() != nullptr && c.n >= 2 * G2_W;
}

size_t gj2_panel_floats(int64_t n)
{
    // rows of the panels padded to the update's 256-row tiles
    return (size_t)ceil_div(n, G2_BN) * G2_BN * G2_W;
}

size_t gj2_workspace_bytes(int64_t n)
{
    // two A panels (hi, lo) and one B panel (hi, lo) of FP32 at most, and the
    // FP16 variant's three scale vectors
    // and the update launches' tile-claim counters (two per block)
    return 6 * sizeof(float) * gj2_panel_floats(n) +
           3 * sizeof(float) * ceil_div(n, G2_BN) * G2_BN +
           2 * sizeof(unsigned long long) * ceil_div(n, G2_BN);
}

// The two-level factorisation of the FP32 matrix M (n x n, column-major) in
// place, in c.d_gj2 (gj2_workspace_bytes(n)): the A operand (the eliminated
// panel G - I_K, split) in two buffers, the B operand (the block row, split),
// and for the FP16 pieces the scales; the inner scaled block row in c.d_gj2_r
// (64 x 256 floats).  f16: the update's products from scaled FP16 pieces
// instead of TF32 ones.  Returns 0, or -1 if the tensor maps could not be made.
//
// Schedule, block b = columns K_b (stream S = c.stream2, U = c.stream):
//   S: [wait N_{b-1}] panel elimination of K_b, A operand of b -> event A
//   U: [wait A] B operand of b (block row M[K_b, :]); the update of the
//      columns K_{b+1} alone -> event N_b; the update of every other column
//      tile but K_b, on all SMs but GJ2_PANEL_SMS
// so the panel of b + 1 runs beside the bulk of the update of b.  The panel
// touches only the columns K_{b+1}, which the bulk does not; the B operand of
// b + 1 reads the block row after the bulk of b, in stream order.  The A
// operand alternates between its two buffers: S writes that of b + 1 after
// N_b, which U records after the bulk of b - 1 (the last reader of that buffer).
int run_gj2_fp32(Ctx &c, float *M, int64_t lda, bool f16)
{
    const int64_t n = c.n;
    const int64_t rows_pad = ceil_div(n, G2_BN) * G2_BN;
    const size_t pf = gj2_panel_floats(n);
    const size_t es = f16 ? 2 : 4;
    uint8_t *w = reinterpret_cast<uint8_t *>(c.d_gj2);
    void *Ah[2] = {w, w + 2 * pf * es}, *Al[2] = {w + pf * es, w + 3 * pf * es};
    void *Bh = w + 4 * pf * es, *Bl = w + 5 * pf * es;
    // the FP16 variant's row scales (one vector per A buffer) and column
    // scales, then the update launches' tile-claim counters
    float *sA[2] = {nullptr, nullptr}, *sB = nullptr;
    unsigned long long *claims = reinterpret_cast<unsigned long long *>(
        w + 6 * pf * sizeof(float) + 3 * sizeof(float) * rows_pad);
    if (f16) {
        sA[0] = reinterpret_cast<float *>(w + 6 * pf * es);
        sA[1] = sA[0] + rows_pad;
        sB = sA[1] + rows_pad;
    }
    CUtensorMap mAh[2], mAl[2], mBh, mBl;
    for (int k = 0; k < 2; ++k)
        if (!make_panel256_map(&mAh[k], Ah[k], rows_pad, G2_BM, f16) ||
            !make_panel256_map(&mAl[k], Al[k], rows_pad, G2_BM, f16))
            return -1;
    if (!make_panel256_map(&mBh, Bh, rows_pad, G2_BN, f16) ||
        !make_panel256_map(&mBl, Bl, rows_pad, G2_BN, f16))
        return -1;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_tc_gj2_update<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             G2_SMEM);
        cudaFuncSetAttribute(k_tc_gj2_update<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             G2_SMEM);
        cudaFuncSetAttribute(k_gj2_panel_update, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             PU_SMEM);
        attr = true;
    }
    const size_t diag_smem = gj_diag_smem();
    gj_diag_prepare();
    cudaMemsetAsync(c.d_info, 0, sizeof(int32_t), c.stream);
    const int nrt = (int)ceil_div(n, G2_BM), nct = (int)ceil_div(n, G2_BN);
    const unsigned gx = (unsigned)ceil_div(rows_pad, 64);
    cudaStream_t S = c.stream2, U = c.stream;

    auto panel = [&](int b) {
        const int64_t k0 = (int64_t)b * G2_W;
        const int W = (int)std::min<int64_t>(G2_W, n - k0);
        const int buf = b & 1;
        c.tbeg(PH_LU_PANEL, S);
        for (int64_t r0 = k0; r0 < k0 + W; r0 += 64) {
            k_gj_diag_launch(c, n, M, lda, r0, c.d_gj_dinv, diag_smem, S);
            k_gj2_rpanel<<<(unsigned)ceil_div(W, 64), 256, 0, S>>>(n, M, lda, k0, W, r0,
                                                                 c.d_gj_dinv, c.d_gj2_r);
            k_gj2_panel_update<<<(unsigned)ceil_div(n, 64), 256, PU_SMEM, S>>>(
                n, M, lda, k0, W, r0, c.d_gj_dinv, c.d_gj2_r);
            c.launches += 3;
        }
        if (f16)
            k_gj2_prep16<<<gx, 256, 0, S>>>(n, M, lda, k0, W, rows_pad, 0, (__half *)Ah[buf],
                                            (__half *)Al[buf], nullptr, nullptr, sA[buf], nullptr);
        else
            k_gj2_prep<<<dim3(gx, 4), 256, 0, S>>>(n, M, lda, k0, W, rows_pad, 0,
                                                  (float *)Ah[buf], (float *)Al[buf], nullptr,
                                                  nullptr);
        c.launches += 1;
        c.tend(PH_LU_PANEL, S);
        cudaEventRecord(c.ev_diag, S);  // A operand of b ready
    };
    // Each update launch claims its tiles from its own counter (zeroed once
    // per factorisation).  The bulk leaves GJ2_PANEL_SMS SMs to the next
    // block's panel kernels (on the higher-priority stream S); its CTAs are
    // persistent and claim tiles until none are left, so CTAs that start late
    // simply take fewer.
    int launch = 0;
    auto update = [&](int b, G2Cols cc, bool bulk) {
        const int buf = b & 1;
        const int64_t tiles = (int64_t)nrt * ((cc.c_hi - cc.c_lo) - (cc.s_hi - cc.s_lo));
        const int sms = bulk ? std::max(1, c.num_sms - GJ2_PANEL_SMS) : c.num_sms;
        const int grid = (int)std::min<int64_t>(tiles, sms);
        const int cap = (int)tiles;  // no cap: the CTAs run until the counter is spent
        unsigned long long *ctr = claims + launch++;
        if (f16)
            k_tc_gj2_update<true><<<grid, G2_THREADS, G2_SMEM, U>>>(
                mAh[buf], mAl[buf], mBh, mBl, n, M, lda, nrt, cc, sA[buf], sB, ctr, cap,
                c.d_status);
        else
            k_tc_gj2_update<false><<<grid, G2_THREADS, G2_SMEM, U>>>(
                mAh[buf], mAl[buf], mBh, mBl, n, M, lda, nrt, cc, nullptr, nullptr, ctr, cap,
                c.d_status);
        c.launches += 1;
    };

    cudaMemsetAsync(claims, 0, sizeof(unsigned long long) * 2 * nct, U);
    cudaEventRecord(c.ev_fin_ready, U);  // the FP32 matrix is ready
    cudaStreamWaitEvent(S, c.ev_fin_ready, 0);
    panel(0);
    for (int b = 0; b < nct; ++b) {
        const int64_t k0 = (int64_t)b * G2_W;
        const int W = (int)std::min<int64_t>(G2_W, n - k0);
        cudaStreamWaitEvent(U, c.ev_diag, 0);
        c.tbeg(PH_LU_UPDATE, U);
        if (f16)
            k_gj2_prep16<<<gx, 256, 0, U>>>(n, M, lda, k0, W, rows_pad, 1, nullptr, nullptr,
                                            (__half *)Bh, (__half *)Bl, nullptr, sB);
        else
            k_gj2_prep<<<dim3(gx, 1), 256, 0, U>>>(n, M, lda, k0, W, rows_pad, 1, nullptr,
                                                  nullptr, (float *)Bh, (float *)Bl);
        c.launches += 1;
        const bool next = b + 1 < nct;
        if (next) {
            update(b, G2Cols{b + 1, b + 2, b + 2, b + 2}, false);
            cudaEventRecord(c.ev_upd, U);  // the columns of K_{b+1} are up to date
            cudaStreamWaitEvent(S, c.ev_upd, 0);
            panel(b + 1);
        }
        // every other column tile but K_b (and K_{b+1}, done above)
        const int s_hi = next ? b + 2 : b + 1;
        if ((nct - (s_hi - b)) > 0) update(b, G2Cols{0, nct, b, s_hi}, true);
        c.tend(PH_LU_UPDATE, U);
    }
    return 0;
}

}  // namespace nrs
