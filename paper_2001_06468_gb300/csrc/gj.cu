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
#include "tc_prims.cuh"

namespace nrs {

constexpr int GJ_NB = 64;

// Shared state of the pipelined elimination below (dynamic shared memory of
// k_gj_diag): per pivot step c an mbarrier, the 64 multipliers, the pivot row
// and 1/pivot; per warp a double-buffered copy of the pivot row's half.
struct GjElimSmem {
    uint64_t bar[GJ_NB];             // step c published (32 arrivals of the leader's lanes)
    float2 f[GJ_NB][32];             // step c: multipliers of rows l (x) and l + 32 (y)
    __align__(16) float prow[2][2][36];  // [warp][step parity]: the pivot row's half, 1/pivot
    int piv[GJ_NB];                  // pivot row of step c
    float rpiv[GJ_NB];               // 1/pivot of step c
};

__device__ __forceinline__ void gje_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tcp::smem_u32(bar)) : "memory");
}

// The elimination of gj_diag_block (threads 0..63) as a two-warp pipeline.
// Warp w holds columns [32 w, 32 w + 32) of all 64 rows; lane l holds rows l
// (X0) and l + 32 (X1).  The 32 steps of the columns in a warp's own half are
// led by that warp: it finds the pivot by itself (the unused row of largest
// |T[c]|, lowest row on ties: one warp max-reduction and two ballots, no
// barrier), passes the pivot row's half to its lanes through shared memory,
// updates its half with its registers rotating as in the one-row-per-lane
// form, and publishes the step -- pivot row, 1/pivot and the 64 multipliers
// f_i = T_i[c] / T_p[c] (0 for the pivot row) -- in a slot of its own,
// completed by an mbarrier.  The other warp follows: it waits for each slot
// (reading the next one while the current update runs), passes the pivot
// row's other half among its lanes and applies T_i[j] -= f_i T_p[j] to all of
// its columns.  The leader never waits for the follower (one slot per step),
// so the two warps' updates overlap and a pivot step costs one warp's search
// plus half a row of updates.  At column 32 the warps swap roles.  Every
// element goes through the same operations as in the one-row-per-lane form
// (same pivot, same multiplier, same fmaf, same deferred scaling), so the
// result is the same bit for bit.  A slot wait that runs out sets
// ST_TIMEOUT in `status` and ends the elimination.
__device__ __forceinline__ void gj_elim_split(float (*sm0)[GJ_NB + 1], GjElimSmem &E, int64_t k0,
                                              int32_t *info, int32_t *status)
{
    constexpr int NB = GJ_NB, H = 32;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __shared__ unsigned zat[2];
    float X0[H], X1[H];
#pragma unroll
    for (int j = 0; j < H; ++j) {
        X0[j] = sm0[lane][H * w + j];
        X1[j] = sm0[lane + H][H * w + j];
    }
    bool used0 = false, used1 = false;
    float scale0 = 1.0f, scale1 = 1.0f;
    int pos0 = 0, pos1 = 0;
    unsigned zero_at = 0xffffffffu;  // step of a zero pivot in this lane's rows, if any
    bool ok = true;
    for (int ph = 0; ph < 2 && ok; ++ph) {
        if (w == ph) {
#pragma unroll 8
            for (int s = 0; s < H; ++s) {
                const int c = H * ph + s, b = c & 1;
                const float colv0 = X0[0], colv1 = X1[0];
                const float myr0 = 1.0f / colv0, myr1 = 1.0f / colv1;
                const unsigned key0 = used0 ? 0u : (0x80000000u | __float_as_uint(fabsf(colv0)));
                const unsigned key1 = used1 ? 0u : (0x80000000u | __float_as_uint(fabsf(colv1)));
                const unsigned mx = __reduce_max_sync(0xffffffffu, max(key0, key1));
                const unsigned bal0 = __ballot_sync(0xffffffffu, key0 == mx);
                const unsigned bal1 = __ballot_sync(0xffffffffu, key1 == mx);
                // rows l come before rows l + 32
                const int p = bal0 ? __ffs(bal0) - 1 : H - 1 + __ffs(bal1);
                const bool in1 = p >= H;
                float4 *buf = reinterpret_cast<float4 *>(&E.prow[w][b][0]);
                if (lane == (p & (H - 1))) {
                    if (in1) {
#pragma unroll
                        for (int q = 0; q < H / 4; ++q)
                            buf[q] = make_float4(X1[4 * q], X1[4 * q + 1], X1[4 * q + 2], X1[4 * q + 3]);
                        buf[H / 4] = make_float4(myr1, 0.0f, 0.0f, 0.0f);
                    } else {
#pragma unroll
                        for (int q = 0; q < H / 4; ++q)
                            buf[q] = make_float4(X0[4 * q], X0[4 * q + 1], X0[4 * q + 2], X0[4 * q + 3]);
                        buf[H / 4] = make_float4(myr0, 0.0f, 0.0f, 0.0f);
                    }
                }
                __syncwarp();
                const float rpiv = E.prow[w][b][H];
                float4 v[H / 4];
#pragma unroll
                for (int q = 0; q < H / 4; ++q) v[q] = buf[q];
                const bool is0 = !in1 && lane == p, is1 = in1 && lane == p - H;
                const float f0 = is0 ? 0.0f : colv0 * rpiv;
                const float f1 = is1 ? 0.0f : colv1 * rpiv;
                E.f[c][lane] = make_float2(f0, f1);
                if (lane == 0) {
                    E.piv[c] = p;
                    E.rpiv[c] = rpiv;
                }
                gje_arrive(&E.bar[c]);
                if (is0) {
                    used0 = true;
                    scale0 = rpiv;
                    pos0 = c;
                    if (colv0 == 0.0f) zero_at = (unsigned)c;
                }
                if (is1) {
                    used1 = true;
                    scale1 = rpiv;
                    pos1 = c;
                    if (colv1 == 0.0f) zero_at = (unsigned)c;
                }
                // the next pivot column first
                X0[1] = fmaf(-f0, v[0].y, X0[1]);
                X1[1] = fmaf(-f1, v[0].y, X1[1]);
                X0[2] = fmaf(-f0, v[0].z, X0[2]);
                X1[2] = fmaf(-f1, v[0].z, X1[2]);
                X0[3] = fmaf(-f0, v[0].w, X0[3]);
                X1[3] = fmaf(-f1, v[0].w, X1[3]);
#pragma unroll
                for (int q = 1; q < H / 4; ++q) {
                    X0[4 * q] = fmaf(-f0, v[q].x, X0[4 * q]);
                    X0[4 * q + 1] = fmaf(-f0, v[q].y, X0[4 * q + 1]);
                    X0[4 * q + 2] = fmaf(-f0, v[q].z, X0[4 * q + 2]);
                    X0[4 * q + 3] = fmaf(-f0, v[q].w, X0[4 * q + 3]);
                    X1[4 * q] = fmaf(-f1, v[q].x, X1[4 * q]);
                    X1[4 * q + 1] = fmaf(-f1, v[q].y, X1[4 * q + 1]);
                    X1[4 * q + 2] = fmaf(-f1, v[q].z, X1[4 * q + 2]);
                    X1[4 * q + 3] = fmaf(-f1, v[q].w, X1[4 * q + 3]);
                }
#pragma unroll
                for (int j = 0; j < H - 1; ++j) {
                    X0[j] = X0[j + 1];
                    X1[j] = X1[j + 1];
                }
                X0[H - 1] = is0 ? 1.0f : -f0;
                X1[H - 1] = is1 ? 1.0f : -f1;
            }
        } else {
            const int c0 = H * ph;
            bool got = tcp::mbar_wait(&E.bar[c0], 0);
            if (!__all_sync(0xffffffffu, got)) {
                ok = false;
                break;
            }
            int pn = E.piv[c0];
            float rpn = E.rpiv[c0];
            float2 fn = E.f[c0][lane];
#pragma unroll 4
            for (int s = 0; s < H; ++s) {
                const int c = c0 + s, b = c & 1;
                const int p = pn;
                const float rp = rpn;
                const float2 f = fn;
                const bool in1 = p >= H;
                float4 *buf = reinterpret_cast<float4 *>(&E.prow[w][b][0]);
                if (lane == (p & (H - 1))) {
                    if (in1) {
#pragma unroll
                        for (int q = 0; q < H / 4; ++q)
                            buf[q] = make_float4(X1[4 * q], X1[4 * q + 1], X1[4 * q + 2], X1[4 * q + 3]);
                    } else {
#pragma unroll
                        for (int q = 0; q < H / 4; ++q)
                            buf[q] = make_float4(X0[4 * q], X0[4 * q + 1], X0[4 * q + 2], X0[4 * q + 3]);
                    }
                }
                __syncwarp();
                float4 v[H / 4];
#pragma unroll
                for (int q = 0; q < H / 4; ++q) v[q] = buf[q];
                if (s + 1 < H) {
                    got = tcp::mbar_wait(&E.bar[c + 1], 0);
                    if (!__all_sync(0xffffffffu, got)) {
                        ok = false;
                        break;
                    }
                    pn = E.piv[c + 1];
                    rpn = E.rpiv[c + 1];
                    fn = E.f[c + 1][lane];
                }
                if (!in1 && lane == p) {
                    used0 = true;
                    scale0 = rp;
                    pos0 = c;
                }
                if (in1 && lane == p - H) {
                    used1 = true;
                    scale1 = rp;
                    pos1 = c;
                }
#pragma unroll
                for (int q = 0; q < H / 4; ++q) {
                    X0[4 * q] = fmaf(-f.x, v[q].x, X0[4 * q]);
                    X0[4 * q + 1] = fmaf(-f.x, v[q].y, X0[4 * q + 1]);
                    X0[4 * q + 2] = fmaf(-f.x, v[q].z, X0[4 * q + 2]);
                    X0[4 * q + 3] = fmaf(-f.x, v[q].w, X0[4 * q + 3]);
                    X1[4 * q] = fmaf(-f.y, v[q].x, X1[4 * q]);
                    X1[4 * q + 1] = fmaf(-f.y, v[q].y, X1[4 * q + 1]);
                    X1[4 * q + 2] = fmaf(-f.y, v[q].z, X1[4 * q + 2]);
                    X1[4 * q + 3] = fmaf(-f.y, v[q].w, X1[4 * q + 3]);
                }
            }
        }
    }
    if (!ok && lane == 0 && status) atomicOr(status, ST_TIMEOUT);
    zero_at = __reduce_min_sync(0xffffffffu, zero_at);
    if (lane == 0) zat[w] = zero_at;
    asm volatile("bar.sync 1, 64;" ::: "memory");  // the pivot order is complete
    if (threadIdx.x == 0 && info) {
        const unsigned z = min(zat[0], zat[1]);
        if (z != 0xffffffffu) atomicCAS(info, 0, (int)(k0 + z + 1));
    }
    // row pos of D^{-1}; this warp's column 32 w + j stands for original row
    // piv[32 w + j] (masked: after a timeout not every slot was written)
#pragma unroll
    for (int j = 0; j < H; ++j) {
        const int col = E.piv[H * w + j] & (NB - 1);
        sm0[pos0][col] = X0[j] * scale0;
        sm0[pos1][col] = X1[j] * scale1;
    }
}

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
// The elimination (SPLIT = false, the fused factorisation, whose 128-register
// budget it fits; SPLIT = true, k_gj_diag, runs the same arithmetic as the
// two-warp pipeline gj_elim_split above): two warps, lane l of warp w holding
// row r = 32 w + l in registers T[64]:
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
// All 256 threads of the CTA enter and leave together.  Every read of data
// that other CTAs write is an L2 load (ld.global.cg), so the same code runs
// inside the fused factorisation.  sraw: two 64 x 68 float buffers in shared
// memory.
template <bool SPLIT>
__device__ __forceinline__ void gj_diag_block(int64_t n, const float *M, int64_t lda,
                                              int64_t k0, float *Dinv, int32_t *info,
                                              const float *Dprev, float *stage, float *sraw,
                                              GjElimSmem *E = nullptr, int32_t *status = nullptr)
{
    constexpr int NB = GJ_NB, LDT = NB + 4;
    // two 64 x 68 buffers: B0 = Dprev^T, then R_PK, then the block D (rows of
    // 65 floats), then the output; B1 = M[P,K], then M[K,P]^T
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
    if (SPLIT && tid == 0)
        for (int c = 0; c < NB; ++c) tcp::mbar_init(&E->bar[c], 32);  // ordered by the barriers below
    {
        // thread owns the 4 x 4 tile rows r0..r0+3, columns j0..j0+3
        const int r0 = 4 * (tid >> 4), j0 = 4 * (tid & 15);
        float L[4][4];
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            const int j = j0 + jj;
            if (r0 + 3 < kb && j < kb) {
                const float4 v = __ldcg(reinterpret_cast<const float4 *>(M + (k0 + r0) + (k0 + j) * lda));
                L[0][jj] = v.x;
                L[1][jj] = v.y;
                L[2][jj] = v.z;
                L[3][jj] = v.w;
            } else {
#pragma unroll
                for (int ii = 0; ii < 4; ++ii) {
                    const int r = r0 + ii;
                    L[ii][jj] = (r < kb && j < kb) ? __ldcg(M + (k0 + r) + (k0 + j) * lda)
                                                   : (r == j ? 1.0f : 0.0f);
                }
            }
        }
        if (Dprev) {
            float dv[16], mv[16], cv[16];  // all loads in flight before the first shared store
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int idx = tid + 256 * q, a = idx & 63, b = idx >> 6;
                mv[q] = b < kb ? __ldcg(M + (kp + a) + (k0 + b) * lda) : 0.0f;  // M[P+a][K+b]
                cv[q] = a < kb ? __ldcg(M + (k0 + a) + (kp + b) * lda) : 0.0f;  // M[K+a][P+b]
            }
            // Launched as a programmatic dependent of the previous diagonal
            // inverse, this kernel may start while that one still runs: the
            // tiles of M above are final already (the previous inverse writes
            // only D^{-1}, the staged tiles and info), Dprev is not until the
            // previous grid has completed and flushed.  Then the next inverse
            // may launch.  (Both instructions do nothing in a kernel launched
            // otherwise.)
            asm volatile("griddepcontrol.wait;" ::: "memory");
            asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int idx = tid + 256 * q, a = idx & 63, b = idx >> 6;
                dv[q] = __ldcg(Dprev + b * NB + a);  // Dprev[b][a]
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
        if (Dprev && wq != 4 && wq != 5) {
            const int u = wq < 4 ? tid - 64 : tid - 128, i0 = 4 * (u & 15), c0 = 8 * (u >> 4);
            float acc[4][8] = {};
#pragma unroll 4
            for (int t = 0; t < NB; ++t) {
                const float4 a4 = *reinterpret_cast<const float4 *>(&B1[t][i0]);
                const float4 d0 = __ldcg(reinterpret_cast<const float4 *>(Dprev + t * NB + c0));
                const float4 d1 = __ldcg(reinterpret_cast<const float4 *>(Dprev + t * NB + c0 + 4));
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
        }
    } else if (SPLIT) {
        gj_elim_split(sm0, *E, k0, info, status);
    } else {
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
        // stores are coalesced and shared by all 256 threads
#pragma unroll
        for (int d = 0; d < NB; ++d) sm0[mypos][pivrow[d]] = T[d] * scale;
    }
    __syncthreads();
    for (int i = tid; i < NB * NB; i += 256) Dinv[i] = sm0[i >> 6][i & 63];
    __syncthreads();  // the caller may reuse sraw
}

// The separate-kernel diagonal inverse, with the pipelined elimination (its
// slots in the dynamic shared memory, which the launch makes large enough to
// keep the SM to itself).
__global__ void __launch_bounds__(256, 1)
    k_gj_diag(int64_t n, const float *M, int64_t lda, int64_t k0, float *Dinv, int32_t *info,
              const float *Dprev, float *stage, int32_t *status)
{
    __shared__ __align__(16) float sraw[2 * GJ_NB * (GJ_NB + 4)];
    extern __shared__ __align__(16) uint8_t gj_diag_dyn[];
    gj_diag_block<true>(n, M, lda, k0, Dinv, info, Dprev, stage, sraw,
                        reinterpret_cast<GjElimSmem *>(gj_diag_dyn), status);
}

// Prep of step K.  grid.y = 0: R[:, j] = D^{-1} M[K, j] for one 64-column tile
// (R[:,K] = 0), stored transposed Rt[j * 64 + r].  grid.y = 1: the block column
// C = M[:, K] for one 64-row tile, stored row-major Cb[i * 64 + c] (rows of K
// zero).  Both through shared memory so every global access is coalesced.
// With `stage` given (K > 0), the tiles M[K-1,K] and M[K,K-1] as left by step
// K-1 are read from there (the diagonal inverse of this step wrote them; the
// finish of step K-1 skips them in M).
// One tile (t0, y) of the prep; sbuf: two 64 x 68 float buffers in shared
// memory.  Ends with every thread past its last shared-memory access.  With
// Rt_lo / Cb_lo given, the panels are stored split for the tensor cores:
// Rt = TF32 rounding of R (cvt.rna) and Rt_lo = the rest, which is exact, so
// that Rt + Rt_lo = R (the same for C).
__device__ __forceinline__ void gj_prep_tile(int64_t n, const float *M, int64_t lda, int64_t k0,
                                             const float *Dinv, float *Rt, float *Cb,
                                             const float *stage, int64_t t0, int y, float *sbuf,
                                             float *Rt_lo = nullptr, float *Cb_lo = nullptr)
{
    constexpr int NB = GJ_NB;
    float(*Ds)[NB + 4] = reinterpret_cast<float(*)[NB + 4]>(sbuf);
    float(*Ms)[NB + 4] = reinterpret_cast<float(*)[NB + 4]>(sbuf + NB * (NB + 4));
    const int tid = threadIdx.x;
    const int kb = (int)min((int64_t)NB, n - k0);
    const int nt = (int)min((int64_t)NB, n - t0);
    const bool staged = stage && t0 == k0 - NB;
    if (y == 1) {
        const bool in_k = (t0 == k0);
        // M[t0 + i][K + c], or column-major 64 x 64 in stage for the tile above
        const float *src = staged ? stage : M + t0 + k0 * lda;
        const int64_t ld = staged ? NB : lda;
        float v[16];  // all loads in flight before the first shared store
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int idx = tid + 256 * q, i = idx & 63, c = idx >> 6;
            v[q] = (i < nt && c < kb && !in_k) ? __ldcg(src + i + c * ld) : 0.0f;
        }
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int idx = tid + 256 * q;
            Ms[idx & 63][idx >> 6] = v[q];
        }
        __syncthreads();
        for (int idx = tid; idx < NB * NB; idx += 256) {
            const int c = idx & 63, i = idx >> 6;
            if (i < nt) {
                if (Cb_lo) {
                    float h, l;
                    tcp::split_tf32(Ms[i][c], h, l);
                    Cb[(t0 + i) * NB + c] = h;
                    Cb_lo[(t0 + i) * NB + c] = l;
                } else {
                    Cb[(t0 + i) * NB + c] = Ms[i][c];
                }
            }
        }
        __syncthreads();
        return;
    }
    const bool tile_is_k = (t0 == k0);
    // D^{-1} transposed and the block row, rows of 68 floats (16-byte loads)
    float(*DT)[NB + 4] = Ds;
    float(*MK)[NB + 4] = Ms;
    {
        // M[K + a][t0 + b], or column-major 64 x 64 in stage for the tile left of K
        const float *src = staged ? stage + NB * NB : M + k0 + t0 * lda;
        const int64_t ld = staged ? NB : lda;
        float dv[16], mv[16];  // all loads in flight before the first shared store
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int idx = tid + 256 * q, a = idx & 63, b = idx >> 6;
            dv[q] = __ldcg(Dinv + b * NB + a);                              // D^{-1}[b][a]
            mv[q] = (a < kb && b < nt) ? __ldcg(src + a + b * ld) : 0.0f;  // M[K+a][t0+b]
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
            for (int yy = 0; yy < 4; ++yy) acc[x][yy] = fmaf(a[x], b[yy], acc[x][yy]);
    }
    __syncthreads();
#pragma unroll
    for (int yy = 0; yy < 4; ++yy) {
        const int c = c0 + yy;
        if (c >= nt) continue;
        float v[4];
#pragma unroll
        for (int x = 0; x < 4; ++x) v[x] = (tile_is_k || r0 + x >= kb) ? 0.0f : acc[x][yy];
        if (Rt_lo) {
            float h[4], l[4];
#pragma unroll
            for (int x = 0; x < 4; ++x) tcp::split_tf32(v[x], h[x], l[x]);
            *reinterpret_cast<float4 *>(&Rt[(t0 + c) * NB + r0]) = make_float4(h[0], h[1], h[2], h[3]);
            *reinterpret_cast<float4 *>(&Rt_lo[(t0 + c) * NB + r0]) =
                make_float4(l[0], l[1], l[2], l[3]);
        } else {
            *reinterpret_cast<float4 *>(&Rt[(t0 + c) * NB + r0]) = make_float4(v[0], v[1], v[2], v[3]);
        }
    }
}

// The R part of a prep tile for one 16-column slice (columns t0 + 16 s ..
// t0 + 16 s + 15): four CTAs share a tile's product.  Each entry gets the same
// FMA sequence as in gj_prep_tile.
// It also finishes block row K for these columns (M[K, :] <- R, M[K,K] <-
// D^{-1}), except for the tile at skip_t0 (the next block's, which its
// diagonal inverse stages): the finish then only does the block column.
__device__ __forceinline__ void gj_prep_slice(int64_t n, float *M, int64_t lda, int64_t k0,
                                              const float *Dinv, float *Rt, const float *stage,
                                              int64_t t0, int s, float *sbuf, float *Rt_lo,
                                              int64_t skip_t0)
{
    constexpr int NB = GJ_NB, SW = 16;
    float(*DT)[NB + 4] = reinterpret_cast<float(*)[NB + 4]>(sbuf);
    float(*MK)[NB + 4] = reinterpret_cast<float(*)[NB + 4]>(sbuf + NB * (NB + 4));
    const int tid = threadIdx.x;
    const int kb = (int)min((int64_t)NB, n - k0);
    const int nt = (int)min((int64_t)NB, n - t0);
    const bool staged = stage && t0 == k0 - NB;
    const bool tile_is_k = (t0 == k0);
    {
        const float *src = staged ? stage + NB * NB : M + k0 + t0 * lda;
        const int64_t ld = staged ? NB : lda;
        float dv[16], mv[4];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int idx = tid + 256 * q, a = idx & 63, b = idx >> 6;
            dv[q] = __ldcg(Dinv + b * NB + a);  // D^{-1}[b][a]
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int idx = tid + 256 * q, a = idx & 63, b = SW * s + (idx >> 6);
            mv[q] = (a < kb && b < nt) ? __ldcg(src + a + b * ld) : 0.0f;  // M[K+a][t0+b]
        }
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int idx = tid + 256 * q;
            DT[idx & 63][idx >> 6] = dv[q];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int idx = tid + 256 * q;
            MK[idx & 63][idx >> 6] = mv[q];
        }
    }
    __syncthreads();
    // thread computes R[r0 + x][t0 + 16 s + c] for x = 0..3
    const int r0 = 4 * (tid & 15), c = tid >> 4;
    float acc[4] = {};
#pragma unroll 8
    for (int t = 0; t < NB; ++t) {
        const float4 a4 = *reinterpret_cast<const float4 *>(&DT[t][r0]);
        const float b = MK[t][c];
        acc[0] = fmaf(a4.x, b, acc[0]);
        acc[1] = fmaf(a4.y, b, acc[1]);
        acc[2] = fmaf(a4.z, b, acc[2]);
        acc[3] = fmaf(a4.w, b, acc[3]);
    }
    const int col = SW * s + c;
    if (col >= nt) return;
    float v[4];
#pragma unroll
    for (int x = 0; x < 4; ++x) v[x] = (tile_is_k || r0 + x >= kb) ? 0.0f : acc[x];
    if (t0 != skip_t0) {
        // block row K of M, column t0 + col: R, or D^{-1} in the diagonal tile
        float mo[4];
#pragma unroll
        for (int x = 0; x < 4; ++x)
            mo[x] = tile_is_k ? (col < kb ? __ldcg(Dinv + (r0 + x) * NB + col) : 0.0f) : v[x];
        float *dst = M + (k0 + r0) + (t0 + col) * lda;
        if (r0 + 3 < kb && !(tile_is_k && col >= kb)) {
            *reinterpret_cast<float4 *>(dst) = make_float4(mo[0], mo[1], mo[2], mo[3]);
        } else {
#pragma unroll
            for (int x = 0; x < 4; ++x)
                if (r0 + x < kb && !(tile_is_k && col >= kb)) dst[x] = mo[x];
        }
    }
    if (Rt_lo) {
        float h[4], l[4];
#pragma unroll
        for (int x = 0; x < 4; ++x) tcp::split_tf32(v[x], h[x], l[x]);
        *reinterpret_cast<float4 *>(&Rt[(t0 + col) * NB + r0]) = make_float4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<float4 *>(&Rt_lo[(t0 + col) * NB + r0]) = make_float4(l[0], l[1], l[2], l[3]);
    } else {
        *reinterpret_cast<float4 *>(&Rt[(t0 + col) * NB + r0]) = make_float4(v[0], v[1], v[2], v[3]);
    }
}

// grid.y = 0..3: the R panel of tile t0, one 16-column slice each; grid.y = 4:
// the C panel of tile t0.
__global__ void __launch_bounds__(256)
    k_gj_prep(int64_t n, float *M, int64_t lda, int64_t k0, const float *Dinv, float *Rt,
              float *Cb, const float *stage, float *Rt_lo, float *Cb_lo, int64_t skip_t0)
{
    __shared__ __align__(16) float sbuf[2 * GJ_NB * (GJ_NB + 4)];
    const int64_t t0 = (int64_t)blockIdx.x * GJ_NB;
    if (t0 >= n) return;
    if (blockIdx.y == 4)
        gj_prep_tile(n, M, lda, k0, Dinv, Rt, Cb, stage, t0, 1, sbuf, Rt_lo, Cb_lo);
    else
        gj_prep_slice(n, M, lda, k0, Dinv, Rt, stage, t0, (int)blockIdx.y, sbuf, Rt_lo, skip_t0);
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

// hi + lo of a split panel entry: the value itself (lo == 0 keeps the sign of a zero)
__device__ __forceinline__ float gj_join(const float *hi, const float *lo, int64_t i)
{
    const float h = __ldcg(hi + i);
    if (!lo) return h;
    const float l = __ldcg(lo + i);
    return l == 0.0f ? h : h + l;
}

// One tile (t0, y) of the finish; sbuf as for the prep; Rt_lo / Cb_lo as
// written by the prep.
__device__ __forceinline__ void gj_finish_tile(int64_t n, float *M, int64_t lda, int64_t k0,
                                               const float *Dinv, const float *Rt,
                                               const float *Cb, int64_t t0, int y, float *sbuf,
                                               const float *Rt_lo = nullptr,
                                               const float *Cb_lo = nullptr)
{
    constexpr int NB = GJ_NB;
    const int tid = threadIdx.x;
    const int kb = (int)min((int64_t)NB, n - k0);
    const int nt = (int)min((int64_t)NB, n - t0);
    if (y == 0) {
        const bool tile_is_k = (t0 == k0);
        float v[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int idx = tid + 256 * q, rr = idx & 63, c = idx >> 6;
            const bool in = rr < kb && c < nt;
            v[q] = !in ? 0.0f
                       : (tile_is_k ? __ldcg(Dinv + rr * NB + c) : gj_join(Rt, Rt_lo, (t0 + c) * NB + rr));
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
    float(*CT)[NB + 4] = reinterpret_cast<float(*)[NB + 4]>(sbuf + NB * (NB + 4));
    float(*DD)[NB + 4] = reinterpret_cast<float(*)[NB + 4]>(sbuf);
    {
        float dv[16], cv[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int idx = tid + 256 * q, a = idx & 63, b = idx >> 6;
            dv[q] = __ldcg(Dinv + b * NB + a);                          // D^{-1}[b][a]
            cv[q] = b < nt ? gj_join(Cb, Cb_lo, (t0 + b) * NB + a) : 0.0f;  // C[t0+b][a]
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
            for (int yy = 0; yy < 4; ++yy) acc[x][yy] = fmaf(a[x], b[yy], acc[x][yy]);
    }
    __syncthreads();
#pragma unroll
    for (int yy = 0; yy < 4; ++yy) {
        const int c = c0 + yy;
        if (c >= kb) continue;
        float *col = M + t0 + (k0 + c) * lda;
        if (i0 + 3 < nt) {
            *reinterpret_cast<float4 *>(col + i0) =
                make_float4(-acc[0][yy], -acc[1][yy], -acc[2][yy], -acc[3][yy]);
        } else {
#pragma unroll
            for (int x = 0; x < 4; ++x)
                if (i0 + x < nt) col[i0 + x] = -acc[x][yy];
        }
    }
}

// Block column K <- -C D^{-1}, in 64-row tiles (the prep has finished block
// row K and the diagonal tile).  The tile at skip_t0 (the next block, whose
// diagonal inverse computes it and leaves it for the next prep) is not written.
__global__ void __launch_bounds__(256)
    k_gj_finish(int64_t n, float *M, int64_t lda, int64_t k0, const float *Dinv, const float *Rt,
                const float *Cb, int64_t skip_t0, const float *Rt_lo, const float *Cb_lo)
{
    __shared__ __align__(16) float sbuf[2 * GJ_NB * (GJ_NB + 4)];
    const int64_t t0 = (int64_t)blockIdx.x * GJ_NB;
    if (t0 < n && t0 != skip_t0)
        gj_finish_tile(n, M, lda, k0, Dinv, Rt, Cb, t0, 1, sbuf, Rt_lo, Cb_lo);
}

// Tensor-core version of the update (tc_gemm.cu); false if not available for
// this precision.
bool launch_tc_gj_update(Ctx &c, float *M, int64_t lda, int64_t k0, const float *Cb,
                         const float *Rt, int prec, int64_t skip0, const float *Cb_lo,
                         const float *Rt_lo);

void launch_simt_rank64(Ctx &c, float *M, int64_t lda, int64_t n, const float *Cb, const float *Rt)
{
    const unsigned g = (unsigned)ceil_div(n, GJ_NB);
    // k0 = -GJ_NB: no tile is skipped
    k_gj_update_simt<<<dim3(g, g), 256, 0, c.stream>>>(n, M, lda, -GJ_NB, Cb, Rt, -GJ_NB);
    c.launches += 1;
}

// ---- the fused factorisation -----------------------------------------------
//
// The whole inversion as ONE cooperative launch, one CTA per SM: CTA 0 runs
// the chain of diagonal inverses (each with its lookahead), the other W CTAs
// ("workers") run prep + finish and the tensor-core update of every step.
// The hand-offs are counters in global memory instead of kernel boundaries
// and stream events:
//   flagD  = diagonal inverses done (CTA 0, after D^{-1} of block k: k + 1),
//   cntP   = workers done with the prep/finish of some step (W per step),
//   cntU   = workers done with the update of some step (W per step).
// Worker, step k:  wait flagD >= k + 1 and cntU >= k W;  prep + finish tiles;
//                  cntP += 1;  wait cntP >= (k + 1) W;  update tiles;  cntU += 1.
// CTA 0, block k:  wait cntU >= (k - 1) W (the update of step k - 2, the last
//                  one that touches the tiles its lookahead reads);  inverse;
//                  flagD = k + 1.
// The same device functions (the same arithmetic, in the same order) as the
// separate kernels below.  Every wait is bounded: a CTA that gives up sets
// ST_TIMEOUT, and every CTA leaves at its next wait once that bit is set.
struct GjFusedArgs {
    int64_t n, lda;
    float *M;
    float *dinv;   // 2 x 64 x 64
    float *rt, *cb;        // the panels, TF32-rounded part
    float *rt_lo, *cb_lo;  // the panels, the rest
    float *stage;  // 2 x 8192
    int32_t *info, *status;
    int32_t *sync;  // [0] flagD, [1] cntP, [2] cntU
    int nblk;
};

constexpr int GJF_THREADS = 256;
// shared memory of a worker: both 32-wide K blocks of a tile's panels (A, B,
// A lo, B lo: 128 KB) and the 128 x 128 tile of M (64 KB)
constexpr int GJF_PANEL_BYTES = 8 * tcp::TC_TILE_BYTES;
constexpr int GJF_MTILE_BYTES = 128 * 128 * 4;
constexpr int GJF_SMEM = GJF_PANEL_BYTES + GJF_MTILE_BYTES + 1024;

__device__ __forceinline__ int32_t gjf_ld_acquire(const int32_t *p)
{
    int32_t v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Thread 0: wait until sync[i] >= v (and sync[j] >= u when j >= 0).  Returns
// false (after setting ST_TIMEOUT) if that takes too long, or if another CTA
// already gave up.
__device__ bool gjf_wait(const GjFusedArgs &a, int i, int32_t v, int j, int32_t u)
{
    long long spins = 0;
    while (gjf_ld_acquire(a.sync + i) < v || (j >= 0 && gjf_ld_acquire(a.sync + j) < u)) {
        ++spins;
        if (spins > kSpinLimit || ((spins & 1023) == 0 && (*(volatile int32_t *)a.status & ST_TIMEOUT))) {
            atomicOr(a.status, ST_TIMEOUT);
            return false;
        }
        __nanosleep(32);
    }
    return true;
}

__device__ __forceinline__ void gjf_signal(int32_t *p)
{
    __threadfence();
    atomicAdd(p, 1);
}

// The update of one step on this worker's tiles (t = first, first + stride,
// ...; 128 x 128 tiles of M, column tile t / rtiles), split TF32 on the
// tensor cores from panels the prep stored already split (hi, lo), pipelined
// over the tiles:
//   thread 0 issues the TMA loads of a tile's panels (hi and lo of both
//   32-wide K blocks) and of its tile of M; once both K blocks are in it
//   issues the 12 MMAs of each; once they are done the next tile's panels are
//   requested; the epilogue subtracts the accumulator (TMEM) from the tile of
//   M (shared memory) and stores the result with coalesced global stores
//   (entries the step must not change are not stored); once every thread has
//   read the tile of M, the next one is requested.
// ph: this CTA's barrier parity, advanced per tile.  Returns false on timeout
// (after bounded waits for its own copies in flight).
__device__ bool gjf_update_step(const CUtensorMap *tmAh, const CUtensorMap *tmAl,
                                const CUtensorMap *tmBh, const CUtensorMap *tmBl,
                                const CUtensorMap *tmM, uint8_t *base, uint64_t *bars,
                                uint32_t tmem, uint32_t &ph, int64_t n, float *M, int64_t lda,
                                int64_t skip0, int64_t kblk, int first, int stride,
                                int32_t *status, int *s_ok)
{
    using namespace tcp;
    uint64_t *bar_pan = bars, *bar_m = bars + 2, *bar_mma = bars + 3;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rtiles = (int)ceil_div(n, TC_BM), total = rtiles * (int)ceil_div(n, TC_BN);
    float *sA[2], *sB[2], *sAl[2], *sBl[2];
#pragma unroll
    for (int kb = 0; kb < 2; ++kb) {
        uint8_t *p = base + (size_t)kb * 4 * TC_TILE_BYTES;
        sA[kb] = reinterpret_cast<float *>(p);
        sB[kb] = reinterpret_cast<float *>(p + TC_TILE_BYTES);
        sAl[kb] = reinterpret_cast<float *>(p + 2 * TC_TILE_BYTES);
        sBl[kb] = reinterpret_cast<float *>(p + 3 * TC_TILE_BYTES);
    }
    const float *Mt = reinterpret_cast<const float *>(base + GJF_PANEL_BYTES);  // [128 cols][128 rows]
    auto load_panels = [&](int t) {
        const int row0 = (t % rtiles) * TC_BM, col0 = (t / rtiles) * TC_BN;
#pragma unroll
        for (int kb = 0; kb < 2; ++kb) {
            mbar_expect_tx(&bar_pan[kb], 4 * TC_TILE_BYTES);
            tma_load_2d(sA[kb], tmAh, kb * TC_KB, row0, &bar_pan[kb]);
            tma_load_2d(sAl[kb], tmAl, kb * TC_KB, row0, &bar_pan[kb]);
            tma_load_2d(sB[kb], tmBh, kb * TC_KB, col0, &bar_pan[kb]);
            tma_load_2d(sBl[kb], tmBl, kb * TC_KB, col0, &bar_pan[kb]);
        }
    };
    auto load_m = [&](int t) {
        mbar_expect_tx(bar_m, GJF_MTILE_BYTES);
        tma_load_2d(const_cast<float *>(Mt), tmM, (t % rtiles) * TC_BM, (t / rtiles) * TC_BN, bar_m);
    };
    if (first >= total) return true;
    if (threadIdx.x == 0) {
        load_panels(first);
        load_m(first);
    }
    constexpr uint32_t idesc = idesc_tf32(TC_BM, TC_BN);
    bool ok = true;
    for (int t = first; t < total; t += stride) {
        const int tn = t + stride;
        const int64_t row0 = (int64_t)(t % rtiles) * TC_BM, col0 = (int64_t)(t / rtiles) * TC_BN;
        if (threadIdx.x == 0) {
#pragma unroll
            for (int kb = 0; kb < 2; ++kb) {
                if (!mbar_wait(&bar_pan[kb], ph)) {
                    atomicOr(status, ST_TIMEOUT);
                    *s_ok = 0;
                    break;
                }
                tc_fence_after();
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const uint32_t kofs = (uint32_t)kk * 32u;
                    const uint64_t ah = desc_sw128_kmajor(smem_u32(sA[kb]) + kofs);
                    const uint64_t bh = desc_sw128_kmajor(smem_u32(sB[kb]) + kofs);
                    const uint64_t al = desc_sw128_kmajor(smem_u32(sAl[kb]) + kofs);
                    const uint64_t bl = desc_sw128_kmajor(smem_u32(sBl[kb]) + kofs);
                    mma_tf32(tmem, al, bh, idesc, (kb > 0 || kk > 0) ? 1u : 0u);
                    mma_tf32(tmem, ah, bl, idesc, 1u);
                    mma_tf32(tmem, ah, bh, idesc, 1u);
                }
            }
            if (*s_ok) {
                mma_commit(bar_mma);
                if (!mbar_wait(bar_mma, ph)) {
                    atomicOr(status, ST_TIMEOUT);
                    *s_ok = 0;
                } else if (tn < total) {
                    load_panels(tn);  // the panels' shared memory is free
                }
            }
        }
        __syncthreads();
        if (!*s_ok) {
            ok = false;
            break;
        }
        if (!mbar_wait(bar_m, ph)) {
            atomicOr(status, ST_TIMEOUT);
            *s_ok = 0;
        }
        __syncthreads();
        if (!*s_ok) {
            ok = false;
            break;
        }
        tc_fence_after();
        {
            const int rl = (warp & 3) * 32 + lane;
            const int64_t row = row0 + rl;
            const int half = warp >> 2;
            const bool row_skip = row >= skip0 && row < skip0 + 64;
            // block row and column kblk were finished by this step's finish
            const bool row_k = row >= kblk && row < kblk + 64;
            const bool row_ok = row < n && !row_k;
            // the accumulator's 64 columns of this thread's row, one wait for all four loads
            uint32_t acc[4][16];
            const uint32_t taddr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(half * 64);
#pragma unroll
            for (int chunk = 0; chunk < 4; ++chunk)
                tmem_ld_16cols_async(taddr + (uint32_t)(chunk * 16), acc[chunk]);
            tmem_wait_ld();
#pragma unroll
            for (int chunk = 0; chunk < 4; ++chunk) {
                const int cl0 = half * 64 + chunk * 16;
                const int64_t cbeg = col0 + cl0;
                const uint32_t *v = acc[chunk];
                if (!row_ok || (cbeg >= kblk && cbeg < kblk + 64)) continue;
                const bool dskip = row_skip && cbeg >= skip0 && cbeg < skip0 + 64;
                if (dskip) continue;  // the 64-aligned diagonal block of the lookahead
                float *p = M + row + cbeg * lda;
                const int64_t ncol = n - cbeg;
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    if (j < ncol) p[j * lda] = Mt[(cl0 + j) * TC_BM + rl] - __uint_as_float(v[j]);
            }
        }
        tc_fence_before();
        __syncthreads();
        // every thread has read the tile of M and its accumulator columns
        if (threadIdx.x == 0 && tn < total) load_m(tn);
        ph ^= 1u;
    }
    if (!ok && threadIdx.x == 0) {
        // bounded waits for this CTA's copies and MMAs still in flight
        mbar_wait(&bar_pan[0], ph);
        mbar_wait(&bar_pan[1], ph);
        mbar_wait(bar_m, ph);
        mbar_wait(bar_mma, ph);
    }
    // the stores of M are read by TMA (the async proxy) in the next step
    asm volatile("fence.proxy.async.global;" ::: "memory");
    __syncthreads();
    return ok;
}

__global__ void __launch_bounds__(GJF_THREADS, 2)
    k_gj_fused(const __grid_constant__ CUtensorMap tmAh, const __grid_constant__ CUtensorMap tmAl,
               const __grid_constant__ CUtensorMap tmBh, const __grid_constant__ CUtensorMap tmBl,
               const __grid_constant__ CUtensorMap tmM, GjFusedArgs a)
{
    using namespace tcp;
    extern __shared__ uint8_t gjf_smem[];
    __shared__ uint64_t bars[4];  // panels K block 0, 1; tile of M; MMAs
    __shared__ uint32_t tmem_slot;
    __shared__ int s_ok;
    uint8_t *base = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(gjf_smem) + 1023) & ~static_cast<uintptr_t>(1023));
    float *sbuf = reinterpret_cast<float *>(base);
    const int64_t n = a.n, lda = a.lda;
    const int nblk = a.nblk;
    const int W = (int)gridDim.x - 1;
    constexpr int NB = GJ_NB;
    if (threadIdx.x == 0) s_ok = 1;
    __syncthreads();
    if (blockIdx.x == 0) {
        // the chain of diagonal inverses
        for (int k = 0; k < nblk; ++k) {
            if (threadIdx.x == 0 && k >= 2 && !gjf_wait(a, 2, (k - 1) * W, -1, 0)) s_ok = 0;
            __syncthreads();
            if (!s_ok) return;
            const int b = k & 1;
            gj_diag_block<false>(n, a.M, lda, (int64_t)k * NB, a.dinv + b * NB * NB, a.info,
                          k ? a.dinv + (b ^ 1) * NB * NB : nullptr,
                          k ? a.stage + b * 2 * NB * NB : nullptr, sbuf);
            if (threadIdx.x == 0) {
                __threadfence();
                asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(a.sync), "r"(k + 1)
                             : "memory");
            }
        }
        return;
    }
    // workers
    const int wid = (int)blockIdx.x - 1;
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        for (int i = 0; i < 4; ++i) mbar_init(&bars[i], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_slot)),
                     "r"(TC_BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    uint32_t ph = 0;
    for (int k = 0; k < nblk; ++k) {
        const int64_t k0 = (int64_t)k * NB, k1 = k0 + NB;
        const bool next = k1 < n;
        const int b = k & 1;
        const float *dk = a.dinv + b * NB * NB;
        if (threadIdx.x == 0 && !gjf_wait(a, 0, k + 1, 2, k * W)) s_ok = 0;
        __syncthreads();
        if (!s_ok) break;
        // prep (and, from the same CTA's panel tile, finish) of step k
        for (int it = wid; it < 2 * nblk; it += W) {
            const int y = it & 1;
            const int64_t t0 = (int64_t)(it >> 1) * NB;
            gj_prep_tile(n, a.M, lda, k0, dk, a.rt, a.cb, k ? a.stage + b * 2 * NB * NB : nullptr,
                         t0, y, sbuf, a.rt_lo, a.cb_lo);
            __syncthreads();
            if (!(next && t0 == k1))
                gj_finish_tile(n, a.M, lda, k0, dk, a.rt, a.cb, t0, y, sbuf, a.rt_lo, a.cb_lo);
            __syncthreads();
        }
        // the panels are read by TMA (the async proxy) in the update, and TMA
        // overwrites the shared memory the prep and finish used
        asm volatile("fence.proxy.async;" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0) {
            gjf_signal(a.sync + 1);
            if (!gjf_wait(a, 1, (k + 1) * W, -1, 0)) s_ok = 0;
            asm volatile("fence.proxy.async.global;" ::: "memory");
        }
        __syncthreads();
        if (!s_ok) break;
        const int64_t skip0 = next ? k1 : -NB;
        if (!gjf_update_step(&tmAh, &tmAl, &tmBh, &tmBl, &tmM, base, bars, tmem, ph, n, a.M, lda,
                             skip0, k0, wid, W, a.status, &s_ok))
            break;
        __syncthreads();
        if (threadIdx.x == 0) gjf_signal(a.sync + 2);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_BN)
                     : "memory");
}

// The fused inversion, if this device and precision allow it (split TF32,
// tensor memory, cooperative launch with one CTA per SM); false otherwise.
bool run_gj_fused(Ctx &c, float *M, int64_t lda)
{
    if (!c.gj_fused || !tc_available()) return false;
    static int attr_state = 0;  // 0 untried, 1 ok, -1 unavailable
    if (attr_state == 0) {
        attr_state = cudaFuncSetAttribute(k_gj_fused, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          GJF_SMEM) == cudaSuccess
                         ? 1
                         : -1;
        cudaGetLastError();
    }
    if (attr_state < 0) return false;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gj_fused, GJF_THREADS, GJF_SMEM) !=
            cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        return false;
    }
    const int G = c.num_sms;
    if (G < 2) return false;
    // the first of the separate-kernel path's panel buffers, split as there
    float *rt_lo = c.d_gj_rt + (size_t)2 * GJ_NB * c.lda, *cb_lo = c.d_gj_cb + (size_t)2 * GJ_NB * c.lda;
    CUtensorMap tmAh, tmAl, tmBh, tmBl, tmM;
    if (!make_panel_map(&tmAh, c.d_gj_cb, c.n) || !make_panel_map(&tmAl, cb_lo, c.n) ||
        !make_panel_map(&tmBh, c.d_gj_rt, c.n) || !make_panel_map(&tmBl, rt_lo, c.n) ||
        !make_matrix_map(&tmM, M, c.n, lda))
        return false;
    GjFusedArgs a{};
    a.n = c.n;
    a.lda = lda;
    a.M = M;
    a.dinv = c.d_gj_dinv;
    a.rt = c.d_gj_rt;
    a.cb = c.d_gj_cb;
    a.rt_lo = rt_lo;
    a.cb_lo = cb_lo;
    a.stage = c.d_gj_stage;
    a.info = c.d_info;
    a.status = c.d_status;
    a.sync = c.d_gj_sync;
    a.nblk = (int)ceil_div(c.n, GJ_NB);
    cudaMemsetAsync(c.d_info, 0, sizeof(int32_t), c.stream);
    cudaMemsetAsync(c.d_gj_sync, 0, 4 * sizeof(int32_t), c.stream);
    void *args[] = {&tmAh, &tmAl, &tmBh, &tmBl, &tmM, &a};
    c.tbeg(PH_LU_UPDATE);
    const cudaError_t e =
        cudaLaunchCooperativeKernel((void *)k_gj_fused, G, GJF_THREADS, args, GJF_SMEM, c.stream);
    c.tend(PH_LU_UPDATE);
    c.launches += 1;
    return e == cudaSuccess;
}

// One inversion.  Streams: main (S), lookahead (S2), finish (S4).  Step k
// (block K, next block K+1):
//   S2: (waits the update of step k-1 and the finish of step k-1) the
//       diagonal inverse of K+1 with its lookahead from D_K^{-1} and the
//       un-finished block row and column K; it also leaves the two finished
//       tiles M[K,K+1], M[K+1,K] in stage[k+1 mod 2]              -> ev_diag
//   S : prep_k: the panels R = D_K^{-1} M[K,:], C = M[:,K]; block row K
//       <- R and M[K,K] <- D_K^{-1} (but the staged tile)     -> ev_fin_ready
//   S4: finish_k: block column K <- -C D_K^{-1} (but the staged
//       tile)                                                 -> ev_fin[k mod 2]
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
static_assert(sizeof(GjElimSmem) <= GJ_DIAG_EXCL_SMEM, "the elimination's slots fit");

size_t gj_diag_smem() { return (sizeof(GjElimSmem) + 1023) / 1024 * 1024; }

void gj_diag_prepare()
{
    static bool done = false;
    if (!done) {
        cudaFuncSetAttribute(k_gj_diag, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             GJ_DIAG_EXCL_SMEM);
        done = true;
    }
}

// D^{-1} of the diagonal block at (k0, k0) alone (no lookahead), for the
// panel elimination of gj2.cu.
void k_gj_diag_launch(Ctx &c, int64_t n, const float *M, int64_t lda, int64_t k0, float *Dinv,
                      size_t smem, cudaStream_t s)
{
    k_gj_diag<<<1, 256, smem, s ? s : c.stream>>>(n, M, lda, k0, Dinv, c.d_info, nullptr, nullptr,
                                                 c.d_status);
}

int run_gj_fp32(Ctx &c, float *M, int64_t lda, int prec)
{
    c.last_factor_two_level = false;
    if (prec == NRS_TF32 && run_gj_fused(c, M, lda)) return 0;
    // large systems: the two-level elimination whose updates are rank-256 products
    const bool two = !c.gj_force_one_level &&
                     (c.gj_schedule >= 3 || (c.gj_schedule == 0 && c.n >= GJ2_MIN_N));
    c.last_factor_two_level = prec == NRS_TF32 && two && gj2_supported(c) && c.d_gj2;
    // the update's pieces: TF32 (schedule 3), scaled FP16 (schedule 4 and auto)
    if (c.last_factor_two_level) return run_gj2_fp32(c, M, lda, c.gj_schedule != 3);
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
    // with the tensor-core update the prep stores the panels split into TF32
    // hi (rt, cb) and lo (these) for it, and the finish joins them again
    const bool split = (prec == NRS_TF32) && tc_available();
    float *rt_lo[2] = {c.d_gj_rt + (size_t)2 * GJ_NB * c.lda, c.d_gj_rt + (size_t)3 * GJ_NB * c.lda};
    float *cb_lo[2] = {c.d_gj_cb + (size_t)2 * GJ_NB * c.lda, c.d_gj_cb + (size_t)3 * GJ_NB * c.lda};
    float *stg[2] = {c.d_gj_stage, c.d_gj_stage + 2 * GJ_NB * GJ_NB};
    c.tbeg(PH_LU_DIAG);
    k_gj_diag<<<1, 256, GJ_DIAG_EXCL_SMEM, c.stream>>>(n, M, lda, 0, dinv[0], c.d_info, nullptr, nullptr,
                                                       c.d_status);
    c.tend(PH_LU_DIAG);
    cudaEventRecord(c.ev_upd, c.stream);
    c.launches += 1;
    int kstep = 0;
    bool failed = false;
    for (int64_t k0 = 0; k0 < n; k0 += GJ_NB, ++kstep) {
        const int b = kstep & 1;
        const int64_t k1 = k0 + GJ_NB;
        const bool next = k1 < n;
        if (next) {
            cudaStreamWaitEvent(c.stream2, c.ev_upd, 0);
            if (kstep > 0) cudaStreamWaitEvent(c.stream2, c.ev_fin[b ^ 1], 0);
            c.tbeg(PH_LU_DIAG, c.stream2);
            // a programmatic dependent of the previous inverse on this stream
            // (it loads its tiles of M while that one finishes)
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(1);
            cfg.blockDim = dim3(256);
            cfg.dynamicSmemBytes = GJ_DIAG_EXCL_SMEM;
            cfg.stream = c.stream2;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
            attr[0].val.programmaticStreamSerializationAllowed = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            cudaLaunchKernelEx(&cfg, k_gj_diag, (int64_t)n, (const float *)M, (int64_t)lda, (int64_t)k1,
                               dinv[b ^ 1], c.d_info, (const float *)dinv[b], stg[b ^ 1], c.d_status);
            c.tend(PH_LU_DIAG, c.stream2);
            cudaEventRecord(c.ev_diag, c.stream2);
            c.launches += 1;
        }
        c.tbeg(PH_LU_PANEL);
        k_gj_prep<<<dim3(gcols, 5), 256, 0, c.stream>>>(n, M, lda, k0, dinv[b], rt[b], cb[b],
                                                        kstep > 0 ? stg[b] : nullptr,
                                                        split ? rt_lo[b] : nullptr,
                                                        split ? cb_lo[b] : nullptr,
                                                        next ? k1 : -1);
        c.tend(PH_LU_PANEL);
        cudaEventRecord(c.ev_fin_ready, c.stream);
        cudaStreamWaitEvent(c.stream4, c.ev_fin_ready, 0);
        c.tbeg(PH_LU_PANEL, c.stream4);
        k_gj_finish<<<dim3(gcols, 1), 256, 0, c.stream4>>>(n, M, lda, k0, dinv[b], rt[b], cb[b],
                                                           next ? k1 : -1,
                                                           split ? rt_lo[b] : nullptr,
                                                           split ? cb_lo[b] : nullptr);
        c.tend(PH_LU_PANEL, c.stream4);
        cudaEventRecord(c.ev_fin[b], c.stream4);
        if (kstep > 0) cudaStreamWaitEvent(c.stream, c.ev_fin[b ^ 1], 0);
        const int64_t skip0 = next ? k1 : -GJ_NB;
        c.tbeg(PH_LU_UPDATE);
        if (split) {
            // split panels have no CUDA-core fallback: a failed launch is an error
            if (!launch_tc_gj_update(c, M, lda, k0, cb[b], rt[b], prec, skip0, cb_lo[b], rt_lo[b]))
                failed = true;
        } else {
            k_gj_update_simt<<<dim3(gcols, gcols), 256, 0, c.stream>>>(n, M, lda, k0, cb[b], rt[b],
                                                                        skip0);
        }
        c.tend(PH_LU_UPDATE);
        cudaEventRecord(c.ev_upd, c.stream);
        if (next) cudaStreamWaitEvent(c.stream, c.ev_diag, 0);
        else cudaStreamWaitEvent(c.stream, c.ev_fin[b], 0);
        c.launches += 3;
    }
    return failed ? -1 : 0;
}

}  // namespace nrs
