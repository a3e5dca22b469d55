// tc_gemm.cu -- the rank-64 update M -= C R of the Gauss-Jordan inverse
// (gj.cu) on the 5th-generation tensor cores: tcgen05.mma kind::tf32 with
// FP32 accumulation in tensor memory, in split precision (3xTF32: every
// operand x = hi + lo, products hi*hi + hi*lo + lo*hi), which keeps FP32
// accuracy.  A single TF32 pass loses too much in the rigid-body Schur
// complement of the bordered system and can leave a useless preconditioner.
//
// One CTA (4 warps) per 128 x 128 output tile; for each of the two 32-wide
// K blocks:
//   * thread 0 loads the A tile (128 rows of Cb) and the B tile (128 rows of
//     Rt) with TMA (128-byte swizzle) onto an mbarrier,
//   * all threads split both tiles in shared memory into hi and lo parts,
//   * thread 0 issues 4 x 3 MMAs of 128 x 128 x 8 (A, B K-major in shared
//     memory, D in 128 TMEM columns) and commits them to an mbarrier;
// then every warp reads its 32 TMEM lanes (rows) with tcgen05.ld and
// subtracts them from M (column-major: a warp writes 32 consecutive rows).
// Every wait is bounded: a wait that runs out sets ST_TIMEOUT, the kernel
// skips the MMA / epilogue, waits once more (bounded) for its own copies and
// frees its tensor memory before returning.
#include <cuda.h>

#include "tc_prims.cuh"

namespace nrs {

namespace {

using namespace tcp;

// PRESPLIT: the panels arrive already split (hi in tmA/tmB, lo in tmAl/tmBl,
// as the prep stores them for this kernel), so the tiles go to the tensor
// cores as loaded; otherwise the FP32 panels are split here.
template <bool PRESPLIT>
__global__ void __launch_bounds__(128, 1)
    k_tc_gj_update(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const __grid_constant__ CUtensorMap tmAl, const __grid_constant__ CUtensorMap tmBl,
                   int64_t n, float *__restrict__ M, int64_t lda, int32_t *status, int64_t skip0,
                   int64_t kblk)
{
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t bar_load[2], bar_mma[2];
    __shared__ uint32_t tmem_slot;
    __shared__ int s_ok;
    uint8_t *base = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    // one 32-wide K block at a time: A (hi after the split), B (hi), A lo, B lo
    float *sA = reinterpret_cast<float *>(base);
    float *sB = reinterpret_cast<float *>(base + TC_TILE_BYTES);
    float *sAl = reinterpret_cast<float *>(base + 2 * TC_TILE_BYTES);
    float *sBl = reinterpret_cast<float *>(base + 3 * TC_TILE_BYTES);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t row0 = (int64_t)blockIdx.x * TC_BM, col0 = (int64_t)blockIdx.y * TC_BN;

    if (threadIdx.x == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(&bar_load[i], 1);
            mbar_init(&bar_mma[i], 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_ok = 1;
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
    constexpr uint32_t idesc = idesc_tf32(TC_BM, TC_BN);
    constexpr int kElems = TC_BM * TC_KB;  // floats per tile

    for (int kb = 0; kb < 2; ++kb) {
        if (threadIdx.x == 0) {
            // the previous K block's MMAs must have finished reading shared memory
            if (kb == 1 && s_ok && !mbar_wait(&bar_mma[0], 0)) {
                atomicOr(status, ST_TIMEOUT);
                s_ok = 0;
            }
            if (s_ok) {
                mbar_expect_tx(&bar_load[kb], (PRESPLIT ? 4 : 2) * TC_TILE_BYTES);
                tma_load_2d(sA, &tmA, kb * TC_KB, (int)row0, &bar_load[kb]);
                tma_load_2d(sB, &tmB, kb * TC_KB, (int)col0, &bar_load[kb]);
                if (PRESPLIT) {
                    tma_load_2d(sAl, &tmAl, kb * TC_KB, (int)row0, &bar_load[kb]);
                    tma_load_2d(sBl, &tmBl, kb * TC_KB, (int)col0, &bar_load[kb]);
                }
            }
        }
        __syncthreads();
        if (!s_ok) break;
        if (!mbar_wait(&bar_load[kb], 0)) {
            atomicOr(status, ST_TIMEOUT);
            s_ok = 0;
        }
        __syncthreads();
        if (!s_ok) break;
        if (!PRESPLIT) {
            // split both tiles in place (element-wise: the swizzled layout is kept)
            for (int i = threadIdx.x; i < kElems; i += 128) {
                float h, l;
                split_tf32(sA[i], h, l);
                sA[i] = h;
                sAl[i] = l;
                split_tf32(sB[i], h, l);
                sB[i] = h;
                sBl[i] = l;
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            tc_fence_after();
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const uint32_t kofs = (uint32_t)kk * 32u;
                const uint64_t ah = desc_sw128_kmajor(smem_u32(sA) + kofs);
                const uint64_t bh = desc_sw128_kmajor(smem_u32(sB) + kofs);
                const uint64_t al = desc_sw128_kmajor(smem_u32(sAl) + kofs);
                const uint64_t bl = desc_sw128_kmajor(smem_u32(sBl) + kofs);
                mma_tf32(tmem, al, bh, idesc, (kb > 0 || kk > 0) ? 1u : 0u);
                mma_tf32(tmem, ah, bl, idesc, 1u);
                mma_tf32(tmem, ah, bh, idesc, 1u);
            }
            mma_commit(&bar_mma[kb]);
        }
    }
    __syncthreads();
    bool ok = s_ok != 0;
    if (ok && !mbar_wait(&bar_mma[1], 0)) {
        atomicOr(status, ST_TIMEOUT);
        ok = false;
    }
    if (!ok && threadIdx.x == 0) {
        // bounded waits for whatever copies or MMAs may still be in flight
        mbar_wait(&bar_load[0], 0);
        mbar_wait(&bar_load[1], 0);
        mbar_wait(&bar_mma[0], 0);
        mbar_wait(&bar_mma[1], 0);
    }
    tc_fence_after();
    if (ok) {
        const int64_t row = row0 + warp * 32 + lane;
        // the 64 x 64 block at (skip0, skip0) is updated separately (lookahead)
        const bool row_skip = row >= skip0 && row < skip0 + 64;
        // block row and column kblk are written by the finish step, which may
        // run concurrently (C R is zero there): this kernel leaves them alone
        const bool row_k = row >= kblk && row < kblk + 64;
        // software-pipelined read-modify-write of this thread's row: the loads
        // of chunk c + 1 are issued before chunk c is subtracted and stored
        float cur[16], nxt[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) cur[j] = (row < n && col0 + j < n) ? M[row + (col0 + j) * lda] : 0.0f;
#pragma unroll 1
        for (int chunk = 0; chunk < TC_BN / 16; ++chunk) {
            const int64_t cbeg = col0 + chunk * 16;
            if (chunk + 1 < TC_BN / 16) {
                const int64_t nbeg = cbeg + 16;
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    nxt[j] = (row < n && nbeg + j < n) ? M[row + (nbeg + j) * lda] : 0.0f;
            }
            uint32_t v[16];
            tmem_ld_16cols(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(chunk * 16), v);
            if (row < n && !row_k && !(cbeg >= kblk && cbeg < kblk + 64)) {
                float *p = M + row + cbeg * lda;
                const int64_t ncol = n - cbeg;
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const bool skip = row_skip && cbeg + j >= skip0 && cbeg + j < skip0 + 64;
                    if (j < ncol && !skip) p[j * lda] = cur[j] - __uint_as_float(v[j]);
                }
            }
#pragma unroll
            for (int j = 0; j < 16; ++j) cur[j] = nxt[j];
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_BN)
                     : "memory");
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

struct TcMaps {
    const float *cb = nullptr, *rt = nullptr;
    int64_t rows = 0;
    CUtensorMap a, b;
    bool ok = false;
};

}  // namespace

// 2-D map over a row-major [rows][64] FP32 panel, boxes of 32 x 128 with
// 128-byte swizzle; rows >= `rows` read as zero.
bool make_panel_map(CUtensorMap *tm, const float *ptr, int64_t rows)
{
    EncodeTiledFn enc = encode_fn();
    if (!enc) return false;
    cuuint64_t dims[2] = {64, (cuuint64_t)rows};
    cuuint64_t strides[1] = {64 * sizeof(float)};
    cuuint32_t box[2] = {TC_KB, TC_BM};
    cuuint32_t estr[2] = {1, 1};
    return enc(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(ptr), dims, strides, box,
               estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool make_matrix_map(CUtensorMap *tm, const float *ptr, int64_t n, int64_t lda)
{
    EncodeTiledFn enc = encode_fn();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)n};
    cuuint64_t strides[1] = {(cuuint64_t)lda * sizeof(float)};
    cuuint32_t box[2] = {128, 128};
    cuuint32_t estr[2] = {1, 1};
    return enc(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(ptr), dims, strides, box,
               estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool tc_available()
{
    int dev = 0, major = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess)
        return false;
    return major >= 10 && encode_fn() != nullptr;
}

bool launch_tc_rank64(Ctx &c, float *M, int64_t lda, int64_t n, const float *Cb, const float *Rt,
                      int prec, int64_t skip0, int64_t kblk, const float *Cb_lo, const float *Rt_lo)
{
    if (prec != NRS_TF32) return false;
    const bool split = Cb_lo != nullptr;
    CUtensorMap a, b, al, bl;
    if (!make_panel_map(&a, Cb, n) || !make_panel_map(&b, Rt, n)) return false;
    if (split && (!make_panel_map(&al, Cb_lo, n) || !make_panel_map(&bl, Rt_lo, n))) return false;
    if (!split) {
        al = a;
        bl = b;
    }
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_tc_gj_update<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             TC_SMEM);
        cudaFuncSetAttribute(k_tc_gj_update<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             TC_SMEM);
        cudaFuncSetAttribute(k_tc_gj_update<false>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
        cudaFuncSetAttribute(k_tc_gj_update<true>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
        attr = true;
    }
    dim3 grid((unsigned)ceil_div(n, TC_BM), (unsigned)ceil_div(n, TC_BN));
    if (split)
        k_tc_gj_update<true><<<grid, 128, TC_SMEM, c.stream>>>(a, b, al, bl, n, M, lda, c.d_status,
                                                                skip0, kblk);
    else
        k_tc_gj_update<false><<<grid, 128, TC_SMEM, c.stream>>>(a, b, al, bl, n, M, lda, c.d_status,
                                                                 skip0, kblk);
    c.launches += 1;
    return true;
}

bool launch_tc_gj_update(Ctx &c, float *M, int64_t lda, int64_t k0, const float *Cb,
                         const float *Rt, int prec, int64_t skip0, const float *Cb_lo,
                         const float *Rt_lo)
{
    return launch_tc_rank64(c, M, lda, c.n, Cb, Rt, prec, skip0, k0, Cb_lo, Rt_lo);
}

}  // namespace nrs
