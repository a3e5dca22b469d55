// assemble.cu -- the NEAREST matrix A_s (Gallagher & Smith, Sec. 3 eq.
// nnrsbie and Sec. 4 step 1):
//
//   A[3m+j, 3n+k] = (1/(8 pi mu)) sum_{q in seg(n)} S^eps_jk(x_m - X_q) w_q,
//   S^eps_jk(r)   = (delta_jk (|r|^2 + 2 eps^2) + r_j r_k) / (|r|^2 + eps^2)^{3/2}.
//
// The 3N x 3Q stokeslet matrix and the sparse nu are never formed: the
// quadrature points are stored in segment order (segment n = the points
// whose nearest force point is n), so each (m, n) block is a register
// reduction over one contiguous run of quadrature points.  One thread owns a
// collocation point m; a block of threads shares a tile of AS_NT segments
// whose quadrature points are staged through shared memory.  Six distinct
// products r_j r_k t and one diagonal term (|r|^2 + 2 eps^2) t are
// accumulated per (m, n); no atomics.
//
// For the mixed-precision path the FP32 copy that the factorisation inverts
// comes from k_assemble32 (FP32 arithmetic after an FP64 difference), so the
// factorisation can start at once; k_assemble64 then builds the FP64 matrix
// that only the refinement's residuals need, on a low-priority stream that
// overlaps the factorisation.
#include <math.h>

#include <algorithm>

#include "nrs_internal.cuh"

namespace nrs {

constexpr int AS_THREADS = (int)kAssembleTileM;
constexpr int AS_NT = (int)kAssembleTileN;
constexpr int AS_CHUNK = 512;
// the FP64 kernel runs beside the fused factorisation, whose CTA takes about
// 195 KB of an SM's shared memory: its staging chunk is kept at 8 KB so that
// up to three of its CTAs still fit beside one (the order of the sums over q
// does not depend on the chunk)
constexpr int AS64_CHUNK = 256;

struct Acc6 {
    double xx, xy, xz, yy, yz, zz;
};

// The FP64 entries are the definition evaluated term by term in one fixed
// order, with every operation rounded on its own (no fused multiply-add,
// correctly rounded square root and division):
//   r = x_m - X_q,  |r|^2 = (r0 r0 + r1 r1) + r2 r2,  rho = |r|^2 + eps^2,
//   s = 1 / (rho sqrt(rho)),  S_jk = (r_j r_k [+ (|r|^2 + 2 eps^2) if j = k]) s,
//   acc_jk += S_jk w_q  (q ascending within the segment),  A = acc_jk / (8 pi mu)
// so each entry is a deterministic function of the inputs, independent of
// the tiling and of the device.
__device__ __forceinline__ void flush_block(int64_t m, int64_t n, const Acc6 &a, double c,
                                            double *__restrict__ A64, float *__restrict__ A32,
                                            float2 *__restrict__ Adf, int64_t lda)
{
    const double v[9] = {__dmul_rn(a.xx, c), __dmul_rn(a.xy, c), __dmul_rn(a.xz, c),
                         __dmul_rn(a.xy, c), __dmul_rn(a.yy, c), __dmul_rn(a.yz, c),
                         __dmul_rn(a.xz, c), __dmul_rn(a.yz, c), __dmul_rn(a.zz, c)};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int64_t col = (3 * n + k) * lda + 3 * m;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            A64[col + j] = v[3 * j + k];
            if (A32) A32[col + j] = (float)v[3 * j + k];
            if (Adf) Adf[col + j] = df_split(v[3 * j + k]);
        }
    }
}

__device__ __forceinline__ void add_pair(double mx, double my, double mz, const D4 &X,
                                         double eps2, double two_e2, Acc6 &a)
{
    const double rx = __dsub_rn(mx, X.x), ry = __dsub_rn(my, X.y), rz = __dsub_rn(mz, X.z);
    const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(rx, rx), __dmul_rn(ry, ry)), __dmul_rn(rz, rz));
    const double rho = __dadd_rn(r2, eps2);
    const double s = __ddiv_rn(1.0, __dmul_rn(rho, __dsqrt_rn(rho)));
    const double dg = __dadd_rn(r2, two_e2);
    const double w = X.w;
    a.xx = __dadd_rn(a.xx, __dmul_rn(__dmul_rn(__dadd_rn(__dmul_rn(rx, rx), dg), s), w));
    a.xy = __dadd_rn(a.xy, __dmul_rn(__dmul_rn(__dmul_rn(rx, ry), s), w));
    a.xz = __dadd_rn(a.xz, __dmul_rn(__dmul_rn(__dmul_rn(rx, rz), s), w));
    a.yy = __dadd_rn(a.yy, __dmul_rn(__dmul_rn(__dadd_rn(__dmul_rn(ry, ry), dg), s), w));
    a.yz = __dadd_rn(a.yz, __dmul_rn(__dmul_rn(__dmul_rn(ry, rz), s), w));
    a.zz = __dadd_rn(a.zz, __dmul_rn(__dmul_rn(__dadd_rn(__dmul_rn(rz, rz), dg), s), w));
}

// One tile = AS_THREADS collocation points x AS_NT segments; tiles are taken
// in grid-stride order (tile = mx + gx * ny), so the kernel also runs on a
// capped grid beside the factorisation.
__global__ void __launch_bounds__(AS_THREADS)
    k_assemble64(int64_t N, const D4 *__restrict__ x, const D4 *__restrict__ Xs,
                 const int32_t *__restrict__ seg_ptr, double eps2, double c,
                 double *__restrict__ A64, float *__restrict__ A32, float2 *__restrict__ Adf,
                 int64_t lda, int64_t gx,
                 int64_t tiles, const uint8_t *__restrict__ mblk_keep,
                 const uint8_t *__restrict__ nblk_keep)
{
    __shared__ D4 sX[AS64_CHUNK];
    __shared__ int32_t sp[AS_NT + 1];
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    // a tile whose collocation points and segments all belong to static rigid
    // bodies keeps the entries of the previous assembly (the same values)
    if (mblk_keep && mblk_keep[tile % gx] && nblk_keep[tile / gx]) continue;
    __syncthreads();  // the previous tile is done with sp and sX
    const int64_t m = (tile % gx) * AS_THREADS + threadIdx.x;
    const int64_t n0 = (tile / gx) * AS_NT;
    const int nt = (int)min((int64_t)AS_NT, N - n0);
    if (threadIdx.x <= nt) sp[threadIdx.x] = seg_ptr[n0 + threadIdx.x];
    const bool active = m < N;
    double mx = 0.0, my = 0.0, mz = 0.0;
    if (active) {
        D4 p = x[m];
        mx = p.x;
        my = p.y;
        mz = p.z;
    }
    const double two_e2 = __dmul_rn(2.0, eps2);
    Acc6 a = {0, 0, 0, 0, 0, 0};
    __syncthreads();
    int cur = 0;
    const int32_t qbeg = sp[0], qend = sp[nt];
    for (int32_t c0 = qbeg; c0 < qend; c0 += AS64_CHUNK) {
        const int cnt = min(AS64_CHUNK, qend - c0);
        const int32_t cend = c0 + cnt;
        __syncthreads();
        for (int i = threadIdx.x; i < cnt; i += AS_THREADS) sX[i] = Xs[c0 + i];
        __syncthreads();
        // segment by segment (bounds uniform across the block): the sums run
        // in ascending q within each segment
        while (cur < nt) {
            const int32_t sb = max(sp[cur], c0), se = min(sp[cur + 1], cend);
            for (int32_t q = sb; q < se; ++q) add_pair(mx, my, mz, sX[q - c0], eps2, two_e2, a);
            if (sp[cur + 1] > cend) break;  // the segment continues in the next chunk
            if (active) flush_block(m, n0 + cur, a, c, A64, A32, Adf, lda);
            a = Acc6{0, 0, 0, 0, 0, 0};
            ++cur;
        }
    }
    while (cur < nt) {
        if (active) flush_block(m, n0 + cur, a, c, A64, A32, Adf, lda);
        a = Acc6{0, 0, 0, 0, 0, 0};
        ++cur;
    }
    }  // tile loop
}

// Coordinates as pairs of floats: p = hi + lo with hi = (float)p and
// lo = (float)(p - hi), so that differences of nearby points are formed in
// FP32 without losing the digits that the FP64 difference keeps.
__global__ void k_split_points(int64_t count, const D4 *__restrict__ p, float4 *__restrict__ hi,
                               float4 *__restrict__ lo)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const D4 v = p[i];
    const float hx = (float)v.x, hy = (float)v.y, hz = (float)v.z;
    hi[i] = make_float4(hx, hy, hz, (float)v.w);
    lo[i] = make_float4((float)(v.x - (double)hx), (float)(v.y - (double)hy),
                        (float)(v.z - (double)hz), 0.0f);
}

// The FP32 copy that the factorisation inverts, on its own: the same sums in
// FP32, with x_m - X_q = (x_hi - X_hi) + (x_lo - X_lo) from the float pairs
// (the hi difference is exact for points closer than their own magnitude),
// so each entry carries a few FP32 roundings.  Each thread owns four
// collocation points (m + h AS_THREADS, h < 4) and evaluates their pairs with
// each staged quadrature point two by two in packed FP32x2 instructions; the
// staged weights carry the factor 1/(8 pi mu); per segment the thread
// accumulates r_j r_k t (six sums) and t, and the diagonal term
// (|r|^2 + 2 eps^2) t is formed at the flush as (r_x^2 + r_y^2 + r_z^2) t +
// 2 eps^2 t from those sums.
constexpr int AS32_P = 4;                // collocation points of a thread
constexpr int AS32_M = AS32_P * AS_THREADS;  // collocation points of a CTA
constexpr int AS32_CHUNK = 256;         // quadrature points staged at a time

// Packed FP32 arithmetic (two lanes of one 64-bit register per instruction,
// sm_100 and later): the thread's two collocation points go through the same
// operations side by side, halving the instructions of the pair loop.
struct F2 {
    float a, b;
};

__device__ __forceinline__ F2 f2_add(F2 x, F2 y)
{
    F2 d;
    asm("{\n\t.reg .b64 p, q, r;\n\t"
        "mov.b64 p, {%2, %3};\n\tmov.b64 q, {%4, %5};\n\t"
        "add.rn.f32x2 r, p, q;\n\tmov.b64 {%0, %1}, r;\n\t}"
        : "=f"(d.a), "=f"(d.b)
        : "f"(x.a), "f"(x.b), "f"(y.a), "f"(y.b));
    return d;
}

__device__ __forceinline__ F2 f2_sub(F2 x, F2 y)
{
    F2 d;
    asm("{\n\t.reg .b64 p, q, r;\n\t"
        "mov.b64 p, {%2, %3};\n\tmov.b64 q, {%4, %5};\n\t"
        "sub.rn.f32x2 r, p, q;\n\tmov.b64 {%0, %1}, r;\n\t}"
        : "=f"(d.a), "=f"(d.b)
        : "f"(x.a), "f"(x.b), "f"(y.a), "f"(y.b));
    return d;
}

__device__ __forceinline__ F2 f2_mul(F2 x, F2 y)
{
    F2 d;
    asm("{\n\t.reg .b64 p, q, r;\n\t"
        "mov.b64 p, {%2, %3};\n\tmov.b64 q, {%4, %5};\n\t"
        "mul.rn.f32x2 r, p, q;\n\tmov.b64 {%0, %1}, r;\n\t}"
        : "=f"(d.a), "=f"(d.b)
        : "f"(x.a), "f"(x.b), "f"(y.a), "f"(y.b));
    return d;
}

// x y + z
__device__ __forceinline__ F2 f2_fma(F2 x, F2 y, F2 z)
{
    F2 d;
    asm("{\n\t.reg .b64 p, q, r, o;\n\t"
        "mov.b64 p, {%2, %3};\n\tmov.b64 q, {%4, %5};\n\tmov.b64 r, {%6, %7};\n\t"
        "fma.rn.f32x2 o, p, q, r;\n\tmov.b64 {%0, %1}, o;\n\t}"
        : "=f"(d.a), "=f"(d.b)
        : "f"(x.a), "f"(x.b), "f"(y.a), "f"(y.b), "f"(z.a), "f"(z.b));
    return d;
}

// A quadrature point staged for the packed loop: every component twice (one
// register pair per operand), the weight times 1/(8 pi mu).
struct alignas(16) StagedQ {
    F2 hx, hy, hz, w;
    F2 lx, ly, lz, pad;
};

__global__ void __launch_bounds__(AS_THREADS)
    k_assemble32(int64_t N, const float4 *__restrict__ xh, const float4 *__restrict__ xl,
                 const float4 *__restrict__ Xh, const float4 *__restrict__ Xl,
                 const int32_t *__restrict__ seg_ptr, float eps2, float c, float *__restrict__ A32,
                 int64_t lda)
{
    __shared__ StagedQ sQ[AS32_CHUNK];
    __shared__ int32_t sp[AS_NT + 1];
    int64_t ms[AS32_P];
    bool act[AS32_P];
    float4 ph[AS32_P], pl[AS32_P];
#pragma unroll
    for (int h = 0; h < AS32_P; ++h) {
        ms[h] = (int64_t)blockIdx.x * AS32_M + threadIdx.x + h * AS_THREADS;
        act[h] = ms[h] < N;
        ph[h] = act[h] ? xh[ms[h]] : make_float4(0.f, 0.f, 0.f, 0.f);
        pl[h] = act[h] ? xl[ms[h]] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const int64_t n0 = (int64_t)blockIdx.y * AS_NT;
    const int nt = (int)min((int64_t)AS_NT, N - n0);
    if (threadIdx.x <= nt) sp[threadIdx.x] = seg_ptr[n0 + threadIdx.x];
    // two packed streams: points (0, 1) and (2, 3)
    F2 px[2], py[2], pz[2], qx[2], qy[2], qz[2];
#pragma unroll
    for (int g = 0; g < 2; ++g) {
        px[g] = F2{ph[2 * g].x, ph[2 * g + 1].x};
        py[g] = F2{ph[2 * g].y, ph[2 * g + 1].y};
        pz[g] = F2{ph[2 * g].z, ph[2 * g + 1].z};
        qx[g] = F2{pl[2 * g].x, pl[2 * g + 1].x};
        qy[g] = F2{pl[2 * g].y, pl[2 * g + 1].y};
        qz[g] = F2{pl[2 * g].z, pl[2 * g + 1].z};
    }
    const F2 e2{eps2, eps2};
    const float two_e2 = 2.0f * eps2;
    const F2 zero{0.0f, 0.0f};
    F2 axx[2], axy[2], axz[2], ayy[2], ayz[2], azz[2], at[2];
#pragma unroll
    for (int g = 0; g < 2; ++g) axx[g] = axy[g] = axz[g] = ayy[g] = ayz[g] = azz[g] = at[g] = zero;
    auto flush = [&](int64_t nn) {
#pragma unroll
        for (int h = 0; h < AS32_P; ++h) {
            const int g = h >> 1;
            const bool lo = (h & 1) == 0;
            const float xx = lo ? axx[g].a : axx[g].b, xy = lo ? axy[g].a : axy[g].b;
            const float xz = lo ? axz[g].a : axz[g].b, yy = lo ? ayy[g].a : ayy[g].b;
            const float yz = lo ? ayz[g].a : ayz[g].b, zz = lo ? azz[g].a : azz[g].b;
            const float tt = lo ? at[g].a : at[g].b;
            if (!act[h]) continue;
            const float d = fmaf(two_e2, tt, (xx + yy) + zz);
            const float v[9] = {xx + d, xy, xz, xy, yy + d, yz, xz, yz, zz + d};
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const int64_t col = (3 * nn + k) * lda + 3 * ms[h];
#pragma unroll
                for (int j = 0; j < 3; ++j) A32[col + j] = v[3 * j + k];
            }
        }
#pragma unroll
        for (int g = 0; g < 2; ++g)
            axx[g] = axy[g] = axz[g] = ayy[g] = ayz[g] = azz[g] = at[g] = zero;
    };
    __syncthreads();
    int cur = 0;
    const int32_t qbeg = sp[0], qend = sp[nt];
    for (int32_t c0 = qbeg; c0 < qend; c0 += AS32_CHUNK) {
        const int cnt = min(AS32_CHUNK, qend - c0);
        const int32_t cend = c0 + cnt;
        __syncthreads();
        for (int i = threadIdx.x; i < cnt; i += AS_THREADS) {
            const float4 h = Xh[c0 + i], l = Xl[c0 + i];
            const float w = h.w * c;  // the weight carries 1/(8 pi mu)
            StagedQ v;
            v.hx = F2{h.x, h.x};
            v.hy = F2{h.y, h.y};
            v.hz = F2{h.z, h.z};
            v.w = F2{w, w};
            v.lx = F2{l.x, l.x};
            v.ly = F2{l.y, l.y};
            v.lz = F2{l.z, l.z};
            v.pad = F2{0.0f, 0.0f};
            sQ[i] = v;
        }
        __syncthreads();
        // segment by segment (bounds uniform across the block), the sums in
        // ascending q
        while (cur < nt) {
            const int32_t sb = max(sp[cur], c0), se = min(sp[cur + 1], cend);
            for (int32_t q = sb; q < se; ++q) {
                const StagedQ Q = sQ[q - c0];
#pragma unroll
                for (int g = 0; g < 2; ++g) {
                    const F2 rx = f2_add(f2_sub(px[g], Q.hx), f2_sub(qx[g], Q.lx));
                    const F2 ry = f2_add(f2_sub(py[g], Q.hy), f2_sub(qy[g], Q.ly));
                    const F2 rz = f2_add(f2_sub(pz[g], Q.hz), f2_sub(qz[g], Q.lz));
                    const F2 r2 = f2_fma(rx, rx, f2_fma(ry, ry, f2_mul(rz, rz)));
                    const F2 u = f2_add(r2, e2);
                    const F2 inv{rsqrtf(u.a), rsqrtf(u.b)};
                    const F2 t = f2_mul(Q.w, f2_mul(inv, f2_mul(inv, inv)));
                    const F2 tx = f2_mul(rx, t), ty = f2_mul(ry, t), tz = f2_mul(rz, t);
                    axx[g] = f2_fma(rx, tx, axx[g]);
                    axy[g] = f2_fma(rx, ty, axy[g]);
                    axz[g] = f2_fma(rx, tz, axz[g]);
                    ayy[g] = f2_fma(ry, ty, ayy[g]);
                    ayz[g] = f2_fma(ry, tz, ayz[g]);
                    azz[g] = f2_fma(rz, tz, azz[g]);
                    at[g] = f2_add(at[g], t);
                }
            }
            if (sp[cur + 1] > cend) break;  // the segment continues in the next chunk
            flush(n0 + cur);
            ++cur;
        }
    }
    while (cur < nt) {
        flush(n0 + cur);
        ++cur;
    }
}

void launch_assemble(Ctx &c, const D4 *x_lab, double *A64, float *A32, int64_t lda,
                     cudaStream_t s, bool from_state)
{
    const bool side = s != nullptr;
    s = side ? s : c.stream;
    static bool attr = false;
    if (!attr) {
        // beside the factorisation, whose diagonal inverse needs a large
        // shared-memory carveout on the SM it lands on
        cudaFuncSetAttribute(k_assemble64, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
        attr = true;
    }
    const int64_t gx = ceil_div(c.N, AS_THREADS), tiles = gx * ceil_div(c.N, AS_NT);
    // beside the factorisation: a few CTAs of four warps per SM (about 25 KB of
    // shared memory and 24K registers), grid-stride over the tiles, so the
    // factorisation's kernels (one CTA per SM each) still find room on every SM
    const int64_t grid = side ? std::min<int64_t>(tiles, (int64_t)c.asm_side_ctas * c.num_sms)
                              : tiles;
    const double coef = 1.0 / (8.0 * kPi * c.mu);
    c.tbeg(PH_ASSEMBLE, s);
    // the blocks among static rigid bodies do not change from one state to the
    // next: kept in the context's FP64 matrix once it holds them (only for an
    // FP64-only pass over the context's own state)
    const bool keep = from_state && A32 == nullptr && A64 == c.d_A64 && c.have_static &&
                      c.static_cache_valid;
    k_assemble64<<<(unsigned)grid, AS_THREADS, 0, s>>>(c.N, x_lab, c.d_Xs, c.d_seg_ptr,
                                                       c.eps * c.eps, coef, A64, A32,
                                                       (c.arnoldi_df && A64 == c.d_A64) ? c.d_Adf
                                                                                        : nullptr,
                                                       lda, gx,
                                                       tiles, keep ? c.d_mblk_keep : nullptr,
                                                       keep ? c.d_nblk_keep : nullptr);
    c.static_cache_valid = from_state && A64 == c.d_A64;
    c.tend(PH_ASSEMBLE, s);
    c.launches += 1;
}

void launch_assemble32(Ctx &c, const D4 *x_lab, float *A32, int64_t lda)
{
    dim3 grid((unsigned)ceil_div(c.N, AS32_M), (unsigned)ceil_div(c.N, AS_NT));
    const float coef = (float)(1.0 / (8.0 * kPi * c.mu));
    c.tbeg(PH_ASSEMBLE32);
    k_split_points<<<(unsigned)ceil_div(c.N, 256), 256, 0, c.stream>>>(c.N, x_lab, c.d_xh, c.d_xl);
    k_split_points<<<(unsigned)ceil_div(c.Q, 256), 256, 0, c.stream>>>(c.Q, c.d_Xs, c.d_Xsh, c.d_Xsl);
    k_assemble32<<<grid, AS_THREADS, 0, c.stream>>>(c.N, c.d_xh, c.d_xl, c.d_Xsh, c.d_Xsl,
                                                    c.d_seg_ptr, (float)(c.eps * c.eps), coef, A32,
                                                    lda);
    c.tend(PH_ASSEMBLE32);
    c.launches += 3;
}

}  // namespace nrs
