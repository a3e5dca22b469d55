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
#include <math.h>

#include "nrs_internal.cuh"

namespace nrs {

constexpr int AS_THREADS = 128;
constexpr int AS_NT = 16;
constexpr int AS_CHUNK = 512;

struct Acc7 {
    double xx, xy, xz, yy, yz, zz, d;
};

__device__ __forceinline__ void flush_block(int64_t m, int64_t n, const Acc7 &a, double c,
                                            double *__restrict__ A64, float *__restrict__ A32,
                                            int64_t lda)
{
    const double v[9] = {c * (a.xx + a.d), c * a.xy,          c * a.xz,
                         c * a.xy,          c * (a.yy + a.d), c * a.yz,
                         c * a.xz,          c * a.yz,          c * (a.zz + a.d)};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int64_t col = (3 * n + k) * lda + 3 * m;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            A64[col + j] = v[3 * j + k];
            if (A32) A32[col + j] = (float)v[3 * j + k];
        }
    }
}

__global__ void __launch_bounds__(AS_THREADS)
    k_assemble64(int64_t N, const D4 *__restrict__ x, const D4 *__restrict__ Xs,
                 const int32_t *__restrict__ seg_ptr, double eps2, double c,
                 double *__restrict__ A64, float *__restrict__ A32, int64_t lda)
{
    __shared__ D4 sX[AS_CHUNK];
    __shared__ int32_t sp[AS_NT + 1];
    const int64_t m = (int64_t)blockIdx.x * AS_THREADS + threadIdx.x;
    const int64_t n0 = (int64_t)blockIdx.y * AS_NT;
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
    const double two_e2 = 2.0 * eps2;
    Acc7 a = {0, 0, 0, 0, 0, 0, 0};
    __syncthreads();
    int cur = 0;
    const int32_t qbeg = sp[0], qend = sp[nt];
    for (int32_t c0 = qbeg; c0 < qend; c0 += AS_CHUNK) {
        const int cnt = min(AS_CHUNK, qend - c0);
        __syncthreads();
        for (int i = threadIdx.x; i < cnt; i += AS_THREADS) sX[i] = Xs[c0 + i];
        __syncthreads();
        int32_t next = sp[cur + 1];
        for (int i = 0; i < cnt; ++i) {
            const int32_t q = c0 + i;
            while (q >= next) {  // uniform across the block
                if (active) flush_block(m, n0 + cur, a, c, A64, A32, lda);
                a = Acc7{0, 0, 0, 0, 0, 0, 0};
                ++cur;
                next = sp[cur + 1];
            }
            const D4 X = sX[i];
            const double rx = mx - X.x, ry = my - X.y, rz = mz - X.z;
            const double r2 = rx * rx + ry * ry + rz * rz;
            const double inv = rsqrt(r2 + eps2);
            const double t = X.w * (inv * inv * inv);
            const double tx = rx * t, ty = ry * t, tz = rz * t;
            a.xx += rx * tx;
            a.xy += rx * ty;
            a.xz += rx * tz;
            a.yy += ry * ty;
            a.yz += ry * tz;
            a.zz += rz * tz;
            a.d += (r2 + two_e2) * t;
        }
    }
    while (cur < nt) {
        if (active) flush_block(m, n0 + cur, a, c, A64, A32, lda);
        a = Acc7{0, 0, 0, 0, 0, 0, 0};
        ++cur;
    }
}

void launch_assemble(Ctx &c, const D4 *x_lab, double *A64, float *A32, int64_t lda)
{
    dim3 grid((unsigned)ceil_div(c.N, AS_THREADS), (unsigned)ceil_div(c.N, AS_NT));
    const double coef = 1.0 / (8.0 * kPi * c.mu);
    c.tbeg(PH_ASSEMBLE);
    k_assemble64<<<grid, AS_THREADS, 0, c.stream>>>(c.N, x_lab, c.d_Xs, c.d_seg_ptr, c.eps * c.eps,
                                                    coef, A64, A32, lda);
    c.tend(PH_ASSEMBLE);
    c.launches += 1;
}

}  // namespace nrs
