// geometry.cu -- kinematics, nearest neighbours, segments of nu, rigid-body
// border and the explicit-midpoint state update (Gallagher & Smith, Sec. 3
// and Sec. 4).
#include <math.h>

#include "nrs_internal.cuh"

namespace nrs {

// ---------------------------------------------------------------------------
// kinematics (Sec. 4: the state Y = [X0; B] places each body)
// ---------------------------------------------------------------------------

// x0 + ((B_r0 p0 + B_r1 p1) + B_r2 p2), rounded step by step (no fused
// multiply-add) so that lab-frame clouds are reproducible bit for bit.
__device__ __forceinline__ double rigid_row(const double *x0, const double *B, int r, double p0,
                                            double p1, double p2)
{
    double s = __dadd_rn(__dmul_rn(B[3 * r + 0], p0), __dmul_rn(B[3 * r + 1], p1));
    s = __dadd_rn(s, __dmul_rn(B[3 * r + 2], p2));
    return __dadd_rn(x0[r], s);
}

__global__ void k_kinematics(int64_t N, int64_t Q, int64_t F, const D4 *__restrict__ xi,
                             const D4 *__restrict__ Xiw, const D4 *__restrict__ xidot,
                             const int32_t *__restrict__ body_x, const int32_t *__restrict__ body_X,
                             const int32_t *__restrict__ kind, const double *__restrict__ x0,
                             const double *__restrict__ B, const double *__restrict__ U,
                             const double *__restrict__ Om, const double *__restrict__ ext,
                             D4 *__restrict__ x, D4 *__restrict__ Xw, double *__restrict__ b)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) {
        int bd = body_x[i];
        const double *o = x0 + 3 * bd;
        const double *Bb = B + 9 * bd;
        D4 p = xi[i];
        D4 r;
        r.x = rigid_row(o, Bb, 0, p.x, p.y, p.z);
        r.y = rigid_row(o, Bb, 1, p.x, p.y, p.z);
        r.z = rigid_row(o, Bb, 2, p.x, p.y, p.z);
        r.w = p.w;
        x[i] = r;
        double v[3] = {0.0, 0.0, 0.0};
        int kd = kind[bd];
        if (kd != NRS_STATIC) {
            D4 d = xidot[i];
            for (int k = 0; k < 3; ++k) {
                double s = __dadd_rn(__dmul_rn(Bb[3 * k + 0], d.x), __dmul_rn(Bb[3 * k + 1], d.y));
                v[k] = __dadd_rn(s, __dmul_rn(Bb[3 * k + 2], d.z));
            }
        }
        if (kd == NRS_PRESCRIBED) {
            double rr[3] = {__dsub_rn(r.x, o[0]), __dsub_rn(r.y, o[1]), __dsub_rn(r.z, o[2])};
            const double *w = Om + 3 * bd;
            double oxr[3] = {__dsub_rn(__dmul_rn(w[1], rr[2]), __dmul_rn(w[2], rr[1])),
                             __dsub_rn(__dmul_rn(w[2], rr[0]), __dmul_rn(w[0], rr[2])),
                             __dsub_rn(__dmul_rn(w[0], rr[1]), __dmul_rn(w[1], rr[0]))};
            for (int k = 0; k < 3; ++k) v[k] = __dadd_rn(v[k], __dadd_rn(U[3 * bd + k], oxr[k]));
        }
        b[3 * i + 0] = v[0];
        b[3 * i + 1] = v[1];
        b[3 * i + 2] = v[2];
    } else if (i < N + Q) {
        int64_t q = i - N;
        int bd = body_X[q];
        const double *o = x0 + 3 * bd;
        const double *Bb = B + 9 * bd;
        D4 p = Xiw[q];
        D4 r;
        r.x = rigid_row(o, Bb, 0, p.x, p.y, p.z);
        r.y = rigid_row(o, Bb, 1, p.x, p.y, p.z);
        r.z = rigid_row(o, Bb, 2, p.x, p.y, p.z);
        r.w = p.w;
        Xw[q] = r;
    } else if (i < N + Q + 6 * F) {
        int64_t c = i - N - Q;
        b[3 * N + c] = ext[c];
    }
}

void launch_kinematics(Ctx &c, const D4 *xi, const D4 *Xiw, const D4 *xidot, D4 *x, D4 *Xw,
                       double *b)
{
    int64_t total = c.N + c.Q + 6 * c.F;
    int threads = 256;
    c.tbeg(PH_KINEMATICS);
    k_kinematics<<<(unsigned)ceil_div(total, threads), threads, 0, c.stream>>>(
        c.N, c.Q, c.F, xi, Xiw, xidot, c.d_body_x, c.d_body_X, c.d_kind, c.d_x0, c.d_B, c.d_U,
        c.d_Om, c.d_ext, x, Xw, b);
    c.tend(PH_KINEMATICS);
    c.launches += 1;
}

// ---------------------------------------------------------------------------
// nearest neighbours (Sec. 3: n-hat(q) = argmin_n |x[n] - X[q]|)
// ---------------------------------------------------------------------------
//
// Two passes over the candidate force points, staged through shared memory.
// Pass 1 finds m_f, the smallest FP32 squared distance.  With C the largest
// coordinate magnitude involved, every FP32 difference component is within
// delta = 2^-24 (|x| + |X| + |dx|) <= 4.01 * 2^-24 * C of the exact one, so
// the difference vector is within e = sqrt(3) delta <= 4.2e-7 C of exact and
// the FP32 squared distance within 4 u of its rounded components.  A force
// point can be (or tie with) the FP64 minimiser only if
//     sqrt(d2_f) <= (sqrt(m_f) (1 + 1e-6) + 2 e) (1 + 1e-6);
// pass 2 evaluates exactly those candidates in FP64 with the operation order
// ((dx*dx + dy*dy) + dz*dz), keeping the first strict minimum in ascending
// index order.  The 1e-6 factors dominate every FP32 rounding of the bound
// itself (u = 2^-24 ~ 6e-8), so the result equals an exhaustive FP64 search.

constexpr int NN_TILE = 512;

// The NN_SPLIT threads of a quadrature point are consecutive lanes; each scans
// the candidates i = sub, sub + NN_SPLIT, ... of every tile in ascending order,
// and the lanes combine their results: the FP32 minimum (exact, order-free)
// and, in pass 2, the lexicographic minimum of (FP64 distance, index), which
// is the first strict minimum of the ascending scan.
__global__ void __launch_bounds__(NN_THREADS)
    k_nearest(const NNTask *__restrict__ tasks, const int64_t *__restrict__ n_off, int nbodies,
              int global, const D4 *__restrict__ x, const D4 *__restrict__ X,
              int32_t *__restrict__ nn, int32_t *status)
{
    __shared__ float4 tile[NN_TILE];
    __shared__ unsigned int s_cmax;
    const NNTask t = tasks[blockIdx.x];
    const int64_t n_lo = global ? 0 : n_off[t.body];
    const int64_t n_hi = global ? n_off[nbodies] : n_off[t.body + 1];
    const int sub = threadIdx.x % NN_SPLIT;
    const int64_t q = (int64_t)t.q0 + threadIdx.x / NN_SPLIT;
    const bool active = q < t.q1;
    double qx = 0.0, qy = 0.0, qz = 0.0;
    if (active) {
        D4 p = X[q];
        qx = p.x;
        qy = p.y;
        qz = p.z;
    }
    const float fx = __double2float_rn(qx), fy = __double2float_rn(qy), fz = __double2float_rn(qz);
    if (threadIdx.x == 0) s_cmax = 0u;
    float best = __int_as_float(0x7f800000);

    for (int64_t base = n_lo; base < n_hi; base += NN_TILE) {
        const int cnt = (int)min((int64_t)NN_TILE, n_hi - base);
        __syncthreads();
        float lmax = 0.0f;
        for (int i = threadIdx.x; i < cnt; i += NN_THREADS) {
            D4 p = x[base + i];
            float4 v = make_float4(__double2float_rn(p.x), __double2float_rn(p.y),
                                   __double2float_rn(p.z), 0.0f);
            tile[i] = v;
            lmax = fmaxf(lmax, fmaxf(fabsf(v.x), fmaxf(fabsf(v.y), fabsf(v.z))));
        }
        for (int o = 16; o > 0; o >>= 1) lmax = fmaxf(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
        if ((threadIdx.x & 31) == 0) atomicMax(&s_cmax, __float_as_uint(lmax));
        __syncthreads();
        if (active) {
#pragma unroll 8
            for (int i = sub; i < cnt; i += NN_SPLIT) {
                float4 v = tile[i];
                float dx = v.x - fx, dy = v.y - fy, dz = v.z - fz;
                float d2 = dx * dx + dy * dy + dz * dz;
                best = fminf(best, d2);
            }
        }
    }
#pragma unroll
    for (int o = 1; o < NN_SPLIT; o <<= 1) best = fminf(best, __shfl_xor_sync(0xffffffffu, best, o));
    __syncthreads();
    const float cmax =
        fmaxf(__uint_as_float(s_cmax), fmaxf(fabsf(fx), fmaxf(fabsf(fy), fabsf(fz))));
    const float e = 4.2e-7f * cmax;
    float th = (sqrtf(best) * (1.0f + 1e-6f) + 2.0f * e + 1e-30f) * (1.0f + 1e-6f);
    th = th * th;

    double best64 = __longlong_as_double(0x7ff0000000000000LL);
    int64_t arg = -1;
    for (int64_t base = n_lo; base < n_hi; base += NN_TILE) {
        const int cnt = (int)min((int64_t)NN_TILE, n_hi - base);
        __syncthreads();
        for (int i = threadIdx.x; i < cnt; i += NN_THREADS) {
            D4 p = x[base + i];
            tile[i] = make_float4(__double2float_rn(p.x), __double2float_rn(p.y),
                                  __double2float_rn(p.z), 0.0f);
        }
        __syncthreads();
        if (active) {
            for (int i = sub; i < cnt; i += NN_SPLIT) {
                float4 v = tile[i];
                float dx = v.x - fx, dy = v.y - fy, dz = v.z - fz;
                float d2 = dx * dx + dy * dy + dz * dz;
                if (d2 <= th) {
                    D4 p = x[base + i];
                    double ex = __dsub_rn(p.x, qx), ey = __dsub_rn(p.y, qy), ez = __dsub_rn(p.z, qz);
                    double s = __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)),
                                         __dmul_rn(ez, ez));
                    if (s < best64) {
                        best64 = s;
                        arg = base + i;
                    }
                }
            }
        }
    }
#pragma unroll
    for (int o = 1; o < NN_SPLIT; o <<= 1) {
        const double os = __shfl_xor_sync(0xffffffffu, best64, o);
        const int64_t oa = __shfl_xor_sync(0xffffffffu, arg, o);
        if (oa >= 0 && (arg < 0 || os < best64 || (os == best64 && oa < arg))) {
            best64 = os;
            arg = oa;
        }
    }
    if (active && sub == 0) {
        nn[q] = (int32_t)arg;  // -1 only when no distance was finite (NaN/Inf input)
        if (arg < 0) atomicOr(status, ST_NONFINITE);
    }
}

void launch_nearest(Ctx &c, const D4 *x, const D4 *Xw, int32_t *nn, bool only_deforming)
{
    const NNTask *tasks = only_deforming ? c.d_tasks_deform : c.d_tasks_all;
    int count = only_deforming ? c.n_tasks_deform : c.n_tasks_all;
    if (count == 0) return;
    c.tbeg(PH_NEAREST);
    k_nearest<<<count, NN_THREADS, 0, c.stream>>>(tasks, c.d_n_off, c.nbodies, c.nn_global, x, Xw,
                                                   nn, c.d_status);
    c.tend(PH_NEAREST);
    c.launches += 1;
}

// ---------------------------------------------------------------------------
// segments of nu: stable counting sort of q by n-hat(q)
// ---------------------------------------------------------------------------

// Quadrature points without a valid nearest force point (non-finite input,
// flagged by k_nearest) are left out of every segment.
__global__ void k_count(int64_t Q, int64_t N, const int32_t *__restrict__ nn,
                        int32_t *__restrict__ cnt)
{
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < Q) {
        const int32_t k = nn[q];
        if (k >= 0 && k < N) atomicAdd(&cnt[k], 1);
    }
}

// Exclusive scan of cnt[0..N) into seg_ptr[0..N] (single block of 1024).
__global__ void __launch_bounds__(1024)
    k_scan(int64_t N, const int32_t *cnt, int32_t *__restrict__ seg_ptr, int32_t *cursor)
{
    __shared__ int32_t part[1024];
    const int tid = threadIdx.x;
    const int64_t chunk = ceil_div(N, 1024);
    const int64_t lo = min(N, tid * chunk), hi = min(N, lo + chunk);
    int32_t s = 0;
    for (int64_t i = lo; i < hi; ++i) s += cnt[i];
    part[tid] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        int32_t v = tid >= off ? part[tid - off] : 0;
        __syncthreads();
        part[tid] += v;
        __syncthreads();
    }
    int32_t run = tid ? part[tid - 1] : 0;
    for (int64_t i = lo; i < hi; ++i) {
        int32_t ci = cnt[i];  // cnt may alias cursor: read before overwriting
        seg_ptr[i] = run;
        cursor[i] = run;
        run += ci;
    }
    if (tid == 1023) {
        seg_ptr[N] = part[1023];
        cursor[N] = part[1023];
    }
}

__global__ void k_scatter(int64_t Q, int64_t N, const int32_t *__restrict__ nn,
                          int32_t *__restrict__ cursor, int32_t *__restrict__ perm)
{
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < Q) {
        const int32_t k = nn[q];
        if (k < 0 || k >= N) return;
        int32_t pos = atomicAdd(&cursor[k], 1);
        perm[pos] = (int32_t)q;
    }
}

// Order each segment by ascending q (insertion sort; segments hold ~Q/N points).
__global__ void k_sort_segments(int64_t N, const int32_t *__restrict__ seg_ptr,
                                int32_t *__restrict__ perm)
{
    int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    int32_t lo = seg_ptr[n], hi = seg_ptr[n + 1];
    for (int32_t i = lo + 1; i < hi; ++i) {
        int32_t v = perm[i];
        int32_t j = i - 1;
        while (j >= lo && perm[j] > v) {
            perm[j + 1] = perm[j];
            --j;
        }
        perm[j + 1] = v;
    }
}

void launch_segments(Ctx &c, const int32_t *nn, int32_t *seg_ptr, int32_t *perm)
{
    int threads = 256;
    c.tbeg(PH_SEGMENTS);
    cudaMemsetAsync(c.d_cursor, 0, sizeof(int32_t) * (c.N + 1), c.stream);
    cudaMemsetAsync(perm, 0, sizeof(int32_t) * c.Q, c.stream);  // tail stays a valid index
    k_count<<<(unsigned)ceil_div(c.Q, threads), threads, 0, c.stream>>>(c.Q, c.N, nn, c.d_cursor);
    // the counts are read from d_cursor, scanned into seg_ptr and back into d_cursor
    k_scan<<<1, 1024, 0, c.stream>>>(c.N, c.d_cursor, seg_ptr, c.d_cursor);
    k_scatter<<<(unsigned)ceil_div(c.Q, threads), threads, 0, c.stream>>>(c.Q, c.N, nn, c.d_cursor,
                                                                          perm);
    k_sort_segments<<<(unsigned)ceil_div(c.N, threads), threads, 0, c.stream>>>(c.N, seg_ptr, perm);
    c.tend(PH_SEGMENTS);
    c.launches += 4;
}

// Lab-frame quadrature points in segment order, and per-segment moments
// W_n = sum w_q, R_n = sum w_q (X_q - x0_b) accumulated in ascending q: one
// thread per segment gathers its points and sums them.  Quadrature points
// left out of every segment (no valid nearest force point) are not gathered.
__global__ void k_gather_moments(int64_t N, const int32_t *__restrict__ seg_ptr,
                                 const int32_t *__restrict__ perm, const D4 *__restrict__ Xw,
                                 D4 *__restrict__ Xs, const int32_t *__restrict__ body_x,
                                 const double *__restrict__ x0, double *__restrict__ W,
                                 double *__restrict__ R)
{
    int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const double *o = x0 + 3 * body_x[n];
    double w_sum = 0.0, r0 = 0.0, r1 = 0.0, r2 = 0.0;
    for (int32_t p = seg_ptr[n]; p < seg_ptr[n + 1]; ++p) {
        const D4 X = Xw[perm[p]];
        Xs[p] = X;
        w_sum = __dadd_rn(w_sum, X.w);
        r0 = __dadd_rn(r0, __dmul_rn(X.w, __dsub_rn(X.x, o[0])));
        r1 = __dadd_rn(r1, __dmul_rn(X.w, __dsub_rn(X.y, o[1])));
        r2 = __dadd_rn(r2, __dmul_rn(X.w, __dsub_rn(X.z, o[2])));
    }
    W[n] = w_sum;
    R[3 * n + 0] = r0;
    R[3 * n + 1] = r1;
    R[3 * n + 2] = r2;
}

void launch_gather(Ctx &c, const D4 *Xw_lab, const int32_t *seg_ptr, const int32_t *perm)
{
    int threads = 128;
    c.tbeg(PH_SEGMENTS);
    k_gather_moments<<<(unsigned)ceil_div(c.N, threads), threads, 0, c.stream>>>(
        c.N, seg_ptr, perm, Xw_lab, c.d_Xs, c.d_body_x, c.d_x0, c.d_W, c.d_R);
    c.tend(PH_SEGMENTS);
    c.launches += 1;
}

// ---------------------------------------------------------------------------
// rigid-body border (Sec. 4: unknown U, Omega; force and moment balance)
// ---------------------------------------------------------------------------

__device__ __forceinline__ double cross_entry(const double v[3], int j, int k)
{
    // [v]x = [[0,-v2,v1],[v2,0,-v0],[-v1,v0,0]]
    if (j == k) return 0.0;
    if (j == 0) return k == 1 ? -v[2] : v[1];
    if (j == 1) return k == 0 ? v[2] : -v[0];
    return k == 0 ? -v[1] : v[0];
}

__global__ void k_border(int64_t N, int64_t n, const int32_t *__restrict__ free_body,
                         const int32_t *__restrict__ body_x, const D4 *__restrict__ x,
                         const double *__restrict__ x0, const double *__restrict__ W,
                         const double *__restrict__ R, double *__restrict__ A64,
                         float *__restrict__ A32, float2 *__restrict__ Adf, int64_t lda)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = blockIdx.y;  // border unknown / row 0 .. 6F-1
    const int f = c / 6, cc = c % 6;
    const int bd = free_body[f];
    const int64_t base = 3 * N + 6 * (int64_t)f;
    double col = 0.0, row = 0.0;
    if (i < 3 * N) {
        const int64_t m = i / 3;
        const int jk = (int)(i % 3);
        if (body_x[m] == bd) {
            if (cc < 3) {
                col = (jk == cc) ? -1.0 : 0.0;
                row = (jk == cc) ? W[m] : 0.0;
            } else {
                D4 p = x[m];
                double r[3] = {__dsub_rn(p.x, x0[3 * bd + 0]), __dsub_rn(p.y, x0[3 * bd + 1]),
                               __dsub_rn(p.z, x0[3 * bd + 2])};
                col = cross_entry(r, jk, cc - 3);
                double Rm[3] = {R[3 * m + 0], R[3 * m + 1], R[3 * m + 2]};
                row = cross_entry(Rm, cc - 3, jk);
            }
        }
    }
    A64[i + (base + cc) * lda] = col;
    A64[(base + cc) + i * lda] = row;
    if (A32) {
        A32[i + (base + cc) * lda] = (float)col;
        A32[(base + cc) + i * lda] = (float)row;
    }
    if (Adf) {
        Adf[i + (base + cc) * lda] = df_split(col);
        Adf[(base + cc) + i * lda] = df_split(row);
    }
}

void launch_border(Ctx &c, const D4 *x_lab, double *A64, float *A32, int64_t lda)
{
    if (c.F == 0) return;
    int threads = 256;
    dim3 grid((unsigned)ceil_div(c.n, threads), (unsigned)(6 * c.F));
    // d_free_index holds nbodies entries (body -> free index) then F entries (free index -> body)
    c.tbeg(PH_BORDER);
    k_border<<<grid, threads, 0, c.stream>>>(c.N, c.n, c.d_free_index + c.nbodies, c.d_body_x, x_lab,
                                             c.d_x0, c.d_W, c.d_R, A64, A32,
                                             (c.arnoldi_df && A64 == c.d_A64) ? c.d_Adf : nullptr,
                                             lda);
    c.tend(PH_BORDER);
    c.launches += 1;
}

// ---------------------------------------------------------------------------
// explicit midpoint update of Y = [X0; B] (Sec. 4), B by modified Gram-Schmidt
// ---------------------------------------------------------------------------

__global__ void k_rk2(int stage, double dt, int nbodies, int64_t N,
                      const int32_t *__restrict__ kind, const int32_t *__restrict__ free_index,
                      const double *__restrict__ sol, const double *__restrict__ U,
                      const double *__restrict__ Om, const double *__restrict__ x0_save,
                      const double *__restrict__ B_save, double *__restrict__ x0,
                      double *__restrict__ B)
{
    int bd = blockIdx.x * blockDim.x + threadIdx.x;
    if (bd >= nbodies) return;
    int kd = kind[bd];
    if (kd == NRS_STATIC) return;
    double u[3], w[3];
    if (kd == NRS_FREE) {
        const double *v = sol + 3 * N + 6 * (int64_t)free_index[bd];
        for (int k = 0; k < 3; ++k) {
            u[k] = v[k];
            w[k] = v[3 + k];
        }
    } else {
        for (int k = 0; k < 3; ++k) {
            u[k] = U[3 * bd + k];
            w[k] = Om[3 * bd + k];
        }
    }
    const double h = stage == 0 ? 0.5 * dt : dt;
    double Bc[9], Bn[9];
    for (int k = 0; k < 9; ++k) Bc[k] = B[9 * bd + k];
    // dB = [w]x Bc ; Bn = B_save + h dB
    for (int r = 0; r < 3; ++r)
        for (int col = 0; col < 3; ++col) {
            double d = 0.0;
            for (int k = 0; k < 3; ++k) {
                double wx = (r == k) ? 0.0
                            : (r == 0) ? (k == 1 ? -w[2] : w[1])
                            : (r == 1) ? (k == 0 ? w[2] : -w[0])
                                       : (k == 0 ? -w[1] : w[0]);
                d += wx * Bc[3 * k + col];
            }
            Bn[3 * r + col] = B_save[9 * bd + 3 * r + col] + h * d;
        }
    for (int k = 0; k < 3; ++k) x0[3 * bd + k] = x0_save[3 * bd + k] + h * u[k];
    // modified Gram-Schmidt on the columns
    for (int j = 0; j < 3; ++j) {
        for (int i = 0; i < j; ++i) {
            double dot = Bn[i] * Bn[j] + Bn[3 + i] * Bn[3 + j] + Bn[6 + i] * Bn[6 + j];
            for (int r = 0; r < 3; ++r) Bn[3 * r + j] -= dot * Bn[3 * r + i];
        }
        double nrm = sqrt(Bn[j] * Bn[j] + Bn[3 + j] * Bn[3 + j] + Bn[6 + j] * Bn[6 + j]);
        for (int r = 0; r < 3; ++r) Bn[3 * r + j] /= nrm;
    }
    for (int k = 0; k < 9; ++k) B[9 * bd + k] = Bn[k];
}

void launch_rk2(Ctx &c, int stage, double dt, const double *sol)
{
    c.tbeg(PH_UPDATE);
    k_rk2<<<(unsigned)ceil_div(c.nbodies, 64), 64, 0, c.stream>>>(
        stage, dt, c.nbodies, c.N, c.d_kind, c.d_free_index, sol, c.d_U, c.d_Om, c.d_x0_save,
        c.d_B_save, c.d_x0, c.d_B);
    c.tend(PH_UPDATE);
    c.launches += 1;
}

}  // namespace nrs
