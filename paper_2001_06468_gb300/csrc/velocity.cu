// velocity.cu -- the fluid velocity at field points and the passive tracers
// it carries (the particle tracking of Gallagher & Smith's mouse-node and
// sperm examples): the NEAREST boundary integral of Sec. 3 evaluated off the
// body,
//   u(x_p) = (1/(8 pi mu)) sum_q S^eps(x_p - X_q) w_q f_{n(q)},
// with f the force density of the stage's solve and n(q) the nearest force
// point of quadrature point q.
//
// One CTA takes 128 field points and a contiguous range of quadrature points
// (staged through shared memory with their f_{n(q)} gathered), one thread
// per field point accumulating the three components in FP64, every term
// evaluated as the assembly evaluates it (correctly rounded square root and
// division, no fused multiply-add).  The ranges' partial sums are added in
// ascending order by a second kernel: deterministic.
#include "nrs_internal.cuh"

namespace nrs {

namespace {

constexpr int VL_THREADS = 128;
constexpr int VL_CHUNK = 256;  // quadrature points staged at a time

// part[(s * P + p) * 3 + j] = sum over quadrature points q of range s of
// (S_jk w_q) f_k(n(q)), k in order, q ascending.
__global__ void __launch_bounds__(VL_THREADS)
    k_velocity_part(int64_t P, const D4 *__restrict__ xp, int64_t Q, const D4 *__restrict__ Xw,
                    const int32_t *__restrict__ nn, const double *__restrict__ f, double eps2,
                    int64_t q_per_split, double *__restrict__ part)
{
    __shared__ D4 sX[VL_CHUNK];
    __shared__ double sF[VL_CHUNK][3];
    const int64_t p = (int64_t)blockIdx.x * VL_THREADS + threadIdx.x;
    const int64_t s = blockIdx.y;
    const int64_t q0 = s * q_per_split, q1 = min(Q, q0 + q_per_split);
    const bool active = p < P;
    double px = 0.0, py = 0.0, pz = 0.0;
    if (active) {
        const D4 v = xp[p];
        px = v.x;
        py = v.y;
        pz = v.z;
    }
    const double two_e2 = __dmul_rn(2.0, eps2);
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    for (int64_t c0 = q0; c0 < q1; c0 += VL_CHUNK) {
        const int cnt = (int)min((int64_t)VL_CHUNK, q1 - c0);
        __syncthreads();
        for (int i = threadIdx.x; i < cnt; i += VL_THREADS) {
            sX[i] = Xw[c0 + i];
            const double *fq = f + 3 * (int64_t)nn[c0 + i];
            sF[i][0] = fq[0];
            sF[i][1] = fq[1];
            sF[i][2] = fq[2];
        }
        __syncthreads();
        for (int i = 0; i < cnt; ++i) {
            const D4 X = sX[i];
            const double rx = __dsub_rn(px, X.x), ry = __dsub_rn(py, X.y), rz = __dsub_rn(pz, X.z);
            const double r2 =
                __dadd_rn(__dadd_rn(__dmul_rn(rx, rx), __dmul_rn(ry, ry)), __dmul_rn(rz, rz));
            const double rho = __dadd_rn(r2, eps2);
            const double inv = __ddiv_rn(1.0, __dmul_rn(rho, __dsqrt_rn(rho)));
            const double dg = __dadd_rn(r2, two_e2);
            const double w = X.w;
            // S_jk w (symmetric: six distinct values)
            const double sxx = __dmul_rn(__dmul_rn(__dadd_rn(__dmul_rn(rx, rx), dg), inv), w);
            const double sxy = __dmul_rn(__dmul_rn(__dmul_rn(rx, ry), inv), w);
            const double sxz = __dmul_rn(__dmul_rn(__dmul_rn(rx, rz), inv), w);
            const double syy = __dmul_rn(__dmul_rn(__dadd_rn(__dmul_rn(ry, ry), dg), inv), w);
            const double syz = __dmul_rn(__dmul_rn(__dmul_rn(ry, rz), inv), w);
            const double szz = __dmul_rn(__dmul_rn(__dadd_rn(__dmul_rn(rz, rz), dg), inv), w);
            const double f0 = sF[i][0], f1 = sF[i][1], f2 = sF[i][2];
            a0 = __dadd_rn(a0, __dadd_rn(__dadd_rn(__dmul_rn(sxx, f0), __dmul_rn(sxy, f1)),
                                         __dmul_rn(sxz, f2)));
            a1 = __dadd_rn(a1, __dadd_rn(__dadd_rn(__dmul_rn(sxy, f0), __dmul_rn(syy, f1)),
                                         __dmul_rn(syz, f2)));
            a2 = __dadd_rn(a2, __dadd_rn(__dadd_rn(__dmul_rn(sxz, f0), __dmul_rn(syz, f1)),
                                         __dmul_rn(szz, f2)));
        }
    }
    if (active) {
        double *o = part + (s * P + p) * 3;
        o[0] = a0;
        o[1] = a1;
        o[2] = a2;
    }
}

// u[p] = (c sum_s part[s][p], 0), the ranges added in ascending order
__global__ void k_velocity_finish(int64_t P, int splits, const double *__restrict__ part, double c,
                                  D4 *__restrict__ u)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    for (int s = 0; s < splits; ++s) {
        const double *o = part + ((int64_t)s * P + p) * 3;
        a0 = __dadd_rn(a0, o[0]);
        a1 = __dadd_rn(a1, o[1]);
        a2 = __dadd_rn(a2, o[2]);
    }
    D4 r;
    r.x = __dmul_rn(a0, c);
    r.y = __dmul_rn(a1, c);
    r.z = __dmul_rn(a2, c);
    r.w = 0.0;
    u[p] = r;
}

// Tracer positions of the explicit midpoint: stage 0 x = x_save + dt/2 u,
// stage 1 x = x_save + dt u (column 3 kept).
__global__ void k_tracer_update(int64_t P, int stage, double dt, const D4 *__restrict__ x_save,
                                const D4 *__restrict__ u, D4 *__restrict__ x)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const double h = stage == 0 ? __dmul_rn(0.5, dt) : dt;
    const D4 a = x_save[p], v = u[p];
    D4 r;
    r.x = __dadd_rn(a.x, __dmul_rn(h, v.x));
    r.y = __dadd_rn(a.y, __dmul_rn(h, v.y));
    r.z = __dadd_rn(a.z, __dmul_rn(h, v.z));
    r.w = a.w;
    x[p] = r;
}

}  // namespace

// Quadrature-range splits of the velocity kernel for P field points: about
// four CTAs per SM in all, each range at least one staging chunk.
int velocity_splits(const Ctx &c, int64_t P)
{
    const int64_t tiles = ceil_div(P, VL_THREADS);
    int64_t s = ceil_div(4 * (int64_t)c.num_sms, tiles);
    s = std::min<int64_t>(s, ceil_div(c.Q, VL_CHUNK));
    return (int)std::max<int64_t>(1, std::min<int64_t>(s, 1024));
}

// u (device [P*4]) at xp (device [P*4]) from the force density f (device,
// 3 per force point), the lab-frame quadrature points Xw (device [Q*4]) and
// the context's nearest-neighbour map; part: device workspace of
// velocity_splits(c, P) * P * 3 doubles.
void launch_velocity(Ctx &c, const D4 *Xw, const D4 *xp, int64_t P, const double *f, D4 *u,
                     double *part, cudaStream_t s)
{
    if (P <= 0) return;
    const int splits = velocity_splits(c, P);
    const int64_t qps = ceil_div(c.Q, splits);
    const double coef = 1.0 / (8.0 * kPi * c.mu);
    dim3 grid((unsigned)ceil_div(P, VL_THREADS), (unsigned)splits);
    k_velocity_part<<<grid, VL_THREADS, 0, s>>>(P, xp, c.Q, Xw, c.d_nn, f, c.eps * c.eps, qps,
                                                part);
    k_velocity_finish<<<(unsigned)ceil_div(P, 256), 256, 0, s>>>(P, splits, part, coef, u);
    c.launches += 2;
}

void launch_tracer_update(Ctx &c, int stage, double dt, cudaStream_t s)
{
    k_tracer_update<<<(unsigned)ceil_div(c.n_tracers, 256), 256, 0, s>>>(
        c.n_tracers, stage, dt, c.d_tr_save, c.d_tr_u, c.d_tr);
    c.launches += 1;
}

}  // namespace nrs
