// dp.cu -- adaptive Dormand-Prince 5(4) stepping of the swimming IVP
// dY/dt = F(Y, t), Y = [X0; B] per body (Sec. 4: the paper integrates it with
// MATLAB's ode45, which is this pair): the state arithmetic of the
// integrator on the device.
//
//   rates    K_i = (U, [Omega]x B) per body from the stage's solution (free
//            bodies), the prescribed motion, or zero (static bodies)
//   combine  Y_i = Y_n + h sum_{j<i} a_ij K_j, then B re-orthonormalised by
//            modified Gram-Schmidt (the projection the RK2 step uses)
//   error    err = max over the state's components of
//            |h sum_j e_j K_j| / (atol + rtol max(|Y_n|, |Y_n+1|)),
//            e = b5 - b4 (the embedded fourth-order solution)
// The stage sequence, the accept/reject decision and the step size are
// host control flow in api.cu.
#include "nrs_internal.cuh"

namespace nrs {

namespace {

__global__ void k_dp_rates(int nbodies, int64_t N, const int32_t *__restrict__ kind,
                           const int32_t *__restrict__ free_index, const double *__restrict__ sol,
                           const double *__restrict__ U, const double *__restrict__ Om,
                           const double *__restrict__ B, double *__restrict__ K)
{
    const int bd = blockIdx.x * blockDim.x + threadIdx.x;
    if (bd >= nbodies) return;
    double *k = K + 12 * bd;
    const int kd = kind[bd];
    if (kd == NRS_STATIC) {
        for (int i = 0; i < 12; ++i) k[i] = 0.0;
        return;
    }
    double u[3], w[3];
    if (kd == NRS_FREE) {
        const double *v = sol + 3 * N + 6 * (int64_t)free_index[bd];
        for (int i = 0; i < 3; ++i) {
            u[i] = v[i];
            w[i] = v[3 + i];
        }
    } else {
        for (int i = 0; i < 3; ++i) {
            u[i] = U[3 * bd + i];
            w[i] = Om[3 * bd + i];
        }
    }
    for (int i = 0; i < 3; ++i) k[i] = u[i];
    // dB = [w]x B, B row-major with the basis vectors as columns
    const double *Bb = B + 9 * bd;
    for (int r = 0; r < 3; ++r)
        for (int col = 0; col < 3; ++col) {
            const double wx0 = r == 0 ? 0.0 : (r == 1 ? w[2] : -w[1]);
            const double wx1 = r == 1 ? 0.0 : (r == 0 ? -w[2] : w[0]);
            const double wx2 = r == 2 ? 0.0 : (r == 0 ? w[1] : -w[0]);
            k[3 + 3 * r + col] = wx0 * Bb[col] + wx1 * Bb[3 + col] + wx2 * Bb[6 + col];
        }
}

struct DpCoef {
    double v[7];
};

// Y = Y_n + h sum_{j < nk} a_j K_j per non-static body, B by modified Gram-Schmidt.
__global__ void k_dp_combine(int nbodies, const int32_t *__restrict__ kind, double h, DpCoef a,
                             int nk, const double *__restrict__ x0n, const double *__restrict__ Bn,
                             const double *__restrict__ K, double *__restrict__ x0,
                             double *__restrict__ B)
{
    const int bd = blockIdx.x * blockDim.x + threadIdx.x;
    if (bd >= nbodies) return;
    if (kind[bd] == NRS_STATIC) {
        for (int i = 0; i < 3; ++i) x0[3 * bd + i] = x0n[3 * bd + i];
        for (int i = 0; i < 9; ++i) B[9 * bd + i] = Bn[9 * bd + i];
        return;
    }
    double y[12];
    for (int i = 0; i < 3; ++i) y[i] = x0n[3 * bd + i];
    for (int i = 0; i < 9; ++i) y[3 + i] = Bn[9 * bd + i];
    for (int i = 0; i < 12; ++i) {
        double s = 0.0;
        for (int j = 0; j < nk; ++j) s += a.v[j] * K[(int64_t)j * 12 * nbodies + 12 * bd + i];
        y[i] += h * s;
    }
    double *M = y + 3;
    for (int j = 0; j < 3; ++j) {
        for (int i = 0; i < j; ++i) {
            const double dot = M[i] * M[j] + M[3 + i] * M[3 + j] + M[6 + i] * M[6 + j];
            for (int r = 0; r < 3; ++r) M[3 * r + j] -= dot * M[3 * r + i];
        }
        const double nrm = sqrt(M[j] * M[j] + M[3 + j] * M[3 + j] + M[6 + j] * M[6 + j]);
        for (int r = 0; r < 3; ++r) M[3 * r + j] /= nrm;
    }
    for (int i = 0; i < 3; ++i) x0[3 * bd + i] = y[i];
    for (int i = 0; i < 9; ++i) B[9 * bd + i] = M[i];
}

// err[0] = the scaled maximum norm of the error estimate (one CTA; a block
// maximum in a fixed order).
__global__ void k_dp_error(int nbodies, const int32_t *__restrict__ kind, double h, DpCoef e,
                           const double *__restrict__ x0n, const double *__restrict__ Bn,
                           const double *__restrict__ x1, const double *__restrict__ B1,
                           const double *__restrict__ K, double rtol, double atol,
                           double *__restrict__ err)
{
    __shared__ double red[256];
    double m = 0.0;
    for (int idx = threadIdx.x; idx < 12 * nbodies; idx += blockDim.x) {
        const int bd = idx / 12, i = idx % 12;
        if (kind[bd] == NRS_STATIC) continue;
        double s = 0.0;
        for (int j = 0; j < 7; ++j) s += e.v[j] * K[(int64_t)j * 12 * nbodies + idx];
        const double y0 = i < 3 ? x0n[3 * bd + i] : Bn[9 * bd + i - 3];
        const double y1 = i < 3 ? x1[3 * bd + i] : B1[9 * bd + i - 3];
        const double sc = atol + rtol * fmax(fabs(y0), fabs(y1));
        const double r = fabs(h * s) / sc;
        m = (r > m || r != r) ? r : m;
    }
    red[threadIdx.x] = m;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            const double a = red[threadIdx.x], b = red[threadIdx.x + o];
            red[threadIdx.x] = (b > a || b != b) ? b : a;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) err[0] = red[0];
}

}  // namespace

// Dormand-Prince 5(4) tableau (Dormand & Prince 1980): nodes, stage
// coefficients (row i for stage i), fifth-order weights (row 6), and the
// difference between the fifth- and fourth-order weights.
static const double kDpC[7] = {0.0, 1.0 / 5, 3.0 / 10, 4.0 / 5, 8.0 / 9, 1.0, 1.0};
static const double kDpA[7][6] = {
    {0, 0, 0, 0, 0, 0},
    {1.0 / 5, 0, 0, 0, 0, 0},
    {3.0 / 40, 9.0 / 40, 0, 0, 0, 0},
    {44.0 / 45, -56.0 / 15, 32.0 / 9, 0, 0, 0},
    {19372.0 / 6561, -25360.0 / 2187, 64448.0 / 6561, -212.0 / 729, 0, 0},
    {9017.0 / 3168, -355.0 / 33, 46732.0 / 5247, 49.0 / 176, -5103.0 / 18656, 0},
    {35.0 / 384, 0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84}};
static const double kDpB4[7] = {5179.0 / 57600, 0, 7571.0 / 16695, 393.0 / 640,
                                -92097.0 / 339200, 187.0 / 2100, 1.0 / 40};

double dp_node(int stage) { return kDpC[stage]; }

void launch_dp_rates(Ctx &c, int stage, const double *sol)
{
    k_dp_rates<<<(unsigned)ceil_div(c.nbodies, 64), 64, 0, c.stream>>>(
        c.nbodies, c.N, c.d_kind, c.d_free_index, sol, c.d_U, c.d_Om, c.d_B,
        c.d_dp_K + (int64_t)stage * 12 * c.nbodies);
    c.launches += 1;
}

void launch_dp_combine(Ctx &c, int stage, double h)
{
    DpCoef a{};
    for (int j = 0; j < stage; ++j) a.v[j] = kDpA[stage][j];
    k_dp_combine<<<(unsigned)ceil_div(c.nbodies, 64), 64, 0, c.stream>>>(
        c.nbodies, c.d_kind, h, a, stage, c.d_x0_save, c.d_B_save, c.d_dp_K, c.d_x0, c.d_B);
    c.launches += 1;
}

void launch_dp_error(Ctx &c, double h, double rtol, double atol, double *err)
{
    DpCoef e{};
    for (int j = 0; j < 7; ++j) e.v[j] = (j < 6 ? kDpA[6][j] : 0.0) - kDpB4[j];
    k_dp_error<<<1, 256, 0, c.stream>>>(c.nbodies, c.d_kind, h, e, c.d_x0_save, c.d_B_save, c.d_x0,
                                       c.d_B, c.d_dp_K, rtol, atol, err);
    c.launches += 1;
}

}  // namespace nrs
