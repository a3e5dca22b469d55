// mlp.cu -- learned starting guess for the refinement: a point-wise MLP that
// predicts each force point's force density f_m (in its body's frame) from
// local features, trained with Adam on the solutions the method produces.
// The paper has no learned component; the prediction only changes where the
// refinement of Sec. 4 step 3 starts, never what it converges to.
//
// Architecture: x (17) -> W1 x + b1 -> SiLU -> W2 h1 + b2 -> SiLU -> W3 h2 + b3 (3),
// SiLU(z) = z / (1 + e^-z).  Parameter vector (FP32, NRS_MLP_PARAMS entries):
//   W1 [64][17] row-major, b1 [64], W2 [64][64], b2 [64], W3 [3][64], b3 [3].
// Features of force point m of body b (body frame; L, V, F are the scales):
//   0-2   xi_m / L                 3-5   xidot_m / V
//   6     s = (m - n_off[b]) / max(1, N_b - 1)  (position in the body's point order)
//   7     W_m / mean_b(W)          8-10  one-hot body kind (free, prescribed, static)
//   11-13 B^T U / V                14-16 B^T Omega L / V
// with (U, Omega) the previous stage's solution for a free body, the
// prescribed motion for a prescribed body, zero for a static one.
// Target: B^T f_m / F.  Loss: mean over points and components of the squared error.
//
// Every sum over points (weight gradients, loss, scales) has a fixed order
// that depends only on the number of points: results are deterministic.
#include <math.h>

#include "nrs_internal.cuh"

namespace nrs {

constexpr int MI = NRS_MLP_IN, MH = NRS_MLP_HID, MO = NRS_MLP_OUT, MP = NRS_MLP_PARAMS;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + MH * MI, OFF_W2 = OFF_B1 + MH,
              OFF_B2 = OFF_W2 + MH * MH, OFF_W3 = OFF_B2 + MH, OFF_B3 = OFF_W3 + MO * MH;
static_assert(OFF_B3 + MO == MP, "parameter layout");

constexpr int ML_THREADS = 128;   // 4 warps; one warp evaluates one point at a time
constexpr int GR_THREADS = 256;   // gradient kernel: threads per block
constexpr int GR_POINTS = 32;     // points per block (chunk) of the gradient sums
constexpr int RD_THREADS = 256;   // single-block reductions

// SiLU(z) = z * sigmoid(z), rounded the same way in every kernel
__device__ __forceinline__ float sigmoid(float z) { return 1.0f / (1.0f + expf(-z)); }
__device__ __forceinline__ float silu(float z) { return z * sigmoid(z); }

// Parameters in shared memory for the warp-per-point kernels: W1 and W2
// transposed so that lane j reads column j without bank conflicts.
struct SmemNet {
    float w1t[MI][MH];   // w1t[i][j] = W1[j][i]
    float w2t[MH][MH];   // w2t[i][j] = W2[j][i]
    float w2[MH][MH];    // W2 as stored (backward: lane i reads W2[j][i])
    float w3[MO][MH];
    float b1[MH], b2[MH], b3[MO];
};

__device__ __forceinline__ void load_net(SmemNet &n, const float *__restrict__ P)
{
    for (int k = threadIdx.x; k < MH * MI; k += blockDim.x) {
        const int j = k / MI, i = k % MI;
        n.w1t[i][j] = P[OFF_W1 + k];
    }
    for (int k = threadIdx.x; k < MH * MH; k += blockDim.x) {
        const int j = k / MH, i = k % MH;
        const float w = P[OFF_W2 + k];
        n.w2t[i][j] = w;
        n.w2[j][i] = w;
    }
    for (int k = threadIdx.x; k < MO * MH; k += blockDim.x) n.w3[k / MH][k % MH] = P[OFF_W3 + k];
    for (int k = threadIdx.x; k < MH; k += blockDim.x) {
        n.b1[k] = P[OFF_B1 + k];
        n.b2[k] = P[OFF_B2 + k];
    }
    if (threadIdx.x < MO) n.b3[threadIdx.x] = P[OFF_B3 + threadIdx.x];
    __syncthreads();
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Forward pass, one warp per point (lane j owns hidden units j and j + 32).
// Same operations in the same order as the forward half of k_mlp_fwd_bwd.
__global__ void __launch_bounds__(ML_THREADS)
    k_mlp_forward(int64_t npts, const float *__restrict__ P, const float *__restrict__ X,
                  float *__restrict__ Y)
{
    __shared__ SmemNet net;
    __shared__ float sh1[ML_THREADS / 32][MH];
    load_net(net, P);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t stride = (int64_t)gridDim.x * (ML_THREADS / 32);
    for (int64_t p = (int64_t)blockIdx.x * (ML_THREADS / 32) + w; p < npts; p += stride) {
        const float xl = lane < MI ? X[p * MI + lane] : 0.0f;
        float za = net.b1[lane], zb = net.b1[lane + 32];
#pragma unroll
        for (int i = 0; i < MI; ++i) {
            const float xi = __shfl_sync(0xffffffffu, xl, i);
            za = fmaf(net.w1t[i][lane], xi, za);
            zb = fmaf(net.w1t[i][lane + 32], xi, zb);
        }
        sh1[w][lane] = silu(za);
        sh1[w][lane + 32] = silu(zb);
        __syncwarp();
        za = net.b2[lane];
        zb = net.b2[lane + 32];
#pragma unroll 16
        for (int i = 0; i < MH; ++i) {
            const float h = sh1[w][i];
            za = fmaf(net.w2t[i][lane], h, za);
            zb = fmaf(net.w2t[i][lane + 32], h, zb);
        }
        __syncwarp();
        const float ha = silu(za), hb = silu(zb);
#pragma unroll
        for (int o = 0; o < MO; ++o) {
            const float part = warp_sum(fmaf(net.w3[o][lane], ha, net.w3[o][lane + 32] * hb));
            if (lane == 0) Y[p * MO + o] = part + net.b3[o];
        }
    }
}

// Forward and backward pass of the training loss, one warp per point
// (lane j owns hidden units j and j + 32):
//   Z1 = W1 x + b1, H1 = SiLU(Z1), Z2 = W2 H1 + b2, H2 = SiLU(Z2), Y = W3 H2 + b3,
//   dY = 2 (Y - T) / (3 npts),  D2 = (W3^T dY) * SiLU'(Z2),  D1 = (W2^T D2) * SiLU'(Z1),
// with SiLU'(z) = s (1 + z (1 - s)), s = 1 / (1 + e^-z).  Writes H1, H2, DY,
// D1, D2 for the parameter-gradient sums, and Y when it is not NULL.
__global__ void __launch_bounds__(ML_THREADS)
    k_mlp_fwd_bwd(int64_t npts, const float *__restrict__ P, const float *__restrict__ X,
                  const float *__restrict__ T, float *__restrict__ Y, float *__restrict__ H1,
                  float *__restrict__ H2, float *__restrict__ DY, float *__restrict__ D1,
                  float *__restrict__ D2)
{
    __shared__ SmemNet net;
    __shared__ float sv[ML_THREADS / 32][MH];
    load_net(net, P);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const float scale = 2.0f / (float)(3 * npts);
    const int64_t stride = (int64_t)gridDim.x * (ML_THREADS / 32);
    for (int64_t p = (int64_t)blockIdx.x * (ML_THREADS / 32) + w; p < npts; p += stride) {
        const float xl = lane < MI ? X[p * MI + lane] : 0.0f;
        float z1a = net.b1[lane], z1b = net.b1[lane + 32];
#pragma unroll
        for (int i = 0; i < MI; ++i) {
            const float xi = __shfl_sync(0xffffffffu, xl, i);
            z1a = fmaf(net.w1t[i][lane], xi, z1a);
            z1b = fmaf(net.w1t[i][lane + 32], xi, z1b);
        }
        const float s1a = sigmoid(z1a), s1b = sigmoid(z1b);
        const float h1a = z1a * s1a, h1b = z1b * s1b;
        H1[p * MH + lane] = h1a;
        H1[p * MH + lane + 32] = h1b;
        sv[w][lane] = h1a;
        sv[w][lane + 32] = h1b;
        __syncwarp();
        float z2a = net.b2[lane], z2b = net.b2[lane + 32];
#pragma unroll 16
        for (int i = 0; i < MH; ++i) {
            const float h = sv[w][i];
            z2a = fmaf(net.w2t[i][lane], h, z2a);
            z2b = fmaf(net.w2t[i][lane + 32], h, z2b);
        }
        __syncwarp();
        const float s2a = sigmoid(z2a), s2b = sigmoid(z2b);
        const float h2a = z2a * s2a, h2b = z2b * s2b;
        H2[p * MH + lane] = h2a;
        H2[p * MH + lane + 32] = h2b;
        float dy[MO];
#pragma unroll
        for (int o = 0; o < MO; ++o) {
            const float y = warp_sum(fmaf(net.w3[o][lane], h2a, net.w3[o][lane + 32] * h2b)) +
                            net.b3[o];
            if (Y && lane == 0) Y[p * MO + o] = y;
            dy[o] = scale * (y - T[p * MO + o]);
        }
        if (lane < MO) DY[p * MO + lane] = lane == 0 ? dy[0] : (lane == 1 ? dy[1] : dy[2]);
        float ga = 0.0f, gb = 0.0f;
#pragma unroll
        for (int o = 0; o < MO; ++o) {
            ga = fmaf(net.w3[o][lane], dy[o], ga);
            gb = fmaf(net.w3[o][lane + 32], dy[o], gb);
        }
        const float d2a = ga * (s2a * (1.0f + z2a * (1.0f - s2a)));
        const float d2b = gb * (s2b * (1.0f + z2b * (1.0f - s2b)));
        D2[p * MH + lane] = d2a;
        D2[p * MH + lane + 32] = d2b;
        sv[w][lane] = d2a;
        sv[w][lane + 32] = d2b;
        __syncwarp();
        ga = 0.0f;
        gb = 0.0f;
#pragma unroll 16
        for (int j = 0; j < MH; ++j) {
            const float d = sv[w][j];
            ga = fmaf(net.w2[j][lane], d, ga);
            gb = fmaf(net.w2[j][lane + 32], d, gb);
        }
        __syncwarp();
        D1[p * MH + lane] = ga * (s1a * (1.0f + z1a * (1.0f - s1a)));
        D1[p * MH + lane + 32] = gb * (s1b * (1.0f + z1b * (1.0f - s1b)));
    }
}

// Partial parameter gradients of GR_POINTS points (one block), summed in
// point order in FP32 from shared-memory tiles:
//   W1[j][i]: D1[p][j] X[p][i]    b1[j]: D1[p][j]    W2[j][i]: D2[p][j] H1[p][i]
//   b2[j]: D2[p][j]               W3[o][j]: DY[p][o] H2[p][j]    b3[o]: DY[p][o]
__global__ void __launch_bounds__(GR_THREADS)
    k_mlp_grad_part(int64_t npts, const float *__restrict__ X, const float *__restrict__ H1,
                    const float *__restrict__ H2, const float *__restrict__ DY,
                    const float *__restrict__ D1, const float *__restrict__ D2,
                    float *__restrict__ part)
{
    __shared__ float sx[GR_POINTS][MI], sh1[GR_POINTS][MH], sh2[GR_POINTS][MH];
    __shared__ float sd1[GR_POINTS][MH], sd2[GR_POINTS][MH], sdy[GR_POINTS][MO];
    const int64_t p0 = (int64_t)blockIdx.x * GR_POINTS;
    const int np = (int)min((int64_t)GR_POINTS, npts - p0);
    for (int k = threadIdx.x; k < GR_POINTS * MH; k += GR_THREADS) {
        const int q = k / MH, j = k % MH;
        const bool in = q < np;
        const int64_t g = (p0 + q) * MH + j;
        sh1[q][j] = in ? H1[g] : 0.0f;
        sh2[q][j] = in ? H2[g] : 0.0f;
        sd1[q][j] = in ? D1[g] : 0.0f;
        sd2[q][j] = in ? D2[g] : 0.0f;
    }
    for (int k = threadIdx.x; k < GR_POINTS * MI; k += GR_THREADS) {
        const int q = k / MI, i = k % MI;
        sx[q][i] = q < np ? X[(p0 + q) * MI + i] : 0.0f;
    }
    if (threadIdx.x < GR_POINTS * MO) {
        const int q = threadIdx.x / MO, o = threadIdx.x % MO;
        sdy[q][o] = q < np ? DY[(p0 + q) * MO + o] : 0.0f;
    }
    __syncthreads();
    float *out = part + (int64_t)blockIdx.x * MP;
    for (int k = threadIdx.x; k < MP; k += GR_THREADS) {
        float s = 0.0f;
        if (k < OFF_B1) {
            const int j = k / MI, i = k % MI;
            for (int q = 0; q < np; ++q) s = fmaf(sd1[q][j], sx[q][i], s);
        } else if (k < OFF_W2) {
            const int j = k - OFF_B1;
            for (int q = 0; q < np; ++q) s += sd1[q][j];
        } else if (k < OFF_B2) {
            const int j = (k - OFF_W2) / MH, i = (k - OFF_W2) % MH;
            for (int q = 0; q < np; ++q) s = fmaf(sd2[q][j], sh1[q][i], s);
        } else if (k < OFF_W3) {
            const int j = k - OFF_B2;
            for (int q = 0; q < np; ++q) s += sd2[q][j];
        } else if (k < OFF_B3) {
            const int o = (k - OFF_W3) / MH, j = (k - OFF_W3) % MH;
            for (int q = 0; q < np; ++q) s = fmaf(sdy[q][o], sh2[q][j], s);
        } else {
            const int o = k - OFF_B3;
            for (int q = 0; q < np; ++q) s += sdy[q][o];
        }
        out[k] = s;
    }
}

// Adam (Kingma & Ba 2015) for parameter k: beta1 = 0.9, beta2 = 0.999,
// epsilon = 1e-8; bc1 = 1 - beta1^t and bc2 = 1 - beta2^t are computed on the
// host in FP64.
__device__ __forceinline__ void adam_update(float *__restrict__ P, float *__restrict__ Mo,
                                            float *__restrict__ Ve, int k, float g, float lr,
                                            float bc1, float bc2)
{
    const float m = fmaf(0.9f, Mo[k], 0.1f * g);
    const float v = fmaf(0.999f, Ve[k], 0.001f * (g * g));
    Mo[k] = m;
    Ve[k] = v;
    P[k] -= lr * (m / bc1) / (sqrtf(v / bc2) + 1e-8f);
}

// G[k] = sum over chunks, in chunk order (FP64 accumulation); with lr > 0
// also one Adam step of the parameters.
__global__ void k_mlp_grad_finish(int chunks, const float *__restrict__ part, float *__restrict__ G,
                                  float *__restrict__ P, float *__restrict__ Mo,
                                  float *__restrict__ Ve, float lr, float bc1, float bc2)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= MP) return;
    double s = 0.0;
    for (int c = 0; c < chunks; ++c) s += (double)part[(int64_t)c * MP + k];
    const float g = (float)s;
    if (G) G[k] = g;
    if (lr > 0.0f) adam_update(P, Mo, Ve, k, g, lr, bc1, bc2);
}

__device__ double block_sum_fixed(double v)
{
    __shared__ double red[RD_THREADS];
    red[threadIdx.x] = v;
    __syncthreads();
    for (int w = RD_THREADS / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    const double r = red[0];
    __syncthreads();
    return r;
}

__device__ double block_max_fixed(double v)
{
    __shared__ double red[RD_THREADS];
    red[threadIdx.x] = v;
    __syncthreads();
    for (int w = RD_THREADS / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    const double r = red[0];
    __syncthreads();
    return r;
}

// loss[0] = mean of (Y - T)^2 and loss[1] = mean of T^2 over the npts * 3
// entries (one block).
__global__ void __launch_bounds__(RD_THREADS)
    k_mlp_loss(int64_t npts, const float *__restrict__ Y, const float *__restrict__ T,
               double *__restrict__ loss)
{
    double s = 0.0, t2 = 0.0;
    for (int64_t i = threadIdx.x; i < npts * MO; i += RD_THREADS) {
        const double d = (double)Y[i] - (double)T[i];
        s += d * d;
        t2 += (double)T[i] * (double)T[i];
    }
    s = block_sum_fixed(s);
    t2 = block_sum_fixed(t2);
    if (threadIdx.x == 0) {
        loss[0] = s / (double)(npts * MO);
        loss[1] = t2 / (double)(npts * MO);
    }
}

// One Adam step with a given gradient G.
__global__ void k_mlp_adam(float *__restrict__ P, float *__restrict__ Mo, float *__restrict__ Ve,
                           const float *__restrict__ G, float lr, float bc1, float bc2)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < MP) adam_update(P, Mo, Ve, k, G[k], lr, bc1, bc2);
}

// Scales from one solved stage: L = max |xi_m|, V = max |b_m| over the force
// rows of the right-hand side, F = sqrt(mean |f_m|^2); a zero scale becomes 1.
__global__ void __launch_bounds__(RD_THREADS)
    k_mlp_scales(int64_t N, const D4 *__restrict__ xi, const double *__restrict__ b,
                 const double *__restrict__ sol, double *__restrict__ out)
{
    double lmax = 0.0, vmax = 0.0, fsum = 0.0;
    for (int64_t m = threadIdx.x; m < N; m += RD_THREADS) {
        const D4 p = xi[m];
        lmax = fmax(lmax, sqrt(p.x * p.x + p.y * p.y + p.z * p.z));
        const double *bm = b + 3 * m, *fm = sol + 3 * m;
        vmax = fmax(vmax, sqrt(bm[0] * bm[0] + bm[1] * bm[1] + bm[2] * bm[2]));
        fsum += fm[0] * fm[0] + fm[1] * fm[1] + fm[2] * fm[2];
    }
    lmax = block_max_fixed(lmax);
    vmax = block_max_fixed(vmax);
    fsum = block_sum_fixed(fsum);
    if (threadIdx.x == 0) {
        const double F = sqrt(fsum / (double)N);
        out[0] = lmax > 0.0 ? lmax : 1.0;
        out[1] = vmax > 0.0 ? vmax : 1.0;
        out[2] = F > 0.0 ? F : 1.0;
    }
}

// Per-body mean of W_n (one thread per body).
__global__ void k_mlp_wmean(int nbodies, const int64_t *__restrict__ n_off,
                            const double *__restrict__ W, double *__restrict__ Wmean)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbodies) return;
    double s = 0.0;
    for (int64_t m = n_off[b]; m < n_off[b + 1]; ++m) s += W[m];
    const int64_t cnt = n_off[b + 1] - n_off[b];
    Wmean[b] = cnt > 0 ? s / (double)cnt : 0.0;
}

// Features of every force point and, when T is not NULL, the body-frame
// targets from the solution sol = [f (3N); (U, Omega) (6F)].
// B row-major per body with the basis vectors as columns: B^T v has
// components sum_r B[r][k] v_r.
__global__ void k_mlp_features(int64_t N, const D4 *__restrict__ xi, const D4 *__restrict__ xidot,
                               const double *__restrict__ W, const double *__restrict__ Wmean,
                               const int64_t *__restrict__ n_off, const int32_t *__restrict__ body_x,
                               const int32_t *__restrict__ kind,
                               const int32_t *__restrict__ free_index, const double *__restrict__ B,
                               const double *__restrict__ Upres, const double *__restrict__ Ompres,
                               const double *__restrict__ vprev, const double *__restrict__ sol,
                               const double *__restrict__ scales, float *__restrict__ X,
                               float *__restrict__ T)
{
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= N) return;
    const double L = scales[0], V = scales[1], F = scales[2];
    const int b = body_x[m];
    const double *Bb = B + 9 * b;
    const D4 p = xi[m], v = xidot[m];
    float *x = X + m * MI;
    x[0] = (float)(p.x / L);
    x[1] = (float)(p.y / L);
    x[2] = (float)(p.z / L);
    x[3] = (float)(v.x / V);
    x[4] = (float)(v.y / V);
    x[5] = (float)(v.z / V);
    const int64_t nb = n_off[b + 1] - n_off[b];
    x[6] = (float)((double)(m - n_off[b]) / (double)(nb > 1 ? nb - 1 : 1));
    x[7] = (float)(Wmean[b] > 0.0 ? W[m] / Wmean[b] : 0.0);
    const int kb = kind[b];
    x[8] = kb == NRS_FREE ? 1.0f : 0.0f;
    x[9] = kb == NRS_PRESCRIBED ? 1.0f : 0.0f;
    x[10] = kb == NRS_STATIC ? 1.0f : 0.0f;
    double U[3] = {0.0, 0.0, 0.0}, Om[3] = {0.0, 0.0, 0.0};
    if (kb == NRS_PRESCRIBED) {
        for (int k = 0; k < 3; ++k) {
            U[k] = Upres[3 * b + k];
            Om[k] = Ompres[3 * b + k];
        }
    } else if (kb == NRS_FREE && vprev) {
        const int f = free_index[b];
        for (int k = 0; k < 3; ++k) {
            U[k] = vprev[6 * f + k];
            Om[k] = vprev[6 * f + 3 + k];
        }
    }
    for (int k = 0; k < 3; ++k) {
        const double ub = Bb[k] * U[0] + Bb[3 + k] * U[1] + Bb[6 + k] * U[2];
        const double ob = Bb[k] * Om[0] + Bb[3 + k] * Om[1] + Bb[6 + k] * Om[2];
        x[11 + k] = (float)(ub / V);
        x[14 + k] = (float)(ob * L / V);
    }
    if (T) {
        const double *fm = sol + 3 * m;
        for (int k = 0; k < 3; ++k)
            T[m * MO + k] =
                (float)((Bb[k] * fm[0] + Bb[3 + k] * fm[1] + Bb[6 + k] * fm[2]) / F);
    }
}

// Start vector from a prediction Y: f_m = F B y_m; (U, Omega) of the free
// bodies from vprev (zero when NULL).  bad[0] is set if any entry is not finite.
__global__ void k_mlp_to_start(int64_t N, int64_t nfree, const float *__restrict__ Y,
                               const int32_t *__restrict__ body_x, const double *__restrict__ B,
                               const double *__restrict__ vprev, const double *__restrict__ scales,
                               double *__restrict__ x0, int32_t *__restrict__ bad)
{
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const double F = scales[2];
    if (m < N) {
        const double *Bb = B + 9 * body_x[m];
        const double y0 = Y[m * MO], y1 = Y[m * MO + 1], y2 = Y[m * MO + 2];
        bool ok = true;
        for (int r = 0; r < 3; ++r) {
            const double f = F * (Bb[3 * r] * y0 + Bb[3 * r + 1] * y1 + Bb[3 * r + 2] * y2);
            ok = ok && isfinite(f);
            x0[3 * m + r] = f;
        }
        if (!ok) atomicOr(bad, 1);
    } else if (m < N + 6 * nfree) {
        const int64_t k = m - N;
        const double v = vprev ? vprev[k] : 0.0;
        if (!isfinite(v)) atomicOr(bad, 1);
        x0[3 * N + k] = v;
    }
}

// x0 = xp if its residual norm is the smaller one (and it is finite), else xc.
// used[0] records the choice; used[1] is the non-finite flag of k_mlp_to_start.
__global__ void k_pick_start(int64_t n, const double *__restrict__ xp, const double *__restrict__ xc,
                             const double *__restrict__ norms, double *__restrict__ x0,
                             int32_t *__restrict__ used)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool pred = used[1] == 0 && norms[0] < norms[1];
    if (i < n) x0[i] = pred ? xp[i] : xc[i];
    if (i == 0) used[0] = pred ? 1 : 0;
}

// ---- host side ---------------------------------------------------------------

int mlp_grad_chunks(int64_t npts) { return (int)ceil_div(npts, GR_POINTS); }

static unsigned warp_grid(const Ctx &c, int64_t npts)
{
    // one warp per point, at most one block of 4 warps per SM (each block
    // stages all parameters in shared memory first)
    return (unsigned)std::max<int64_t>(
        1, std::min<int64_t>(ceil_div(npts, ML_THREADS / 32), (int64_t)c.num_sms));
}

static void bias_corrections(int t, float *bc1, float *bc2)
{
    *bc1 = (float)(1.0 - pow(0.9, (double)t));
    *bc2 = (float)(1.0 - pow(0.999, (double)t));
}

void mlp_eval(Ctx &c, const float *X, int64_t npts, const float *T, float *Y, float *G,
              double *loss_dev)
{
    if (!T || !G) {
        k_mlp_forward<<<warp_grid(c, npts), ML_THREADS, 0, c.stream>>>(npts, c.d_mlp_params, X, Y);
        c.launches += 1;
        if (T && loss_dev) {
            k_mlp_loss<<<1, RD_THREADS, 0, c.stream>>>(npts, Y, T, loss_dev);
            c.launches += 1;
        }
    }
    if (T && G) mlp_train_step(c, X, npts, T, G, 0.0f, Y);
    if (T && G && loss_dev) {
        k_mlp_loss<<<1, RD_THREADS, 0, c.stream>>>(npts, Y, T, loss_dev);
        c.launches += 1;
    }
}

void mlp_train_step(Ctx &c, const float *X, int64_t npts, const float *T, float *G, float lr,
                    float *Y)
{
    k_mlp_fwd_bwd<<<warp_grid(c, npts), ML_THREADS, 0, c.stream>>>(
        npts, c.d_mlp_params, X, T, Y, c.d_mlp_z1, c.d_mlp_z2, c.d_mlp_dy, c.d_mlp_d1, c.d_mlp_d2);
    const int chunks = mlp_grad_chunks(npts);
    k_mlp_grad_part<<<(unsigned)chunks, GR_THREADS, 0, c.stream>>>(
        npts, X, c.d_mlp_z1, c.d_mlp_z2, c.d_mlp_dy, c.d_mlp_d1, c.d_mlp_d2, c.d_mlp_part);
    float bc1 = 1.0f, bc2 = 1.0f;
    if (lr > 0.0f) {
        c.mlp_t += 1;
        bias_corrections(c.mlp_t, &bc1, &bc2);
    }
    k_mlp_grad_finish<<<(unsigned)ceil_div(MP, 256), 256, 0, c.stream>>>(
        chunks, c.d_mlp_part, G, c.d_mlp_params, c.d_mlp_m, c.d_mlp_v, lr, bc1, bc2);
    c.launches += 3;
}

void mlp_adam(Ctx &c, const float *G, float lr)
{
    c.mlp_t += 1;
    float bc1, bc2;
    bias_corrections(c.mlp_t, &bc1, &bc2);
    k_mlp_adam<<<(unsigned)ceil_div(MP, 256), 256, 0, c.stream>>>(c.d_mlp_params, c.d_mlp_m,
                                                                  c.d_mlp_v, G, lr, bc1, bc2);
    c.launches += 1;
}

void mlp_scales(Ctx &c, const D4 *xi, const double *b, const double *sol, double *out)
{
    k_mlp_scales<<<1, RD_THREADS, 0, c.stream>>>(c.N, xi, b, sol, out);
    c.launches += 1;
}

void mlp_features(Ctx &c, const D4 *xi, const D4 *xidot, const double *vprev, const double *sol,
                  float *X, float *T)
{
    k_mlp_wmean<<<(unsigned)ceil_div(c.nbodies, 64), 64, 0, c.stream>>>(c.nbodies, c.d_n_off, c.d_W,
                                                                         c.d_mlp_wmean);
    k_mlp_features<<<(unsigned)ceil_div(c.N, 128), 128, 0, c.stream>>>(
        c.N, xi, xidot, c.d_W, c.d_mlp_wmean, c.d_n_off, c.d_body_x, c.d_kind, c.d_free_index,
        c.d_B, c.d_U, c.d_Om, vprev, sol, c.d_mlp_scal, X, T);
    c.launches += 2;
}

void mlp_start(Ctx &c, const float *Y, const double *vprev, double *x0)
{
    cudaMemsetAsync(c.d_mlp_used, 0, 2 * sizeof(int32_t), c.stream);
    k_mlp_to_start<<<(unsigned)ceil_div(c.N + 6 * c.F, 128), 128, 0, c.stream>>>(
        c.N, c.F, Y, c.d_body_x, c.d_B, vprev, c.d_mlp_scal, x0, c.d_mlp_used + 1);
    c.launches += 1;
}

void pick_start(Ctx &c, const double *xp, const double *xc, const double *norms, double *x0)
{
    k_pick_start<<<(unsigned)ceil_div(c.n, 256), 256, 0, c.stream>>>(c.n, xp, xc, norms, x0,
                                                                       c.d_mlp_used);
    c.launches += 1;
}

}  // namespace nrs
