// nrs_internal.cuh -- shared declarations of the libnrs CUDA sources.
//
// Layout conventions (see include/nrs.h): points are rows of 4 doubles,
// matrices column-major with leading dimension lda, unknown 3m+j for force
// point m, then 6 per free body.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/nrs.h"

namespace nrs {

struct __align__(32) D4 {
    double x, y, z, w;
};

// Device status word bits (ORed by kernels, read by the host after a sync).
enum : int32_t {
    ST_SINGULAR = 1,
    ST_NOCONV = 2,
    ST_NONFINITE = 4,
    ST_TIMEOUT = 8,
};

constexpr double kPi = 3.14159265358979323846;

// tile of the FP64 assembly: collocation points x segments
constexpr int64_t kAssembleTileM = 128, kAssembleTileN = 16;

// Upper bound on spins of any device-side wait (each spin sleeps ~100 ns):
// a wait that runs out sets ST_TIMEOUT and returns instead of hanging.
constexpr long long kSpinLimit = 1LL << 24;

// Nearest-neighbour block task: quadrature points [q0, q1) of body b.
struct NNTask {
    int32_t body, q0, q1, pad;
};
// A nearest-neighbour task (one block of k_nearest) covers NN_QPB quadrature
// points of one body, with NN_SPLIT threads per point.
constexpr int NN_QPB = 128;
constexpr int NN_SPLIT = 4;
constexpr int NN_THREADS = NN_QPB * NN_SPLIT;

struct Ctx;

// Phases timed with CUDA events when timing is enabled (nrs_set_timing).
enum Phase {
    PH_KINEMATICS = NRS_PH_KINEMATICS,
    PH_NEAREST = NRS_PH_NEAREST,
    PH_SEGMENTS = NRS_PH_SEGMENTS,
    PH_ASSEMBLE = NRS_PH_ASSEMBLE,
    PH_BORDER = NRS_PH_BORDER,
    PH_CONVERT = NRS_PH_CONVERT,
    PH_LU_PANEL = NRS_PH_LU_PANEL,
    PH_LU_UPDATE = NRS_PH_LU_UPDATE,
    PH_TRSV = NRS_PH_TRSV,
    PH_GEMV = NRS_PH_GEMV,
    PH_KRYLOV = NRS_PH_KRYLOV,
    PH_UPDATE = NRS_PH_UPDATE,
    PH_LU_DIAG = NRS_PH_LU_DIAG,
    PH_ASSEMBLE32 = NRS_PH_ASSEMBLE32,
    NPH = NRS_NPHASE
};

// ---- geometry kernels (geometry.cu) -------------------------------------
void launch_kinematics(Ctx &c, const D4 *xi, const D4 *Xiw, const D4 *xidot, D4 *x, D4 *Xw,
                       double *b);
void launch_nearest(Ctx &c, const D4 *x, const D4 *Xw, int32_t *nn, bool only_deforming);
void launch_segments(Ctx &c, const int32_t *nn, int32_t *seg_ptr, int32_t *perm);
void launch_gather(Ctx &c, const D4 *Xw_lab, const int32_t *seg_ptr, const int32_t *perm);
void launch_border(Ctx &c, const D4 *x_lab, double *A64, float *A32, int64_t lda);
void launch_rk2(Ctx &c, int stage, double dt, const double *sol);

// ---- assembly (assemble.cu) ----------------------------------------------
// from_state: x_lab and the quadrature points come from the context's state
// (nrs_step, the Dormand-Prince stages), so the blocks among static rigid
// bodies may be kept from the previous assembly of that matrix
void launch_assemble(Ctx &c, const D4 *x_lab, double *A64, float *A32, int64_t lda,
                     cudaStream_t s = nullptr, bool from_state = false);
void launch_assemble32(Ctx &c, const D4 *x_lab, float *A32, int64_t lda);
// make c.stream wait for the FP64 assembly running on the side stream, if any
void join_assembly(Ctx &c);

// ---- velocity at field points and tracers (velocity.cu) --------------------
int velocity_splits(const Ctx &c, int64_t P);
void launch_velocity(Ctx &c, const D4 *Xw, const D4 *xp, int64_t P, const double *f, D4 *u,
                     double *part, cudaStream_t s);
void launch_tracer_update(Ctx &c, int stage, double dt, cudaStream_t s);

// ---- Dormand-Prince 5(4) stepping (dp.cu) ----------------------------------
double dp_node(int stage);
void launch_dp_rates(Ctx &c, int stage, const double *sol);
void launch_dp_combine(Ctx &c, int stage, double h);
void launch_dp_error(Ctx &c, double h, double rtol, double atol, double *err);

// ---- factorisation (lu.cu) -------------------------------------------------
int run_lu_fp64(Ctx &c, double *A, int64_t lda);
int run_gj_fp32(Ctx &c, float *M, int64_t lda, int prec);

// two-level Gauss-Jordan with rank-256 tensor-core updates (gj2.cu), used by
// run_gj_fp32 for TF32 from n = GJ2_MIN_N on
constexpr int64_t GJ2_MIN_N = 8192;
bool gj2_supported(const Ctx &c);
size_t gj2_panel_floats(int64_t n);
size_t gj2_workspace_bytes(int64_t n);
int run_gj2_fp32(Ctx &c, float *M, int64_t lda, bool f16);
size_t gj_diag_smem();
void gj_diag_prepare();
void k_gj_diag_launch(Ctx &c, int64_t n, const float *M, int64_t lda, int64_t k0, float *Dinv,
                      size_t smem, cudaStream_t s = nullptr);

bool tc_available();
bool launch_tc_rank64(Ctx &c, float *M, int64_t lda, int64_t n, const float *Cb, const float *Rt,
                      int prec, int64_t skip0, int64_t kblk, const float *Cb_lo = nullptr,
                      const float *Rt_lo = nullptr);
void launch_simt_rank64(Ctx &c, float *M, int64_t lda, int64_t n, const float *Cb, const float *Rt);

// ---- solve (solve.cu) ------------------------------------------------------
nrs_status run_gmres_ir(Ctx &c, const double *b, double *x, const double *x0,
                        nrs_solve_report *rep, int *inner_out = nullptr);
// The whole refinement as one cooperative launch (gmres_persistent.cu), for
// explicit-inverse factors and restart lengths up to 64.
bool pg_supported(const Ctx &c);
size_t pg_dpart_doubles(int max_inner);
int pg_max_coresident(const Ctx &c);  // CTAs of the solve kernel that fit on the device at once
cudaError_t launch_gmres_persistent(Ctx &c, const double *b, double *x, bool cold, double *stats);
// out3[0..2] (device) = ||b - A x||_inf, ||A||_inf, ||b||_inf
void enqueue_backward_error(Ctx &c, const double *b, const double *x, double *out3);
// r = b - A x with the FP64 matrix, in the context's residual precision
void enqueue_residual(Ctx &c, const double *x, const double *b, double *r);
// One RK2 step enqueued with no host synchronisation (api.cu); valid when
// graph_capable(c).  stats: 8 doubles per stage (outer, inner, converged,
// ||d||, ||x||, then with berr ||b - A x||, ||A||, ||b||).
bool graph_capable(const Ctx &c);
nrs_status enqueue_step(Ctx *c, const nrs_shapes *s0, const nrs_shapes *sh, double dt,
                        double *stats, bool berr);
// x0 = whichever of xp and the cold start xc = M^{-1} b has the smaller
// ||b - A x||_inf (norms[0], norms[1]); c.d_mlp_used[0] records the choice.
cudaError_t choose_start(Ctx &c, const double *b, const double *xp, double *xc, double *x0,
                         double *norms);

// ---- learned starting guess (mlp.cu) ---------------------------------------
void mlp_eval(Ctx &c, const float *X, int64_t npts, const float *T, float *Y, float *G,
              double *loss_dev);
void mlp_adam(Ctx &c, const float *G, float lr);
// one training iteration: forward, backward, gradient (into G if not NULL)
// and, for lr > 0, an Adam step
void mlp_train_step(Ctx &c, const float *X, int64_t npts, const float *T, float *G, float lr,
                    float *Y = nullptr);
void mlp_scales(Ctx &c, const D4 *xi, const double *b, const double *sol, double *out);
void mlp_features(Ctx &c, const D4 *xi, const D4 *xidot, const double *vprev, const double *sol,
                  float *X, float *T);
void mlp_start(Ctx &c, const float *Y, const double *vprev, double *x0);
void pick_start(Ctx &c, const double *xp, const double *xc, const double *norms, double *x0);
int mlp_grad_chunks(int64_t npts);

struct Ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t stream2 = nullptr;              // lookahead stream of the factorisation
    cudaStream_t stream3 = nullptr;              // FP64 assembly overlapping the factorisation
    cudaEvent_t ev_asm = nullptr, ev_asm_done = nullptr;
    bool asm_pending = false;                    // stream3 holds an FP64 assembly not yet joined
    int lo_eval = 0;  // FP32 copy for the factor: 0 evaluated in FP32 (overlapped), 1 rounded FP64
    int asm_side_ctas = 3;  // CTAs per SM of the FP64 assembly beside the factorisation
    cudaEvent_t ev_upd = nullptr, ev_diag = nullptr;
    cudaStream_t stream4 = nullptr;              // finish step of the factorisation
    cudaEvent_t ev_fin_ready = nullptr, ev_fin[2] = {nullptr, nullptr};
    int num_sms = 0;
    std::string err;

    // problem
    int nbodies = 0;
    int64_t N = 0, Q = 0, F = 0, n = 0, lda = 0;
    std::vector<int64_t> n_off, q_off;
    std::vector<int32_t> kind, rigid, free_index;
    double eps = 0, mu = 0;
    int nn_global = 0, factor_prec = NRS_FP32, nb = 64;
    double tol = 1e-12;
    double tol_in = 1e-4;      // GMRES tolerance of each refinement step (preconditioned residual)
    int max_outer = 20, max_inner = 30;

    // device body tables
    int32_t *d_body_x = nullptr, *d_body_X = nullptr, *d_kind = nullptr, *d_free_index = nullptr;
    int64_t *d_n_off = nullptr, *d_q_off = nullptr;
    double *d_U = nullptr, *d_Om = nullptr, *d_ext = nullptr;
    double *d_x0 = nullptr, *d_B = nullptr, *d_x0_save = nullptr, *d_B_save = nullptr;
    NNTask *d_tasks_all = nullptr, *d_tasks_deform = nullptr;
    int n_tasks_all = 0, n_tasks_deform = 0;
    bool nn_valid = false;

    // clouds and right-hand side (lab frame)
    D4 *d_x = nullptr, *d_Xw = nullptr;
    double *d_b = nullptr, *d_sol = nullptr;

    // passive tracers carried by the flow (nrs_set_tracers), and the workspace
    // of nrs_velocity
    int64_t n_tracers = 0;
    bool kin_valid = false;    // d_Xw holds the lab-frame quadrature points of the last stage
    bool map_built = false;    // d_nn holds a map from nrs_nearest_build
    D4 *d_tr = nullptr, *d_tr_save = nullptr, *d_tr_u = nullptr;
    double *d_tr_part = nullptr;
    double *d_vel_part = nullptr;
    size_t vel_part_doubles = 0;

    // adaptive Dormand-Prince integration (nrs_dp_*): the accepted state Y_n
    // lives in d_x0_save / d_B_save, the stage rates K in d_dp_K [7][nbodies][12]
    bool dp_active = false;
    int dp_stage = 0, dp_accepted = 0, dp_rejected = 0, dp_last_accepted = 0, dp_done = 0;
    double dp_t = 0, dp_t_end = 0, dp_h = 0, dp_rtol = 0, dp_atol = 0, dp_hmin = 0, dp_hmax = 0;
    double dp_err = 0;
    double *d_dp_K = nullptr, *d_dp_err = nullptr;

    // nearest neighbours and segments
    int32_t *d_nn = nullptr, *d_seg_ptr = nullptr, *d_perm = nullptr, *d_cursor = nullptr;
    D4 *d_Xs = nullptr;        // lab-frame quadrature points in segment order
    float4 *d_Xsh = nullptr, *d_Xsl = nullptr;  // the same as float pairs (FP32 assembly)
    float4 *d_xh = nullptr, *d_xl = nullptr;    // force points as float pairs
    double *d_W = nullptr;     // W_n
    double *d_R = nullptr;     // R_n (N x 3)
    bool seg_valid = false;

    // matrices
    double *d_A64 = nullptr;   // FP64 system (residual)
    // 128-point collocation blocks and 16-segment blocks made only of static
    // rigid bodies' points: their A_s entries never change (k_assemble64 keeps them)
    uint8_t *d_mblk_keep = nullptr, *d_nblk_keep = nullptr;
    bool have_static = false, static_cache_valid = false;
    float *d_A32 = nullptr;    // FP32 copy, factored in place for the FP32/TF32/BF16 paths
    double *d_LU64 = nullptr;  // FP64 factor (plain path)
    int32_t *d_rowperm = nullptr;  // row order after pivoting: position i holds original row
    int32_t *d_lperm = nullptr;    // row exchange of the current diagonal block
    bool a32_fresh = false;        // d_A32 holds the last assembly (not yet factored)
    float *d_gj_dinv = nullptr;    // Gauss-Jordan workspaces: D^{-1} (64 x 64)
    float *d_gj_rt = nullptr;      //   scaled block row, transposed (2 buffers of n x 64, then their TF32 lo parts)
    float *d_gj_cb = nullptr;      //   block column (2 buffers of n x 64, then their TF32 lo parts)
    float *d_gj_stage = nullptr;   //   two finished 64 x 64 tiles (2 buffers)
    float *d_gj2 = nullptr;        //   two-level factorisation: operands (gj2_workspace_bytes)
    float *d_gj2_r = nullptr;      //   its inner scaled block row (64 x 256)
    int32_t *d_gj_sync = nullptr;  //   counters of the fused factorisation (4)
    bool gj_fused = false;         //   use the fused (one-launch) factorisation when possible
    int gj_schedule = 0;           //   nrs_problem_desc.factor_schedule
    bool gj_force_one_level = false;  // the next factorisation: one level whatever the schedule
    bool last_factor_two_level = false;  // the last factorisation was the two-level one
    int32_t *d_info = nullptr;
    int factored_prec = -1;
    bool assembled = false;
    // factor reuse across stages (nrs_step)
    int reuse_factor = 0, reuse_max_inner = 8, reuse_max_stages = 16, warm_start = 0;
    int stages_since_factor = 0, last_inner = 0;
    bool have_sol = false;
    int64_t factorizations = 0;
    int64_t retries = 0;       // stages solved again after a non-converged refinement (nrs_step)
    int64_t solves = 0, outer_total = 0, inner_total = 0;  // solves finished on the host side
    int64_t res_exact_total = 0, res_work_total = 0;  // their residuals: exact, working precision

    // learned starting guess (mlp.cu); allocated by the first nrs_mlp_* call
    bool mlp_alloc = false, mlp_params_set = false, mlp_scales_set = false;
    float *d_mlp_params = nullptr, *d_mlp_m = nullptr, *d_mlp_v = nullptr, *d_mlp_g = nullptr;
    float *d_mlp_x = nullptr, *d_mlp_t = nullptr, *d_mlp_y = nullptr;   // features, targets, output
    float *d_mlp_z1 = nullptr, *d_mlp_z2 = nullptr;                      // pre-activations
    float *d_mlp_dy = nullptr, *d_mlp_d1 = nullptr, *d_mlp_d2 = nullptr; // back-propagated terms
    float *d_mlp_part = nullptr;    // per-chunk partial gradients
    double *d_mlp_wmean = nullptr;  // mean W_n per body
    double *d_mlp_scal = nullptr;   // [0..2] scales L, V, F; [3..4] residual norms;
                                    // [5] loss, [6] mean square of the targets
    double *d_mlp_xp = nullptr, *d_mlp_xc = nullptr, *d_mlp_x0 = nullptr;  // start vectors
    int32_t *d_mlp_used = nullptr;  // [0] prediction chosen, [1] prediction not finite
    int32_t *h_mlp_used = nullptr;  // pinned host copy of d_mlp_used
    double *h_mlp_loss = nullptr;   // pinned host copy of the loss and mean square target
    int mlp_t = 0, mlp_train_iters = 0, mlp_predict = 0, mlp_backoff = 0;
    float mlp_lr = 1e-3f;
    double cold_inner_sum = 0.0;
    int64_t cold_inner_cnt = 0;

    // solve workspaces
    int solve_mode = 0;        // 0: persistent device loop where supported; 1: host-driven loop
    double *d_dpart = nullptr; // reduction partials of the persistent solve
    int32_t *d_bar = nullptr;  // its grid barrier
    double *d_pg_stats = nullptr;  // its outcome: outer, inner, converged, ||d||, ||x||
    int pg_grid = 0;           // its CTA count (0 = from occupancy)
    bool pg_shared = false;    // solves share the SMs with other problems' (a batch)

    // CUDA-graph replay of nrs_step (graph mode)
    struct GraphKey {
        const void *p[6];
        double dt;
        bool berr;
        bool operator==(const GraphKey &o) const
        {
            for (int i = 0; i < 6; ++i)
                if (p[i] != o.p[i]) return false;
            return dt == o.dt && berr == o.berr;
        }
    };
    int graph_mode = 0;
    cudaStream_t gstream = nullptr;     // capture stream (the legacy stream cannot be captured)
    cudaGraphExec_t gexec = nullptr;
    GraphKey gkey{};
    int64_t graph_launches = 0;         // kernels in the recorded step
    int64_t graph_captures = 0;
    double *d_step_stats = nullptr;     // 16 doubles: per stage outcome of the device solve
    double *d_r = nullptr, *d_xk = nullptr, *d_w = nullptr, *d_V = nullptr, *d_H = nullptr;
    double *d_gv = nullptr;    // Givens state: cs[m], sn[m], g[m+1], y[m]
    double *d_scal = nullptr;  // scalars (norms, flags as doubles)
    double *d_part = nullptr;  // partial sums of matrix-vector products
    double *d_part32 = nullptr;  // partial sums of the FP32 products of the persistent solve
    unsigned long long *d_part_fx = nullptr; // the residual's exact partial sums [splits][3][n]
    int arnoldi_df = 0;            // GMRES products with the float-pair copy of A (desc.arnoldi)
    float2 *d_Adf = nullptr;       //   that copy: (hi, lo) per entry, A64's layout
    float2 *d_vf2 = nullptr;       //   the raw Krylov vector as float pairs
    float2 *d_vf = nullptr;      // the preconditioner product's input vector as float pairs
    int residual_dd = 1;       // refinement residual b - A x: 1 double-double, 0 FP64
    int splits64 = 1, splits32 = 1;  // column splits of the FP64 / FP32 matrix-vector products
    float *d_t32 = nullptr;    // FP32 work vector for the triangular solves
    double *d_t64 = nullptr;   // FP64 work vector for the triangular solves
    int32_t *d_flags = nullptr;
    int32_t *d_status = nullptr;
    int32_t *h_pinned = nullptr;  // pinned host mirror of small status values
    int trsv_epoch = 0;
    int trsv_grid = 0;

    // timing (CUDA events on `stream`) and the count of kernels launched
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    struct Span {
        int ph;
        cudaEvent_t a, b;
    };
    std::vector<Span> spans;
    cudaEvent_t open_ev[NPH] = {};
    int64_t launches = 0;

    cudaEvent_t next_event()
    {
        if (ev_used == ev_pool.size()) {
            cudaEvent_t e = nullptr;
            cudaEventCreate(&e);
            ev_pool.push_back(e);
        }
        return ev_pool[ev_used++];
    }
    void tbeg(int ph, cudaStream_t s = nullptr)
    {
        if (!timing) return;
        open_ev[ph] = next_event();
        cudaEventRecord(open_ev[ph], s ? s : stream);
    }
    void tend(int ph, cudaStream_t s = nullptr)
    {
        if (!timing || !open_ev[ph]) return;
        cudaEvent_t e = next_event();
        cudaEventRecord(e, s ? s : stream);
        spans.push_back(Span{ph, open_ev[ph], e});
        open_ev[ph] = nullptr;
    }
};

__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// ---- error-free sum --------------------------------------------------------
// Knuth's TwoSum: s + e = a + b exactly.  Every step is an explicitly rounded
// intrinsic, so the compiler cannot fuse or reorder.
__device__ __forceinline__ void dd_two_sum(double a, double b, double &s, double &e)
{
    s = __dadd_rn(a, b);
    const double bb = __dsub_rn(s, a);
    e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
}

// ---- exact fixed-point sums of FP64 products (the refinement's residual) ----
// The residual b - A x is needed to about u^2 of |A| |x| (the extended
// residual precision of three-precision GMRES-IR).  Double-double sums cost 7
// FP64 operations per matrix entry, and GB300 issues FP64 at about two lanes
// per SM per clock, so they bound the product far above its memory time.
// Here each product p = A_ij x_j is rounded in FP64 (one multiply), its
// rounding error e = A_ij x_j - p taken exactly by one fused multiply-add, and
// the errors summed in FP64 (one add): 3 FP64 operations.  The rounded
// products themselves are added EXACTLY on the integer pipe to a 192-bit
// two's-complement integer S standing for S 2^L.  The anchor L comes from a
// bound on every partial sum, |sum_j A_ij x_j| <= ||A||_inf ||x||_inf < 2^E:
// with L = E - 189 the sums never overflow (|S| < 2^191), and a product loses
// less than 2^L (about 2^-187 ||A|| ||x||) when its bits below 2^L are
// dropped.  Integer addition is associative, so splitting the sum over
// threads, column groups and column splits changes nothing: the product's
// integer part is exact and deterministic whatever the order.  A non-finite
// product makes its FP64 error term NaN, so it still reaches the residual.
struct Fx192 {
    unsigned long long w0, w1, w2;  // little-endian 64-bit words
};

// c = 1075 + L for sums bounded by an * xn (an, xn >= 0).  When the bound is
// zero every product is zero; when it is not finite, products overflow to
// non-finite error terms; any anchor serves then (E = 0).
__device__ __forceinline__ int fx_anchor(double an, double xn)
{
    const bool ok = an > 0.0 && xn > 0.0 && isfinite(an) && isfinite(xn);
    const int E = ok ? ilogb(an) + ilogb(xn) + 2 : 0;
    return 1075 + E - 189;
}

// S += p 2^-L exactly, truncated toward zero below bit 0 (c = 1075 + L).  The
// double is m 2^(e - 1075) with m its 53-bit integer significand (no implicit
// bit for subnormals, e raised to 1), so m lands at bit s = e - c of S; the
// magnitude is placed in three words and added, or subtracted as its one's
// complement with a carry in, by one chain of extended-precision adds.
__device__ __forceinline__ void fx_add(Fx192 &a, double p, int c)
{
    const unsigned long long bits = (unsigned long long)__double_as_longlong(p);
    const int ex = (int)(bits >> 52) & 0x7ff;
    unsigned long long m = (bits & 0xfffffffffffffULL) | ((unsigned long long)(ex != 0) << 52);
    int s = max(ex, 1) - c;
    m >>= min(max(-s, 0), 63);  // the bits below 2^L
    s = max(s, 0);
    const int wi = s >> 6, b = s & 63;
    const unsigned long long lo = m << b, hi = (m >> 1) >> (63 - b);
    const unsigned long long neg = (unsigned long long)((long long)bits >> 63);
    const unsigned long long x0 = (wi == 0 ? lo : 0ULL) ^ neg;
    const unsigned long long x1 = (wi == 0 ? hi : (wi == 1 ? lo : 0ULL)) ^ neg;
    const unsigned long long x2 = (wi == 1 ? hi : (wi == 2 ? lo : 0ULL)) ^ neg;
    // carry in = 1 for negative p: neg + neg carries out exactly when neg != 0
    asm("{\n\t.reg .u64 t;\n\t"
        "add.cc.u64 t, %3, %3;\n\t"
        "addc.cc.u64 %0, %0, %4;\n\t"
        "addc.cc.u64 %1, %1, %5;\n\t"
        "addc.u64 %2, %2, %6;\n\t}"
        : "+l"(a.w0), "+l"(a.w1), "+l"(a.w2)
        : "l"(neg), "l"(x0), "l"(x1), "l"(x2));
}

// a += b (exact, modulo 2^192)
__device__ __forceinline__ void fx_merge(Fx192 &a, const Fx192 &b)
{
    asm("add.cc.u64 %0, %0, %3;\n\t"
        "addc.cc.u64 %1, %1, %4;\n\t"
        "addc.u64 %2, %2, %5;"
        : "+l"(a.w0), "+l"(a.w1), "+l"(a.w2)
        : "l"(b.w0), "l"(b.w1), "l"(b.w2));
}

// (hi, lo) = S 2^L as an unevaluated sum of two doubles (relative error about
// 2^-104): the magnitude's six 32-bit limbs, each exact in FP64, scaled and
// added from the top by TwoSum.
__device__ __forceinline__ void fx_to_dd(Fx192 a, int c, double &hi, double &lo)
{
    const bool negative = (long long)a.w2 < 0;
    if (negative) {
        a.w0 = ~a.w0;
        a.w1 = ~a.w1;
        a.w2 = ~a.w2;
        const Fx192 one{1ULL, 0ULL, 0ULL};
        fx_merge(a, one);
    }
    const int L = c - 1075;
    const unsigned long long w[3] = {a.w0, a.w1, a.w2};
    hi = 0.0;
    lo = 0.0;
#pragma unroll
    for (int k = 5; k >= 0; --k) {
        const unsigned int limb = (unsigned int)(w[k >> 1] >> (32 * (k & 1)));
        const double t = scalbn((double)limb, L + 32 * k);
        double s, e;
        dd_two_sum(hi, t, s, e);
        hi = s;
        lo = __dadd_rn(lo, e);
    }
    const double s = __dadd_rn(hi, lo);
    lo = __dsub_rn(lo, __dsub_rn(s, hi));
    hi = s;
    if (negative) {
        hi = -hi;
        lo = -lo;
    }
}

// b - (S 2^L + es) in double-double, rounded once: the residual of one row
// from its exact integer product sum S and the FP64 sum es of the products'
// rounding errors.
__device__ __forceinline__ double fx_residual(double b, const Fx192 &S, int c, double es)
{
    double h, l, s, e;
    fx_to_dd(S, c, h, l);
    dd_two_sum(b, -h, s, e);
    return __dadd_rn(s, __dsub_rn(__dsub_rn(e, l), es));
}

// ---- double-float arithmetic of the preconditioner's product ----------------
// v = hi + lo as two floats (hi = v rounded to FP32, lo = the rest rounded).
__device__ __forceinline__ float2 df_split(double v)
{
    const float h = __double2float_rn(v);
    return make_float2(h, __double2float_rn(__dsub_rn(v, (double)h)));
}

// (s, c) += m (vh + vl) on the FP32 pipe: the product m vh exactly (one
// fused multiply-add gives its rounding error), TwoSum into s, every error
// term gathered in c; carries about 2^-46 of |m v| where plain FP32 carries
// 2^-24.
__device__ __forceinline__ void df_fma(float m, float2 v, float &s, float &c)
{
    const float p = __fmul_rn(m, v.x);
    const float pe = __fmaf_rn(m, v.x, -p);
    const float t = __fadd_rn(s, p);
    const float bb = __fsub_rn(t, s);
    const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bb)), __fsub_rn(p, bb));
    s = t;
    c = __fadd_rn(c, __fadd_rn(e, __fmaf_rn(m, v.y, pe)));
}


}  // namespace nrs
