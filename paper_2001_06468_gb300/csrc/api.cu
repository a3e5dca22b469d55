// api.cu -- the extern "C" entry points of libnrs (declared in include/nrs.h).
//
// The host code here validates arguments, owns the device workspaces and
// enqueues kernels; every arithmetic step of the method runs in the kernels
// of geometry.cu, assemble.cu, lu.cu, tc_gemm.cu and solve.cu.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <string>
#include <vector>

#include "nrs_internal.cuh"

using nrs::Ctx;
using nrs::D4;

namespace {

nrs_status fail(Ctx *c, nrs_status s, const std::string &msg)
{
    if (c) c->err = msg;
    return s;
}

#define CK(call)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return fail(c, NRS_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

template <typename T>
cudaError_t dalloc(T **p, size_t count)
{
    *p = nullptr;
    if (count == 0) count = 1;
    return cudaMalloc((void **)p, sizeof(T) * count);
}

nrs_status alloc_all(Ctx *c)
{
    const int64_t N = c->N, Q = c->Q, n = c->n, lda = c->lda, m = c->max_inner;
    // workspaces of the two-level factorisation where it may run
    const bool gj2 = c->factor_prec == NRS_TF32 && n >= 512 &&
                     (c->gj_schedule >= 3 || (c->gj_schedule == 0 && n >= nrs::GJ2_MIN_N));
    const int nb = c->nbodies;
    struct {
        void **p;
        size_t bytes;
    } req[] = {
        {(void **)&c->d_body_x, sizeof(int32_t) * N},
        {(void **)&c->d_body_X, sizeof(int32_t) * Q},
        {(void **)&c->d_kind, sizeof(int32_t) * nb},
        {(void **)&c->d_free_index, sizeof(int32_t) * (nb + c->F)},
        {(void **)&c->d_n_off, sizeof(int64_t) * (nb + 1)},
        {(void **)&c->d_q_off, sizeof(int64_t) * (nb + 1)},
        {(void **)&c->d_U, sizeof(double) * 3 * nb},
        {(void **)&c->d_Om, sizeof(double) * 3 * nb},
        {(void **)&c->d_ext, sizeof(double) * 6 * c->F},
        {(void **)&c->d_x0, sizeof(double) * 3 * nb},
        {(void **)&c->d_B, sizeof(double) * 9 * nb},
        {(void **)&c->d_x0_save, sizeof(double) * 3 * nb},
        {(void **)&c->d_B_save, sizeof(double) * 9 * nb},
        {(void **)&c->d_x, sizeof(D4) * N},
        {(void **)&c->d_Xw, sizeof(D4) * Q},
        {(void **)&c->d_b, sizeof(double) * lda},
        {(void **)&c->d_sol, sizeof(double) * 2 * lda},
        {(void **)&c->d_nn, sizeof(int32_t) * Q},
        {(void **)&c->d_seg_ptr, sizeof(int32_t) * (N + 1)},
        {(void **)&c->d_perm, sizeof(int32_t) * Q},
        {(void **)&c->d_cursor, sizeof(int32_t) * (N + 1)},
        {(void **)&c->d_Xs, sizeof(D4) * Q},
        {(void **)&c->d_W, sizeof(double) * N},
        {(void **)&c->d_R, sizeof(double) * 3 * N},
        {(void **)&c->d_A64, sizeof(double) * lda * n},
        {(void **)&c->d_A32, sizeof(float) * lda * n},
        {(void **)&c->d_rowperm, sizeof(int32_t) * n},
        {(void **)&c->d_lperm, sizeof(int32_t) * 64},
        {(void **)&c->d_gj_dinv, sizeof(float) * 2 * 64 * 64},
        {(void **)&c->d_gj_rt, sizeof(float) * 4 * 64 * lda},
        {(void **)&c->d_gj_cb, sizeof(float) * 4 * 64 * lda},
        {(void **)&c->d_gj_stage, sizeof(float) * 4 * 64 * 64},
        {(void **)&c->d_gj_sync, sizeof(int32_t) * 4},
        {(void **)&c->d_info, sizeof(int32_t)},
        {(void **)&c->d_r, sizeof(double) * lda},
        {(void **)&c->d_w, sizeof(double) * lda},
        {(void **)&c->d_V, sizeof(double) * lda * (m + 1)},
        {(void **)&c->d_H, sizeof(double) * (m + 1) * m},
        {(void **)&c->d_gv, sizeof(double) * (4 * m + 2)},
        {(void **)&c->d_scal, sizeof(double) * (16 + 2 * (m + 1))},
        {(void **)&c->d_part, sizeof(double) * 64 * lda},
        {(void **)&c->d_part32, sizeof(double) * 64 * lda},
        {(void **)&c->d_part_fx, sizeof(unsigned long long) * 3 * 64 * lda},
        {(void **)&c->d_vf, sizeof(float2) * lda},
        {(void **)&c->d_vf2, sizeof(float2) * lda},
        {(void **)&c->d_Adf, c->arnoldi_df ? sizeof(float2) * (size_t)lda * (size_t)n : 0},
        {(void **)&c->d_gj2, gj2 ? nrs::gj2_workspace_bytes(n) : 0},
        {(void **)&c->d_gj2_r, gj2 ? sizeof(float) * 64 * 256 : 0},
        {(void **)&c->d_t32, sizeof(float) * 2 * lda},
        {(void **)&c->d_t64, sizeof(double) * 2 * lda},
        {(void **)&c->d_flags, sizeof(int32_t) * nrs::ceil_div(n, 64)},
        {(void **)&c->d_status, sizeof(int32_t)},
        {(void **)&c->d_dpart, sizeof(double) * nrs::pg_dpart_doubles(c->max_inner)},
        {(void **)&c->d_bar, sizeof(int32_t) * 2},
        {(void **)&c->d_pg_stats, sizeof(double) * 8},
        {(void **)&c->d_step_stats, sizeof(double) * 16},
        {(void **)&c->d_Xsh, sizeof(float4) * Q},
        {(void **)&c->d_Xsl, sizeof(float4) * Q},
        {(void **)&c->d_xh, sizeof(float4) * N},
        {(void **)&c->d_xl, sizeof(float4) * N},
    };
    for (auto &r : req) {
        *r.p = nullptr;
        cudaError_t e = cudaMalloc(r.p, r.bytes ? r.bytes : 1);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(c, NRS_ENOMEM,
                        "device allocation of " + std::to_string(r.bytes) + " bytes failed");
        }
    }
    return NRS_OK;
}

void free_all(Ctx *c)
{
    void *ptrs[] = {c->d_body_x, c->d_body_X, c->d_kind,   c->d_free_index, c->d_n_off,
                    c->d_q_off,  c->d_U,      c->d_Om,     c->d_ext,        c->d_x0,
                    c->d_B,      c->d_x0_save, c->d_B_save, c->d_tasks_all, c->d_tasks_deform,
                    c->d_x,      c->d_Xw,     c->d_b,      c->d_sol,        c->d_nn,
                    c->d_seg_ptr, c->d_perm,  c->d_cursor, c->d_Xs,         c->d_W,
                    c->d_R,      c->d_A64,    c->d_A32,    c->d_LU64,       c->d_rowperm,
                    c->d_lperm,  c->d_info,   c->d_r,      c->d_xk,         c->d_w,
                    c->d_V,      c->d_H,      c->d_gv,     c->d_scal,       c->d_part,
                    c->d_t32,    c->d_t64,    c->d_flags,  c->d_status,     c->d_gj_dinv,
                    c->d_gj_rt,  c->d_gj_cb,  c->d_dpart,  c->d_bar,        c->d_pg_stats,
                    c->d_step_stats, c->d_Xsh, c->d_Xsl, c->d_xh, c->d_xl, c->d_gj_stage, c->d_gj_sync, c->d_part32,
                    c->d_part_fx, c->d_vf, c->d_gj2, c->d_gj2_r,
                    c->d_vf2, c->d_Adf};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    void *tr[] = {c->d_tr, c->d_tr_save, c->d_tr_u, c->d_tr_part, c->d_vel_part, c->d_dp_K,
                  c->d_dp_err, c->d_mblk_keep, c->d_nblk_keep};
    for (void *p : tr)
        if (p) cudaFree(p);
    void *mlp[] = {c->d_mlp_params, c->d_mlp_m,  c->d_mlp_v,     c->d_mlp_g,    c->d_mlp_x,
                   c->d_mlp_t,      c->d_mlp_y,  c->d_mlp_z1,    c->d_mlp_z2,   c->d_mlp_dy,
                   c->d_mlp_d1,     c->d_mlp_d2, c->d_mlp_part,  c->d_mlp_wmean, c->d_mlp_scal,
                   c->d_mlp_xp,     c->d_mlp_xc, c->d_mlp_x0,    c->d_mlp_used};
    for (void *p : mlp)
        if (p) cudaFree(p);
    if (c->h_mlp_used) cudaFreeHost(c->h_mlp_used);
    if (c->h_mlp_loss) cudaFreeHost(c->h_mlp_loss);
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    c->ev_pool.clear();
    if (c->ev_upd) cudaEventDestroy(c->ev_upd);
    if (c->ev_diag) cudaEventDestroy(c->ev_diag);
    if (c->ev_fin_ready) cudaEventDestroy(c->ev_fin_ready);
    for (auto &e : c->ev_fin)
        if (e) cudaEventDestroy(e);
    if (c->stream2) cudaStreamDestroy(c->stream2);
    if (c->stream4) cudaStreamDestroy(c->stream4);
    if (c->stream3) cudaStreamSynchronize(c->stream3), cudaStreamDestroy(c->stream3);
    if (c->ev_asm) cudaEventDestroy(c->ev_asm);
    if (c->ev_asm_done) cudaEventDestroy(c->ev_asm_done);
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->gstream) cudaStreamDestroy(c->gstream);
    c->ev_upd = c->ev_diag = nullptr;
    c->ev_fin_ready = c->ev_fin[0] = c->ev_fin[1] = nullptr;
    c->stream2 = nullptr;
    c->stream4 = nullptr;
    c->stream3 = nullptr;
    c->ev_asm = c->ev_asm_done = nullptr;
    c->gexec = nullptr;
    c->gstream = nullptr;
}

// NRS_BF16 is reserved: no BF16 factorisation is built, so it is rejected
// rather than run in another precision
bool is_prec(int p) { return p == NRS_FP64 || p == NRS_FP32 || p == NRS_TF32; }

__global__ void k_cvt_f64_f32(int64_t count, const double *__restrict__ a, float *__restrict__ b)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) b[i] = (float)a[i];
}

nrs_status do_factor(Ctx *c, int prec)
{
    if (!c->assembled) return fail(c, NRS_EINVAL, "nrs_factor before nrs_assemble");
    if (prec == NRS_TF32 && !nrs::tc_available())
        return fail(c, NRS_EINVAL, "tensor-core factor precision needs a tcgen05 device and the tensor-map driver entry point");
    const size_t elems = (size_t)c->lda * c->n;
    if (prec == NRS_FP64) {
        nrs::join_assembly(*c);
        if (!c->d_LU64) {
            cudaError_t e = cudaMalloc(&c->d_LU64, sizeof(double) * elems);
            if (e != cudaSuccess) {
                cudaGetLastError();
                c->d_LU64 = nullptr;
                return fail(c, NRS_ENOMEM, "FP64 factor workspace does not fit");
            }
        }
        c->tbeg(nrs::PH_CONVERT);
        CK(cudaMemcpyAsync(c->d_LU64, c->d_A64, sizeof(double) * elems, cudaMemcpyDeviceToDevice,
                           c->stream));
        c->tend(nrs::PH_CONVERT);
        nrs::run_lu_fp64(*c, c->d_LU64, c->lda);
    } else {
        if (!c->a32_fresh) {
            nrs::join_assembly(*c);  // the conversion reads the FP64 matrix
            c->tbeg(nrs::PH_CONVERT);
            k_cvt_f64_f32<<<(unsigned)nrs::ceil_div((int64_t)elems, 256), 256, 0, c->stream>>>(
                (int64_t)elems, c->d_A64, c->d_A32);
            c->tend(nrs::PH_CONVERT);
            c->launches += 1;
        }
        if (nrs::run_gj_fp32(*c, c->d_A32, c->lda, prec) != 0)
            return fail(c, NRS_EINVAL, "nrs_factor: the tensor-core update could not be launched");
        c->a32_fresh = false;
    }
    CK(cudaGetLastError());
    c->factored_prec = prec;
    c->factorizations += 1;
    return NRS_OK;
}

// write_lo: also write the FP32 copy (which a Gauss-Jordan factor replaces by
// its inverse: writing it destroys that factor).
nrs_status do_segments_and_assemble(Ctx *c, const D4 *x_lab, const D4 *Xw_lab, bool write_lo = true,
                                    bool from_state = false)
{
    nrs::launch_gather(*c, Xw_lab, c->d_seg_ptr, c->d_perm);
    float *a32 = (c->factor_prec == NRS_FP64 || !write_lo) ? nullptr : c->d_A32;
    if (a32 && c->factored_prec != NRS_FP64) c->factored_prec = -1;
    nrs::join_assembly(*c);  // an earlier FP64 assembly must not overlap this one
    if (a32 && c->lo_eval == 0) {
        // the FP32 copy first, alone on the GPU, so the factorisation can start;
        // then the FP64 matrix on the side stream beside the factorisation,
        // joined before the refinement uses it
        nrs::launch_assemble32(*c, x_lab, a32, c->lda);
        CK(cudaEventRecord(c->ev_asm, c->stream));
        CK(cudaStreamWaitEvent(c->stream3, c->ev_asm, 0));
        nrs::launch_assemble(*c, x_lab, c->d_A64, nullptr, c->lda, c->stream3, from_state);
        CK(cudaEventRecord(c->ev_asm_done, c->stream3));
        c->asm_pending = true;
    } else {
        // one FP64 pass; with an FP32 copy, that copy is the rounded FP64 entries
        nrs::launch_assemble(*c, x_lab, c->d_A64, a32, c->lda, nullptr, from_state);
    }
    // the border rows and columns: disjoint from the block the side stream writes
    nrs::launch_border(*c, x_lab, c->d_A64, a32, c->lda);
    CK(cudaGetLastError());
    c->a32_fresh = a32 != nullptr;
    c->assembled = true;
    return NRS_OK;
}

// Workspaces of the learned starting guess, allocated by the first nrs_mlp_* call.
nrs_status mlp_alloc(Ctx *c)
{
    if (c->mlp_alloc) return NRS_OK;
    const int64_t N = c->N, P = NRS_MLP_PARAMS, H = NRS_MLP_HID;
    struct {
        void **p;
        size_t bytes;
    } req[] = {
        {(void **)&c->d_mlp_params, sizeof(float) * P},
        {(void **)&c->d_mlp_m, sizeof(float) * P},
        {(void **)&c->d_mlp_v, sizeof(float) * P},
        {(void **)&c->d_mlp_g, sizeof(float) * P},
        {(void **)&c->d_mlp_x, sizeof(float) * N * NRS_MLP_IN},
        {(void **)&c->d_mlp_t, sizeof(float) * N * NRS_MLP_OUT},
        {(void **)&c->d_mlp_y, sizeof(float) * N * NRS_MLP_OUT},
        {(void **)&c->d_mlp_z1, sizeof(float) * N * H},
        {(void **)&c->d_mlp_z2, sizeof(float) * N * H},
        {(void **)&c->d_mlp_dy, sizeof(float) * N * NRS_MLP_OUT},
        {(void **)&c->d_mlp_d1, sizeof(float) * N * H},
        {(void **)&c->d_mlp_d2, sizeof(float) * N * H},
        {(void **)&c->d_mlp_part, sizeof(float) * P * nrs::mlp_grad_chunks(N)},
        {(void **)&c->d_mlp_wmean, sizeof(double) * c->nbodies},
        {(void **)&c->d_mlp_scal, sizeof(double) * 8},
        {(void **)&c->d_mlp_xp, sizeof(double) * c->lda},
        {(void **)&c->d_mlp_xc, sizeof(double) * c->lda},
        {(void **)&c->d_mlp_x0, sizeof(double) * c->lda},
        {(void **)&c->d_mlp_used, sizeof(int32_t) * 2},
    };
    for (auto &r : req) {
        cudaError_t e = cudaMalloc(r.p, r.bytes ? r.bytes : 1);
        if (e != cudaSuccess) {
            cudaGetLastError();
            *r.p = nullptr;
            return fail(c, NRS_ENOMEM, "MLP workspace allocation failed");
        }
    }
    CK(cudaHostAlloc((void **)&c->h_mlp_used, sizeof(int32_t) * 2, cudaHostAllocDefault));
    CK(cudaHostAlloc((void **)&c->h_mlp_loss, sizeof(double) * 2, cudaHostAllocDefault));
    CK(cudaMemsetAsync(c->d_mlp_scal, 0, sizeof(double) * 8, c->stream));
    CK(cudaMemsetAsync(c->d_mlp_used, 0, sizeof(int32_t) * 2, c->stream));
    c->mlp_alloc = true;
    return NRS_OK;
}

}  // namespace

namespace nrs {

void join_assembly(Ctx &c)
{
    if (!c.asm_pending) return;
    cudaStreamWaitEvent(c.stream, c.ev_asm_done, 0);
    c.asm_pending = false;
}

bool graph_capable(const Ctx &c)
{
    return c.factor_prec != NRS_FP64 && c.solve_mode == 0 && c.max_inner <= 64 &&
           !c.reuse_factor && !c.mlp_predict && c.mlp_train_iters == 0 && !c.timing &&
           c.nn_valid && c.seg_valid;
}

nrs_status enqueue_step(Ctx *c, const nrs_shapes *s0, const nrs_shapes *sh, double dt,
                        double *stats, bool berr)
{
    CK(cudaMemcpyAsync(c->d_x0_save, c->d_x0, sizeof(double) * 3 * c->nbodies,
                       cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpyAsync(c->d_B_save, c->d_B, sizeof(double) * 9 * c->nbodies,
                       cudaMemcpyDeviceToDevice, c->stream));
    if (c->n_tracers > 0)
        CK(cudaMemcpyAsync(c->d_tr_save, c->d_tr, sizeof(D4) * c->n_tracers,
                           cudaMemcpyDeviceToDevice, c->stream));
    for (int stage = 0; stage < 2; ++stage) {
        const nrs_shapes *s = stage ? sh : s0;
        launch_kinematics(*c, (const D4 *)s->xi, (const D4 *)s->Xiw, (const D4 *)s->xidot, c->d_x,
                          c->d_Xw, c->d_b);
        c->kin_valid = true;
        if (c->nn_global) {
            launch_nearest(*c, c->d_x, c->d_Xw, c->d_nn, false);
            launch_segments(*c, c->d_nn, c->d_seg_ptr, c->d_perm);
        } else if (c->n_tasks_deform > 0) {
            launch_nearest(*c, (const D4 *)s->xi, (const D4 *)s->Xiw, c->d_nn, true);
            launch_segments(*c, c->d_nn, c->d_seg_ptr, c->d_perm);
        }
        nrs_status st = do_segments_and_assemble(c, c->d_x, c->d_Xw, true, true);
        if (st != NRS_OK) return st;
        st = do_factor(c, c->factor_prec);
        if (st != NRS_OK) return st;
        double *out = c->d_sol + (int64_t)stage * c->lda;
        const double *prev = c->have_sol ? c->d_sol + (int64_t)(1 - stage) * c->lda : nullptr;
        const bool warm = c->warm_start && prev;
        if (warm)
            CK(cudaMemcpyAsync(out, prev, sizeof(double) * c->n, cudaMemcpyDeviceToDevice,
                               c->stream));
        double *so = stats + 8 * stage;
        join_assembly(*c);
        CK(launch_gmres_persistent(*c, c->d_b, out, !warm, so));
        if (berr) enqueue_backward_error(*c, c->d_b, out, so + 5);
        if (c->n_tracers > 0) {
            launch_velocity(*c, c->d_Xw, c->d_tr, c->n_tracers, out, c->d_tr_u, c->d_tr_part,
                            c->stream);
            launch_tracer_update(*c, stage, dt, c->stream);
        }
        launch_rk2(*c, stage, dt, out);
        CK(cudaGetLastError());
    }
    return NRS_OK;
}

}  // namespace nrs

namespace {

// nrs_step through a recorded CUDA graph (graph mode, see include/nrs.h).
nrs_status step_graph(Ctx *c, const nrs_shapes *s0, const nrs_shapes *sh, double dt, double *sol,
                      nrs_step_report *report)
{
    Ctx::GraphKey key{{s0->xi, s0->Xiw, s0->xidot, sh->xi, sh->Xiw, sh->xidot}, dt,
                      report != nullptr};
    if (!c->gexec || !(key == c->gkey)) {
        cudaStream_t user = c->stream;
        c->stream = c->gstream;
        const int64_t l0 = c->launches;
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
        nrs_status st = e == cudaSuccess ? nrs::enqueue_step(c, s0, sh, dt, c->d_step_stats,
                                                             key.berr)
                                         : NRS_ECUDA;
        cudaError_t e2 = e == cudaSuccess ? cudaStreamEndCapture(c->stream, &g) : e;
        c->stream = user;
        c->graph_launches = c->launches - l0;
        c->launches = l0;
        if (st != NRS_OK || e2 != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return fail(c, st != NRS_OK ? st : NRS_ECUDA,
                        std::string("recording the step graph failed: ") + cudaGetErrorString(e2));
        }
        if (c->gexec) cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
        e = cudaGraphInstantiate(&c->gexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            c->gexec = nullptr;
            return fail(c, NRS_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
        }
        c->gkey = key;
        c->graph_captures += 1;
    }
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (report) {
        CK(cudaEventCreate(&ev0));
        CK(cudaEventCreate(&ev1));
        CK(cudaEventRecord(ev0, c->stream));
    }
    CK(cudaGraphLaunch(c->gexec, c->stream));
    c->launches += c->graph_launches;
    c->have_sol = true;
    c->factored_prec = c->factor_prec;
    c->factorizations += 2;
    if (sol) {
        CK(cudaMemcpyAsync(sol, c->d_sol, sizeof(double) * c->n, cudaMemcpyDeviceToDevice, c->stream));
        CK(cudaMemcpyAsync(sol + c->n, c->d_sol + c->lda, sizeof(double) * c->n,
                           cudaMemcpyDeviceToDevice, c->stream));
    }
    if (!report) return NRS_OK;
    CK(cudaEventRecord(ev1, c->stream));
    CK(cudaEventSynchronize(ev1));
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, ev0, ev1);
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    double st[16];
    int32_t word = 0;
    CK(cudaMemcpy(st, c->d_step_stats, sizeof(st), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(&word, c->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost));
    CK(cudaMemset(c->d_status, 0, sizeof(int32_t)));
    nrs_status worst = NRS_OK;
    for (int k = 0; k < 2; ++k) {
        const double *q = st + 8 * k;
        nrs_solve_report &r = report->stage[k];
        r.outer = (int32_t)q[0];
        r.inner = (int32_t)q[1];
        r.converged = q[2] != 0.0;
        r.last_update = q[4] > 0 ? q[3] / q[4] : 0.0;
        r.backward_err = q[5] / (q[6] * q[4] + q[7]);
        r.status = (word & nrs::ST_TIMEOUT)     ? NRS_ETIMEOUT
                   : (word & nrs::ST_NONFINITE) ? NRS_ENONFINITE
                   : !r.converged               ? NRS_ENOCONV
                                                : NRS_OK;
        if (r.status != NRS_OK && worst == NRS_OK) worst = (nrs_status)r.status;
        report->start[k] = c->warm_start ? 1 : 0;
    }
    report->ms_total = ms;
    report->factorizations = 2;
    report->mlp_rel_err = -1.0;
    report->retried[0] = report->retried[1] = 0;
    if (worst != NRS_OK) c->err = "a stage of the recorded step did not converge cleanly";
    return worst;
}

}  // namespace

extern "C" {

nrs_status nrs_create(nrs_ctx **out, const nrs_problem_desc *d, void *stream)
{
    Ctx *c = nullptr;
    if (!out || !d) return NRS_EINVAL;
    *out = nullptr;
    if (d->nbodies <= 0 || !d->n_off || !d->q_off || !d->kind) return NRS_EINVAL;
    if (!(d->eps > 0.0) || !(d->mu > 0.0)) return NRS_EINVAL;
    if (d->n_off[0] != 0 || d->q_off[0] != 0) return NRS_EINVAL;
    if (!is_prec(d->factor_prec)) return NRS_EINVAL;
    for (int b = 0; b < d->nbodies; ++b) {
        if (d->n_off[b + 1] < d->n_off[b] || d->q_off[b + 1] < d->q_off[b]) return NRS_EINVAL;
        if (d->kind[b] < NRS_FREE || d->kind[b] > NRS_STATIC) return NRS_EINVAL;
        if (d->q_off[b + 1] > d->q_off[b] && d->n_off[b + 1] == d->n_off[b] && !d->nn_global)
            return NRS_EINVAL;
    }
    const int64_t N = d->n_off[d->nbodies], Q = d->q_off[d->nbodies];
    if (N <= 0 || Q <= 0 || N > (1LL << 28) || Q > (1LL << 30)) return NRS_EINVAL;
    c = new (std::nothrow) Ctx();
    if (!c) return NRS_ENOMEM;
    c->stream = (cudaStream_t)stream;
    cudaGetDevice(&c->device);
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    c->nbodies = d->nbodies;
    c->N = N;
    c->Q = Q;
    c->n_off.assign(d->n_off, d->n_off + d->nbodies + 1);
    c->q_off.assign(d->q_off, d->q_off + d->nbodies + 1);
    c->kind.assign(d->kind, d->kind + d->nbodies);
    c->rigid.assign(d->nbodies, 0);
    if (d->rigid)
        for (int b = 0; b < d->nbodies; ++b) c->rigid[b] = d->rigid[b] ? 1 : 0;
    c->free_index.assign(d->nbodies, -1);
    std::vector<int32_t> free_body;
    for (int b = 0; b < d->nbodies; ++b)
        if (c->kind[b] == NRS_FREE) {
            c->free_index[b] = (int32_t)free_body.size();
            free_body.push_back(b);
        }
    c->F = (int64_t)free_body.size();
    c->n = 3 * N + 6 * c->F;
    c->lda = nrs::ceil_div(c->n, 32) * 32;
    c->eps = d->eps;
    c->mu = d->mu;
    c->nn_global = d->nn_global ? 1 : 0;
    c->factor_prec = d->factor_prec;
    c->nb = 64;
    c->tol = d->tol > 0 ? d->tol : 1e-12;
    c->max_outer = d->max_outer > 0 ? d->max_outer : 20;
    c->max_inner = d->max_inner > 0 ? d->max_inner : 30;
    c->reuse_factor = d->reuse_factor ? 1 : 0;
    c->reuse_max_inner = d->reuse_max_inner > 0 ? d->reuse_max_inner : 8;
    c->reuse_max_stages = d->reuse_max_stages > 0 ? d->reuse_max_stages : 16;
    c->warm_start = d->warm_start ? 1 : 0;
    c->solve_mode = d->solve_mode ? 1 : 0;
    if (d->inner_tol < 0.0 || !(d->inner_tol < 1.0)) {
        delete c;
        return NRS_EINVAL;
    }
    c->tol_in = d->inner_tol > 0.0 ? d->inner_tol : 1e-4;
    c->lo_eval = d->factor_input ? 1 : 0;
    c->residual_dd = d->residual == 0 ? 1 : 0;
    if (d->arnoldi < 0 || d->arnoldi > 1) {
        delete c;
        return NRS_EINVAL;
    }
    c->arnoldi_df = d->arnoldi == 1 && d->factor_prec != NRS_FP64;
    if (d->factor_schedule < 0 || d->factor_schedule > 4) {
        delete c;
        return NRS_EINVAL;
    }
    c->gj_schedule = d->factor_schedule;
    c->gj_fused = d->factor_schedule == 1;
    c->graph_mode = d->graph ? 1 : 0;
    if (c->graph_mode && (d->factor_prec == NRS_FP64 || c->solve_mode != 0 || d->reuse_factor ||
                          (d->max_inner > 64))) {
        delete c;
        return NRS_EINVAL;
    }
    {
        // enough column splits for about two CTAs per SM in the matrix-vector products
        auto splits = [&](int64_t rows_per_cta) {
            int64_t rowblocks = nrs::ceil_div(c->n, rows_per_cta);
            int64_t s = nrs::ceil_div(2 * (int64_t)c->num_sms, rowblocks);
            return (int)std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(s, 64), c->n));
        };
        c->splits64 = splits(256);
        c->splits32 = splits(512);
    }
    nrs_status st = alloc_all(c);
    if (st != NRS_OK) {
        std::string msg = c->err;
        free_all(c);
        delete c;
        return st;
    }
    // body tables
    std::vector<int32_t> bx(N), bX(Q);
    for (int b = 0; b < d->nbodies; ++b) {
        for (int64_t i = d->n_off[b]; i < d->n_off[b + 1]; ++i) bx[i] = b;
        for (int64_t i = d->q_off[b]; i < d->q_off[b + 1]; ++i) bX[i] = b;
    }
    std::vector<int32_t> fi(c->free_index);
    fi.insert(fi.end(), free_body.begin(), free_body.end());
    std::vector<double> U(3 * d->nbodies, 0.0), Om(3 * d->nbodies, 0.0);
    if (d->U) memcpy(U.data(), d->U, sizeof(double) * 3 * d->nbodies);
    if (d->Omega) memcpy(Om.data(), d->Omega, sizeof(double) * 3 * d->nbodies);
    std::vector<double> x0(3 * d->nbodies, 0.0), B(9 * d->nbodies, 0.0);
    for (int b = 0; b < d->nbodies; ++b) B[9 * b + 0] = B[9 * b + 4] = B[9 * b + 8] = 1.0;
    // nearest-neighbour tasks: 128 quadrature points of one body each
    std::vector<nrs::NNTask> all, deform;
    for (int b = 0; b < d->nbodies; ++b)
        for (int64_t q0 = d->q_off[b]; q0 < d->q_off[b + 1]; q0 += nrs::NN_QPB) {
            nrs::NNTask t{b, (int32_t)q0,
                          (int32_t)std::min<int64_t>(q0 + nrs::NN_QPB, d->q_off[b + 1]), 0};
            all.push_back(t);
            if (!c->rigid[b] || c->nn_global) deform.push_back(t);
        }
    c->n_tasks_all = (int)all.size();
    c->n_tasks_deform = (int)deform.size();
    // blocks of the assembly made only of static rigid bodies' points (per-body
    // nearest neighbours: their segments hold only their own quadrature points)
    std::vector<uint8_t> keep_pt(N, 0);
    if (!c->nn_global)
        for (int b = 0; b < d->nbodies; ++b)
            if (c->kind[b] == NRS_STATIC && c->rigid[b])
                for (int64_t i = d->n_off[b]; i < d->n_off[b + 1]; ++i) keep_pt[i] = 1;
    auto blocks = [&](int64_t bs) {
        std::vector<uint8_t> f((size_t)nrs::ceil_div(N, bs), 0);
        for (size_t k = 0; k < f.size(); ++k) {
            uint8_t all_keep = 1;
            for (int64_t i = (int64_t)k * bs; i < std::min<int64_t>(N, (int64_t)(k + 1) * bs); ++i)
                all_keep &= keep_pt[i];
            f[k] = all_keep;
        }
        return f;
    };
    const std::vector<uint8_t> mblk = blocks(nrs::kAssembleTileM), nblk = blocks(nrs::kAssembleTileN);
    for (uint8_t v : mblk) c->have_static |= v != 0;
    cudaError_t e = cudaSuccess;
    if (c->have_static) {
        e = cudaMalloc(&c->d_mblk_keep, mblk.size());
        if (e == cudaSuccess) e = cudaMalloc(&c->d_nblk_keep, nblk.size());
        if (e == cudaSuccess) e = cudaMemcpy(c->d_mblk_keep, mblk.data(), mblk.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(c->d_nblk_keep, nblk.data(), nblk.size(), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess)
        e = cudaMalloc(&c->d_tasks_all, sizeof(nrs::NNTask) * std::max<size_t>(1, all.size()));
    if (e == cudaSuccess)
        e = cudaMalloc(&c->d_tasks_deform, sizeof(nrs::NNTask) * std::max<size_t>(1, deform.size()));
    auto h2d = [&](void *dst, const void *src, size_t bytes) {
        if (e == cudaSuccess && bytes) e = cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
    };
    h2d(c->d_tasks_all, all.data(), sizeof(nrs::NNTask) * all.size());
    h2d(c->d_tasks_deform, deform.data(), sizeof(nrs::NNTask) * deform.size());
    h2d(c->d_body_x, bx.data(), sizeof(int32_t) * N);
    h2d(c->d_body_X, bX.data(), sizeof(int32_t) * Q);
    h2d(c->d_kind, c->kind.data(), sizeof(int32_t) * d->nbodies);
    h2d(c->d_free_index, fi.data(), sizeof(int32_t) * fi.size());
    h2d(c->d_n_off, d->n_off, sizeof(int64_t) * (d->nbodies + 1));
    h2d(c->d_q_off, d->q_off, sizeof(int64_t) * (d->nbodies + 1));
    h2d(c->d_U, U.data(), sizeof(double) * U.size());
    h2d(c->d_Om, Om.data(), sizeof(double) * Om.size());
    h2d(c->d_x0, x0.data(), sizeof(double) * x0.size());
    h2d(c->d_B, B.data(), sizeof(double) * B.size());
    if (e == cudaSuccess && c->F) e = cudaMemset(c->d_ext, 0, sizeof(double) * 6 * c->F);
    if (e == cudaSuccess) e = cudaMemset(c->d_flags, 0, sizeof(int32_t) * nrs::ceil_div(c->n, 64));
    if (e == cudaSuccess) e = cudaMemset(c->d_status, 0, sizeof(int32_t));
    if (e == cudaSuccess) {
        // the lookahead stream runs single-CTA kernels on the critical path:
        // highest priority, so the block scheduler serves them first
        int least = 0, greatest = 0;
        cudaDeviceGetStreamPriorityRange(&least, &greatest);
        e = cudaStreamCreateWithPriority(&c->stream2, cudaStreamNonBlocking, greatest);
        if (e == cudaSuccess)
            e = cudaStreamCreateWithPriority(&c->stream4, cudaStreamNonBlocking, greatest);
    }
    if (e == cudaSuccess && c->graph_mode)
        e = cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking);
    if (e == cudaSuccess) {
        // the FP64 assembly fills what the latency-bound factorisation leaves idle
        int least = 0, greatest = 0;
        cudaDeviceGetStreamPriorityRange(&least, &greatest);
        e = cudaStreamCreateWithPriority(&c->stream3, cudaStreamNonBlocking, least);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_asm, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_asm_done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_upd, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_diag, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_fin_ready, cudaEventDisableTiming);
    for (auto &ev : c->ev_fin)
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        free_all(c);
        delete c;
        return NRS_ECUDA;
    }
    *out = reinterpret_cast<nrs_ctx *>(c);
    return NRS_OK;
}

nrs_status nrs_destroy(nrs_ctx *ctx)
{
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c) return NRS_EINVAL;
    cudaStreamSynchronize(c->stream);
    free_all(c);
    delete c;
    return NRS_OK;
}

const char *nrs_last_error(const nrs_ctx *ctx)
{
    const Ctx *c = reinterpret_cast<const Ctx *>(ctx);
    return c ? c->err.c_str() : "null context";
}

nrs_status nrs_sizes(const nrs_ctx *ctx, int64_t *N, int64_t *Q, int64_t *F, int64_t *n)
{
    const Ctx *c = reinterpret_cast<const Ctx *>(ctx);
    if (!c) return NRS_EINVAL;
    if (N) *N = c->N;
    if (Q) *Q = c->Q;
    if (F) *F = c->F;
    if (n) *n = c->n;
    return NRS_OK;
}

nrs_status nrs_set_state(nrs_ctx *ctx, const double *x0, const double *B)
{
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c || !x0 || !B) return fail(c, NRS_EINVAL, "nrs_set_state: null argument");
    CK(cudaMemcpyAsync(c->d_x0, x0, sizeof(double) * 3 * c->nbodies, cudaMemcpyHostToDevice,
                       c->stream));
    CK(cudaMemcpyAsync(c->d_B, B, sizeof(double) * 9 * c->nbodies, cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    // static bodies may have moved: the kept blocks of A_s and a recorded step are stale
    c->static_cache_valid = false;
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
    return NRS_OK;
}

nrs_status nrs_get_state(nrs_ctx *ctx, double *x0, double *B)
{
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c || !x0 || !B) return fail(c, NRS_EINVAL, "nrs_get_state: null argument");
    CK(cudaMemcpyAsync(x0, c->d_x0, sizeof(double) * 3 * c->nbodies, cudaMemcpyDeviceToHost,
                       c->stream));
    CK(cudaMemcpyAsync(B, c->d_B, sizeof(double) * 9 * c->nbodies, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return NRS_OK;
}

nrs_status nrs_set_external(nrs_ctx *ctx, const double *ext)
{
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c) return NRS_EINVAL;
    if (c->F == 0) return NRS_OK;
    if (ext)
        CK(cudaMemcpyAsync(c->d_ext, ext, sizeof(double) * 6 * c->F, cudaMemcpyHostToDevice,
                           c->stream));
    else
        CK(cudaMemsetAsync(c->d_ext, 0, sizeof(double) * 6 * c->F, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return NRS_OK;
}

nrs_status nrs_kinematics(nrs_ctx *ctx, const nrs_shapes *s, double *x, double *Xw, double *b)
{
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c || !s || !s->xi || !s->Xiw || !s->xidot || !x || !Xw || !b)
        return fail(c, NRS_EINVAL, "nrs_kinematics: null argument");
    nrs::launch_kinematics(*c, (const D4 *)s->xi, (const D4 *)s->Xiw, (const D4 *)s->xidot, (D4 *)x,
                           (D4 *)Xw, b);
    CK(cudaGetLastError());
    return NRS_OK;
}

nrs_status nrs_nearest_build(nrs_ctx *ctx, const double *x, const double *Xw, int32_t *nn,
                             int32_t *seg_ptr, int32_t *perm)
{
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c || !x || !Xw) return fail(c, NRS_EINVAL, "nrs_nearest_build: null argument");
    nrs::launch_nearest(*c, (const D4 *)x, (const D4 *)Xw, c->d_nn, false);
    nrs::launch_segments(*c, c->d_nn, c->d_seg_ptr, c->d_perm);
    CK(cudaGetLastError());
    c->map_built = true;
    if (nn) CK(cudaMemcpyAsync(nn, c->d_nn, sizeof(int32_t) * c->Q, cudaMemcpyDeviceToDevice, c->stream));
    if (seg_ptr)
        CK(cudaMemcpyAsync(seg_ptr, c->d_seg_ptr, sizeof(int32_t) * (c->N + 1),
                           cudaMemcpyDeviceToDevice, c->stream));
    if (perm)
        CK(cudaMemcpyAsync(perm, c->d_perm, sizeof(int32_t) * c->Q, cudaMemcpyDeviceToDevice,
                           c->stream));
    c->seg_valid = true;
    c->nn_valid = false;  // the step path recomputes its own map
    return NRS_OK;
}

nrs_status nrs_assemble(nrs_ctx *ctx, const double *x, const double *Xw, double *A64, int64_t lda)
{
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c || !x || !Xw) return fail(c, NRS_EINVAL, "nrs_assemble: null argument");
    if (!c->seg_valid) return fail(c, NRS_EINVAL, "nrs_assemble before nrs_nearest_build");
    if (A64 && lda < c->n) return fail(c, NRS_EINVAL, "nrs_assemble: lda < n");
    nrs_status st = do_segments_and_assemble(c, (const D4 *)x, (const D4 *)Xw);
    if (st != NRS_OK) return st;
    if (A64) {
        nrs::join_assembly(*c);
        CK(cudaMemcpy2DAsync(A64, sizeof(double) * lda, c->d_A64, sizeof(double) * c->lda,
                             sizeof(double) * c->n, c->n, cudaMemcpyDeviceToDevice, c->stream));
    }
    return NRS_OK;
}

nrs_status nrs_factor(nrs_ctx *ctx, int32_t prec, int32_t *info)
{
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c) return NRS_EINVAL;
    if (!is_prec(prec))
        return fail(c, NRS_EINVAL,
                    prec == NRS_BF16 ? "nrs_factor: NRS_BF16 has no factorisation in this library "
                                       "(use NRS_TF32: split-TF32 tensor-core updates)"
                                     : "nrs_factor: unknown precision");
    nrs_status st = do_factor(c, prec);
    if (st != NRS_OK) return st;
    if (info) {
        CK(cudaMemcpyAsync(info, c->d_info, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        if (*info != 0) return fail(c, NRS_ESINGULAR, "exactly zero pivot");
    }
    return NRS_OK;
}

nrs_status nrs_solve(nrs_ctx *ctx, const double *b, double *x, int32_t nrhs, const double *x0,
                     nrs_solve_report *report)
{
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c || !b || !x || nrhs <= 0) return fail(c, NRS_EINVAL, "nrs_solve: bad argument");
    if (c->factored_prec < 0) return fail(c, NRS_EINVAL, "nrs_solve before nrs_factor");
    nrs_status worst = NRS_OK;
    for (int k = 0; k < nrhs; ++k) {
        nrs_status st = nrs::run_gmres_ir(*c, b + (int64_t)k * c->n, x + (int64_t)k * c->n,
                                          x0 ? x0 + (int64_t)k * c->n : nullptr,
                                          report ? report + k : nullptr);
        if (st == NRS_ECUDA) return st;
        if (st != NRS_OK && worst == NRS_OK) worst = st;
    }
    return worst;
}

nrs_status nrs_residual(nrs_ctx *ctx, const double *b, const double *x, double *r)
{
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c || !b || !x || !r) return fail(c, NRS_EINVAL, "nrs_residual: null argument");
    if (!c->assembled) return fail(c, NRS_EINVAL, "nrs_residual before an assembly");
    nrs::join_assembly(*c);
    nrs::enqueue_residual(*c, x, b, r);
    CK(cudaGetLastError());
    return NRS_OK;
}

namespace {

// One evaluation of the swimming problem's right-hand side up to the factor
// (Sec. 4 steps 1-3): kinematics at the context's state, nearest neighbours
// (deforming bodies; rigid ones keep their map), segments, assembly, border,
// and the factorisation if the reuse policy asks for one (*need_factor).
nrs_status prepare_stage(Ctx *c, const nrs_shapes *s, bool *need_factor)
{
    nrs::launch_kinematics(*c, (const D4 *)s->xi, (const D4 *)s->Xiw, (const D4 *)s->xidot, c->d_x,
                           c->d_Xw, c->d_b);
    c->kin_valid = true;
    bool ran = true;
    if (c->nn_global) {
        nrs::launch_nearest(*c, c->d_x, c->d_Xw, c->d_nn, false);
    } else if (!c->nn_valid) {
        nrs::launch_nearest(*c, (const D4 *)s->xi, (const D4 *)s->Xiw, c->d_nn, false);
        c->nn_valid = true;
    } else if (c->n_tasks_deform > 0) {
        nrs::launch_nearest(*c, (const D4 *)s->xi, (const D4 *)s->Xiw, c->d_nn, true);
    } else {
        ran = false;
    }
    if (ran || !c->seg_valid) nrs::launch_segments(*c, c->d_nn, c->d_seg_ptr, c->d_perm);
    c->seg_valid = true;
    *need_factor = !c->reuse_factor || c->factored_prec != c->factor_prec ||
                   c->stages_since_factor >= c->reuse_max_stages ||
                   c->last_inner > c->reuse_max_inner;
    nrs_status st = do_segments_and_assemble(c, c->d_x, c->d_Xw, *need_factor, true);
    if (st != NRS_OK) return st;
    if (*need_factor) {
        st = do_factor(c, c->factor_prec);
        if (st != NRS_OK) return st;
        c->stages_since_factor = 0;
    } else {
        c->stages_since_factor += 1;
    }
    return NRS_OK;
}

// The stage's refinement, and the retry of nrs_step when it does not converge.
nrs_status solve_stage(Ctx *c, double *out, const double *x0, bool need_factor,
                       nrs_solve_report *rep, int *inner_out, int *retried)
{
    int inner = 0;
    *retried = 0;
    nrs_status st = nrs::run_gmres_ir(*c, c->d_b, out, x0, rep, &inner);
    if (st == NRS_ECUDA) return st;
    if (st == NRS_ENOCONV && c->factor_prec != NRS_FP64) {
        // The refinement did not converge with this factor.  An FP32 inverse
        // of a system with kappa(A) u_fp32 >> 1 is sometimes a poor
        // preconditioner; another one usually is not: a two-level factor
        // is replaced by the one-level elimination of the same input (the
        // more robust of the two on such systems), a one-level one by that
        // of the other FP32 input (the rounded FP64 entries instead of the
        // FP32 evaluation, or the reverse), a reused factor by a fresh one
        // of the configured input.  One retry, from the same start.
        const bool was_two = need_factor && c->last_factor_two_level;
        const bool other = need_factor && !was_two ? c->lo_eval == 1 : c->lo_eval == 0;
        if (was_two) c->gj_force_one_level = true;
        nrs::join_assembly(*c);
        if (other) {
            nrs::launch_assemble32(*c, c->d_x, c->d_A32, c->lda);
            c->a32_fresh = true;
        } else {
            c->a32_fresh = false;  // do_factor rounds the FP64 entries
        }
        c->factored_prec = -1;
        st = do_factor(c, c->factor_prec);
        c->gj_force_one_level = false;
        if (st != NRS_OK) return st;
        c->stages_since_factor = 0;
        c->retries += 1;
        *retried = 1;
        inner = 0;
        st = nrs::run_gmres_ir(*c, c->d_b, out, x0, rep, &inner);
        if (st == NRS_ECUDA) return st;
    }
    *inner_out = inner;
    return st;
}

}  // namespace

nrs_status nrs_step(nrs_ctx *ctx, const nrs_shapes *s0, const nrs_shapes *sh, double dt, double *sol,
                    nrs_step_report *report)
{
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c || !s0 || !sh || !s0->xi || !s0->Xiw || !s0->xidot || !sh->xi || !sh->Xiw || !sh->xidot)
        return fail(c, NRS_EINVAL, "nrs_step: null argument");
    if (!(dt > 0.0)) return fail(c, NRS_EINVAL, "nrs_step: dt must be positive");
    if (c->graph_mode && nrs::graph_capable(*c)) return step_graph(c, s0, sh, dt, sol, report);
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (report) {
        CK(cudaEventCreate(&ev0));
        CK(cudaEventCreate(&ev1));
        CK(cudaEventRecord(ev0, c->stream));
    }
    CK(cudaMemcpyAsync(c->d_x0_save, c->d_x0, sizeof(double) * 3 * c->nbodies,
                       cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpyAsync(c->d_B_save, c->d_B, sizeof(double) * 9 * c->nbodies,
                       cudaMemcpyDeviceToDevice, c->stream));
    if (c->n_tracers > 0)
        CK(cudaMemcpyAsync(c->d_tr_save, c->d_tr, sizeof(D4) * c->n_tracers,
                           cudaMemcpyDeviceToDevice, c->stream));
    nrs_status worst = NRS_OK;
    const int64_t fact0 = c->factorizations;
    bool trained = false;
    if (report) report->mlp_rel_err = -1.0;
    for (int stage = 0; stage < 2; ++stage) {
        const nrs_shapes *s = stage ? sh : s0;
        bool need_factor = false;
        nrs_status st = prepare_stage(c, s, &need_factor);
        if (st != NRS_OK) return st;
        double *out = c->d_sol + (int64_t)stage * c->lda;
        const double *prev = c->have_sol ? c->d_sol + (int64_t)(1 - stage) * c->lda : nullptr;
        const double *vprev = (prev && c->F) ? prev + 3 * c->N : nullptr;
        const double *x0 = (c->warm_start && prev) ? prev : nullptr;
        int start = x0 ? 1 : 0;
        // learned starting guess: prediction or cold start, whichever has the smaller residual
        bool learned = false;
        if (c->mlp_predict && c->mlp_scales_set) {
            if (c->mlp_backoff > 0) {
                c->mlp_backoff -= 1;
            } else {
                learned = true;
                nrs::mlp_features(*c, (const D4 *)s->xi, (const D4 *)s->xidot, vprev, nullptr,
                                  c->d_mlp_x, nullptr);
                nrs::mlp_eval(*c, c->d_mlp_x, c->N, nullptr, c->d_mlp_y, nullptr, nullptr);
                nrs::mlp_start(*c, c->d_mlp_y, vprev, c->d_mlp_xp);
                CK(nrs::choose_start(*c, c->d_b, c->d_mlp_xp, c->d_mlp_xc, c->d_mlp_x0,
                                     c->d_mlp_scal + 3));
                CK(cudaMemcpyAsync(c->h_mlp_used, c->d_mlp_used, sizeof(int32_t) * 2,
                                   cudaMemcpyDeviceToHost, c->stream));
                x0 = c->d_mlp_x0;
                start = 0;
            }
        }
        int inner = 0;
        int retried = 0;
        st = solve_stage(c, out, x0, need_factor, report ? &report->stage[stage] : nullptr, &inner,
                         &retried);
        if (st == NRS_ECUDA) return st;
        if (report) report->retried[stage] = retried;
        if (st != NRS_OK && worst == NRS_OK) worst = st;
        // run_gmres_ir synchronised the stream: the pinned copy of the choice has landed
        if (learned && c->h_mlp_used[0]) {
            start = 2;
            if (c->cold_inner_cnt > 0 &&
                inner > c->cold_inner_sum / (double)c->cold_inner_cnt + 2.0)
                c->mlp_backoff = 8;
        }
        if (start == 0) {
            c->cold_inner_sum += inner;
            c->cold_inner_cnt += 1;
        }
        if (report) report->start[stage] = start;
        if (c->mlp_train_iters > 0 && st == NRS_OK) {
            if (!c->mlp_scales_set) {
                nrs::mlp_scales(*c, (const D4 *)s->xi, c->d_b, out, c->d_mlp_scal);
                c->mlp_scales_set = true;
            }
            nrs::mlp_features(*c, (const D4 *)s->xi, (const D4 *)s->xidot, vprev, out, c->d_mlp_x,
                              c->d_mlp_t);
            if (report) {  // error on this stage before training on it (held out)
                nrs::mlp_eval(*c, c->d_mlp_x, c->N, c->d_mlp_t, c->d_mlp_y, nullptr,
                              c->d_mlp_scal + 5);
                CK(cudaMemcpyAsync(c->h_mlp_loss, c->d_mlp_scal + 5, sizeof(double) * 2,
                                   cudaMemcpyDeviceToHost, c->stream));
                trained = true;
            }
            for (int it = 0; it < c->mlp_train_iters; ++it)
                nrs::mlp_train_step(*c, c->d_mlp_x, c->N, c->d_mlp_t, nullptr, c->mlp_lr);
        }
        c->last_inner = inner;
        c->have_sol = true;
        if (c->n_tracers > 0) {
            // tracers: the stage's velocity at their current positions, then
            // the explicit-midpoint update (x_half, then x_new)
            nrs::launch_velocity(*c, c->d_Xw, c->d_tr, c->n_tracers, out, c->d_tr_u, c->d_tr_part,
                                 c->stream);
            nrs::launch_tracer_update(*c, stage, dt, c->stream);
        }
        nrs::launch_rk2(*c, stage, dt, out);
        CK(cudaGetLastError());
    }
    if (sol) {
        CK(cudaMemcpyAsync(sol, c->d_sol, sizeof(double) * c->n, cudaMemcpyDeviceToDevice, c->stream));
        CK(cudaMemcpyAsync(sol + c->n, c->d_sol + c->lda, sizeof(double) * c->n,
                           cudaMemcpyDeviceToDevice, c->stream));
    }
    if (report) {
        CK(cudaEventRecord(ev1, c->stream));
        CK(cudaEventSynchronize(ev1));
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, ev0, ev1);
        report->ms_total = ms;
        report->factorizations = (int32_t)(c->factorizations - fact0);
        if (trained)
            report->mlp_rel_err = c->h_mlp_loss[1] > 0.0 ? sqrt(c->h_mlp_loss[0] / c->h_mlp_loss[1])
                                                         : 0.0;
        cudaEventDestroy(ev0);
        cudaEventDestroy(ev1);
    }
    return worst;
}

nrs_status nrs_set_timing(nrs_ctx *ctx, int32_t enable)
{
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c) return NRS_EINVAL;
    CK(cudaStreamSynchronize(c->stream));
    c->spans.clear();
    c->ev_used = 0;
    for (auto &e : c->open_ev) e = nullptr;
    c->timing = enable != 0;
    if (c->timing) c->launches = 0;
    return NRS_OK;
}

nrs_status nrs_get_trace(nrs_ctx *ctx, int32_t *phase, double *begin_ms, double *end_ms,
                         int64_t capacity, int64_t *count)
{
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c || capacity < 0) return NRS_EINVAL;
    CK(cudaStreamSynchronize(c->stream));
    const int64_t m = std::min<int64_t>(capacity, (int64_t)c->spans.size());
    for (int64_t i = 0; i < m; ++i) {
        const auto &s = c->spans[i];
        float t0 = 0.0f, t1 = 0.0f;
        CK(cudaEventElapsedTime(&t0, c->spans[0].a, s.a));
        CK(cudaEventElapsedTime(&t1, c->spans[0].a, s.b));
        if (phase) phase[i] = s.ph;
        if (begin_ms) begin_ms[i] = t0;
        if (end_ms) end_ms[i] = t1;
    }
    if (count) *count = (int64_t)c->spans.size();
    return NRS_OK;
}

nrs_status nrs_get_timing(nrs_ctx *ctx, double *ms, int64_t *spans, int64_t *launches)
{
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c) return NRS_EINVAL;
    CK(cudaStreamSynchronize(c->stream));
    double acc[nrs::NPH] = {};
    int64_t cnt[nrs::NPH] = {};
    for (const auto &s : c->spans) {
        float t = 0.0f;
        CK(cudaEventElapsedTime(&t, s.a, s.b));
        acc[s.ph] += t;
        cnt[s.ph] += 1;
    }
    if (ms)
        for (int i = 0; i < nrs::NPH; ++i) ms[i] = acc[i];
    if (spans)
        for (int i = 0; i < nrs::NPH; ++i) spans[i] = cnt[i];
    if (launches) *launches = c->launches;
    c->spans.clear();
    c->ev_used = 0;
    c->launches = 0;
    return NRS_OK;
}

nrs_status nrs_rank64_update(nrs_ctx *ctx, float *M, int64_t lda, int64_t n, const float *C,
                             const float *Rt, int32_t prec)
{
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c || !M || !C || !Rt || n <= 0 || lda < n || n > (1LL << 31))
        return fail(c, NRS_EINVAL, "nrs_rank64_update: bad argument");
    if ((reinterpret_cast<uintptr_t>(C) | reinterpret_cast<uintptr_t>(Rt)) & 15u)
        return fail(c, NRS_EINVAL, "nrs_rank64_update: panels must be 16-byte aligned");
    if (prec == NRS_FP32) {
        nrs::launch_simt_rank64(*c, M, lda, n, C, Rt);
    } else if (prec == NRS_TF32) {
        if (!nrs::tc_available() || !nrs::launch_tc_rank64(*c, M, lda, n, C, Rt, prec, -64, -64))
            return fail(c, NRS_EINVAL, "nrs_rank64_update: no tensor-core kernel on this device");
    } else {
        return fail(c, NRS_EINVAL, "nrs_rank64_update: precision must be NRS_FP32 or NRS_TF32");
    }
    CK(cudaGetLastError());
    return NRS_OK;
}

nrs_status nrs_mlp_set_params(nrs_ctx *ctx, const float *params, const float *adam_m,
                              const float *adam_v, int32_t t)
{
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c || !params || t < 0) return fail(c, NRS_EINVAL, "nrs_mlp_set_params: bad argument");
    nrs_status st = mlp_alloc(c);
    if (st != NRS_OK) return st;
    const size_t bytes = sizeof(float) * NRS_MLP_PARAMS;
    CK(cudaMemcpyAsync(c->d_mlp_params, params, bytes, cudaMemcpyHostToDevice, c->stream));
    if (adam_m) CK(cudaMemcpyAsync(c->d_mlp_m, adam_m, bytes, cudaMemcpyHostToDevice, c->stream));
    else CK(cudaMemsetAsync(c->d_mlp_m, 0, bytes, c->stream));
    if (adam_v) CK(cudaMemcpyAsync(c->d_mlp_v, adam_v, bytes, cudaMemcpyHostToDevice, c->stream));
    else CK(cudaMemsetAsync(c->d_mlp_v, 0, bytes, c->stream));
    CK(cudaStreamSynchronize(c->stream));  // the host arrays may be freed on return
    c->mlp_t = t;
    c->mlp_params_set = true;
    c->mlp_backoff = 0;
    return NRS_OK;
}

nrs_status nrs_mlp_get_params(nrs_ctx *ctx, float *params, float *adam_m, float *adam_v,
                              int32_t *t, double *scales)
{
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c) return NRS_EINVAL;
    if (!c->mlp_params_set) return fail(c, NRS_EINVAL, "nrs_mlp_get_params: no parameters set");
    const size_t bytes = sizeof(float) * NRS_MLP_PARAMS;
    CK(cudaStreamSynchronize(c->stream));
    if (params) CK(cudaMemcpy(params, c->d_mlp_params, bytes, cudaMemcpyDeviceToHost));
    if (adam_m) CK(cudaMemcpy(adam_m, c->d_mlp_m, bytes, cudaMemcpyDeviceToHost));
    if (adam_v) CK(cudaMemcpy(adam_v, c->d_mlp_v, bytes, cudaMemcpyDeviceToHost));
    if (t) *t = c->mlp_t;
    if (scales) CK(cudaMemcpy(scales, c->d_mlp_scal, sizeof(double) * 3, cudaMemcpyDeviceToHost));
    return NRS_OK;
}

nrs_status nrs_mlp_config(nrs_ctx *ctx, int32_t train_iters, int32_t predict, float lr,
                          const double *scales)
{
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c || train_iters < 0) return fail(c, NRS_EINVAL, "nrs_mlp_config: bad argument");
    if (!c->mlp_params_set) return fail(c, NRS_EINVAL, "nrs_mlp_config: no parameters set");
    if (train_iters > 0 && !(lr > 0.0f)) return fail(c, NRS_EINVAL, "nrs_mlp_config: lr <= 0");
    if (scales) {
        for (int k = 0; k < 3; ++k)
            if (!(scales[k] > 0.0) || !(scales[k] < 1e300))
                return fail(c, NRS_EINVAL, "nrs_mlp_config: scales must be positive and finite");
        CK(cudaMemcpyAsync(c->d_mlp_scal, scales, sizeof(double) * 3, cudaMemcpyHostToDevice,
                           c->stream));
        CK(cudaStreamSynchronize(c->stream));
        c->mlp_scales_set = true;
    }
    if (predict && !c->mlp_scales_set && train_iters == 0)
        return fail(c, NRS_EINVAL, "nrs_mlp_config: prediction needs scales or training");
    c->mlp_train_iters = train_iters;
    c->mlp_predict = predict ? 1 : 0;
    c->mlp_lr = lr;
    c->mlp_backoff = 0;
    return NRS_OK;
}

nrs_status nrs_mlp_eval(nrs_ctx *ctx, const float *X, const float *T, int64_t npts, float *Y,
                        float *G, double *loss)
{
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c || !X || !Y || npts <= 0) return fail(c, NRS_EINVAL, "nrs_mlp_eval: bad argument");
    if (!c->mlp_params_set) return fail(c, NRS_EINVAL, "nrs_mlp_eval: no parameters set");
    if (npts > c->N) return fail(c, NRS_EINVAL, "nrs_mlp_eval: npts exceeds the context's N");
    if ((G || loss) && !T) return fail(c, NRS_EINVAL, "nrs_mlp_eval: gradient or loss needs T");
    nrs::mlp_eval(*c, X, npts, T, Y, G, loss ? c->d_mlp_scal + 5 : nullptr);
    CK(cudaGetLastError());
    if (loss) {
        CK(cudaMemcpyAsync(c->h_mlp_loss, c->d_mlp_scal + 5, sizeof(double),
                           cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        *loss = *c->h_mlp_loss;
    }
    return NRS_OK;
}

nrs_status nrs_mlp_adam(nrs_ctx *ctx, const float *G, float lr)
{
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c || !G || !(lr > 0.0f)) return fail(c, NRS_EINVAL, "nrs_mlp_adam: bad argument");
    if (!c->mlp_params_set) return fail(c, NRS_EINVAL, "nrs_mlp_adam: no parameters set");
    nrs::mlp_adam(*c, G, lr);
    CK(cudaGetLastError());
    return NRS_OK;
}

nrs_status nrs_mlp_features(nrs_ctx *ctx, const nrs_shapes *s, const double *vprev,
                            const double *sol, float *X, float *T)
{
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c || !s || !s->xi || !s->xidot || !X || (T && !sol))
        return fail(c, NRS_EINVAL, "nrs_mlp_features: bad argument");
    if (!c->mlp_alloc || !c->mlp_scales_set)
        return fail(c, NRS_EINVAL, "nrs_mlp_features: scales not set");
    if (!c->assembled) return fail(c, NRS_EINVAL, "nrs_mlp_features before nrs_assemble");
    nrs::mlp_features(*c, (const D4 *)s->xi, (const D4 *)s->xidot, vprev, sol, X, T);
    CK(cudaGetLastError());
    return NRS_OK;
}

nrs_status nrs_mlp_start(nrs_ctx *ctx, const float *Y, const double *vprev, double *x0)
{
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c || !Y || !x0) return fail(c, NRS_EINVAL, "nrs_mlp_start: bad argument");
    if (!c->mlp_alloc || !c->mlp_scales_set)
        return fail(c, NRS_EINVAL, "nrs_mlp_start: scales not set");
    nrs::mlp_start(*c, Y, vprev, x0);
    CK(cudaGetLastError());
    return NRS_OK;
}

namespace {

void dp_fill(const Ctx *c, nrs_dp_info *info)
{
    if (!info) return;
    info->t = c->dp_t;
    info->h = c->dp_h;
    info->err = c->dp_err;
    info->stage = c->dp_stage;
    info->accepted = c->dp_accepted;
    info->rejected = c->dp_rejected;
    info->last_accepted = c->dp_last_accepted;
    info->done = c->dp_done;
}

// the next trial step: h grown or shrunk by 0.9 err^(-1/5) within [0.2, 5],
// clamped to [h_min, h_max] and to the end of the interval
double dp_next_h(const Ctx *c, double h, double err, bool accepted)
{
    double f = err > 0.0 && std::isfinite(err) ? 0.9 * std::pow(err, -0.2) : (err == 0.0 ? 5.0 : 0.2);
    f = std::min(accepted ? 5.0 : 1.0, std::max(0.2, f));
    double hn = std::min(c->dp_hmax, std::max(c->dp_hmin, h * f));
    return std::min(hn, c->dp_t_end - c->dp_t);
}

}  // namespace

nrs_status nrs_dp_start(nrs_ctx *ctx, double t0, double t_end, double h0, double rtol, double atol,
                        double h_min, double h_max)
{
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c) return NRS_EINVAL;
    if (!(t_end > t0) || !(h0 > 0.0) || !(rtol > 0.0) || !(atol >= 0.0) || !(h_min > 0.0) ||
        !(h_max >= h_min) || c->graph_mode)
        return fail(c, NRS_EINVAL, "nrs_dp_start: bad arguments (or a context in graph mode)");
    if (!c->d_dp_K) {
        if (cudaMalloc(&c->d_dp_K, sizeof(double) * 7 * 12 * c->nbodies) != cudaSuccess ||
            cudaMalloc(&c->d_dp_err, sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, NRS_ENOMEM, "Dormand-Prince workspace allocation failed");
        }
    }
    // Y_n = the context's state
    CK(cudaMemcpyAsync(c->d_x0_save, c->d_x0, sizeof(double) * 3 * c->nbodies,
                       cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpyAsync(c->d_B_save, c->d_B, sizeof(double) * 9 * c->nbodies,
                       cudaMemcpyDeviceToDevice, c->stream));
    c->dp_active = true;
    c->dp_t = t0;
    c->dp_t_end = t_end;
    c->dp_rtol = rtol;
    c->dp_atol = atol;
    c->dp_hmin = h_min;
    c->dp_hmax = h_max;
    c->dp_h = std::min(std::min(h0, h_max), t_end - t0);
    c->dp_stage = 0;
    c->dp_accepted = c->dp_rejected = c->dp_last_accepted = c->dp_done = 0;
    c->dp_err = 0.0;
    return NRS_OK;
}

nrs_status nrs_dp_next_time(const nrs_ctx *ctx, double *t_stage)
{
    const Ctx *c = reinterpret_cast<const Ctx *>(ctx);
    if (!c || !t_stage || !c->dp_active) return NRS_EINVAL;
    *t_stage = c->dp_t + nrs::dp_node(c->dp_stage) * c->dp_h;
    return NRS_OK;
}

nrs_status nrs_dp_info_get(const nrs_ctx *ctx, nrs_dp_info *info)
{
    const Ctx *c = reinterpret_cast<const Ctx *>(ctx);
    if (!c || !info) return NRS_EINVAL;
    dp_fill(c, info);
    return NRS_OK;
}

nrs_status nrs_dp_stage(nrs_ctx *ctx, const nrs_shapes *s, double *sol, nrs_dp_info *info)
{
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c || !s || !s->xi || !s->Xiw || !s->xidot) return fail(c, NRS_EINVAL, "nrs_dp_stage: null argument");
    if (!c->dp_active || c->dp_done) return fail(c, NRS_EINVAL, "nrs_dp_stage: no integration in progress");
    const int i = c->dp_stage;
    if (i >= 1) nrs::launch_dp_combine(*c, i, c->dp_h);  // the stage's state
    bool need_factor = false;
    nrs_status st = prepare_stage(c, s, &need_factor);
    if (st != NRS_OK) return st;
    double *out = c->d_sol + (int64_t)(i & 1) * c->lda;
    const double *prev = c->have_sol ? c->d_sol + (int64_t)(1 - (i & 1)) * c->lda : nullptr;
    const double *x0 = (c->warm_start && prev) ? prev : nullptr;
    int inner = 0, retried = 0;
    st = solve_stage(c, out, x0, need_factor, nullptr, &inner, &retried);
    if (st != NRS_OK) return st;
    c->last_inner = inner;
    c->have_sol = true;
    if (sol) CK(cudaMemcpyAsync(sol, out, sizeof(double) * c->n, cudaMemcpyDeviceToDevice, c->stream));
    nrs::launch_dp_rates(*c, i, out);
    CK(cudaGetLastError());
    if (i < 6) {
        c->dp_stage = i + 1;
        dp_fill(c, info);
        return NRS_OK;
    }
    // all seven stages: error estimate, accept or reject, next step size
    nrs::launch_dp_error(*c, c->dp_h, c->dp_rtol, c->dp_atol, c->d_dp_err);
    double err = 0.0;
    CK(cudaMemcpyAsync(&err, c->d_dp_err, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->dp_err = err;
    const bool ok = std::isfinite(err) && err <= 1.0;
    const int64_t nb = c->nbodies;
    if (ok) {
        // Y_n+1 = the last stage's state (first same as last: its rates are K_0 of the next step)
        c->dp_t += c->dp_h;
        CK(cudaMemcpyAsync(c->d_x0_save, c->d_x0, sizeof(double) * 3 * nb, cudaMemcpyDeviceToDevice,
                           c->stream));
        CK(cudaMemcpyAsync(c->d_B_save, c->d_B, sizeof(double) * 9 * nb, cudaMemcpyDeviceToDevice,
                           c->stream));
        CK(cudaMemcpyAsync(c->d_dp_K, c->d_dp_K + 6 * 12 * nb, sizeof(double) * 12 * nb,
                           cudaMemcpyDeviceToDevice, c->stream));
        c->dp_accepted += 1;
        c->dp_last_accepted = 1;
        if (c->dp_t >= c->dp_t_end * (1.0 - 1e-14) - 1e-300) c->dp_done = 1;
    } else {
        CK(cudaMemcpyAsync(c->d_x0, c->d_x0_save, sizeof(double) * 3 * nb, cudaMemcpyDeviceToDevice,
                           c->stream));
        CK(cudaMemcpyAsync(c->d_B, c->d_B_save, sizeof(double) * 9 * nb, cudaMemcpyDeviceToDevice,
                           c->stream));
        c->dp_rejected += 1;
        c->dp_last_accepted = 0;
    }
    const double h_old = c->dp_h;
    if (!c->dp_done) {
        c->dp_h = dp_next_h(c, h_old, err, ok);
        if (!ok && h_old <= c->dp_hmin * (1.0 + 1e-12)) {
            dp_fill(c, info);
            return fail(c, NRS_ENOCONV, "nrs_dp_stage: error above tolerance at the smallest step");
        }
    }
    c->dp_stage = 1;
    dp_fill(c, info);
    return NRS_OK;
}

nrs_status nrs_set_tracers(nrs_ctx *ctx, const double *xp, int64_t P)
{
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c) return NRS_EINVAL;
    if (P < 0 || (P > 0 && !xp)) return fail(c, NRS_EINVAL, "nrs_set_tracers: bad arguments");
    CK(cudaStreamSynchronize(c->stream));
    // a recorded step does not carry a changed tracer set: record it again
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
    void *old[] = {c->d_tr, c->d_tr_save, c->d_tr_u, c->d_tr_part};
    for (void *p : old)
        if (p) cudaFree(p);
    c->d_tr = c->d_tr_save = c->d_tr_u = nullptr;
    c->d_tr_part = nullptr;
    c->n_tracers = 0;
    if (P == 0) return NRS_OK;
    const size_t part = (size_t)nrs::velocity_splits(*c, P) * (size_t)P * 3;
    cudaError_t e = cudaMalloc(&c->d_tr, sizeof(D4) * P);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_tr_save, sizeof(D4) * P);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_tr_u, sizeof(D4) * P);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_tr_part, sizeof(double) * part);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, NRS_ENOMEM, "tracer workspace allocation failed");
    }
    CK(cudaMemcpy(c->d_tr, xp, sizeof(D4) * P, cudaMemcpyHostToDevice));
    c->n_tracers = P;
    return NRS_OK;
}

nrs_status nrs_get_tracers(nrs_ctx *ctx, double *xp)
{
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c) return NRS_EINVAL;
    if (c->n_tracers == 0) return NRS_OK;
    if (!xp) return fail(c, NRS_EINVAL, "nrs_get_tracers: null output");
    CK(cudaStreamSynchronize(c->stream));
    CK(cudaMemcpy(xp, c->d_tr, sizeof(D4) * c->n_tracers, cudaMemcpyDeviceToHost));
    return NRS_OK;
}

nrs_status nrs_velocity(nrs_ctx *ctx, const double *Xw, const double *xp, int64_t P, const double *f,
                        double *u)
{
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c) return NRS_EINVAL;
    if (P < 0 || (P > 0 && (!xp || !f || !u)))
        return fail(c, NRS_EINVAL, "nrs_velocity: bad arguments");
    if (!(c->nn_valid || c->map_built) || (!Xw && !c->kin_valid))
        return fail(c, NRS_EINVAL, "nrs_velocity: no nearest-neighbour map or quadrature points yet");
    const D4 *Xq = Xw ? reinterpret_cast<const D4 *>(Xw) : c->d_Xw;
    if (P == 0) return NRS_OK;
    const size_t need = (size_t)nrs::velocity_splits(*c, P) * (size_t)P * 3;
    if (need > c->vel_part_doubles) {
        CK(cudaStreamSynchronize(c->stream));
        if (c->d_vel_part) cudaFree(c->d_vel_part);
        c->d_vel_part = nullptr;
        c->vel_part_doubles = 0;
        if (cudaMalloc(&c->d_vel_part, sizeof(double) * need) != cudaSuccess) {
            cudaGetLastError();
            c->d_vel_part = nullptr;
            return fail(c, NRS_ENOMEM, "velocity workspace allocation failed");
        }
        c->vel_part_doubles = need;
    }
    nrs::launch_velocity(*c, Xq, reinterpret_cast<const D4 *>(xp), P, f, reinterpret_cast<D4 *>(u),
                         c->d_vel_part, c->stream);
    CK(cudaGetLastError());
    return NRS_OK;
}

nrs_status nrs_counters(const nrs_ctx *ctx, int64_t *factorizations, int64_t *solves,
                        int64_t *outer, int64_t *inner, int64_t *retries)
{
    const Ctx *c = reinterpret_cast<const Ctx *>(ctx);
    if (!c) return NRS_EINVAL;
    if (retries) *retries = c->retries;
    if (factorizations) *factorizations = c->factorizations;
    if (solves) *solves = c->solves;
    if (outer) *outer = c->outer_total;
    if (inner) *inner = c->inner_total;
    return NRS_OK;
}

nrs_status nrs_residual_counters(const nrs_ctx *ctx, int64_t *exact, int64_t *working)
{
    const Ctx *c = reinterpret_cast<const Ctx *>(ctx);
    if (!c) return NRS_EINVAL;
    if (exact) *exact = c->res_exact_total;
    if (working) *working = c->res_work_total;
    return NRS_OK;
}

nrs_status nrs_sync(nrs_ctx *ctx)
{
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c) return NRS_EINVAL;
    nrs::join_assembly(*c);
    CK(cudaStreamSynchronize(c->stream));
    int32_t st = 0;
    CK(cudaMemcpy(&st, c->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost));
    CK(cudaMemset(c->d_status, 0, sizeof(int32_t)));
    if (st & nrs::ST_TIMEOUT) return fail(c, NRS_ETIMEOUT, "a device wait ran out");
    if (st & nrs::ST_NONFINITE) return fail(c, NRS_ENONFINITE, "non-finite value");
    return NRS_OK;
}

}  // extern "C"
