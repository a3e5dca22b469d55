// batch.cu -- many independent problems of uneven size stepped together:
// the time steps of all problems recorded into ONE CUDA graph and replayed
// with one cudaGraphLaunch per batch step.
//
// The problems are split into K chains by longest-processing-time-first
// (LPT) on an estimate of each problem's step time; the problems of a chain
// run one after the other, the chains run concurrently (independent
// branches of the graph).  Each problem's refinement is one cooperative
// launch of G CTAs (gmres_persistent.cu).  K and G are chosen by measuring
// candidate plans on the device (nrs_batch_tune); the choice can be cached
// in a small text file keyed by the device and the problem sizes.  With
// K * G at most the co-resident CTA count of the solve kernel, the
// refinements of all chains fit on the device together, so no cooperative
// launch waits on another chain's.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <string>
#include <vector>

#include "nrs_internal.cuh"

using nrs::Ctx;

struct nrs_batch {
    std::vector<Ctx *> ctx;
    std::vector<cudaStream_t> streams;  // one per problem (owned)
    cudaStream_t stream = nullptr;      // the caller's stream
    cudaStream_t cap = nullptr;         // capture stream (owned)
    cudaEvent_t ev_fork = nullptr;
    std::vector<cudaEvent_t> ev;        // one per problem
    int num_sms = 0, max_coresident = 0;
    int chains = 1, grid = 0;
    std::vector<int32_t> chain_of, order;
    cudaGraphExec_t exec = nullptr;
    std::vector<const void *> key_ptrs;
    double key_dt = 0.0;
    bool key_berr = false;
    int64_t graph_launches = 0;
    std::string err;
};

namespace {

nrs_status bfail(nrs_batch *b, nrs_status s, const std::string &m)
{
    if (b) b->err = m;
    return s;
}

// Rough step time of one problem on GB300 (seconds): the Gauss-Jordan
// inverse moves n^3 / 8 bytes twice per step at about 2.3 TB/s, the FP64
// assembly evaluates N Q pairs twice per step at about 1.4e10 pairs/s.
double step_cost(const Ctx &c)
{
    const double n = (double)c.n;
    return 2.0 * (n * n * n / 8.0 / 2.3e12 + (double)c.N * (double)c.Q / 1.4e10);
}

void plan_lpt(const std::vector<double> &cost, int chains, std::vector<int32_t> &chain_of,
              std::vector<int32_t> &order)
{
    const int count = (int)cost.size();
    order.resize(count);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int32_t a, int32_t b) { return cost[a] > cost[b]; });
    std::vector<double> load(chains, 0.0);
    chain_of.assign(count, 0);
    for (int32_t i : order) {
        int best = 0;
        for (int k = 1; k < chains; ++k)
            if (load[k] < load[best]) best = k;
        chain_of[i] = best;
        load[best] += cost[i];
    }
}

void drop_graph(nrs_batch *b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    b->key_ptrs.clear();
}

nrs_status apply_config(nrs_batch *b, int chains, int grid)
{
    const int count = (int)b->ctx.size();
    if (chains < 1 || chains > count || grid < 1 || (int64_t)chains * grid > b->max_coresident)
        return bfail(b, NRS_EINVAL, "nrs_batch_config: need 1 <= chains <= count and "
                                    "chains * grid <= co-resident solve CTAs");
    b->chains = chains;
    b->grid = grid;
    std::vector<double> cost(count);
    for (int i = 0; i < count; ++i) cost[i] = step_cost(*b->ctx[i]);
    plan_lpt(cost, chains, b->chain_of, b->order);
    for (Ctx *c : b->ctx) c->pg_grid = grid;
    drop_graph(b);
    return NRS_OK;
}

nrs_status record(nrs_batch *b, const nrs_shapes *s0, const nrs_shapes *sh, double dt, bool berr)
{
    const int count = (int)b->ctx.size();
    drop_graph(b);
    cudaGraph_t g = nullptr;
    int64_t l0 = 0;
    for (Ctx *c : b->ctx) l0 += c->launches;
    cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    nrs_status st = e == cudaSuccess ? NRS_OK : NRS_ECUDA;
    if (st == NRS_OK) e = cudaEventRecord(b->ev_fork, b->cap);
    std::vector<int32_t> last(b->chains, -1);
    for (int32_t i : b->order) {
        if (st != NRS_OK || e != cudaSuccess) break;
        Ctx *c = b->ctx[i];
        const int k = b->chain_of[i];
        e = cudaStreamWaitEvent(c->stream, last[k] < 0 ? b->ev_fork : b->ev[last[k]], 0);
        if (e != cudaSuccess) break;
        st = nrs::enqueue_step(c, s0 + i, sh + i, dt, c->d_step_stats, berr);
        if (st != NRS_OK) break;
        e = cudaEventRecord(b->ev[i], c->stream);
        last[k] = i;
    }
    for (int k = 0; k < b->chains && st == NRS_OK && e == cudaSuccess; ++k)
        if (last[k] >= 0) e = cudaStreamWaitEvent(b->cap, b->ev[last[k]], 0);
    cudaError_t e2 = cudaStreamEndCapture(b->cap, &g);
    int64_t l1 = 0;
    for (Ctx *c : b->ctx) l1 += c->launches;
    if (st != NRS_OK || e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return bfail(b, st != NRS_OK ? st : NRS_ECUDA,
                     std::string("recording the batch graph failed: ") +
                         cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    e = cudaGraphInstantiate(&b->exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        b->exec = nullptr;
        return bfail(b, NRS_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    }
    // the launches counted while recording are the kernels of one replay
    b->graph_launches = l1 - l0;
    for (int i = 0; i < count; ++i) {
        b->key_ptrs.push_back(s0[i].xi);
        b->key_ptrs.push_back(s0[i].Xiw);
        b->key_ptrs.push_back(s0[i].xidot);
        b->key_ptrs.push_back(sh[i].xi);
        b->key_ptrs.push_back(sh[i].Xiw);
        b->key_ptrs.push_back(sh[i].xidot);
    }
    b->key_dt = dt;
    b->key_berr = berr;
    return NRS_OK;
}

bool key_matches(const nrs_batch *b, const nrs_shapes *s0, const nrs_shapes *sh, double dt,
                 bool berr)
{
    if (!b->exec || b->key_dt != dt || b->key_berr != berr) return false;
    const size_t count = b->ctx.size();
    if (b->key_ptrs.size() != 6 * count) return false;
    for (size_t i = 0; i < count; ++i) {
        const void *p[6] = {s0[i].xi, s0[i].Xiw, s0[i].xidot, sh[i].xi, sh[i].Xiw, sh[i].xidot};
        for (int k = 0; k < 6; ++k)
            if (b->key_ptrs[6 * i + k] != p[k]) return false;
    }
    return true;
}

std::string tune_key(const nrs_batch *b)
{
    cudaDeviceProp prop{};
    int dev = 0;
    cudaGetDevice(&dev);
    cudaGetDeviceProperties(&prop, dev);
    std::vector<int64_t> ns;
    for (const Ctx *c : b->ctx) ns.push_back(c->n);
    std::sort(ns.begin(), ns.end());
    uint64_t h = 1469598103934665603ull;  // FNV-1a over the sorted sizes
    for (int64_t v : ns)
        for (int k = 0; k < 8; ++k) {
            h ^= (uint64_t)((v >> (8 * k)) & 0xff);
            h *= 1099511628211ull;
        }
    char buf[256];
    snprintf(buf, sizeof(buf), "sm%d%d-%dsm-count%zu-sizes%016llx", prop.major, prop.minor,
             prop.multiProcessorCount, ns.size(), (unsigned long long)h);
    std::string k(buf);
    for (char &ch : k)
        if (ch == ' ') ch = '_';
    return k;
}

// The cache is a text file of lines "<key> <chains> <grid> <ms>".
bool cache_lookup(const char *path, const std::string &key, int *chains, int *grid)
{
    if (!path) return false;
    FILE *f = fopen(path, "r");
    if (!f) return false;
    char k[256];
    int ch = 0, gr = 0;
    double ms = 0.0;
    bool found = false;
    while (fscanf(f, "%255s %d %d %lf", k, &ch, &gr, &ms) == 4)
        if (key == k) {
            *chains = ch;
            *grid = gr;
            found = true;
        }
    fclose(f);
    return found;
}

void cache_store(const char *path, const std::string &key, int chains, int grid, double ms)
{
    if (!path) return;
    FILE *f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s %d %d %.6f\n", key.c_str(), chains, grid, ms);
    fclose(f);
}

}  // namespace

extern "C" {

nrs_status nrs_batch_plan(const double *cost, int32_t count, int32_t chains, int32_t *chain_of,
                          int32_t *order)
{
    if (!cost || count <= 0 || chains <= 0 || !chain_of || !order) return NRS_EINVAL;
    std::vector<double> c(cost, cost + count);
    std::vector<int32_t> ch, ord;
    plan_lpt(c, chains, ch, ord);
    std::copy(ch.begin(), ch.end(), chain_of);
    std::copy(ord.begin(), ord.end(), order);
    return NRS_OK;
}

nrs_status nrs_batch_create(nrs_batch **out, const nrs_problem_desc *descs, int32_t count,
                            void *stream)
{
    if (!out || !descs || count <= 0) return NRS_EINVAL;
    *out = nullptr;
    for (int i = 0; i < count; ++i) {
        const nrs_problem_desc &d = descs[i];
        if (d.factor_prec == NRS_FP64 || d.solve_mode != 0 || d.reuse_factor ||
            d.max_inner > 64)
            return NRS_EINVAL;
    }
    nrs_batch *b = new (std::nothrow) nrs_batch();
    if (!b) return NRS_ENOMEM;
    b->stream = (cudaStream_t)stream;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev);
    nrs_status st = NRS_OK;
    cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
    for (int i = 0; i < count && e == cudaSuccess && st == NRS_OK; ++i) {
        cudaStream_t s = nullptr;
        e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e != cudaSuccess) break;
        b->streams.push_back(s);
        cudaEvent_t ev = nullptr;
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e != cudaSuccess) break;
        b->ev.push_back(ev);
        nrs_problem_desc d = descs[i];
        d.graph = 0;
        // the problems of a batch run side by side: the fused factorisation,
        // one cooperative launch taking every SM, would serialise them; the
        // automatic choice stays (two-level from n = 8192 on: its update CTAs
        // claim their tiles dynamically, so they share the SMs with the other
        // chains' kernels instead of waiting for all of them)
        if (d.factor_schedule == 1) d.factor_schedule = 2;
        nrs_ctx *h = nullptr;
        st = nrs_create(&h, &d, s);
        if (st == NRS_OK) {
            b->ctx.push_back(reinterpret_cast<Ctx *>(h));
            b->ctx.back()->pg_shared = true;
        }
    }
    if (e != cudaSuccess && st == NRS_OK) st = NRS_ECUDA;
    if (st == NRS_OK) {
        b->max_coresident = nrs::pg_max_coresident(*b->ctx[0]);
        const int chains = std::min(count, 4);
        st = apply_config(b, chains, std::max(1, std::min(b->num_sms, b->max_coresident / chains)));
    }
    if (st != NRS_OK) {
        nrs_batch_destroy(b);
        return st;
    }
    *out = b;
    return NRS_OK;
}

nrs_status nrs_batch_destroy(nrs_batch *b)
{
    if (!b) return NRS_EINVAL;
    if (b->stream) cudaStreamSynchronize(b->stream);
    drop_graph(b);
    for (Ctx *c : b->ctx) nrs_destroy(reinterpret_cast<nrs_ctx *>(c));
    for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
    return NRS_OK;
}

const char *nrs_batch_last_error(const nrs_batch *b) { return b ? b->err.c_str() : ""; }

nrs_status nrs_batch_info(const nrs_batch *b, int32_t *chains, int32_t *grid, int64_t *graph_kernels)
{
    if (!b) return NRS_EINVAL;
    if (chains) *chains = b->chains;
    if (grid) *grid = b->grid;
    if (graph_kernels) *graph_kernels = b->exec ? b->graph_launches : 0;
    return NRS_OK;
}

nrs_status nrs_batch_context(nrs_batch *b, int32_t i, nrs_ctx **ctx)
{
    if (!b || !ctx || i < 0 || i >= (int32_t)b->ctx.size()) return NRS_EINVAL;
    *ctx = reinterpret_cast<nrs_ctx *>(b->ctx[i]);
    return NRS_OK;
}

nrs_status nrs_batch_config(nrs_batch *b, int32_t chains, int32_t grid, int32_t *chain_of)
{
    if (!b) return NRS_EINVAL;
    nrs_status st = apply_config(b, chains, grid);
    if (st == NRS_OK && chain_of) std::copy(b->chain_of.begin(), b->chain_of.end(), chain_of);
    return st;
}

nrs_status nrs_batch_step(nrs_batch *b, const nrs_shapes *s0, const nrs_shapes *sh, double dt,
                          double *const *sol, nrs_step_report *reports)
{
    if (!b || !s0 || !sh || !(dt > 0.0)) return bfail(b, NRS_EINVAL, "nrs_batch_step: bad argument");
    const int count = (int)b->ctx.size();
    for (int i = 0; i < count; ++i)
        if (!s0[i].xi || !s0[i].Xiw || !s0[i].xidot || !sh[i].xi || !sh[i].Xiw || !sh[i].xidot)
            return bfail(b, NRS_EINVAL, "nrs_batch_step: null shape pointer");
    bool capable = true;
    for (Ctx *c : b->ctx) capable = capable && nrs::graph_capable(*c);
    const bool berr = reports != nullptr;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if (reports) {
        if (cudaEventCreate(&t0) != cudaSuccess || cudaEventCreate(&t1) != cudaSuccess)
            return bfail(b, NRS_ECUDA, "cudaEventCreate");
        cudaEventRecord(t0, b->stream);
    }
    nrs_status worst = NRS_OK;
    if (!capable) {
        // first step (nearest-neighbour maps of the rigid bodies) or an option
        // that needs the eager step: each problem on its own stream, ordered
        // after the caller's stream and joined back into it
        if (cudaEventRecord(b->ev_fork, b->stream) != cudaSuccess)
            return bfail(b, NRS_ECUDA, "cudaEventRecord");
        for (int32_t i : b->order) {
            Ctx *c = b->ctx[i];
            cudaStreamWaitEvent(c->stream, b->ev_fork, 0);
            nrs_status st = nrs_step(reinterpret_cast<nrs_ctx *>(c), s0 + i, sh + i, dt,
                                     sol ? sol[i] : nullptr, reports ? reports + i : nullptr);
            if (st == NRS_ECUDA || st == NRS_EINVAL) return bfail(b, st, c->err);
            if (st != NRS_OK && worst == NRS_OK) worst = st;
            cudaEventRecord(b->ev[i], c->stream);
            cudaStreamWaitEvent(b->stream, b->ev[i], 0);
        }
    } else {
        if (!key_matches(b, s0, sh, dt, berr)) {
            nrs_status st = record(b, s0, sh, dt, berr);
            if (st != NRS_OK) return st;
        }
        if (cudaGraphLaunch(b->exec, b->stream) != cudaSuccess)
            return bfail(b, NRS_ECUDA, "cudaGraphLaunch");
        for (int i = 0; i < count; ++i) {
            Ctx *c = b->ctx[i];
            c->have_sol = true;
            c->factorizations += 2;
            if (sol && sol[i]) {
                cudaMemcpyAsync(sol[i], c->d_sol, sizeof(double) * c->n, cudaMemcpyDeviceToDevice,
                                b->stream);
                cudaMemcpyAsync(sol[i] + c->n, c->d_sol + c->lda, sizeof(double) * c->n,
                                cudaMemcpyDeviceToDevice, b->stream);
            }
        }
        if (reports) {
            if (cudaStreamSynchronize(b->stream) != cudaSuccess)
                return bfail(b, NRS_ECUDA, "cudaStreamSynchronize");
            for (int i = 0; i < count; ++i) {
                Ctx *c = b->ctx[i];
                double q[16];
                int32_t word = 0;
                cudaMemcpy(q, c->d_step_stats, sizeof(q), cudaMemcpyDeviceToHost);
                cudaMemcpy(&word, c->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost);
                cudaMemset(c->d_status, 0, sizeof(int32_t));
                nrs_step_report &r = reports[i];
                r.retried[0] = r.retried[1] = 0;
                for (int k = 0; k < 2; ++k) {
                    const double *s = q + 8 * k;
                    nrs_solve_report &sr = r.stage[k];
                    sr.outer = (int32_t)s[0];
                    sr.inner = (int32_t)s[1];
                    sr.converged = s[2] != 0.0;
                    sr.last_update = s[4] > 0 ? s[3] / s[4] : 0.0;
                    sr.backward_err = s[5] / (s[6] * s[4] + s[7]);
                    sr.status = (word & nrs::ST_TIMEOUT)     ? NRS_ETIMEOUT
                                : (word & nrs::ST_NONFINITE) ? NRS_ENONFINITE
                                : !sr.converged              ? NRS_ENOCONV
                                                             : NRS_OK;
                    if (sr.status != NRS_OK && worst == NRS_OK) worst = (nrs_status)sr.status;
                    r.start[k] = c->warm_start ? 1 : 0;
                }
                r.factorizations = 2;
                r.mlp_rel_err = -1.0;
                r.ms_total = 0.0;
            }
        }
    }
    if (reports) {
        cudaEventRecord(t1, b->stream);
        cudaEventSynchronize(t1);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, t0, t1);
        for (int i = 0; i < count; ++i) reports[i].ms_total = ms;
        cudaEventDestroy(t0);
        cudaEventDestroy(t1);
    }
    if (worst != NRS_OK) b->err = "a problem of the batch did not converge cleanly";
    return worst;
}

nrs_status nrs_batch_tune(nrs_batch *b, const nrs_shapes *s0, const nrs_shapes *sh, double dt,
                          const char *cache_path, int32_t *chains_out, int32_t *grid_out,
                          double *ms_out)
{
    if (!b || !s0 || !sh || !(dt > 0.0)) return bfail(b, NRS_EINVAL, "nrs_batch_tune: bad argument");
    for (Ctx *c : b->ctx)
        if (!nrs::graph_capable(*c))
            return bfail(b, NRS_EINVAL, "nrs_batch_tune: take one nrs_batch_step first");
    const int count = (int)b->ctx.size();
    const std::string key = tune_key(b);
    int best_k = 0, best_g = 0;
    double best_ms = -1.0;
    if (cache_lookup(cache_path, key, &best_k, &best_g) &&
        apply_config(b, best_k, best_g) == NRS_OK) {
        if (chains_out) *chains_out = best_k;
        if (grid_out) *grid_out = best_g;
        if (ms_out) *ms_out = -1.0;
        return NRS_OK;
    }
    // save every problem's state; each trial restores it before it runs
    std::vector<double *> save(count, nullptr);
    for (int i = 0; i < count; ++i) {
        Ctx *c = b->ctx[i];
        const size_t bytes = sizeof(double) * (12 * c->nbodies + 2 * c->lda);
        if (cudaMalloc(&save[i], bytes) != cudaSuccess) {
            for (double *p : save)
                if (p) cudaFree(p);
            return bfail(b, NRS_ENOMEM, "nrs_batch_tune: state copy does not fit");
        }
        cudaMemcpyAsync(save[i], c->d_x0, sizeof(double) * 3 * c->nbodies, cudaMemcpyDeviceToDevice,
                        b->stream);
        cudaMemcpyAsync(save[i] + 3 * c->nbodies, c->d_B, sizeof(double) * 9 * c->nbodies,
                        cudaMemcpyDeviceToDevice, b->stream);
        cudaMemcpyAsync(save[i] + 12 * c->nbodies, c->d_sol, sizeof(double) * 2 * c->lda,
                        cudaMemcpyDeviceToDevice, b->stream);
    }
    auto restore = [&]() {
        for (int i = 0; i < count; ++i) {
            Ctx *c = b->ctx[i];
            cudaMemcpyAsync(c->d_x0, save[i], sizeof(double) * 3 * c->nbodies,
                            cudaMemcpyDeviceToDevice, b->stream);
            cudaMemcpyAsync(c->d_B, save[i] + 3 * c->nbodies, sizeof(double) * 9 * c->nbodies,
                            cudaMemcpyDeviceToDevice, b->stream);
            cudaMemcpyAsync(c->d_sol, save[i] + 12 * c->nbodies, sizeof(double) * 2 * c->lda,
                            cudaMemcpyDeviceToDevice, b->stream);
        }
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int ks[] = {1, 2, 4, 8, 16};
    const int gdiv[] = {1, 2, 4};
    nrs_status st = NRS_OK;
    for (int k : ks) {
        if (k > count) break;
        for (int gd : gdiv) {
            const int g = std::min(b->num_sms / gd, b->max_coresident / k);
            if (g < 1 || apply_config(b, k, g) != NRS_OK) continue;
            restore();
            st = nrs_batch_step(b, s0, sh, dt, nullptr, nullptr);  // records and warms up
            if (st != NRS_OK) break;
            restore();
            cudaEventRecord(e0, b->stream);
            st = nrs_batch_step(b, s0, sh, dt, nullptr, nullptr);
            cudaEventRecord(e1, b->stream);
            cudaEventSynchronize(e1);
            if (st != NRS_OK) break;
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (best_ms < 0.0 || ms < best_ms) {
                best_ms = ms;
                best_k = k;
                best_g = g;
            }
        }
        if (st != NRS_OK) break;
    }
    restore();
    cudaStreamSynchronize(b->stream);
    for (double *p : save) cudaFree(p);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != NRS_OK) return st;
    if (best_ms < 0.0) return bfail(b, NRS_EINVAL, "nrs_batch_tune: no valid plan");
    apply_config(b, best_k, best_g);
    cache_store(cache_path, key, best_k, best_g, best_ms);
    if (chains_out) *chains_out = best_k;
    if (grid_out) *grid_out = best_g;
    if (ms_out) *ms_out = best_ms;
    return NRS_OK;
}

}  // extern "C"
