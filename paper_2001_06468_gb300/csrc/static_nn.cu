// static_nn.cu -- nrs_nearest_build_static: nearest neighbours and segments of
// nu without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need the
// nearest-neighbour map: code that runs inside a memory pool or arena it does
// not control, a time-critical loop in which cudaMalloc/cudaFree would
// synchronise the device, or a process that reserved all device memory up
// front.  This entry point takes the caller's inputs and outputs and keeps its
// scratch (segment counters and cursors, the block task table, the body
// offsets and a status word) in file-scope __device__ arrays of a fixed size,
// which every GPU that loads the library holds until the process exits.
//
// The kernels are the ones nrs_nearest_build runs (geometry.cu); nothing in
// that path changes.
#include <mutex>

#include "nrs_internal.cuh"

namespace nrs {

// kernels defined in geometry.cu
__global__ void k_nearest(const NNTask *tasks, const int64_t *n_off, int nbodies, int global,
                          const D4 *x, const D4 *X, int32_t *nn, int32_t *status);
__global__ void k_count(int64_t Q, int64_t N, const int32_t *nn, int32_t *cnt);
__global__ void k_scan(int64_t N, const int32_t *cnt, int32_t *seg_ptr, int32_t *cursor);
__global__ void k_scatter(int64_t Q, int64_t N, const int32_t *nn, int32_t *cursor, int32_t *perm);
__global__ void k_sort_segments(int64_t N, const int32_t *seg_ptr, int32_t *perm);

namespace {

constexpr int64_t kMaxN = NRS_STATIC_MAX_N;
constexpr int64_t kMaxQ = NRS_STATIC_MAX_Q;
constexpr int kMaxBodies = NRS_STATIC_MAX_BODIES;
constexpr int64_t kMaxTasks = kMaxQ / NN_QPB + kMaxBodies;

// The scratch.  Host code must not pass these names to a kernel: on the host
// they are stand-ins, not device addresses.  Their device addresses come from
// cudaGetSymbolAddress (setup_device below).
static __device__ __align__(256) int32_t g_cursor[kMaxN + 1];
static __device__ __align__(256) NNTask g_tasks[kMaxTasks];
static __device__ __align__(256) int64_t g_n_off[kMaxBodies + 1];
static __device__ __align__(256) int64_t g_q_off[kMaxBodies + 1];
static __device__ __align__(256) int32_t g_status[1];

struct DevScratch {
    bool ready = false;
    int32_t *cursor = nullptr;
    NNTask *tasks = nullptr;
    int64_t *n_off = nullptr;
    int64_t *q_off = nullptr;
    int32_t *status = nullptr;
};

constexpr int kMaxDevices = 64;
DevScratch g_dev[kMaxDevices];
std::mutex g_mu;

// Device addresses of the scratch for the current device (looked up once per
// device, with that device current).
cudaError_t setup_device(int dev, DevScratch **out)
{
    std::lock_guard<std::mutex> lock(g_mu);
    DevScratch &s = g_dev[dev];
    if (!s.ready) {
        cudaError_t e;
        if ((e = cudaGetSymbolAddress((void **)&s.cursor, g_cursor)) != cudaSuccess) return e;
        if ((e = cudaGetSymbolAddress((void **)&s.tasks, g_tasks)) != cudaSuccess) return e;
        if ((e = cudaGetSymbolAddress((void **)&s.n_off, g_n_off)) != cudaSuccess) return e;
        if ((e = cudaGetSymbolAddress((void **)&s.q_off, g_q_off)) != cudaSuccess) return e;
        if ((e = cudaGetSymbolAddress((void **)&s.status, g_status)) != cudaSuccess) return e;
        s.ready = true;
    }
    *out = &s;
    return cudaSuccess;
}

// Block tasks (NN_QPB quadrature points of one body each) from the body offsets,
// written by one thread into the static task table.
__global__ void k_static_tasks(int nbodies, const int64_t *__restrict__ q_off,
                               NNTask *__restrict__ tasks)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    int64_t t = 0;
    for (int b = 0; b < nbodies; ++b)
        for (int64_t q0 = q_off[b]; q0 < q_off[b + 1]; q0 += NN_QPB)
            tasks[t++] = NNTask{b, (int32_t)q0, (int32_t)min(q0 + NN_QPB, q_off[b + 1]), 0};
}

}  // namespace
}  // namespace nrs

extern "C" nrs_status nrs_nearest_build_static(const double *x, const double *Xw, int32_t nbodies,
                                               const int64_t *n_off, const int64_t *q_off,
                                               int32_t global, int32_t *nn, int32_t *seg_ptr,
                                               int32_t *perm, int32_t *status, void *stream)
{
    using namespace nrs;
    if (!x || !Xw || !n_off || !q_off || !nn || !seg_ptr || !perm) return NRS_EINVAL;
    if (nbodies <= 0 || nbodies > kMaxBodies) return NRS_EINVAL;
    if (n_off[0] != 0 || q_off[0] != 0) return NRS_EINVAL;
    int64_t ntasks = 0;
    for (int b = 0; b < nbodies; ++b) {
        if (n_off[b + 1] < n_off[b] || q_off[b + 1] < q_off[b]) return NRS_EINVAL;
        if (!global && q_off[b + 1] > q_off[b] && n_off[b + 1] == n_off[b]) return NRS_EINVAL;
        ntasks += (q_off[b + 1] - q_off[b] + NN_QPB - 1) / NN_QPB;
    }
    const int64_t N = n_off[nbodies], Q = q_off[nbodies];
    if (N <= 0 || Q <= 0 || N > kMaxN || Q > kMaxQ || ntasks > kMaxTasks) return NRS_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return NRS_ECUDA;
    DevScratch *s = nullptr;
    if (setup_device(dev, &s) != cudaSuccess) return NRS_ECUDA;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t ob = sizeof(int64_t) * (nbodies + 1);
    if (cudaMemcpyAsync(s->n_off, n_off, ob, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(s->q_off, q_off, ob, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return NRS_ECUDA;
    // the shared scratch keeps the previous call's contents: clear what must start at zero
    if (cudaMemsetAsync(s->status, 0, sizeof(int32_t), st) != cudaSuccess ||
        cudaMemsetAsync(s->cursor, 0, sizeof(int32_t) * (N + 1), st) != cudaSuccess ||
        cudaMemsetAsync(perm, 0, sizeof(int32_t) * Q, st) != cudaSuccess)
        return NRS_ECUDA;
    k_static_tasks<<<1, 1, 0, st>>>(nbodies, s->q_off, s->tasks);
    k_nearest<<<(unsigned)ntasks, NN_THREADS, 0, st>>>(s->tasks, s->n_off, nbodies, global ? 1 : 0,
                                                 (const D4 *)x, (const D4 *)Xw, nn, s->status);
    const int threads = 256;
    k_count<<<(unsigned)ceil_div(Q, threads), threads, 0, st>>>(Q, N, nn, s->cursor);
    k_scan<<<1, 1024, 0, st>>>(N, s->cursor, seg_ptr, s->cursor);
    k_scatter<<<(unsigned)ceil_div(Q, threads), threads, 0, st>>>(Q, N, nn, s->cursor, perm);
    k_sort_segments<<<(unsigned)ceil_div(N, threads), threads, 0, st>>>(N, seg_ptr, perm);
    if (cudaGetLastError() != cudaSuccess) return NRS_ECUDA;
    // the device status word (ST_NONFINITE: a non-finite coordinate; those
    // quadrature points have nn < 0 and belong to no segment) to the caller's
    // word, in stream order, before a later call clears the shared one
    if (status &&
        cudaMemcpyAsync(status, s->status, sizeof(int32_t), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return NRS_ECUDA;
    return NRS_OK;
}
