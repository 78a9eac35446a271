// C ABI of libpwa: context, device store, and the per-call path of the
// likelihood (declared and documented in include/pwa.h).
//
// Per call only the parameters cross to the device and only the likelihood
// and gradient come back (Sec. 5): V is staged in pinned memory, copied in
// one transfer together with a zeroed status word, the fused kernel runs,
// and one transfer brings back [nll | grad | status].
#include <cudaTypedefs.h>

#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <numeric>
#include <string>
#include <vector>

#include <cmath>

#include "pwa_internal.cuh"

using namespace pwa;

struct pwa_ctx {
    int device = 0;
    pwa_config cfg{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int num_sms = 0;
    int N = 0;
    int form = PWA_FORM_AMP;

    // sample
    int64_t n_data = 0, n_mc = 0;
    double n_gen = 0;
    Planes data{}, mc{};
    float *table = nullptr;
    int64_t table_pitch = 0;
    float *tmax = nullptr;  // [N^2] max over events of |t_p|
    void *xbf = nullptr;    // BF16 slices of the data in 64-event blocks (tensor-core form)
    long long *xsum = nullptr;  // sum of the per-event exponents (inside xbf)
    int xs = 2;                 // BF16 slices of the amplitudes (tensor-core form)
    int n_lambda = 1;           // incoherent components per event (data planes hold L N waves)
    bool incoh_tma = false;     // incoherent direct form through the TMA-fed kernel
    int tune_groups = 0;        // direct form: consumer groups (0 = default rule)
    int tune_tc_nxs = 0;        // tensor-core form: X stages (0 = as many as fit)
    int tune_tc_per = 0;        // tensor-core form: sets per launch (0 = the even split)
    // host evaluations replayed as CUDA graphs (copy in, kernels, copy out),
    // one per (K, with gradient); stale once `epoch` moves (a new sample, form
    // or launch shape)
    struct EvalGraph {
        int K;
        bool grad;
        unsigned epoch;
        cudaGraphExec_t exec;
    };
    std::vector<EvalGraph> graphs;
    unsigned epoch = 0;
    bool graphs_off = false;
    int tune_res_cps = 1;       // free-resonance kernel: blocks per SM
    // free-resonance form
    float *res_data = nullptr, *res_mc = nullptr;
    int64_t res_data_pitch = 0, res_mc_pitch = 0, res_n_data = 0, res_n_mc = 0;
    int res_R = 0;
    double res_ngen = 0.0;
    bool res_loaded = false;
    bool res_tma = false;       // the TMA-fed free-resonance kernel serves this sample
    CUtensorMap res_dmap, res_mmap;
    float *res_amax = nullptr;  // [N] max over both samples of |Y_a|_1 or |A_a|_1
    double *d_res = nullptr;    // partials, ticket, io
    double *h_res = nullptr;    // pinned io mirror
    // Hessian, projection weights, fit fractions (allocated on first use)
    double *d_fx = nullptr;     // V [2N] | status [1] | out [4N^2] | Hessian partials
    double *h_fx = nullptr;     // pinned mirror of V | status | out
    size_t fx_bytes = 0;
    float *d_w = nullptr;       // projection weights when the caller's buffer is on the host
    int64_t w_len = 0;
    CUtensorMap data_map, table_map;
    size_t work_bytes = 0;
    bool loaded = false, has_norm = false;
    double *M = nullptr;     // [N][N] complex
    float *amax = nullptr;   // [N] max over data events of |Re A_a| + |Im A_a|
    float *mc_amax = nullptr;  // [N] the same over the accepted MC events (projection weights)
    CUtensorMap mc_map;        // over the MC planes, as data_map over the data
    CUtensorMap hess_map;      // over the data planes, tiles of the tensor-core Hessian
    bool hess_tc = false;      // hess_map is set: the tensor-core Hessian serves this sample

    // per-call buffers
    double *d_io = nullptr;  // [nll K | grad 2NK | status,done | V 2NK]
    double *h_io = nullptr;  // pinned mirror (and, at io_flags_at, max_k result flags)
    double *h_io_dev = nullptr;  // h_io as a device address (null: not mapped)
    int *zc_status = nullptr;    // device word the zero-copy launches OR their status into
    unsigned zc_seq = 0;         // sequence number of the last zero-copy call
    double *d_work = nullptr;  // partials + work flag, then ticket and async status
    unsigned *ticket = nullptr;
    int *async_status = nullptr;

    char err[512] = {0};
};

namespace {

thread_local char g_create_err[512];

int fail(pwa_ctx *ctx, int code, const char *fmt, ...)
{
    char *buf = ctx ? ctx->err : g_create_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, 512, fmt, ap);
    va_end(ap);
    return code;
}

// Host-side fault injection for tests of the error paths: PWA_FAULT=alloc:N
// makes the N-th device allocation of the process fail (no GPU state is
// touched by the failure itself).
std::atomic<long> g_alloc_count{0};

bool injected_alloc_failure()
{
    static long target = [] {
        const char *f = getenv("PWA_FAULT");
        if (f && strncmp(f, "alloc:", 6) == 0)
            return atol(f + 6);
        return 0L;
    }();
    const long n = ++g_alloc_count;
    return target > 0 && n == target;
}

int dev_alloc(pwa_ctx *ctx, void **p, size_t bytes, const char *what)
{
    *p = nullptr;
    if (injected_alloc_failure())
        return fail(ctx, PWA_ENOMEM, "injected allocation failure (%s, %zu bytes)", what, bytes);
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(ctx, PWA_ENOMEM, "cudaMalloc(%s, %zu bytes): %s", what, bytes,
                    cudaGetErrorString(e));
    }
    return PWA_OK;
}

template <typename T>
void dev_free(T *&p)
{
    if (p)
        cudaFree(p);
    p = nullptr;
}

#define CK(ctx, call)                                                                      \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            cudaGetLastError();                                                            \
            return fail(ctx, PWA_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
        }                                                                                  \
    } while (0)

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        cudaGetDevice(&prev);
        if (prev != dev)
            cudaSetDevice(dev);
        else
            prev = -1;
    }
    ~DeviceGuard()
    {
        if (prev >= 0)
            cudaSetDevice(prev);
    }
};

bool is_device_pointer(const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// Device inputs may come from work on any stream (another library's, the
// caller's default stream): before the library's own stream reads them, all
// work already issued to the device completes. Used by the calls that read
// caller-provided device buffers at load time (one-time calls).
int device_input_ready(pwa_ctx *c)
{
    const cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, PWA_ECUDA, "waiting for device inputs: %s", cudaGetErrorString(e));
    }
    return PWA_OK;
}

// [nll K | grad 2NK | status,done | V 2NK] for K <= max_k, then max_k flags
size_t io_flags_at(int N, int max_k) { return (size_t)max_k * (1 + 4 * (size_t)N) + 1; }
size_t io_doubles(int N, int max_k) { return io_flags_at(N, max_k) + max_k; }

void free_res(pwa_ctx *c)
{
    dev_free(c->res_data);
    dev_free(c->res_mc);
    dev_free(c->d_res);
    dev_free(c->res_amax);
    if (c->h_res)
        cudaFreeHost(c->h_res);
    c->h_res = nullptr;
    c->res_loaded = false;
    c->res_tma = false;
}

void free_sample(pwa_ctx *c)
{
    dev_free(c->data.ptr);
    dev_free(c->mc.ptr);
    dev_free(c->table);
    dev_free(c->tmax);
    dev_free(c->xbf);
    c->loaded = c->has_norm = false;
    c->hess_tc = false;
    c->n_lambda = 1;
    ++c->epoch;
}

// Copy n events of nw complex waves (event-major, host or device) into the
// 2 nw planes starting at dst (pitch floats apart): device sources are packed
// directly; host sources go through a bounded device staging buffer.
int pack_rows(pwa_ctx *c, const void *src, int64_t n, int dtype, int nw, float *dst, int64_t pitch)
{
    if (nw == 0 || n == 0)
        return PWA_OK;
    const size_t esz = (dtype == PWA_C64 ? 8 : 16) * (size_t)nw;
    if (is_device_pointer(src)) {
        if (int rc = device_input_ready(c))
            return rc;
        CK(c, launch_pack(src, dtype, n, nw, dst, pitch, c->stream));
        return PWA_OK;
    }
    const int64_t chunk = (int64_t)((64u << 20) / esz) > 0 ? (int64_t)((64u << 20) / esz) : 1;
    void *staging = nullptr;
    int rc = dev_alloc(c, &staging, (size_t)std::min<int64_t>(chunk, n) * esz, "staging");
    if (rc)
        return rc;
    for (int64_t s = 0; s < n; s += chunk) {
        const int64_t m = std::min(chunk, n - s);
        cudaError_t e = cudaMemcpyAsync(staging, static_cast<const char *>(src) + s * esz, m * esz,
                                        cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess)
            e = launch_pack(staging, dtype, m, nw, dst + s, pitch, c->stream);
        if (e != cudaSuccess) {
            cudaStreamSynchronize(c->stream);
            cudaFree(staging);
            cudaGetLastError();
            return fail(c, PWA_ECUDA, "loading amplitudes: %s", cudaGetErrorString(e));
        }
    }
    cudaError_t e = cudaStreamSynchronize(c->stream);
    cudaFree(staging);
    if (e != cudaSuccess)
        return fail(c, PWA_ECUDA, "loading amplitudes: %s", cudaGetErrorString(e));
    return PWA_OK;
}

// Copy one sample into planes [2N][pitch].
int load_planes(pwa_ctx *c, const void *src, int64_t n, int dtype, Planes *out)
{
    const int N = c->N;
    out->n = n;
    out->n_waves = N;
    out->pitch = round_up(n, 256);
    int rc = dev_alloc(c, (void **)&out->ptr, (size_t)2 * N * out->pitch * sizeof(float), "planes");
    if (rc)
        return rc;
    CK(c, cudaMemsetAsync(out->ptr, 0, (size_t)2 * N * out->pitch * sizeof(float), c->stream));
    return pack_rows(c, src, n, dtype, N, out->ptr, out->pitch);
}

// n doubles (host or device) rounded to floats at dst.
int load_floats(pwa_ctx *c, const double *src, int64_t n, float *dst)
{
    if (is_device_pointer(src)) {
        if (int rc = device_input_ready(c))
            return rc;
        CK(c, launch_to_float(src, n, dst, c->stream));
        return PWA_OK;
    }
    const int64_t chunk = 8 << 20;
    double *staging = nullptr;
    int rc = dev_alloc(c, (void **)&staging, (size_t)std::min<int64_t>(chunk, n) * 8, "staging");
    if (rc)
        return rc;
    cudaError_t e = cudaSuccess;
    for (int64_t s = 0; s < n && e == cudaSuccess; s += chunk) {
        const int64_t m = std::min(chunk, n - s);
        e = cudaMemcpyAsync(staging, src + s, m * 8, cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess)
            e = launch_to_float(staging, m, dst + s, c->stream);
    }
    const cudaError_t e2 = cudaStreamSynchronize(c->stream);
    cudaFree(staging);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        cudaGetLastError();
        return fail(c, PWA_ECUDA, "loading masses: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    return PWA_OK;
}

// One sample of the free-resonance form: planes [1 + 2N][pitch] + padding.
int load_res_sample(pwa_ctx *c, int R, const double *m, const void *Y, const void *Afix, int64_t n,
                    int dtype, float **out, int64_t *pitch)
{
    const int N = c->N;
    *pitch = round_up(n, 256);
    const size_t bytes = ((size_t)(1 + 2 * N) * *pitch + 256) * sizeof(float);
    int rc = dev_alloc(c, (void **)out, bytes, "resonance planes");
    if (rc)
        return rc;
    CK(c, cudaMemsetAsync(*out, 0, bytes, c->stream));
    if ((rc = load_floats(c, m, n, *out)))
        return rc;
    if ((rc = pack_rows(c, Y, n, dtype, R, *out + *pitch, *pitch)))
        return rc;
    return pack_rows(c, Afix, n, dtype, N - R, *out + (size_t)(1 + 2 * R) * *pitch, *pitch);
}


int status_from_flags(pwa_ctx *c, int flags)
{
    if (flags & FLAG_TIMEOUT)
        return fail(c, PWA_ETIMEOUT, "a device-side wait timed out; results are invalid");
    if (flags & FLAG_DOMAIN)
        return fail(c, PWA_EDOMAIN, "an intensity was not positive and finite (nll = +inf)");
    return PWA_OK;
}

int check_eval_args(pwa_ctx *c, const void *V, int K, const void *nll)
{
    if (!V || !nll)
        return fail(c, PWA_EINVAL, "null V or nll");
    if (K < 1 || K > c->cfg.max_k)
        return fail(c, PWA_EINVAL, "K=%d outside [1, max_k=%d]", K, c->cfg.max_k);
    if (!c->loaded || !c->has_norm)
        return fail(c, PWA_ESTATE, "pwa_load_events and pwa_build_norm must come first");
    return PWA_OK;
}

// PWA_TEST_TIMEOUT_NS=<ns> (tests of the timeout path): the direct form's
// copies are not issued and its consumers give up after <ns>, so that the
// call reports PWA_ETIMEOUT without anything left in flight. Read per call.
unsigned long long test_stall_ns()
{
    const char *v = getenv("PWA_TEST_TIMEOUT_NS");
    return v ? strtoull(v, nullptr, 10) : 0ull;
}

// Enqueue the evaluation of K parameter sets (device pointers).
int enqueue_eval(pwa_ctx *c, const double *dV, int K, double *dnll, double *dgrad, int *status,
                 int *done)
{
    const int N = c->N;
    if (c->form == PWA_FORM_TC) {
        // launches of near-equal size (multiples of 64 sets): each launch reads the data once
        const int kmax = batched_max_k(N, c->xs);
        const int nl = (K + kmax - 1) / kmax;
        int per = ((K + nl - 1) / nl + 63) / 64 * 64;
        if (c->tune_tc_per > 0)
            per = std::min(c->tune_tc_per, kmax);
        for (int k0 = 0; k0 < K; k0 += per) {
            const int kk = std::min(per, K - k0);
            cudaError_t e = launch_batched(c->xbf, c->n_data, N, c->xs, c->xsum, dV + (size_t)2 * N * k0,
                                           kk, c->M, c->d_work, c->num_sms, status, done, dnll + k0,
                                           dgrad ? dgrad + (size_t)2 * N * k0 : nullptr, c->stream,
                                           c->tune_tc_nxs);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return fail(c, PWA_ECUDA, "batched launch: %s", cudaGetErrorString(e));
            }
        }
        return PWA_OK;
    }
    for (int k = 0; k < K; ++k) {
        EvalArgs a{};
        a.n_waves = N;
        a.n_events = c->n_data;
        a.V = dV + (size_t)2 * N * k;
        a.M = c->M;
        a.amax = c->amax;
        a.partials = c->d_work;
        a.ticket = c->ticket;
        a.status = status;
        a.done = done;
        a.nll = dnll + k;
        a.grad = dgrad ? dgrad + (size_t)2 * N * k : nullptr;
        a.stall_ns = test_stall_ns();
        cudaError_t e = cudaSuccess;
        if (c->form == PWA_FORM_AMP && c->n_lambda > 1 && c->incoh_tma)
            e = launch_nll_incoh_tma(&c->data_map, c->n_lambda, a, amp_grid(N, c->num_sms), c->stream);
        else if (c->form == PWA_FORM_AMP && c->n_lambda > 1)
            e = launch_nll_incoh(c->data, c->n_lambda, a, c->num_sms, c->stream);
        else if (c->form == PWA_FORM_AMP)
            e = launch_nll_amp(c->data, &c->data_map, a, c->num_sms, c->stream, c->tune_groups);
        else if (c->form == PWA_FORM_TABLE)
            e = launch_nll_table(c->n_data, N, &c->table_map, a, c->tmax, c->num_sms, c->stream);
        else
            return fail(c, PWA_EINVAL, "internal: tensor-core form in the per-set loop");
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(c, PWA_ECUDA, "kernel launch: %s", cudaGetErrorString(e));
        }
    }
    return PWA_OK;
}

// The copy of [status | V] in, the evaluation kernels and the copy of
// [nll | grad | status] out, enqueued on the context's stream.
int enqueue_host_eval(pwa_ctx *c, int K, bool with_grad)
{
    const size_t gK = (size_t)2 * c->N * K;
    double *h_stat = c->h_io + K + gK, *d_stat = c->d_io + K + gK;
    CK(c, cudaMemcpyAsync(d_stat, h_stat, (1 + gK) * sizeof(double), cudaMemcpyHostToDevice,
                          c->stream));
    int *ds = reinterpret_cast<int *>(d_stat);
    int rc = enqueue_eval(c, d_stat + 1, K, c->d_io, with_grad ? c->d_io + K : nullptr, ds, ds + 1);
    if (rc)
        return rc;
    CK(c, cudaMemcpyAsync(c->h_io, c->d_io, (K + gK + 1) * sizeof(double), cudaMemcpyDeviceToHost,
                          c->stream));
    return PWA_OK;
}

// The graph of enqueue_host_eval for (K, with_grad) at the current epoch,
// captured on first use (null if capture is not possible here: the stream is
// being captured by the caller, or PWA_EVAL_GRAPHS=0).
cudaGraphExec_t eval_graph(pwa_ctx *c, int K, bool with_grad)
{
    const char *v = getenv("PWA_EVAL_GRAPHS");
    if ((v && strcmp(v, "0") == 0) || c->graphs_off)
        return nullptr;
    for (size_t i = 0; i < c->graphs.size();) {
        if (c->graphs[i].epoch != c->epoch) {
            cudaGraphExecDestroy(c->graphs[i].exec);
            c->graphs.erase(c->graphs.begin() + i);
        } else if (c->graphs[i].K == K && c->graphs[i].grad == with_grad) {
            return c->graphs[i].exec;
        } else {
            ++i;
        }
    }
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(c->stream, &st) != cudaSuccess || st != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return nullptr;
    }
    if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        c->graphs_off = true;
        return nullptr;
    }
    const int rc = enqueue_host_eval(c, K, with_grad);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
    cudaGraphExec_t exec = nullptr;
    if (rc == PWA_OK && e == cudaSuccess && graph &&
        cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess) {
        if (c->graphs.size() >= 8) {
            cudaGraphExecDestroy(c->graphs.front().exec);
            c->graphs.erase(c->graphs.begin());
        }
        c->graphs.push_back({K, with_grad, c->epoch, exec});
    } else {
        cudaGetLastError();
        c->graphs_off = true;   // fall back to direct enqueueing for this context
        exec = nullptr;
    }
    if (graph)
        cudaGraphDestroy(graph);
    return exec;
}

// The direct form's host call without copies: the kernels read V from the
// pinned buffer and write nll, grad and a flag (sequence number, status
// bits) straight back into it, and the host spins on the flags instead of
// synchronising the stream. Used for coherent samples in the direct form
// unless PWA_ZERO_COPY=0.
bool zero_copy_ok(const pwa_ctx *c)
{
    static const bool off = [] {
        const char *v = getenv("PWA_ZERO_COPY");
        return v && strcmp(v, "0") == 0;
    }();
    return !off && c->h_io_dev && c->form == PWA_FORM_AMP && c->n_lambda == 1;
}

int eval_host_zc(pwa_ctx *c, const double *V, int K, double *nll, double *grad)
{
    const int N = c->N;
    const size_t gK = (size_t)2 * N * K;
    double *h_stat = c->h_io + K + gK;
    const ptrdiff_t to_dev = reinterpret_cast<char *>(c->h_io_dev) - reinterpret_cast<char *>(c->h_io);
    auto dev = [&](void *p) { return reinterpret_cast<char *>(p) + to_dev; };
    unsigned long long *flags =
        reinterpret_cast<unsigned long long *>(c->h_io + io_flags_at(N, c->cfg.max_k));
    memcpy(h_stat + 1, V, gK * sizeof(double));
    const unsigned seq = ++c->zc_seq;
    std::atomic_thread_fence(std::memory_order_seq_cst);  // V is in memory before the launch
    for (int k = 0; k < K; ++k) {
        EvalArgs a{};
        a.n_waves = N;
        a.n_events = c->n_data;
        a.V = reinterpret_cast<const double *>(dev(h_stat + 1 + (size_t)2 * N * k));
        a.M = c->M;
        a.amax = c->amax;
        a.partials = c->d_work;
        a.ticket = c->ticket;
        a.status = c->zc_status;
        a.nll = reinterpret_cast<double *>(dev(c->h_io + k));
        a.grad = grad ? reinterpret_cast<double *>(dev(c->h_io + K + (size_t)2 * N * k)) : nullptr;
        a.host_flag = reinterpret_cast<unsigned long long *>(dev(flags + k));
        a.seq = seq;
        a.stall_ns = test_stall_ns();
        const cudaError_t e = launch_nll_amp(c->data, &c->data_map, a, c->num_sms, c->stream,
                                             c->tune_groups);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(c, PWA_ECUDA, "kernel launch: %s", cudaGetErrorString(e));
        }
    }
    // spin on the flags; look at the stream now and then, so that a failed
    // launch or a kernel that ended without its flag cannot hold the caller
    int status = 0;
    for (int k = 0; k < K; ++k) {
        unsigned long long f;
        for (long it = 0;; ++it) {
            f = __atomic_load_n(&flags[k], __ATOMIC_ACQUIRE);
            if ((unsigned)(f >> 32) == seq)
                break;
            if ((it & 1023) == 1023) {
                const cudaError_t q = cudaStreamQuery(c->stream);
                if (q == cudaSuccess) {
                    f = __atomic_load_n(&flags[k], __ATOMIC_ACQUIRE);
                    if ((unsigned)(f >> 32) == seq)
                        break;
                    return fail(c, PWA_ETIMEOUT, "evaluation %d of %d ended without its result", k, K);
                }
                if (q != cudaErrorNotReady) {
                    cudaGetLastError();
                    return fail(c, PWA_ECUDA, "evaluation: %s", cudaGetErrorString(q));
                }
            }
        }
        status |= (int)(unsigned)(f & 0xffffffffu);
    }
    memcpy(nll, c->h_io, K * sizeof(double));
    if (grad)
        memcpy(grad, c->h_io + K, gK * sizeof(double));
    return status_from_flags(c, status);
}

int eval_host(pwa_ctx *c, const double *V, int K, double *nll, double *grad)
{
    int rc = check_eval_args(c, V, K, nll);
    if (rc)
        return rc;
    DeviceGuard g(c->device);
    if (zero_copy_ok(c))
        return eval_host_zc(c, V, K, nll, grad);
    const int N = c->N;
    const size_t gK = (size_t)2 * N * K;
    double *h_stat = c->h_io + K + gK;
    int *hs = reinterpret_cast<int *>(h_stat);
    hs[0] = 0;
    hs[1] = 0;
    memcpy(h_stat + 1, V, gK * sizeof(double));
    if (cudaGraphExec_t ex = eval_graph(c, K, grad != nullptr)) {
        CK(c, cudaGraphLaunch(ex, c->stream));
    } else if ((rc = enqueue_host_eval(c, K, grad != nullptr))) {
        return rc;
    }
    CK(c, cudaStreamSynchronize(c->stream));
    if (hs[1] != K)
        return fail(c, PWA_ETIMEOUT, "only %d of %d evaluations finished", hs[1], K);
    memcpy(nll, c->h_io, K * sizeof(double));
    if (grad)
        memcpy(grad, c->h_io + K, gK * sizeof(double));
    return status_from_flags(c, hs[0]);
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }();
    return fn;
}

}  // namespace

namespace pwa {

cudaError_t encode_planes_map(CUtensorMap *map, const float *base, int64_t n, int64_t pitch,
                              int rows, int box_x, int box_y)
{
    auto fn = get_encode_fn();
    if (!fn)
        return cudaErrorNotSupported;
    cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)pitch * sizeof(float)};
    cuuint32_t box[2] = {(cuuint32_t)box_x, (cuuint32_t)box_y};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(base), dims, strides,
                    box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace pwa

extern "C" {

static int finish_load(pwa_ctx *c, int rc, int64_t n_data, int64_t n_mc_acc, double n_mc_gen);

int pwa_version(void) { return 100; }

const char *pwa_last_error(const pwa_ctx *ctx) { return ctx ? ctx->err : g_create_err; }

constexpr int kResMaxBlocksPerSm = 3;
static size_t res_grid(const pwa_ctx *c) { return (size_t)c->num_sms * c->tune_res_cps; }

int pwa_load_resonance_events(pwa_ctx *c, int n_free, const double *m_data, const void *Y_data,
                              const void *Afix_data, int64_t n_data, const double *m_mc,
                              const void *Y_mc, const void *Afix_mc, int64_t n_mc_acc,
                              double n_mc_gen, int amp_dtype)
{
    if (!c)
        return PWA_EINVAL;
    const int N = c->N;
    if (N > res_max_waves() || n_free > res_max_free())
        return fail(c, PWA_ENOTSUP, "free resonances need n_waves <= %d and n_free <= %d",
                    res_max_waves(), res_max_free());
    if (n_free < 1 || n_free > N)
        return fail(c, PWA_EINVAL, "n_free=%d outside [1, n_waves=%d]", n_free, N);
    if (!m_data || !Y_data || !m_mc || !Y_mc || (n_free < N && (!Afix_data || !Afix_mc)))
        return fail(c, PWA_EINVAL, "null sample pointer");
    if (n_data < 1 || n_mc_acc < 1 || n_data > ((int64_t)1 << 31) - 1024 ||
        n_mc_acc > ((int64_t)1 << 31) - 1024)
        return fail(c, PWA_EINVAL, "sample sizes must be in [1, 2^31 - 1024]");
    if (!(n_mc_gen >= (double)n_mc_acc))
        return fail(c, PWA_EINVAL, "n_mc_gen=%g must be >= n_mc_acc=%lld", n_mc_gen,
                    (long long)n_mc_acc);
    if (amp_dtype != PWA_C64 && amp_dtype != PWA_C128)
        return fail(c, PWA_EINVAL, "amp_dtype=%d is neither PWA_C64 nor PWA_C128", amp_dtype);
    DeviceGuard g(c->device);
    cudaStreamSynchronize(c->stream);
    free_res(c);
    int rc = load_res_sample(c, n_free, m_data, Y_data, Afix_data, n_data, amp_dtype, &c->res_data,
                             &c->res_data_pitch);
    if (!rc)
        rc = load_res_sample(c, n_free, m_mc, Y_mc, Afix_mc, n_mc_acc, amp_dtype, &c->res_mc,
                             &c->res_mc_pitch);
    const size_t npart = res_partials_doubles(N, n_free, c->num_sms * kResMaxBlocksPerSm);
    const size_t nio = 4 * (size_t)N + 4 * (size_t)n_free + 2;
    if (!rc)
        rc = dev_alloc(c, (void **)&c->d_res, (npart + 1 + nio) * sizeof(double), "resonance io");
    if (!rc && cudaMemsetAsync(c->d_res, 0, (npart + 1 + nio) * sizeof(double), c->stream) != cudaSuccess)
        rc = fail(c, PWA_ECUDA, "memset");
    if (!rc && cudaMallocHost((void **)&c->h_res, nio * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        c->h_res = nullptr;
        rc = fail(c, PWA_ENOMEM, "pinned host buffer");
    }
    // The TMA-fed kernel (PWA_RES_KERNEL=generic selects the per-event one):
    // per-wave maxima over both samples bound its exact product split.
    const char *kv = getenv("PWA_RES_KERNEL");
    const bool tma = res_tma_available(N, n_free) && !(kv && strcmp(kv, "generic") == 0);
    if (!rc && tma) {
        float *tmp = nullptr;
        rc = dev_alloc(c, (void **)&c->res_amax, N * sizeof(float), "resonance maxima");
        if (!rc)
            rc = dev_alloc(c, (void **)&tmp, N * sizeof(float), "resonance maxima");
        cudaError_t e = cudaSuccess;
        if (!rc) {
            const Planes pd{c->res_data + c->res_data_pitch, c->res_data_pitch, n_data, N};
            const Planes pm{c->res_mc + c->res_mc_pitch, c->res_mc_pitch, n_mc_acc, N};
            e = cudaMemsetAsync(c->res_amax, 0, N * sizeof(float), c->stream);
            if (e == cudaSuccess)
                e = cudaMemsetAsync(tmp, 0, N * sizeof(float), c->stream);
            if (e == cudaSuccess)
                e = launch_amp_max(pd, c->res_amax, c->stream);
            if (e == cudaSuccess)
                e = launch_amp_max(pm, tmp, c->stream);
            std::vector<float> h1(N), h2(N);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(h1.data(), c->res_amax, N * sizeof(float), cudaMemcpyDeviceToHost,
                                    c->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(h2.data(), tmp, N * sizeof(float), cudaMemcpyDeviceToHost,
                                    c->stream);
            if (e == cudaSuccess)
                e = cudaStreamSynchronize(c->stream);
            for (int k = 0; k < N && e == cudaSuccess; ++k)
                h1[k] = std::max(h1[k], h2[k]);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(c->res_amax, h1.data(), N * sizeof(float), cudaMemcpyHostToDevice,
                                    c->stream);
            if (e == cudaSuccess)
                e = cudaStreamSynchronize(c->stream);
            if (e == cudaSuccess)
                e = encode_planes_map(&c->res_dmap, c->res_data, n_data, c->res_data_pitch, 1 + 2 * N,
                                      res_tma_box_events(), 1 + 2 * N);
            if (e == cudaSuccess)
                e = encode_planes_map(&c->res_mmap, c->res_mc, n_mc_acc, c->res_mc_pitch, 1 + 2 * N,
                                      res_tma_box_events(), 1 + 2 * N);
            if (e != cudaSuccess)
                rc = fail(c, PWA_ECUDA, "free-resonance set-up: %s", cudaGetErrorString(e));
        }
        dev_free(tmp);
    }
    if (!rc && cudaStreamSynchronize(c->stream) != cudaSuccess)
        rc = fail(c, PWA_ECUDA, "loading the resonance samples");
    if (rc) {
        free_res(c);
        return rc;
    }
    c->res_tma = tma;
    c->res_R = n_free;
    c->res_n_data = n_data;
    c->res_n_mc = n_mc_acc;
    c->res_ngen = n_mc_gen;
    c->res_loaded = true;
    return PWA_OK;
}

// The free-resonance evaluation with device pointers: V, mass, width in,
// [nll | gV | gM | gW] out, status into `status`, `done` incremented (may be null).
static int enqueue_res(pwa_ctx *c, const double *dV, const double *dmass, const double *dwidth,
                       double *dout, int *status, int *done)
{
    const int N = c->N, R = c->res_R;
    const size_t npart = res_partials_doubles(N, R, c->num_sms * kResMaxBlocksPerSm);
    ResArgs a{};
    a.n_waves = N;
    a.n_free = R;
    a.data = c->res_data;
    a.data_pitch = c->res_data_pitch;
    a.n_data = c->res_n_data;
    a.mc = c->res_mc;
    a.mc_pitch = c->res_mc_pitch;
    a.n_mc = c->res_n_mc;
    a.inv_ngen = 1.0 / c->res_ngen;
    a.V = dV;
    a.mass = dmass;
    a.width = dwidth;
    a.partials = c->d_res;
    a.ticket = reinterpret_cast<unsigned *>(c->d_res + npart);
    a.status = status;
    a.done = done;
    a.out = dout;
    cudaError_t e = c->res_tma
                        ? launch_nll_res_tma(&c->res_dmap, &c->res_mmap, a, c->res_amax, c->num_sms,
                                             c->stream)
                        : launch_nll_res(a, (int)res_grid(c), c->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, PWA_ECUDA, "resonance kernel launch: %s", cudaGetErrorString(e));
    }
    return PWA_OK;
}

int pwa_nll_grad_res_async(pwa_ctx *c, const double *d_V, const double *d_mass,
                           const double *d_width, double *d_out)
{
    if (!c)
        return PWA_EINVAL;
    if (!d_V || !d_mass || !d_width || !d_out)
        return fail(c, PWA_EINVAL, "null V, mass, width or out");
    if (!c->res_loaded)
        return fail(c, PWA_ESTATE, "pwa_load_resonance_events must come first");
    DeviceGuard g(c->device);
    return enqueue_res(c, d_V, d_mass, d_width, d_out, c->async_status, nullptr);
}

int pwa_nll_grad_res(pwa_ctx *c, const double *V, const double *mass, const double *width,
                     double *nll, double *gV, double *gM, double *gW)
{
    if (!c)
        return PWA_EINVAL;
    if (!V || !mass || !width || !nll)
        return fail(c, PWA_EINVAL, "null V, mass, width or nll");
    if (!c->res_loaded)
        return fail(c, PWA_ESTATE, "pwa_load_resonance_events must come first");
    DeviceGuard g(c->device);
    const int N = c->N, R = c->res_R;
    const size_t npart = res_partials_doubles(N, R, c->num_sms * kResMaxBlocksPerSm);
    double *d_io = c->d_res + npart + 1, *h = c->h_res;
    // io: V [2N] | mass [R] | width [R] | status, done | out [1 + 2N + 2R]
    memcpy(h, V, 2 * N * sizeof(double));
    memcpy(h + 2 * N, mass, R * sizeof(double));
    memcpy(h + 2 * N + R, width, R * sizeof(double));
    int *hs = reinterpret_cast<int *>(h + 2 * N + 2 * R);
    hs[0] = hs[1] = 0;
    const size_t nin = 2 * (size_t)N + 2 * R + 1, nout = 1 + 2 * (size_t)N + 2 * R;
    CK(c, cudaMemcpyAsync(d_io, h, nin * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    int *ds = reinterpret_cast<int *>(d_io + 2 * N + 2 * R);
    int rc = enqueue_res(c, d_io, d_io + 2 * N, d_io + 2 * N + R, d_io + nin, ds, ds + 1);
    if (rc)
        return rc;
    CK(c, cudaMemcpyAsync(h + 2 * N + 2 * R, d_io + 2 * N + 2 * R, (1 + nout) * sizeof(double),
                          cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    if (hs[1] != 1)
        return fail(c, PWA_ETIMEOUT, "the resonance evaluation did not finish");
    const double *o = h + nin;
    *nll = o[0];
    if (gV)
        memcpy(gV, o + 1, 2 * N * sizeof(double));
    if (gM)
        memcpy(gM, o + 1 + 2 * N, R * sizeof(double));
    if (gW)
        memcpy(gW, o + 1 + 2 * N + R, R * sizeof(double));
    return status_from_flags(c, hs[0]);
}

// ---- Hessian, projection weights, fit fractions -----------------------------

// Device scratch and its pinned host mirror for the Hessian, weight and
// fraction calls; copies V in (through the mirror) and clears the status word.
static int fx_alloc(pwa_ctx *c)
{
    const int N = c->N;
    const size_t nio = 2 * (size_t)N + 1 + 4 * (size_t)N * N;
    const size_t npart = std::max(hess_partials_doubles(N, c->num_sms),
                                  hess_tc_partials_doubles(N, c->num_sms));
    const size_t bytes = (nio + npart) * sizeof(double);
    if (c->fx_bytes < bytes) {
        dev_free(c->d_fx);
        if (c->h_fx)
            cudaFreeHost(c->h_fx);
        c->h_fx = nullptr;
        c->fx_bytes = 0;
        int rc = dev_alloc(c, (void **)&c->d_fx, bytes, "Hessian scratch");
        if (rc)
            return rc;
        if (cudaMallocHost((void **)&c->h_fx, nio * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            c->h_fx = nullptr;
            dev_free(c->d_fx);
            return fail(c, PWA_ENOMEM, "pinned host buffer");
        }
        c->fx_bytes = bytes;
    }
    return PWA_OK;
}

static int fx_buffer(pwa_ctx *c, const double *V, double **dV, int **dstat, double **dout,
                     double **dpart)
{
    int rc = fx_alloc(c);
    if (rc)
        return rc;
    const int N = c->N;
    *dV = c->d_fx;
    *dstat = reinterpret_cast<int *>(c->d_fx + 2 * N);
    *dout = c->d_fx + 2 * N + 1;
    *dpart = *dout + 4 * (size_t)N * N;
    memcpy(c->h_fx, V, 2 * N * sizeof(double));
    c->h_fx[2 * N] = 0.0;  // status word(s)
    CK(c, cudaMemcpyAsync(*dV, c->h_fx, (2 * N + 1) * sizeof(double), cudaMemcpyHostToDevice,
                          c->stream));
    return PWA_OK;
}

// Copies `count` doubles of the output area back through the pinned mirror
// (with the status word in front of them), waits, and returns the flags.
static int fx_result(pwa_ctx *c, size_t count, double *out, int *flags)
{
    const int N = c->N;
    CK(c, cudaMemcpyAsync(c->h_fx + 2 * N, c->d_fx + 2 * N, (1 + count) * sizeof(double),
                          cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    *flags = *reinterpret_cast<const int *>(c->h_fx + 2 * N);
    if (out)
        memcpy(out, c->h_fx + 2 * N + 1, count * sizeof(double));
    return PWA_OK;
}

// The tensor-core kernel where it serves the sample (PWA_HESS_KERNEL=generic
// selects the CUDA-core kernel), else the CUDA-core one.
static cudaError_t enqueue_hessian(pwa_ctx *c, const double *dV, double *dpart, int *ds, double *dH,
                                   int *async_or)
{
    const char *kv = getenv("PWA_HESS_KERNEL");
    if (c->hess_tc && !(kv && strcmp(kv, "generic") == 0))
        return launch_hessian_tc(&c->hess_map, c->data, dV, c->amax, dpart, c->num_sms, ds, dH,
                                 async_or, c->stream);
    return launch_hessian(c->data, dV, dpart, c->num_sms, ds, dH, async_or, c->stream);
}

int pwa_hessian(pwa_ctx *c, const double *V, double *H)
{
    if (!c)
        return PWA_EINVAL;
    if (!V || !H)
        return fail(c, PWA_EINVAL, "null V or H");
    if (!c->loaded)
        return fail(c, PWA_ESTATE, "pwa_load_events must come first");
    if (c->n_lambda > 1)
        return fail(c, PWA_ENOTSUP, "the Hessian takes coherent samples only");
    DeviceGuard g(c->device);
    double *dV, *dH, *dpart;
    int *ds;
    int rc = fx_buffer(c, V, &dV, &ds, &dH, &dpart);
    if (rc)
        return rc;
    CK(c, enqueue_hessian(c, dV, dpart, ds, dH, nullptr));
    const int P = 2 * c->N;
    int flags = 0;
    if ((rc = fx_result(c, (size_t)P * P, H, &flags)))
        return rc;
    return status_from_flags(c, flags);
}

int pwa_hessian_async(pwa_ctx *c, const double *d_V, double *d_H)
{
    if (!c)
        return PWA_EINVAL;
    if (!d_V || !d_H)
        return fail(c, PWA_EINVAL, "null V or H");
    if (!c->loaded)
        return fail(c, PWA_ESTATE, "pwa_load_events must come first");
    if (c->n_lambda > 1)
        return fail(c, PWA_ENOTSUP, "the Hessian takes coherent samples only");
    DeviceGuard g(c->device);
    int rc = fx_alloc(c);
    if (rc)
        return rc;
    const int N = c->N;
    int *ds = reinterpret_cast<int *>(c->d_fx + 2 * N);
    double *dpart = c->d_fx + 2 * N + 1 + 4 * (size_t)N * N;
    CK(c, cudaMemsetAsync(ds, 0, sizeof(double), c->stream));
    CK(c, enqueue_hessian(c, d_V, dpart, ds, d_H, c->async_status));
    return PWA_OK;
}

int pwa_mc_weights(pwa_ctx *c, const double *V, float *w)
{
    if (!c)
        return PWA_EINVAL;
    if (!V || !w)
        return fail(c, PWA_EINVAL, "null V or w");
    if (!c->loaded)
        return fail(c, PWA_ESTATE, "pwa_load_events must come first");
    if (c->n_lambda > 1)
        return fail(c, PWA_ENOTSUP, "projection weights take coherent samples only");
    DeviceGuard g(c->device);
    double *dV, *dout, *dpart;
    int *ds;
    int rc = fx_buffer(c, V, &dV, &ds, &dout, &dpart);
    if (rc)
        return rc;
    const bool on_dev = is_device_pointer(w);
    float *dw = w;
    if (!on_dev) {
        if (c->w_len < c->n_mc) {
            dev_free(c->d_w);
            c->w_len = 0;
            if ((rc = dev_alloc(c, (void **)&c->d_w, (size_t)c->n_mc * sizeof(float), "weights")))
                return rc;
            c->w_len = c->n_mc;
        }
        dw = c->d_w;
    }
    const char *kv = getenv("PWA_WEIGHTS_KERNEL");
    if (kv && strcmp(kv, "generic") == 0) {
        CK(c, launch_mc_weights(c->mc, dV, c->n_gen, dw, c->num_sms * 8, c->stream));
    } else {
        CK(c, launch_mc_weights_tma(&c->mc_map, c->mc, dV, c->mc_amax, c->n_gen, dw, ds, c->num_sms,
                                    c->stream));
    }
    if (!on_dev)
        CK(c, cudaMemcpyAsync(w, dw, (size_t)c->n_mc * sizeof(float), cudaMemcpyDeviceToHost,
                              c->stream));
    int flags = 0;
    if ((rc = fx_result(c, 0, nullptr, &flags)))
        return rc;
    return status_from_flags(c, flags);
}

int pwa_fit_fractions(pwa_ctx *c, const double *V, double *F)
{
    if (!c)
        return PWA_EINVAL;
    if (!V || !F)
        return fail(c, PWA_EINVAL, "null V or F");
    if (!c->has_norm)
        return fail(c, PWA_ESTATE, "pwa_build_norm must come first");
    DeviceGuard g(c->device);
    double *dV, *dF, *dpart;
    int *ds;
    int rc = fx_buffer(c, V, &dV, &ds, &dF, &dpart);
    if (rc)
        return rc;
    CK(c, launch_fit_fractions(c->M, dV, c->N, dF, c->stream));
    int flags = 0;
    return fx_result(c, (size_t)c->N * c->N, F, &flags);
}

int pwa_table_bytes(int n_waves, int64_t n_events, int64_t *bytes)
{
    if (!bytes || n_waves < 1 || n_waves > kMaxWaves || n_events < 0)
        return PWA_EINVAL;
    *bytes = (int64_t)n_waves * n_waves * (int64_t)sizeof(float) * n_events;
    return PWA_OK;
}

int pwa_create(pwa_ctx **out, int device, const pwa_config *cfg)
{
    g_create_err[0] = 0;
    if (!out || !cfg)
        return fail(nullptr, PWA_EINVAL, "null out or cfg");
    *out = nullptr;
    if (cfg->n_waves < 1 || cfg->n_waves > kMaxWaves)
        return fail(nullptr, PWA_EINVAL, "n_waves=%d outside [1, %d]", cfg->n_waves, kMaxWaves);
    if (cfg->max_k < 1 || cfg->max_k > 65536)
        return fail(nullptr, PWA_EINVAL, "max_k=%d outside [1, 65536]", cfg->max_k);
    const int forms = cfg->forms ? cfg->forms : PWA_FORM_AMP;
    if (forms & ~(PWA_FORM_AMP | PWA_FORM_TABLE | PWA_FORM_TC))
        return fail(nullptr, PWA_EINVAL, "unknown form bits 0x%x", forms);
    if (cfg->precision != PWA_PREC_DEFAULT && cfg->precision != PWA_PREC_BFP16 &&
        cfg->precision != PWA_PREC_BFP8)
        return fail(nullptr, PWA_EINVAL, "unknown precision %d", cfg->precision);
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return fail(nullptr, PWA_ECUDA, "device %d not available (%d devices)", device, ndev);
    }
    DeviceGuard g(device);
    cudaSetDevice(device);
    pwa_ctx *c = new pwa_ctx();
    c->device = device;
    c->cfg = *cfg;
    c->cfg.forms = forms;
    c->N = cfg->n_waves;
    c->xs = cfg->precision == PWA_PREC_BFP8 ? 1 : 2;
    c->form = (forms & PWA_FORM_AMP) ? PWA_FORM_AMP
              : (forms & PWA_FORM_TABLE) ? PWA_FORM_TABLE : PWA_FORM_TC;
    int rc = PWA_OK;
    auto bail = [&](int code) {
        snprintf(g_create_err, sizeof g_create_err, "%s", c->err);
        pwa_destroy(c);
        return code;
    };
    if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return bail(fail(c, PWA_ECUDA, "cannot query the SM count"));
    if (cfg->stream) {
        c->stream = static_cast<cudaStream_t>(cfg->stream);
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess)
            return bail(fail(c, PWA_ECUDA, "cudaStreamCreate failed"));
        c->own_stream = true;
    }
    if ((forms & PWA_FORM_TABLE) && c->N > table_max_waves())
        return bail(fail(c, PWA_ENOTSUP, "the table form supports up to %d waves", table_max_waves()));
    cudaError_t e = amp_configure();
    if (e == cudaSuccess && (forms & PWA_FORM_TABLE))
        e = table_configure();
    if (e == cudaSuccess && (forms & PWA_FORM_TC))
        e = batched_configure();
    if (e != cudaSuccess)
        return bail(fail(c, PWA_ECUDA, "kernel configuration: %s", cudaGetErrorString(e)));
    const size_t nio = io_doubles(c->N, cfg->max_k);
    if ((rc = dev_alloc(c, (void **)&c->d_io, nio * sizeof(double), "io")))
        return bail(rc);
    if (cudaHostAlloc((void **)&c->h_io, nio * sizeof(double), cudaHostAllocMapped) != cudaSuccess) {
        cudaGetLastError();
        c->h_io = nullptr;
        return bail(fail(c, PWA_ENOMEM, "pinned host buffer"));
    }
    memset(c->h_io, 0, nio * sizeof(double));
    // the device address of the pinned buffer, for the zero-copy host call
    if (cudaHostGetDevicePointer((void **)&c->h_io_dev, c->h_io, 0) != cudaSuccess) {
        cudaGetLastError();
        c->h_io_dev = nullptr;
    }
    size_t nwork = std::max(amp_partials_doubles(c->N, c->num_sms),
                            incoh_partials_doubles(c->N, c->num_sms)) + 8;
    if (forms & PWA_FORM_TABLE)
        nwork = std::max(nwork, table_scratch_bytes(c->N, c->num_sms) / sizeof(double) + 16);
    if (forms & PWA_FORM_TC)
        nwork = std::max(nwork, batched_scratch_bytes(c->N, c->xs,
                                                      std::min(cfg->max_k, batched_max_k(c->N, c->xs)),
                                                      c->num_sms) / sizeof(double) + 16);
    c->work_bytes = nwork * sizeof(double);
    if ((rc = dev_alloc(c, (void **)&c->d_work, nwork * sizeof(double), "work")))
        return bail(rc);
    if (cudaMemset(c->d_work, 0, nwork * sizeof(double)) != cudaSuccess)
        return bail(fail(c, PWA_ECUDA, "memset"));
    c->ticket = reinterpret_cast<unsigned *>(c->d_work + nwork - 4);
    c->async_status = reinterpret_cast<int *>(c->d_work + nwork - 2);
    c->zc_status = reinterpret_cast<int *>(c->d_work + nwork - 6);
    if ((rc = dev_alloc(c, (void **)&c->M, (size_t)2 * c->N * c->N * sizeof(double), "M")))
        return bail(rc);
    if ((rc = dev_alloc(c, (void **)&c->amax, (size_t)c->N * sizeof(float), "amax")))
        return bail(rc);
    if ((rc = dev_alloc(c, (void **)&c->mc_amax, (size_t)c->N * sizeof(float), "MC amax")))
        return bail(rc);
    *out = c;
    return PWA_OK;
}

int pwa_destroy(pwa_ctx *c)
{
    if (!c)
        return PWA_OK;
    DeviceGuard g(c->device);
    if (c->stream)
        cudaStreamSynchronize(c->stream);
    for (auto &g : c->graphs)
        cudaGraphExecDestroy(g.exec);
    c->graphs.clear();
    free_sample(c);
    free_res(c);
    dev_free(c->M);
    dev_free(c->mc_amax);
    dev_free(c->amax);
    dev_free(c->d_io);
    dev_free(c->d_fx);
    dev_free(c->d_w);
    if (c->h_fx)
        cudaFreeHost(c->h_fx);
    dev_free(c->d_work);
    if (c->h_io)
        cudaFreeHost(c->h_io);
    if (c->own_stream && c->stream)
        cudaStreamDestroy(c->stream);
    delete c;
    return PWA_OK;
}

int pwa_load_events(pwa_ctx *c, const void *data_amp, int64_t n_data, const void *mc_amp,
                    int64_t n_mc_acc, double n_mc_gen, int amp_dtype)
{
    if (!c)
        return PWA_EINVAL;
    if (!data_amp || !mc_amp)
        return fail(c, PWA_EINVAL, "null amplitude pointer");
    if (n_data < 1 || n_mc_acc < 1)
        return fail(c, PWA_EINVAL, "n_data=%lld and n_mc_acc=%lld must be >= 1",
                    (long long)n_data, (long long)n_mc_acc);
    if (!(n_mc_gen >= (double)n_mc_acc))
        return fail(c, PWA_EINVAL, "n_mc_gen=%g must be >= n_mc_acc=%lld", n_mc_gen,
                    (long long)n_mc_acc);
    if (amp_dtype != PWA_C64 && amp_dtype != PWA_C128)
        return fail(c, PWA_EINVAL, "amp_dtype=%d is neither PWA_C64 nor PWA_C128", amp_dtype);
    if (n_data > ((int64_t)1 << 31) - 1024 || n_mc_acc > ((int64_t)1 << 31) - 1024)
        return fail(c, PWA_EINVAL, "samples are limited to 2^31 - 1024 events");
    DeviceGuard g(c->device);
    cudaStreamSynchronize(c->stream);
    free_sample(c);
    c->n_lambda = 1;
    int rc = load_planes(c, data_amp, n_data, amp_dtype, &c->data);
    if (!rc)
        rc = load_planes(c, mc_amp, n_mc_acc, amp_dtype, &c->mc);
    return finish_load(c, rc, n_data, n_mc_acc, n_mc_gen);
}

// After the data and MC planes of a coherent sample are filled (rc = the
// status so far): the table, the tensor-core store, the amplitude maxima and
// the direct form's tensor map; then the sample is marked loaded.
static int finish_load(pwa_ctx *c, int rc, int64_t n_data, int64_t n_mc_acc, double n_mc_gen)
{
    if (!rc && (c->cfg.forms & PWA_FORM_TABLE)) {
        c->table_pitch = c->data.pitch;
        rc = dev_alloc(c, (void **)&c->table, (size_t)c->N * c->N * c->table_pitch * sizeof(float),
                       "table");
        if (!rc)
            rc = dev_alloc(c, (void **)&c->tmax, (size_t)c->N * c->N * sizeof(float), "tmax");
        if (!rc) {
            const int P = c->N * c->N;
            cudaError_t e = launch_table_build(c->data, c->table, c->table_pitch, c->stream);
            if (e == cudaSuccess)
                e = cudaMemsetAsync(c->tmax, 0, P * sizeof(float), c->stream);
            if (e == cudaSuccess)
                e = launch_plane_absmax(c->table, c->table_pitch, n_data, P, c->tmax, c->stream);
            if (e == cudaSuccess)
                e = encode_planes_map(&c->table_map, c->table, n_data, c->table_pitch, P,
                                      table_box_events(c->N), table_box_rows(c->N));
            if (e != cudaSuccess)
                rc = fail(c, PWA_ECUDA, "table build: %s", cudaGetErrorString(e));
        }
    }
    if (!rc && (c->cfg.forms & PWA_FORM_TC)) {
        const int F = batched_features(c->N);
        const size_t slice_bytes = (size_t)c->xs * F * c->data.pitch * 2;
        rc = dev_alloc(c, &c->xbf, slice_bytes + 256, "bf16 planes");
        if (!rc) {
            // the exponent sum sits after the slices
            c->xsum = reinterpret_cast<long long *>(static_cast<char *>(c->xbf) + slice_bytes);
            cudaError_t e = launch_batched_encode(c->data.ptr, c->data.pitch, c->data.n, c->N, c->xs,
                                                  c->xbf, c->xsum, c->stream);
            if (e != cudaSuccess)
                rc = fail(c, PWA_ECUDA, "block-floating-point store: %s", cudaGetErrorString(e));
        }
    }
    if (!rc) {
        cudaError_t e = cudaMemsetAsync(c->amax, 0, c->N * sizeof(float), c->stream);
        if (e == cudaSuccess)
            e = launch_amp_max(c->data, c->amax, c->stream);
        if (e != cudaSuccess)
            rc = fail(c, PWA_ECUDA, "amplitude maxima: %s", cudaGetErrorString(e));
    }
    if (!rc) {
        cudaError_t e = encode_planes_map(&c->data_map, c->data.ptr, c->data.n, c->data.pitch,
                                          2 * c->N, amp_box_events(c->N), amp_box_rows(c->N));
        // the MC sample's map and maxima serve the projection weights
        if (e == cudaSuccess)
            e = encode_planes_map(&c->mc_map, c->mc.ptr, c->mc.n, c->mc.pitch, 2 * c->N,
                                  amp_box_events(c->N), amp_box_rows(c->N));
        c->hess_tc = false;
        if (e == cudaSuccess && hess_tc_available(c->N)) {
            e = encode_planes_map(&c->hess_map, c->data.ptr, c->data.n, c->data.pitch, 2 * c->N,
                                  hess_tc_box_events(), 2 * c->N);
            c->hess_tc = e == cudaSuccess;
        }
        if (e == cudaSuccess)
            e = cudaMemsetAsync(c->mc_amax, 0, c->N * sizeof(float), c->stream);
        if (e == cudaSuccess)
            e = launch_amp_max(c->mc, c->mc_amax, c->stream);
        if (e != cudaSuccess)
            rc = fail(c, PWA_ECUDA, "tensor map encode failed");
    }
    if (!rc) {
        cudaError_t e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess)
            rc = fail(c, PWA_ECUDA, "loading: %s", cudaGetErrorString(e));
    }
    if (rc) {
        free_sample(c);
        return rc;
    }
    c->n_data = n_data;
    c->n_mc = n_mc_acc;
    c->n_gen = n_mc_gen;
    c->loaded = true;
    c->has_norm = false;
    return PWA_OK;
}

// ---- amplitudes on the device --------------------------------------------

// Checks the wave list and converts it (with N_lm) into the device table at
// *d_waves (allocated here, freed by the caller); *max_m = max |m|.
static int upload_waves(pwa_ctx *c, const pwa_wave *waves, GenWave **d_waves, int *max_m)
{
    *d_waves = nullptr;
    if (!waves)
        return fail(c, PWA_EINVAL, "null wave list");
    std::vector<GenWave> h(c->N);
    *max_m = 0;
    for (int a = 0; a < c->N; ++a) {
        const pwa_wave &w = waves[a];
        const int am = w.m < 0 ? -w.m : w.m;
        if (w.l < 0 || w.l > ampgen_max_l() || am > w.l)
            return fail(c, PWA_EINVAL, "wave %d: (l, m) = (%d, %d) needs 0 <= |m| <= l <= %d", a, w.l,
                        w.m, ampgen_max_l());
        if (!(w.mass > 0) || !(w.width > 0) || !std::isfinite(w.mass) || !std::isfinite(w.width))
            return fail(c, PWA_EINVAL, "wave %d: mass and width must be positive and finite", a);
        double ratio = 1.0;  // (l - |m|)! / (l + |m|)!
        for (int k = w.l - am + 1; k <= w.l + am; ++k)
            ratio /= k;
        h[a] = GenWave{w.mass, w.width, std::sqrt((2.0 * w.l + 1.0) / (4.0 * 3.14159265358979323846) * ratio),
                       w.l, w.m};
        *max_m = std::max(*max_m, am);
    }
    int rc = dev_alloc(c, (void **)d_waves, c->N * sizeof(GenWave), "wave table");
    if (rc)
        return rc;
    CK(c, cudaMemcpyAsync(*d_waves, h.data(), c->N * sizeof(GenWave), cudaMemcpyHostToDevice,
                          c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return PWA_OK;
}

// Generates the amplitudes of n events (kin host or device) into `out`
// (device): SoA planes of `pitch` floats, or event-major complex64.
static int generate(pwa_ctx *c, const GenWave *d_waves, int max_m, const double *kin, int64_t n,
                    float *out, bool soa, int64_t pitch)
{
    const double *dk = kin;
    double *staging = nullptr;
    if (is_device_pointer(kin)) {
        if (int rc = device_input_ready(c))
            return rc;
    } else {
        int rc = dev_alloc(c, (void **)&staging, (size_t)n * 3 * sizeof(double), "kinematics");
        if (rc)
            return rc;
        cudaError_t e = cudaMemcpyAsync(staging, kin, (size_t)n * 3 * sizeof(double),
                                        cudaMemcpyHostToDevice, c->stream);
        if (e != cudaSuccess) {
            cudaStreamSynchronize(c->stream);
            cudaFree(staging);
            return fail(c, PWA_ECUDA, "kinematics copy: %s", cudaGetErrorString(e));
        }
        dk = staging;
    }
    cudaError_t e = launch_amp_gen(dk, n, c->N, d_waves, max_m, out, soa, pitch, c->num_sms * 8,
                                   c->stream);
    cudaError_t e2 = cudaStreamSynchronize(c->stream);
    if (staging)
        cudaFree(staging);
    if (e == cudaSuccess)
        e = e2;
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, PWA_ECUDA, "amplitude generation: %s", cudaGetErrorString(e));
    }
    return PWA_OK;
}

int pwa_compute_amplitudes(pwa_ctx *c, const pwa_wave *waves, const double *kin, int64_t n,
                           void *out)
{
    if (!c)
        return PWA_EINVAL;
    if (!kin || !out)
        return fail(c, PWA_EINVAL, "null kinematics or output");
    if (n < 1 || n > ((int64_t)1 << 31) - 1024)
        return fail(c, PWA_EINVAL, "n=%lld outside [1, 2^31 - 1024]", (long long)n);
    DeviceGuard g(c->device);
    GenWave *dw;
    int max_m;
    int rc = upload_waves(c, waves, &dw, &max_m);
    if (rc) {
        dev_free(dw);
        return rc;
    }
    const bool on_dev = is_device_pointer(out);
    float *dout = static_cast<float *>(out);
    if (!on_dev)
        rc = dev_alloc(c, (void **)&dout, (size_t)n * c->N * 8, "amplitudes");
    if (!rc)
        rc = generate(c, dw, max_m, kin, n, dout, false, 0);
    if (!rc && !on_dev) {
        cudaError_t e = cudaMemcpy(out, dout, (size_t)n * c->N * 8, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess)
            rc = fail(c, PWA_ECUDA, "amplitude copy: %s", cudaGetErrorString(e));
    }
    if (!on_dev)
        dev_free(dout);
    dev_free(dw);
    return rc;
}

int pwa_load_events_generated(pwa_ctx *c, const pwa_wave *waves, const double *data_kin,
                              int64_t n_data, const double *mc_kin, int64_t n_mc_acc,
                              double n_mc_gen)
{
    if (!c)
        return PWA_EINVAL;
    if (!data_kin || !mc_kin)
        return fail(c, PWA_EINVAL, "null kinematics");
    if (n_data < 1 || n_mc_acc < 1)
        return fail(c, PWA_EINVAL, "n_data=%lld and n_mc_acc=%lld must be >= 1",
                    (long long)n_data, (long long)n_mc_acc);
    if (!(n_mc_gen >= (double)n_mc_acc))
        return fail(c, PWA_EINVAL, "n_mc_gen=%g must be >= n_mc_acc=%lld", n_mc_gen,
                    (long long)n_mc_acc);
    if (n_data > ((int64_t)1 << 31) - 1024 || n_mc_acc > ((int64_t)1 << 31) - 1024)
        return fail(c, PWA_EINVAL, "samples are limited to 2^31 - 1024 events");
    DeviceGuard g(c->device);
    cudaStreamSynchronize(c->stream);
    GenWave *dw;
    int max_m;
    int rc = upload_waves(c, waves, &dw, &max_m);
    if (rc) {
        dev_free(dw);
        return rc;
    }
    free_sample(c);
    c->n_lambda = 1;
    const int N = c->N;
    for (int which = 0; which < 2 && !rc; ++which) {
        Planes &p = which == 0 ? c->data : c->mc;
        const int64_t n = which == 0 ? n_data : n_mc_acc;
        p.n = n;
        p.n_waves = N;
        p.pitch = round_up(n, 256);
        rc = dev_alloc(c, (void **)&p.ptr, (size_t)2 * N * p.pitch * sizeof(float), "planes");
        if (!rc && cudaMemsetAsync(p.ptr, 0, (size_t)2 * N * p.pitch * sizeof(float), c->stream) !=
                       cudaSuccess)
            rc = fail(c, PWA_ECUDA, "memset");
        if (!rc)
            rc = generate(c, dw, max_m, which == 0 ? data_kin : mc_kin, n, p.ptr, true, p.pitch);
    }
    dev_free(dw);
    return finish_load(c, rc, n_data, n_mc_acc, n_mc_gen);
}

// ---- covariant amplitudes ------------------------------------------------

// Checks the covariant wave list and uploads it to *d_waves (freed by the caller).
static int upload_cov_waves(pwa_ctx *c, const pwa_cov_wave *waves, CovWave **d_waves)
{
    *d_waves = nullptr;
    if (!waves)
        return fail(c, PWA_EINVAL, "null wave list");
    std::vector<CovWave> h(c->N);
    for (int a = 0; a < c->N; ++a) {
        const pwa_cov_wave &w = waves[a];
        if (w.spin != 0 && w.spin != 2)
            return fail(c, PWA_EINVAL, "wave %d: spin %d is neither 0 nor 2", a, w.spin);
        if (!(w.mass > 0) || !(w.width > 0) || !std::isfinite(w.mass) || !std::isfinite(w.width))
            return fail(c, PWA_EINVAL, "wave %d: mass and width must be positive and finite", a);
        h[a] = CovWave{w.mass, w.width, w.spin};
    }
    int rc = dev_alloc(c, (void **)d_waves, c->N * sizeof(CovWave), "wave table");
    if (rc)
        return rc;
    CK(c, cudaMemcpyAsync(*d_waves, h.data(), c->N * sizeof(CovWave), cudaMemcpyHostToDevice,
                          c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return PWA_OK;
}

// Covariant amplitudes of n events (p3 host or device) into `out` (device,
// event-major [n][4][N] complex64).
static int generate_cov(pwa_ctx *c, const CovWave *d_waves, const double *p3, int64_t n, float *out)
{
    const double *dk = p3;
    double *staging = nullptr;
    if (is_device_pointer(p3)) {
        if (int rc = device_input_ready(c))
            return rc;
    } else {
        int rc = dev_alloc(c, (void **)&staging, (size_t)n * 9 * sizeof(double), "momenta");
        if (rc)
            return rc;
        cudaError_t e = cudaMemcpyAsync(staging, p3, (size_t)n * 9 * sizeof(double),
                                        cudaMemcpyHostToDevice, c->stream);
        if (e != cudaSuccess) {
            cudaStreamSynchronize(c->stream);
            cudaFree(staging);
            return fail(c, PWA_ECUDA, "momenta copy: %s", cudaGetErrorString(e));
        }
        dk = staging;
    }
    cudaError_t e = launch_cov_amp_gen(dk, n, c->N, d_waves, out, false, 0, c->num_sms * 8, c->stream);
    cudaError_t e2 = cudaStreamSynchronize(c->stream);
    if (staging)
        cudaFree(staging);
    if (e == cudaSuccess)
        e = e2;
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, PWA_ECUDA, "covariant amplitudes: %s", cudaGetErrorString(e));
    }
    return PWA_OK;
}

int pwa_compute_covariant_amplitudes(pwa_ctx *c, const pwa_cov_wave *waves, const double *p3,
                                     int64_t n, void *out)
{
    if (!c)
        return PWA_EINVAL;
    if (!p3 || !out)
        return fail(c, PWA_EINVAL, "null momenta or output");
    if (n < 1 || n > ((int64_t)1 << 31) - 1024)
        return fail(c, PWA_EINVAL, "n=%lld outside [1, 2^31 - 1024]", (long long)n);
    DeviceGuard g(c->device);
    CovWave *dw;
    int rc = upload_cov_waves(c, waves, &dw);
    if (rc) {
        dev_free(dw);
        return rc;
    }
    const size_t bytes = (size_t)n * 4 * c->N * 8;
    const bool on_dev = is_device_pointer(out);
    float *dout = static_cast<float *>(out);
    if (!on_dev)
        rc = dev_alloc(c, (void **)&dout, bytes, "amplitudes");
    if (!rc)
        rc = generate_cov(c, dw, p3, n, dout);
    if (!rc && !on_dev) {
        cudaError_t e = cudaMemcpy(out, dout, bytes, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess)
            rc = fail(c, PWA_ECUDA, "amplitude copy: %s", cudaGetErrorString(e));
    }
    if (!on_dev)
        dev_free(dout);
    dev_free(dw);
    return rc;
}

// The amplitudes of both samples go through device buffers of this call into
// the incoherent loader (which copies them into its planes), so that every
// check and store that loader makes applies unchanged.
int pwa_load_events_covariant(pwa_ctx *c, const pwa_cov_wave *waves, const double *data_p3,
                              int64_t n_data, const double *mc_p3, int64_t n_mc_acc,
                              double n_mc_gen)
{
    if (!c)
        return PWA_EINVAL;
    if (!data_p3 || !mc_p3)
        return fail(c, PWA_EINVAL, "null momenta");
    if (n_data < 1 || n_mc_acc < 1)
        return fail(c, PWA_EINVAL, "n_data=%lld and n_mc_acc=%lld must be >= 1",
                    (long long)n_data, (long long)n_mc_acc);
    if (n_data > ((int64_t)1 << 31) - 1024 || n_mc_acc * 4 > ((int64_t)1 << 31) - 1024)
        return fail(c, PWA_EINVAL, "samples are limited to 2^31 - 1024 events (MC: 4 x events)");
    DeviceGuard g(c->device);
    CovWave *dw;
    int rc = upload_cov_waves(c, waves, &dw);
    float *amp[2] = {nullptr, nullptr};
    const int64_t n[2] = {n_data, n_mc_acc};
    for (int k = 0; k < 2 && !rc; ++k) {
        rc = dev_alloc(c, (void **)&amp[k], (size_t)n[k] * 4 * c->N * 8, "amplitudes");
        if (!rc)
            rc = generate_cov(c, dw, k == 0 ? data_p3 : mc_p3, n[k], amp[k]);
    }
    dev_free(dw);
    if (!rc)
        rc = pwa_load_events_incoherent(c, 4, amp[0], n_data, amp[1], n_mc_acc, n_mc_gen, PWA_C64);
    cudaStreamSynchronize(c->stream);
    dev_free(amp[0]);
    dev_free(amp[1]);
    return rc;
}

int pwa_load_events_incoherent(pwa_ctx *c, int n_lambda, const void *data_amp, int64_t n_data,
                               const void *mc_amp, int64_t n_mc_acc, double n_mc_gen,
                               int amp_dtype)
{
    if (!c)
        return PWA_EINVAL;
    if (n_lambda == 1)
        return pwa_load_events(c, data_amp, n_data, mc_amp, n_mc_acc, n_mc_gen, amp_dtype);
    if (n_lambda < 1 || n_lambda > incoh_max_components())
        return fail(c, PWA_EINVAL, "n_lambda=%d outside [1, %d]", n_lambda, incoh_max_components());
    if (!data_amp || !mc_amp)
        return fail(c, PWA_EINVAL, "null amplitude pointer");
    if (n_data < 1 || n_mc_acc < 1)
        return fail(c, PWA_EINVAL, "n_data=%lld and n_mc_acc=%lld must be >= 1",
                    (long long)n_data, (long long)n_mc_acc);
    if (!(n_mc_gen >= (double)n_mc_acc))
        return fail(c, PWA_EINVAL, "n_mc_gen=%g must be >= n_mc_acc=%lld", n_mc_gen,
                    (long long)n_mc_acc);
    if (amp_dtype != PWA_C64 && amp_dtype != PWA_C128)
        return fail(c, PWA_EINVAL, "amp_dtype=%d is neither PWA_C64 nor PWA_C128", amp_dtype);
    if (n_data > ((int64_t)1 << 31) - 1024 || n_mc_acc * n_lambda > ((int64_t)1 << 31) - 1024)
        return fail(c, PWA_EINVAL, "samples are limited to 2^31 - 1024 events (MC: events x n_lambda)");
    if (c->cfg.forms & PWA_FORM_TC)
        return fail(c, PWA_ENOTSUP, "the tensor-core form takes coherent samples only");
    if ((c->cfg.forms & PWA_FORM_AMP) && c->N > incoh_max_waves(n_lambda))
        return fail(c, PWA_ENOTSUP, "the direct form takes up to %d waves at n_lambda=%d",
                    incoh_max_waves(n_lambda), n_lambda);
    DeviceGuard g(c->device);
    cudaStreamSynchronize(c->stream);
    free_sample(c);
    const int N = c->N, L = n_lambda;
    // data: [n][L][N] complex = n events of L N waves, plane 2 (l N + a) = Re A_a^l
    Planes &d = c->data;
    d.n = n_data;
    d.n_waves = L * N;
    d.pitch = round_up(n_data, 256);
    int rc = dev_alloc(c, (void **)&d.ptr, (size_t)2 * L * N * d.pitch * sizeof(float), "planes");
    if (!rc && cudaMemsetAsync(d.ptr, 0, (size_t)2 * L * N * d.pitch * sizeof(float), c->stream) !=
                   cudaSuccess)
        rc = fail(c, PWA_ECUDA, "memset");
    if (!rc)
        rc = pack_rows(c, data_amp, n_data, amp_dtype, L * N, d.ptr, d.pitch);
    // MC: the same bytes read as n L pseudo-events of N waves, so that M sums
    // the products over components as well as over events
    if (!rc)
        rc = load_planes(c, mc_amp, n_mc_acc * L, amp_dtype, &c->mc);
    if (!rc && (c->cfg.forms & PWA_FORM_TABLE)) {
        c->table_pitch = d.pitch;
        rc = dev_alloc(c, (void **)&c->table, (size_t)N * N * c->table_pitch * sizeof(float),
                       "table");
        if (!rc)
            rc = dev_alloc(c, (void **)&c->tmax, (size_t)N * N * sizeof(float), "tmax");
        if (!rc) {
            const int P = N * N;
            cudaError_t e = launch_table_build_incoh(d, L, c->table, c->table_pitch, c->stream);
            if (e == cudaSuccess)
                e = cudaMemsetAsync(c->tmax, 0, P * sizeof(float), c->stream);
            if (e == cudaSuccess)
                e = launch_plane_absmax(c->table, c->table_pitch, n_data, P, c->tmax, c->stream);
            if (e == cudaSuccess)
                e = encode_planes_map(&c->table_map, c->table, n_data, c->table_pitch, P,
                                      table_box_events(N), table_box_rows(N));
            if (e != cudaSuccess)
                rc = fail(c, PWA_ECUDA, "table build: %s", cudaGetErrorString(e));
        }
    }
    // The TMA-fed kernel (N_pad L <= 48) bounds its exact product split by
    // amax[a] = max over components and events of |Re A_a^l| + |Im A_a^l|; it
    // reads all 2 L n planes as one box per tile. PWA_INCOH_KERNEL=generic
    // selects the one-event-per-thread kernel instead.
    const char *kv = getenv("PWA_INCOH_KERNEL");
    const bool tma = (c->cfg.forms & PWA_FORM_AMP) && incoh_tma_available(N, L) &&
                     !(kv && strcmp(kv, "generic") == 0);
    if (!rc && cudaMemsetAsync(c->amax, 0, N * sizeof(float), c->stream) != cudaSuccess)
        rc = fail(c, PWA_ECUDA, "memset");
    // the MC planes hold n_mc_acc L pseudo-events of N waves: their maxima
    // scale the tensor-core build of M
    if (!rc && (cudaMemsetAsync(c->mc_amax, 0, N * sizeof(float), c->stream) != cudaSuccess ||
                launch_amp_max(c->mc, c->mc_amax, c->stream) != cudaSuccess))
        rc = fail(c, PWA_ECUDA, "MC amplitude maxima");
    if (!rc && tma) {
        float *dmax = nullptr;
        rc = dev_alloc(c, (void **)&dmax, (size_t)L * N * sizeof(float), "component maxima");
        std::vector<float> hmax((size_t)L * N), amax(N, 0.f);
        cudaError_t e = cudaSuccess;
        if (!rc) {
            e = cudaMemsetAsync(dmax, 0, (size_t)L * N * sizeof(float), c->stream);
            if (e == cudaSuccess)
                e = launch_amp_max(d, dmax, c->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(hmax.data(), dmax, (size_t)L * N * sizeof(float),
                                    cudaMemcpyDeviceToHost, c->stream);
            if (e == cudaSuccess)
                e = cudaStreamSynchronize(c->stream);
            for (int l = 0; l < L && e == cudaSuccess; ++l)
                for (int a = 0; a < N; ++a)
                    amax[a] = std::max(amax[a], hmax[(size_t)l * N + a]);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(c->amax, amax.data(), N * sizeof(float), cudaMemcpyHostToDevice,
                                    c->stream);
            if (e == cudaSuccess)
                e = encode_planes_map(&c->data_map, d.ptr, n_data, d.pitch, 2 * L * N,
                                      incoh_tma_box_events(), 2 * L * N);
            if (e != cudaSuccess)
                rc = fail(c, PWA_ECUDA, "incoherent direct-form set-up: %s", cudaGetErrorString(e));
        }
        if (dmax) {
            cudaStreamSynchronize(c->stream);
            cudaFree(dmax);
        }
    }
    if (!rc) {
        cudaError_t e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess)
            rc = fail(c, PWA_ECUDA, "loading: %s", cudaGetErrorString(e));
    }
    if (rc) {
        free_sample(c);
        return rc;
    }
    c->n_lambda = L;
    c->incoh_tma = tma;
    c->n_data = n_data;
    c->n_mc = n_mc_acc;
    c->n_gen = n_mc_gen;
    c->loaded = true;
    c->has_norm = false;
    return PWA_OK;
}

int pwa_build_norm(pwa_ctx *c, double *M_out)
{
    if (!c)
        return PWA_EINVAL;
    if (!c->loaded)
        return fail(c, PWA_ESTATE, "pwa_load_events must come first");
    DeviceGuard g(c->device);
    // The tensor-core kernel serves up to 20 waves when every wave's scale is
    // in its range; the FP64 kernel everything else (or PWA_NORM_KERNEL=fp64).
    bool tc = norm_tc_available(c->N);
    if (const char *v = getenv("PWA_NORM_KERNEL"))
        if (strcmp(v, "fp64") == 0)
            tc = false;
    if (tc) {
        std::vector<float> am(c->N);
        CK(c, cudaMemcpy(am.data(), c->mc_amax, c->N * sizeof(float), cudaMemcpyDeviceToHost));
        for (float x : am)
            tc = tc && norm_tc_scale_ok(x);
    }
    if (tc) {
        CUtensorMap map;
        CK(c, encode_planes_map(&map, c->mc.ptr, c->mc.n, c->mc.pitch, 2 * c->N,
                                norm_tc_box_events(), 2 * c->N));
        const int grid = c->num_sms;
        const size_t nd = norm_tc_partials_doubles(c->N, grid);
        double *scratch = nullptr;
        int rc = dev_alloc(c, (void **)&scratch, (nd + 1) * sizeof(double), "norm scratch");
        if (rc)
            return rc;
        int *dstat = reinterpret_cast<int *>(scratch + nd);
        int flags = 0;
        cudaError_t e = cudaMemsetAsync(dstat, 0, sizeof(int), c->stream);
        if (e == cudaSuccess)
            e = launch_build_norm_tc(&map, c->mc, c->mc_amax, c->n_gen, scratch, grid, dstat, c->M,
                                     c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&flags, dstat, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(c->stream);
        cudaFree(scratch);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(c, PWA_ECUDA, "build_norm: %s", cudaGetErrorString(e));
        }
        if (flags & FLAG_TIMEOUT)
            return fail(c, PWA_ETIMEOUT, "build_norm: a device-side wait timed out");
    } else {
        double *scratch = nullptr;
        int rc = dev_alloc(c, (void **)&scratch, norm_scratch_bytes(c->N, c->num_sms), "norm scratch");
        if (rc)
            return rc;
        cudaError_t e = launch_build_norm(c->mc, c->n_gen, c->M, scratch, c->num_sms, c->stream);
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(c->stream);
        cudaFree(scratch);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(c, PWA_ECUDA, "build_norm: %s", cudaGetErrorString(e));
        }
    }
    if (M_out)
        CK(c, cudaMemcpy(M_out, c->M, (size_t)2 * c->N * c->N * sizeof(double),
                         cudaMemcpyDeviceToHost));
    c->has_norm = true;
    return PWA_OK;
}

int pwa_set_form(pwa_ctx *c, int form)
{
    if (!c)
        return PWA_EINVAL;
    if (form != PWA_FORM_AMP && form != PWA_FORM_TABLE && form != PWA_FORM_TC)
        return fail(c, PWA_EINVAL, "unknown form %d", form);
    if (!(c->cfg.forms & form))
        return fail(c, PWA_ESTATE, "form %d was not requested at pwa_create", form);
    if (form == PWA_FORM_TC && c->n_lambda > 1)
        return fail(c, PWA_ENOTSUP, "the tensor-core form takes coherent samples only");
    if (form != c->form) {
        // the two kernels lay out the shared scratch differently: start clean
        DeviceGuard g(c->device);
        CK(c, cudaMemsetAsync(c->d_work, 0, c->work_bytes, c->stream));
        CK(c, cudaStreamSynchronize(c->stream));
    }
    c->form = form;
    ++c->epoch;
    return PWA_OK;
}

int pwa_nll(pwa_ctx *c, const double *V, int K, double *nll)
{
    if (!c)
        return PWA_EINVAL;
    return eval_host(c, V, K, nll, nullptr);
}

int pwa_nll_grad(pwa_ctx *c, const double *V, int K, double *nll, double *grad)
{
    if (!c)
        return PWA_EINVAL;
    if (!grad)
        return fail(c, PWA_EINVAL, "null grad");
    return eval_host(c, V, K, nll, grad);
}

int pwa_nll_grad_async(pwa_ctx *c, const double *d_V, int K, double *d_nll, double *d_grad)
{
    if (!c)
        return PWA_EINVAL;
    int rc = check_eval_args(c, d_V, K, d_nll);
    if (rc)
        return rc;
    DeviceGuard g(c->device);
    return enqueue_eval(c, d_V, K, d_nll, d_grad, c->async_status, nullptr);
}

int pwa_sync(pwa_ctx *c)
{
    if (!c)
        return PWA_EINVAL;
    DeviceGuard g(c->device);
    int flags = 0;
    CK(c, cudaMemcpyAsync(&flags, c->async_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaMemsetAsync(c->async_status, 0, sizeof(int), c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return status_from_flags(c, flags);
}

// ---- uneven model batch ------------------------------------------------------
constexpr int kBatchStreams = 4;

struct pwa_batch {
    int device = 0;
    std::vector<pwa_ctx *> models;
    std::vector<int> n_waves;
    std::vector<int> order;      // models by sample size, largest first
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t side[kBatchStreams] = {};
    cudaEvent_t ev_fork = nullptr, ev_join[kBatchStreams] = {};
    int max_k = 0, sum_n = 0;
    double *d_buf = nullptr, *h_buf = nullptr;  // V | nll | grad | status
    cudaGraphExec_t exec = nullptr;
    int graph_k = 0;
    // one launch over work items of every model (the default), or, with
    // PWA_BATCH_MODE=graph, a graph of per-model launches
    bool per_model = false;
    void *plan = nullptr;        // device plan of the one-launch form (for graph_k)
    size_t plan_bytes = 0;
    int items_per_sm = 16;       // work granularity (pwa_batch_autotune picks it)
    int tune_nxs = 0;            // X stages of the tensor-core kernel (0 = as many as fit)
    int num_sms = 0;
    char err[512] = {0};
};

static int bfail(pwa_batch *b, int code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    if (b)
        vsnprintf(b->err, sizeof b->err, fmt, ap);
    else
        vsnprintf(g_create_err, sizeof g_create_err, fmt, ap);
    va_end(ap);
    return code;
}

static void batch_drop_graph(pwa_batch *b)
{
    if (b->exec)
        cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    b->graph_k = 0;
    if (b->plan)
        cudaFree(b->plan);
    b->plan = nullptr;
    b->plan_bytes = 0;
}

// The models as the one-launch form sees them, for K sets per model.
static std::vector<BatchModelDesc> batch_descs(pwa_batch *b, int K)
{
    const int nm = (int)b->models.size();
    const size_t nv = 2 * (size_t)K * b->sum_n;
    double *dV = b->d_buf, *dN = dV + nv, *dG = dN + (size_t)nm * K;
    int *dS = reinterpret_cast<int *>(dG + nv);
    std::vector<BatchModelDesc> d(nm);
    size_t off = 0;
    for (int m = 0; m < nm; ++m) {
        const pwa_ctx *c = b->models[m];
        d[m].xbf = c->xbf;
        d[m].n_events = c->n_data;
        d[m].n_waves = c->N;
        d[m].sum_e = c->xsum;
        d[m].M = c->M;
        d[m].V = dV + off;
        d[m].nll = dN + (size_t)m * K;
        d[m].grad = dG + off;
        d[m].status = dS + 2 * m;
        d[m].done = dS + 2 * m + 1;
        off += 2 * (size_t)K * b->n_waves[m];
    }
    return d;
}

int pwa_batch_destroy(pwa_batch *b)
{
    if (!b)
        return PWA_OK;
    DeviceGuard g(b->device);
    if (b->stream)
        cudaStreamSynchronize(b->stream);
    batch_drop_graph(b);
    for (pwa_ctx *c : b->models)
        pwa_destroy(c);
    for (int s = 0; s < kBatchStreams; ++s) {
        if (b->side[s])
            cudaStreamDestroy(b->side[s]);
        if (b->ev_join[s])
            cudaEventDestroy(b->ev_join[s]);
    }
    if (b->ev_fork)
        cudaEventDestroy(b->ev_fork);
    if (b->d_buf)
        cudaFree(b->d_buf);
    if (b->h_buf)
        cudaFreeHost(b->h_buf);
    if (b->own_stream && b->stream)
        cudaStreamDestroy(b->stream);
    delete b;
    return PWA_OK;
}

const char *pwa_batch_last_error(const pwa_batch *b) { return b ? b->err : g_create_err; }

int pwa_batch_create(pwa_batch **out, int device, int n_models, const int *n_waves, int max_k,
                     int precision, void *stream)
{
    if (!out || !n_waves || n_models < 1 || n_models > 65536)
        return bfail(nullptr, PWA_EINVAL, "null out or n_waves, or n_models outside [1, 65536]");
    *out = nullptr;
    const int xs = precision == PWA_PREC_BFP8 ? 1 : 2;
    for (int m = 0; m < n_models; ++m) {
        if (n_waves[m] < 1 || n_waves[m] > kMaxWaves)
            return bfail(nullptr, PWA_EINVAL, "model %d: n_waves=%d outside [1, %d]", m, n_waves[m],
                         kMaxWaves);
        if (max_k < 1 || max_k > batched_max_k(n_waves[m], xs))
            return bfail(nullptr, PWA_ENOTSUP, "model %d: max_k=%d outside [1, %d]", m, max_k,
                         batched_max_k(n_waves[m], xs));
    }
    DeviceGuard g(device);
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return bfail(nullptr, PWA_ECUDA, "device %d not available", device);
    }
    pwa_batch *b = new pwa_batch();
    b->device = device;
    b->max_k = max_k;
    if (const char *v = getenv("PWA_BATCH_MODE"))
        b->per_model = strcmp(v, "graph") == 0;
    if (cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        cudaGetLastError();
        b->num_sms = 1;
    }
    b->n_waves.assign(n_waves, n_waves + n_models);
    b->sum_n = std::accumulate(b->n_waves.begin(), b->n_waves.end(), 0);
    auto bail = [&](int code) {
        snprintf(g_create_err, sizeof g_create_err, "%s", b->err);
        pwa_batch_destroy(b);
        return code;
    };
    if (stream) {
        b->stream = static_cast<cudaStream_t>(stream);
    } else {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess)
            return bail(bfail(b, PWA_ECUDA, "cudaStreamCreate failed"));
        b->own_stream = true;
    }
    for (int s = 0; s < kBatchStreams; ++s)
        if (cudaStreamCreateWithFlags(&b->side[s], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&b->ev_join[s], cudaEventDisableTiming) != cudaSuccess)
            return bail(bfail(b, PWA_ECUDA, "stream or event creation failed"));
    if (cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) != cudaSuccess)
        return bail(bfail(b, PWA_ECUDA, "event creation failed"));
    for (int m = 0; m < n_models; ++m) {
        pwa_config cfg{};
        cfg.n_waves = n_waves[m];
        cfg.forms = PWA_FORM_TC;
        cfg.precision = precision;
        cfg.max_k = max_k;
        cfg.stream = b->side[m % kBatchStreams];
        pwa_ctx *c = nullptr;
        const int rc = pwa_create(&c, device, &cfg);
        if (rc)
            return bail(bfail(b, rc, "model %d: %s", m, g_create_err));
        b->models.push_back(c);
    }
    const size_t nd = 4 * (size_t)max_k * b->sum_n + (size_t)n_models * max_k + n_models;
    if (cudaMalloc((void **)&b->d_buf, nd * sizeof(double)) != cudaSuccess ||
        cudaMallocHost((void **)&b->h_buf, nd * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return bail(bfail(b, PWA_ENOMEM, "batch io buffers (%zu doubles)", nd));
    }
    b->order.resize(n_models);
    std::iota(b->order.begin(), b->order.end(), 0);
    *out = b;
    return PWA_OK;
}

int pwa_batch_load_model(pwa_batch *b, int model, const void *data_amp, int64_t n_data,
                         const void *mc_amp, int64_t n_mc_acc, double n_mc_gen, int amp_dtype)
{
    if (!b)
        return PWA_EINVAL;
    if (model < 0 || model >= (int)b->models.size())
        return bfail(b, PWA_EINVAL, "model %d outside [0, %zu)", model, b->models.size());
    pwa_ctx *c = b->models[model];
    DeviceGuard g(b->device);
    cudaStreamSynchronize(b->stream);
    batch_drop_graph(b);
    int rc = pwa_load_events(c, data_amp, n_data, mc_amp, n_mc_acc, n_mc_gen, amp_dtype);
    if (!rc)
        rc = pwa_build_norm(c, nullptr);
    if (!rc)
        rc = pwa_set_form(c, PWA_FORM_TC);
    if (rc)
        return bfail(b, rc, "model %d: %s", model, c->err);
    // largest samples first: they set the length of the graph
    std::stable_sort(b->order.begin(), b->order.end(), [&](int x, int y) {
        const pwa_ctx *cx = b->models[x], *cy = b->models[y];
        return (double)cx->n_data * cx->N > (double)cy->n_data * cy->N;
    });
    return PWA_OK;
}

// The graph of one evaluation of every model for K sets (and, in the
// one-launch form, its plan), built on first use for K and kept until a
// model is reloaded or the launch shape changes.
static int batch_prepare(pwa_batch *b, int K)
{
    const int nm = (int)b->models.size();
    const size_t nv = 2 * (size_t)K * b->sum_n;  // doubles of V (and of grad)
    double *dV = b->d_buf, *dN = dV + nv, *dG = dN + (size_t)nm * K;
    int *dS = reinterpret_cast<int *>(dG + nv);  // [nm][2]: flags, done
    std::vector<size_t> off(nm);
    for (int m = 1; m < nm; ++m)
        off[m] = off[m - 1] + 2 * (size_t)K * b->n_waves[m - 1];
    if (!b->exec || b->graph_k != K) {
        batch_drop_graph(b);
        std::vector<BatchModelDesc> descs;
        const int xs = b->models[0]->xs;
        if (!b->per_model) {
            // the plan of the one-launch form: arguments, maps and work items
            descs = batch_descs(b, K);
            b->plan_bytes = batched_plan_bytes(descs.data(), nm, xs, K, b->num_sms,
                                               b->items_per_sm, nullptr);
            if (cudaMalloc(&b->plan, b->plan_bytes) != cudaSuccess) {
                cudaGetLastError();
                b->plan = nullptr;
                return bfail(b, PWA_ENOMEM, "batch plan (%zu bytes)", b->plan_bytes);
            }
            const cudaError_t pe = batched_plan_build(b->plan, descs.data(), nm, xs, K, b->num_sms,
                                                      b->items_per_sm, b->tune_nxs, b->stream);
            if (pe != cudaSuccess) {
                cudaGetLastError();
                return bfail(b, PWA_ECUDA, "batch plan: %s", cudaGetErrorString(pe));
            }
        }
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
        int rc = PWA_OK;
        if (e == cudaSuccess)
            e = cudaMemsetAsync(dS, 0, (size_t)nm * 2 * sizeof(int), b->stream);
        if (e == cudaSuccess && !b->per_model)
            e = launch_batched_items(b->plan, descs.data(), nm, xs, K, b->num_sms, b->items_per_sm,
                                     b->tune_nxs, b->stream);
        if (e == cudaSuccess && b->per_model)
            e = cudaEventRecord(b->ev_fork, b->stream);
        for (int s = 0; s < kBatchStreams && e == cudaSuccess && b->per_model; ++s)
            e = cudaStreamWaitEvent(b->side[s], b->ev_fork, 0);
        for (int i = 0; i < nm && e == cudaSuccess && !rc && b->per_model; ++i) {
            const int m = b->order[i];
            pwa_ctx *c = b->models[m];
            c->stream = b->side[i % kBatchStreams];
            rc = enqueue_eval(c, dV + off[m], K, dN + (size_t)m * K, dG + off[m], dS + 2 * m,
                              dS + 2 * m + 1);
            if (rc)
                bfail(b, rc, "model %d: %s", m, c->err);
        }
        for (int s = 0; s < kBatchStreams && e == cudaSuccess && b->per_model; ++s) {
            e = cudaEventRecord(b->ev_join[s], b->side[s]);
            if (e == cudaSuccess)
                e = cudaStreamWaitEvent(b->stream, b->ev_join[s], 0);
        }
        const cudaError_t e2 = cudaStreamEndCapture(b->stream, &graph);
        if (e == cudaSuccess)
            e = e2;
        if (e == cudaSuccess && !rc)
            e = cudaGraphInstantiate(&b->exec, graph, 0);
        if (graph)
            cudaGraphDestroy(graph);
        if (rc || e != cudaSuccess) {
            cudaGetLastError();
            b->exec = nullptr;
            return rc ? rc : bfail(b, PWA_ECUDA, "graph capture: %s", cudaGetErrorString(e));
        }
        b->graph_k = K;
    }
    return PWA_OK;
}

int pwa_batch_nll_grad(pwa_batch *b, const double *V_all, int K, double *nll, double *grad)
{
    if (!b)
        return PWA_EINVAL;
    if (!V_all || !nll)
        return bfail(b, PWA_EINVAL, "null V_all or nll");
    if (K < 1 || K > b->max_k)
        return bfail(b, PWA_EINVAL, "K=%d outside [1, max_k=%d]", K, b->max_k);
    const int nm = (int)b->models.size();
    for (int m = 0; m < nm; ++m)
        if (!b->models[m]->loaded || !b->models[m]->has_norm)
            return bfail(b, PWA_ESTATE, "model %d has no samples (pwa_batch_load_model)", m);
    DeviceGuard g(b->device);
    const size_t nv = 2 * (size_t)K * b->sum_n;  // doubles of V (and of grad)
    double *dV = b->d_buf, *dN = dV + nv, *dG = dN + (size_t)nm * K;
    int *dS = reinterpret_cast<int *>(dG + nv);  // [nm][2]: flags, done
    int rc = batch_prepare(b, K);
    if (rc)
        return rc;
    double *h = b->h_buf;
    memcpy(h, V_all, nv * sizeof(double));
    cudaError_t e = cudaMemcpyAsync(dV, h, nv * sizeof(double), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaGraphLaunch(b->exec, b->stream);
    const size_t nout = (size_t)nm * K + (grad ? nv : 0);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h + nv, dN, nout * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h + nv + (size_t)nm * K + nv, dS, (size_t)nm * 2 * sizeof(int),
                            cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return bfail(b, PWA_ECUDA, "batch launch: %s", cudaGetErrorString(e));
    }
    const int *hs = reinterpret_cast<const int *>(h + nv + (size_t)nm * K + nv);
    int flags = 0;
    for (int m = 0; m < nm; ++m) {
        if (hs[2 * m + 1] != K)
            return bfail(b, PWA_ETIMEOUT, "model %d: only %d of %d evaluations finished", m,
                         hs[2 * m + 1], K);
        flags |= hs[2 * m];
    }
    memcpy(nll, h + nv, (size_t)nm * K * sizeof(double));
    if (grad)
        memcpy(grad, h + nv + (size_t)nm * K, nv * sizeof(double));
    if (flags & FLAG_TIMEOUT)
        return bfail(b, PWA_ETIMEOUT, "a device-side wait timed out; results are invalid");
    if (flags & FLAG_DOMAIN)
        return bfail(b, PWA_EDOMAIN, "an intensity was not positive and finite (nll = +inf)");
    return PWA_OK;
}

// ---- autotuner -------------------------------------------------------------------
// Cache file: a JSON object, one entry per line, "key": {"choice": C, "us": T}.
extern "C++" {

static std::string tune_key(const pwa_ctx *c, const char *what)
{
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, c->device) != cudaSuccess) {
        cudaGetLastError();
        snprintf(p.name, sizeof p.name, "device%d", c->device);
    }
    char buf[320];
    snprintf(buf, sizeof buf, "%s|sm%d|%s|N%d", p.name, c->num_sms, what, c->N);
    for (char *q = buf; *q; ++q)
        if (*q == '"' || *q == '\\')
            *q = '_';
    return buf;
}

static bool read_cache(const char *path, std::vector<std::pair<std::string, std::string>> &rows)
{
    rows.clear();
    FILE *f = fopen(path, "r");
    if (!f)
        return true;  // no file yet
    char line[1024];
    while (fgets(line, sizeof line, f)) {
        const char *a = strchr(line, '"');
        const char *b = a ? strchr(a + 1, '"') : nullptr;
        const char *v = b ? strchr(b, '{') : nullptr;
        const char *w = v ? strchr(v, '}') : nullptr;
        if (!w)
            continue;
        rows.emplace_back(std::string(a + 1, b), std::string(v, w + 1));
    }
    fclose(f);
    return true;
}

static bool cache_lookup(const char *path, const std::string &key, int *choice)
{
    std::vector<std::pair<std::string, std::string>> rows;
    if (!path || !read_cache(path, rows))
        return false;
    for (auto &r : rows)
        if (r.first == key) {
            const char *q = strstr(r.second.c_str(), "\"choice\":");
            return q && sscanf(q + 9, "%d", choice) == 1;
        }
    return false;
}

static bool cache_store(const char *path, const std::string &key, int choice, double us)
{
    std::vector<std::pair<std::string, std::string>> rows;
    read_cache(path, rows);
    char val[96];
    snprintf(val, sizeof val, "{\"choice\": %d, \"us\": %.3f}", choice, us);
    bool found = false;
    for (auto &r : rows)
        if (r.first == key) {
            r.second = val;
            found = true;
        }
    if (!found)
        rows.emplace_back(key, val);
    const std::string tmp = std::string(path) + ".tmp";
    FILE *f = fopen(tmp.c_str(), "w");
    if (!f)
        return false;
    fprintf(f, "{\n");
    for (size_t i = 0; i < rows.size(); ++i)
        fprintf(f, "\"%s\": %s%s\n", rows[i].first.c_str(), rows[i].second.c_str(),
                i + 1 < rows.size() ? "," : "");
    fprintf(f, "}\n");
    const bool ok = fclose(f) == 0;
    return ok && rename(tmp.c_str(), path) == 0;
}

// Mean time in microseconds of `reps` calls of enqueue() after `warm` untimed ones.
template <typename F>
static int time_variant(pwa_ctx *c, F enqueue, int warm, int reps, double *us)
{
    cudaEvent_t e0, e1;
    CK(c, cudaEventCreate(&e0));
    CK(c, cudaEventCreate(&e1));
    int rc = PWA_OK;
    for (int i = 0; i < warm && !rc; ++i)
        rc = enqueue();
    cudaEventRecord(e0, c->stream);
    for (int i = 0; i < reps && !rc; ++i)
        rc = enqueue();
    cudaEventRecord(e1, c->stream);
    float ms = 0.f;
    if (!rc && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
        rc = fail(c, PWA_ECUDA, "timing events failed");
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *us = 1e3 * ms / reps;
    return rc;
}

}  // extern "C++"

int pwa_autotune(pwa_ctx *c, const char *cache_path, char *choice, int choice_len)
{
    if (!c)
        return PWA_EINVAL;
    if (!(c->loaded && c->has_norm) && !c->res_loaded)
        return fail(c, PWA_ESTATE, "nothing to tune: load a sample first");
    DeviceGuard g(c->device);
    std::string summary;
    char buf[256];
    if (c->loaded && c->has_norm) {
        if (c->form == PWA_FORM_AMP && c->n_lambda > 1) {
            summary += "incoherent direct form: one launch shape";
        } else if (c->form == PWA_FORM_AMP) {
            const std::string key = tune_key(c, "amp-groups");
            int best = 0;
            double best_us = 0.0;
            if (!cache_lookup(cache_path, key, &best)) {
                // one parameter set, V_a = 1 for every wave, in the io buffer
                const int N = c->N;
                std::vector<double> V(2 * N, 0.0);
                for (int a = 0; a < N; ++a)
                    V[2 * a] = 1.0;
                double *dV = c->d_io + 1 + 2 * N + 1;
                int *ds = reinterpret_cast<int *>(c->d_io + 1 + 2 * N);
                CK(c, cudaMemcpyAsync(dV, V.data(), 2 * N * sizeof(double), cudaMemcpyHostToDevice,
                                      c->stream));
                for (int gr : {2, 3}) {
                    if (gr == 3 && !amp_groups3_available(N))
                        continue;
                    c->tune_groups = gr;
                    CK(c, cudaMemsetAsync(c->d_work, 0, c->work_bytes, c->stream));
                    double us = 0.0;
                    const int rc = time_variant(
                        c, [&] { return enqueue_eval(c, dV, 1, c->d_io, c->d_io + 1, ds, ds + 1); },
                        3, 20, &us);
                    if (rc)
                        return rc;
                    if (!best || us < best_us) {
                        best = gr;
                        best_us = us;
                    }
                }
                CK(c, cudaMemsetAsync(c->d_work, 0, c->work_bytes, c->stream));
                CK(c, cudaStreamSynchronize(c->stream));
                if (cache_path && !cache_store(cache_path, key, best, best_us))
                    return fail(c, PWA_EINVAL, "cannot write the tuning cache %s", cache_path);
                snprintf(buf, sizeof buf, "direct form: %d consumer groups (%.1f us, timed)", best, best_us);
            } else {
                snprintf(buf, sizeof buf, "direct form: %d consumer groups (cached)", best);
            }
            c->tune_groups = best;
            ++c->epoch;
            summary += buf;
        } else if (c->form == PWA_FORM_TC) {
            // tile parameters of the tensor-core form for K = max_k sets: sets
            // per launch (multiples of 64 up to the launch limit) and X
            // pipeline stages (2 up to what shared memory takes)
            const int N = c->N, K = c->cfg.max_k;
            char what[64];
            snprintf(what, sizeof what, "tc-tiles|K%d|xs%d", K, c->xs);
            const std::string key = tune_key(c, what);
            int best = 0;
            double best_us = 0.0;
            if (!cache_lookup(cache_path, key, &best)) {
                const size_t gK = (size_t)2 * N * K;
                std::vector<double> V(gK, 0.0);
                for (size_t i = 0; i < gK; i += 2)
                    V[i] = 1.0;
                double *dV = c->d_io + K + gK + 1;
                int *ds = reinterpret_cast<int *>(c->d_io + K + gK);
                CK(c, cudaMemcpyAsync(dV, V.data(), gK * sizeof(double), cudaMemcpyHostToDevice,
                                      c->stream));
                const int kmax = batched_max_k(N, c->xs);
                for (int per = 64; per <= std::max(64, std::min(kmax, ((K + 63) / 64) * 64)); per += 64) {
                    const int top = batched_max_x_stages(N, c->xs, std::min(per, K));
                    for (int nxs = 2; nxs <= top; ++nxs) {
                        c->tune_tc_per = per;
                        c->tune_tc_nxs = nxs;
                        double us = 0.0;
                        const int rc = time_variant(
                            c, [&] { return enqueue_eval(c, dV, K, c->d_io, c->d_io + K, ds, ds + 1); },
                            2, 5, &us);
                        if (rc)
                            return rc;
                        if (!best || us < best_us) {
                            best = nxs * 10000 + per;
                            best_us = us;
                        }
                    }
                }
                CK(c, cudaStreamSynchronize(c->stream));
                if (cache_path && !cache_store(cache_path, key, best, best_us))
                    return fail(c, PWA_EINVAL, "cannot write the tuning cache %s", cache_path);
                snprintf(buf, sizeof buf,
                         "tensor-core form: %d sets per launch, %d X stages (%.1f us for %d sets, timed)",
                         best % 10000, best / 10000, best_us, K);
            } else {
                snprintf(buf, sizeof buf, "tensor-core form: %d sets per launch, %d X stages (cached)",
                         best % 10000, best / 10000);
            }
            c->tune_tc_per = best % 10000;
            c->tune_tc_nxs = best / 10000;
            ++c->epoch;
            summary += buf;
        } else {
            summary += "table form: one launch shape";
        }
    }
    if (c->res_loaded && c->res_tma) {
        summary += summary.empty() ? "" : "; ";
        summary += "free resonances: TMA-fed kernel, one launch shape";
    } else if (c->res_loaded) {
        const std::string key = tune_key(c, "res-blocks-per-sm");
        int best = 0;
        double best_us = 0.0;
        if (!cache_lookup(cache_path, key, &best)) {
            const int N = c->N, R = c->res_R;
            const size_t npart = res_partials_doubles(N, R, c->num_sms * kResMaxBlocksPerSm);
            double *d_io = c->d_res + npart + 1;
            std::vector<double> h(2 * N + 2 * R, 0.0);
            for (int a = 0; a < N; ++a)
                h[2 * a] = 1.0;
            for (int r = 0; r < R; ++r) {
                h[2 * N + r] = 1.5;
                h[2 * N + R + r] = 0.1;
            }
            CK(c, cudaMemcpyAsync(d_io, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice,
                                  c->stream));
            ResArgs a{};
            a.n_waves = N;
            a.n_free = R;
            a.data = c->res_data;
            a.data_pitch = c->res_data_pitch;
            a.n_data = c->res_n_data;
            a.mc = c->res_mc;
            a.mc_pitch = c->res_mc_pitch;
            a.n_mc = c->res_n_mc;
            a.inv_ngen = 1.0 / c->res_ngen;
            a.V = d_io;
            a.mass = d_io + 2 * N;
            a.width = d_io + 2 * N + R;
            a.partials = c->d_res;
            a.ticket = reinterpret_cast<unsigned *>(c->d_res + npart);
            int *ds = reinterpret_cast<int *>(d_io + 2 * N + 2 * R);
            a.status = ds;
            a.done = nullptr;
            a.out = d_io + 2 * N + 2 * R + 1;
            for (int cps = 1; cps <= kResMaxBlocksPerSm; ++cps) {
                double us = 0.0;
                const int rc = time_variant(
                    c,
                    [&] {
                        const cudaError_t e = launch_nll_res(a, c->num_sms * cps, c->stream);
                        return e == cudaSuccess ? PWA_OK
                                                : fail(c, PWA_ECUDA, "%s", cudaGetErrorString(e));
                    },
                    2, 10, &us);
                if (rc)
                    return rc;
                if (!best || us < best_us) {
                    best = cps;
                    best_us = us;
                }
            }
            CK(c, cudaStreamSynchronize(c->stream));
            if (cache_path && !cache_store(cache_path, key, best, best_us))
                return fail(c, PWA_EINVAL, "cannot write the tuning cache %s", cache_path);
            snprintf(buf, sizeof buf, "%sfree resonances: %d blocks per SM (%.1f us, timed)",
                     summary.empty() ? "" : "; ", best, best_us);
        } else {
            snprintf(buf, sizeof buf, "%sfree resonances: %d blocks per SM (cached)",
                     summary.empty() ? "" : "; ", best);
        }
        c->tune_res_cps = best;
        summary += buf;
    }
    if (choice && choice_len > 0)
        snprintf(choice, (size_t)choice_len, "%s", summary.c_str());
    return PWA_OK;
}

int pwa_batch_autotune(pwa_batch *b, const char *cache_path, char *choice, int choice_len)
{
    if (!b)
        return PWA_EINVAL;
    const int nm = (int)b->models.size();
    for (int m = 0; m < nm; ++m)
        if (!b->models[m]->loaded || !b->models[m]->has_norm)
            return bfail(b, PWA_ESTATE, "model %d has no samples (pwa_batch_load_model)", m);
    char buf[256];
    if (b->per_model) {
        snprintf(buf, sizeof buf, "model batch: per-model graph, the models' own launch shapes");
        if (choice && choice_len > 0)
            snprintf(choice, (size_t)choice_len, "%s", buf);
        return PWA_OK;
    }
    DeviceGuard g(b->device);
    const int K = b->max_k, xs = b->models[0]->xs;
    // the key: device, models (count, total waves and events), K, precision
    int64_t n_events = 0;
    for (pwa_ctx *c : b->models)
        n_events += c->n_data;
    char what[128];
    snprintf(what, sizeof what, "batch|M%d|W%d|E%lld|K%d|xs%d", nm, b->sum_n, (long long)n_events,
             K, xs);
    const std::string key = tune_key(b->models[0], what);
    int best = 0;
    double best_us = 0.0;
    if (!cache_lookup(cache_path, key, &best)) {
        // V_a = 1 for every set of every model
        const size_t nv = 2 * (size_t)K * b->sum_n;
        std::vector<double> V(nv, 0.0);
        for (size_t i = 0; i < nv; i += 2)
            V[i] = 1.0;
        if (cudaMemcpy(b->d_buf, V.data(), nv * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaGetLastError();
            return bfail(b, PWA_ECUDA, "autotune: copy of V failed");
        }
        int top = 2;
        for (int m = 0; m < nm; ++m)
            top = std::max(top, batched_max_x_stages(b->n_waves[m], xs, K));
        cudaEvent_t e0, e1;
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
            cudaGetLastError();
            return bfail(b, PWA_ECUDA, "autotune: event creation failed");
        }
        int rc = PWA_OK;
        for (int ips : {4, 8, 16, 32}) {
            for (int nxs = 2; nxs <= top && !rc; ++nxs) {
                b->items_per_sm = ips;
                b->tune_nxs = nxs;
                batch_drop_graph(b);
                if ((rc = batch_prepare(b, K)))
                    break;
                float ms = 0.f;
                cudaError_t e = cudaGraphLaunch(b->exec, b->stream);   // warm-up
                if (e == cudaSuccess)
                    e = cudaEventRecord(e0, b->stream);
                for (int r = 0; r < 3 && e == cudaSuccess; ++r)
                    e = cudaGraphLaunch(b->exec, b->stream);
                if (e == cudaSuccess)
                    e = cudaEventRecord(e1, b->stream);
                if (e == cudaSuccess)
                    e = cudaEventSynchronize(e1);
                if (e == cudaSuccess)
                    e = cudaEventElapsedTime(&ms, e0, e1);
                if (e != cudaSuccess) {
                    cudaGetLastError();
                    rc = bfail(b, PWA_ECUDA, "autotune: %s", cudaGetErrorString(e));
                    break;
                }
                const double us = 1e3 * ms / 3;
                if (!best || us < best_us) {
                    best = nxs * 100 + ips;
                    best_us = us;
                }
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (rc)
            return rc;
        if (cache_path && !cache_store(cache_path, key, best, best_us))
            return bfail(b, PWA_EINVAL, "cannot write the tuning cache %s", cache_path);
        snprintf(buf, sizeof buf, "model batch: %d work items per SM, %d X stages (%.1f us for %d sets, timed)",
                 best % 100, best / 100, best_us, K);
    } else {
        snprintf(buf, sizeof buf, "model batch: %d work items per SM, %d X stages (cached)", best % 100,
                 best / 100);
    }
    b->items_per_sm = best % 100;
    b->tune_nxs = best / 100;
    batch_drop_graph(b);
    if (choice && choice_len > 0)
        snprintf(choice, (size_t)choice_len, "%s", buf);
    return PWA_OK;
}

}  // extern "C"
