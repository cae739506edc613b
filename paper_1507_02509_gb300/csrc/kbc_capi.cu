// C ABI of the D2Q9 KBC library (declarations and contracts: include/kbc.h).
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include <cufft.h>

#include "../../include/kbc.h"
#include "kbc_launch.cuh"
#include "kbc_spectrum.cuh"

namespace kbc {

__global__ void diag_final(const double* __restrict__ part, int nblocks, double* __restrict__ out,
                           long long total, int raw)
{
    // one block; thread t folds blocks t, t + blockDim, ... in a fixed order,
    // then a fixed tree combines the threads
    __shared__ double sm[kDiagParts][kDiagBlock];
    double acc[kDiagParts] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 1e300, -1e300};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
        diag_fold(acc, 1, part + (long long)b * kDiagParts, 1);
#pragma unroll
    for (int k = 0; k < kDiagParts; ++k) sm[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int s = kDiagBlock / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) diag_fold(&sm[0][threadIdx.x], kDiagBlock, &sm[0][threadIdx.x + s], kDiagBlock);
        __syncthreads();
    }
    if (threadIdx.x == 0 && raw) {
#pragma unroll
        for (int k = 0; k < kDiagParts; ++k) out[k] = sm[k][0];
    } else if (threadIdx.x == 0) {
        out[0] = sm[0][0];
        out[1] = sm[1][0];
        out[2] = sm[2][0];
        out[3] = sm[4][0];
        out[4] = sm[6][0];
        out[5] = sm[8][0] / (double)total;
        out[6] = sm[9][0];
        out[7] = sm[10][0];
        out[8] = sqrt(fmax(sm[5][0], 0.0) / (double)total);
        out[9] = sqrt(fmax(sm[7][0], 0.0) / (double)total);
    }
}

__global__ void diag_ext_final(const double* __restrict__ part, int nblocks, double* __restrict__ out,
                               long long total)
{
    __shared__ double sm[kDiagExtParts][kDiagBlock];
    double acc[kDiagExtParts] = {0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
        diag_ext_fold(acc, 1, part + (long long)b * kDiagExtParts, 1);
#pragma unroll
    for (int k = 0; k < kDiagExtParts; ++k) sm[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int s = kDiagBlock / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            diag_ext_fold(&sm[0][threadIdx.x], kDiagBlock, &sm[0][threadIdx.x + s], kDiagBlock);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = sm[1][0];
        out[1] = sqrt(fmax(sm[2][0], 0.0) / (double)total);
        out[2] = sm[3][0];
        out[3] = sqrt(fmax(sm[4][0], 0.0) / (double)total);
    }
}

__global__ void sum_partials(const double* __restrict__ part, int n, double* __restrict__ out)
{
    __shared__ double sm[256];
    double acc = 0.0;
    for (int b = threadIdx.x; b < n; b += blockDim.x) acc += part[b];
    sm[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sm[0];
}

}  // namespace kbc

using namespace kbc;

namespace {

struct Allocator {
    kbc_alloc_fn alloc = nullptr;
    kbc_free_fn release = nullptr;
    void* user = nullptr;
};

std::mutex g_alloc_mu;
Allocator g_alloc;
std::string g_create_error;

}  // namespace

// The message kbc_last_error(NULL) returns, for the calls that have no
// handle (declared in kbc_launch.cuh).
int kbc::handle_free_error(int code, const char* msg)
{
    g_create_error = msg;
    return code;
}

// Row chunks of the host <-> device pipelines of kbc_init and kbc_moments;
// staging below kPipeMinBytes uses one copy and one kernel.
constexpr int kPipeChunks = 32;
constexpr size_t kPipeMinBytes = (size_t)64 << 20;

struct kbc_ctx {
    int nx = 0, ny = 0, variant = 0, dtype = 0, device = 0, num_sms = 1;
    double beta = 1.0;
    int gamma_mode = KBC_GAMMA_ENTROPIC;
    double gamma_fixed = 2.0;
    double guard = 0.0;
    float f16_scale = 1.0f;
    long long plane = 0;  // elements per population plane
    size_t elem = 8;      // bytes per stored element
    // y-slab handle: each plane holds a ghost row below and above the ny
    // interior rows; buf[k] points at interior row 0 of allocation alloc[k]
    bool slab = false;
    int ghosts_full = 0;  // bit f: face f's ghost row holds a full halo of the current state
    void* alloc[2] = {nullptr, nullptr};
    void* buf[2] = {nullptr, nullptr};
    int cur = 0;          // buffer holding the current state
    int* fix = nullptr;   // [0..1] counters, [64..] list of node indices
    int fix_slot = 0;
    int* flag_dev = nullptr;
    int* flag_host = nullptr;  // pinned
    double* diag_part = nullptr;
    int diag_nblocks = 0;
    double* diag_out = nullptr;  // device, KBC_DIAG_N doubles
    void* stage = nullptr;       // device staging for host pointers
    size_t stage_bytes = 0;
    bool initialized = false;
    int kernel = KBC_KERNEL_AUTO;
    // CUDA graphs of graph_steps (even) steps, one per (cur, fix_slot) parity,
    // valid while config_version == graph_version[k]
    int graph_steps = 32;
    unsigned config_version = 1;
    unsigned graph_version[4] = {0, 0, 0, 0};
    cudaGraphExec_t graph[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaStream_t capture_stream = nullptr;
    // host <-> device pipelines: copies of one row chunk overlap the kernel
    // of the neighbouring chunk on this second stream, ordered by events
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t pipe_ev[kPipeChunks + 2] = {};
    cudaStream_t stream = nullptr;
    Allocator al;
    std::string err;
};

namespace {

int fail(kbc_ctx* h, int code, const std::string& msg)
{
    if (h) h->err = msg;
    else g_create_error = msg;
    return code;
}

int cuda_fail(kbc_ctx* h, cudaError_t e, const char* where)
{
    return fail(h, KBC_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

void* dev_alloc(kbc_ctx* h, size_t bytes)
{
    if (bytes == 0) bytes = 256;
    if (h->al.alloc) return h->al.alloc(bytes, (void*)h->stream, h->al.user);
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void dev_free(kbc_ctx* h, void* p)
{
    if (!p) return;
    if (h->al.release) h->al.release(p, (void*)h->stream, h->al.user);
    else cudaFree(p);
}

bool is_device_ptr(const void* p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

size_t elem_size(int dtype) { return dtype == KBC_F64 ? 8 : dtype == KBC_F32_DEV ? 4 : 2; }
int vec_width(int dtype)
{
    return dtype == KBC_F64 ? CodecF64::kVec : dtype == KBC_F32_DEV ? CodecF32::kVec : CodecF16::kVec;
}

StepArgs args_of(const kbc_ctx* h)
{
    StepArgs a;
    a.nx = h->nx;
    a.ny = h->ny;
    a.plane = h->plane;
    a.cs = make_scale(h->f16_scale);
    const int fixed = (h->gamma_mode == KBC_GAMMA_FIXED) ? 1 : (h->gamma_mode == KBC_GAMMA_EXACT ? 2 : 0);
    const double guard = (h->dtype == KBC_F64) ? 0.0 : h->guard;
    a.pf = make_params<float>(h->beta, fixed, h->gamma_fixed, guard);
    a.pd = make_params<double>(h->beta, fixed, h->gamma_fixed, guard);
    if (h->dtype == KBC_F16_DEV) {  // the FP16 step kernels collide in storage units
        const double s = h->f16_scale, c = 1.0 / (36.0 * s);
        a.pf.unit_s = (float)s;
        a.pf.unit_c = (float)c;
        a.pf.guard_u = (float)(guard / (c * c));
    }
    a.beta = h->beta;
    a.fix_count = h->fix;
    a.fix_list = h->fix ? h->fix + 64 : nullptr;
    a.fix_slot = h->fix_slot;
    a.flag = h->flag_dev;
    a.ywrap = h->slab ? 0 : 1;
    return a;
}

int reject_slab(kbc_ctx* h, const char* what)
{
    return fail(h, KBC_ERR_ARG, std::string(what) + " is not available on a y-slab handle");
}

// Stage `bytes` from a host or device pointer into device memory.
int stage_in(kbc_ctx* h, const void* src, size_t bytes, const void** dev)
{
    if (is_device_ptr(src)) {
        *dev = src;
        return KBC_OK;
    }
    if (h->stage_bytes < bytes) {
        dev_free(h, h->stage);
        h->stage = dev_alloc(h, bytes);
        h->stage_bytes = h->stage ? bytes : 0;
        if (!h->stage) return fail(h, KBC_ERR_NOMEM, "staging allocation failed");
    }
    cudaError_t e = cudaMemcpyAsync(h->stage, src, bytes, cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "host-to-device copy");
    *dev = h->stage;
    return KBC_OK;
}

int wait_stream(kbc_ctx* h, double timeout_s)
{
    if (timeout_s <= 0) timeout_s = 600.0;
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaStreamQuery(h->stream);
        if (e == cudaSuccess) break;
        if (e != cudaErrorNotReady) return cuda_fail(h, e, "stream");
        const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (el > timeout_s) return fail(h, KBC_ERR_TIMEOUT, "timed out waiting for the stream");
        std::this_thread::sleep_for(std::chrono::microseconds(el < 0.01 ? 5 : 200));
    }
    return KBC_OK;
}

template <class F>
cudaError_t by_codec(int dtype, F&& fn)
{
    switch (dtype) {
    case KBC_F64: return fn(CodecF64{});
    case KBC_F32_DEV: return fn(CodecF32{});
    case KBC_F16_DEV: return fn(CodecF16{});
    default: return cudaErrorInvalidValue;
    }
}

int check_h(kbc_ctx* h)
{
    if (!h) return KBC_ERR_ARG;
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
    return KBC_OK;
}

}  // namespace

// One step from src to dst with the handle's settings (guard pass and its
// alternating counters included).
static int step_into(kbc_handle h, const void* src, void* dst, cudaStream_t stream = nullptr,
                     bool use_stream = false)
{
    Launch L;
    L.variant = h->variant;
    L.rows = h->kernel != KBC_KERNEL_NODES && (h->nx % (32 * vec_width(h->dtype))) == 0;
    // AUTO takes the bulk-copy kernel for FP16 KBC (measured 1-3% faster than
    // the vector rows there; the rows win for LBGK and for FP32 by 12-16%)
    const bool bulk = h->kernel == KBC_KERNEL_BULK ||
                      (h->kernel == KBC_KERNEL_AUTO && h->dtype == KBC_F16_DEV &&
                       h->variant != KBC_LBGK);
    L.tma = bulk && h->dtype != KBC_F64 && (h->nx % kTmaTile) == 0;
    L.all_f64 = h->gamma_mode == KBC_GAMMA_EXACT && h->variant != KBC_LBGK;
    L.stream = use_stream ? stream : h->stream;
    L.num_sms = h->num_sms;
    const bool guard_on = h->dtype != KBC_F64 && h->variant != KBC_LBGK &&
                          h->gamma_mode == KBC_GAMMA_ENTROPIC && h->guard > 0.0 && h->fix;
    L.fixup = guard_on;
    L.src = src;
    L.dst = dst;
    L.a = args_of(h);
    if (!guard_on) L.a.fix_list = nullptr;
    cudaError_t e = by_codec(h->dtype, [&](auto c) {
        using C = decltype(c);
        return launch_step<C>(L);
    });
    if (e != cudaSuccess) return cuda_fail(h, e, "step launch");
    if (guard_on) h->fix_slot ^= 1;
    return KBC_OK;
}

static void drop_graphs(kbc_handle h)
{
    for (int k = 0; k < 4; ++k) {
        if (h->graph[k]) cudaGraphExecDestroy(h->graph[k]);
        h->graph[k] = nullptr;
        h->graph_version[k] = 0;
    }
}

// The instantiated graph of graph_steps steps starting from the current
// (cur, fix_slot) parity, captured on a private stream; nullptr if capture
// is not possible (the step then runs launch by launch).
static cudaGraphExec_t step_graph(kbc_handle h)
{
    const int key = h->cur | (h->fix_slot << 1);
    if (h->graph[key] && h->graph_version[key] == h->config_version) return h->graph[key];
    if (h->graph[key]) {
        cudaGraphExecDestroy(h->graph[key]);
        h->graph[key] = nullptr;
    }
    if (!h->capture_stream &&
        cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        h->capture_stream = nullptr;
        return nullptr;
    }
    const int slot0 = h->fix_slot;
    if (cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    int c = h->cur;
    bool ok = true;
    for (int s = 0; s < h->graph_steps && ok; ++s) {
        ok = step_into(h, h->buf[c], h->buf[c ^ 1], h->capture_stream, true) == KBC_OK;
        c ^= 1;
    }
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(h->capture_stream, &g);
    h->fix_slot = slot0;  // graph_steps is even: the replay returns to this parity
    cudaGraphExec_t exec = nullptr;
    if (ok && e == cudaSuccess && g && cudaGraphInstantiate(&exec, g, 0) == cudaSuccess) {
        h->graph[key] = exec;
        h->graph_version[key] = h->config_version;
    } else {
        exec = nullptr;
    }
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return exec;
}

// Instantiated graph of the work `issue(stream)` enqueues on the private
// capture stream (returns false on a failed launch); nullptr when capture or
// instantiation fails, with the handle's guard parity restored, so that the
// caller can fall back to launching the same work directly.
template <class F>
static cudaGraphExec_t capture_work(kbc_handle h, F&& issue)
{
    if (!h->capture_stream &&
        cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        h->capture_stream = nullptr;
        return nullptr;
    }
    const int slot0 = h->fix_slot;
    if (cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    const bool ok = issue(h->capture_stream);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(h->capture_stream, &g);
    cudaGraphExec_t exec = nullptr;
    if (!(ok && e == cudaSuccess && g && cudaGraphInstantiate(&exec, g, 0) == cudaSuccess)) {
        exec = nullptr;
        h->fix_slot = slot0;
    }
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return exec;
}

// Graphs of one kbc_adjoint call (its buffers are the call's own).
struct AdjointGraphs {
    cudaGraphExec_t fwd = nullptr;              // ckpt_every forward steps from work[0]
    cudaGraphExec_t rec[2] = {nullptr, nullptr}; // segment recompute, by starting guard parity
    int rec_flip[2] = {0, 0};                    // guard parity change of one recompute
    cudaGraphExec_t rev[2] = {nullptr, nullptr}; // reverse segment, by lambda parity
    ~AdjointGraphs()
    {
        for (cudaGraphExec_t g : {fwd, rec[0], rec[1], rev[0], rev[1]})
            if (g) cudaGraphExecDestroy(g);
    }
};

// device buffers owned by one call, released on every exit path
struct CallBuffers {
    kbc_ctx* h;
    void* p[64];
    int n = 0;
    explicit CallBuffers(kbc_ctx* hh) : h(hh) {}
    void* get(size_t bytes)
    {
        if (n >= 64) return nullptr;
        void* q = dev_alloc(h, bytes);
        if (q) p[n++] = q;
        return q;
    }
    ~CallBuffers()
    {
        cudaStreamSynchronize(h->stream);
        for (int i = n - 1; i >= 0; --i) dev_free(h, p[i]);
    }
};

// Device staging buffer of at least `bytes` (kept between calls).
static int ensure_stage(kbc_ctx* h, size_t bytes)
{
    if (h->stage_bytes >= bytes) return KBC_OK;
    dev_free(h, h->stage);
    h->stage = dev_alloc(h, bytes);
    h->stage_bytes = h->stage ? bytes : 0;
    return h->stage ? KBC_OK : fail(h, KBC_ERR_NOMEM, "staging allocation failed");
}

// The copy stream and events of the pipelines (created on first use).
static int pipe_ready(kbc_ctx* h)
{
    if (!h->copy_stream) {
        cudaError_t e = cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            h->copy_stream = nullptr;
            return cuda_fail(h, e, "copy stream");
        }
    }
    for (cudaEvent_t& ev : h->pipe_ev) {
        if (ev) continue;
        cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            ev = nullptr;
            return cuda_fail(h, e, "pipeline event");
        }
    }
    return KBC_OK;
}

// Rows [y0, y0 + rows) of chunk k of the pipelines.
static void pipe_chunk(const kbc_ctx* h, int k, int* y0, int* rows)
{
    const int per = (h->ny + kPipeChunks - 1) / kPipeChunks;
    *y0 = k * per;
    *rows = (*y0 >= h->ny) ? 0 : ((h->ny - *y0 < per) ? h->ny - *y0 : per);
}

// f = f^eq(rho, u) from host (or mixed) pointers: chunk k's uploads on the
// copy stream overlap the init kernel of chunk k - 1 on the handle's stream
// (init_feq works node by node, so a chunk is the same launch on fewer rows).
static int init_feq_pipelined(kbc_ctx* h, const double* rho, const double* u)
{
    const size_t n = (size_t)h->nx * h->ny;
    int rc = pipe_ready(h);
    if (rc) return rc;
    double* st = static_cast<double*>(h->stage);
    // the staging buffer is free once earlier work on the handle's stream is done
    cudaError_t e = cudaEventRecord(h->pipe_ev[kPipeChunks], h->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->copy_stream, h->pipe_ev[kPipeChunks], 0);
    for (int k = 0; k < kPipeChunks && e == cudaSuccess; ++k) {
        int y0, rows;
        pipe_chunk(h, k, &y0, &rows);
        if (rows == 0) break;
        const size_t off = (size_t)y0 * h->nx, cnt = (size_t)rows * h->nx * sizeof(double);
        e = cudaMemcpyAsync(st + off, rho + off, cnt, cudaMemcpyDefault, h->copy_stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(st + n + off, u + off, cnt, cudaMemcpyDefault, h->copy_stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(st + 2 * n + off, u + n + off, cnt, cudaMemcpyDefault, h->copy_stream);
        if (e == cudaSuccess) e = cudaEventRecord(h->pipe_ev[k], h->copy_stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, h->pipe_ev[k], 0);
        if (e != cudaSuccess) break;
        StepArgs a = args_of(h);
        a.ny = rows;
        void* dst = static_cast<char*>(h->buf[h->cur]) + off * h->elem;
        e = by_codec(h->dtype, [&](auto c) {
            using C = decltype(c);
            return launch_init<C>(st + off, st + n + off, st + 2 * n + off, dst, a, false,
                                  h->stream, h->num_sms);
        });
    }
    return e == cudaSuccess ? KBC_OK : cuda_fail(h, e, "pipelined field upload");
}

static int init_common(kbc_handle h, const double* rho, const double* u, bool grad)
{
    int rc = check_h(h);
    if (rc) return rc;
    if (!rho || !u) return fail(h, KBC_ERR_ARG, "NULL field");
    const size_t n = (size_t)h->nx * h->ny;
    const double *drho, *du;

    // stage both fields through one buffer when they are on the host
    const bool hr = !is_device_ptr(rho), hu = !is_device_ptr(u);
    if (hr || hu) {
        const size_t need = 3 * n * sizeof(double);
        rc = ensure_stage(h, need);
        if (rc) return rc;
        if (!grad && need >= kPipeMinBytes) {
            rc = init_feq_pipelined(h, rho, u);
            if (rc) return rc;
            h->initialized = true;
            h->ghosts_full = 0;
            return KBC_OK;
        }
        double* st = static_cast<double*>(h->stage);
        cudaError_t e = cudaMemcpyAsync(st, rho, n * sizeof(double), cudaMemcpyDefault, h->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(st + n, u, 2 * n * sizeof(double), cudaMemcpyDefault, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "field upload");
        drho = st;
        du = st + n;
    } else {
        drho = rho;
        du = u;
    }

    StepArgs a = args_of(h);
    cudaError_t e = by_codec(h->dtype, [&](auto c) {
        using C = decltype(c);
        return launch_init<C>(drho, du, du + n, h->buf[h->cur], a, grad, h->stream, h->num_sms);
    });
    if (e != cudaSuccess) return cuda_fail(h, e, "init launch");
    h->initialized = true;
    h->ghosts_full = 0;
    return KBC_OK;
}

// Run `kernel(dst_device)` writing `bytes` of output, into `out` (host or device).
template <class K>
static int produce(kbc_handle h, void* out, size_t bytes, K&& kernel)
{
    const bool dev = is_device_ptr(out);
    void* target = out;
    if (!dev) {
        if (h->stage_bytes < bytes) {
            dev_free(h, h->stage);
            h->stage = dev_alloc(h, bytes);
            h->stage_bytes = h->stage ? bytes : 0;
            if (!h->stage) return fail(h, KBC_ERR_NOMEM, "staging allocation failed");
        }
        target = h->stage;
    }
    cudaError_t e = kernel(target);
    if (e != cudaSuccess) return cuda_fail(h, e, "launch");
    if (!dev) {
        e = cudaMemcpyAsync(out, target, bytes, cudaMemcpyDeviceToHost, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "device-to-host copy");
        return wait_stream(h, 0);
    }
    return KBC_OK;
}

extern "C" {

int kbc_set_allocator(kbc_alloc_fn alloc, kbc_free_fn release, void* user)
{
    if ((alloc == nullptr) != (release == nullptr)) return KBC_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_alloc.alloc = alloc;
    g_alloc.release = release;
    g_alloc.user = user;
    return KBC_OK;
}

static int create_common(int nx, int ny, int variant, double beta, int dtype, bool slab,
                         kbc_handle* out)
{
    if (!out) return fail(nullptr, KBC_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (nx < 1 || ny < 1 || (long long)nx * (ny + (slab ? 2 : 0)) > 2147483647LL)
        return fail(nullptr, KBC_ERR_ARG, "grid size out of range");
    if (!(beta > 0.0 && beta <= 1.0)) return fail(nullptr, KBC_ERR_ARG, "beta must lie in (0, 1]");
    if (variant < KBC_LBGK || variant > KBC_D) return fail(nullptr, KBC_ERR_ARG, "bad variant");
    if (dtype < KBC_F64 || dtype > KBC_F16_DEV) return fail(nullptr, KBC_ERR_ARG, "bad dtype");
    kbc_ctx* h = new (std::nothrow) kbc_ctx;
    if (!h) return fail(nullptr, KBC_ERR_NOMEM, "host allocation failed");
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        h->al = g_alloc;
    }
    h->nx = nx;
    h->ny = ny;
    h->slab = slab;
    h->variant = variant;
    h->beta = beta;
    h->dtype = dtype;
    h->elem = elem_size(dtype);
    h->guard = (dtype == KBC_F32_DEV) ? 1e-16 : 0.0;
    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e != cudaSuccess) {
        cudaGetLastError();
        std::string m = std::string("no CUDA device: ") + cudaGetErrorString(e);
        delete h;
        return fail(nullptr, KBC_ERR_CUDA, m);
    }
    const long long per = 256 / (long long)h->elem;
    const long long rows = (long long)ny + (slab ? 2 : 0);
    h->plane = (((long long)nx * rows + per - 1) / per) * per;
    const size_t field = (size_t)9 * h->plane * h->elem;
    for (int k = 0; k < 2; ++k) {
        h->alloc[k] = dev_alloc(h, field);
        h->buf[k] = h->alloc[k] && slab ? static_cast<char*>(h->alloc[k]) + (size_t)nx * h->elem
                                        : h->alloc[k];
    }
    h->flag_dev = static_cast<int*>(dev_alloc(h, 256));
    const long long total = (long long)nx * ny;
    h->diag_nblocks = diag_blocks(total, h->num_sms);
    h->diag_part = static_cast<double*>(dev_alloc(h, (size_t)h->diag_nblocks * kDiagParts * sizeof(double)));
    h->diag_out = static_cast<double*>(dev_alloc(h, 256));
    if (dtype != KBC_F64 && variant != KBC_LBGK)
        h->fix = static_cast<int*>(dev_alloc(h, (size_t)(64 + total) * sizeof(int)));
    if (!h->buf[0] || !h->buf[1] || !h->flag_dev || !h->diag_part || !h->diag_out ||
        (dtype != KBC_F64 && variant != KBC_LBGK && !h->fix)) {
        kbc_destroy(h);
        return fail(nullptr, KBC_ERR_NOMEM, "device allocation failed");
    }
    e = cudaHostAlloc((void**)&h->flag_host, 4 * sizeof(int), cudaHostAllocDefault);
    if (e != cudaSuccess) {
        cudaGetLastError();
        h->flag_host = nullptr;
        kbc_destroy(h);
        return fail(nullptr, KBC_ERR_CUDA, "pinned allocation failed");
    }
    h->flag_host[0] = h->flag_host[1] = h->flag_host[2] = h->flag_host[3] = 0;
    e = cudaMemsetAsync(h->flag_dev, 0, 256, h->stream);
    if (e == cudaSuccess && h->fix) e = cudaMemsetAsync(h->fix, 0, 64 * sizeof(int), h->stream);
    // ghost rows start at f = W (zero deviation) until the first halo arrives
    for (int k = 0; k < 2 && slab && e == cudaSuccess; ++k) e = cudaMemsetAsync(h->alloc[k], 0, field, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        std::string m = std::string("initial memset: ") + cudaGetErrorString(e);
        kbc_destroy(h);
        return fail(nullptr, KBC_ERR_CUDA, m);
    }
    *out = h;
    return KBC_OK;
}

int kbc_create(int nx, int ny, int variant, double beta, int dtype, kbc_handle* out)
{
    return create_common(nx, ny, variant, beta, dtype, false, out);
}

int kbc_create_slab(int nx, int ny, int variant, double beta, int dtype, kbc_handle* out)
{
    return create_common(nx, ny, variant, beta, dtype, true, out);
}

int kbc_destroy(kbc_handle h)
{
    if (!h) return KBC_ERR_ARG;
    cudaSetDevice(h->device);
    cudaStreamSynchronize(h->stream);
    dev_free(h, h->alloc[0]);
    dev_free(h, h->alloc[1]);
    dev_free(h, h->fix);
    dev_free(h, h->flag_dev);
    dev_free(h, h->diag_part);
    dev_free(h, h->diag_out);
    dev_free(h, h->stage);
    if (h->flag_host) cudaFreeHost(h->flag_host);
    drop_graphs(h);
    if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
    if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
    for (cudaEvent_t ev : h->pipe_ev)
        if (ev) cudaEventDestroy(ev);
    cudaGetLastError();
    delete h;
    return KBC_OK;
}

int kbc_set_stream(kbc_handle h, void* stream)
{
    if (!h) return KBC_ERR_ARG;
    h->stream = static_cast<cudaStream_t>(stream);
    return KBC_OK;
}

int kbc_set_gamma_mode(kbc_handle h, int mode, double gamma_fixed)
{
    if (!h) return KBC_ERR_ARG;
    if (mode != KBC_GAMMA_ENTROPIC && mode != KBC_GAMMA_FIXED && mode != KBC_GAMMA_EXACT)
        return fail(h, KBC_ERR_ARG, "bad gamma mode");
    if (mode == KBC_GAMMA_FIXED && !std::isfinite(gamma_fixed))
        return fail(h, KBC_ERR_ARG, "gamma must be finite");
    h->gamma_mode = mode;
    h->gamma_fixed = gamma_fixed;
    ++h->config_version;
    return KBC_OK;
}

int kbc_set_kernel(kbc_handle h, int kernel)
{
    if (!h) return KBC_ERR_ARG;
    if (kernel < KBC_KERNEL_AUTO || kernel > KBC_KERNEL_BULK) return fail(h, KBC_ERR_ARG, "bad kernel");
    h->kernel = kernel;
    ++h->config_version;
    return KBC_OK;
}

int kbc_set_graph_steps(kbc_handle h, int steps)
{
    if (!h) return KBC_ERR_ARG;
    if (steps < 0 || steps % 2 != 0) return fail(h, KBC_ERR_ARG, "graph steps must be even and >= 0");
    h->graph_steps = steps;
    drop_graphs(h);
    return KBC_OK;
}

int kbc_set_guard(kbc_handle h, double threshold)
{
    if (!h) return KBC_ERR_ARG;
    if (!(threshold >= 0.0)) return fail(h, KBC_ERR_ARG, "guard must be >= 0");
    if (threshold > 0.0 && h->dtype != KBC_F64 && h->variant != KBC_LBGK && !h->fix) {
        h->fix = static_cast<int*>(dev_alloc(h, (size_t)(64 + (long long)h->nx * h->ny) * sizeof(int)));
        if (!h->fix) return fail(h, KBC_ERR_NOMEM, "guard list allocation failed");
        cudaError_t e = cudaMemsetAsync(h->fix, 0, 64 * sizeof(int), h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "memset");
    }
    h->guard = threshold;
    ++h->config_version;
    return KBC_OK;
}

int kbc_guard_count(kbc_handle h, long long* count)
{
    int rc = check_h(h);
    if (rc) return rc;
    if (!count) return fail(h, KBC_ERR_ARG, "NULL output");
    *count = 0;
    if (!h->fix) return KBC_OK;
    // the last step used slot fix_slot ^ 1 (the slot flips after every step)
    cudaError_t e = cudaMemcpyAsync(h->flag_host + 2, h->fix + (h->fix_slot ^ 1), sizeof(int),
                                    cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "guard count copy");
    rc = wait_stream(h, 0);
    if (rc) return rc;
    *count = h->flag_host[2];
    return KBC_OK;
}

int kbc_set_f16_scale(kbc_handle h, double scale)
{
    if (!h) return KBC_ERR_ARG;
    if (!(scale >= 0x1p-24 && scale <= 0x1p24))
        return fail(h, KBC_ERR_ARG, "scale must lie in [2^-24, 2^24]");
    if (h->initialized) return fail(h, KBC_ERR_STATE, "set the scale before kbc_init");
    h->f16_scale = (float)scale;
    ++h->config_version;
    return KBC_OK;
}

int kbc_init(kbc_handle h, const double* rho, const double* u)
{
    return init_common(h, rho, u, false);
}

int kbc_init_grad(kbc_handle h, const double* rho, const double* u)
{
    if (h && h->slab) return reject_slab(h, "kbc_init_grad (y gradients across the slab faces)");
    return init_common(h, rho, u, true);
}

int kbc_set_populations(kbc_handle h, const double* f)
{
    int rc = check_h(h);
    if (rc) return rc;
    if (!f) return fail(h, KBC_ERR_ARG, "NULL field");
    const void* df;
    rc = stage_in(h, f, (size_t)9 * h->nx * h->ny * sizeof(double), &df);
    if (rc) return rc;
    StepArgs a = args_of(h);
    cudaError_t e = by_codec(h->dtype, [&](auto c) {
        using C = decltype(c);
        return launch_set<C>(static_cast<const double*>(df), h->buf[h->cur], a, h->stream, h->num_sms);
    });
    if (e != cudaSuccess) return cuda_fail(h, e, "set launch");
    h->initialized = true;
    h->ghosts_full = 0;
    return KBC_OK;
}

int kbc_get_populations(kbc_handle h, double* f)
{
    int rc = check_h(h);
    if (rc) return rc;
    if (!f) return fail(h, KBC_ERR_ARG, "NULL field");
    if (!h->initialized) return fail(h, KBC_ERR_STATE, "field not initialised");
    const size_t n = (size_t)h->nx * h->ny;
    StepArgs a = args_of(h);
    return produce(h, f, 9 * n * sizeof(double), [&](void* t) {
        return by_codec(h->dtype, [&](auto c) {
            using C = decltype(c);
            return launch_get<C>(h->buf[h->cur], static_cast<double*>(t), a, h->stream, h->num_sms);
        });
    });
}

int kbc_step(kbc_handle h, int nsteps)
{
    int rc = check_h(h);
    if (rc) return rc;
    if (nsteps < 0) return fail(h, KBC_ERR_ARG, "nsteps must be >= 0");
    if (h->slab && nsteps > 1)
        return fail(h, KBC_ERR_ARG, "a y-slab handle steps once between halo exchanges (nsteps <= 1)");
    if (!h->initialized) return fail(h, KBC_ERR_STATE, "field not initialised");
    if (h->flag_host[0] & 2) return fail(h, KBC_ERR_TIMEOUT, "a device-side wait ran out");
    if (h->flag_host[0]) return fail(h, KBC_ERR_NONFINITE, "non-finite populations detected");
    if (nsteps == 0) return KBC_OK;
    h->ghosts_full = 0;
    int done = 0;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const bool capturing = cudaStreamIsCapturing(h->stream, &cs) != cudaSuccess ||
                           cs != cudaStreamCaptureStatusNone;
    cudaGetLastError();
    if (h->graph_steps > 0 && nsteps >= h->graph_steps && !capturing) {
        cudaGraphExec_t g = step_graph(h);
        if (g) {
            for (; done + h->graph_steps <= nsteps; done += h->graph_steps) {
                cudaError_t e = cudaGraphLaunch(g, h->stream);
                if (e != cudaSuccess) return cuda_fail(h, e, "graph launch");
            }
        }
    }
    for (int s = done; s < nsteps; ++s) {
        rc = step_into(h, h->buf[h->cur], h->buf[h->cur ^ 1]);
        if (rc) return rc;
        h->cur ^= 1;
    }
    cudaError_t e = cudaMemcpyAsync(h->flag_host, h->flag_dev, sizeof(int), cudaMemcpyDeviceToHost,
                                    h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "flag copy");
    return KBC_OK;
}

int kbc_sync(kbc_handle h, double timeout_s)
{
    int rc = check_h(h);
    if (rc) return rc;
    rc = wait_stream(h, timeout_s);
    if (rc) return rc;
    if (h->flag_host[0] & 2) return fail(h, KBC_ERR_TIMEOUT, "a device-side wait ran out");
    if (h->flag_host[0]) return fail(h, KBC_ERR_NONFINITE, "non-finite populations detected");
    return KBC_OK;
}

int kbc_probe(kbc_handle h, int count, const long long* nodes, double* f)
{
    int rc = check_h(h);
    if (rc) return rc;
    if (count < 0 || (count > 0 && (!nodes || !f))) return fail(h, KBC_ERR_ARG, "bad probe arguments");
    if (!h->initialized) return fail(h, KBC_ERR_STATE, "field not initialised");
    if (count == 0) return KBC_OK;
    const bool dn = is_device_ptr(nodes), df = is_device_ptr(f);
    const size_t nb = (size_t)count * sizeof(long long), fb = (size_t)count * 9 * sizeof(double);
    const size_t need = 256 + (dn ? 0 : nb) + (df ? 0 : fb);
    if (h->stage_bytes < need) {
        dev_free(h, h->stage);
        h->stage = dev_alloc(h, need);
        h->stage_bytes = h->stage ? need : 0;
        if (!h->stage) return fail(h, KBC_ERR_NOMEM, "staging allocation failed");
    }
    char* st = static_cast<char*>(h->stage);
    int* bad = reinterpret_cast<int*>(st);
    const long long* dnodes = nodes;
    double* dfo = f;
    size_t off = 256;
    if (!dn) {
        dnodes = reinterpret_cast<const long long*>(st + off);
        off += nb;
    }
    if (!df) dfo = reinterpret_cast<double*>(st + off);
    cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(int), h->stream);
    if (e == cudaSuccess && !dn)
        e = cudaMemcpyAsync((void*)dnodes, nodes, nb, cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "probe upload");
    StepArgs a = args_of(h);
    e = by_codec(h->dtype, [&](auto c) {
        using C = decltype(c);
        return launch_probe<C>(h->buf[h->cur], dnodes, count, dfo, bad, a, h->stream, h->num_sms);
    });
    if (e != cudaSuccess) return cuda_fail(h, e, "probe launch");
    if (!df) {
        e = cudaMemcpyAsync(f, dfo, fb, cudaMemcpyDeviceToHost, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "probe download");
    }
    int bad_host = 0;
    e = cudaMemcpyAsync(h->flag_host + 1, bad, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "probe status");
    rc = wait_stream(h, 0);
    if (rc) return rc;
    bad_host = h->flag_host[1];
    if (bad_host) return fail(h, KBC_ERR_ARG, "probe node index out of range");
    return KBC_OK;
}

int kbc_moments(kbc_handle h, double* rho, double* u)
{
    int rc = check_h(h);
    if (rc) return rc;
    if (!rho || !u) return fail(h, KBC_ERR_ARG, "NULL field");
    if (!h->initialized) return fail(h, KBC_ERR_STATE, "field not initialised");
    const size_t n = (size_t)h->nx * h->ny;
    StepArgs a = args_of(h);
    const bool dr = is_device_ptr(rho), du = is_device_ptr(u);
    if (dr && du) {
        cudaError_t e = by_codec(h->dtype, [&](auto c) {
            using C = decltype(c);
            return launch_moments<C>(h->buf[h->cur], rho, u, u + n, a, h->stream, h->num_sms);
        });
        return e == cudaSuccess ? KBC_OK : cuda_fail(h, e, "moments launch");
    }
    // at least one host output: compute all three fields into staging
    const size_t bytes = 3 * n * sizeof(double);
    rc = ensure_stage(h, bytes);
    if (rc) return rc;
    double* st = static_cast<double*>(h->stage);
    if (bytes >= kPipeMinBytes) {
        // chunk k's downloads on the copy stream overlap the moments kernel of
        // chunk k + 1 (the kernel works node by node)
        rc = pipe_ready(h);
        if (rc) return rc;
        cudaError_t e = cudaSuccess;
        for (int k = 0; k < kPipeChunks && e == cudaSuccess; ++k) {
            int y0, rows;
            pipe_chunk(h, k, &y0, &rows);
            if (rows == 0) break;
            const size_t off = (size_t)y0 * h->nx, cnt = (size_t)rows * h->nx * sizeof(double);
            StepArgs ak = a;
            ak.ny = rows;
            const void* src = static_cast<const char*>(h->buf[h->cur]) + off * h->elem;
            e = by_codec(h->dtype, [&](auto c) {
                using C = decltype(c);
                return launch_moments<C>(src, st + off, st + n + off, st + 2 * n + off, ak,
                                         h->stream, h->num_sms);
            });
            if (e == cudaSuccess) e = cudaEventRecord(h->pipe_ev[k], h->stream);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(h->copy_stream, h->pipe_ev[k], 0);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(rho + off, st + off, cnt, cudaMemcpyDefault, h->copy_stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(u + off, st + n + off, cnt, cudaMemcpyDefault, h->copy_stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(u + n + off, st + 2 * n + off, cnt, cudaMemcpyDefault, h->copy_stream);
        }
        // the handle's stream resumes once the last download is done
        if (e == cudaSuccess) e = cudaEventRecord(h->pipe_ev[kPipeChunks + 1], h->copy_stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, h->pipe_ev[kPipeChunks + 1], 0);
        if (e != cudaSuccess) return cuda_fail(h, e, "pipelined moments");
        return wait_stream(h, 0);
    }
    cudaError_t e = by_codec(h->dtype, [&](auto c) {
        using C = decltype(c);
        return launch_moments<C>(h->buf[h->cur], st, st + n, st + 2 * n, a, h->stream, h->num_sms);
    });
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(rho, st, n * sizeof(double), cudaMemcpyDefault, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(u, st + n, 2 * n * sizeof(double), cudaMemcpyDefault, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "moments");
    return wait_stream(h, 0);
}

int kbc_diagnostics(kbc_handle h, double* out)
{
    int rc = check_h(h);
    if (rc) return rc;
    if (h->slab) return reject_slab(h, "kbc_diagnostics");
    if (!out) return fail(h, KBC_ERR_ARG, "NULL output");
    if (!h->initialized) return fail(h, KBC_ERR_STATE, "field not initialised");
    StepArgs a = args_of(h);
    cudaError_t e = by_codec(h->dtype, [&](auto c) {
        using C = decltype(c);
        return launch_diag<C>(h->buf[h->cur], h->diag_part, h->diag_nblocks, h->diag_out,
                              h->variant, a, h->stream, 0);
    });
    if (e != cudaSuccess) return cuda_fail(h, e, "diagnostics launch");
    e = cudaMemcpyAsync(out, h->diag_out, KBC_DIAG_N * sizeof(double), cudaMemcpyDefault, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "diagnostics copy");
    return wait_stream(h, 0);
}

int kbc_diagnostics_partial(kbc_handle h, double* out)
{
    int rc = check_h(h);
    if (rc) return rc;
    if (!out) return fail(h, KBC_ERR_ARG, "NULL output");
    if (!h->initialized) return fail(h, KBC_ERR_STATE, "field not initialised");
    if (h->slab && h->ghosts_full != 3)
        return fail(h, KBC_ERR_STATE,
                    "a y-slab needs full halos (kbc_halo_recv, full = 1) of the current state in "
                    "both ghost rows");
    StepArgs a = args_of(h);
    cudaError_t e = by_codec(h->dtype, [&](auto c) {
        using C = decltype(c);
        return launch_diag<C>(h->buf[h->cur], h->diag_part, h->diag_nblocks, h->diag_out,
                              h->variant, a, h->stream, 1);
    });
    if (e != cudaSuccess) return cuda_fail(h, e, "diagnostics launch");
    e = cudaMemcpyAsync(out, h->diag_out, KBC_DIAG_PART_N * sizeof(double), cudaMemcpyDefault,
                        h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "diagnostics copy");
    return wait_stream(h, 0);
}

int kbc_diagnostics_merge(int n, const double* parts, double* out)
{
    if (n < 1 || !parts || !out) return fail(nullptr, KBC_ERR_ARG, "merge: bad argument");
    // host arithmetic: device pointers are refused (where the runtime can
    // tell; without a device every pointer is host memory)
    for (const void* q : {static_cast<const void*>(parts), static_cast<const void*>(out)}) {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, q) == cudaSuccess && at.type == cudaMemoryTypeDevice)
            return fail(nullptr, KBC_ERR_ARG, "merge: parts and out must be host memory");
        cudaGetLastError();
    }
    // Chan, Golub and LeVeque's pairwise combination of the (count, mean,
    // M2) sets, the sums added, min and max taken, in the order given
    double acc[KBC_DIAG_PART_N];
    for (int k = 0; k < KBC_DIAG_PART_N; ++k) acc[k] = parts[k];
    for (int j = 1; j < n; ++j) {
        const double* b = parts + (size_t)j * KBC_DIAG_PART_N;
        const double na = acc[3], nb = b[3], nn = na + nb;
        acc[0] += b[0];
        acc[1] += b[1];
        acc[2] += b[2];
        for (int k = 4; k <= 6 && nb > 0.0; k += 2) {
            if (na == 0.0) {
                acc[k] = b[k];
                acc[k + 1] = b[k + 1];
            } else {
                const double dlt = b[k] - acc[k];
                acc[k] += dlt * (nb / nn);
                acc[k + 1] += b[k + 1] + dlt * dlt * (na * nb / nn);
            }
        }
        acc[3] = nn;
        acc[8] += b[8];
        acc[9] = std::fmin(acc[9], b[9]);
        acc[10] = std::fmax(acc[10], b[10]);
    }
    if (!(acc[3] > 0.0)) return fail(nullptr, KBC_ERR_ARG, "merge: no nodes");
    out[0] = acc[0];
    out[1] = acc[1];
    out[2] = acc[2];
    out[3] = acc[4];
    out[4] = acc[6];
    out[5] = acc[8] / acc[3];
    out[6] = acc[9];
    out[7] = acc[10];
    out[8] = std::sqrt(std::fmax(acc[5], 0.0) / acc[3]);
    out[9] = std::sqrt(std::fmax(acc[7], 0.0) / acc[3]);
    return KBC_OK;
}

int kbc_adjoint(kbc_handle h, const double* rho0, const double* u0, int nsteps, int ckpt_every,
                int objective, const double* u_target, double* J, double* grad_u0,
                double* grad_beta)
{
    int rc = check_h(h);
    if (rc) return rc;
    if (h->slab) return reject_slab(h, "kbc_adjoint");
    if (!rho0 || !u0 || !J || !grad_u0 || !grad_beta) return fail(h, KBC_ERR_ARG, "NULL argument");
    if (nsteps < 0 || ckpt_every < 1) return fail(h, KBC_ERR_ARG, "nsteps >= 0, ckpt_every >= 1");
    if (objective != 0 && objective != 1) return fail(h, KBC_ERR_ARG, "objective must be 0 or 1");
    if (objective == 1 && !u_target) return fail(h, KBC_ERR_ARG, "objective 1 needs u_target");
    if (h->gamma_mode == KBC_GAMMA_EXACT && h->variant != KBC_LBGK)
        return fail(h, KBC_ERR_ARG, "the adjoint supports the entropic and fixed gamma modes");
    const long long n = (long long)h->nx * h->ny;
    const size_t field = (size_t)9 * h->plane * h->elem;
    const size_t tsize = (h->dtype == KBC_F64) ? sizeof(double) : sizeof(float);
    const size_t lamf = (size_t)9 * h->plane * tsize;
    const int K = ckpt_every;
    const int nseg = (nsteps + K - 1) / K;
    const int seglen = nsteps < K ? nsteps : K;
    const int nb = adj_blocks(n, h->num_sms);
    CallBuffers B(h);
    // inputs on the device: rho0, u0 (and the target)
    double* in = static_cast<double*>(B.get((size_t)(objective == 1 ? 5 : 3) * n * sizeof(double)));
    double* gdev = static_cast<double*>(B.get((size_t)2 * n * sizeof(double)));
    double* part = static_cast<double*>(B.get((size_t)(2 * nb + 8) * sizeof(double)));
    void* work[2] = {B.get(field), B.get(field)};
    void* lam[2] = {B.get(lamf), B.get(lamf)};
    // one bit per node: single-precision reverse steps left to the double redo
    const size_t maskbytes = (size_t)((n + 31) / 32) * sizeof(unsigned);
    unsigned* fixmask = static_cast<unsigned*>(B.get(maskbytes));
    if (!in || !gdev || !part || !work[0] || !work[1] || !lam[0] || !lam[1] || !fixmask)
        return fail(h, KBC_ERR_NOMEM, "adjoint buffers");
    // checkpoints and segment states in two slabs
    char* ckslab = nseg ? static_cast<char*>(B.get(field * (size_t)nseg)) : nullptr;
    char* segslab = seglen > 1 ? static_cast<char*>(B.get(field * (size_t)(seglen - 1))) : nullptr;
    if ((nseg && !ckslab) || (seglen > 1 && !segslab))
        return fail(h, KBC_ERR_NOMEM, "adjoint checkpoint storage");
    // Full segments (ckpt_every steps, even) replay captured graphs: the
    // sweep is otherwise launch-bound on small grids.  The recompute starts
    // from a fixed copy of the segment's checkpoint so that its graph's
    // pointers do not change from segment to segment.
    AdjointGraphs G;
    void* ckwork = (K % 2 == 0 && h->graph_steps > 0 && nsteps >= K) ? B.get(field) : nullptr;
    const bool graphs = ckwork != nullptr;
    cudaError_t e = cudaMemcpyAsync(in, rho0, n * sizeof(double), cudaMemcpyDefault, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(in + n, u0, 2 * n * sizeof(double), cudaMemcpyDefault, h->stream);
    if (e == cudaSuccess && objective == 1)
        e = cudaMemcpyAsync(in + 3 * n, u_target, 2 * n * sizeof(double), cudaMemcpyDefault, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(part, 0, (size_t)(2 * nb + 8) * sizeof(double), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(fixmask, 0, maskbytes, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->flag_dev, 0, sizeof(int), h->stream);  // fresh field
    if (e != cudaSuccess) return cuda_fail(h, e, "adjoint inputs");
    StepArgs a = args_of(h);
    e = by_codec(h->dtype, [&](auto c) {
        using C = decltype(c);
        return launch_init<C>(in, in + n, in + 2 * n, work[0], a, false, h->stream, h->num_sms);
    });
    if (e != cudaSuccess) return cuda_fail(h, e, "adjoint init");
    // forward sweep, keeping g^{sK}
    int cur = 0;
    for (int t = 0; t < nsteps;) {
        if (t % K == 0) {
            e = cudaMemcpyAsync(ckslab + field * (size_t)(t / K), work[cur], field,
                                cudaMemcpyDeviceToDevice, h->stream);
            if (e != cudaSuccess) return cuda_fail(h, e, "checkpoint copy");
            if (graphs && cur == 0 && t + K <= nsteps) {
                // K (even) steps return to work[0] and to the same guard parity
                if (!G.fwd) {
                    G.fwd = capture_work(h, [&](cudaStream_t cs) {
                        int c = 0;
                        for (int j = 0; j < K; ++j, c ^= 1)
                            if (step_into(h, work[c], work[c ^ 1], cs, true) != KBC_OK) return false;
                        return true;
                    });
                }
                if (G.fwd) {
                    e = cudaGraphLaunch(G.fwd, h->stream);
                    if (e != cudaSuccess) return cuda_fail(h, e, "adjoint forward graph");
                    t += K;
                    continue;
                }
            }
        }
        rc = step_into(h, work[cur], work[cur ^ 1]);
        if (rc) return rc;
        cur ^= 1;
        ++t;
    }
    const void* gN = work[cur];
    // J and lambda^N
    a = args_of(h);
    e = by_codec(h->dtype, [&](auto c) {
        using C = decltype(c);
        return launch_adj_objective<C>(gN, objective == 1 ? in + 3 * n : nullptr,
                                       objective == 1 ? in + 4 * n : nullptr, objective, lam[0],
                                       part, nb, a, h->stream);
    });
    if (e != cudaSuccess) return cuda_fail(h, e, "objective");
    // the handle keeps g^N
    e = cudaMemcpyAsync(h->buf[h->cur], gN, field, cudaMemcpyDeviceToDevice, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "final state copy");
    h->initialized = true;
    h->ghosts_full = 0;
    // reverse sweep over segments, recomputing each from its checkpoint
    int lc = 0;
    for (int sgi = nseg - 1; sgi >= 0; --sgi) {
        const int n0 = sgi * K;
        const int n1 = (n0 + K < nsteps) ? n0 + K : nsteps;
        const int len = n1 - n0;
        std::vector<const void*> states((size_t)len);
        const bool full = graphs && len == K;
        states[0] = ckslab + field * (size_t)sgi;
        if (full) {
            e = cudaMemcpyAsync(ckwork, states[0], field, cudaMemcpyDeviceToDevice, h->stream);
            if (e != cudaSuccess) return cuda_fail(h, e, "checkpoint copy");
            states[0] = ckwork;
        }
        for (int j = 1; j < len; ++j) states[j] = segslab + field * (size_t)(j - 1);
        bool done = false;
        if (full) {
            const int slot = h->fix_slot & 1;
            if (G.rec[slot]) {
                e = cudaGraphLaunch(G.rec[slot], h->stream);
                if (e != cudaSuccess) return cuda_fail(h, e, "adjoint recompute graph");
                h->fix_slot ^= G.rec_flip[slot];
                done = true;
            } else {
                G.rec[slot] = capture_work(h, [&](cudaStream_t cs) {
                    for (int j = 1; j < len; ++j)
                        if (step_into(h, states[j - 1], const_cast<void*>(states[j]), cs, true) != KBC_OK)
                            return false;
                    return true;
                });
                if (G.rec[slot]) {
                    // capture advanced the parity as the replay will
                    G.rec_flip[slot] = (h->fix_slot ^ slot) & 1;
                    e = cudaGraphLaunch(G.rec[slot], h->stream);
                    if (e != cudaSuccess) return cuda_fail(h, e, "adjoint recompute graph");
                    done = true;
                }
            }
        }
        for (int j = 1; j < len && !done; ++j) {
            rc = step_into(h, states[j - 1], const_cast<void*>(states[j]));
            if (rc) return rc;
        }
        if (full) {
            if (!G.rev[lc]) {
                const int l0 = lc;
                G.rev[lc] = capture_work(h, [&](cudaStream_t cs) {
                    int l = l0;
                    StepArgs ar = args_of(h);
                    for (int t = n1 - 1; t >= n0; --t, l ^= 1) {
                        cudaError_t ec = by_codec(h->dtype, [&](auto c) {
                            using C = decltype(c);
                            return launch_adj_step<C>(h->variant, states[t - n0], lam[l], lam[l ^ 1],
                                                      part + nb, fixmask, nb, ar, cs);
                        });
                        if (ec != cudaSuccess) return false;
                    }
                    return true;
                });
            }
            if (G.rev[lc]) {
                e = cudaGraphLaunch(G.rev[lc], h->stream);
                if (e != cudaSuccess) return cuda_fail(h, e, "adjoint reverse graph");
                continue;  // K (even) reverse steps leave lc unchanged
            }
        }
        for (int t = n1 - 1; t >= n0; --t) {
            a = args_of(h);
            e = by_codec(h->dtype, [&](auto c) {
                using C = decltype(c);
                return launch_adj_step<C>(h->variant, states[t - n0], lam[lc], lam[lc ^ 1],
                                          part + nb, fixmask, nb, a, h->stream);
            });
            if (e != cudaSuccess) return cuda_fail(h, e, "adjoint step");
            lc ^= 1;
        }
    }
    // dJ/du0 and the two sums
    e = by_codec(h->dtype, [&](auto c) {
        using C = decltype(c);
        return launch_adj_grad_u0<C>(in, in + n, in + 2 * n, lam[lc], gdev, gdev + n, a, h->stream,
                                     h->num_sms);
    });
    if (e != cudaSuccess) return cuda_fail(h, e, "grad u0");
    double* sums = part + 2 * nb;
    sum_partials<<<1, 256, 0, h->stream>>>(part, nb, sums);
    sum_partials<<<1, 256, 0, h->stream>>>(part + nb, nb, sums + 1);
    e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(grad_u0, gdev, 2 * n * sizeof(double), cudaMemcpyDefault, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->flag_host + 0, h->flag_dev, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    double host_sums[2] = {0.0, 0.0};
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(host_sums, sums, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "adjoint outputs");
    rc = wait_stream(h, 0);
    if (rc) return rc;
    *J = host_sums[0];
    *grad_beta = host_sums[1];
    if (h->flag_host[0] & 2) return fail(h, KBC_ERR_TIMEOUT, "a device-side wait ran out");
    if (h->flag_host[0] & 1) return fail(h, KBC_ERR_NONFINITE, "non-finite populations in the forward sweep");
    if ((h->flag_host[0] & 8) || !std::isfinite(*J) || !std::isfinite(*grad_beta))
        return fail(h, KBC_ERR_NONFINITE,
                    "the adjoint overflowed: where <dh|dh> is tiny gamma* leaves [0, 2/beta] "
                    "and the linearised step amplifies by |1 - beta gamma| > 1 (smooth fields, "
                    "many steps); use FP64 storage or fewer steps");
    return KBC_OK;
}

int kbc_diagnostics_ext(kbc_handle h, double* out)
{
    int rc = check_h(h);
    if (rc) return rc;
    if (h->slab) return reject_slab(h, "kbc_diagnostics_ext");
    if (!out) return fail(h, KBC_ERR_ARG, "NULL output");
    if (!h->initialized) return fail(h, KBC_ERR_STATE, "field not initialised");
    StepArgs a = args_of(h);
    cudaError_t e = by_codec(h->dtype, [&](auto c) {
        using C = decltype(c);
        return launch_diag_ext<C>(h->buf[h->cur], h->diag_part, h->diag_nblocks, h->diag_out, a,
                                  h->stream);
    });
    if (e != cudaSuccess) return cuda_fail(h, e, "diagnostics launch");
    e = cudaMemcpyAsync(out, h->diag_out, KBC_DIAG_EXT_N * sizeof(double), cudaMemcpyDefault, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "diagnostics copy");
    return wait_stream(h, 0);
}

// Rows of the halo of one face: the first of its populations and the row
// (relative to interior row 0) in the current field.  A full halo is all
// nine populations of the row.
static void halo_rows(const kbc_ctx* h, int face, bool ghost, bool full, int* pop0, long long* row)
{
    if (!ghost) {
        // outgoing: the bottom row's b = -1 populations, the top row's b = +1
        *pop0 = full ? 0 : (face == 0 ? 0 : 6);
        *row = face == 0 ? 0 : h->ny - 1;
    } else {
        // incoming: the lower ghost row's b = +1 populations, the upper's b = -1
        *pop0 = full ? 0 : (face == 0 ? 6 : 0);
        *row = face == 0 ? -1 : h->ny;
    }
}

static int halo_copy(kbc_handle h, int face, int full, void* out, const void* in)
{
    int rc = check_h(h);
    if (rc) return rc;
    if (!h->slab) return fail(h, KBC_ERR_ARG, "halo exchange needs a y-slab handle (kbc_create_slab)");
    if (face != 0 && face != 1) return fail(h, KBC_ERR_ARG, "face must be 0 (lower) or 1 (upper)");
    if (full != 0 && full != 1) return fail(h, KBC_ERR_ARG, "full must be 0 or 1");
    if (!(out ? (const void*)out : in)) return fail(h, KBC_ERR_ARG, "NULL buffer");
    if (out && !h->initialized) return fail(h, KBC_ERR_STATE, "field not initialised");
    int pop0;
    long long row;
    halo_rows(h, face, in != nullptr, full != 0, &pop0, &row);
    char* field = static_cast<char*>(h->buf[h->cur]) + ((long long)pop0 * h->plane + row * h->nx) * (long long)h->elem;
    const size_t width = (size_t)h->nx * h->elem, pitch = (size_t)h->plane * h->elem;
    const size_t rows = full ? 9 : 3;
    cudaError_t e = out ? cudaMemcpy2DAsync(out, width, field, pitch, width, rows, cudaMemcpyDefault, h->stream)
                        : cudaMemcpy2DAsync(field, pitch, in, width, width, rows, cudaMemcpyDefault, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "halo copy");
    if (in) h->ghosts_full = full ? (h->ghosts_full | (1 << face)) : (h->ghosts_full & ~(1 << face));
    const bool host = !is_device_ptr(out ? (const void*)out : in);
    return host ? wait_stream(h, 0) : KBC_OK;
}

int kbc_halo_send(kbc_handle h, int face, int full, void* buf)
{
    return halo_copy(h, face, full, buf, nullptr);
}

int kbc_halo_recv(kbc_handle h, int face, int full, const void* buf)
{
    return halo_copy(h, face, full, nullptr, buf);
}

int kbc_halo_bytes(kbc_handle h, int full, size_t* bytes)
{
    if (!h || !bytes || (full != 0 && full != 1)) return KBC_ERR_ARG;
    *bytes = (size_t)(full ? 9 : 3) * h->nx * h->elem;
    return KBC_OK;
}

int kbc_bytes_per_update(kbc_handle h, double* bytes)
{
    if (!h || !bytes) return KBC_ERR_ARG;
    *bytes = 18.0 * (double)h->elem;
    return KBC_OK;
}

int kbc_spectrum(int n, const double* u, int nbins, double* E, double* Z, void* stream)
{
    if (n < 2 || n % 2 != 0 || (long long)n * n > 2147483647LL)
        return fail(nullptr, KBC_ERR_ARG, "spectrum: n must be even, 2 <= n, n^2 < 2^31");
    if (nbins < 1 || !u || !E || !Z) return fail(nullptr, KBC_ERR_ARG, "spectrum: bad argument");
    Allocator al;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        al = g_alloc;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // scratch owned by this call (the handle-free form of CallBuffers)
    struct Scratch {
        Allocator al;
        cudaStream_t s;
        void* p[4] = {nullptr, nullptr, nullptr, nullptr};
        int k = 0;
        cufftHandle plan = 0;
        bool planned = false;
        void* get(size_t bytes)
        {
            if (bytes == 0) bytes = 256;
            void* q = nullptr;
            if (al.alloc) q = al.alloc(bytes, (void*)s, al.user);
            else if (cudaMalloc(&q, bytes) != cudaSuccess) {
                cudaGetLastError();
                q = nullptr;
            }
            if (q) p[k++] = q;
            return q;
        }
        ~Scratch()
        {
            cudaStreamSynchronize(s);
            if (planned) cufftDestroy(plan);
            for (int j = 0; j < k; ++j) {
                if (al.release) al.release(p[j], (void*)s, al.user);
                else cudaFree(p[j]);
            }
            cudaGetLastError();
        }
    } sc{al, s};
    const size_t nn = (size_t)n * n;
    const double* du = u;
    if (!is_device_ptr(u)) {
        double* st = static_cast<double*>(sc.get(2 * nn * sizeof(double)));
        if (!st) return fail(nullptr, KBC_ERR_NOMEM, "spectrum: staging allocation failed");
        cudaError_t e = cudaMemcpyAsync(st, u, 2 * nn * sizeof(double), cudaMemcpyDefault, s);
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "spectrum: upload");
        du = st;
    }
    double2* uh = static_cast<double2*>(sc.get((size_t)n * (n / 2 + 1) * sizeof(double2)));
    double* acc = static_cast<double*>(sc.get(2 * (size_t)nbins * sizeof(double)));
    if (!uh || !acc) return fail(nullptr, KBC_ERR_NOMEM, "spectrum: scratch allocation failed");
    // cuFFT (a library step) with its work area from the same allocator
    size_t ws = 0;
    if (cufftCreate(&sc.plan) != CUFFT_SUCCESS) return fail(nullptr, KBC_ERR_CUDA, "spectrum: cufftCreate");
    sc.planned = true;
    if (cufftSetAutoAllocation(sc.plan, 0) != CUFFT_SUCCESS ||
        cufftMakePlan2d(sc.plan, n, n, CUFFT_D2Z, &ws) != CUFFT_SUCCESS)
        return fail(nullptr, KBC_ERR_CUDA, "spectrum: cuFFT plan");
    void* work = sc.get(ws);
    if (!work) return fail(nullptr, KBC_ERR_NOMEM, "spectrum: cuFFT work area allocation failed");
    if (cufftSetWorkArea(sc.plan, work) != CUFFT_SUCCESS || cufftSetStream(sc.plan, s) != CUFFT_SUCCESS)
        return fail(nullptr, KBC_ERR_CUDA, "spectrum: cuFFT work area / stream");
    cudaError_t e = cudaMemsetAsync(acc, 0, (size_t)nbins * sizeof(double), s);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "spectrum: memset");
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = (size_t)nbins * sizeof(double);
    const int use_smem = smem <= (size_t)160 * 1024 ? 1 : 0;
    if (use_smem && smem > 48 * 1024)
        cudaFuncSetAttribute(spectrum_bin, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const double scale = 1.0 / ((double)nn * (double)nn);
    for (int c = 0; c < 2; ++c) {
        if (cufftExecD2Z(sc.plan, const_cast<double*>(du) + c * nn, reinterpret_cast<cufftDoubleComplex*>(uh)) !=
            CUFFT_SUCCESS)
            return fail(nullptr, KBC_ERR_CUDA, "spectrum: cuFFT execution");
        spectrum_bin<<<sms * 4, 256, use_smem ? smem : 0, s>>>(uh, n, nbins, scale, acc, use_smem);
    }
    spectrum_enstrophy<<<(nbins + 255) / 256, 256, 0, s>>>(acc, acc + nbins, nbins, n);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(E, acc, (size_t)nbins * sizeof(double), cudaMemcpyDefault, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(Z, acc + nbins, (size_t)nbins * sizeof(double), cudaMemcpyDefault, s);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "spectrum");
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "spectrum");
    return KBC_OK;
}

const char* kbc_last_error(kbc_handle h)
{
    return h ? h->err.c_str() : g_create_error.c_str();
}

}  // extern "C"
