// gbem_unit_rates: throughput of the arithmetic units the assembly leans on,
// measured on the context's GPU.  The assembly is bound by arithmetic, not by
// memory: its far field by the MUFU reciprocal square root of every 1/r
// evaluation, its near field by the FP64 closed forms (log, atan, sqrt and
// plain FP64 arithmetic).  Its roofline therefore needs the rate of each of
// these units on this part, which no vendor table states for the FP64 library
// calls; this probe measures them.
//
// Each probe kernel runs `CH` independent dependency chains per thread, a
// whole number of CTAs per SM, and times `iters` steps of every chain with
// CUDA events (best of three after one warm-up launch).  Every chain stays
// finite and data-dependent, and each thread stores its sum, so nothing can
// be folded or dropped.  A step is the operation plus, for the library calls,
// one FP64 add that keeps the argument in range; the add is counted as part
// of the call.
#include <algorithm>
#include <cmath>

#include "gbem_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kCtasPerSm = 8;

__device__ __forceinline__ float mufu_rsqrt(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <int OP>
struct Step;
template <>
struct Step<GBEM_RATE_DFMA> {   // x <- x a + b, fixed point 1
    using T = double;
    static __device__ __forceinline__ T f(T x) { return fma(x, 0.9999999, 1e-7); }
};
template <>
struct Step<GBEM_RATE_FFMA> {
    using T = float;
    static __device__ __forceinline__ T f(T x) { return fmaf(x, 0.9999999f, 1e-7f); }
};
template <>
struct Step<GBEM_RATE_MUFU_RSQRT> {   // x <- 1/sqrt(x), fixed point 1
    using T = float;
    static __device__ __forceinline__ T f(T x) { return mufu_rsqrt(x); }
};
template <>
struct Step<GBEM_RATE_DSQRT> {   // x <- sqrt(x + 1)
    using T = double;
    static __device__ __forceinline__ T f(T x) { return sqrt(x + 1.0); }
};
template <>
struct Step<GBEM_RATE_DLOG> {   // x <- log(x + 2), positive
    using T = double;
    static __device__ __forceinline__ T f(T x) { return log(x + 2.0); }
};
template <>
struct Step<GBEM_RATE_DATAN> {   // x <- atan(x) + 1/2, bounded
    using T = double;
    static __device__ __forceinline__ T f(T x) { return atan(x) + 0.5; }
};
template <>
struct Step<GBEM_RATE_DRSQRT> {   // x <- 1/sqrt(x + 1)
    using T = double;
    static __device__ __forceinline__ T f(T x) { return rsqrt(x + 1.0); }
};

template <int OP, int CH>
__global__ void __launch_bounds__(kThreads) unit_rate_probe(typename Step<OP>::T* __restrict__ out, int iters)
{
    using T = typename Step<OP>::T;
    const int g = blockIdx.x * kThreads + threadIdx.x;
    T x[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) x[c] = T(1) + T(1e-6) * T((g + 7 * c) & 1023);
#pragma unroll 4
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < CH; ++c) x[c] = Step<OP>::f(x[c]);
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < CH; ++c) s += x[c];
    out[g] = s;
}

struct ProbeShape {
    int chains;
    int iters;
};

// Chains per thread and steps per chain: enough chains to cover each unit's
// latency, enough steps for a launch of several milliseconds.
constexpr ProbeShape kShape[GBEM_RATE_COUNT] = {
    {4, 4096},    // DFMA
    {8, 65536},   // FFMA
    {8, 16384},   // MUFU rsqrt
    {4, 512},     // FP64 sqrt
    {4, 1024},    // FP64 log
    {4, 128},     // FP64 atan
    {4, 512},     // FP64 rsqrt
};

template <int OP>
cudaError_t launch_probe(void* out, int grid, cudaStream_t s)
{
    using T = typename Step<OP>::T;
    constexpr int CH = OP == GBEM_RATE_FFMA || OP == GBEM_RATE_MUFU_RSQRT ? 8 : 4;
    static_assert(CH == kShape[OP].chains, "chain count");
    unit_rate_probe<OP, CH><<<grid, kThreads, 0, s>>>(static_cast<T*>(out), kShape[OP].iters);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_op(int op, void* out, int grid, cudaStream_t s)
{
    switch (op) {
    case GBEM_RATE_DFMA: return launch_probe<GBEM_RATE_DFMA>(out, grid, s);
    case GBEM_RATE_FFMA: return launch_probe<GBEM_RATE_FFMA>(out, grid, s);
    case GBEM_RATE_MUFU_RSQRT: return launch_probe<GBEM_RATE_MUFU_RSQRT>(out, grid, s);
    case GBEM_RATE_DSQRT: return launch_probe<GBEM_RATE_DSQRT>(out, grid, s);
    case GBEM_RATE_DLOG: return launch_probe<GBEM_RATE_DLOG>(out, grid, s);
    case GBEM_RATE_DATAN: return launch_probe<GBEM_RATE_DATAN>(out, grid, s);
    default: return launch_probe<GBEM_RATE_DRSQRT>(out, grid, s);
    }
}

}  // namespace

gbem_status gbem_unit_rates(gbem_ctx* ctx, double* rates, int n_rates, gbem_stream stream)
{
    if (!ctx || !rates || n_rates < 1 || n_rates > GBEM_RATE_COUNT) return GBEM_ERR_ARG;
    if (ctx->device < 0) return ctx_fail(ctx, GBEM_ERR_NODEV, "context has no device");
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int sms = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    const int grid = std::max(1, sms) * kCtasPerSm;
    const size_t bytes = sizeof(double) * (size_t)grid * kThreads;
    void* out = e == cudaSuccess ? ctx_alloc(ctx, bytes, s) : nullptr;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    if (e == cudaSuccess && out) e = cudaEventCreate(&ev[0]);
    if (e == cudaSuccess && out) e = cudaEventCreate(&ev[1]);
    for (int op = 0; op < n_rates && e == cudaSuccess && out; ++op) {
        float best = 0.0f;
        for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {   // one warm-up, best of three
            e = cudaEventRecord(ev[0], s);
            if (e == cudaSuccess) e = launch_op(op, out, grid, s);
            if (e == cudaSuccess) e = cudaEventRecord(ev[1], s);
            if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
            float ms = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
            if (e == cudaSuccess && rep > 0 && (best == 0.0f || ms < best)) best = ms;
        }
        if (e == cudaSuccess)
            rates[op] = (double)grid * kThreads * kShape[op].chains * kShape[op].iters / (best * 1e-3);
    }
    if (ev[0]) cudaEventDestroy(ev[0]);
    if (ev[1]) cudaEventDestroy(ev[1]);
    if (out) ctx_free(ctx, out, bytes, s);
    if (prev >= 0) cudaSetDevice(prev);
    if (!out && e == cudaSuccess) return ctx_fail(ctx, GBEM_ERR_OOM, "unit-rate probe buffer");
    if (e != cudaSuccess) return ctx_fail(ctx, GBEM_ERR_CUDA, std::string("unit-rate probe: ") + cudaGetErrorString(e));
    return GBEM_OK;
}
