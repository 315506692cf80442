// C ABI of libgbem (declared and documented in include/gbem.h): contexts,
// device memory through the caller's allocator, mesh and matrix handles, and
// the orchestration of the extraction steps of Wu & Li, Sec. 3.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "gbem_internal.h"

std::atomic<long long> g_gbem_launches{0};

namespace {

constexpr double kEps0 = 8.8541878128e-12;  // F/m

// Records CUDA events around a phase on the call's stream when timing is on.
struct PhaseTimer {
    gbem_ctx* ctx;
    int phase;
    cudaStream_t s;
    cudaEvent_t a = nullptr;
    PhaseTimer(gbem_ctx* c, int ph, cudaStream_t st) : ctx(c), phase(ph), s(st)
    {
        if (ctx->timing && cudaEventCreate(&a) == cudaSuccess) cudaEventRecord(a, s);
        else a = nullptr;
    }
    ~PhaseTimer()
    {
        if (!a) return;
        cudaEvent_t b = nullptr;
        if (cudaEventCreate(&b) == cudaSuccess && cudaEventRecord(b, s) == cudaSuccess)
            ctx->pending.push_back({phase, a, b});
        else {
            cudaEventDestroy(a);
            if (b) cudaEventDestroy(b);
        }
    }
};

}  // namespace

thread_local KernelTrace* g_trace = nullptr;

cudaEvent_t trace_begin(cudaStream_t s)
{
    if (!g_trace) return nullptr;
    cudaEvent_t a = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventRecord(a, s) != cudaSuccess) {
        if (a) cudaEventDestroy(a);
        cudaGetLastError();
        return nullptr;
    }
    return a;
}

void trace_end(int kind, cudaEvent_t a, cudaStream_t s, double bytes, double flops)
{
    if (!g_trace || !a) return;
    cudaEvent_t b = nullptr;
    if (cudaEventCreate(&b) == cudaSuccess && cudaEventRecord(b, s) == cudaSuccess) {
        g_trace->recs.push_back({kind, a, b, bytes, flops});
        return;
    }
    cudaGetLastError();
    cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
}

TraceScope::TraceScope(gbem_ctx* ctx) : prev(g_trace) { g_trace = (ctx && ctx->ktiming) ? &ctx->ktrace : nullptr; }
TraceScope::~TraceScope() { g_trace = prev; }

namespace {

gbem_tuning default_tuning()
{
    gbem_tuning t{};
    t.q_near_fp64 = 12.0;
    // below q = 1 the FP32 6-point rule misses its 3e-7 target on large
    // panels next to small ones (40 x 10 um enclosure walls beside 1 um
    // panels: 7.7e-6); the FP64 closed form is exact there.  Pairs of similar
    // sizes keep the 6-point rule down to q = 0.5 (the assembly's switch)
    t.q_near_mixed = 1.0;
    // |B - A X| / |B| <= 1e-11 makes X the exact solution of a system whose
    // matrix differs from the assembled one by at most 1e-11 relative (the
    // normwise backward error); the mixed assembly's own FP32 far field is
    // about 1e-7 away from the exact integrals, so refining further moves
    // the capacitances by nothing measurable
    t.ir_tol = 1e-11;
    t.ir_max_iter = 10;
    t.nb = 64;
    return t;
}

bool cuda_ok(gbem_ctx* ctx, cudaError_t e, const char* what)
{
    if (e == cudaSuccess) return true;
    ctx->err = std::string(what) + ": " + cudaGetErrorString(e);
    return false;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (dev >= 0 && cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

size_t round_up(size_t x, size_t m) { return (x + m - 1) / m * m; }

// A spare buffer of exactly `bytes` (idle), or null.
void* take_spare(gbem_ctx* ctx, size_t bytes)
{
    for (size_t i = ctx->spare.size(); i-- > 0;) {
        if (ctx->spare[i].bytes != bytes) continue;
        void* p = ctx->spare[i].p;
        ctx->spare.erase(ctx->spare.begin() + (long)i);
        return p;
    }
    return nullptr;
}

// Allocate from the context (a spare buffer of the same size first) and
// remember it in the matrix for release.
template <typename T>
T* mat_alloc(gbem_matrix_t* m, size_t count, cudaStream_t s)
{
    size_t bytes = round_up(std::max<size_t>(count * sizeof(T), 256), 256);
    void* p = take_spare(m->ctx, bytes);
    if (!p) p = ctx_alloc(m->ctx, bytes, s);
    if (p) m->allocs.emplace_back(p, bytes);
    return static_cast<T*>(p);
}

gbem_status upload_mesh(gbem_ctx* ctx, gbem_mesh_t* m)
{
    if (ctx->device < 0 || m->n == 0) return GBEM_OK;
    DeviceGuard g(ctx->device);
    PhaseTimer pt(ctx, GBEM_PHASE_MESH, nullptr);
    const size_t n = (size_t)m->n;
    const size_t bytes = round_up(5 * n * sizeof(double), 256) + round_up(n, 256) +
                         round_up(n * sizeof(int32_t), 256);
    void* buf = ctx_alloc(ctx, bytes, nullptr);
    if (!buf) return GBEM_ERR_OOM;
    m->dbuf = buf;
    m->dbytes = bytes;
    std::vector<unsigned char> host(bytes, 0);
    double* gd = reinterpret_cast<double*>(host.data());
    for (size_t i = 0; i < n; ++i)
        for (int e = 0; e < 5; ++e) gd[e * n + i] = m->geo[5 * i + e];
    size_t off_axis = round_up(5 * n * sizeof(double), 256);
    size_t off_cond = off_axis + round_up(n, 256);
    std::memcpy(host.data() + off_axis, m->axis.data(), n);
    std::memcpy(host.data() + off_cond, m->cond.data(), n * sizeof(int32_t));
    if (!cuda_ok(ctx, cudaMemcpy(buf, host.data(), bytes, cudaMemcpyHostToDevice), "mesh upload"))
        return GBEM_ERR_CUDA;
    const double* d = static_cast<const double*>(buf);
    m->dev.c = d;
    m->dev.lo0 = d + n;
    m->dev.hi0 = d + 2 * n;
    m->dev.lo1 = d + 3 * n;
    m->dev.hi1 = d + 4 * n;
    m->dev.axis = reinterpret_cast<const int8_t*>(static_cast<unsigned char*>(buf) + off_axis);
    m->dev.cond = reinterpret_cast<const int32_t*>(static_cast<unsigned char*>(buf) + off_cond);
    m->dev.n = m->n;
    return GBEM_OK;
}

// Compact caller conductor ids to 0..n_c-1 in ascending id order.
void compact_conductors(gbem_mesh_t* m, const std::vector<int32_t>& raw)
{
    std::vector<int32_t> ids(raw);
    std::sort(ids.begin(), ids.end());
    ids.erase(std::unique(ids.begin(), ids.end()), ids.end());
    std::map<int32_t, int32_t> idx;
    for (size_t k = 0; k < ids.size(); ++k) idx[ids[k]] = (int32_t)k;
    m->cond.resize(raw.size());
    for (size_t i = 0; i < raw.size(); ++i) m->cond[i] = idx[raw[i]];
    m->cond_ids = ids;
    m->n_cond = (int)ids.size();
}

gbem_status ensure_solve_buffers(gbem_matrix_t* m, int nrhs, cudaStream_t s)
{
    if (m->cap_rhs >= nrhs) return GBEM_OK;
    const size_t np = (size_t)m->np;
    // older buffers stay in the allocation list until the matrix is destroyed;
    // the matrix takes the new set only once all of it is allocated, so a
    // refusal leaves the previous, smaller set in use
    double* X = mat_alloc<double>(m, np * nrhs, s);
    double* R = X ? mat_alloc<double>(m, np * nrhs, s) : nullptr;
    double* B = R ? mat_alloc<double>(m, np * nrhs, s) : nullptr;
    unsigned long long* chk = B ? mat_alloc<unsigned long long>(m, 2 * (size_t)nrhs + 1, s) : nullptr;
    // W: FP64 mode, solve vectors and work (2 x np x nrhs doubles); mixed
    // mode, FP32 solve vectors and work, then X as float pairs (4 x np x nrhs
    // floats): the same bytes
    double* W = chk ? mat_alloc<double>(m, 2 * np * nrhs, s) : nullptr;
    if (!W) return GBEM_ERR_OOM;
    if (cudaMemsetAsync(chk, 0, (2 * (size_t)nrhs + 1) * sizeof(unsigned long long), s) != cudaSuccess) {
        cudaGetLastError();
        return GBEM_ERR_CUDA;
    }
    m->X = X;
    m->R = R;
    m->B = B;
    m->dchk = chk;
    m->W = W;
    m->cap_rhs = nrhs;
    return GBEM_OK;
}

// Solve with the padded right-hand sides already in m->B (np x nrhs); the
// solution ends in m->X.  Mixed mode refines in FP64.
gbem_status solve_padded(gbem_matrix_t* m, int nrhs, cudaStream_t s, int* iters, double* resid)
{
    gbem_ctx* ctx = m->ctx;
    PhaseTimer pt(ctx, GBEM_PHASE_SOLVE, s);
    const int np = m->np;
    if (m->prec == GBEM_FP64) {
        double* W = static_cast<double*>(m->W);
        if (!cuda_ok(ctx, cudaMemcpyAsync(W, m->B, sizeof(double) * np * nrhs, cudaMemcpyDeviceToDevice, s),
                     "solve copy"))
            return GBEM_ERR_CUDA;
        if (!cuda_ok(ctx,
                     launch_trsv_f64(m->L64, static_cast<const double*>(m->Linv), np, m->nb, W, nrhs, m->dsync,
                                     m->dflags + 3, s),
                     "trsv"))
            return GBEM_ERR_CUDA;
        if (!cuda_ok(ctx, cudaMemcpyAsync(m->X, W, sizeof(double) * np * nrhs, cudaMemcpyDeviceToDevice, s),
                     "solve copy"))
            return GBEM_ERR_CUDA;
        if (iters) *iters = 0;
        if (resid) {
            if (!cuda_ok(ctx, launch_residual(m->A64, np, m->B, m->X, nrhs, m->R, nullptr, s), "residual"))
                return GBEM_ERR_CUDA;
            if (!cuda_ok(ctx, cudaMemsetAsync(m->dflags + 1, 0, 2 * sizeof(int), s), "memset"))
                return GBEM_ERR_CUDA;
            if (!cuda_ok(ctx, launch_ir_check(m->R, m->B, np, nrhs, m->dnorm, 0.0, m->dflags, s), "check"))
                return GBEM_ERR_CUDA;
            double h = 0.0;
            if (!cuda_ok(ctx, cudaMemcpyAsync(&h, m->dnorm, sizeof(double), cudaMemcpyDeviceToHost, s), "d2h") ||
                !cuda_ok(ctx, cudaStreamSynchronize(s), "sync"))
                return GBEM_ERR_CUDA;
            *resid = h;
        }
        return GBEM_OK;
    }
    // mixed: X = 0, R = B; repeat { W = f32(R); W = L^-T L^-1 W; X += W; R = B - A X }
    float* W = static_cast<float*>(m->W);
    float2* Xdf = reinterpret_cast<float2*>(W + 2 * (size_t)np * nrhs);
    const float* Lf = m->A32;
    const float* Li = static_cast<const float*>(m->Linv);
    int* done = m->dflags + 1;
    if (!cuda_ok(ctx, launch_ir_begin(m->B, np, nrhs, m->X, m->R, m->dnorm, m->dflags, s), "ir begin"))
        return GBEM_ERR_CUDA;
    const int maxit = std::max(1, ctx->tune.ir_max_iter);
    int host_flags[3] = {0, 0, 0};
    for (int it = 0; it < maxit; ++it) {
        if (!cuda_ok(ctx, launch_to_f32(m->R, np, nrhs, W, done, s), "to_f32") ||
            !cuda_ok(ctx, launch_trsv_f32_guarded(Lf, Li, np, m->nb, W, nrhs, m->dsync, m->dflags + 3, done, s),
                     "trsv") ||
            !cuda_ok(ctx, launch_add_f32(W, np, nrhs, m->X, Xdf, done, s), "add") ||
            !cuda_ok(ctx,
                     launch_residual_df(reinterpret_cast<const float2*>(m->A64), np, m->B, Xdf, nrhs, m->R, done, s,
                                        m->dchk, m->dnorm, ctx->tune.ir_tol, m->dflags),
                     "residual"))
            return GBEM_ERR_CUDA;
        // read the flags back: stop once converged.  The first two
        // iterations go out together (a converged iteration leaves the next
        // one's kernels without work), saving one host round trip.
        if (it == 0 && maxit > 1) continue;
        if (!cuda_ok(ctx, cudaMemcpyAsync(host_flags, m->dflags, 3 * sizeof(int), cudaMemcpyDeviceToHost, s),
                     "d2h") ||
            !cuda_ok(ctx, cudaStreamSynchronize(s), "sync"))
            return GBEM_ERR_CUDA;
        if (host_flags[1]) break;
    }
    double h = 0.0;
    if (!cuda_ok(ctx, cudaMemcpyAsync(&h, m->dnorm, sizeof(double), cudaMemcpyDeviceToHost, s), "d2h") ||
        !cuda_ok(ctx, cudaStreamSynchronize(s), "sync"))
        return GBEM_ERR_CUDA;
    if (iters) *iters = host_flags[2];
    if (resid) *resid = h;
    if (!host_flags[1]) {
        ctx->err = "iterative refinement did not reach the tolerance (residual " + std::to_string(h) + ")";
        return GBEM_ERR_NOCONV;
    }
    return GBEM_OK;
}

}  // namespace

// ------------------------------------------------------------------ helpers

gbem_status ctx_fail(gbem_ctx* ctx, gbem_status st, const std::string& msg)
{
    if (ctx) ctx->err = msg;
    return st;
}

static void* raw_alloc(gbem_ctx* ctx, size_t bytes, cudaStream_t s)
{
    void* p = nullptr;
    if (ctx->alloc) {
        p = ctx->alloc(bytes, (gbem_stream)s, ctx->user);
        if (!p) ctx->err = "allocator refused " + std::to_string(bytes) + " bytes";
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
        ctx->err = "cudaMalloc failed for " + std::to_string(bytes) + " bytes";
    }
    return p;
}

void* ctx_alloc(gbem_ctx* ctx, size_t bytes, cudaStream_t s)
{
    if (ctx->budget && ctx->in_use + bytes > ctx->budget) ctx_drop_spare(ctx);
    if (ctx->budget && ctx->in_use + bytes > ctx->budget) {
        ctx->err = "HBM budget exceeded: " + std::to_string(ctx->in_use + bytes) + " > " +
                   std::to_string(ctx->budget) + " bytes";
        return nullptr;
    }
    void* p = raw_alloc(ctx, bytes, s);
    if (!p && !ctx->spare.empty()) {   // the spare buffers may be what is missing
        ctx_drop_spare(ctx);
        p = raw_alloc(ctx, bytes, s);
    }
    if (p) ctx->in_use += bytes;
    return p;
}

void ctx_free(gbem_ctx* ctx, void* p, size_t bytes, cudaStream_t s)
{
    if (!p) return;
    if (ctx->free_fn) ctx->free_fn(p, bytes, (gbem_stream)s, ctx->user);
    else cudaFree(p);
    ctx->in_use -= std::min(ctx->in_use, bytes);
}

void ctx_drop_spare(gbem_ctx* ctx)
{
    std::vector<gbem_ctx::Spare> sp;
    sp.swap(ctx->spare);
    for (auto& a : sp) ctx_free(ctx, a.p, a.bytes, a.stream);
}

// ------------------------------------------------------------------ ABI

extern "C" {

gbem_status gbem_create(gbem_ctx** out, int device, size_t hbm_budget, gbem_alloc_fn alloc,
                        gbem_free_fn free_fn, void* user)
{
    if (!out) return GBEM_ERR_ARG;
    *out = nullptr;
    if ((alloc == nullptr) != (free_fn == nullptr)) return GBEM_ERR_ARG;
    gbem_ctx* ctx = new (std::nothrow) gbem_ctx();
    if (!ctx) return GBEM_ERR_OOM;
    ctx->device = device;
    ctx->budget = hbm_budget;
    ctx->alloc = alloc;
    ctx->free_fn = free_fn;
    ctx->user = user;
    ctx->tune = default_tuning();
    if (device >= 0) {
        int count = 0;
        if (cudaGetDeviceCount(&count) != cudaSuccess || device >= count) {
            cudaGetLastError();
            delete ctx;
            return GBEM_ERR_NODEV;
        }
        DeviceGuard g(device);
        cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
        if (gl_upload() != cudaSuccess) {
            cudaGetLastError();
            delete ctx;
            return GBEM_ERR_CUDA;
        }
        ctx->gl_uploaded = true;
    }
    *out = ctx;
    return GBEM_OK;
}

void gbem_destroy(gbem_ctx* ctx)
{
    if (!ctx) return;
    if (!ctx->spare.empty()) {
        DeviceGuard g(ctx->device);
        ctx_drop_spare(ctx);
    }
    for (auto& p : ctx->pending) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    if (!ctx->side_pool.empty()) {
        DeviceGuard g(ctx->device);
        for (auto& sd : ctx->side_pool) {
            cudaEventDestroy(sd.ready);
            cudaEventDestroy(sd.done);
            cudaStreamDestroy(sd.stream);
        }
    }
    delete ctx;
}

const char* gbem_last_error(const gbem_ctx* ctx) { return ctx ? ctx->err.c_str() : "no context"; }

gbem_status gbem_set_tuning(gbem_ctx* ctx, const gbem_tuning* t)
{
    if (!ctx || !t) return GBEM_ERR_ARG;
    gbem_tuning d = default_tuning();
    ctx->tune.q_near_fp64 = t->q_near_fp64 > 0 ? t->q_near_fp64 : d.q_near_fp64;
    ctx->tune.q_near_mixed = t->q_near_mixed > 0 ? t->q_near_mixed : d.q_near_mixed;
    ctx->tune.ir_tol = t->ir_tol > 0 ? t->ir_tol : d.ir_tol;
    ctx->tune.ir_max_iter = t->ir_max_iter > 0 ? t->ir_max_iter : d.ir_max_iter;
    if (t->nb != 0 && t->nb != 64) return ctx_fail(ctx, GBEM_ERR_ARG, "nb must be 64");
    ctx->tune.nb = 64;
    return GBEM_OK;
}

size_t gbem_bytes_in_use(const gbem_ctx* ctx) { return ctx ? ctx->in_use : 0; }

gbem_status gbem_set_timing(gbem_ctx* ctx, int enable)
{
    if (!ctx || enable < 0 || enable > 2) return GBEM_ERR_ARG;
    ctx->timing = enable != 0;
    ctx->ktiming = enable == 2;
    return GBEM_OK;
}

gbem_status gbem_get_kernel_stats(gbem_ctx* ctx, gbem_kernel_stats* out, int reset)
{
    if (!ctx || !out) return GBEM_ERR_ARG;
    DeviceGuard g(ctx->device);
    gbem_status st = GBEM_OK;
    KernelTrace& T = ctx->ktrace;
    for (auto& r : T.recs) {
        float ms = 0.0f;
        if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            T.ms[r.kind] += ms;
            T.launches[r.kind] += 1;
            T.bytes[r.kind] += r.bytes;
            T.flops[r.kind] += r.flops;
        } else {
            cudaGetLastError();
            st = ctx_fail(ctx, GBEM_ERR_CUDA, "event timing failed");
        }
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    T.recs.clear();
    for (int k = 0; k < GBEM_NKERNEL; ++k) {
        out->ms[k] = T.ms[k];
        out->launches[k] = T.launches[k];
        out->bytes[k] = T.bytes[k];
        out->flops[k] = T.flops[k];
        if (reset) T.ms[k] = T.bytes[k] = T.flops[k] = 0.0, T.launches[k] = 0;
    }
    return st;
}

gbem_status gbem_get_stats(gbem_ctx* ctx, gbem_stats* out, int reset)
{
    if (!ctx || !out) return GBEM_ERR_ARG;
    DeviceGuard g(ctx->device);
    gbem_status st = GBEM_OK;
    for (auto& p : ctx->pending) {
        float ms = 0.0f;
        if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            ctx->ms[p.phase] += ms;
            ctx->calls[p.phase] += 1;
        } else {
            cudaGetLastError();
            st = ctx_fail(ctx, GBEM_ERR_CUDA, "event timing failed");
        }
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    ctx->pending.clear();
    for (int k = 0; k < GBEM_NPHASE; ++k) {
        out->ms[k] = ctx->ms[k];
        out->calls[k] = ctx->calls[k];
    }
    out->launches = g_gbem_launches.load();
    if (reset) {
        for (int k = 0; k < GBEM_NPHASE; ++k) {
            ctx->ms[k] = 0.0;
            ctx->calls[k] = 0;
        }
        g_gbem_launches.store(0);
    }
    return st;
}

gbem_status gbem_mesh(gbem_ctx* ctx, const gbem_box* boxes, int nbox, const gbem_mesh_params* params,
                      gbem_mesh_t** out)
{
    if (!ctx || !out) return GBEM_ERR_ARG;
    *out = nullptr;
    gbem_mesh_t* m = new (std::nothrow) gbem_mesh_t();
    if (!m) return GBEM_ERR_OOM;
    m->ctx = ctx;
    std::vector<int32_t> raw;
    gbem_status st = mesh_build_boxes(boxes, nbox, params, m->axis, m->geo, raw, ctx->err);
    if (st != GBEM_OK) {
        delete m;
        return st;
    }
    compact_conductors(m, raw);
    mesh_order(m->axis, m->geo, m->cond);
    m->n = (int)m->axis.size();
    if ((st = upload_mesh(ctx, m)) != GBEM_OK) {
        delete m;
        return st;
    }
    *out = m;
    return GBEM_OK;
}

gbem_status gbem_mesh_graded(gbem_ctx* ctx, const gbem_box* boxes, int nbox, const gbem_partition_params* params,
                             gbem_mesh_t** out)
{
    if (!ctx || !out) return GBEM_ERR_ARG;
    *out = nullptr;
    gbem_mesh_t* m = new (std::nothrow) gbem_mesh_t();
    if (!m) return GBEM_ERR_OOM;
    m->ctx = ctx;
    std::vector<int32_t> raw;
    gbem_status st = mesh_build_graded(boxes, nbox, params, m->axis, m->geo, raw, ctx->err);
    if (st != GBEM_OK) {
        delete m;
        return st;
    }
    compact_conductors(m, raw);
    mesh_order(m->axis, m->geo, m->cond);
    m->n = (int)m->axis.size();
    if ((st = upload_mesh(ctx, m)) != GBEM_OK) {
        delete m;
        return st;
    }
    *out = m;
    return GBEM_OK;
}

gbem_status gbem_mesh_refine(const gbem_mesh_t* mesh, const double* density, double theta, double* eta,
                             gbem_mesh_t** out, int* n_marked)
{
    if (!mesh || !density || !out) return GBEM_ERR_ARG;
    *out = nullptr;
    gbem_ctx* ctx = mesh->ctx;
    if (!(theta >= 0.0 && theta <= 1.0)) return ctx_fail(ctx, GBEM_ERR_ARG, "theta outside [0, 1]");
    if (!mesh->tri.empty()) return ctx_fail(ctx, GBEM_ERR_STATE, "refinement takes rectangle meshes");
    for (int i = 0; i < mesh->n; ++i)
        if (!std::isfinite(density[i])) return ctx_fail(ctx, GBEM_ERR_ARG, "density not finite");
    std::vector<int8_t> a;
    std::vector<double> g, e;
    std::vector<int32_t> c;
    int nm = 0;
    gbem_status st = mesh_refine(mesh->axis, mesh->geo, mesh->cond, density, theta, a, g, c, e, nm);
    if (st != GBEM_OK) return st;
    if (a.size() > 2000000) return ctx_fail(ctx, GBEM_ERR_ARG, "gbem_mesh_refine: more than 2e6 panels");
    gbem_mesh_t* m = new (std::nothrow) gbem_mesh_t();
    if (!m) return GBEM_ERR_OOM;
    m->ctx = ctx;
    m->axis = std::move(a);
    m->geo = std::move(g);
    std::vector<int32_t> raw(c.size());
    for (size_t i = 0; i < c.size(); ++i) raw[i] = mesh->cond_ids[c[i]];   // the caller's conductor ids
    compact_conductors(m, raw);
    mesh_order(m->axis, m->geo, m->cond);
    m->n = (int)m->axis.size();
    if ((st = upload_mesh(ctx, m)) != GBEM_OK) {
        delete m;
        return st;
    }
    if (eta) std::memcpy(eta, e.data(), sizeof(double) * (size_t)mesh->n);
    if (n_marked) *n_marked = nm;
    *out = m;
    return GBEM_OK;
}

gbem_status gbem_mesh_from_panels(gbem_ctx* ctx, int n, const int8_t* axis, const double* geo,
                                  const int32_t* cond, gbem_mesh_t** out)
{
    if (!ctx || !out) return GBEM_ERR_ARG;
    *out = nullptr;
    if (n <= 0 || !axis || !geo || !cond) return ctx_fail(ctx, GBEM_ERR_ARG, "empty panel list");
    for (int i = 0; i < n; ++i) {
        if (axis[i] < 0 || axis[i] > 2) return ctx_fail(ctx, GBEM_ERR_MESH, "panel axis out of range");
        const double* g = geo + 5 * (size_t)i;
        for (int e = 0; e < 5; ++e)
            if (!std::isfinite(g[e])) return ctx_fail(ctx, GBEM_ERR_MESH, "panel coordinate not finite");
        if (!(g[2] > g[1]) || !(g[4] > g[3]))
            return ctx_fail(ctx, GBEM_ERR_MESH, "panel " + std::to_string(i) + " has zero area");
    }
    gbem_mesh_t* m = new (std::nothrow) gbem_mesh_t();
    if (!m) return GBEM_ERR_OOM;
    m->ctx = ctx;
    m->n = n;
    m->axis.assign(axis, axis + n);
    m->geo.assign(geo, geo + 5 * (size_t)n);
    std::vector<int32_t> raw(cond, cond + n);
    compact_conductors(m, raw);
    gbem_status st = upload_mesh(ctx, m);
    if (st != GBEM_OK) {
        delete m;
        return st;
    }
    *out = m;
    return GBEM_OK;
}

// Device copy of a triangle mesh: the vertices (9 doubles a panel) and the
// conductor indices.
static gbem_status upload_triangles(gbem_ctx* ctx, gbem_mesh_t* m)
{
    if (ctx->device < 0) return GBEM_OK;
    DeviceGuard g(ctx->device);
    const size_t n = (size_t)m->n;
    const size_t off_cond = round_up(9 * n * sizeof(double), 256);
    const size_t bytes = off_cond + round_up(n * sizeof(int32_t), 256);
    void* buf = ctx_alloc(ctx, bytes, nullptr);
    if (!buf) return GBEM_ERR_OOM;
    m->dbuf = buf;
    m->dbytes = bytes;
    std::vector<unsigned char> host(bytes, 0);
    std::memcpy(host.data(), m->tri.data(), 9 * n * sizeof(double));
    std::memcpy(host.data() + off_cond, m->cond.data(), n * sizeof(int32_t));
    if (!cuda_ok(ctx, cudaMemcpy(buf, host.data(), bytes, cudaMemcpyHostToDevice), "mesh upload"))
        return GBEM_ERR_CUDA;
    m->dev = DevPanels{};
    m->dev.tri = static_cast<const double*>(buf);
    m->dev.cond = reinterpret_cast<const int32_t*>(static_cast<unsigned char*>(buf) + off_cond);
    m->dev.n = m->n;
    return GBEM_OK;
}

gbem_status gbem_mesh_from_triangles(gbem_ctx* ctx, int n, const double* tri, const int32_t* cond, gbem_mesh_t** out)
{
    if (!ctx || !out) return GBEM_ERR_ARG;
    *out = nullptr;
    if (n <= 0 || !tri || !cond) return ctx_fail(ctx, GBEM_ERR_ARG, "empty triangle list");
    if (n > 2000000) return ctx_fail(ctx, GBEM_ERR_ARG, "more than 2e6 triangles");
    for (int i = 0; i < n; ++i) {
        const double* t = tri + 9 * (size_t)i;
        for (int e = 0; e < 9; ++e)
            if (!std::isfinite(t[e])) return ctx_fail(ctx, GBEM_ERR_MESH, "triangle coordinate not finite");
        const double e1[3] = {t[3] - t[0], t[4] - t[1], t[5] - t[2]}, e2[3] = {t[6] - t[0], t[7] - t[1], t[8] - t[2]};
        const double c0 = e1[1] * e2[2] - e1[2] * e2[1], c1 = e1[2] * e2[0] - e1[0] * e2[2],
                     c2 = e1[0] * e2[1] - e1[1] * e2[0];
        const double l2 = std::max({e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2], e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2]});
        if (!(c0 * c0 + c1 * c1 + c2 * c2 > 1e-24 * l2 * l2))
            return ctx_fail(ctx, GBEM_ERR_MESH, "triangle " + std::to_string(i) + " has zero area");
    }
    gbem_mesh_t* m = new (std::nothrow) gbem_mesh_t();
    if (!m) return GBEM_ERR_OOM;
    m->ctx = ctx;
    m->n = n;
    m->tri.assign(tri, tri + 9 * (size_t)n);
    std::vector<int32_t> raw(cond, cond + n);
    compact_conductors(m, raw);
    gbem_status st = upload_triangles(ctx, m);
    if (st != GBEM_OK) {
        if (m->dbuf) ctx_free(ctx, m->dbuf, m->dbytes, nullptr);
        delete m;
        return st;
    }
    *out = m;
    return GBEM_OK;
}

gbem_status gbem_mesh_triangles(const gbem_mesh_t* mesh, double* tri, int32_t* cond)
{
    if (!mesh) return GBEM_ERR_ARG;
    if (mesh->tri.empty()) return GBEM_ERR_STATE;
    if (tri) std::memcpy(tri, mesh->tri.data(), sizeof(double) * 9 * mesh->n);
    if (cond)
        for (int i = 0; i < mesh->n; ++i) cond[i] = mesh->cond_ids[mesh->cond[i]];
    return GBEM_OK;
}

gbem_status gbem_mesh_info(const gbem_mesh_t* mesh, int* n_panels, int* n_cond)
{
    if (!mesh) return GBEM_ERR_ARG;
    if (n_panels) *n_panels = mesh->n;
    if (n_cond) *n_cond = mesh->n_cond;
    return GBEM_OK;
}

gbem_status gbem_mesh_panels(const gbem_mesh_t* mesh, int8_t* axis, double* geo, int32_t* cond,
                             int32_t* cond_ids)
{
    if (!mesh) return GBEM_ERR_ARG;
    if (!mesh->tri.empty() && (axis || geo)) return GBEM_ERR_STATE;   // a triangle mesh has no rectangles
    if (axis) std::memcpy(axis, mesh->axis.data(), mesh->n);
    if (geo) std::memcpy(geo, mesh->geo.data(), sizeof(double) * 5 * mesh->n);
    if (cond)
        for (int i = 0; i < mesh->n; ++i) cond[i] = mesh->cond_ids[mesh->cond[i]];
    if (cond_ids) std::memcpy(cond_ids, mesh->cond_ids.data(), sizeof(int32_t) * mesh->n_cond);
    return GBEM_OK;
}

void gbem_mesh_destroy(gbem_mesh_t* mesh)
{
    if (!mesh) return;
    if (mesh->dbuf) {
        DeviceGuard g(mesh->ctx->device);
        ctx_free(mesh->ctx, mesh->dbuf, mesh->dbytes, nullptr);
    }
    delete mesh;
}

gbem_status gbem_assemble(gbem_mesh_t* mesh, gbem_precision prec, gbem_stream stream,
                          gbem_matrix_t** out)
{
    if (!mesh || !out) return GBEM_ERR_ARG;
    *out = nullptr;
    gbem_ctx* ctx = mesh->ctx;
    if (ctx->device < 0) return ctx_fail(ctx, GBEM_ERR_NODEV, "context has no device");
    if (prec != GBEM_FP64 && prec != GBEM_MIXED) return ctx_fail(ctx, GBEM_ERR_ARG, "bad precision");
    DeviceGuard g(ctx->device);
    TraceScope ts(ctx);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    gbem_matrix_t* m = new (std::nothrow) gbem_matrix_t();
    if (!m) return GBEM_ERR_OOM;
    m->ctx = ctx;
    m->mesh = mesh;
    m->n = mesh->n;
    m->np = (int)round_up((size_t)mesh->n, GBEM_PAD);
    m->nb = ctx->tune.nb;
    m->prec = prec;
    const size_t np = (size_t)m->np;
    m->A64 = mat_alloc<double>(m, np * np, s);
    if (prec == GBEM_MIXED) m->A32 = mat_alloc<float>(m, np * np, s);
    m->dflags = mat_alloc<int>(m, 4, s);
    m->dcounts = mat_alloc<unsigned long long>(m, 16, s);
    m->dnorm = mat_alloc<double>(m, 4, s);
    if (!m->A64 || (prec == GBEM_MIXED && !m->A32) || !m->dflags || !m->dcounts || !m->dnorm) {
        gbem_matrix_destroy(m);
        return GBEM_ERR_OOM;
    }
    PhaseTimer pt(ctx, GBEM_PHASE_ASSEMBLE, s);
    const double qn = prec == GBEM_MIXED ? ctx->tune.q_near_mixed : ctx->tune.q_near_fp64;
    const bool ok = cuda_ok(ctx, cudaMemsetAsync(m->dflags, 0, 4 * sizeof(int), s), "memset") &&
                    cuda_ok(ctx, cudaMemsetAsync(m->dcounts, 0, 16 * sizeof(unsigned long long), s), "memset") &&
                    cuda_ok(ctx, launch_pad(m->A64, m->A32, m->n, m->np, s), "pad") &&
                    cuda_ok(ctx,
                            mesh->tri.empty()
                                ? launch_assemble(mesh->dev, m->np, prec, qn, m->A64, m->A32, m->dcounts, s)
                                : launch_assemble_tri(mesh->dev.tri, m->n, m->np, prec, m->A64, m->A32, m->dcounts, s),
                            "assemble");
    if (!ok) {
        gbem_matrix_destroy(m);
        return GBEM_ERR_CUDA;
    }
    m->last = s;
    m->used = true;
    *out = m;
    return GBEM_OK;
}

gbem_status gbem_factor(gbem_matrix_t* m, gbem_stream stream)
{
    if (!m) return GBEM_ERR_ARG;
    gbem_ctx* ctx = m->ctx;
    DeviceGuard g(ctx->device);
    TraceScope ts(ctx);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t np = (size_t)m->np;
    const size_t nblk = np / m->nb;
    PhaseTimer pt(ctx, GBEM_PHASE_FACTOR, s);
    if (!m->dsync) {
        m->dsync = mat_alloc<unsigned>(m, nblk, s);
        if (!m->dsync) return GBEM_ERR_OOM;
        if (!cuda_ok(ctx, cudaMemsetAsync(m->dsync, 0, nblk * sizeof(unsigned), s), "memset")) return GBEM_ERR_CUDA;
    }
    if (m->prec == GBEM_FP64) {
        if (!m->L64) m->L64 = mat_alloc<double>(m, np * np, s);
        if (!m->Linv) m->Linv = mat_alloc<double>(m, nblk * m->nb * m->nb, s);
        if (!m->L64 || !m->Linv) return GBEM_ERR_OOM;
        if (!cuda_ok(ctx, launch_copy_lower(m->A64, m->L64, m->np, s), "copy") ||
            !cuda_ok(ctx, launch_cholesky_f64(m->L64, m->np, m->nb, static_cast<double*>(m->Linv), m->dflags, s),
                     "cholesky"))
            return GBEM_ERR_CUDA;
    } else {
        if (m->factored) return ctx_fail(ctx, GBEM_ERR_STATE, "mixed factor is in place; assemble again");
        if (!m->Linv) m->Linv = mat_alloc<float>(m, nblk * m->nb * m->nb, s);
        if (!m->split) m->split = mat_alloc<unsigned char>(m, cholesky_f32_split_bytes(m->np), s);
        if (!m->Linv || !m->split) return GBEM_ERR_OOM;
        if (ctx->side_stream && !m->side.stream && !ctx->side_pool.empty()) {
            m->side = ctx->side_pool.back();
            ctx->side_pool.pop_back();
        }
        if (ctx->side_stream && !m->side.stream) {
            // the stream of the rest updates, at the lowest priority (the
            // factorisation's own launches take the highest); without it they
            // run on the caller's stream
            int least = 0, greatest = 0;
            SideStream sd;
            if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess ||
                cudaStreamCreateWithPriority(&sd.stream, cudaStreamNonBlocking, least) != cudaSuccess ||
                cudaEventCreateWithFlags(&sd.ready, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&sd.done, cudaEventDisableTiming) != cudaSuccess) {
                cudaGetLastError();
                if (sd.done) cudaEventDestroy(sd.done);
                if (sd.ready) cudaEventDestroy(sd.ready);
                if (sd.stream) cudaStreamDestroy(sd.stream);
                sd = SideStream{};
            }
            m->side = sd;
        }
        if (!cuda_ok(ctx,
                     launch_cholesky_f32(m->A32, m->np, m->nb, static_cast<float*>(m->Linv), m->dflags, m->split, s,
                                         &m->side),
                     "cholesky")) {
            // a launch failed after the rest updates were forked: let them
            // finish before the caller may free what they use
            if (m->side.stream) cudaStreamSynchronize(m->side.stream);
            return GBEM_ERR_CUDA;
        }
    }
    m->factored = true;
    m->last = s;
    m->used = true;
    return GBEM_OK;
}

gbem_status gbem_solve(gbem_matrix_t* m, const double* B_dev, int nrhs, int ldb, double* X_dev, int ldx,
                       int* ir_iters, gbem_stream stream)
{
    if (!m || !B_dev || !X_dev || nrhs <= 0) return GBEM_ERR_ARG;
    gbem_ctx* ctx = m->ctx;
    if (ldb < m->n || ldx < m->n) return ctx_fail(ctx, GBEM_ERR_ARG, "leading dimension below N");
    if (!m->factored) return ctx_fail(ctx, GBEM_ERR_STATE, "solve before factor");
    DeviceGuard g(ctx->device);
    TraceScope ts(ctx);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    gbem_status st = ensure_solve_buffers(m, nrhs, s);
    if (st != GBEM_OK) return st;
    if (!cuda_ok(ctx, launch_pack_rhs(B_dev, ldb, m->n, m->np, nrhs, m->B, s), "pack")) return GBEM_ERR_CUDA;
    int it = 0;
    st = solve_padded(m, nrhs, s, ir_iters ? &it : nullptr, nullptr);
    if (st != GBEM_OK && st != GBEM_ERR_NOCONV) return st;
    if (!cuda_ok(ctx, launch_unpack(m->X, m->np, m->n, nrhs, X_dev, ldx, s), "unpack")) return GBEM_ERR_CUDA;
    if (ir_iters) {
        if (!cuda_ok(ctx, cudaStreamSynchronize(s), "sync")) return GBEM_ERR_CUDA;
        *ir_iters = it;
    }
    m->last = s;
    m->used = true;
    return st;
}

gbem_status gbem_capacitance(gbem_mesh_t* mesh, gbem_matrix_t* m, double eps_r, double* C_host,
                             double* resid_out, gbem_stream stream)
{
    if (!mesh || !m || !C_host || !(eps_r > 0)) return GBEM_ERR_ARG;
    gbem_ctx* ctx = m->ctx;
    if (m->mesh != mesh) return ctx_fail(ctx, GBEM_ERR_ARG, "matrix was assembled from another mesh");
    DeviceGuard g(ctx->device);
    TraceScope ts(ctx);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    gbem_status st;
    if (!m->factored && (st = gbem_factor(m, stream)) != GBEM_OK) return st;
    const int nc = mesh->n_cond;
    if ((st = ensure_solve_buffers(m, nc, s)) != GBEM_OK) return st;
    {
        PhaseTimer pt(ctx, GBEM_PHASE_REDUCE, s);
        if (!cuda_ok(ctx, launch_indicator_rhs(mesh->dev.cond, m->n, m->np, nc, m->B, s), "rhs"))
            return GBEM_ERR_CUDA;
    }
    double resid = 0.0;
    int it = 0;
    st = solve_padded(m, nc, s, &it, &resid);
    if (st != GBEM_OK && st != GBEM_ERR_NOCONV) return st;
    gbem_status solve_st = st;
    // C (n_c x n_c) in the dnorm scratch would be too small: reuse R's head
    double* dC = m->R;
    {
        PhaseTimer pt(ctx, GBEM_PHASE_REDUCE, s);
        if (!cuda_ok(ctx, launch_capacitance(mesh->dev.cond, m->n, m->np, nc, m->X, kEps0 * eps_r * 1e-6, dC, s),
                     "capacitance"))
            return GBEM_ERR_CUDA;
    }
    if (!cuda_ok(ctx, cudaMemcpyAsync(C_host, dC, sizeof(double) * nc * nc, cudaMemcpyDeviceToHost, s), "d2h"))
        return GBEM_ERR_CUDA;
    int flags[4] = {0, 0, 0, 0};
    if (!cuda_ok(ctx, cudaMemcpyAsync(flags, m->dflags, sizeof(flags), cudaMemcpyDeviceToHost, s), "d2h") ||
        !cuda_ok(ctx, cudaStreamSynchronize(s), "sync"))
        return GBEM_ERR_CUDA;
    if (resid_out) *resid_out = resid;
    m->last = s;
    m->used = true;
    if (flags[0]) return ctx_fail(ctx, GBEM_ERR_NOT_SPD, "Cholesky met a non-positive pivot");
    if (flags[3]) return ctx_fail(ctx, GBEM_ERR_TIMEOUT, "a bounded device wait in the solve gave up");
    return solve_st;
}

gbem_status gbem_selftest_wait(gbem_ctx* ctx, int set_flag, double limit_ms, gbem_stream stream)
{
    if (!ctx || !(limit_ms > 0.0) || limit_ms > 10000.0) return GBEM_ERR_ARG;
    if (ctx->device < 0) return ctx_fail(ctx, GBEM_ERR_NODEV, "context has no device");
    DeviceGuard g(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // word 0: the flag the CTA waits for; word 1: the status it reports
    unsigned* buf = static_cast<unsigned*>(ctx_alloc(ctx, 256, s));
    if (!buf) return GBEM_ERR_OOM;
    int status = 0;
    const unsigned one = 1u;
    bool ok = cuda_ok(ctx, cudaMemsetAsync(buf, 0, 256, s), "memset") &&
              (!set_flag || cuda_ok(ctx, cudaMemcpyAsync(buf, &one, sizeof(one), cudaMemcpyHostToDevice, s), "h2d")) &&
              cuda_ok(ctx, launch_wait_selftest(buf, reinterpret_cast<int*>(buf + 1), limit_ms, s), "launch") &&
              cuda_ok(ctx, cudaMemcpyAsync(&status, buf + 1, sizeof(int), cudaMemcpyDeviceToHost, s), "d2h") &&
              cuda_ok(ctx, cudaStreamSynchronize(s), "sync");
    ctx_free(ctx, buf, 256, s);
    if (!ok) return GBEM_ERR_CUDA;
    if (status == GBEM_ERR_TIMEOUT) return ctx_fail(ctx, GBEM_ERR_TIMEOUT, "the bounded wait gave up (flag withheld)");
    return status == 0 ? GBEM_OK : ctx_fail(ctx, GBEM_ERR_CUDA, "unexpected self-test status");
}

gbem_status gbem_matrix_download(gbem_matrix_t* m, double* host)
{
    if (!m || !host) return GBEM_ERR_ARG;
    gbem_ctx* ctx = m->ctx;
    DeviceGuard g(ctx->device);
    const int n = m->n, np = m->np;
    if (!cuda_ok(ctx, cudaStreamSynchronize(m->last), "sync")) return GBEM_ERR_CUDA;
    // column j of the lower triangle: rows j..n-1
    if (!cuda_ok(ctx,
                 cudaMemcpy2D(host, sizeof(double) * n, m->A64, sizeof(double) * np, sizeof(double) * n, n,
                              cudaMemcpyDeviceToHost),
                 "download"))
        return GBEM_ERR_CUDA;
    if (m->prec == GBEM_MIXED) {
        // mixed-mode storage holds float pairs: the entry is hi + lo
        for (size_t e = 0; e < (size_t)n * n; ++e) {
            float p[2];
            std::memcpy(p, host + e, sizeof(p));
            host[e] = (double)p[0] + (double)p[1];
        }
    }
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < j; ++i) host[i + (size_t)j * n] = host[j + (size_t)i * n];
    return GBEM_OK;
}

gbem_status gbem_matrix_status(gbem_matrix_t* m)
{
    if (!m) return GBEM_ERR_ARG;
    gbem_ctx* ctx = m->ctx;
    DeviceGuard g(ctx->device);
    int flags[4] = {0, 0, 0, 0};
    if (!cuda_ok(ctx, cudaStreamSynchronize(m->last), "sync") ||
        !cuda_ok(ctx, cudaMemcpy(flags, m->dflags, sizeof(flags), cudaMemcpyDeviceToHost), "d2h"))
        return GBEM_ERR_CUDA;
    if (flags[0]) return ctx_fail(ctx, GBEM_ERR_NOT_SPD, "Cholesky met a non-positive pivot");
    if (flags[3]) return ctx_fail(ctx, GBEM_ERR_TIMEOUT, "a bounded device wait in the solve gave up");
    return GBEM_OK;
}

// The 14 class counts of the assembly (near parallel, near perpendicular,
// far order n parallel at 2n and perpendicular at 2n + 1).
static gbem_status read_class_counts(gbem_matrix_t* m, long long* cls)
{
    gbem_ctx* ctx = m->ctx;
    unsigned long long c[16] = {};
    if (!cuda_ok(ctx, cudaStreamSynchronize(m->last), "sync") ||
        !cuda_ok(ctx, cudaMemcpy(c, m->dcounts, sizeof(c), cudaMemcpyDeviceToHost), "d2h"))
        return GBEM_ERR_CUDA;
    for (int k = 0; k < 14; ++k) cls[k] = (long long)c[k];
    return GBEM_OK;
}

gbem_status gbem_matrix_info(gbem_matrix_t* m, int* n, long long* counts)
{
    if (!m) return GBEM_ERR_ARG;
    DeviceGuard g(m->ctx->device);
    if (n) *n = m->n;
    if (counts) {
        long long cls[14];
        gbem_status st = read_class_counts(m, cls);
        if (st != GBEM_OK) return st;
        counts[0] = cls[0] + cls[1];
        for (int k = 1; k <= 6; ++k) counts[k] = cls[2 * k] + cls[2 * k + 1];
    }
    return GBEM_OK;
}

gbem_status gbem_matrix_class_counts(gbem_matrix_t* m, long long* counts)
{
    if (!m || !counts) return GBEM_ERR_ARG;
    DeviceGuard g(m->ctx->device);
    return read_class_counts(m, counts);
}

void gbem_matrix_destroy(gbem_matrix_t* m)
{
    if (!m) return;
    DeviceGuard g(m->ctx->device);
    if (m->used) cudaStreamSynchronize(m->last);
    gbem_ctx* ctx = m->ctx;
    if (m->side.stream) {
        cudaStreamSynchronize(m->side.stream);
        ctx->side_pool.push_back(m->side);   // idle: kept for the next matrix
    }
    // the previous matrix's buffers that this one did not take go now; this
    // one's wait for the next matrix if they are known to be idle (a matrix
    // that never finished its assembly call has no synchronised stream)
    ctx_drop_spare(ctx);
    const bool keep = ctx->keep_spare && m->used;
    for (auto& a : m->allocs) {
        if (keep) ctx->spare.push_back({a.first, a.second, m->last});
        else ctx_free(ctx, a.first, a.second, m->last);
    }
    delete m;
}

}  // extern "C"
