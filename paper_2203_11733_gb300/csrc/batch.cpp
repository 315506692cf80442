// Batched extraction of many independent structures (mixed precision):
// pooled device buffers, per-structure offsets and prefix sums, and one CUDA
// graph holding the whole pipeline (assembly, factorisation, refinement,
// residuals, capacitances), replayed by gbem_batch_run.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "gbem_internal.h"

namespace {

constexpr double kEps0 = 8.8541878128e-12;
constexpr int kNB = 64;

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

// One group of structures: pooled buffers, views and its own graph.
struct BatchPart {
    gbem_ctx* ctx = nullptr;
    int nb = 0;
    int iters = 3;
    int max_nc = 0;
    int nsteps = 0;
    long long tiles = 0, row_blocks = 0;
    size_t vec_total = 0, c_total = 0;
    std::vector<long long> coff_host;
    std::vector<long long> steps_host;
    void* buf = nullptr;
    size_t bytes = 0;
    BatchView v;
    const long long* steps_dev = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    cudaGraphExec_t exec = nullptr;
    long long graph_kernels = 0;
};

static void part_destroy(BatchPart* B);

static gbem_status part_create(gbem_ctx* ctx, int count, gbem_mesh_t* const* meshes, int iters, BatchPart** out)
{
    if (!ctx || !out || count <= 0 || !meshes) return GBEM_ERR_ARG;
    *out = nullptr;
    if (ctx->device < 0) return ctx_fail(ctx, GBEM_ERR_NODEV, "context has no device");
    for (int b = 0; b < count; ++b) {
        if (!meshes[b] || meshes[b]->ctx != ctx) return ctx_fail(ctx, GBEM_ERR_ARG, "mesh from another context");
        if (meshes[b]->n_cond > 16) return ctx_fail(ctx, GBEM_ERR_ARG, "batched structures have at most 16 conductors");
        if (!meshes[b]->tri.empty()) return ctx_fail(ctx, GBEM_ERR_STATE, "batches take rectangle meshes");
    }
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(ctx->device);
    BatchPart* B = new (std::nothrow) BatchPart();
    if (!B) return GBEM_ERR_OOM;
    B->ctx = ctx;
    B->nb = count;
    B->iters = iters > 0 ? iters : 3;
    const int nb = count;
    std::vector<int> n(nb), np(nb), nc(nb);
    std::vector<long long> poff(nb), moff(nb), voff(nb), ioff(nb), coff(nb), tile_prefix(nb + 1, 0),
        rows_prefix(nb + 1, 0);
    long long P = 0, M = 0, V = 0, I = 0, C = 0;
    int max_nblk = 0;
    for (int b = 0; b < nb; ++b) {
        const gbem_mesh_t* m = meshes[b];
        n[b] = m->n;
        np[b] = (int)((m->n + GBEM_PAD - 1) / GBEM_PAD * GBEM_PAD);
        nc[b] = m->n_cond;
        poff[b] = P;
        moff[b] = M;
        voff[b] = V;
        ioff[b] = I;
        coff[b] = C;
        P += n[b];
        M += (long long)np[b] * np[b];
        V += (long long)np[b] * nc[b];
        I += (long long)(np[b] / kNB) * kNB * kNB;
        C += (long long)nc[b] * nc[b];
        const long long nt = (n[b] + GBEM_TILE - 1) / GBEM_TILE;
        tile_prefix[b + 1] = tile_prefix[b] + nt * (nt + 1) / 2;
        rows_prefix[b + 1] = rows_prefix[b] + np[b] / 16;
        max_nblk = std::max(max_nblk, np[b] / kNB);
        B->max_nc = std::max(B->max_nc, nc[b]);
    }
    B->nsteps = max_nblk;
    B->tiles = tile_prefix[nb];
    B->row_blocks = rows_prefix[nb];
    B->vec_total = (size_t)V;
    B->c_total = (size_t)C;
    B->coff_host = coff;
    // per-step prefix sums: trsm blocks (m_b) then syrk tiles (m_b (m_b + 1) / 2)
    const int nb1 = nb + 1;
    B->steps_host.assign((size_t)2 * max_nblk * nb1, 0);
    for (int k = 0; k < max_nblk; ++k)
        for (int b = 0; b < nb; ++b) {
            const long long m = std::max(0, np[b] / kNB - k - 1);
            B->steps_host[(size_t)k * nb1 + b + 1] = B->steps_host[(size_t)k * nb1 + b] + m;
            B->steps_host[(size_t)(max_nblk + k) * nb1 + b + 1] =
                B->steps_host[(size_t)(max_nblk + k) * nb1 + b] + m * (m + 1) / 2;
        }

    // one allocation: metadata, panels, matrices, vectors, results
    std::vector<std::pair<size_t*, size_t>> parts;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += align256(std::max<size_t>(bytes, 1));
        return o;
    };
    const size_t o_n = take(sizeof(int) * nb), o_np = take(sizeof(int) * nb), o_nc = take(sizeof(int) * nb);
    const size_t o_poff = take(8 * nb), o_moff = take(8 * nb), o_voff = take(8 * nb), o_ioff = take(8 * nb),
                 o_coff = take(8 * nb);
    const size_t o_tp = take(8 * (size_t)nb1), o_rp = take(8 * (size_t)nb1);
    const size_t o_steps = take(8 * B->steps_host.size());
    const size_t o_geo = take(sizeof(double) * 5 * (size_t)P), o_axis = take((size_t)P),
                 o_cond = take(sizeof(int32_t) * (size_t)P);
    const size_t o_A64 = take(sizeof(double) * (size_t)M), o_A32 = take(sizeof(float) * (size_t)M);
    const size_t o_Linv = take(sizeof(float) * (size_t)I);
    const size_t o_B = take(8 * (size_t)V), o_X = take(8 * (size_t)V), o_R = take(8 * (size_t)V),
                 o_W = take(4 * (size_t)V), o_Y = take(4 * (size_t)V), o_Xdf = take(8 * (size_t)V);
    const size_t o_flags = take(sizeof(int) * 4 * (size_t)nb), o_C = take(8 * (size_t)C), o_res = take(8 * (size_t)nb);
    B->bytes = off;
    B->buf = ctx_alloc(ctx, B->bytes, nullptr);
    if (!B->buf) {
        delete B;
        if (prev >= 0) cudaSetDevice(prev);
        return GBEM_ERR_OOM;
    }
    // host image of the metadata and panels
    std::vector<unsigned char> host(o_A64, 0);
    auto put = [&](size_t o, const void* src, size_t bytes) { std::memcpy(host.data() + o, src, bytes); };
    put(o_n, n.data(), sizeof(int) * nb);
    put(o_np, np.data(), sizeof(int) * nb);
    put(o_nc, nc.data(), sizeof(int) * nb);
    put(o_poff, poff.data(), 8 * nb);
    put(o_moff, moff.data(), 8 * nb);
    put(o_voff, voff.data(), 8 * nb);
    put(o_ioff, ioff.data(), 8 * nb);
    put(o_coff, coff.data(), 8 * nb);
    put(o_tp, tile_prefix.data(), 8 * (size_t)nb1);
    put(o_rp, rows_prefix.data(), 8 * (size_t)nb1);
    put(o_steps, B->steps_host.data(), 8 * B->steps_host.size());
    double* geo = reinterpret_cast<double*>(host.data() + o_geo);
    int8_t* axis = reinterpret_cast<int8_t*>(host.data() + o_axis);
    int32_t* cond = reinterpret_cast<int32_t*>(host.data() + o_cond);
    for (int b = 0; b < nb; ++b) {
        const gbem_mesh_t* m = meshes[b];
        for (int i = 0; i < m->n; ++i) {
            const long long g = poff[b] + i;
            for (int e = 0; e < 5; ++e) geo[(size_t)e * P + g] = m->geo[5 * (size_t)i + e];
            axis[g] = m->axis[i];
            cond[g] = m->cond[i];
        }
    }
    cudaError_t e = cudaMemcpy(B->buf, host.data(), host.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        ctx_fail(ctx, GBEM_ERR_CUDA, std::string("batch set-up: ") + cudaGetErrorString(e));
        part_destroy(B);
        if (prev >= 0) cudaSetDevice(prev);
        return GBEM_ERR_CUDA;
    }
    unsigned char* d = static_cast<unsigned char*>(B->buf);
    BatchView& v = B->v;
    v.nb = nb;
    v.n = reinterpret_cast<const int*>(d + o_n);
    v.np = reinterpret_cast<const int*>(d + o_np);
    v.nc = reinterpret_cast<const int*>(d + o_nc);
    v.poff = reinterpret_cast<const long long*>(d + o_poff);
    v.moff = reinterpret_cast<const long long*>(d + o_moff);
    v.voff = reinterpret_cast<const long long*>(d + o_voff);
    v.ioff = reinterpret_cast<const long long*>(d + o_ioff);
    v.coff = reinterpret_cast<const long long*>(d + o_coff);
    v.tile_prefix = reinterpret_cast<const long long*>(d + o_tp);
    v.rows_prefix = reinterpret_cast<const long long*>(d + o_rp);
    B->steps_dev = reinterpret_cast<const long long*>(d + o_steps);
    const double* gd = reinterpret_cast<const double*>(d + o_geo);
    v.c = gd;
    v.lo0 = gd + P;
    v.hi0 = gd + 2 * P;
    v.lo1 = gd + 3 * P;
    v.hi1 = gd + 4 * P;
    v.axis = reinterpret_cast<const int8_t*>(d + o_axis);
    v.cond = reinterpret_cast<const int32_t*>(d + o_cond);
    v.A64 = reinterpret_cast<double*>(d + o_A64);
    v.A32 = reinterpret_cast<float*>(d + o_A32);
    v.Linv = reinterpret_cast<float*>(d + o_Linv);
    v.B = reinterpret_cast<double*>(d + o_B);
    v.X = reinterpret_cast<double*>(d + o_X);
    v.R = reinterpret_cast<double*>(d + o_R);
    v.W = reinterpret_cast<float*>(d + o_W);
    v.Y = reinterpret_cast<float*>(d + o_Y);
    v.Xdf = reinterpret_cast<float2*>(d + o_Xdf);
    v.flags = reinterpret_cast<int*>(d + o_flags);
    v.C = reinterpret_cast<double*>(d + o_C);
    v.resid = reinterpret_cast<double*>(d + o_res);
    if (prev >= 0) cudaSetDevice(prev);
    *out = B;
    return GBEM_OK;
}

static gbem_status batch_capture(BatchPart* B)
{
    gbem_ctx* ctx = B->ctx;
    const BatchView& v = B->v;
    cudaStream_t s = B->stream;
    const long long before = g_gbem_launches.load();
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return ctx_fail(ctx, GBEM_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e));
    cudaError_t err = cudaMemsetAsync(v.flags, 0, sizeof(int) * 4 * (size_t)v.nb, s);
    if (err == cudaSuccess) err = launch_assemble_batched(v, B->tiles, GBEM_MIXED, ctx->tune.q_near_mixed, s);
    if (err == cudaSuccess) err = launch_cholesky_batched(v, B->nsteps, B->steps_dev, B->steps_host.data(), s);
    if (err == cudaSuccess) err = launch_batch_begin(v, s);
    for (int it = 0; it < B->iters && err == cudaSuccess; ++it)
        err = launch_batch_iteration(v, B->vec_total, B->row_blocks, B->max_nc, s);
    if (err == cudaSuccess) err = launch_batch_finish(v, kEps0 * 1e-6, s);
    e = cudaStreamEndCapture(s, &graph);
    if (err != cudaSuccess || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return ctx_fail(ctx, GBEM_ERR_CUDA,
                        std::string("capture: ") + cudaGetErrorString(err != cudaSuccess ? err : e));
    }
    B->graph_kernels = g_gbem_launches.load() - before;
    g_gbem_launches.fetch_sub(B->graph_kernels);   // counted when the graph runs
    e = cudaGraphInstantiate(&B->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return ctx_fail(ctx, GBEM_ERR_CUDA, std::string("instantiate: ") + cudaGetErrorString(e));
    return GBEM_OK;
}

// Enqueue the part's graph on its stream after `fork`, and the reads of its
// results into the part's host buffers.
static cudaError_t part_launch(BatchPart* B, cudaEvent_t fork, std::vector<double>& C, std::vector<double>& res,
                               std::vector<int>& flags)
{
    C.resize(B->c_total);
    res.resize(B->nb);
    flags.resize(4 * (size_t)B->nb);
    cudaError_t e = cudaStreamWaitEvent(B->stream, fork, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(B->exec, B->stream);
    count_launch(B->graph_kernels);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(C.data(), B->v.C, sizeof(double) * B->c_total, cudaMemcpyDeviceToHost, B->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(res.data(), B->v.resid, sizeof(double) * B->nb, cudaMemcpyDeviceToHost, B->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(flags.data(), B->v.flags, sizeof(int) * flags.size(), cudaMemcpyDeviceToHost, B->stream);
    return e;
}

static void part_destroy(BatchPart* B)
{
    if (!B) return;
    if (B->stream) cudaStreamSynchronize(B->stream);
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->ev) cudaEventDestroy(B->ev);
    if (B->stream) cudaStreamDestroy(B->stream);
    if (B->buf) ctx_free(B->ctx, B->buf, B->bytes, nullptr);
    delete B;
}

// A batch: its structures split into groups (parts) whose graphs run
// concurrently on their own streams; results are gathered back into the
// order the structures were given.
struct gbem_batch_s {
    gbem_ctx* ctx = nullptr;
    int nb = 0;
    int groups = 1;
    int iters = 3;
    std::vector<BatchPart*> parts;
    std::vector<int> part_of, index_in_part;   // per structure
    std::vector<long long> coff;               // per structure, caller's order
    long long c_total = 0;
    cudaEvent_t fork = nullptr;
};

namespace {

struct DeviceScope {
    int prev = -1;
    explicit DeviceScope(int dev)
    {
        cudaGetDevice(&prev);
        cudaSetDevice(dev);
    }
    ~DeviceScope()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// Split the structures into `groups` parts of similar factorisation work
// (sum of np^3, largest first onto the lightest part), keeping each part's
// structures in the caller's order.
std::vector<std::vector<int>> split_groups(gbem_mesh_t* const* meshes, int count, int groups)
{
    std::vector<int> idx(count);
    for (int b = 0; b < count; ++b) idx[b] = b;
    auto work = [&](int b) {
        const double np = (double)((meshes[b]->n + GBEM_PAD - 1) / GBEM_PAD * GBEM_PAD);
        return np * np * np;
    };
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return work(a) > work(b); });
    std::vector<std::vector<int>> g(groups);
    std::vector<double> load(groups, 0.0);
    for (int b : idx) {
        const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        g[k].push_back(b);
        load[k] += work(b);
    }
    for (auto& v : g) std::sort(v.begin(), v.end());
    g.erase(std::remove_if(g.begin(), g.end(), [](const std::vector<int>& v) { return v.empty(); }), g.end());
    return g;
}

gbem_status batch_build(gbem_ctx* ctx, int count, gbem_mesh_t* const* meshes, int groups, int iters,
                        gbem_batch_t** out)
{
    gbem_batch_t* B = new (std::nothrow) gbem_batch_t();
    if (!B) return GBEM_ERR_OOM;
    B->ctx = ctx;
    B->nb = count;
    B->iters = iters > 0 ? iters : 3;
    B->part_of.assign(count, 0);
    B->index_in_part.assign(count, 0);
    const auto g = split_groups(meshes, count, std::max(1, std::min(groups, count)));
    B->groups = (int)g.size();
    gbem_status st = GBEM_OK;
    for (int k = 0; k < (int)g.size() && st == GBEM_OK; ++k) {
        std::vector<gbem_mesh_t*> m;
        for (int j = 0; j < (int)g[k].size(); ++j) {
            m.push_back(meshes[g[k][j]]);
            B->part_of[g[k][j]] = k;
            B->index_in_part[g[k][j]] = j;
        }
        BatchPart* P = nullptr;
        st = part_create(ctx, (int)m.size(), m.data(), B->iters, &P);
        if (st == GBEM_OK) B->parts.push_back(P);
    }
    if (st == GBEM_OK && cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        st = ctx_fail(ctx, GBEM_ERR_CUDA, "batch event");
    }
    if (st != GBEM_OK) {
        gbem_batch_destroy(B);
        return st;
    }
    B->coff.assign(count, 0);
    long long off = 0;
    for (int b = 0; b < count; ++b) {
        B->coff[b] = off;
        off += (long long)meshes[b]->n_cond * meshes[b]->n_cond;
    }
    B->c_total = off;
    *out = B;
    return GBEM_OK;
}

// Re-capture every part's graph for another number of refinement passes.
gbem_status batch_set_iters(gbem_batch_t* B, int iters)
{
    B->iters = iters;
    for (BatchPart* P : B->parts) {
        if (P->stream) cudaStreamSynchronize(P->stream);
        if (P->exec) cudaGraphExecDestroy(P->exec);
        P->exec = nullptr;
        P->iters = iters;
    }
    return GBEM_OK;
}

}  // namespace

extern "C" {

gbem_status gbem_batch_create(gbem_ctx* ctx, int count, gbem_mesh_t* const* meshes, int iters, gbem_batch_t** out)
{
    return gbem_batch_create_grouped(ctx, count, meshes, 1, iters, out);
}

gbem_status gbem_batch_create_grouped(gbem_ctx* ctx, int count, gbem_mesh_t* const* meshes, int groups, int iters,
                                      gbem_batch_t** out)
{
    if (!ctx || !out || count <= 0 || !meshes || groups <= 0) return GBEM_ERR_ARG;
    *out = nullptr;
    if (ctx->device < 0) return ctx_fail(ctx, GBEM_ERR_NODEV, "context has no device");
    for (int b = 0; b < count; ++b) {
        if (!meshes[b] || meshes[b]->ctx != ctx) return ctx_fail(ctx, GBEM_ERR_ARG, "mesh from another context");
        if (meshes[b]->n_cond > 16) return ctx_fail(ctx, GBEM_ERR_ARG, "batched structures have at most 16 conductors");
    }
    DeviceScope dev(ctx->device);
    return batch_build(ctx, count, meshes, groups, iters, out);
}

gbem_status gbem_batch_run(gbem_batch_t* B, double eps_r, double* C_host, double* resid_host, gbem_stream stream)
{
    if (!B || !C_host || !(eps_r > 0)) return GBEM_ERR_ARG;
    gbem_ctx* ctx = B->ctx;
    DeviceScope dev(ctx->device);
    gbem_status st;
    for (BatchPart* P : B->parts)
        if (!P->exec && (st = batch_capture(P)) != GBEM_OK) return st;
    cudaStream_t user = static_cast<cudaStream_t>(stream);
    const size_t np = B->parts.size();
    std::vector<std::vector<double>> C(np), res(np);
    std::vector<std::vector<int>> flags(np);
    cudaError_t e = cudaEventRecord(B->fork, user);
    for (size_t k = 0; k < np && e == cudaSuccess; ++k) e = part_launch(B->parts[k], B->fork, C[k], res[k], flags[k]);
    for (size_t k = 0; k < np && e == cudaSuccess; ++k) e = cudaStreamSynchronize(B->parts[k]->stream);
    if (e != cudaSuccess) return ctx_fail(ctx, GBEM_ERR_CUDA, std::string("batch run: ") + cudaGetErrorString(e));
    for (int b = 0; b < B->nb; ++b) {
        const int k = B->part_of[b], j = B->index_in_part[b];
        const BatchPart* P = B->parts[k];
        const long long o = P->coff_host[j];
        const long long nc2 = (b + 1 < B->nb ? B->coff[b + 1] : B->c_total) - B->coff[b];
        for (long long q = 0; q < nc2; ++q) C_host[B->coff[b] + q] = C[k][o + q] * eps_r;
        if (resid_host) resid_host[b] = res[k][j];
        if (flags[k][4 * (size_t)j])
            return ctx_fail(ctx, GBEM_ERR_NOT_SPD, "structure " + std::to_string(b) + ": non-positive pivot");
        if (flags[k][4 * (size_t)j + 3])
            return ctx_fail(ctx, GBEM_ERR_TIMEOUT, "structure " + std::to_string(b) + ": bounded wait gave up");
    }
    return GBEM_OK;
}

gbem_status gbem_batch_info(const gbem_batch_t* B, int* count, long long* c_total, long long* c_offset)
{
    if (!B) return GBEM_ERR_ARG;
    if (count) *count = B->nb;
    if (c_total) *c_total = B->c_total;
    if (c_offset) std::memcpy(c_offset, B->coff.data(), sizeof(long long) * B->nb);
    return GBEM_OK;
}

gbem_status gbem_batch_config(const gbem_batch_t* B, int* groups, int* iters)
{
    if (!B) return GBEM_ERR_ARG;
    if (groups) *groups = B->groups;
    if (iters) *iters = B->iters;
    return GBEM_OK;
}

gbem_status gbem_batch_autotune(gbem_ctx* ctx, int count, gbem_mesh_t* const* meshes, int max_iters,
                                const char* cache_path, gbem_batch_t** out, gbem_batch_tuning* report)
{
    if (!ctx || !out || count <= 0 || !meshes) return GBEM_ERR_ARG;
    *out = nullptr;
    if (max_iters <= 0) max_iters = 3;
    // the cache key: structure count, every structure's order and conductors
    unsigned long long h = 1469598103934665603ull;   // FNV-1a
    auto mix = [&h](unsigned long long x) {
        for (int k = 0; k < 8; ++k) {
            h ^= (x >> (8 * k)) & 0xff;
            h *= 1099511628211ull;
        }
    };
    mix((unsigned long long)count);
    for (int b = 0; b < count; ++b) {
        if (!meshes[b]) return GBEM_ERR_ARG;
        mix((unsigned long long)meshes[b]->n);
        mix((unsigned long long)meshes[b]->n_cond);
    }
    mix((unsigned long long)max_iters);
    char key[32];
    std::snprintf(key, sizeof(key), "%016llx", h);
    gbem_batch_tuning best{};
    best.ms = -1.0;
    // a cached decision: lines "<key> <groups> <iters> <ms>"
    if (cache_path) {
        if (FILE* f = std::fopen(cache_path, "r")) {
            char k[64];
            int g = 0, it = 0;
            double ms = 0.0;
            while (std::fscanf(f, "%63s %d %d %lf", k, &g, &it, &ms) == 4)
                if (std::strcmp(k, key) == 0 && g > 0 && it > 0) {
                    best.groups = g;
                    best.iters = it;
                    best.ms = ms;
                    best.from_cache = 1;
                }
            std::fclose(f);
        }
    }
    if (best.from_cache) {
        gbem_status st = gbem_batch_create_grouped(ctx, count, meshes, best.groups, best.iters, out);
        if (st == GBEM_OK && report) *report = best;
        return st;
    }
    DeviceScope dev(ctx->device);
    std::vector<double> C;
    std::vector<double> res(count);
    gbem_batch_t* keep = nullptr;
    const int cand[3] = {1, 2, 4};
    for (int ci = 0; ci < 3; ++ci) {
        const int groups = cand[ci];
        if (groups > count) break;
        gbem_batch_t* B = nullptr;
        gbem_status st = gbem_batch_create_grouped(ctx, count, meshes, groups, max_iters, &B);
        if (st != GBEM_OK) {
            if (keep) gbem_batch_destroy(keep);
            return st;
        }
        C.resize(B->c_total);
        // the fewest refinement passes that reach the tolerance on every structure
        int iters = max_iters;
        for (int it = 1; it <= max_iters; ++it) {
            batch_set_iters(B, it);
            if (gbem_batch_run(B, 1.0, C.data(), res.data(), nullptr) != GBEM_OK) continue;
            bool ok = true;
            for (int b = 0; b < count; ++b) ok = ok && res[b] <= ctx->tune.ir_tol;
            if (ok) {
                iters = it;
                break;
            }
        }
        batch_set_iters(B, iters);
        // time three runs after one warm-up
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        float ms = 0.0f;
        gbem_status rs = gbem_batch_run(B, 1.0, C.data(), res.data(), nullptr);
        cudaEventRecord(e0, nullptr);
        for (int r = 0; r < 3 && rs == GBEM_OK; ++r) rs = gbem_batch_run(B, 1.0, C.data(), res.data(), nullptr);
        cudaEventRecord(e1, nullptr);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        const double per = ms / 3.0;
        if (rs == GBEM_OK && (best.ms < 0 || per < best.ms)) {
            if (keep) gbem_batch_destroy(keep);
            keep = B;
            best.groups = B->groups;
            best.iters = iters;
            best.ms = per;
        } else {
            gbem_batch_destroy(B);
        }
    }
    if (!keep) return ctx_fail(ctx, GBEM_ERR_CUDA, "autotune: no candidate ran");
    if (cache_path) {
        if (FILE* f = std::fopen(cache_path, "a")) {
            std::fprintf(f, "%s %d %d %.6f\n", key, best.groups, best.iters, best.ms);
            std::fclose(f);
        }
    }
    if (report) *report = best;
    *out = keep;
    return GBEM_OK;
}

void gbem_batch_destroy(gbem_batch_t* B)
{
    if (!B) return;
    DeviceScope dev(B->ctx->device);
    for (BatchPart* P : B->parts) part_destroy(P);
    if (B->fork) cudaEventDestroy(B->fork);
    delete B;
}

}  // extern "C"
