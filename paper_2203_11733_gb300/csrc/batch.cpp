// Batched extraction of many independent structures (mixed precision):
// pooled device buffers, per-structure offsets and prefix sums, and one CUDA
// graph holding the whole pipeline (assembly, factorisation, refinement,
// residuals, capacitances), replayed by gbem_batch_run.
#include <cuda_runtime.h>

#include <algorithm>
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

struct gbem_batch_s {
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

extern "C" {

gbem_status gbem_batch_create(gbem_ctx* ctx, int count, gbem_mesh_t* const* meshes, int iters, gbem_batch_t** out)
{
    if (!ctx || !out || count <= 0 || !meshes) return GBEM_ERR_ARG;
    *out = nullptr;
    if (ctx->device < 0) return ctx_fail(ctx, GBEM_ERR_NODEV, "context has no device");
    for (int b = 0; b < count; ++b) {
        if (!meshes[b] || meshes[b]->ctx != ctx) return ctx_fail(ctx, GBEM_ERR_ARG, "mesh from another context");
        if (meshes[b]->n_cond > 16) return ctx_fail(ctx, GBEM_ERR_ARG, "batched structures have at most 16 conductors");
    }
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(ctx->device);
    gbem_batch_t* B = new (std::nothrow) gbem_batch_t();
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
        gbem_batch_destroy(B);
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

static gbem_status batch_capture(gbem_batch_t* B)
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

gbem_status gbem_batch_run(gbem_batch_t* B, double eps_r, double* C_host, double* resid_host, gbem_stream stream)
{
    if (!B || !C_host || !(eps_r > 0)) return GBEM_ERR_ARG;
    gbem_ctx* ctx = B->ctx;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(ctx->device);
    struct Restore {
        int dev;
        ~Restore()
        {
            if (dev >= 0) cudaSetDevice(dev);
        }
    } restore{prev};
    gbem_status st;
    if (!B->exec && (st = batch_capture(B)) != GBEM_OK) return st;
    cudaStream_t user = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaEventRecord(B->ev, user);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(B->stream, B->ev, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(B->exec, B->stream);
    count_launch(B->graph_kernels);
    if (e == cudaSuccess) e = cudaMemcpyAsync(C_host, B->v.C, sizeof(double) * B->c_total, cudaMemcpyDeviceToHost, B->stream);
    std::vector<double> res(B->nb);
    std::vector<int> flags(4 * (size_t)B->nb);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(res.data(), B->v.resid, sizeof(double) * B->nb, cudaMemcpyDeviceToHost, B->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(flags.data(), B->v.flags, sizeof(int) * flags.size(), cudaMemcpyDeviceToHost, B->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(B->stream);
    if (e != cudaSuccess) return ctx_fail(ctx, GBEM_ERR_CUDA, std::string("batch run: ") + cudaGetErrorString(e));
    for (size_t i = 0; i < B->c_total; ++i) C_host[i] *= eps_r;
    if (resid_host) std::memcpy(resid_host, res.data(), sizeof(double) * B->nb);
    for (int b = 0; b < B->nb; ++b) {
        if (flags[4 * (size_t)b])
            return ctx_fail(ctx, GBEM_ERR_NOT_SPD, "structure " + std::to_string(b) + ": non-positive pivot");
        if (flags[4 * (size_t)b + 3])
            return ctx_fail(ctx, GBEM_ERR_TIMEOUT, "structure " + std::to_string(b) + ": bounded wait gave up");
    }
    return GBEM_OK;
}

gbem_status gbem_batch_info(const gbem_batch_t* B, int* count, long long* c_total, long long* c_offset)
{
    if (!B) return GBEM_ERR_ARG;
    if (count) *count = B->nb;
    if (c_total) *c_total = (long long)B->c_total;
    if (c_offset) std::memcpy(c_offset, B->coff_host.data(), sizeof(long long) * B->nb);
    return GBEM_OK;
}

void gbem_batch_destroy(gbem_batch_t* B)
{
    if (!B) return;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(B->ctx->device);
    if (B->stream) cudaStreamSynchronize(B->stream);
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->ev) cudaEventDestroy(B->ev);
    if (B->stream) cudaStreamDestroy(B->stream);
    if (B->buf) ctx_free(B->ctx, B->buf, B->bytes, nullptr);
    if (prev >= 0) cudaSetDevice(prev);
    delete B;
}

}  // extern "C"
