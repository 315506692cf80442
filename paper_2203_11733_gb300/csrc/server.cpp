// Extraction server: continuous batching of independent extraction requests
// on one GPU.
//
// Requests are meshed on the host at submission (so their device footprint
// is known), queued in arrival order, and admitted by a pool of worker
// threads whenever a worker is free: the first queued request, in arrival
// order, that fits in the HBM budget next to the requests already running.
// A smaller request may so pass a head request that waits for memory, but
// the head is passed at most kMaxBypass times; after that nothing is
// admitted before it, so a large request cannot starve.  Every worker owns a context and a
// stream, so admitted requests run concurrently and their kernels overlap on
// the device; a request that arrives while others run starts as soon as a
// worker and memory free up.  Completed results (capacitance matrix, residual,
// submit/start/finish times) are collected by gbem_server_poll.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "gbem_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    long long id = 0;
    std::vector<int8_t> axis;
    std::vector<double> geo;
    std::vector<int32_t> cond;   // caller ids
    double eps_r = 1.0;
    size_t bytes = 0;
    double t_submit = 0.0;
    int bypassed = 0;   // admissions of later requests while this one led the queue
};

// Times the head of the queue may be passed by a later request that fits.
constexpr int kMaxBypass = 8;

struct Result {
    gbem_result_info info{};
    std::vector<double> C;
};

// Device bytes one mixed (or FP64) extraction of order n with nc conductors holds.
size_t request_bytes(int n, int nc, gbem_precision prec)
{
    const size_t np = (size_t)((n + GBEM_PAD - 1) / GBEM_PAD * GBEM_PAD);
    size_t b = 8 * np * np;                                   // A64
    b += (prec == GBEM_MIXED ? 4 : 8) * np * np;              // A32 or the FP64 factor
    b += 8 * np * 64;                                         // diagonal-block inverses
    if (prec == GBEM_MIXED) b += cholesky_f32_split_bytes((int)np);   // split panels, flags
    b += np * (size_t)std::max(nc, 1) * 40;                   // solve vectors
    b += 45 * (size_t)n + (1u << 20);                         // panels, flags, slack
    return b;
}

// Stream-ordered allocation for the workers: no device-wide synchronisation
// on allocate or free, so one worker's allocations never stall another's
// kernels.
void* srv_alloc(size_t bytes, gbem_stream s, void*)
{
    void* p = nullptr;
    if (cudaMallocAsync(&p, bytes, static_cast<cudaStream_t>(s)) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void srv_free(void* p, size_t, gbem_stream s, void*) { cudaFreeAsync(p, static_cast<cudaStream_t>(s)); }

}  // namespace

struct gbem_server_s {
    int device = 0;
    size_t budget = 0;
    size_t reserved = 0;
    gbem_precision prec = GBEM_MIXED;
    Clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request> queue;
    std::deque<Result> done;
    std::vector<std::thread> workers;
    std::vector<gbem_ctx*> ctxs;
    std::vector<cudaStream_t> streams;
    int running = 0;
    long long peak_reserved = 0;
    bool stop = false;
    std::string err;

    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }

    void work(int w)
    {
        cudaSetDevice(device);
        gbem_ctx* ctx = ctxs[w];
        cudaStream_t s = streams[w];
        for (;;) {
            Request req;
            {
                std::unique_lock<std::mutex> lk(mu);
                for (;;) {
                    if (stop) return;
                    // requests larger than the whole budget can never run: reject them
                    for (auto it = queue.begin(); it != queue.end();) {
                        if (it->bytes <= budget) {
                            ++it;
                            continue;
                        }
                        Result r;
                        r.info.id = it->id;
                        r.info.status = GBEM_ERR_OOM;
                        r.info.submit_s = it->t_submit;
                        r.info.start_s = r.info.done_s = now();
                        it = queue.erase(it);
                        done.push_back(std::move(r));
                        cv_done.notify_all();
                    }
                    // the first request in arrival order that fits; the head
                    // alone once it has been passed kMaxBypass times
                    auto pick = queue.end();
                    for (auto it = queue.begin(); it != queue.end(); ++it) {
                        if (reserved + it->bytes <= budget) {
                            pick = it;
                            break;
                        }
                        if (it == queue.begin() && it->bypassed >= kMaxBypass) break;
                    }
                    if (pick != queue.end()) {
                        if (pick != queue.begin()) ++queue.front().bypassed;
                        req = std::move(*pick);
                        queue.erase(pick);
                        reserved += req.bytes;
                        peak_reserved = std::max<long long>(peak_reserved, (long long)reserved);
                        ++running;
                        break;
                    }
                    cv_work.wait(lk);
                }
            }
            Result r;
            r.info.id = req.id;
            r.info.submit_s = req.t_submit;
            r.info.start_s = now();
            r.info.n_panels = (int)req.axis.size();
            gbem_mesh_t* mesh = nullptr;
            gbem_matrix_t* mat = nullptr;
            gbem_status st = gbem_mesh_from_panels(ctx, (int)req.axis.size(), req.axis.data(), req.geo.data(),
                                                   req.cond.data(), &mesh);
            if (st == GBEM_OK) {
                r.info.n_cond = mesh->n_cond;
                r.C.assign((size_t)mesh->n_cond * mesh->n_cond, 0.0);
                st = gbem_assemble(mesh, prec, s, &mat);
            }
            if (st == GBEM_OK) st = gbem_capacitance(mesh, mat, req.eps_r, r.C.data(), &r.info.residual, s);
            if (mat) gbem_matrix_destroy(mat);
            if (mesh) gbem_mesh_destroy(mesh);
            cudaStreamSynchronize(s);
            r.info.status = st;
            r.info.done_s = now();
            {
                std::lock_guard<std::mutex> lk(mu);
                reserved -= req.bytes;
                --running;
                done.push_back(std::move(r));
            }
            cv_work.notify_all();
            cv_done.notify_all();
        }
    }
};

extern "C" {

gbem_status gbem_server_create(int device, size_t hbm_budget, int slots, gbem_precision prec,
                               gbem_server_t** out)
{
    if (!out || slots <= 0 || slots > 64 || hbm_budget == 0) return GBEM_ERR_ARG;
    if (prec != GBEM_FP64 && prec != GBEM_MIXED) return GBEM_ERR_ARG;
    *out = nullptr;
    gbem_server_t* S = new (std::nothrow) gbem_server_t();
    if (!S) return GBEM_ERR_OOM;
    S->device = device;
    S->budget = hbm_budget;
    S->prec = prec;
    S->t0 = Clock::now();
    int prev = -1;
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        delete S;
        return GBEM_ERR_NODEV;
    }
    {
        // keep freed blocks in the device's pool between requests
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
            unsigned long long keep = ~0ull;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
        cudaGetLastError();
    }
    for (int w = 0; w < slots; ++w) {
        gbem_ctx* ctx = nullptr;
        cudaStream_t s = nullptr;
        gbem_status st = gbem_create(&ctx, device, 0, srv_alloc, srv_free, nullptr);
        // a worker's next request has its own size and its memory is
        // reserved at admission: keep no buffers between requests
        if (st == GBEM_OK) ctx->keep_spare = false;
        // the workers already run factorisations side by side: each keeps
        // its rest updates on its own stream instead of forking a second one
        if (st == GBEM_OK) ctx->side_stream = false;
        if (st == GBEM_OK && cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) st = GBEM_ERR_CUDA;
        if (st != GBEM_OK) {
            if (ctx) gbem_destroy(ctx);
            for (auto* c : S->ctxs) gbem_destroy(c);
            for (auto st2 : S->streams) cudaStreamDestroy(st2);
            delete S;
            if (prev >= 0) cudaSetDevice(prev);
            return st;
        }
        S->ctxs.push_back(ctx);
        S->streams.push_back(s);
    }
    for (int w = 0; w < slots; ++w) S->workers.emplace_back([S, w] { S->work(w); });
    if (prev >= 0) cudaSetDevice(prev);
    *out = S;
    return GBEM_OK;
}

gbem_status gbem_server_submit(gbem_server_t* S, long long id, const gbem_box* boxes, int nbox,
                               const gbem_mesh_params* params, double eps_r, size_t* bytes_needed)
{
    if (!S || !boxes || !params || !(eps_r > 0)) return GBEM_ERR_ARG;
    Request req;
    req.id = id;
    req.eps_r = eps_r;
    std::string err;
    gbem_status st = mesh_build_boxes(boxes, nbox, params, req.axis, req.geo, req.cond, err);
    if (st != GBEM_OK) {
        std::lock_guard<std::mutex> lk(S->mu);
        S->err = err;
        return st;
    }
    mesh_order(req.axis, req.geo, req.cond);
    std::vector<int32_t> ids(req.cond);
    std::sort(ids.begin(), ids.end());
    const int nc = (int)(std::unique(ids.begin(), ids.end()) - ids.begin());
    req.bytes = request_bytes((int)req.axis.size(), nc, S->prec);
    if (bytes_needed) *bytes_needed = req.bytes;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        req.t_submit = S->now();
        S->queue.push_back(std::move(req));
    }
    S->cv_work.notify_all();
    return GBEM_OK;
}

gbem_status gbem_server_poll(gbem_server_t* S, gbem_result_info* infos, double* C, long long c_capacity,
                             int max_results, int* count, int wait_ms)
{
    if (!S || !infos || !count || max_results <= 0) return GBEM_ERR_ARG;
    *count = 0;
    std::unique_lock<std::mutex> lk(S->mu);
    if (S->done.empty() && wait_ms > 0)
        S->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), [S] { return !S->done.empty(); });
    long long used = 0;
    while (!S->done.empty() && *count < max_results) {
        Result& r = S->done.front();
        const long long need = (long long)r.C.size();
        if (C && used + need > c_capacity) break;
        r.info.c_offset = used;
        if (C && need) std::memcpy(C + used, r.C.data(), sizeof(double) * need);
        used += need;
        infos[(*count)++] = r.info;
        S->done.pop_front();
    }
    return GBEM_OK;
}

gbem_status gbem_server_stats(gbem_server_t* S, int* queued, int* running, size_t* reserved, size_t* peak)
{
    if (!S) return GBEM_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    if (queued) *queued = (int)S->queue.size();
    if (running) *running = S->running;
    if (reserved) *reserved = S->reserved;
    if (peak) *peak = (size_t)S->peak_reserved;
    return GBEM_OK;
}

void gbem_server_destroy(gbem_server_t* S)
{
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    for (auto& t : S->workers) t.join();
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(S->device);
    for (auto* c : S->ctxs) gbem_destroy(c);
    for (auto s : S->streams) cudaStreamDestroy(s);
    if (prev >= 0) cudaSetDevice(prev);
    delete S;
}

}  // extern "C"
