// gbem_solve_noalloc: the solve of gbem_solve with every scratch buffer taken
// from one fixed, file-scope device array instead of the context's allocator.
//
// Who needs it: callers that cannot allocate device memory at solve time.  A
// serving worker that reserved its whole HBM budget at start-up and must not
// grow it per request; an application whose memory is owned by its own arena
// or pool manager and forbids libraries from calling cudaMalloc; code that
// must not risk the implicit device synchronisation that cudaMalloc/cudaFree
// can cause in the middle of a latency-critical loop.  gbem_solve allocates
// its work buffers on first use of a matrix; this variant never does.
//
// The array costs GBEM_NOALLOC_SCRATCH_BYTES of device memory on every GPU
// that loads the library, held until the process exits.  All calls share it
// and it keeps the contents of the last call, so everything a call reads is
// first written by that call (padded right-hand sides, solution, residual,
// flags).  Calls that overlap on the GPU (different streams, or different
// host threads) race on the array and must be serialised by the caller.
#include <algorithm>
#include <mutex>

#include "gbem_internal.h"

namespace {

constexpr size_t kScratchBytes = GBEM_NOALLOC_SCRATCH_BYTES;

// The scratch itself.  Host code must not use this symbol as a pointer: on the
// host it names a stand-in, not the device address.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch on `device` (current), looked up once.
cudaError_t scratch_address(int device, unsigned char** out)
{
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_ptr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[device] = p;
    }
    *out = static_cast<unsigned char*>(g_scratch_ptr[device]);
    return cudaSuccess;
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

extern "C" gbem_status gbem_solve_noalloc(gbem_matrix_t* m, const double* B_dev, int nrhs, int ldb,
                                          double* X_dev, int ldx, int* ir_iters, gbem_stream stream)
{
    if (!m || !B_dev || !X_dev || nrhs <= 0) return GBEM_ERR_ARG;
    gbem_ctx* ctx = m->ctx;
    if (ldb < m->n || ldx < m->n) return ctx_fail(ctx, GBEM_ERR_ARG, "leading dimension below N");
    if (!m->factored) return ctx_fail(ctx, GBEM_ERR_STATE, "solve before factor");
    const size_t np = (size_t)m->np;
    const size_t vec = align256(np * nrhs * sizeof(double));
    const size_t nblk = np / 64;
    const size_t need = 5 * vec + 256 + align256(nblk * sizeof(unsigned));   // B, X, R, W (two halves),
                                                                             // flags and norm, block flags
    if (need > kScratchBytes)
        return ctx_fail(ctx, GBEM_ERR_ARG,
                        "gbem_solve_noalloc: needs " + std::to_string(need) + " bytes of scratch (padded N " +
                            std::to_string(np) + " x " + std::to_string(nrhs) + " right-hand sides), limit " +
                            std::to_string(kScratchBytes));
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return ctx_fail(ctx, GBEM_ERR_CUDA, "cudaGetDevice failed");
    if (prev != ctx->device && cudaSetDevice(ctx->device) != cudaSuccess)
        return ctx_fail(ctx, GBEM_ERR_CUDA, "cudaSetDevice failed");
    struct Restore {
        int dev;
        ~Restore()
        {
            if (dev >= 0) cudaSetDevice(dev);
        }
    } restore{prev != ctx->device ? prev : -1};

    unsigned char* base = nullptr;
    cudaError_t e = scratch_address(ctx->device, &base);
    if (e != cudaSuccess) return ctx_fail(ctx, GBEM_ERR_CUDA, std::string("scratch set-up: ") + cudaGetErrorString(e));
    double* Bp = reinterpret_cast<double*>(base);
    double* X = reinterpret_cast<double*>(base + vec);
    double* R = reinterpret_cast<double*>(base + 2 * vec);
    void* W = base + 3 * vec;                       // 2 np nrhs entries of the solve type
    int* flags = reinterpret_cast<int*>(base + 5 * vec);
    double* norm = reinterpret_cast<double*>(base + 5 * vec + 64);
    // block flags of the FP64 persistent solves: compared against a fresh
    // epoch on every sweep; cleared below so that no leftover word of an
    // earlier call (right-hand sides, solutions) can equal a later epoch
    unsigned* sync = reinterpret_cast<unsigned*>(base + 5 * vec + 256);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int n = m->n, npi = m->np;

    auto fail = [&](cudaError_t err, const char* what) {
        return ctx_fail(ctx, GBEM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(err));
    };
    if ((e = cudaMemsetAsync(flags, 0, 64, s)) != cudaSuccess) return fail(e, "clear flags");
    if ((e = cudaMemsetAsync(sync, 0, nblk * sizeof(unsigned), s)) != cudaSuccess) return fail(e, "clear sync");
    if ((e = launch_pack_rhs(B_dev, ldb, n, npi, nrhs, Bp, s)) != cudaSuccess) return fail(e, "pack");
    int iters = 0;
    if (m->prec == GBEM_FP64) {
        double* Wd = static_cast<double*>(W);
        if ((e = cudaMemcpyAsync(Wd, Bp, sizeof(double) * np * nrhs, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
            return fail(e, "copy");
        if ((e = launch_trsv_f64(m->L64, static_cast<const double*>(m->Linv), npi, m->nb, Wd, nrhs, sync,
                                 flags + 3, s)) != cudaSuccess)
            return fail(e, "trsv");
        if ((e = launch_unpack(Wd, npi, n, nrhs, X_dev, ldx, s)) != cudaSuccess) return fail(e, "unpack");
    } else {
        float* Wf = static_cast<float*>(W);                       // W and its work half: the first vec
        float2* Xdf = reinterpret_cast<float2*>(base + 4 * vec);  // X as float pairs: the second vec
        const int* done = flags + 1;
        if ((e = launch_ir_begin(Bp, npi, nrhs, X, R, norm, flags, s)) != cudaSuccess) return fail(e, "ir begin");
        int host_flags[3] = {0, 0, 0};
        const int maxit = std::max(1, ctx->tune.ir_max_iter);   // as gbem_solve
        for (int it = 0; it < maxit && !host_flags[1]; ++it) {
            if ((e = launch_to_f32(R, npi, nrhs, Wf, done, s)) != cudaSuccess ||
                (e = launch_trsv_f32_guarded(m->A32, static_cast<const float*>(m->Linv), npi, m->nb, Wf, nrhs,
                                             sync, flags + 3, done, s)) != cudaSuccess ||
                (e = launch_add_f32(Wf, npi, nrhs, X, Xdf, done, s)) != cudaSuccess ||
                (e = launch_residual_df(reinterpret_cast<const float2*>(m->A64), npi, Bp, Xdf, nrhs, R, done, s)) !=
                    cudaSuccess ||
                (e = launch_ir_check(R, Bp, npi, nrhs, norm, ctx->tune.ir_tol, flags, s)) != cudaSuccess)
                return fail(e, "refinement");
            if ((e = cudaMemcpyAsync(host_flags, flags, sizeof(host_flags), cudaMemcpyDeviceToHost, s)) !=
                    cudaSuccess ||
                (e = cudaStreamSynchronize(s)) != cudaSuccess)
                return fail(e, "flags");
        }
        if ((e = launch_unpack(X, npi, n, nrhs, X_dev, ldx, s)) != cudaSuccess) return fail(e, "unpack");
    }
    // every path ends here: the status words live in the shared scratch, so
    // read them (and let X_dev be written) before returning
    int fl[4] = {0, 0, 0, 0};
    if ((e = cudaMemcpyAsync(fl, flags, sizeof(fl), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return fail(e, "sync");
    if (m->prec != GBEM_FP64) iters = fl[2];
    if (ir_iters) *ir_iters = iters;
    if (fl[3]) return ctx_fail(ctx, GBEM_ERR_TIMEOUT, "gbem_solve_noalloc: a bounded device wait gave up");
    if (m->prec != GBEM_FP64 && !fl[1])
        return ctx_fail(ctx, GBEM_ERR_NOCONV, "gbem_solve_noalloc: refinement missed its tolerance");
    return GBEM_OK;
}
