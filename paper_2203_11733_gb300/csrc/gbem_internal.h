// Internal declarations shared by the translation units of libgbem.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <string>
#include <vector>

#include "gbem.h"

// Matrices are padded to a multiple of this with the identity.
constexpr int GBEM_PAD = 128;
// Assembly tile edge (panels).
constexpr int GBEM_TILE = 32;
// Largest Gauss-Legendre order used by the far-field rule.
constexpr int GBEM_GL_MAX = 6;

// Kernel-level tracing (gbem_set_timing level 2).  The entry points install
// their context's trace for the calling thread (TraceScope); launchers wrap
// their main kernels in trace_begin / trace_end, which do nothing when no
// trace is installed.
struct KernelTrace {
    struct Rec {
        int kind;
        cudaEvent_t a, b;
        double bytes, flops;
    };
    std::vector<Rec> recs;
    double ms[GBEM_NKERNEL] = {};
    double bytes[GBEM_NKERNEL] = {};
    double flops[GBEM_NKERNEL] = {};
    long long launches[GBEM_NKERNEL] = {};
};
extern thread_local KernelTrace* g_trace;
cudaEvent_t trace_begin(cudaStream_t s);
void trace_end(int kind, cudaEvent_t a, cudaStream_t s, double bytes, double flops);

// A second stream of the FP32 factorisation, owned by the matrix: the
// trailing updates beyond each panel run on it beside the panel's steps,
// ordered by the two events.  With no stream they run on the main stream.
struct SideStream {
    cudaStream_t stream = nullptr;
    cudaEvent_t ready = nullptr, done = nullptr;
};

struct gbem_ctx_s {
    int device = -1;
    int num_sms = 0;
    size_t budget = 0;
    size_t in_use = 0;
    gbem_alloc_fn alloc = nullptr;
    gbem_free_fn free_fn = nullptr;
    void* user = nullptr;
    std::string err;
    gbem_tuning tune{};
    bool gl_uploaded = false;
    // tracing
    bool timing = false;
    bool ktiming = false;
    KernelTrace ktrace;
    struct Pending {
        int phase;
        cudaEvent_t a, b;
    };
    std::vector<Pending> pending;
    double ms[GBEM_NPHASE] = {};
    long long calls[GBEM_NPHASE] = {};
    // buffers of the last destroyed matrix (idle: its stream was synchronised
    // before they came here), offered to the next matrix's allocations of the
    // same size so that repeated extractions of one size make no allocator
    // calls; still counted in in_use.  Dropped at the next matrix destroy,
    // under budget pressure, when the allocator refuses, and with the context.
    struct Spare {
        void* p;
        size_t bytes;
        cudaStream_t stream;   // where the buffer was last used
    };
    std::vector<Spare> spare;
    bool keep_spare = true;
    // side streams of destroyed matrices (idle), for the next matrices' factors
    std::vector<SideStream> side_pool;
    // mixed factors run their rest updates on a second stream; off, they run
    // on the caller's stream (the server's workers, already concurrent)
    bool side_stream = true;
};

// Kernels launched by the library in this process.
extern std::atomic<long long> g_gbem_launches;
inline void count_launch(long long k = 1) { g_gbem_launches.fetch_add(k, std::memory_order_relaxed); }

// Device view of a mesh: structure of arrays, one entry per panel.
struct DevPanels {
    const double* c = nullptr;    // plane coordinate
    const double* lo0 = nullptr;  // extents on the first in-plane axis
    const double* hi0 = nullptr;
    const double* lo1 = nullptr;  // extents on the second in-plane axis
    const double* hi1 = nullptr;
    const int8_t* axis = nullptr; // normal axis
    const double* tri = nullptr;  // triangle meshes: 9 per panel (vertices), else null
    const int32_t* cond = nullptr;// conductor index 0..n_c-1
    int n = 0;
};

// Device view of a batch of independent structures (pooled buffers; every
// per-structure array has nb entries, prefix arrays nb + 1).
struct BatchView {
    int nb = 0;
    const int* n = nullptr;           // panels
    const int* np = nullptr;          // padded order (multiple of 128)
    const int* nc = nullptr;          // conductors
    const long long* poff = nullptr;  // panel offset in the panel pools
    const long long* moff = nullptr;  // matrix offset (elements) in A64 / A32
    const long long* voff = nullptr;  // vector offset (elements) in B, X, R, W, Y (np x nc)
    const long long* ioff = nullptr;  // inverse-block offset (elements) in Linv (np/64 * 4096)
    const long long* coff = nullptr;  // capacitance offset (nc x nc) in C
    const long long* tile_prefix = nullptr;   // assembly tiles
    const long long* rows_prefix = nullptr;   // 16-row blocks (residual)
    const double *c = nullptr, *lo0 = nullptr, *hi0 = nullptr, *lo1 = nullptr, *hi1 = nullptr;
    const int8_t* axis = nullptr;
    const int32_t* cond = nullptr;
    double* A64 = nullptr;            // float pairs (hi, lo) per entry: batches are mixed
    float* A32 = nullptr;
    float* Linv = nullptr;
    double *B = nullptr, *X = nullptr, *R = nullptr;
    float *W = nullptr, *Y = nullptr;
    float2* Xdf = nullptr;            // X as float pairs for the compensated residual
    int* flags = nullptr;             // 4 per structure: [0] not SPD, [3] wait timeout
    double* C = nullptr;
    double* resid = nullptr;          // per structure: final relative residual
};

// Structure owning global index x given prefix sums p[0..nb] (p[0] = 0).
__host__ __device__ inline int batch_find(const long long* p, int nb, long long x)
{
    int lo = 0, hi = nb - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (p[mid] <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

struct gbem_mesh_s {
    gbem_ctx* ctx = nullptr;
    int n = 0;
    int n_cond = 0;
    std::vector<int8_t> axis;
    std::vector<double> geo;        // 5 per panel
    std::vector<int32_t> cond;      // conductor index (0..n_c-1)
    std::vector<int32_t> cond_ids;  // conductor index -> caller's id
    std::vector<double> tri;        // flat triangles: 9 per panel (empty for rectangles)
    void* dbuf = nullptr;
    size_t dbytes = 0;
    DevPanels dev;
};


struct gbem_matrix_s {
    gbem_ctx* ctx = nullptr;
    gbem_mesh_t* mesh = nullptr;
    int n = 0;
    int np = 0;                 // padded order
    int nb = 64;                // factor block
    gbem_precision prec = GBEM_FP64;
    double* A64 = nullptr;      // np x np col-major, lower triangle: FP64 entries, or in
                                // mixed mode float pairs (hi, lo) with hi + lo the FP64 entry
    float* A32 = nullptr;       // mixed: FP32 copy, factored in place
    double* L64 = nullptr;      // FP64 mode: the factor
    void* Linv = nullptr;       // inverses of the diagonal blocks (T)
    unsigned char* split = nullptr;  // mixed: hi/lo copies of one panel for the tensor-core update
    int* dflags = nullptr;      // [0] not-SPD pivot, [1] IR done, [2] IR iters, [3] wait timeout
    unsigned* dsync = nullptr;  // one flag per 64-row block for the persistent solves
    unsigned long long* dcounts = nullptr; // pair class counts (8)
    double* dnorm = nullptr;    // IR: [0] residual, [1..] scratch
    unsigned long long* dchk = nullptr;   // IR test folded into the residual: 2 cap_rhs + 1 words
    // solve work buffers (np x cap_rhs)
    int cap_rhs = 0;
    double* X = nullptr;
    double* R = nullptr;
    double* B = nullptr;
    void* W = nullptr;          // T: triangular-solve work
    bool factored = false;
    SideStream side;               // mixed factor: the stream of its rest updates (created at first use)
    cudaStream_t last = nullptr;   // the stream of the last call (null: the default stream)
    bool used = false;             // `last` holds a stream that work was enqueued on
    std::vector<std::pair<void*, size_t>> allocs;
};

// ---- context helpers (api.cpp)
struct TraceScope {
    KernelTrace* prev;
    explicit TraceScope(gbem_ctx* ctx);
    ~TraceScope();
};
gbem_status ctx_fail(gbem_ctx* ctx, gbem_status st, const std::string& msg);
void* ctx_alloc(gbem_ctx* ctx, size_t bytes, cudaStream_t s);
void ctx_free(gbem_ctx* ctx, void* p, size_t bytes, cudaStream_t s);
void ctx_drop_spare(gbem_ctx* ctx);

// ---- mesher (mesh.cpp)
gbem_status mesh_build_boxes(const gbem_box* boxes, int nbox, const gbem_mesh_params* p,
                             std::vector<int8_t>& axis, std::vector<double>& geo,
                             std::vector<int32_t>& cond_raw, std::string& err);
gbem_status mesh_build_graded(const gbem_box* boxes, int nbox, const gbem_partition_params* p,
                              std::vector<int8_t>& axis, std::vector<double>& geo, std::vector<int32_t>& cond_raw,
                              std::string& err);
void mesh_order(std::vector<int8_t>& axis, std::vector<double>& geo, std::vector<int32_t>& cond);
// Error-driven refinement of a panel list (gbem_mesh_refine): eta receives
// the indicator per input panel, n_marked the number of bisected panels.
gbem_status mesh_refine(const std::vector<int8_t>& axis, const std::vector<double>& geo,
                        const std::vector<int32_t>& cond, const double* density, double theta,
                        std::vector<int8_t>& axis_out, std::vector<double>& geo_out,
                        std::vector<int32_t>& cond_out, std::vector<double>& eta, int& n_marked);
void mesh_divide(double lo, double hi, const gbem_mesh_params* p, std::vector<double>& nodes);

// ---- kernels (assemble.cu, factor.cu, solve.cu)
cudaError_t gl_upload();
// Gauss-Legendre nodes and weights of order n on [-1, 1] (host).
void gl_nodes(int n, double* x, double* w);
// Every lower entry, tiles in band order.  Mixed mode writes the float pairs
// and the FP32 copy.  counts (8 words, zeroed) receives the pairs of each
// class; the traced work counts the quadrature evaluations and corner terms.
cudaError_t launch_assemble(const DevPanels& g, int np, gbem_precision prec, double q_near,
                            double* A64, float* A32, unsigned long long* counts, cudaStream_t s);
cudaError_t launch_pad(double* A64, float* A32, int n, int np, cudaStream_t s);
// Every lower entry of a mesh of flat triangles (tri: 9 per panel), FP64,
// stored as for rectangles (float pairs and the FP32 copy in mixed mode);
// counts (zeroed) receives the pairs of each class: self, touching, near,
// far of order 3..6.
cudaError_t launch_assemble_tri(const double* tri, int n, int np, gbem_precision prec, double* A64, float* A32,
                                unsigned long long* counts, cudaStream_t s);
cudaError_t launch_assemble_batched(const BatchView& v, long long tiles, gbem_precision prec, double q_near,
                                    cudaStream_t s);
cudaError_t launch_cholesky_batched(const BatchView& v, int nsteps, const long long* steps_dev,
                                    const long long* steps_host, cudaStream_t s);
// Batched solve: begin (right-hand sides, X = 0, R = B), then per refinement
// iteration W = f32(R), W = A32^-1 W, X += W, R = B - A64 X; finish writes the
// residual and the capacitance matrix of every structure.
cudaError_t launch_batch_begin(const BatchView& v, cudaStream_t s);
cudaError_t launch_batch_iteration(const BatchView& v, size_t vec_total, long long row_blocks, int max_nc,
                                   cudaStream_t s);
cudaError_t launch_batch_finish(const BatchView& v, double scale, cudaStream_t s);
cudaError_t launch_copy_lower(const double* A, double* L, int np, cudaStream_t s);
cudaError_t launch_cholesky_f64(double* L, int np, int nb, double* Linv, int* info, cudaStream_t s);
// The FP32 factor's tensor-core update needs `split` work space of
// cholesky_f32_split_bytes(np) bytes (the hi/lo copies of one panel).
size_t cholesky_f32_split_bytes(int np);
cudaError_t launch_cholesky_f32(float* L, int np, int nb, float* Linv, int* info, unsigned char* split,
                                cudaStream_t s, const SideStream* side);
// One CTA waits, through the factorisation's bounded release-flag wait, for
// flag[0] to reach 1 (limit limit_ms); status receives GBEM_ERR_TIMEOUT if
// it gives up.
cudaError_t launch_wait_selftest(const unsigned* flag, int* status, double limit_ms, cudaStream_t s);
// W (np x nrhs, followed by np x nrhs of work space) := A^-1 W with the
// factor L and its diagonal-block inverses; sync: np/64 flags, status: word
// that receives GBEM_ERR_TIMEOUT if a bounded device wait gives up.
cudaError_t launch_trsv_f64(const double* L, const double* Linv, int np, int nb, double* W, int nrhs,
                            unsigned* sync, int* status, cudaStream_t s);
cudaError_t launch_pack_rhs(const double* B, int ldb, int n, int np, int nrhs, double* Bp,
                            cudaStream_t s);
cudaError_t launch_unpack(const double* Xp, int np, int n, int nrhs, double* X, int ldx,
                          cudaStream_t s);
cudaError_t launch_ir_begin(const double* Bp, int np, int nrhs, double* X, double* R, double* norm,
                            int* flags, cudaStream_t s);
cudaError_t launch_to_f32(const double* R, int np, int nrhs, float* W, const int* done,
                          cudaStream_t s);
// X += W; with Xdf, also X as float pairs for launch_residual_df.
cudaError_t launch_add_f32(const float* W, int np, int nrhs, double* X, float2* Xdf, const int* done,
                           cudaStream_t s);
// FP32: W (np x nrhs) is followed by 3 x np x nrhs floats of work space (the
// forward result, then 64-bit epoch-tagged words through which the CTAs of a
// sweep exchange solved blocks); sync is unused.  Skipped once *done is set.
cudaError_t launch_trsv_f32_guarded(const float* L, const float* Linv, int np, int nb, float* W,
                                    int nrhs, unsigned* sync, int* status, const int* done, cudaStream_t s);
cudaError_t launch_residual(const double* A, int np, const double* Bp, const double* X, int nrhs,
                            double* R, const int* done, cudaStream_t s);
// R = B - A X with A and X stored as float pairs (mixed mode's FP64 storage),
// in compensated FP32 arithmetic.  With chk (2 nrhs + 1 zeroed words), the
// refinement test of launch_ir_check is folded in: norm[0] = max over columns
// of max|R| / max|B|, flags[2] += 1, flags[1] = 1 if that is at most tol.
cudaError_t launch_residual_df(const float2* A, int np, const double* Bp, const float2* Xdf, int nrhs,
                               double* R, const int* done, cudaStream_t s, unsigned long long* chk = nullptr,
                               double* norm = nullptr, double tol = 0.0, int* flags = nullptr);
cudaError_t launch_ir_check(const double* R, const double* Bp, int np, int nrhs, double* norm,
                            double tol, int* flags, cudaStream_t s);
cudaError_t launch_indicator_rhs(const int32_t* cond, int n, int np, int n_cond, double* Bp,
                                 cudaStream_t s);
cudaError_t launch_capacitance(const int32_t* cond, int n, int np, int n_cond, const double* X,
                               double scale, double* C, cudaStream_t s);

// ---- multi-dielectric system (stack.cpp, dielectric.cu)
// Device view of a layered stack's system.  Panels as DevPanels; rows of
// region a are reg_off[a] .. reg_off[a+1]-1, row r belongs to panel
// row_panel[r]; ucol / qcol: the column of the panel's unknown u / q (-1:
// known); bcol: the right-hand side of a panel held at a conductor's
// potential (-1: none); cidx: the conductor index of a conductor or
// electrode panel (-1: none).  Matrices np x np column-major: M0 the
// assembled system (FP64), factored in place as M (FP64 mode) or M32 (mixed
// mode); B, X, R: np x nc FP64; W, Y: np x nc in the factor's type.
struct StackView {
    int n = 0, n_eq = 0, np = 0, nc = 0, R_layers = 0;
    const double *c = nullptr, *lo0 = nullptr, *hi0 = nullptr, *lo1 = nullptr, *hi1 = nullptr;
    const int8_t *axis = nullptr, *sign = nullptr;
    const int32_t *ra = nullptr, *ucol = nullptr, *qcol = nullptr, *bcol = nullptr, *cidx = nullptr;
    const int32_t *row_panel = nullptr, *reg_off = nullptr;
    const long long* tile_off = nullptr;
    const double* eps = nullptr;
    double *M0 = nullptr, *M = nullptr;
    float* M32 = nullptr;
    double *B = nullptr, *X = nullptr, *R = nullptr, *P = nullptr, *C = nullptr;
    void* W = nullptr;
    void* Y = nullptr;      // np x nc, the forward sweep's result (factor's type)
    void* Inv = nullptr;    // np/64 x 2 inverses of the factor's 64 x 64 diagonal blocks
    int *ipiv = nullptr, *perm = nullptr, *status = nullptr;
    int* plan = nullptr;    // 1 + 4 * 64 ints: one panel's row moves
    unsigned long long* norms = nullptr;
};
cudaError_t stack_gl_upload(cudaStream_t s);
// M0 and B from the geometry (entries FP64, or FP32 far field in mixed
// mode), then the copy to factor (M, or M32 in mixed mode).
cudaError_t launch_stack_assemble(const StackView& v, long long tiles, bool mixed, cudaStream_t s);
// LU with partial pivoting of M (M32), ipiv, and perm from ipiv.  In mixed
// mode with a side stream (and two events) each panel after the first runs
// there beside the previous panel's trailing update.
cudaError_t launch_stack_lu(const StackView& v, bool mixed, cudaStream_t s, cudaStream_t side, cudaEvent_t ready,
                            cudaEvent_t done);
// One correction: W = (LU)^-1 P R in the factor's type, X += W.
cudaError_t launch_stack_correct(const StackView& v, bool mixed, cudaStream_t s);
// R = B - M0 X in FP64; norms[m] = max_r |R[r, m]|, norms[nc + m] = max_r
// |B[r, m]| (bit patterns of non-negative doubles).
cudaError_t launch_stack_residual(const StackView& v, cudaStream_t s);
size_t stack_partial_bytes(int np, int nc);
// C (nc x nc) from X.
cudaError_t launch_stack_charges(const StackView& v, double eps0, cudaStream_t s);
