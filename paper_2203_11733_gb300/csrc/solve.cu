// Solve A X = B with the Cholesky factor (Wu & Li, Sec. 3.1 Eq. "lineareq1"
// and Sec. 3.2), iterative refinement in FP64 for the mixed-precision factor,
// and the charge on each conductor (Eq. "electriccharge").
//
// Triangular solves are blocked by the factor's 64-wide diagonal blocks and
// use their stored inverses: the forward sweep takes, for k = 0..nblk-1,
//     Y_k = Linv_kk W_k,   W_i -= L_ik Y_k (i > k)
// and the backward sweep, for k = nblk-1..0,
//     X_k = Linv_kk^T Y_k, Y_i -= L_ki^T X_k (i < k).
// One launch per block step; every CTA recomputes the small diagonal product
// itself so that no CTA waits on another.
#include "gbem_internal.h"

namespace {

constexpr int NB = 64;
constexpr int MAXR = 16;   // right-hand sides per pass

// Forward step k: rows of block k and the rows below.
template <typename T>
__global__ void __launch_bounds__(256) trsv_fwd_step(const T* __restrict__ L, const T* __restrict__ Linv,
                                                     int np, int k, T* __restrict__ W,
                                                     T* __restrict__ Y, int nrhs, const int* done)
{
    if (done && *done) return;
    __shared__ T w[NB][MAXR];
    __shared__ T y[NB][MAXR];
    const int tid = threadIdx.x;
    const int k0 = k * NB;
    const T* Lb = Linv + (size_t)k * NB * NB;
    for (int r0 = 0; r0 < nrhs; r0 += MAXR) {
        const int nr = min(MAXR, nrhs - r0);
        for (int e = tid; e < NB * nr; e += blockDim.x) {
            int r = e % NB, c = e / NB;
            w[r][c] = W[(size_t)(k0 + r) + (size_t)(r0 + c) * np];
        }
        __syncthreads();
        for (int e = tid; e < NB * nr; e += blockDim.x) {
            int r = e % NB, c = e / NB;
            T s = T(0);
            for (int t = 0; t <= r; ++t) s += Lb[r + (size_t)t * NB] * w[t][c];
            y[r][c] = s;
        }
        __syncthreads();
        if (blockIdx.x == 0)
            for (int e = tid; e < NB * nr; e += blockDim.x) {
                int r = e % NB, c = e / NB;
                Y[(size_t)(k0 + r) + (size_t)(r0 + c) * np] = y[r][c];
            }
        // rows below, one row per thread
        for (int row = k0 + NB + blockIdx.x * blockDim.x + tid; row < np;
             row += gridDim.x * blockDim.x) {
            T acc[MAXR];
#pragma unroll
            for (int c = 0; c < MAXR; ++c) acc[c] = T(0);
            for (int t = 0; t < NB; ++t) {
                T l = L[(size_t)row + (size_t)(k0 + t) * np];
#pragma unroll
                for (int c = 0; c < MAXR; ++c) acc[c] += l * y[t][c];
            }
            for (int c = 0; c < nr; ++c) W[(size_t)row + (size_t)(r0 + c) * np] -= acc[c];
        }
        __syncthreads();
    }
}

// Backward step k: X_k = Linv_kk^T Y_k written into W; rows above updated in Y.
template <typename T>
__global__ void __launch_bounds__(256) trsv_bwd_step(const T* __restrict__ L, const T* __restrict__ Linv,
                                                     int np, int k, T* __restrict__ Y,
                                                     T* __restrict__ W, int nrhs, const int* done)
{
    if (done && *done) return;
    __shared__ T yk[NB][MAXR];
    __shared__ T x[NB][MAXR];
    const int tid = threadIdx.x;
    const int k0 = k * NB;
    const T* Lb = Linv + (size_t)k * NB * NB;
    for (int r0 = 0; r0 < nrhs; r0 += MAXR) {
        const int nr = min(MAXR, nrhs - r0);
        for (int e = tid; e < NB * nr; e += blockDim.x) {
            int r = e % NB, c = e / NB;
            yk[r][c] = Y[(size_t)(k0 + r) + (size_t)(r0 + c) * np];
        }
        __syncthreads();
        for (int e = tid; e < NB * nr; e += blockDim.x) {
            int r = e % NB, c = e / NB;
            T s = T(0);
            for (int t = r; t < NB; ++t) s += Lb[t + (size_t)r * NB] * yk[t][c];
            x[r][c] = s;
        }
        __syncthreads();
        if (blockIdx.x == 0)
            for (int e = tid; e < NB * nr; e += blockDim.x) {
                int r = e % NB, c = e / NB;
                W[(size_t)(k0 + r) + (size_t)(r0 + c) * np] = x[r][c];
            }
        // rows above: Y_i -= (L_ki)^T X_k, i.e. for row `row` < k0:
        // sum_t L[k0 + t][row] * x[t]  (column `row` of L, rows k0..k0+63)
        for (int row = blockIdx.x * blockDim.x + tid; row < k0; row += gridDim.x * blockDim.x) {
            T acc[MAXR];
#pragma unroll
            for (int c = 0; c < MAXR; ++c) acc[c] = T(0);
            const T* col = L + (size_t)row * np + k0;
            for (int t = 0; t < NB; ++t) {
                T l = col[t];
#pragma unroll
                for (int c = 0; c < MAXR; ++c) acc[c] += l * x[t][c];
            }
            for (int c = 0; c < nr; ++c) Y[(size_t)row + (size_t)(r0 + c) * np] -= acc[c];
        }
        __syncthreads();
    }
}

template <typename T>
cudaError_t trsv(const T* L, const T* Linv, int np, T* W, T* Y, int nrhs, const int* done,
                 cudaStream_t s)
{
    const int nblk = np / NB;
    for (int k = 0; k < nblk; ++k) {
        int rows = np - (k + 1) * NB;
        int grid = max(1, min(1024, (rows + 255) / 256));
        trsv_fwd_step<T><<<grid, 256, 0, s>>>(L, Linv, np, k, W, Y, nrhs, done);
        count_launch();
    }
    for (int k = nblk - 1; k >= 0; --k) {
        int rows = k * NB;
        int grid = max(1, min(1024, (rows + 255) / 256));
        trsv_bwd_step<T><<<grid, 256, 0, s>>>(L, Linv, np, k, Y, W, nrhs, done);
        count_launch();
    }
    return cudaGetLastError();
}

__global__ void pack_rhs(const double* __restrict__ B, int ldb, int n, int np, int nrhs,
                         double* __restrict__ Bp)
{
    size_t total = (size_t)np * nrhs;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        int r = (int)(e % np), c = (int)(e / np);
        Bp[e] = (r < n) ? B[(size_t)r + (size_t)c * ldb] : 0.0;
    }
}

__global__ void unpack(const double* __restrict__ Xp, int np, int n, int nrhs, double* __restrict__ X,
                       int ldx)
{
    size_t total = (size_t)n * nrhs;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        int r = (int)(e % n), c = (int)(e / n);
        X[(size_t)r + (size_t)c * ldx] = Xp[(size_t)r + (size_t)c * np];
    }
}

__global__ void ir_begin(const double* __restrict__ Bp, int np, int nrhs, double* __restrict__ X,
                         double* __restrict__ R, double* norm, int* flags)
{
    size_t total = (size_t)np * nrhs;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        X[e] = 0.0;
        R[e] = Bp[e];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        flags[1] = 0;
        flags[2] = 0;
        norm[0] = 1.0;
    }
}

__global__ void to_f32(const double* __restrict__ R, size_t total, float* __restrict__ W,
                       const int* done)
{
    if (*done) return;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x)
        W[e] = (float)R[e];
}

__global__ void add_f32(const float* __restrict__ W, size_t total, double* __restrict__ X,
                        const int* done)
{
    if (*done) return;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x)
        X[e] += (double)W[e];
}

// R = B - A X with A symmetric, only its lower triangle stored.  CTA owns 32
// rows and walks every 32-column block in order (deterministic sums): lower
// blocks are read directly, blocks above the diagonal through the transpose.
constexpr int RT = 32;
__global__ void __launch_bounds__(256) residual(const double* __restrict__ A, int np,
                                                const double* __restrict__ Bp,
                                                const double* __restrict__ X, int nrhs,
                                                double* __restrict__ R, const int* done)
{
    if (done && *done) return;
    __shared__ double a[RT][RT + 1];
    __shared__ double xs[RT][MAXR];
    __shared__ double part[8][RT][MAXR];
    const int tid = threadIdx.x;
    const int i0 = blockIdx.x * RT;
    const int ri = tid % RT, grp = tid / RT;  // 8 column groups
    for (int c0 = 0; c0 < nrhs; c0 += MAXR) {
        const int nr = min(MAXR, nrhs - c0);
        double acc[MAXR];
#pragma unroll
        for (int c = 0; c < MAXR; ++c) acc[c] = 0.0;
        for (int j0 = 0; j0 < np; j0 += RT) {
            __syncthreads();
            // tile a[r][c] = A(i0 + r, j0 + c)
            for (int e = tid; e < RT * RT; e += blockDim.x) {
                int r = e % RT, c = e / RT;
                double v;
                if (j0 < i0) v = A[(size_t)(i0 + r) + (size_t)(j0 + c) * np];
                else if (j0 > i0) v = A[(size_t)(j0 + r) + (size_t)(i0 + c) * np];
                else v = A[(size_t)(i0 + max(r, c)) + (size_t)(i0 + min(r, c)) * np];
                if (j0 > i0) a[c][r] = v;
                else a[r][c] = v;
            }
            for (int e = tid; e < RT * nr; e += blockDim.x) {
                int r = e % RT, c = e / RT;
                xs[r][c] = X[(size_t)(j0 + r) + (size_t)(c0 + c) * np];
            }
            __syncthreads();
            for (int jj = grp; jj < RT; jj += 8) {
                double av = a[ri][jj];
#pragma unroll
                for (int c = 0; c < MAXR; ++c)
                    if (c < nr) acc[c] = fma(av, xs[jj][c], acc[c]);
            }
        }
#pragma unroll
        for (int c = 0; c < MAXR; ++c) part[grp][ri][c] = acc[c];
        __syncthreads();
        for (int e = tid; e < RT * nr; e += blockDim.x) {
            int r = e % RT, c = e / RT;
            double s = 0.0;
            for (int g = 0; g < 8; ++g) s += part[g][r][c];
            size_t idx = (size_t)(i0 + r) + (size_t)(c0 + c) * np;
            R[idx] = Bp[idx] - s;
        }
    }
}

// max_k |R_k|_inf / |B_k|_inf -> norm[0]; converged -> flags[1] = 1, else
// flags[2] += 1 (iterations taken).
__global__ void ir_check(const double* __restrict__ R, const double* __restrict__ Bp, int np,
                         int nrhs, double* norm, double tol, int* flags)
{
    __shared__ double red[256];
    if (flags[1]) return;
    double worst = 0.0;
    for (int c = 0; c < nrhs; ++c) {
        double mr = 0.0, mb = 0.0;
        for (int r = threadIdx.x; r < np; r += blockDim.x) {
            mr = fmax(mr, fabs(R[(size_t)r + (size_t)c * np]));
            mb = fmax(mb, fabs(Bp[(size_t)r + (size_t)c * np]));
        }
        red[threadIdx.x] = mr;
        __syncthreads();
        for (int s = 128; s > 0; s >>= 1) {
            if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
            __syncthreads();
        }
        mr = red[0];
        __syncthreads();
        red[threadIdx.x] = mb;
        __syncthreads();
        for (int s = 128; s > 0; s >>= 1) {
            if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
            __syncthreads();
        }
        mb = red[0];
        __syncthreads();
        double rel = (mb > 0.0) ? mr / mb : mr;
        worst = fmax(worst, rel);
    }
    if (threadIdx.x == 0) {
        norm[0] = worst;
        flags[2] += 1;
        if (worst <= tol) flags[1] = 1;
    }
}

__global__ void indicator_rhs(const int32_t* __restrict__ cond, int n, int np, int n_cond,
                              double* __restrict__ Bp)
{
    size_t total = (size_t)np * n_cond;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        int r = (int)(e % np), k = (int)(e / np);
        Bp[e] = (r < n && cond[r] == k) ? 1.0 : 0.0;
    }
}

// C[m][k] = scale * sum_{i : cond[i] == m} X[i][k]; one CTA per (m, k), a
// fixed-order reduction so the result does not depend on scheduling.
__global__ void capacitance(const int32_t* __restrict__ cond, int n, int np, int n_cond,
                            const double* __restrict__ X, double scale, double* __restrict__ C)
{
    __shared__ double red[256];
    const int m = blockIdx.x / n_cond, k = blockIdx.x % n_cond;
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        if (cond[i] == m) s += X[(size_t)i + (size_t)k * np];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) C[(size_t)m * n_cond + k] = scale * red[0];
}

static int grid_for(size_t total)
{
    size_t g = (total + 255) / 256;
    return (int)(g < 1 ? 1 : (g > 4096 ? 4096 : g));
}

}  // namespace

cudaError_t launch_trsv_f64(const double* L, const double* Linv, int np, int nb, double* W, int nrhs,
                            cudaStream_t s)
{
    if (nb != NB || nrhs <= 0) return cudaErrorInvalidValue;
    // Y shares the tail of W's allocation: W holds 2 * np * nrhs entries
    return trsv<double>(L, Linv, np, W, W + (size_t)np * nrhs, nrhs, nullptr, s);
}

cudaError_t launch_trsv_f32(const float* L, const float* Linv, int np, int nb, float* W, int nrhs,
                            cudaStream_t s)
{
    if (nb != NB || nrhs <= 0) return cudaErrorInvalidValue;
    return trsv<float>(L, Linv, np, W, W + (size_t)np * nrhs, nrhs, nullptr, s);
}

cudaError_t launch_trsv_f32_guarded(const float* L, const float* Linv, int np, int nb, float* W,
                                    int nrhs, const int* done, cudaStream_t s)
{
    if (nb != NB || nrhs <= 0) return cudaErrorInvalidValue;
    return trsv<float>(L, Linv, np, W, W + (size_t)np * nrhs, nrhs, done, s);
}

cudaError_t launch_pack_rhs(const double* B, int ldb, int n, int np, int nrhs, double* Bp,
                            cudaStream_t s)
{
    pack_rhs<<<grid_for((size_t)np * nrhs), 256, 0, s>>>(B, ldb, n, np, nrhs, Bp);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_unpack(const double* Xp, int np, int n, int nrhs, double* X, int ldx,
                          cudaStream_t s)
{
    unpack<<<grid_for((size_t)n * nrhs), 256, 0, s>>>(Xp, np, n, nrhs, X, ldx);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_ir_begin(const double* Bp, int np, int nrhs, double* X, double* R, double* norm,
                            int* flags, cudaStream_t s)
{
    ir_begin<<<grid_for((size_t)np * nrhs), 256, 0, s>>>(Bp, np, nrhs, X, R, norm, flags);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_to_f32(const double* R, int np, int nrhs, float* W, const int* done,
                          cudaStream_t s)
{
    size_t total = (size_t)np * nrhs;
    to_f32<<<grid_for(total), 256, 0, s>>>(R, total, W, done);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_add_f32(const float* W, int np, int nrhs, double* X, const int* done,
                           cudaStream_t s)
{
    size_t total = (size_t)np * nrhs;
    add_f32<<<grid_for(total), 256, 0, s>>>(W, total, X, done);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_residual(const double* A, int np, const double* Bp, const double* X, int nrhs,
                            double* R, const int* done, cudaStream_t s)
{
    if (np % RT) return cudaErrorInvalidValue;
    residual<<<np / RT, 256, 0, s>>>(A, np, Bp, X, nrhs, R, done);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_ir_check(const double* R, const double* Bp, int np, int nrhs, double* norm,
                            double tol, int* flags, cudaStream_t s)
{
    ir_check<<<1, 256, 0, s>>>(R, Bp, np, nrhs, norm, tol, flags);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_indicator_rhs(const int32_t* cond, int n, int np, int n_cond, double* Bp,
                                 cudaStream_t s)
{
    indicator_rhs<<<grid_for((size_t)np * n_cond), 256, 0, s>>>(cond, n, np, n_cond, Bp);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_capacitance(const int32_t* cond, int n, int np, int n_cond, const double* X,
                               double scale, double* C, cudaStream_t s)
{
    capacitance<<<n_cond * n_cond, 256, 0, s>>>(cond, n, np, n_cond, X, scale, C);
    count_launch();
    return cudaGetLastError();
}
