// Blocked right-looking Cholesky factorisation A = L L^T of the Galerkin
// matrix, which is symmetric positive definite (Wu & Li, Sec. 3.2, Theorem 1:
// the single-layer operator is elliptic, hence Cholesky).
//
// The matrix is np x np column-major (np a multiple of the block size nb = 64,
// padding rows carry the identity), lower triangle significant.  For each
// block column k:
//   1. potrf_diag:  L_kk = chol(A_kk) in shared memory, and Linv_kk = L_kk^-1
//                   (kept for the triangular solves);
//   2. trsm_panel:  L_ik = A_ik Linv_kk^T for the blocks below;
//   3. syrk_update: A_ij -= L_ik L_jk^T on the lower tiles of the trailing
//                   matrix.
// T is the storage and arithmetic type: double in FP64 mode, float in mixed
// mode (whose FP64 refinement restores the solution's accuracy).  A
// non-positive pivot sets info[0] = 1 and is replaced by 1 so that the
// factorisation completes without NaNs; the host reports GBEM_ERR_NOT_SPD.
#include "gbem_internal.h"

namespace {

constexpr int NB = 64;

template <typename T>
__global__ void __launch_bounds__(256) potrf_diag(T* __restrict__ L, int ld, int k0,
                                                  T* __restrict__ Linv, int* __restrict__ info)
{
    extern __shared__ unsigned char smem_raw[];
    T(*a)[NB + 1] = reinterpret_cast<T(*)[NB + 1]>(smem_raw);
    T(*inv)[NB + 1] = a + NB;
    const int tid = threadIdx.x;
    for (int e = tid; e < NB * NB; e += blockDim.x) {
        int r = e % NB, c = e / NB;
        a[r][c] = (r >= c) ? L[(size_t)(k0 + r) + (size_t)(k0 + c) * ld] : T(0);
    }
    __syncthreads();
    for (int j = 0; j < NB; ++j) {
        if (tid == 0) {
            T d = a[j][j];
            if (!(d > T(0))) {
                info[0] = 1;
                d = T(1);
            }
            a[j][j] = sqrt(d);
        }
        __syncthreads();
        T djj = a[j][j];
        for (int r = j + 1 + tid; r < NB; r += blockDim.x) a[r][j] /= djj;
        __syncthreads();
        // rank-1 update of the trailing lower triangle
        const int m = NB - 1 - j;
        for (int e = tid; e < m * m; e += blockDim.x) {
            int r = j + 1 + e % m, c = j + 1 + e / m;
            if (r >= c) a[r][c] -= a[r][j] * a[c][j];
        }
        __syncthreads();
    }
    // inverse of the lower-triangular factor, one column per thread
    if (tid < NB) {
        const int c = tid;
        for (int r = 0; r < c; ++r) inv[r][c] = T(0);
        inv[c][c] = T(1) / a[c][c];
        for (int r = c + 1; r < NB; ++r) {
            T s = T(0);
            for (int k = c; k < r; ++k) s += a[r][k] * inv[k][c];
            inv[r][c] = -s / a[r][r];
        }
    }
    __syncthreads();
    T* Lb = Linv + (size_t)(k0 / NB) * NB * NB;
    for (int e = tid; e < NB * NB; e += blockDim.x) {
        int r = e % NB, c = e / NB;
        if (r >= c) L[(size_t)(k0 + r) + (size_t)(k0 + c) * ld] = a[r][c];
        Lb[e] = inv[r][c];
    }
}

// L_ik = A_ik Linv_kk^T for the row block starting at k0 + NB * (1 + blockIdx.x)
template <typename T>
__global__ void __launch_bounds__(256) trsm_panel(T* __restrict__ L, int ld, int k0,
                                                  const T* __restrict__ Linv)
{
    extern __shared__ unsigned char smem_raw[];
    T(*a)[NB + 1] = reinterpret_cast<T(*)[NB + 1]>(smem_raw);
    T(*iv)[NB + 1] = a + NB;
    const int tid = threadIdx.x;
    const int r0 = k0 + NB * (1 + blockIdx.x);
    const T* Lb = Linv + (size_t)(k0 / NB) * NB * NB;
    for (int e = tid; e < NB * NB; e += blockDim.x) {
        int r = e % NB, c = e / NB;
        a[r][c] = L[(size_t)(r0 + r) + (size_t)(k0 + c) * ld];
        iv[r][c] = Lb[e];
    }
    __syncthreads();
    // out[r][c] = sum_{t <= c} a[r][t] * iv[c][t]; 4x4 outputs per thread
    const int tr = (tid % 16) * 4, tc = (tid / 16) * 4;
    T acc[4][4] = {};
    for (int t = 0; t < NB; ++t) {
        T x[4], y[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            x[u] = a[tr + u][t];
            y[u] = iv[tc + u][t];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] += x[u] * y[v];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) L[(size_t)(r0 + tr + u) + (size_t)(k0 + tc + v) * ld] = acc[u][v];
}

// A_IJ -= L_Ik L_Jk^T for the lower tiles (I >= J) of the trailing matrix.
template <typename T>
__global__ void __launch_bounds__(256) syrk_update(T* __restrict__ L, int ld, int k0)
{
    extern __shared__ unsigned char smem_raw[];
    T* sa = reinterpret_cast<T*>(smem_raw);   // [NB][NB+1]  rows of block I
    T* sb = sa + NB * (NB + 1);               // [NB][NB+1]  rows of block J
    long long b = blockIdx.x;
    int I = (int)((sqrt(8.0 * (double)b + 1.0) - 1.0) * 0.5);
    while ((long long)(I + 1) * (I + 2) / 2 <= b) ++I;
    while ((long long)I * (I + 1) / 2 > b) --I;
    int J = (int)(b - (long long)I * (I + 1) / 2);
    const int rI = k0 + NB * (1 + I), rJ = k0 + NB * (1 + J);
    const int tid = threadIdx.x;
    for (int e = tid; e < NB * NB; e += blockDim.x) {
        int r = e % NB, c = e / NB;
        sa[r * (NB + 1) + c] = L[(size_t)(rI + r) + (size_t)(k0 + c) * ld];
        sb[r * (NB + 1) + c] = L[(size_t)(rJ + r) + (size_t)(k0 + c) * ld];
    }
    __syncthreads();
    const int tr = (tid % 16) * 4, tc = (tid / 16) * 4;
    T acc[4][4] = {};
    for (int t = 0; t < NB; ++t) {
        T x[4], y[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            x[u] = sa[(tr + u) * (NB + 1) + t];
            y[u] = sb[(tc + u) * (NB + 1) + t];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] += x[u] * y[v];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            size_t idx = (size_t)(rI + tr + u) + (size_t)(rJ + tc + v) * ld;
            L[idx] -= acc[u][v];
        }
}

template <typename T>
cudaError_t cholesky(T* L, int np, T* Linv, int* info, cudaStream_t s)
{
    const int nblk = np / NB;
    const size_t smem = 2 * NB * (NB + 1) * sizeof(T);
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(potrf_diag<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(trsm_panel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(syrk_update<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem)) != cudaSuccess)
        return e;
    for (int k = 0; k < nblk; ++k) {
        const int k0 = k * NB;
        potrf_diag<T><<<1, 256, smem, s>>>(L, np, k0, Linv, info);
        count_launch();
        const int m = nblk - k - 1;
        if (m > 0) {
            trsm_panel<T><<<m, 256, smem, s>>>(L, np, k0, Linv);
            count_launch();
            long long tiles = (long long)m * (m + 1) / 2;
            syrk_update<T><<<(unsigned)tiles, 256, smem, s>>>(L, np, k0);
            count_launch();
        }
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_cholesky_f64(double* L, int np, int nb, double* Linv, int* info, cudaStream_t s)
{
    if (nb != NB || np % NB) return cudaErrorInvalidValue;
    return cholesky<double>(L, np, Linv, info, s);
}

cudaError_t launch_cholesky_f32(float* L, int np, int nb, float* Linv, int* info, cudaStream_t s)
{
    if (nb != NB || np % NB) return cudaErrorInvalidValue;
    return cholesky<float>(L, np, Linv, info, s);
}
