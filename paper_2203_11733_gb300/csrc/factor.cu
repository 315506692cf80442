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
#include "tc_syrk.cuh"

namespace {

constexpr int NB = 64;

// Cholesky of one 64x64 diagonal block fused with the inverse of its factor.
// Each of the 256 threads keeps a fixed 4x4 sub-block of the matrix A and of
// X = L^-1 (started as the identity) in registers.  Step j publishes, through
// double-buffered shared memory, the current column j of A (unscaled) and
// row j of X; then every thread
//   - subtracts a_rj a_cj / a_jj from its entries of A right of column j,
//   - finalises X_j = X_j / l_jj and subtracts l_ij X_j from its rows i > j
//     of X (l_ij = a_ij / sqrt(a_jj): forward elimination of the identity).
// One barrier per column.  Column j of L is a_.j / sqrt(a_jj) at the end.
// A non-positive pivot sets info[0] = 1 and is replaced by 1 so that the
// factorisation completes without NaNs.
template <typename T>
struct PotrfSmem {
    T col[2][NB];
    T rowx[2][NB];
    T piv[NB];
};

__device__ __forceinline__ float rsqrt_t(float d) { return rsqrtf(d); }
__device__ __forceinline__ double rsqrt_t(double d) { return 1.0 / sqrt(d); }

template <typename T>
__device__ __forceinline__ void potrf_body(T* __restrict__ L, int ld, int k0, T* __restrict__ Linv,
                                           int* __restrict__ info)
{
    extern __shared__ unsigned char smem_raw[];
    PotrfSmem<T>& S = *reinterpret_cast<PotrfSmem<T>*>(smem_raw);
    const int tid = threadIdx.x;
    const int r0 = (tid & 15) * 4, c0 = (tid >> 4) * 4;   // this thread's 4x4 sub-block
    T x[4][4], y[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int r = r0 + u, c = c0 + v;
            x[u][v] = (r >= c) ? L[(size_t)(k0 + r) + (size_t)(k0 + c) * ld] : T(0);
            y[u][v] = (r == c) ? T(1) : T(0);
        }
    for (int j = 0; j < NB; ++j) {
        const int b = j & 1;
        if (c0 <= j && j < c0 + 4) {
#pragma unroll
            for (int v = 0; v < 4; ++v)
                if (c0 + v == j)
#pragma unroll
                    for (int u = 0; u < 4; ++u) S.col[b][r0 + u] = x[u][v];
        }
        if (r0 <= j && j < r0 + 4) {
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (r0 + u == j)
#pragma unroll
                    for (int v = 0; v < 4; ++v) S.rowx[b][c0 + v] = y[u][v];
        }
        __syncthreads();
        T d = S.col[b][j];
        if (tid == 0) S.piv[j] = d;
        if (!(d > T(0))) d = T(1);
        const T rs = rsqrt_t(d);          // 1 / l_jj
        const T rd = rs * rs;             // 1 / a_jj
        if (r0 + 3 < j) continue;   // rows above j: nothing left to update
        T cr[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) cr[u] = S.col[b][r0 + u];
        if (c0 + 3 > j) {            // entries of A right of column j
            T cc[4];
#pragma unroll
            for (int v = 0; v < 4; ++v) cc[v] = S.col[b][c0 + v] * rd;
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v)
                    if (c0 + v > j && r0 + u >= c0 + v) x[u][v] -= cr[u] * cc[v];
        }
        T xj[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) xj[v] = S.rowx[b][c0 + v] * rs;   // final row j of X
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const T l = cr[u] * rs;
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                if (r0 + u > j) y[u][v] -= l * xj[v];
                else if (r0 + u == j) y[u][v] = xj[v];
            }
        }
    }
    __syncthreads();
    if (tid < NB && !(S.piv[tid] > T(0))) info[0] = 1;
    T* Lb = Linv + (size_t)(k0 / NB) * NB * NB;
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int r = r0 + u, c = c0 + v;
            T p = S.piv[c];
            if (!(p > T(0))) p = T(1);
            if (r > c) L[(size_t)(k0 + r) + (size_t)(k0 + c) * ld] = x[u][v] * rsqrt_t(p);
            else if (r == c) L[(size_t)(k0 + r) + (size_t)(k0 + c) * ld] = p * rsqrt_t(p);
            Lb[r + (size_t)c * NB] = y[u][v];
        }
}

template <typename T>
__global__ void __launch_bounds__(256) potrf_diag(T* __restrict__ L, int ld, int k0, T* __restrict__ Linv,
                                                  int* __restrict__ info)
{
    potrf_body<T>(L, ld, k0, Linv, info);
}

// L_ik = A_ik Linv_kk^T for the row block starting at k0 + NB * (1 + i)
template <typename T>
__device__ __forceinline__ void trsm_body(T* __restrict__ L, int ld, int k0, const T* __restrict__ Linv, int i)
{
    extern __shared__ unsigned char smem_raw[];
    T(*a)[NB + 1] = reinterpret_cast<T(*)[NB + 1]>(smem_raw);
    T(*iv)[NB + 1] = a + NB;
    const int tid = threadIdx.x;
    const int r0 = k0 + NB * (1 + i);
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

template <typename T>
__global__ void __launch_bounds__(256) trsm_panel(T* __restrict__ L, int ld, int k0, const T* __restrict__ Linv)
{
    trsm_body<T>(L, ld, k0, Linv, blockIdx.x);
}

// A_IJ -= L_Ik L_Jk^T for the lower tile b (I >= J) of the trailing matrix.
template <typename T>
__device__ __forceinline__ void syrk_body(T* __restrict__ L, int ld, int k0, long long b)
{
    extern __shared__ unsigned char smem_raw[];
    T* sa = reinterpret_cast<T*>(smem_raw);   // [NB][NB+1]  rows of block I
    T* sb = sa + NB * (NB + 1);               // [NB][NB+1]  rows of block J
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
__global__ void __launch_bounds__(256) syrk_update(T* __restrict__ L, int ld, int k0)
{
    syrk_body<T>(L, ld, k0, blockIdx.x);
}

// The leading column strip of the trailing matrix, gridDim.y 64-wide column
// blocks wide: tiles (t0 + 64 I, t0 + 64 J) with I >= J, t0 = k0 + 64.
template <typename T>
__global__ void __launch_bounds__(256) syrk_strip(T* __restrict__ L, int ld, int k0)
{
    if (blockIdx.x < blockIdx.y) return;
    extern __shared__ unsigned char smem_raw[];
    T* sa = reinterpret_cast<T*>(smem_raw);
    T* sb = sa + NB * (NB + 1);
    const int t0 = k0 + NB;
    const int rI = t0 + NB * blockIdx.x, rJ = t0 + NB * blockIdx.y;
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
        for (int v = 0; v < 4; ++v) L[(size_t)(rI + tr + u) + (size_t)(rJ + tc + v) * ld] -= acc[u][v];
}

// Tensor-core trailing update of the lower 128 x 128 tiles of [r0, np)^2
// (FP32 storage, 3xTF32 arithmetic) from the split panel; a bounded wait that
// gives up sets status[0] = GBEM_ERR_TIMEOUT.
__global__ void __launch_bounds__(256) syrk_tc(float* __restrict__ L, int ld, int r0,
                                               const unsigned char* __restrict__ hi,
                                               const unsigned char* __restrict__ lo, int* status)
{
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    long long b = blockIdx.x;
    int I = (int)((sqrt(8.0 * (double)b + 1.0) - 1.0) * 0.5);
    while ((long long)(I + 1) * (I + 2) / 2 <= b) ++I;
    while ((long long)I * (I + 1) / 2 > b) --I;
    const int J = (int)(b - (long long)I * (I + 1) / 2);
    if (!tc::syrk_tile(L, ld, r0 + tc::TM * I, r0 + tc::TM * J, hi, lo, I, J, tc_smem) && threadIdx.x == 0)
        atomicCAS(status, 0, (int)GBEM_ERR_TIMEOUT);
}

// One launch of the FP32 factorisation step: CTA 0 factors the next
// diagonal block (k0n, already brought up to date by the strip kernel) while
// the other CTAs apply the current panel to the tensor-core region [r0, np)^2,
// which does not touch that block.  The diagonal factorisation is thereby
// hidden behind the trailing update.
__global__ void __launch_bounds__(256) step_fused(float* __restrict__ L, int ld, int k0n, float* __restrict__ Linv,
                                                  int* __restrict__ info, int r0, const unsigned char* __restrict__ hi,
                                                  const unsigned char* __restrict__ lo)
{
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    if (blockIdx.x == 0) {
        potrf_body<float>(L, ld, k0n, Linv, info);
        return;
    }
    long long b = blockIdx.x - 1;
    int I = (int)((sqrt(8.0 * (double)b + 1.0) - 1.0) * 0.5);
    while ((long long)(I + 1) * (I + 2) / 2 <= b) ++I;
    while ((long long)I * (I + 1) / 2 > b) --I;
    const int J = (int)(b - (long long)I * (I + 1) / 2);
    if (!tc::syrk_tile(L, ld, r0 + tc::TM * I, r0 + tc::TM * J, hi, lo, I, J, tc_smem) && threadIdx.x == 0)
        atomicCAS(info + 3, 0, (int)GBEM_ERR_TIMEOUT);
}

template <typename T>
cudaError_t cholesky(T* L, int np, T* Linv, int* info, unsigned char* split, cudaStream_t s)
{
    const int nblk = np / NB;
    const size_t smem = 2 * NB * (NB + 1) * sizeof(T);
    constexpr bool kTensor = sizeof(T) == 4;   // FP32 storage: trailing update on tcgen05
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(potrf_diag<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)sizeof(PotrfSmem<T>))) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(trsm_panel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(syrk_update<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(syrk_strip<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
        cudaSuccess)
        return e;
    if (kTensor &&
        (e = cudaFuncSetAttribute(syrk_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM_BYTES)) !=
            cudaSuccess)
        return e;
    if (kTensor) {
        if ((e = cudaFuncSetAttribute(step_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM_BYTES)) !=
            cudaSuccess)
            return e;
        // block 0 is factored alone; every later diagonal block is factored
        // inside the fused launch of the previous step
        potrf_diag<T><<<1, 256, sizeof(PotrfSmem<T>), s>>>(L, np, 0, Linv, info);
        count_launch();
        for (int k = 0; k + 1 < nblk; ++k) {
            const int k0 = k * NB;
            const int m = nblk - k - 1;   // trailing order in 64-blocks
            trsm_panel<T><<<m, 256, smem, s>>>(L, np, k0, Linv);
            count_launch();
            // strip: one or two column blocks, leaving an even number of
            // blocks (whole 128-tiles) for the tensor cores
            const int sw = ((m - 1) & 1) ? 2 : 1;
            syrk_strip<T><<<dim3(m, sw), 256, smem, s>>>(L, np, k0);
            count_launch();
            const int r0 = k0 + NB + NB * sw;
            const long long nt = (np - r0) / tc::TM;
            // one split buffer suffices: the next step's split follows this
            // step's fused launch in stream order
            unsigned char* hi = split;
            unsigned char* lo = split + (size_t)(np / tc::TM + 1) * tc::OPER_BYTES;
            if (nt > 0) {
                const long long elems = (long long)(np - r0) * tc::TK;
                const int sgrid = (int)std::min<long long>(4096, (elems + 255) / 256);
                tc::split_panel<<<sgrid, 256, 0, s>>>(reinterpret_cast<const float*>(L), np, k0, r0, np, hi, lo);
                count_launch();
            }
            step_fused<<<(unsigned)(1 + nt * (nt + 1) / 2), 256, tc::SMEM_BYTES, s>>>(
                reinterpret_cast<float*>(L), np, k0 + NB, reinterpret_cast<float*>(Linv), info, r0, hi, lo);
            count_launch();
        }
        return cudaGetLastError();
    }
    for (int k = 0; k < nblk; ++k) {
        const int k0 = k * NB;
        potrf_diag<T><<<1, 256, sizeof(PotrfSmem<T>), s>>>(L, np, k0, Linv, info);
        count_launch();
        const int m = nblk - k - 1;   // trailing order in 64-blocks
        if (m <= 0) continue;
        trsm_panel<T><<<m, 256, smem, s>>>(L, np, k0, Linv);
        count_launch();
        long long tiles = (long long)m * (m + 1) / 2;
        syrk_update<T><<<(unsigned)tiles, 256, smem, s>>>(L, np, k0);
        count_launch();
    }
    return cudaGetLastError();
}

// ---- batched factorisation: elimination step k of every structure of a
// batch at once (FP32 storage).  steps[k * (nb + 1) ..] holds, per step, the
// prefix sums over structures of their panel blocks below the diagonal
// (trsm) and, at offset nsteps * (nb + 1), of their trailing tiles (syrk).
__global__ void __launch_bounds__(256) potrf_batched(BatchView v, int k)
{
    const int b = blockIdx.x;
    const int np = v.np[b];
    if (k * NB >= np) return;
    potrf_body<float>(v.A32 + v.moff[b], np, k * NB, v.Linv + v.ioff[b], v.flags + 4 * b);
}

__global__ void __launch_bounds__(256) trsm_batched(BatchView v, int k, const long long* __restrict__ prefix)
{
    __shared__ int sb;
    if (threadIdx.x == 0) sb = batch_find(prefix, v.nb, (long long)blockIdx.x);
    __syncthreads();
    const int b = sb;
    trsm_body<float>(v.A32 + v.moff[b], v.np[b], k * NB, v.Linv + v.ioff[b], (int)(blockIdx.x - prefix[b]));
}

__global__ void __launch_bounds__(256) syrk_batched(BatchView v, int k, const long long* __restrict__ prefix)
{
    __shared__ int sb;
    if (threadIdx.x == 0) sb = batch_find(prefix, v.nb, (long long)blockIdx.x);
    __syncthreads();
    const int b = sb;
    syrk_body<float>(v.A32 + v.moff[b], v.np[b], k * NB, (long long)blockIdx.x - prefix[b]);
}

}  // namespace

cudaError_t launch_cholesky_f64(double* L, int np, int nb, double* Linv, int* info, cudaStream_t s)
{
    if (nb != NB || np % NB) return cudaErrorInvalidValue;
    return cholesky<double>(L, np, Linv, info, nullptr, s);
}

size_t cholesky_f32_split_bytes(int np) { return 2 * (size_t)(np / tc::TM + 1) * tc::OPER_BYTES; }

cudaError_t launch_cholesky_f32(float* L, int np, int nb, float* Linv, int* info, unsigned char* split,
                                cudaStream_t s)
{
    if (nb != NB || np % tc::TM || !split) return cudaErrorInvalidValue;
    return cholesky<float>(L, np, Linv, info, split, s);
}

cudaError_t launch_cholesky_batched(const BatchView& v, int nsteps, const long long* steps_dev,
                                    const long long* steps_host, cudaStream_t s)
{
    const size_t smem = 2 * NB * (NB + 1) * sizeof(float);
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(potrf_batched, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)sizeof(PotrfSmem<float>))) != cudaSuccess ||
        (e = cudaFuncSetAttribute(trsm_batched, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
            cudaSuccess ||
        (e = cudaFuncSetAttribute(syrk_batched, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
            cudaSuccess)
        return e;
    const int nb1 = v.nb + 1;
    for (int k = 0; k < nsteps; ++k) {
        potrf_batched<<<v.nb, 256, sizeof(PotrfSmem<float>), s>>>(v, k);
        count_launch();
        const long long ntrsm = steps_host[(size_t)k * nb1 + v.nb];
        const long long nsyrk = steps_host[(size_t)(nsteps + k) * nb1 + v.nb];
        if (ntrsm > 0) {
            trsm_batched<<<(unsigned)ntrsm, 256, smem, s>>>(v, k, steps_dev + (size_t)k * nb1);
            count_launch();
        }
        if (nsyrk > 0) {
            syrk_batched<<<(unsigned)nsyrk, 256, smem, s>>>(v, k, steps_dev + (size_t)(nsteps + k) * nb1);
            count_launch();
        }
    }
    return cudaGetLastError();
}
