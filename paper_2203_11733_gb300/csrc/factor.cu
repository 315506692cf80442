// Blocked right-looking Cholesky factorisation A = L L^T of the Galerkin
// matrix, which is symmetric positive definite (Wu & Li, Sec. 3.2, Theorem 1:
// the single-layer operator is elliptic, hence Cholesky).
//
// The matrix is np x np column-major (np a multiple of the block size nb = 64,
// padding rows carry the identity), lower triangle significant.
//
// FP64 storage, for each block column k:
//   1. potrf_diag:  L_kk = chol(A_kk) and Linv_kk = L_kk^-1 (kept for the
//                   panel products and the triangular solves);
//   2. trsm_panel:  L_ik = A_ik Linv_kk^T for the blocks below;
//   3. syrk_update: A_ij -= L_ik L_jk^T on the lower tiles of the trailing
//                   matrix.
// FP32 storage (mixed mode, whose FP64 refinement restores the solution's
// accuracy): one launch per block column k (factor_step), whose CTAs take,
// in the order they start, the panel work of every row block below the
// diagonal (products, strip update of the next one or two block columns,
// TF32 hi/lo split), the factorisation and inverse of diagonal block k+1, and
// the tensor-core update of the remaining trailing tiles (tc_syrk.cuh); each
// waits on release flags for exactly the panel rows it needs.
// A non-positive pivot sets info[0] = 1 and is replaced by 1 so that the
// factorisation completes without NaNs; the host reports GBEM_ERR_NOT_SPD.
#include <cuda_fp16.h>

#include <algorithm>

#include "gbem_internal.h"
#include "tc_syrk.cuh"

namespace {

constexpr int NB = 64;

// Cholesky of one 64x64 diagonal block and the inverse X = L^-1 of its factor
// (kept for the panel products and the triangular solves), in 16 steps of 4
// columns with one barrier each.
//
// The 136 threads below index 136 each own one 4x4 block (R, C), R >= C, of
// the lower triangle, in registers.  At step s:
//   1. the owners of column block s publish it through double-buffered
//      shared memory;
//   2. every thread with R >= s factors the 4x4 pivot block
//      P_ss = L_ss L_ss^T itself and solves its own rows against it, which
//      gives its block L_Rs;
//   3. threads right of column block s apply the rank-4 update
//      A_RC -= L_Rs L_Cs^T; the owners store L_Rs, and from then on their
//      registers accumulate block (R, s) of X;
//   4. X follows by block forward substitution one step behind the factor:
//      threads with C < s <= R subtract L_R,s-1 X_s-1,C (X_s-1,C was
//      published at step s-1), and the threads of row block s finish
//      X_sC = L_ss^-1 (I_sC - sum_J L_sJ X_JC) and publish it.
// A non-positive pivot sets info[0] = 1 and is replaced by 1 so that the
// factorisation completes without NaNs.
template <typename T>
struct PotrfSmem {
    T pan[2][NB][4];   // column block s of the reduced matrix, pan[b][r][w]
    T xr[2][4][NB];    // row block s of X, xr[b][w][c]
};

__device__ __forceinline__ float rsqrt_t(float d) { return rsqrtf(d); }
__device__ __forceinline__ double rsqrt_t(double d) { return 1.0 / sqrt(d); }

// barrier 1 over warps 0-4 (the threads that own a block of the triangle)
__device__ __forceinline__ void bar_factor() { asm volatile("bar.sync 1, 160;" ::: "memory"); }

// four consecutive elements (16- or 32-byte aligned)
__device__ __forceinline__ void load4(const float* p, float v[4])
{
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x, v[1] = q.y, v[2] = q.z, v[3] = q.w;
}
__device__ __forceinline__ void load4(const double* p, double v[4])
{
    const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
    v[0] = a.x, v[1] = a.y, v[2] = b.x, v[3] = b.y;
}
// Global memory only, through L2: the block may have been written by another
// CTA of the same launch.
__device__ __forceinline__ void load4_l2(const float* p, float v[4])
{
    const float4 q = __ldcg(reinterpret_cast<const float4*>(p));
    v[0] = q.x, v[1] = q.y, v[2] = q.z, v[3] = q.w;
}
__device__ __forceinline__ void load4_l2(const double* p, double v[4])
{
    const double2 a = __ldcg(reinterpret_cast<const double2*>(p)), b = __ldcg(reinterpret_cast<const double2*>(p) + 1);
    v[0] = a.x, v[1] = a.y, v[2] = b.x, v[3] = b.y;
}
__device__ __forceinline__ void store4(float* p, float a, float b, float c, float d)
{
    *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
}
__device__ __forceinline__ void store4(double* p, double a, double b, double c, double d)
{
    reinterpret_cast<double2*>(p)[0] = make_double2(a, b);
    reinterpret_cast<double2*>(p)[1] = make_double2(c, d);
}

// P = Ld Ld^T for a 4x4 block (lower entries of p); dv[w] = 1 / Ld[w][w].
template <typename T>
__device__ __forceinline__ void chol4(const T p[4][4], T Ld[4][4], T dv[4], bool& bad)
{
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        T d = p[w][w];
#pragma unroll
        for (int q = 0; q < w; ++q) d -= Ld[w][q] * Ld[w][q];
        if (!(d > T(0))) {
            bad = true;
            d = T(1);
        }
        const T rs = rsqrt_t(d);
        dv[w] = rs;
        Ld[w][w] = d * rs;
#pragma unroll
        for (int i = w + 1; i < 4; ++i) {
            T a = p[i][w];
#pragma unroll
            for (int q = 0; q < w; ++q) a -= Ld[i][q] * Ld[w][q];
            Ld[i][w] = a * rs;
        }
    }
}

// l = a Ld^-T: the row of L whose row of the reduced matrix is a.
template <typename T>
__device__ __forceinline__ void solve_row(const T a[4], const T Ld[4][4], const T dv[4], T l[4])
{
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        T x = a[w];
#pragma unroll
        for (int q = 0; q < w; ++q) x -= l[q] * Ld[w][q];
        l[w] = x * dv[w];
    }
}

template <typename T>
__device__ __forceinline__ void potrf_work(T* __restrict__ L, int ld, int k0, T* __restrict__ Linv,
                                           int* __restrict__ info)
{
    extern __shared__ unsigned char smem_raw[];
    PotrfSmem<T>& S = *reinterpret_cast<PotrfSmem<T>*>(smem_raw);
    const int tid = threadIdx.x;
    // triangular thread map: tid -> (R, C), R >= C, column blocks in order
    const bool act = tid < 136;
    int C = 0, R = act ? tid : 0;
    while (R >= 16 - C) {
        R -= 16 - C;
        ++C;
    }
    R += C;
    const int r0 = 4 * R, c0 = 4 * C;
    T z[4][4], lr[4][4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        T col[4] = {T(0), T(0), T(0), T(0)};
        if (act) load4_l2(L + (size_t)(k0 + r0) + (size_t)(k0 + c0 + v) * ld, col);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            z[u][v] = col[u];
            lr[u][v] = T(0);
        }
    }
    bool bad = false;
#pragma unroll 1
    for (int s = 0; s < 16; ++s) {
        const int b = s & 1;
        if (act && C == s) {
#pragma unroll
            for (int u = 0; u < 4; ++u) store4(&S.pan[b][r0 + u][0], z[u][0], z[u][1], z[u][2], z[u][3]);
        }
        bar_factor();
        if (!act || R < s) continue;
        T p[4][4], Ld[4][4], dv[4], nr[4][4];
#pragma unroll
        for (int w = 0; w < 4; ++w) load4(&S.pan[b][4 * s + w][0], p[w]);
        chol4(p, Ld, dv, bad);
        if (R == s) {
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int w = 0; w < 4; ++w) nr[u][w] = Ld[u][w];
        } else {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                T a[4];
                load4(&S.pan[b][r0 + u][0], a);
                solve_row(a, Ld, dv, nr[u]);
            }
        }
        if (C == s) {
            // the block of L is final: store it and start the block of X
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                T* dst = L + (size_t)(k0 + r0) + (size_t)(k0 + c0 + v) * ld;
                if (R > C) store4(dst, nr[0][v], nr[1][v], nr[2][v], nr[3][v]);
                else {
#pragma unroll
                    for (int u = v; u < 4; ++u) dst[u] = nr[u][v];
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) z[u][v] = (R == C && u == v) ? T(1) : T(0);
            }
            if (R == C && bad) info[0] = 1;
        } else {
            T P[4][4], Q[4][4];   // z -= P Q^T
            if (C > s) {
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    T a[4];
                    load4(&S.pan[b][c0 + v][0], a);
                    solve_row(a, Ld, dv, Q[v]);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int w = 0; w < 4; ++w) P[u][w] = nr[u][w];
            } else {
#pragma unroll
                for (int w = 0; w < 4; ++w) {
                    T x[4];
                    load4(&S.xr[b ^ 1][w][c0], x);
#pragma unroll
                    for (int v = 0; v < 4; ++v) Q[v][w] = x[v];
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int w = 0; w < 4; ++w) P[u][w] = lr[u][w];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v)
#pragma unroll
                    for (int w = 0; w < 4; ++w) z[u][v] -= P[u][w] * Q[v][w];
        }
        if (R == s) {
            // finish row block s of X: z = L_ss^-1 z, column by column
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                T col[4] = {z[0][v], z[1][v], z[2][v], z[3][v]}, x[4];
#pragma unroll
                for (int w = 0; w < 4; ++w) {
                    T t = col[w];
#pragma unroll
                    for (int q = 0; q < w; ++q) t -= Ld[w][q] * x[q];
                    x[w] = t * dv[w];
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) z[u][v] = x[u];
            }
#pragma unroll
            for (int w = 0; w < 4; ++w) store4(&S.xr[b][w][c0], z[w][0], z[w][1], z[w][2], z[w][3]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int w = 0; w < 4; ++w) lr[u][w] = nr[u][w];
    }
    if (!act) return;
    // X: this block and zeros in its mirror above the diagonal
    T* Lb = Linv + (size_t)(k0 / NB) * NB * NB;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        store4(Lb + r0 + (size_t)(c0 + v) * NB, z[0][v], z[1][v], z[2][v], z[3][v]);
        if (R > C) store4(Lb + c0 + (size_t)(r0 + v) * NB, T(0), T(0), T(0), T(0));
    }
}

// Warps 0-4 factor; the other threads of the CTA pass through.
template <typename T>
__device__ __forceinline__ void potrf_body(T* __restrict__ L, int ld, int k0, T* __restrict__ Linv,
                                           int* __restrict__ info)
{
    if (threadIdx.x < 160) potrf_work<T>(L, ld, k0, Linv, info);
}

// Programmatic dependent launch: wait for the previous kernel of the stream
// (a no-op when launched without the attribute), and let the next one be
// scheduled early; it waits in turn before touching memory.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }


__device__ __forceinline__ unsigned ld_acquire(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(unsigned* p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Waits until every flag in f0[0..n0) and f1[0..n1) has reached `token`
// (n0 + n1 <= blockDim.x): thread q polls one flag, so the polls' latencies
// overlap, and the CTA then proceeds together.  Bounded by limit_ns of
// wall-clock time: false (and status = GBEM_ERR_TIMEOUT) if a wait gave up
// or another CTA's already had.
__device__ bool wait_flags(const unsigned* f0, int n0, const unsigned* f1, int n1, unsigned token, int* status,
                           uint64_t limit_ns = bw::kDependencyNs)
{
    const int q = threadIdx.x;
    int ok = 1;
    if (q < n0 + n1) {
        const unsigned* f = q < n0 ? f0 + q : f1 + (q - n0);
        bw::Deadline dl(limit_ns);
        while (ld_acquire(f) < token) {
            if (dl.expired() || *(volatile int*)status != 0) {
                atomicCAS(status, 0, (int)GBEM_ERR_TIMEOUT);
                ok = 0;
                break;
            }
            __nanosleep(20);
        }
    }
    return __syncthreads_and(ok) != 0;
}

__device__ __forceinline__ bool wait_flags(const unsigned* f, int n, unsigned token, int* status)
{
    return wait_flags(f, n, nullptr, 0, token, status);
}

// Self-test of the release-flag wait above: one CTA waits for flag[0] to
// reach 1 with the given limit (gbem_selftest_wait).
__global__ void __launch_bounds__(256) wait_selftest(const unsigned* flag, int* status, unsigned long long limit_ns)
{
    wait_flags(flag, 1, nullptr, 0, 1u, status, limit_ns);
}

constexpr int PT = NB + 4;   // padded row of a t-major 64 x 64 block in shared memory

// The work that follows the factorisation of diagonal block k (k0 = 64 k) in
// the same CTA, all 256 threads, arranged so that every global read is
// issued in one phase:
//   1. the strip rows of step k: L_ck = A_ck Linv_kk^T for the ns row blocks
//      c = k+1 .. k+ns, stored t-major in lsT[s * 4096 + t * 64 + r] =
//      L_ck[r][t] for the strip update of that step's panel work;
//   2. the lookahead panel work of row block c = k+1 for step k: L_ck is
//      written to L, and A_cc -= L_ck L_ck^T once A_cc has every earlier
//      panel applied (after `ready`, when given: the tile that applies the
//      previous panel to it); then pflag_c = token.  The next launch orders
//      these writes before its reads, so the flag needs no fence.
// Shared memory: four t-major 64 x 68 blocks.
__device__ void diag_tail(float* __restrict__ L, int ld, int k0, const float* __restrict__ Linv,
                          float* __restrict__ lsT, int ns, const unsigned* ready, unsigned* pflag_c, unsigned token,
                          int* status)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float(*ivT)[PT] = reinterpret_cast<float(*)[PT]>(smem_raw);   // ivT[t][c] = Linv_kk[c][t]
    float(*aT)[PT] = ivT + NB;                                    // aT[s * 64 + t][r] = A_ck[r][t]
    float(*lT)[PT] = ivT + 3 * NB;                                // lT[t][r] = L_ck[r][t], c = k+1
    const int tid = threadIdx.x;
    const int tr = (tid & 15) * 4, tc = (tid >> 4) * 4;
    const int rc = k0 + NB;
    const float* Lb = Linv + (size_t)(k0 / NB) * NB * NB;
    __syncthreads();   // the factorisation is done with shared memory, its stores are issued
    // 1. every read at once: the inverse (just written by this CTA), the
    // strip blocks, and A_cc unless it still waits for a tile
    float4 cc[4];
    if (!ready)
#pragma unroll
        for (int v = 0; v < 4; ++v)
            cc[v] = __ldcg(reinterpret_cast<const float4*>(L + (size_t)(rc + tr) + (size_t)(rc + tc + v) * ld));
    for (int e = tid; e < NB * NB / 4; e += blockDim.x) {
        const int t = e >> 4, r = (e & 15) * 4;
        *reinterpret_cast<float4*>(&ivT[t][r]) = __ldcg(reinterpret_cast<const float4*>(Lb) + e);
        for (int sidx = 0; sidx < ns; ++sidx)
            *reinterpret_cast<float4*>(&aT[sidx * NB + t][r]) = __ldcg(
                reinterpret_cast<const float4*>(L + (size_t)(rc + sidx * NB + r) + (size_t)(k0 + t) * ld));
    }
    __syncthreads();
    for (int sidx = 0; sidx < ns; ++sidx) {
        float acc[4][4] = {};
        for (int t = 0; t < tc + 4; ++t) {   // Linv_kk is lower triangular
            const float4 x = *reinterpret_cast<const float4*>(&aT[sidx * NB + t][tr]);
            const float4 y = *reinterpret_cast<const float4*>(&ivT[t][tc]);
            const float xs[4] = {x.x, x.y, x.z, x.w}, ys[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] += xs[u] * ys[v];
        }
        float* dst = lsT + (size_t)sidx * NB * NB;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const float4 q = make_float4(acc[0][v], acc[1][v], acc[2][v], acc[3][v]);
            *reinterpret_cast<float4*>(dst + (size_t)(tc + v) * NB + tr) = q;
            if (sidx == 0) {
                *reinterpret_cast<float4*>(&lT[tc + v][tr]) = q;
                // L_ck into L: column k0 + tc + v, rows rc + tr ..
                *reinterpret_cast<float4*>(L + (size_t)(rc + tr) + (size_t)(k0 + tc + v) * ld) = q;
            }
        }
    }
    if (ns <= 0) return;
    // 2. the lookahead update of A_cc
    if (ready) {
        if (!wait_flags(ready, 1, 1u, status)) return;
#pragma unroll
        for (int v = 0; v < 4; ++v)
            cc[v] = __ldcg(reinterpret_cast<const float4*>(L + (size_t)(rc + tr) + (size_t)(rc + tc + v) * ld));
    } else {
        __syncthreads();   // lT complete
    }
    float acc[4][4] = {};
    for (int t = 0; t < NB; ++t) {
        const float4 x = *reinterpret_cast<const float4*>(&lT[t][tr]);
        const float4 y = *reinterpret_cast<const float4*>(&lT[t][tc]);
        const float xs[4] = {x.x, x.y, x.z, x.w}, ys[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] += xs[u] * ys[v];
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        float4 o = cc[v];
        o.x -= acc[0][v];
        o.y -= acc[1][v];
        o.z -= acc[2][v];
        o.w -= acc[3][v];
        *reinterpret_cast<float4*>(L + (size_t)(rc + tr) + (size_t)(rc + tc + v) * ld) = o;
    }
    if (tid == 0) *(volatile unsigned*)pflag_c = token;
}

// A helper CTA of step k (k0 = 64 (k+1), the diagonal block the step's
// diagonal CTA factors): strip row s of step k+1, L_c,k+1 = A_c,k+1 Linv^T
// with c = k+2+s, into lsT[s] (t-major); for s = 0 also the lookahead panel
// work of row block k+2 (L_k+2,k+1 into L, A_k+2,k+2 -= L L^T, then
// pflag_c = token + 1).  The blocks of A are read as soon as the panel rows
// are done, before the inverse is ready, so only the inverse's read and the
// products follow the diagonal block.  When block (k+2, k+2) lies in step k's
// tensor-core tile (0, 0), lk points at L_k+2,k (step k's panel row k+2) and
// the helper applies step k's update to the block too, before the inverse is
// ready; the tile leaves that quadrant alone.  All 256 threads; shared
// memory: four t-major blocks.
__device__ void tail_helper(float* __restrict__ L, int ld, int k0, const float* __restrict__ Linv,
                            float* __restrict__ lsT_s, int sidx, const unsigned* pflag_row, const float* lk,
                            const unsigned* dflag, unsigned token, unsigned* pflag_c, int* status)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float(*ivT)[PT] = reinterpret_cast<float(*)[PT]>(smem_raw);   // ivT[t][c] = Linv[c][t]
    float(*aT)[PT] = ivT + NB;                                    // aT[t][r] = A_c,k+1[r][t]
    float(*lT)[PT] = ivT + 2 * NB;                                // lT[t][r] = L_c,k+1[r][t]
    float(*lkT)[PT] = ivT + 3 * NB;                               // lkT[t][r] = L_c,k[r][t], then A_cc
    const int tid = threadIdx.x;
    const int tr = (tid & 15) * 4, tc = (tid >> 4) * 4;
    const int rc = k0 + NB * (1 + sidx);
    const bool look = sidx == 0;
    if (!wait_flags(pflag_row, 1, token, status)) return;
    for (int e = tid; e < NB * NB / 4; e += blockDim.x) {
        const int t = e >> 4, r = (e & 15) * 4;
        *reinterpret_cast<float4*>(&aT[t][r]) =
            __ldcg(reinterpret_cast<const float4*>(L + (size_t)(rc + r) + (size_t)(k0 + t) * ld));
    }
    if (look) {
        float4 cc[4];
#pragma unroll
        for (int v = 0; v < 4; ++v)
            cc[v] = __ldcg(reinterpret_cast<const float4*>(L + (size_t)(rc + tr) + (size_t)(rc + tc + v) * ld));
        if (lk) {
            for (int e = tid; e < NB * NB / 4; e += blockDim.x) {
                const int t = e >> 4, r = (e & 15) * 4;
                *reinterpret_cast<float4*>(&lkT[t][r]) =
                    __ldcg(reinterpret_cast<const float4*>(lk + (size_t)r + (size_t)t * ld));
            }
            __syncthreads();
            // step k's update of A_cc: A_cc -= L_ck L_ck^T
            float acc0[4][4] = {};
#pragma unroll 4
            for (int t = 0; t < NB; ++t) {
                const float4 x = *reinterpret_cast<const float4*>(&lkT[t][tr]);
                const float4 y = *reinterpret_cast<const float4*>(&lkT[t][tc]);
                const float xs[4] = {x.x, x.y, x.z, x.w}, ys[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) acc0[u][v] += xs[u] * ys[v];
            }
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                cc[v].x -= acc0[0][v];
                cc[v].y -= acc0[1][v];
                cc[v].z -= acc0[2][v];
                cc[v].w -= acc0[3][v];
            }
            __syncthreads();   // lkT is read
        }
        // A_cc waits in shared memory for the lookahead update
#pragma unroll
        for (int v = 0; v < 4; ++v) *reinterpret_cast<float4*>(&lkT[tc + v][tr]) = cc[v];
    }
    if (!wait_flags(dflag, 1, token, status)) return;
    const float* Lb = Linv + (size_t)(k0 / NB) * NB * NB;
    for (int e = tid; e < NB * NB / 4; e += blockDim.x)
        *reinterpret_cast<float4*>(&ivT[e >> 4][(e & 15) * 4]) = __ldcg(reinterpret_cast<const float4*>(Lb) + e);
    __syncthreads();
    float acc[4][4] = {};
    for (int t = 0; t < tc + 4; ++t) {   // the inverse is lower triangular
        const float4 x = *reinterpret_cast<const float4*>(&aT[t][tr]);
        const float4 y = *reinterpret_cast<const float4*>(&ivT[t][tc]);
        const float xs[4] = {x.x, x.y, x.z, x.w}, ys[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] += xs[u] * ys[v];
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const float4 q = make_float4(acc[0][v], acc[1][v], acc[2][v], acc[3][v]);
        *reinterpret_cast<float4*>(lsT_s + (size_t)(tc + v) * NB + tr) = q;
        if (look) {
            *reinterpret_cast<float4*>(&lT[tc + v][tr]) = q;
            *reinterpret_cast<float4*>(L + (size_t)(rc + tr) + (size_t)(k0 + tc + v) * ld) = q;
        }
    }
    if (!look) return;
    __syncthreads();   // lT complete
    float acc2[4][4] = {};
    for (int t = 0; t < NB; ++t) {
        const float4 x = *reinterpret_cast<const float4*>(&lT[t][tr]);
        const float4 y = *reinterpret_cast<const float4*>(&lT[t][tc]);
        const float xs[4] = {x.x, x.y, x.z, x.w}, ys[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc2[u][v] += xs[u] * ys[v];
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        float4 o = *reinterpret_cast<const float4*>(&lkT[tc + v][tr]);
        o.x -= acc2[0][v];
        o.y -= acc2[1][v];
        o.z -= acc2[2][v];
        o.w -= acc2[3][v];
        *reinterpret_cast<float4*>(L + (size_t)(rc + tr) + (size_t)(rc + tc + v) * ld) = o;
    }
    if (tid == 0) *(volatile unsigned*)pflag_c = token + 1;
}

constexpr size_t kStripSmem = 4 * NB * PT * sizeof(float);
// Panels of kPanel 64-column blocks; the split of a panel holds
// kPanelStages K stages of 32 columns.
constexpr int kPanel = 4;
constexpr int kPanelStages = kPanel * tc::CHUNK_STAGES;
// Bytes between two K stages of one part of a panel split: one stage of every
// 128-row block of the matrix, and one more.
inline size_t split_stage_stride(int np) { return (size_t)(np / tc::TM + 1) * tc::STAGE_BYTES; }
constexpr size_t kPanelRowSmem = 4 * NB * PT * sizeof(float);
// every role of factor_step within one dynamic allocation: two CTAs per SM
constexpr size_t kFactorSmem = kPanelRowSmem > (size_t)tc::SMEM_BYTES ? kPanelRowSmem : (size_t)tc::SMEM_BYTES;

// The split scale of the FP16 tensor-core operands: s = 2^(15 - e) with
// 2^e > the largest sqrt(A_rr) over the diagonal (one CTA), so that every
// entry of the factor, |L_rt| <= sqrt(A_rr), has |s L_rt| < 2^15 (FP16's
// largest finite value is 65504).  scale[0] = s, scale[1] = 1 / s^2.
__global__ void __launch_bounds__(1024) split_scale(const float* __restrict__ L, int ld, float* __restrict__ scale)
{
    __shared__ float wmax[32];
    float m = 0.0f;
    for (int r = threadIdx.x; r < ld; r += blockDim.x) m = fmaxf(m, L[(size_t)r * ld + r]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < (blockDim.x >> 5) ? wmax[threadIdx.x] : 0.0f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (threadIdx.x == 0) {
            int e = 0;
            frexpf(sqrtf(fmaxf(m, 1e-30f)), &e);   // sqrt(max) < 2^e
            e = max(-100, min(100, e));
            scale[0] = ldexpf(1.0f, 15 - e);
            scale[1] = ldexpf(1.0f, 2 * (e - 15));
        }
    }
}

// The first diagonal block b0 of a panel (every earlier update of it done by
// the launches before), the strip rows of step b0 and the lookahead panel
// work of row block b0 + 1 (diag_tail).
__global__ void __launch_bounds__(256) panel_start(float* __restrict__ L, int ld, int b0, float* __restrict__ Linv,
                                                   int* __restrict__ info, float* __restrict__ lsT, int ns,
                                                   unsigned* __restrict__ pflag)
{
    potrf_body<float>(L, ld, b0 * NB, Linv, info);
    if (ns > 0) diag_tail(L, ld, b0 * NB, Linv, lsT, ns, nullptr, pflag + b0 + 1, (unsigned)b0 + 1, info + 3);
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
    int I = (int)((sqrtf(8.0f * (float)b + 1.0f) - 1.0f) * 0.5f);
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

// Panel work of the row blocks i = i0, i0 + di, ... < iend at step k (one
// CTA; Linv_kk and the strip blocks L_ck are loaded once for all of them):
//   1. L_ik = A_ik Linv_kk^T, written in place (Linv_kk is lower triangular,
//      so the sum over t stops at the output column);
//   2. row blocks at or below srow0 write the FP16 hi/lo split of the block,
//      scaled by split_scale, in the tensor-core operand layout, as the 2
//      stages st_base .. of the panel's split;
//   3. A_ic -= L_ik L_ck^T for the sw strip blocks c = k+1 .. k+sw, c <= i,
//      with L_ck (lsT, t-major) computed by the helpers of the previous step;
//   4. the block's panel flag is released (token), so that the diagonal
//      block, the helpers and the tiles of its rows can go on.
// A thread owns 4 rows x 4 columns of a block.  The strip targets of a block
// are read before its product, so their latency overlaps it.
__device__ void panel_rows(float* __restrict__ L, int ld, int k, const float* __restrict__ Linv, int sw, int srow0,
                           int st_base, size_t stage_stride, unsigned char* __restrict__ hi,
                           unsigned char* __restrict__ lo, const float* __restrict__ lsT, int i0, int di, int iend,
                           unsigned char* smem, float split_scale, unsigned* pflag, unsigned token)
{
    // Blocks are stored t-major (rows padded to 68 floats) so that a
    // thread's rows or columns at one t are one 16-byte load.
    float(*ivT)[PT] = reinterpret_cast<float(*)[PT]>(smem);   // ivT[t][c] = Linv_kk[c][t]
    float(*aT)[PT] = ivT + NB;                                // aT[t][r] = A_ik, then L_ik
    float(*lcT)[PT] = aT + NB;                                // lcT[s * 64 + t][c] = L_ck[c][t]
    const int tid = threadIdx.x;
    const int tr = (tid & 15) * 4, tc = (tid >> 4) * 4;
    const int k0 = k * NB;
    const float* Lb = Linv + (size_t)k * NB * NB;
    for (int e = tid; e < NB * NB / 4; e += blockDim.x)   // Linv_kk column-major: 4e = c + 64 t
        *reinterpret_cast<float4*>(&ivT[e >> 4][(e & 15) * 4]) = reinterpret_cast<const float4*>(Lb)[e];
    for (int e = tid; e < sw * NB * NB / 4; e += blockDim.x)
        *reinterpret_cast<float4*>(&lcT[e >> 4][(e & 15) * 4]) = reinterpret_cast<const float4*>(lsT)[e];
    for (int i = i0; i < iend; i += di) {
        const int rI = i * NB;
        const int nstrip = min(sw, i - k);   // strip blocks c = k+1 .. with c <= i
        float4 tgt[2][4];
#pragma unroll
        for (int sidx = 0; sidx < 2; ++sidx)
            if (sidx < nstrip)
#pragma unroll
                for (int v = 0; v < 4; ++v)
                    tgt[sidx][v] =
                        *reinterpret_cast<const float4*>(L + (size_t)(rI + tr) + (size_t)((k + 1 + sidx) * NB + tc + v) * ld);
        for (int e = tid; e < NB * NB / 4; e += blockDim.x) {
            const int t = e >> 4, r = (e & 15) * 4;
            *reinterpret_cast<float4*>(&aT[t][r]) =
                *reinterpret_cast<const float4*>(L + (size_t)(rI + r) + (size_t)(k0 + t) * ld);
        }
        __syncthreads();   // Linv, the strip blocks and A_ik are in shared memory
        float acc[4][4] = {};
        for (int t = 0; t < tc + 4; ++t) {
            const float4 x = *reinterpret_cast<const float4*>(&aT[t][tr]);
            const float4 y = *reinterpret_cast<const float4*>(&ivT[t][tc]);
            const float xs[4] = {x.x, x.y, x.z, x.w}, ys[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] += xs[u] * ys[v];
        }
        __syncthreads();   // every thread is done reading A_ik
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const float4 q = make_float4(acc[0][v], acc[1][v], acc[2][v], acc[3][v]);
            *reinterpret_cast<float4*>(&aT[tc + v][tr]) = q;
            *reinterpret_cast<float4*>(L + (size_t)(rI + tr) + (size_t)(k0 + tc + v) * ld) = q;
        }
        if (rI >= srow0) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int rr = rI - srow0 + tr + u;
                const size_t off = tc::split_offset(rr, tc, stage_stride) + (size_t)st_base * stage_stride;
                __half hv[4], lv[4];
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const float x = acc[u][v] * split_scale;   // exact: a power of two
                    hv[v] = __float2half_rn(x);
                    lv[v] = __float2half_rn(x - __half2float(hv[v]));
                }
                *reinterpret_cast<uint2*>(hi + off) = make_uint2(
                    (uint32_t)__half_as_ushort(hv[0]) | ((uint32_t)__half_as_ushort(hv[1]) << 16),
                    (uint32_t)__half_as_ushort(hv[2]) | ((uint32_t)__half_as_ushort(hv[3]) << 16));
                *reinterpret_cast<uint2*>(lo + off) = make_uint2(
                    (uint32_t)__half_as_ushort(lv[0]) | ((uint32_t)__half_as_ushort(lv[1]) << 16),
                    (uint32_t)__half_as_ushort(lv[2]) | ((uint32_t)__half_as_ushort(lv[3]) << 16));
            }
        }
        __syncthreads();   // aT holds L_ik
#pragma unroll
        for (int sidx = 0; sidx < 2; ++sidx) {
            if (sidx >= nstrip) break;
            const float(*bT)[PT] = lcT + sidx * NB;
            float acc2[4][4] = {};
            for (int t = 0; t < NB; ++t) {
                const float4 x = *reinterpret_cast<const float4*>(&aT[t][tr]);
                const float4 y = *reinterpret_cast<const float4*>(&bT[t][tc]);
                const float xs[4] = {x.x, x.y, x.z, x.w}, ys[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) acc2[u][v] += xs[u] * ys[v];
            }
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                float4 o = tgt[sidx][v];
                o.x -= acc2[0][v];
                o.y -= acc2[1][v];
                o.z -= acc2[2][v];
                o.w -= acc2[3][v];
                *reinterpret_cast<float4*>(L + (size_t)(rI + tr) + (size_t)((k + 1 + sidx) * NB + tc + v) * ld) = o;
            }
        }
        __syncthreads();   // the block is stored; aT is free for the next one
        if (tid == 0) {
            asm volatile("fence.proxy.async.global;" ::: "memory");   // the split is read by bulk copies
            __threadfence();
            st_release(pflag + i, token);
        }
    }
}

// Arguments of one elimination step of the FP32 factorisation (factor_step).
// The factorisation runs by panels of up to four 64-column blocks
// [b0, e): the elimination steps k = b0 .. e-1 of a panel update only the
// panel's own columns (strip updates, the lookahead, and inner 128-tiles),
// and write the FP16 hi/lo split of every panel row as the panel's 8 K
// stages.  The update of the rest of the trailing matrix by the whole panel
// (K = 256) is done by tensor-core tiles: the next panel's columns ("front"
// tiles, in the panel's last step, after the flags of their rows) and
// everything beyond ("rest" tiles: one rest_update launch on a second
// stream, which runs beside the next panel's steps but its last; it needs
// no flags, since the panel's split is complete before it starts, and it
// touches no column the next panel's steps read or write).  The split is
// double-buffered by panel parity.
struct StepArgs {
    float* L;
    int ld, k, nblk;
    int pctas;                    // panel CTAs: the row blocks p0 + j, p0 + j + pctas, ... for CTA j
    float* Linv;
    int* info;
    int sw;        // strip width of step k: 0, 1 or 2 blocks, within the panel
    int p0;        // first panel row block (k+2; k+1 when row block k+1 had no lookahead)
    int has_diag;  // factor diagonal block k+1 (in the panel) in this launch
    int ns_next;   // strip-row helpers for step k+1 (the first also does the lookahead)
    // the panel's split: rows from srow0, this step's chunk at stage st_base
    unsigned char* hi;
    unsigned char* lo;
    int srow0, st_base;
    size_t stage_stride;
    int r0, icols;                // inner tiles: rows [r0, np), icols 128-columns from r0
    int f0, fcols;                // front tiles: rows [f0, np), fcols 128-columns from f0 (16 stages)
    int next_start;               // start the next panel (its first block f0 / 64) after front tile (0, 0)
    int f00;                      // apply this step's chunk to front tile (0, 0) now (one CTA, K = 64)
    int f00_rest;                 // ... after applying the previous panel's rest tile (0, 0) to it
    int f00_last;                 // front tile (0, 0) holds the earlier chunks: only this step's remains
    int ns_start;                 // strip rows of the next panel's first step
    const unsigned char* hi_p;    // f00_rest: the previous panel's split (rows from srow0_p)
    const unsigned char* lo_p;    // and the block (c0r, c0r) it updates
    int srow0_p, c0r;
    const float* lsT_in;
    float* lsT_out;
    unsigned* pflag;
    unsigned* tickets;
    unsigned* dflag;
    const float* scale;   // [0] the split scale s, [1] 1 / s^2 (split_scale)
};

// Tile (I, J), I >= J, of a column band of `cols` 128-columns over nrow
// 128-rows: index t over J = 0 .. cols-1, I = J .. nrow-1.  False if t is
// past the band.
__device__ __forceinline__ bool band_tile(long long t, int nrow, int cols, int& I, int& J)
{
    for (int j = 0; j < cols; ++j) {
        const long long nj = nrow - j;
        if (t < nj) {
            I = j + (int)t;
            J = j;
            return true;
        }
        t -= nj;
    }
    return false;
}

__host__ __device__ __forceinline__ long long band_tiles(int nrow, int cols)
{
    long long n = 0;
    for (int j = 0; j < cols; ++j) n += nrow - j;
    return n;
}

// Elimination step k of the FP32 factorisation in one launch.  Row block
// k+1 was already done by the previous launch (lookahead) when p0 = k+2.
// Every CTA draws a ticket in the order the CTAs start (an atomic counter
// per step), and the ticket gives its role:
//   pctas           panel work (panel_rows) of the row blocks
//                   i = p0 + ticket, p0 + ticket + pctas, ... (at most one
//                   CTA per SM: the panel is one wave and the tiles take the
//                   other slots); each block, once done, sets its release
//                   flag pflag[i] = k + 1;
//   has_diag        factor and invert diagonal block k+1, then dflag[k];
//   ns_next         helpers (tail_helper): the strip rows of step k+1 and,
//                   for the first, the lookahead panel work of row block
//                   k+2 (pflag[k+2] = k + 2);
//   rest tiles      the previous panel's update of the matrix beyond this
//                   panel (K = 256), no waits: they fill the SMs while the
//                   panel rows are computed;
//   inner tiles     the panel's 128-tiles right of the strip, after the
//                   flags of their four row blocks (this step's chunk);
//   f00             in a panel's first steps: this step's chunk applied at
//                   once to front tile (0, 0) (the next panel's first two
//                   diagonal blocks), so that the last step applies only its
//                   own chunk there; in the step whose share of the
//                   previous panel's rest tiles holds rest tile (0, 0), which
//                   covers the same block, the same CTA applies it first;
//   front tiles     the next panel's columns with the whole panel (K = 256),
//                   after the flags of their row blocks; with next_start,
//                   right after front tile (0, 0) (which holds the next
//                   panel's first diagonal block, its strip and lookahead
//                   blocks) comes the next panel's start: it waits for that
//                   tile (dflag[k], unused by a step without a diagonal
//                   block), factors block f0 / 64 and does the strip rows and
//                   lookahead of the next step (panel_start's work).
// Every wait is on a smaller ticket, a CTA that has already started: panel
// CTAs wait for nothing, the diagonal CTA for the previous launch, helpers
// for their panel row and the diagonal CTA, tiles for panel rows, the next
// panel's start for front tile (0, 0).  So the launch cannot deadlock however
// many CTAs are resident.  Waits are bounded; one that gives up sets status
// GBEM_ERR_TIMEOUT and its CTA skips its work.
__global__ void __launch_bounds__(256, 2) factor_step(const StepArgs a)
{
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    __shared__ int s_ticket;
    // the next step's launch begins as this one's CTAs exit (no early
    // trigger): CTAs of the next step waiting here would hold SM slots, at
    // the highest priority, that the concurrent rest update needs
    pdl_wait();
    if (threadIdx.x == 0) s_ticket = (int)atomicAdd(a.tickets + a.k, 1u);
    __syncthreads();
    const int t_raw = s_ticket;
    const int k = a.k, ld = a.ld;
    float* __restrict__ L = a.L;
    const unsigned token = (unsigned)k + 1;
    int* status = a.info + 3;
    const float sc = a.scale[0], unsc = a.scale[1];
    long long t = (long long)t_raw - a.pctas;   // index among the other roles
    // roles without tensor-core work give up the CTA's TMEM allocation permit
    // at once: while a CTA holds it, no second CTA of the kernel is placed on
    // its SM
    const int nin = (a.ld - a.r0) / tc::TM;
    const long long n_inner = band_tiles(nin, a.icols);
    const long long t_start = a.has_diag + a.ns_next + n_inner + a.f00 + 1;   // the next panel's start, when present
    if ((t < a.has_diag + a.ns_next || (a.next_start && t == t_start)) && threadIdx.x < 32)
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    if (t < 0) {
        // panel row blocks p0 + t_raw, p0 + t_raw + pctas, ...
        panel_rows(L, ld, k, a.Linv, a.sw, a.srow0, a.st_base, a.stage_stride, a.hi, a.lo, a.lsT_in, a.p0 + t_raw,
                   a.pctas, a.nblk, tc_smem, sc, a.pflag, token);
        return;
    }
    if (a.has_diag) {
        if (t == 0) {
            if (!wait_flags(a.pflag + k + 1, 1, token, status)) return;
            potrf_body<float>(L, ld, (k + 1) * NB, a.Linv, a.info);
            __syncthreads();   // the inverse is stored
            if (threadIdx.x == 0) {
                __threadfence();
                st_release(a.dflag + k, token);
            }
            return;
        }
        --t;
    }
    // with a strip one block wide and a lookahead helper, block (k+2, k+2)
    // lies in inner tile (0, 0) and the helper applies this step's update to it
    const bool la = a.sw == 1 && a.ns_next >= 1;
    if (t < a.ns_next) {
        const int sidx = (int)t;
        const float* lk = la ? L + (size_t)((k + 2) * NB) + (size_t)(k * NB) * ld : nullptr;
        tail_helper(L, ld, (k + 1) * NB, a.Linv, a.lsT_out + (size_t)sidx * NB * NB, sidx, a.pflag + k + 2 + sidx,
                    lk, a.dflag + k, token, a.pflag + k + 2, status);
        return;
    }
    t -= a.ns_next;
    const int np = ld;
    // the tile role's work as one or two tile jobs, run through a single
    // inlined tensor-core tile (tc::syrk_tile)
    struct TileJob {
        int rI, rJ, ia, ja, st0, nst;
        const unsigned char* hi;
        const unsigned char* lo;
        int fb0, fb1;   // row blocks whose two release flags the tile waits for (-1: none)
        bool skip00;
    };
    TileJob jobs[2];
    int njobs = 1;
    bool release_start = false;   // front tile (0, 0): release the next panel's start after it
    int I, J;
    if (t < n_inner) {
        band_tile(t, nin, a.icols, I, J);
        const int rI = a.r0 + tc::TM * I, rJ = a.r0 + tc::TM * J;
        const int off = (a.r0 - a.srow0) / tc::TM;
        jobs[0] = TileJob{rI, rJ, off + I, off + J, a.st_base, tc::CHUNK_STAGES, a.hi, a.lo, rI / NB, rJ / NB,
                          la && I == 0 && J == 0};
    } else if (a.f00 && t == n_inner) {
        // this step's chunk on front tile (0, 0), after the flags of its rows;
        // first the previous panel's rest tile (0, 0) when it is this step's
        const int off = (a.f0 - a.srow0) / tc::TM;
        const TileJob mine{a.f0, a.f0, off, off, a.st_base, tc::CHUNK_STAGES, a.hi, a.lo, a.f0 / NB, -1, false};
        if (a.f00_rest) {
            const int offp = (a.c0r - a.srow0_p) / tc::TM;
            jobs[0] = TileJob{a.c0r, a.c0r, offp, offp, 0, 4 * tc::CHUNK_STAGES, a.hi_p, a.lo_p, -1, -1, false};
            jobs[1] = mine;
            njobs = 2;
        } else {
            jobs[0] = mine;
        }
    } else {
        t -= n_inner + a.f00;
        const int nf = a.fcols > 0 ? (np - a.f0) / tc::TM : 0;
        const long long n_front = band_tiles(nf, a.fcols);
        if (a.next_start && t == 1) {
            // the next panel's start, once front tile (0, 0) is stored
            if (!wait_flags(a.dflag + k, 1, token, status)) return;
            const int b0n = a.f0 / NB;
            potrf_body<float>(L, ld, a.f0, a.Linv, a.info);
            if (a.ns_start > 0)
                diag_tail(L, ld, a.f0, a.Linv, a.lsT_out, a.ns_start, nullptr, a.pflag + b0n + 1, (unsigned)b0n + 1,
                          status);
            return;
        }
        if (a.next_start && t > 1) --t;
        if (t < n_front) {
            band_tile(t, nf, a.fcols, I, J);
            const int rI = a.f0 + tc::TM * I, rJ = a.f0 + tc::TM * J;
            const int off = (a.f0 - a.srow0) / tc::TM;
            // tile (0, 0) already holds the panel's earlier chunks when f00_last
            const bool last_only = a.f00_last && I == 0 && J == 0;
            jobs[0] = TileJob{rI, rJ, off + I, off + J, last_only ? a.st_base : 0,
                              last_only ? tc::CHUNK_STAGES : 4 * tc::CHUNK_STAGES, a.hi, a.lo, rI / NB, rJ / NB,
                              false};
            release_start = t == 0 && a.next_start;
        } else {
            njobs = 0;   // beyond the step's roles (not launched)
        }
    }
    bool ok = true;
    for (int jb = 0; jb < njobs && ok; ++jb) {
        const TileJob& T = jobs[jb];
        auto ready = [&]() {
            const int n0 = T.fb0 >= 0 ? 2 : 0, n1 = T.fb1 >= 0 ? 2 : 0;
            if (n0 + n1 == 0) return true;   // uniform over the CTA
            return wait_flags(a.pflag + (T.fb0 >= 0 ? T.fb0 : 0), n0, a.pflag + (T.fb1 >= 0 ? T.fb1 : 0), n1, token,
                              status);
        };
        // a CTA with two jobs keeps the TMEM allocation permit for the second,
        // which takes fresh mbarriers
        ok = tc::syrk_tile(L, ld, T.rI, T.rJ, T.hi, T.lo, a.stage_stride, T.ia, T.ja, T.st0, T.nst, tc_smem, ready,
                           T.skip00, unsc, jb + 1 == njobs, jb);
    }
    if (ok && release_start) {
        // front tile (0, 0) is stored: release the next panel's start
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            st_release(a.dflag + k, token);
        }
    }
    if (!ok && threadIdx.x == 0) atomicCAS(status, 0, (int)GBEM_ERR_TIMEOUT);
}

// The previous panel's update of the matrix beyond the current panel (the
// "rest" tiles): the lower 128-tiles tb0, tb0 + 1, ... of [c0r, np)^2 in
// lower-triangle order, one warp-specialised CTA each, with the previous
// panel's split (rows from srow0).  Launched on a second stream beside the
// panel's steps: it waits for nothing.
struct RestArgs {
    float* L;
    int ld;
    const unsigned char* hi;
    const unsigned char* lo;
    size_t stage_stride;
    int c0r, srow0;
    long long tb0;
    const float* scale;
    int* status;
};

__global__ void __launch_bounds__(tc::WS_THREADS, 2) rest_update(const RestArgs a)
{
    extern __shared__ __align__(1024) unsigned char ws_smem[];
    const long long b = a.tb0 + blockIdx.x;
    int I = (int)((sqrtf(8.0f * (float)b + 1.0f) - 1.0f) * 0.5f);
    while ((long long)(I + 1) * (I + 2) / 2 <= b) ++I;
    while ((long long)I * (I + 1) / 2 > b) --I;
    const int J = (int)(b - (long long)I * (I + 1) / 2);
    const int off = (a.c0r - a.srow0) / tc::TM;
    const bool ok = tc::syrk_tile_ws(a.L, a.ld, a.c0r + tc::TM * I, a.c0r + tc::TM * J, a.hi, a.lo, a.stage_stride,
                                     off + I, off + J, 0, 4 * tc::CHUNK_STAGES, ws_smem, a.scale[1]);
    if (!ok && threadIdx.x == 0) atomicCAS(a.status, 0, (int)GBEM_ERR_TIMEOUT);
}

template <typename T>
cudaError_t cholesky(T* L, int np, T* Linv, int* info, unsigned char* split, cudaStream_t s,
                     const SideStream* side = nullptr)
{
    const int nblk = np / NB;
    const size_t smem = 2 * NB * (NB + 1) * sizeof(T);
    constexpr bool kTensor = sizeof(T) == 4;   // FP32 storage: trailing update on tcgen05
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(potrf_diag<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)sizeof(PotrfSmem<T>))) != cudaSuccess)
        return e;
    if constexpr (kTensor) {
        if ((e = cudaFuncSetAttribute(factor_step, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFactorSmem)) !=
                cudaSuccess ||
            (e = cudaFuncSetAttribute(panel_start, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kStripSmem)) !=
                cudaSuccess)
            return e;
        // work space (cholesky_f32_split_bytes): the hi and lo split of two
        // panels (by parity), two strip-row buffers, then per 64-row block
        // the panel flag, the step's ticket and the diagonal-block flag
        const size_t stage_stride = split_stage_stride(np);
        const size_t part = (size_t)kPanelStages * stage_stride;
        float* lsT = reinterpret_cast<float*>(split + 4 * part);   // 2 x (2 x 64 x 64)
        unsigned* pflag = reinterpret_cast<unsigned*>(split + 4 * part + 4 * NB * NB * sizeof(float));
        float* scale = reinterpret_cast<float*>(pflag + 3 * (size_t)nblk);   // 2 floats
        unsigned* tickets = pflag + nblk;
        unsigned* dflag = tickets + nblk;
        float* Lf = reinterpret_cast<float*>(L);
        float* Linvf = reinterpret_cast<float*>(Linv);
        if ((e = cudaMemsetAsync(pflag, 0, 3 * (size_t)nblk * sizeof(unsigned), s)) != cudaSuccess) return e;
        // panel CTAs of a step: one per SM at most (each takes a share of the
        // row blocks), so that the panel work is one wave beside the tiles
        int dev = 0, nsm = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
            (e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
            return e;
        split_scale<<<1, 1024, 0, s>>>(reinterpret_cast<const float*>(L), np, scale);
        count_launch();
        // strip width of a step with m blocks of its panel right of the
        // diagonal: one or two column blocks, leaving an even number (whole
        // 128-tiles) to the tensor cores
        auto strip_width = [](int m) { return m <= 0 ? 0 : (((m - 1) & 1) ? 2 : 1); };
        // the per-step launches on the main stream at the highest priority,
        // so that the block scheduler gives their CTAs the SM slots that the
        // concurrent rest updates (second stream, lowest priority) free up
        int prio_least = 0, prio_greatest = 0;
        if ((e = cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest)) != cudaSuccess) return e;
        cudaLaunchAttribute attrs[2];
        attrs[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attrs[0].val.programmaticStreamSerializationAllowed = 1;
        attrs[1].id = cudaLaunchAttributePriority;
        attrs[1].val.priority = prio_greatest;
        if ((e = cudaFuncSetAttribute(rest_update, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      tc::WS_SMEM_BYTES)) != cudaSuccess)
            return e;
        cudaStream_t rs = side && side->stream ? side->stream : s;   // where the rest updates run
        bool joined = true;                                          // no rest update pending on rs
        // the whole factorisation is one traced span (its launches overlap);
        // algorithmic bytes and useful flops are summed over the launches
        double tr_bytes = 0.0, tr_flops = 0.0;
        cudaEvent_t ev_all = trace_begin(s);
        const double blk = 4.0 * NB * NB, tb = 4.0 * tc::TM * tc::TM;
        int prev_srow0 = 0;
        for (int q = 0, b0 = 0; b0 < nblk; ++q, b0 += kPanel) {
            const int e0 = std::min(b0 + kPanel, nblk);   // the panel is [b0, e0)
            unsigned char* hi = split + (size_t)(q & 1) * 2 * part;
            unsigned char* lo = hi + part;
            const unsigned char* hi_p = split + (size_t)((q + 1) & 1) * 2 * part;
            const unsigned char* lo_p = hi_p + part;
            const int srow0 = (b0 + 1 + strip_width(e0 - b0 - 1)) * NB;   // the panel's first tile row
            // the first diagonal block, the strip rows and lookahead of step
            // b0: a launch of its own for the first panel, the previous
            // panel's last step for the others
            if (q == 0) {
                panel_start<<<1, 256, kStripSmem, s>>>(Lf, np, b0, Linvf, info, lsT + (size_t)(b0 & 1) * 2 * NB * NB,
                                                       strip_width(e0 - b0 - 1), pflag);
                count_launch();
                tr_bytes += 4.0 * blk;
                tr_flops += 2.0 * NB * NB * NB / 3.0;
            }
            // a full panel followed by another: its first steps apply their
            // chunks to front tile (0, 0) at once, the last step its own only
            const bool incr = e0 - b0 == kPanel && e0 < nblk;
            // the previous panel's update of [e0, np)^2 (one rest_update
            // launch, beside this panel's steps but the last).  Its tile 0 is
            // block (e0, e0), front tile (0, 0) of this panel: with incr the
            // f00 CTA of the first step applies it, before that step's chunk.
            const int c0r = e0 * NB;
            const long long ntr = (np - c0r) / tc::TM;
            const long long rest = q > 0 ? ntr * (ntr + 1) / 2 : 0;
            const bool f00_rest = incr && rest > 0;
            const long long tb0 = f00_rest ? 1 : 0;
            if (rest - tb0 > 0) {
                if (rs != s) {
                    // the previous panel's split is complete once the launches
                    // issued so far on the main stream are
                    if ((e = cudaEventRecord(side->ready, s)) != cudaSuccess ||
                        (e = cudaStreamWaitEvent(rs, side->ready, 0)) != cudaSuccess)
                        return e;
                }
                RestArgs ra{Lf, np, hi_p, lo_p, stage_stride, c0r, prev_srow0, tb0, scale, info + 3};
                rest_update<<<(unsigned)(rest - tb0), tc::WS_THREADS, tc::WS_SMEM_BYTES, rs>>>(ra);
                count_launch();
                if ((e = cudaGetLastError()) != cudaSuccess) return e;
                if (rs != s) {
                    if ((e = cudaEventRecord(side->done, rs)) != cudaSuccess) return e;
                    joined = false;
                }
                const double kt = (double)(rest - tb0) * 4 * tc::TK;   // K summed over tiles
                tr_bytes += 2.0 * (rest - tb0) * tb + 2.0 * 4.0 * tc::TM * kt;
                tr_flops += 2.0 * tc::TM * tc::TM * kt;
            }
            for (int k = b0; k < e0; ++k) {
                // the last step's front tiles overlap the rest region
                if (k == e0 - 1 && !joined) {
                    if ((e = cudaStreamWaitEvent(s, side->done, 0)) != cudaSuccess) return e;
                    joined = true;
                }
                StepArgs a{};
                a.L = Lf;
                a.ld = np;
                a.k = k;
                a.nblk = nblk;
                a.Linv = Linvf;
                a.info = info;
                a.sw = strip_width(e0 - k - 1);
                a.p0 = a.sw >= 1 ? k + 2 : k + 1;
                a.has_diag = k + 1 < e0;
                a.ns_next = a.has_diag ? strip_width(e0 - k - 2) : 0;
                a.hi = hi;
                a.lo = lo;
                a.srow0 = srow0;
                a.st_base = (k - b0) * tc::CHUNK_STAGES;
                a.stage_stride = stage_stride;
                a.r0 = (k + 1 + a.sw) * NB;
                a.icols = (e0 * NB - a.r0) / tc::TM;
                a.f0 = e0 * NB;
                a.fcols = (k == e0 - 1 && e0 < nblk) ? (std::min(e0 + kPanel, nblk) - e0) * NB / tc::TM : 0;
                a.next_start = a.fcols > 0;
                a.ns_start = a.next_start ? strip_width(std::min(e0 + kPanel, nblk) - e0 - 1) : 0;
                a.f00 = incr && k < e0 - 1;
                a.f00_last = incr && k == e0 - 1;
                a.f00_rest = f00_rest && k == b0;
                a.hi_p = hi_p;
                a.lo_p = lo_p;
                a.srow0_p = prev_srow0;
                a.c0r = c0r;
                a.lsT_in = lsT + (size_t)(k & 1) * 2 * NB * NB;
                a.lsT_out = lsT + (size_t)((k + 1) & 1) * 2 * NB * NB;
                a.pflag = pflag;
                a.tickets = tickets;
                a.dflag = dflag;
                a.scale = scale;
                // a lookahead helper that applies this step's update to block
                // (k+2, k+2) needs the inner tile (0, 0) that leaves it alone
                if (a.sw == 1 && a.ns_next >= 1 && a.icols < 1) return cudaErrorInvalidValue;
                const long long npan = nblk - a.p0;
                a.pctas = (int)std::min<long long>(npan, nsm);
                const long long n_in = band_tiles((np - a.r0) / tc::TM, a.icols);
                const long long n_fr = a.fcols > 0 ? band_tiles((np - a.f0) / tc::TM, a.fcols) : 0;
                const long long grid = a.pctas + a.has_diag + a.ns_next + n_in + a.f00 + n_fr + a.next_start;
                if (grid == 0) continue;
                cudaLaunchConfig_t cfg = {};
                cfg.gridDim = dim3((unsigned)grid);
                cfg.blockDim = dim3(256);
                cfg.dynamicSmemBytes = kFactorSmem;
                cfg.stream = s;
                cfg.attrs = attrs;
                cfg.numAttrs = 2;
                if ((e = cudaLaunchKernelEx(&cfg, factor_step, a)) != cudaSuccess) return e;
                count_launch();
                // algorithmic bytes: per panel row block A_ik read, L_ik and
                // its hi/lo split written, strip blocks read and written;
                // every tile read and written once and its split rows read
                // once; the diagonal block read, its factor and inverse
                // written.  Useful flops: panel products, strip and tile
                // updates (2mnk), diagonal factor and inverse.
                const double strips = (double)npan * a.sw;
                const double kt = (double)(n_fr + a.f00_rest) * 4 * tc::TK + (double)(n_in + a.f00) * tc::TK -
                                  (a.f00_last ? 3.0 * tc::TK : 0.0);   // K summed over tiles
                const int diags = a.has_diag + a.next_start;
                tr_bytes += 2.0 * npan * blk + 8.0 * npan * NB * NB + 2.0 * strips * blk +
                            2.0 * (n_in + n_fr + a.f00_rest) * tb + 2.0 * 4.0 * tc::TM * kt + 3.0 * diags * blk;
                tr_flops += (double)npan * NB * NB * (NB + 1) + 2.0 * strips * NB * NB * NB +
                            2.0 * tc::TM * tc::TM * kt + diags * 2.0 * NB * NB * NB / 3.0;
            }
            prev_srow0 = srow0;
        }
        if (!joined && (e = cudaStreamWaitEvent(s, side->done, 0)) != cudaSuccess) return e;
        trace_end(GBEM_KERNEL_FACTOR, ev_all, s, tr_bytes, tr_flops);
        return cudaGetLastError();
    }
    if ((e = cudaFuncSetAttribute(trsm_panel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
            cudaSuccess ||
        (e = cudaFuncSetAttribute(syrk_update<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
            cudaSuccess)
        return e;
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

size_t cholesky_f32_split_bytes(int np)
{
    // hi/lo split of two panels, two strip-row buffers, panel flags, step
    // tickets and diagonal-block flags
    return 4 * (size_t)kPanelStages * split_stage_stride(np) + 4 * NB * NB * sizeof(float) +
           3 * (size_t)(np / NB) * sizeof(unsigned) + 2 * sizeof(float);
}

cudaError_t launch_cholesky_f32(float* L, int np, int nb, float* Linv, int* info, unsigned char* split,
                                cudaStream_t s, const SideStream* side)
{
    if (nb != NB || np % tc::TM || !split) return cudaErrorInvalidValue;
    return cholesky<float>(L, np, Linv, info, split, s, side);
}

cudaError_t launch_wait_selftest(const unsigned* flag, int* status, double limit_ms, cudaStream_t s)
{
    wait_selftest<<<1, 256, 0, s>>>(flag, status, (unsigned long long)(limit_ms * 1e6));
    count_launch();
    return cudaGetLastError();
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
