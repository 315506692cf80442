// Solve A X = B with the Cholesky factor (Wu & Li, Sec. 3.1 Eq. "lineareq1"
// and Sec. 3.2), iterative refinement in FP64 for the mixed-precision factor,
// and the charge on each conductor (Eq. "electriccharge").
//
// Triangular solves are blocked by the factor's 64-wide diagonal blocks and
// use their stored inverses.  Forward sweep, block rows b = 0..nblk-1:
//     Y_b = Linv_bb (W_b - sum_{j<b} L_bj Y_j)
// backward sweep, b = nblk-1..0:
//     X_b = Linv_bb^T (Y_b - sum_{j>b} L_jb^T X_j).
// Each sweep is one persistent cooperative launch: CTA c owns block rows
// c, c + G, ... and consumes the solved blocks of other CTAs as their flags
// appear.  All CTAs are co-resident (cooperative launch), so every wait ends;
// each wait is also bounded and reports GBEM_ERR_TIMEOUT through a status word
// instead of spinning forever.
#include <atomic>

#include "bounded_wait.cuh"
#include "gbem_internal.h"

namespace {

constexpr int NB = 64;
constexpr int MAXR = 16;          // right-hand sides per pass

std::atomic<unsigned> g_epoch{1};

__device__ __forceinline__ unsigned load_acquire(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void store_release(unsigned* p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Thread 0 waits until flag == epoch (bounded in wall-clock time); the CTA
// then proceeds together.  Returns false if the wait gave up (status set).
__device__ bool wait_flag(const unsigned* flag, unsigned epoch, int* status, int* s_ok)
{
    if (threadIdx.x == 0) {
        bw::Deadline dl(bw::kDependencyNs);
        int ok = 1;
        while (load_acquire(flag) != epoch) {
            if (dl.expired() || atomicAdd(status, 0) != 0) {
                atomicCAS(status, 0, (int)GBEM_ERR_TIMEOUT);
                ok = 0;
                break;
            }
            __nanosleep(32);
        }
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

template <typename T, int R>
struct SweepSmem {
    T iv[NB][NB + 1];      // diagonal-block inverse
    T v[NB][R];            // solved block of another row (Y_j or X_j)
    T part[4][NB][R];      // partial sums of the four column quarters
    T w[NB][R];            // right-hand side block of this row, then the result
    int ok;
};

// Forward sweep on right-hand-side columns [0, nr) of W (np x nrhs, col-major).
// Per block row, everything that does not depend on other blocks -- the
// diagonal-block inverse, the right-hand side and the next L tile -- is
// loaded before the CTA waits, so only the solved block crosses the critical
// path.
template <typename T, int R>
__global__ void __launch_bounds__(256) trsv_fwd(const T* __restrict__ L, const T* __restrict__ Linv, int np,
                                                const T* __restrict__ W, T* __restrict__ Y, int nr,
                                                unsigned* sync, unsigned epoch, int* status, const int* done)
{
    if (done && *done) return;
    extern __shared__ unsigned char smem_raw[];
    SweepSmem<T, R>& S = *reinterpret_cast<SweepSmem<T, R>*>(smem_raw);
    const int tid = threadIdx.x;
    const int r = tid & (NB - 1), q = tid >> 6;   // row of the block, column quarter
    const int nblk = np / NB;
    constexpr int QW = NB / 4;
    for (int b = blockIdx.x; b < nblk; b += gridDim.x) {
        const int b0 = b * NB;
        for (int e = tid; e < NB * NB; e += blockDim.x) S.iv[e % NB][e / NB] = Linv[(size_t)b * NB * NB + e];
        T rhs[R];
#pragma unroll
        for (int c = 0; c < R; ++c) rhs[c] = (q == 0 && c < nr) ? W[(size_t)(b0 + r) + (size_t)c * np] : T(0);
        T acc[R];
#pragma unroll
        for (int c = 0; c < R; ++c) acc[c] = T(0);
        T lnext[QW];
        if (b > 0)
#pragma unroll
            for (int tt = 0; tt < QW; ++tt) lnext[tt] = L[(size_t)(b0 + r) + (size_t)(q * QW + tt) * np];
        for (int j = 0; j < b; ++j) {
            T lcur[QW];
#pragma unroll
            for (int tt = 0; tt < QW; ++tt) lcur[tt] = lnext[tt];
            if (j + 1 < b)
#pragma unroll
                for (int tt = 0; tt < QW; ++tt)
                    lnext[tt] = L[(size_t)(b0 + r) + (size_t)((j + 1) * NB + q * QW + tt) * np];
            if (!wait_flag(sync + j, epoch, status, &S.ok)) return;
            const int j0 = j * NB;
            for (int e = tid; e < NB * R; e += blockDim.x) {
                const int t = e % NB, c = e / NB;
                S.v[t][c] = (c < nr) ? __ldcg(Y + (size_t)(j0 + t) + (size_t)c * np) : T(0);
            }
            __syncthreads();
#pragma unroll
            for (int tt = 0; tt < QW; ++tt) {
                const int t = q * QW + tt;
#pragma unroll
                for (int c = 0; c < R; ++c) acc[c] += lcur[tt] * S.v[t][c];
            }
            __syncthreads();
        }
        // w = W_b - sum of the four partial sums; Y_b = Linv_bb w
#pragma unroll
        for (int c = 0; c < R; ++c) S.part[q][r][c] = acc[c];
        if (q == 0)
#pragma unroll
            for (int c = 0; c < R; ++c) S.w[r][c] = rhs[c];
        __syncthreads();
        for (int e = tid; e < NB * R; e += blockDim.x) {
            const int t = e % NB, c = e / NB;
            S.w[t][c] -= ((S.part[0][t][c] + S.part[1][t][c]) + S.part[2][t][c]) + S.part[3][t][c];
        }
        __syncthreads();
        for (int e = tid; e < NB * R; e += blockDim.x) {
            const int t = e % NB, c = e / NB;
            if (c >= nr) continue;
            T sum = T(0);
            for (int k = 0; k <= t; ++k) sum += S.iv[t][k] * S.w[k][c];
            Y[(size_t)(b0 + t) + (size_t)c * np] = sum;
        }
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            store_release(sync + b, epoch);
        }
    }
}

// Backward sweep: X = L^-T Y, written into W; block rows in falling order.
template <typename T, int R>
__global__ void __launch_bounds__(256) trsv_bwd(const T* __restrict__ L, const T* __restrict__ Linv, int np,
                                                const T* __restrict__ Y, T* __restrict__ X, int nr,
                                                unsigned* sync, unsigned epoch, int* status, const int* done)
{
    if (done && *done) return;
    extern __shared__ unsigned char smem_raw[];
    SweepSmem<T, R>& S = *reinterpret_cast<SweepSmem<T, R>*>(smem_raw);
    const int tid = threadIdx.x;
    const int r = tid & (NB - 1), q = tid >> 6;
    const int nblk = np / NB;
    constexpr int QW = NB / 4;
    for (int b = nblk - 1 - blockIdx.x; b >= 0; b -= gridDim.x) {
        const int b0 = b * NB;
        for (int e = tid; e < NB * NB; e += blockDim.x) S.iv[e % NB][e / NB] = Linv[(size_t)b * NB * NB + e];
        T rhs[R];
#pragma unroll
        for (int c = 0; c < R; ++c) rhs[c] = (q == 0 && c < nr) ? Y[(size_t)(b0 + r) + (size_t)c * np] : T(0);
        T acc[R];
#pragma unroll
        for (int c = 0; c < R; ++c) acc[c] = T(0);
        // row r of L_jb^T is column (b0 + r) of L, rows j0 + q * 16 ..
        const T* col = L + (size_t)(b0 + r) * np + q * QW;
        T lnext[QW];
        if (b < nblk - 1)
#pragma unroll
            for (int tt = 0; tt < QW; ++tt) lnext[tt] = col[(size_t)(nblk - 1) * NB + tt];
        for (int j = nblk - 1; j > b; --j) {
            T lcur[QW];
#pragma unroll
            for (int tt = 0; tt < QW; ++tt) lcur[tt] = lnext[tt];
            if (j - 1 > b)
#pragma unroll
                for (int tt = 0; tt < QW; ++tt) lnext[tt] = col[(size_t)(j - 1) * NB + tt];
            if (!wait_flag(sync + j, epoch, status, &S.ok)) return;
            const int j0 = j * NB;
            for (int e = tid; e < NB * R; e += blockDim.x) {
                const int t = e % NB, c = e / NB;
                S.v[t][c] = (c < nr) ? __ldcg(X + (size_t)(j0 + t) + (size_t)c * np) : T(0);
            }
            __syncthreads();
#pragma unroll
            for (int tt = 0; tt < QW; ++tt) {
#pragma unroll
                for (int c = 0; c < R; ++c) acc[c] += lcur[tt] * S.v[q * QW + tt][c];
            }
            __syncthreads();
        }
#pragma unroll
        for (int c = 0; c < R; ++c) S.part[q][r][c] = acc[c];
        if (q == 0)
#pragma unroll
            for (int c = 0; c < R; ++c) S.w[r][c] = rhs[c];
        __syncthreads();
        for (int e = tid; e < NB * R; e += blockDim.x) {
            const int t = e % NB, c = e / NB;
            S.w[t][c] -= ((S.part[0][t][c] + S.part[1][t][c]) + S.part[2][t][c]) + S.part[3][t][c];
        }
        __syncthreads();
        for (int e = tid; e < NB * R; e += blockDim.x) {
            const int t = e % NB, c = e / NB;
            if (c >= nr) continue;
            T sum = T(0);
            for (int k = t; k < NB; ++k) sum += S.iv[k][t] * S.w[k][c];
            X[(size_t)(b0 + t) + (size_t)c * np] = sum;
        }
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            store_release(sync + b, epoch);
        }
    }
}

// ---- FP32 sweeps with self-validating data.  A solved block is published
// as 64-bit words (epoch << 32 | value bits), each single-copy atomic, so a
// consumer polls the words it needs until they carry this launch's epoch:
// one L2 round trip instead of a flag, a fence and a second load.

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Waits for the tagged word and returns its value; gives up, setting status,
// after a second of wall-clock time or once another wait has given up.
__device__ __forceinline__ float poll_tagged(const unsigned long long* p, unsigned epoch, int* status)
{
    bw::Deadline dl(bw::kDependencyNs);
    for (;;) {
        const unsigned long long w = ld_relaxed_u64(p);
        if ((unsigned)(w >> 32) == epoch) return __uint_as_float((unsigned)w);
        if (dl.expired() || *(volatile int*)status != 0) {
            atomicCAS(status, 0, (int)GBEM_ERR_TIMEOUT);
            return 0.0f;
        }
    }
}

__device__ __forceinline__ unsigned long long tagged(float v, unsigned epoch)
{
    return ((unsigned long long)epoch << 32) | __float_as_uint(v);
}

// The 64 x R tagged block of rows j0 .. j0 + 63 (columns c < nr; zero for
// c >= nr) into shared memory at dst(t, c), 256 threads.  Every thread issues
// its R / 4 loads at once and polls again only the words not yet tagged with
// this epoch, so a block that is ready costs one L2 round trip, not R / 4.
template <int R, typename Dst>
__device__ __forceinline__ void load_tagged_block(const unsigned long long* __restrict__ tag, int j0, int np, int nr,
                                                  unsigned epoch, int* status, Dst dst)
{
    constexpr int K = NB * R / 256;
    static_assert(K * 256 == NB * R, "R a multiple of 4");
    const int tid = threadIdx.x;
    unsigned long long w[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int e = tid + 256 * k, t = e % NB, c = e / NB;
        w[k] = c < nr ? ld_relaxed_u64(tag + (size_t)(j0 + t) + (size_t)c * np) : 0ull;
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int e = tid + 256 * k, t = e % NB, c = e / NB;
        float v = 0.f;
        if (c < nr)
            v = ((unsigned)(w[k] >> 32) == epoch) ? __uint_as_float((unsigned)w[k])
                                                   : poll_tagged(tag + (size_t)(j0 + t) + (size_t)c * np, epoch, status);
        dst(t, c) = v;
    }
}

// acc += aj with Kahan compensation: a thread sums one 16-term product per
// earlier block, so the long sum over blocks carries no rounding drift into
// the solve (the refinement's contraction, about the square of the solve's
// error per two iterations, depends on it).
template <int R>
__device__ __forceinline__ void kahan_add(float (&acc)[R], float (&comp)[R], const float (&aj)[R])
{
#pragma unroll
    for (int c = 0; c < R; ++c) {
        const float y = __fsub_rn(aj[c], comp[c]);
        const float t = __fadd_rn(acc[c], y);
        comp[c] = __fsub_rn(__fsub_rn(t, acc[c]), y);
        acc[c] = t;
    }
}

// Shared memory of the FP32 sweeps.  Per block row b the solution is split
// as x_b = z_b - M_b x_p, with p the neighbouring row solved just before
// (b - 1 forward, b + 1 backward), M_b = Linv_b L_bp (forward) or
// Linv_b^T L_pb^T (backward), and z_b the inverse applied to the right-hand
// side minus the compensated sum over every other earlier row.  M_b and z_b
// are ready before x_p arrives, so the critical path from one row to the
// next is one polled block and one 64-term dot product per output.  The row
// of M_b a thread needs is held in its registers, and the vectors are laid
// out so that a thread reads four of them with one 16-byte shared load (all
// lanes of a warp read the same address).
constexpr int SG = 2;          // earlier blocks taken per step of a sweep's sum
template <int R>
struct SweepF32Smem {
    float v[SG][NB][R];        // solved blocks of other rows, v[g][t][c]
    float part[4][NB][R];      // partial sums of the four column quarters
    float wT[R][NB];           // right-hand side minus the sums, wT[c][k]
    float vT[R][NB];           // the neighbouring row's solved block, vT[c][k]
    float lp[NB][NB + 4];      // L_bp (forward: lp[j][k] = L_bp[j][k]; backward: lp[j][k] = L_pb[k][j])
    float m[NB][NB + 4];       // M_b, m[t][k]
    float iv[NB][NB + 4];      // the inverse (forward) or its transpose (backward), iv[t][k]
};
template <int R>
struct SweepBwdSmem {
    SweepF32Smem<R> base;
    float lt[SG][NB][NB + 1];  // lt[g][r][t] = L[j0 + t][b0 + r] of block g
};

// sum_k li[k] w[k] with w in shared memory (16-byte aligned), four chains
__device__ __forceinline__ float dot64(const float (&li)[NB], const float* __restrict__ w)
{
    float a[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < NB; k += 4) {
        const float4 x = *reinterpret_cast<const float4*>(w + k);
        a[0] = fmaf(li[k], x.x, a[0]);
        a[1] = fmaf(li[k + 1], x.y, a[1]);
        a[2] = fmaf(li[k + 2], x.z, a[2]);
        a[3] = fmaf(li[k + 3], x.w, a[3]);
    }
    return (a[0] + a[1]) + (a[2] + a[3]);
}

// sum_k a[k] w[k] for two 16-byte aligned rows of shared memory
__device__ __forceinline__ float dot64s(const float* __restrict__ a, const float* __restrict__ w)
{
    float s4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < NB; k += 4) {
        const float4 x = *reinterpret_cast<const float4*>(a + k);
        const float4 y = *reinterpret_cast<const float4*>(w + k);
        s4[0] = fmaf(x.x, y.x, s4[0]);
        s4[1] = fmaf(x.y, y.y, s4[1]);
        s4[2] = fmaf(x.z, y.z, s4[2]);
        s4[3] = fmaf(x.w, y.w, s4[3]);
    }
    return (s4[0] + s4[1]) + (s4[2] + s4[3]);
}

// aj[c] += l * v[c] for c < R, v 16-byte aligned
template <int R>
__device__ __forceinline__ void axpy_row(float (&aj)[R], float l, const float* __restrict__ v)
{
#pragma unroll
    for (int c = 0; c < R; c += 4) {
        const float4 x = *reinterpret_cast<const float4*>(v + c);
        aj[c] = fmaf(l, x.x, aj[c]);
        if (c + 1 < R) aj[c + 1] = fmaf(l, x.y, aj[c + 1]);
        if (c + 2 < R) aj[c + 2] = fmaf(l, x.z, aj[c + 2]);
        if (c + 3 < R) aj[c + 3] = fmaf(l, x.w, aj[c + 3]);
    }
}

// Row r of M_b into mrow: m[r][k] = sum_j iv[r][j] lp[j][k] (the caller has
// filled iv and lp); thread (r, q) forms the 16 columns of quarter q, then
// every thread reads its whole row back.
__device__ __forceinline__ void form_m(float (*m)[NB + 4], const float (*lp)[NB + 4], const float (*iv)[NB + 4],
                                       float (&mrow)[NB])
{
    const int tid = threadIdx.x;
    const int r = tid & (NB - 1), q = tid >> 6;
    float a[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) a[i] = 0.f;
    for (int j0 = 0; j0 < NB; j0 += 4) {
        const float4 l4 = *reinterpret_cast<const float4*>(&iv[r][j0]);
        const float ls[4] = {l4.x, l4.y, l4.z, l4.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float l = ls[u];
#pragma unroll
            for (int i = 0; i < 16; i += 4) {
                const float4 x = *reinterpret_cast<const float4*>(&lp[j0 + u][16 * q + i]);
                a[i] = fmaf(l, x.x, a[i]);
                a[i + 1] = fmaf(l, x.y, a[i + 1]);
                a[i + 2] = fmaf(l, x.z, a[i + 2]);
                a[i + 3] = fmaf(l, x.w, a[i + 3]);
            }
        }
    }
#pragma unroll
    for (int i = 0; i < 16; i += 4)
        *reinterpret_cast<float4*>(&m[r][16 * q + i]) = make_float4(a[i], a[i + 1], a[i + 2], a[i + 3]);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NB; k += 4) {
        const float4 x = *reinterpret_cast<const float4*>(&m[r][k]);
        mrow[k] = x.x, mrow[k + 1] = x.y, mrow[k + 2] = x.z, mrow[k + 3] = x.w;
    }
}

// z_b for thread (t = r, c = q + 4 i): acc (this thread's compensated sum
// for row r, quarter q) and rhs (row r's right-hand side, held by quarter 0)
// give w = rhs - sum over quarters in wT; then z = iv[r] . w.
template <int R>
__device__ __forceinline__ void form_z(SweepF32Smem<R>& S, const float (&acc)[R], const float (&rhs)[R],
                                       float (&z)[(R + 3) / 4])
{
    const int tid = threadIdx.x;
    const int r = tid & (NB - 1), q = tid >> 6;
#pragma unroll
    for (int c = 0; c < R; ++c) S.part[q][r][c] = acc[c];
    if (q == 0)
#pragma unroll
        for (int c = 0; c < R; ++c) S.wT[c][r] = rhs[c];
    __syncthreads();
    for (int c = q; c < R; c += 4)
        S.wT[c][r] -= ((S.part[0][r][c] + S.part[1][r][c]) + S.part[2][r][c]) + S.part[3][r][c];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < (R + 3) / 4; ++i) z[i] = (q + 4 * i < R) ? dot64s(&S.iv[r][0], &S.wT[q + 4 * i][0]) : 0.f;
}

// The last step of a row: wait for the neighbouring row p's solved block
// (skipped when there is none), x = z - M_b x_p, publish x.
template <int R>
__device__ __forceinline__ void finish_row(SweepF32Smem<R>& S, const float (&z)[(R + 3) / 4],
                                           const float (&mrow)[NB], bool has_p, int p0, int b0, int np, int nr,
                                           unsigned epoch, unsigned long long* __restrict__ tag,
                                           float* __restrict__ out, int* status)
{
    const int tid = threadIdx.x;
    const int r = tid & (NB - 1), q = tid >> 6;
    if (has_p) {
        load_tagged_block<R>(tag, p0, np, nr, epoch, status, [&](int t, int c) -> float& { return S.vT[c][t]; });
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < (R + 3) / 4; ++i) {
        const int c = q + 4 * i;
        if (c >= nr) break;
        const float y = has_p ? z[i] - dot64(mrow, &S.vT[c][0]) : z[i];
        const size_t idx = (size_t)(b0 + r) + (size_t)c * np;
        tag[idx] = tagged(y, epoch);
        out[idx] = y;
    }
}

// Forward sweep Y = L^-1 W on columns [0, nr) (FP32).
template <int R>
__global__ void __launch_bounds__(256) sweep_fwd_f32(const float* __restrict__ L, const float* __restrict__ Linv,
                                                     int np, const float* __restrict__ W, float* __restrict__ Y,
                                                     unsigned long long* __restrict__ tag, int nr, unsigned epoch,
                                                     int* status, const int* done)
{
    if (done && *done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SweepF32Smem<R>& S = *reinterpret_cast<SweepF32Smem<R>*>(smem_raw);
    const int tid = threadIdx.x;
    const int r = tid & (NB - 1), q = tid >> 6;   // row of the block, column quarter
    const int nblk = np / NB;
    constexpr int QW = NB / 4;
    for (int b = blockIdx.x; b < nblk; b += gridDim.x) {
        const int b0 = b * NB;
        // the diagonal-block inverse (stored column-major, zeros above), iv[t][k]
        for (int e = tid; e < NB * NB; e += blockDim.x) S.iv[e % NB][e / NB] = Linv[(size_t)b * NB * NB + e];
        float rhs[R], acc[R], comp[R];
#pragma unroll
        for (int c = 0; c < R; ++c) {
            rhs[c] = (q == 0 && c < nr) ? W[(size_t)(b0 + r) + (size_t)c * np] : 0.f;
            acc[c] = comp[c] = 0.f;
        }
        // M_b = Linv_b L_b,b-1, row r
        float mrow[NB];
        if (b > 0) {
            for (int e = tid; e < NB * NB; e += blockDim.x) {
                const int j = e % NB, k = e / NB;
                S.lp[j][k] = L[(size_t)(b0 + j) + (size_t)(b0 - NB + k) * np];
            }
            __syncthreads();
            form_m(S.m, S.lp, S.iv, mrow);
        } else {
            __syncthreads();   // iv complete
        }
        // the compensated sum over rows j < b - 1, SG blocks a step: this
        // thread's L_bj entries and the solved blocks are loaded together
        for (int j = 0; j + 1 < b; j += SG) {
            const int gn = min(SG, b - 1 - j);
            float lc[SG][QW];
#pragma unroll
            for (int g = 0; g < SG; ++g)
                if (g < gn)
#pragma unroll
                    for (int tt = 0; tt < QW; ++tt)
                        lc[g][tt] = L[(size_t)(b0 + r) + (size_t)((j + g) * NB + q * QW + tt) * np];
#pragma unroll
            for (int g = 0; g < SG; ++g)
                if (g < gn)
                    load_tagged_block<R>(tag, (j + g) * NB, np, nr, epoch, status,
                                         [&](int t, int c) -> float& { return S.v[g][t][c]; });
            __syncthreads();
            float aj[R];
#pragma unroll
            for (int c = 0; c < R; ++c) aj[c] = 0.f;
#pragma unroll
            for (int g = 0; g < SG; ++g)
                if (g < gn)
#pragma unroll
                    for (int tt = 0; tt < QW; ++tt) axpy_row<R>(aj, lc[g][tt], &S.v[g][q * QW + tt][0]);
            kahan_add(acc, comp, aj);
            __syncthreads();
        }
        float z[(R + 3) / 4];
        form_z<R>(S, acc, rhs, z);
        finish_row<R>(S, z, mrow, b > 0, b0 - NB, b0, np, nr, epoch, tag, Y, status);
        __syncthreads();
    }
}

// Backward sweep X = L^-T Y, written into X; block rows in falling order.
// Block (j, b) of L is read along its columns (coalesced) into registers one
// step ahead and staged through shared memory as its transpose.
template <int R>
__global__ void __launch_bounds__(256) sweep_bwd_f32(const float* __restrict__ L, const float* __restrict__ Linv,
                                                     int np, const float* __restrict__ Y, float* __restrict__ X,
                                                     unsigned long long* __restrict__ tag, int nr, unsigned epoch,
                                                     int* status, const int* done)
{
    if (done && *done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SweepBwdSmem<R>& SB = *reinterpret_cast<SweepBwdSmem<R>*>(smem_raw);
    SweepF32Smem<R>& S = SB.base;
    const int tid = threadIdx.x;
    const int r = tid & (NB - 1), q = tid >> 6;
    const int nblk = np / NB;
    constexpr int QW = NB / 4;
    for (int b = nblk - 1 - blockIdx.x; b >= 0; b -= gridDim.x) {
        const int b0 = b * NB;
        // the transpose of the diagonal-block inverse, iv[t][k] = Linv[k][t]
        for (int e = tid; e < NB * NB; e += blockDim.x) S.iv[e / NB][e % NB] = Linv[(size_t)b * NB * NB + e];
        float rhs[R], acc[R], comp[R];
#pragma unroll
        for (int c = 0; c < R; ++c) {
            rhs[c] = (q == 0 && c < nr) ? Y[(size_t)(b0 + r) + (size_t)c * np] : 0.f;
            acc[c] = comp[c] = 0.f;
        }
        // M_b = Linv_b^T L_b+1,b^T, row r: m[r][k] = sum_j Linv[j][r] L_b+1,b[k][j]
        float mrow[NB];
        if (b < nblk - 1) {
            for (int e = tid; e < NB * NB; e += blockDim.x) {
                const int k = e % NB, j = e / NB;
                S.lp[j][k] = L[(size_t)(b0 + NB + k) + (size_t)(b0 + j) * np];
            }
            __syncthreads();
            form_m(S.m, S.lp, S.iv, mrow);
        } else {
            __syncthreads();   // iv complete
        }
        // the compensated sum over rows j > b + 1, SG blocks a step (falling
        // j): thread tid reads L[j0 + (tid & 63)][b0 + (tid >> 6) + 4 k],
        // k < 16, of each block (coalesced along the columns) into lt
        const float* colb = L + (size_t)(tid & 63) + (size_t)(b0 + (tid >> 6)) * np;
        for (int j = nblk - 1; j > b + 1; j -= SG) {
            const int gn = min(SG, j - b - 1);
            float lc[SG][QW];
#pragma unroll
            for (int g = 0; g < SG; ++g)
                if (g < gn)
#pragma unroll
                    for (int k = 0; k < QW; ++k) lc[g][k] = colb[(size_t)(j - g) * NB + (size_t)(4 * k) * np];
#pragma unroll
            for (int g = 0; g < SG; ++g)
                if (g < gn)
                    load_tagged_block<R>(tag, (j - g) * NB, np, nr, epoch, status,
                                         [&](int t, int c) -> float& { return S.v[g][t][c]; });
#pragma unroll
            for (int g = 0; g < SG; ++g)
                if (g < gn)
#pragma unroll
                    for (int k = 0; k < QW; ++k) SB.lt[g][(tid >> 6) + 4 * k][tid & 63] = lc[g][k];
            __syncthreads();
            float aj[R];
#pragma unroll
            for (int c = 0; c < R; ++c) aj[c] = 0.f;
#pragma unroll
            for (int g = 0; g < SG; ++g)
                if (g < gn)
#pragma unroll
                    for (int tt = 0; tt < QW; ++tt)
                        axpy_row<R>(aj, SB.lt[g][r][q * QW + tt], &S.v[g][q * QW + tt][0]);
            kahan_add(acc, comp, aj);
            __syncthreads();
        }
        float z[(R + 3) / 4];
        form_z<R>(S, acc, rhs, z);
        finish_row<R>(S, z, mrow, b < nblk - 1, b0 + NB, b0, np, nr, epoch, tag, X, status);
        __syncthreads();
    }
}

template <typename K>
int coop_grid(K kernel, size_t smem, int nblk)
{
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, 256, smem) != cudaSuccess) {
        cudaGetLastError();
        per = 1;
    }
    return std::max(1, std::min(nblk, std::max(1, per) * sms));
}

template <typename T, int R>
cudaError_t sweep_pair(const T* L, const T* Linv, int np, T* W, T* Y, int nr, unsigned* sync, int* status,
                       const int* done, cudaStream_t s)
{
    const size_t smem = sizeof(SweepSmem<T, R>);
    const int nblk = np / NB;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(trsv_fwd<T, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
            cudaSuccess ||
        (e = cudaFuncSetAttribute(trsv_bwd<T, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
            cudaSuccess)
        return e;
    unsigned e1 = g_epoch.fetch_add(2);
    if (e1 + 1 == 0) e1 = g_epoch.fetch_add(2);   // 0 marks a cleared flag
    unsigned e2 = e1 + 1;
    // one sweep reads the lower triangle of L and the diagonal-block
    // inverses once and the right-hand sides twice
    const double sweep_bytes =
        sizeof(T) * ((double)np * (np + NB) / 2 + (double)np * NB + 3.0 * np * nr);
    const double sweep_flops = (double)np * np * nr;
    {
        const T* Wc = W;
        int grid = coop_grid(trsv_fwd<T, R>, smem, nblk);
        void* args[] = {(void*)&L, (void*)&Linv, (void*)&np, (void*)&Wc, (void*)&Y, (void*)&nr,
                        (void*)&sync, (void*)&e1, (void*)&status, (void*)&done};
        cudaEvent_t ev = trace_begin(s);
        if ((e = cudaLaunchCooperativeKernel((void*)trsv_fwd<T, R>, grid, 256, args, smem, s)) != cudaSuccess)
            return e;
        count_launch();
        trace_end(GBEM_KERNEL_SWEEP, ev, s, sweep_bytes, sweep_flops);
    }
    {
        const T* Yc = Y;
        int grid = coop_grid(trsv_bwd<T, R>, smem, nblk);
        void* args[] = {(void*)&L, (void*)&Linv, (void*)&np, (void*)&Yc, (void*)&W, (void*)&nr,
                        (void*)&sync, (void*)&e2, (void*)&status, (void*)&done};
        cudaEvent_t ev = trace_begin(s);
        if ((e = cudaLaunchCooperativeKernel((void*)trsv_bwd<T, R>, grid, 256, args, smem, s)) != cudaSuccess)
            return e;
        count_launch();
        trace_end(GBEM_KERNEL_SWEEP, ev, s, sweep_bytes, sweep_flops);
    }
    return cudaSuccess;
}

template <int R>
cudaError_t sweep_pair_f32(const float* L, const float* Linv, int np, float* W, float* Y, unsigned long long* tag,
                           int nr, int* status, const int* done, cudaStream_t s)
{
    const size_t smem = sizeof(SweepF32Smem<R>), smem_b = sizeof(SweepBwdSmem<R>);
    const int nblk = np / NB;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(sweep_fwd_f32<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
            cudaSuccess ||
        (e = cudaFuncSetAttribute(sweep_bwd_f32<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_b)) !=
            cudaSuccess)
        return e;
    unsigned e1 = g_epoch.fetch_add(2);
    if (e1 == 0) e1 = g_epoch.fetch_add(2);   // 0 marks a cleared word
    unsigned e2 = e1 + 1;
    const double sweep_bytes = 4.0 * ((double)np * (np + NB) / 2 + (double)np * NB + 3.0 * np * nr);
    const double sweep_flops = (double)np * np * nr;
    {
        const float* Wc = W;
        int grid = coop_grid(sweep_fwd_f32<R>, smem, nblk);
        void* args[] = {(void*)&L, (void*)&Linv, (void*)&np, (void*)&Wc, (void*)&Y, (void*)&tag,
                        (void*)&nr, (void*)&e1, (void*)&status, (void*)&done};
        cudaEvent_t ev = trace_begin(s);
        if ((e = cudaLaunchCooperativeKernel((void*)sweep_fwd_f32<R>, grid, 256, args, smem, s)) != cudaSuccess)
            return e;
        count_launch();
        trace_end(GBEM_KERNEL_SWEEP, ev, s, sweep_bytes, sweep_flops);
    }
    {
        const float* Yc = Y;
        int grid = coop_grid(sweep_bwd_f32<R>, smem_b, nblk);
        void* args[] = {(void*)&L, (void*)&Linv, (void*)&np, (void*)&Yc, (void*)&W, (void*)&tag,
                        (void*)&nr, (void*)&e2, (void*)&status, (void*)&done};
        cudaEvent_t ev = trace_begin(s);
        if ((e = cudaLaunchCooperativeKernel((void*)sweep_bwd_f32<R>, grid, 256, args, smem_b, s)) != cudaSuccess)
            return e;
        count_launch();
        trace_end(GBEM_KERNEL_SWEEP, ev, s, sweep_bytes, sweep_flops);
    }
    return cudaSuccess;
}

// W (np x nrhs) := L^-T L^-1 W, with Y (same size) as work; sync holds one
// flag per 64-row block.
template <typename T>
cudaError_t trsv(const T* L, const T* Linv, int np, T* W, T* Y, int nrhs, unsigned* sync, int* status,
                 const int* done, cudaStream_t s)
{
    for (int c0 = 0; c0 < nrhs; c0 += MAXR) {
        const int nr = std::min(MAXR, nrhs - c0);
        T* Wc = W + (size_t)c0 * np;
        T* Yc = Y + (size_t)c0 * np;
        cudaError_t e;
        if (nr <= 4) e = sweep_pair<T, 4>(L, Linv, np, Wc, Yc, nr, sync, status, done, s);
        else if (nr <= 8) e = sweep_pair<T, 8>(L, Linv, np, Wc, Yc, nr, sync, status, done, s);
        else e = sweep_pair<T, 16>(L, Linv, np, Wc, Yc, nr, sync, status, done, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
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

// X += W, and X as an unevaluated float pair (hi + lo) for the compensated
// residual when Xdf is given.
__device__ __forceinline__ float2 split_df(double x)
{
    const float h = __double2float_rn(x);
    return make_float2(h, __double2float_rn(x - (double)h));
}

__global__ void add_f32(const float* __restrict__ W, size_t total, double* __restrict__ X,
                        float2* __restrict__ Xdf, const int* done)
{
    if (*done) return;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const double x = X[e] + (double)W[e];
        X[e] = x;
        if (Xdf) Xdf[e] = split_df(x);
    }
}

// R = B - A X with A symmetric, only its lower triangle stored.  A CTA owns 16
// rows and walks the 64-column blocks in order; blocks left of the diagonal
// are read directly, blocks right of it through the transpose (coalesced in
// both cases).  16 column groups per CTA and a fixed-order final sum keep the
// result independent of scheduling; small row blocks spread the FP64 work
// over every SM.
constexpr int RT = 16;
constexpr int CT = 64;
template <int RR>
__device__ __forceinline__ void residual_body(const double* __restrict__ A, int np, const double* __restrict__ Bp,
                                              const double* __restrict__ X, int nrhs, double* __restrict__ R,
                                              int blk)
{
    __shared__ double a[RT][CT + 1];
    __shared__ double xs[CT][RR + 1];
    __shared__ double part[8][RT][RR];
    const int tid = threadIdx.x;
    const int i0 = blk * RT;
    const int ri = tid % RT, grp = tid / RT;  // 16 column groups
    for (int c0 = 0; c0 < nrhs; c0 += RR) {
        const int nr = min(RR, nrhs - c0);
        double acc[RR];
#pragma unroll
        for (int c = 0; c < RR; ++c) acc[c] = 0.0;
        for (int j0 = 0; j0 < np; j0 += CT) {
            __syncthreads();
            // a[r][c] = A(i0 + r, j0 + c)
            if (j0 + CT <= i0) {
                for (int e = tid; e < RT * CT; e += blockDim.x) {
                    int r = e % RT, c = e / RT;
                    a[r][c] = A[(size_t)(i0 + r) + (size_t)(j0 + c) * np];
                }
            } else if (j0 >= i0 + RT) {
                for (int e = tid; e < RT * CT; e += blockDim.x) {
                    int c = e % CT, r = e / CT;
                    a[r][c] = A[(size_t)(j0 + c) + (size_t)(i0 + r) * np];
                }
            } else {
                for (int e = tid; e < RT * CT; e += blockDim.x) {
                    int r = e % RT, c = e / RT;
                    int gi = i0 + r, gj = j0 + c;
                    a[r][c] = A[(size_t)max(gi, gj) + (size_t)min(gi, gj) * np];
                }
            }
            for (int e = tid; e < CT * RR; e += blockDim.x) {
                int r = e % CT, c = e / CT;
                xs[r][c] = (c < nr) ? X[(size_t)(j0 + r) + (size_t)(c0 + c) * np] : 0.0;
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < CT / 16; ++q) {
                const int jj = grp + 16 * q;
                const double av = a[ri][jj];
#pragma unroll
                for (int c = 0; c < RR; ++c) acc[c] = fma(av, xs[jj][c], acc[c]);
            }
        }
        // the two column groups of a warp first, then 8 partial sums
#pragma unroll
        for (int c = 0; c < RR; ++c) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], 16);
        if ((grp & 1) == 0)
#pragma unroll
            for (int c = 0; c < RR; ++c) part[grp >> 1][ri][c] = acc[c];
        __syncthreads();
        for (int e = tid; e < RT * nr; e += blockDim.x) {
            int r = e % RT, c = e / RT;
            double s = 0.0;
            for (int g = 0; g < 8; ++g) s += part[g][r][c];
            size_t idx = (size_t)(i0 + r) + (size_t)(c0 + c) * np;
            R[idx] = Bp[idx] - s;
        }
        __syncthreads();
    }
}

// The same product with A and X stored as unevaluated float pairs
// (a = a.x + a.y, |a.y| <= ulp(a.x) / 2) and compensated FP32 arithmetic
// throughout (double-float: Dekker's product via FMA and Knuth's two-sum):
//   a x = a.x x.x + e + (a.x x.y + a.y x.x),  e = fma(a.x, x.x, -a.x x.x) exact,
// summed into (s, c) with s + p = s' + err exactly.  The dropped a.y x.y term
// and the FP32 rounding of the tail sums leave a relative error of a few
// 2^-48 per term; each thread folds its pair into an FP64 sum every 64 terms
// (residual_df_body), which keeps the residual accurate to about 1e-13 at
// any order.  The explicit _rn intrinsics keep the compiler from contracting
// the exact steps.
__device__ __forceinline__ void df_acc(float& s, float& c, float2 a, float2 x)
{
    const float p = __fmul_rn(a.x, x.x);
    const float e = __fmaf_rn(a.x, x.x, -p);
    const float t = __fmaf_rn(a.x, x.y, __fmul_rn(a.y, x.x));
    const float sn = __fadd_rn(s, p);
    const float bb = __fsub_rn(sn, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(sn, bb)), __fsub_rn(p, bb));
    s = sn;
    c = __fadd_rn(c, __fadd_rn(err, __fadd_rn(e, t)));
}

__device__ __forceinline__ void cp_async8(void* dst, const void* src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// The 64-column blocks of A and X stream through a STAGES-deep cp.async
// ring, so a CTA keeps several blocks of loads in flight while it computes.
template <int RR>
struct DfRes {
    static constexpr int STAGES = RR <= 8 ? 3 : 2;
    struct Ring {
        float2 a[STAGES][RT][CT + 1];
        float2 xs[STAGES][CT][RR + 1];
    };
    static constexpr size_t BYTES =
        sizeof(Ring) > sizeof(double) * 8 * RT * RR ? sizeof(Ring) : sizeof(double) * 8 * RT * RR;
};

// The refinement's convergence test folded into the residual: per column c
// the largest |R| and |B| (non-negative doubles ordered as their bit
// patterns) are combined with atomicMax into chk[2 c], chk[2 c + 1]; the last
// CTA of the launch (counted in chk[2 nrhs_all]) forms max_c |R|/|B|, stores
// it in norm[0], counts the iteration in flags[2], sets flags[1] if it is at
// most tol, and clears chk for the next call.
struct IrCheck {
    unsigned long long* chk = nullptr;   // 2 per column, then the CTA counter
    int col0 = 0;                         // this launch's first column
    int ncols = 0;                        // columns of every launch of the call
    bool finalize = false;                // the call's last launch: test and clear
    double* norm = nullptr;
    double tol = 0.0;
    int* flags = nullptr;
};

template <int RR>
__device__ __forceinline__ void residual_df_body(const float2* __restrict__ A, int np, const double* __restrict__ Bp,
                                                 const float2* __restrict__ X, int nrhs, double* __restrict__ R,
                                                 int blk, const IrCheck& ck)
{
    __shared__ unsigned long long smax[2][RR];
    constexpr int S = DfRes<RR>::STAGES;
    __shared__ __align__(16) unsigned char smem[DfRes<RR>::BYTES];
    auto& ring = *reinterpret_cast<typename DfRes<RR>::Ring*>(smem);
    auto part = reinterpret_cast<double(*)[RT][RR]>(smem);   // after the ring is drained
    const int tid = threadIdx.x;
    const int i0 = blk * RT;
    const int ri = tid % RT, grp = tid / RT;  // 16 column groups
    const int nblk = np / CT;
    for (int c0 = 0; c0 < nrhs; c0 += RR) {
        const int nr = min(RR, nrhs - c0);
        __syncthreads();   // the previous pass is done reading its partial sums
        if (tid < 2 * RR) smax[tid / RR][tid % RR] = 0ull;
        for (int e = tid; e < S * CT * RR; e += blockDim.x) {   // unused columns read as zero
            const int st = e / (CT * RR), r = (e / RR) % CT, c = e % RR;
            if (c >= nr) ring.xs[st][r][c] = make_float2(0.0f, 0.0f);
        }
        auto issue = [&](int jb) {
            const int st = jb % S, j0 = jb * CT;
            if (j0 + CT <= i0) {
                for (int e = tid; e < RT * CT; e += blockDim.x) {
                    int r = e % RT, c = e / RT;
                    cp_async8(&ring.a[st][r][c], A + (size_t)(i0 + r) + (size_t)(j0 + c) * np);
                }
            } else if (j0 >= i0 + RT) {
                for (int e = tid; e < RT * CT; e += blockDim.x) {
                    int c = e % CT, r = e / CT;
                    cp_async8(&ring.a[st][r][c], A + (size_t)(j0 + c) + (size_t)(i0 + r) * np);
                }
            } else {
                for (int e = tid; e < RT * CT; e += blockDim.x) {
                    int r = e % RT, c = e / RT;
                    int gi = i0 + r, gj = j0 + c;
                    cp_async8(&ring.a[st][r][c], A + (size_t)max(gi, gj) + (size_t)min(gi, gj) * np);
                }
            }
            for (int e = tid; e < CT * nr; e += blockDim.x) {
                int r = e % CT, c = e / CT;
                cp_async8(&ring.xs[st][r][c], X + (size_t)(j0 + r) + (size_t)(c0 + c) * np);
            }
        };
        __syncthreads();   // zeros written
#pragma unroll
        for (int q = 0; q < S - 1; ++q) {
            if (q < nblk) issue(q);
            cp_async_commit();
        }
        float sh[RR], sl[RR];
        double sd[RR];   // FP64 sum of the flushed float pairs
#pragma unroll
        for (int c = 0; c < RR; ++c) {
            sh[c] = sl[c] = 0.0f;
            sd[c] = 0.0;
        }
        for (int jb = 0; jb < nblk; ++jb) {
            if (jb + S - 1 < nblk) issue(jb + S - 1);
            cp_async_commit();
            cp_async_wait<S - 1>();   // block jb has landed (this thread's copies)
            __syncthreads();          // ... and every thread's
            const int st = jb % S;
#pragma unroll
            for (int q = 0; q < CT / 16; ++q) {
                const int jj = grp + 16 * q;
                const float2 av = ring.a[st][ri][jj];
#pragma unroll
                for (int c = 0; c < RR; ++c) df_acc(sh[c], sl[c], av, ring.xs[st][jj][c]);
            }
            // a float pair loses about 2^-48 of the partial sum per term: fold
            // it into FP64 every 64 terms, so the error stays near 1e-13 of
            // the largest partial sum whatever the order
            if ((jb & 15) == 15)
#pragma unroll
                for (int c = 0; c < RR; ++c) {
                    sd[c] += (double)sh[c] + (double)sl[c];
                    sh[c] = sl[c] = 0.0f;
                }
            __syncthreads();          // the stage is free for the copy issued next
        }
        cp_async_wait<0>();
        double acc[RR];
#pragma unroll
        for (int c = 0; c < RR; ++c) {
            acc[c] = sd[c] + ((double)sh[c] + (double)sl[c]);
            acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], 16);
        }
        __syncthreads();
        if ((grp & 1) == 0)
#pragma unroll
            for (int c = 0; c < RR; ++c) part[grp >> 1][ri][c] = acc[c];
        __syncthreads();
        for (int e = tid; e < RT * nr; e += blockDim.x) {
            int r = e % RT, c = e / RT;
            double sum = 0.0;
            for (int g = 0; g < 8; ++g) sum += part[g][r][c];
            size_t idx = (size_t)(i0 + r) + (size_t)(c0 + c) * np;
            const double b = Bp[idx], rv = b - sum;
            R[idx] = rv;
            if (ck.chk) {
                atomicMax(&smax[0][c], (unsigned long long)__double_as_longlong(fabs(rv)));
                atomicMax(&smax[1][c], (unsigned long long)__double_as_longlong(fabs(b)));
            }
        }
        if (ck.chk) {
            __syncthreads();
            if (tid < 2 * nr) {
                const int c = tid % nr, w = tid / nr;
                atomicMax(&ck.chk[2 * (ck.col0 + c0 + c) + w], smax[w][c]);
                __threadfence();   // performed before this CTA is counted
            }
        }
    }
    if (!ck.chk) return;
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        unsigned long long* counter = ck.chk + 2 * ck.ncols;
        if (atomicAdd(counter, 1ull) == (unsigned long long)gridDim.x - 1) {
            __threadfence();
            if (ck.finalize) {
                double worst = 0.0;
                for (int c = 0; c < ck.ncols; ++c) {
                    const double mr = __longlong_as_double((long long)atomicExch(&ck.chk[2 * c], 0ull));
                    const double mb = __longlong_as_double((long long)atomicExch(&ck.chk[2 * c + 1], 0ull));
                    worst = fmax(worst, (mb > 0.0) ? mr / mb : mr);
                }
                ck.norm[0] = worst;
                ck.flags[2] += 1;
                if (worst <= ck.tol) ck.flags[1] = 1;
            }
            *counter = 0ull;
        }
    }
}

template <int RR>
__global__ void __launch_bounds__(256) residual_df(const float2* __restrict__ A, int np,
                                                   const double* __restrict__ Bp, const float2* __restrict__ X,
                                                   int nrhs, double* __restrict__ R, const int* done, IrCheck ck)
{
    if (done && *done) return;
    residual_df_body<RR>(A, np, Bp, X, nrhs, R, blockIdx.x, ck);
}

template <int RR>
__global__ void __launch_bounds__(256) residual(const double* __restrict__ A, int np, const double* __restrict__ Bp,
                                                const double* __restrict__ X, int nrhs, double* __restrict__ R,
                                                const int* done)
{
    if (done && *done) return;
    residual_body<RR>(A, np, Bp, X, nrhs, R, blockIdx.x);
}

// max_k |R_k|_inf / |B_k|_inf -> norm[0]; converged -> flags[1] = 1, else
// flags[2] += 1 (iterations taken).
__device__ __forceinline__ double block_max_1024(double v, double* red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    v = red[threadIdx.x & 31];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    return v;
}

// One CTA of 1024 threads; each thread keeps eight loads in flight.
__global__ void __launch_bounds__(1024) ir_check(const double* __restrict__ R, const double* __restrict__ Bp,
                                                 int np, int nrhs, double* norm, double tol, int* flags)
{
    __shared__ double red[32];
    if (flags[1]) return;
    double worst = 0.0;
    for (int c = 0; c < nrhs; ++c) {
        const double* Rc = R + (size_t)c * np;
        const double* Bc = Bp + (size_t)c * np;
        double mr = 0.0, mb = 0.0;
        int r = threadIdx.x;
        for (; r + 3 * 1024 < np; r += 4 * 1024) {
            double a[4], b[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                a[q] = Rc[r + q * 1024];
                b[q] = Bc[r + q * 1024];
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                mr = fmax(mr, fabs(a[q]));
                mb = fmax(mb, fabs(b[q]));
            }
        }
        for (; r < np; r += 1024) {
            mr = fmax(mr, fabs(Rc[r]));
            mb = fmax(mb, fabs(Bc[r]));
        }
        mr = block_max_1024(mr, red);
        mb = block_max_1024(mb, red);
        worst = fmax(worst, (mb > 0.0) ? mr / mb : mr);
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

// ------------------------------------------------------------------ batches

// Right-hand sides (indicator of each conductor), X = 0, R = B, per structure.
__global__ void batch_begin(BatchView v)
{
    const int b = blockIdx.y;
    const int n = v.n[b], np = v.np[b], nc = v.nc[b];
    const int32_t* cond = v.cond + v.poff[b];
    const long long o = v.voff[b];
    const size_t total = (size_t)np * nc;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(e % np), k = (int)(e / np);
        const double bv = (r < n && cond[r] == k) ? 1.0 : 0.0;
        v.B[o + e] = bv;
        v.R[o + e] = bv;
        v.X[o + e] = 0.0;
    }
}

__global__ void batch_to_f32(const double* __restrict__ R, float* __restrict__ W, size_t total)
{
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x)
        W[e] = (float)R[e];
}

__global__ void batch_add(const float* __restrict__ W, double* __restrict__ X, float2* __restrict__ Xdf,
                          size_t total)
{
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const double x = X[e] + (double)W[e];
        X[e] = x;
        Xdf[e] = split_df(x);
    }
}

// W := L^-T L^-1 W for one structure per CTA: the block sweeps of the
// persistent solve, run by a single CTA so no CTA waits on another.
template <int R>
__global__ void __launch_bounds__(256) trsv_batched(BatchView v)
{
    const int b = blockIdx.x;
    const int np = v.np[b], nr = v.nc[b], nblk = np / NB;
    const float* __restrict__ L = v.A32 + v.moff[b];
    const float* __restrict__ Linv = v.Linv + v.ioff[b];
    float* W = v.W + v.voff[b];
    float* Y = v.Y + v.voff[b];
    __shared__ float iv[NB][NB + 1];
    __shared__ float sv[NB][R];
    __shared__ float part[4][NB][R];
    __shared__ float sw[NB][R];
    const int tid = threadIdx.x, r = tid & (NB - 1), q = tid >> 6;
    for (int dir = 0; dir < 2; ++dir) {
        const float* src = dir == 0 ? W : Y;   // right-hand side of this sweep
        float* dst = dir == 0 ? Y : W;          // its solution
        for (int s = 0; s < nblk; ++s) {
            const int bk = dir == 0 ? s : nblk - 1 - s;
            const int b0 = bk * NB;
            float acc[R];
#pragma unroll
            for (int c = 0; c < R; ++c) acc[c] = 0.f;
            for (int t2 = 0; t2 < s; ++t2) {
                const int j = dir == 0 ? t2 : nblk - 1 - t2;
                const int j0 = j * NB;
                for (int e = tid; e < NB * R; e += blockDim.x) {
                    const int t = e % NB, c = e / NB;
                    sv[t][c] = (c < nr) ? dst[(size_t)(j0 + t) + (size_t)c * np] : 0.f;
                }
                __syncthreads();
#pragma unroll
                for (int tt = 0; tt < NB / 4; ++tt) {
                    const int t = q * (NB / 4) + tt;
                    // forward: L[b0 + r][j0 + t]; backward: L[j0 + t][b0 + r]
                    const float l = dir == 0 ? L[(size_t)(b0 + r) + (size_t)(j0 + t) * np]
                                             : L[(size_t)(j0 + t) + (size_t)(b0 + r) * np];
#pragma unroll
                    for (int c = 0; c < R; ++c) acc[c] += l * sv[t][c];
                }
                __syncthreads();
            }
            for (int e = tid; e < NB * NB; e += blockDim.x) iv[e % NB][e / NB] = Linv[(size_t)bk * NB * NB + e];
#pragma unroll
            for (int c = 0; c < R; ++c) part[q][r][c] = acc[c];
            __syncthreads();
            for (int e = tid; e < NB * R; e += blockDim.x) {
                const int t = e % NB, c = e / NB;
                const float rhs = (c < nr) ? src[(size_t)(b0 + t) + (size_t)c * np] : 0.f;
                sw[t][c] = rhs - (((part[0][t][c] + part[1][t][c]) + part[2][t][c]) + part[3][t][c]);
            }
            __syncthreads();
            for (int e = tid; e < NB * R; e += blockDim.x) {
                const int t = e % NB, c = e / NB;
                if (c >= nr) continue;
                float sum = 0.f;
                if (dir == 0)
                    for (int k = 0; k <= t; ++k) sum += iv[t][k] * sw[k][c];
                else
                    for (int k = t; k < NB; ++k) sum += iv[k][t] * sw[k][c];
                dst[(size_t)(b0 + t) + (size_t)c * np] = sum;
            }
            __syncthreads();
        }
    }
}

// R = B - A X over every 16-row block of every structure.
template <int RR>
__global__ void __launch_bounds__(256) residual_batched(BatchView v)
{
    __shared__ int sb;
    if (threadIdx.x == 0) sb = batch_find(v.rows_prefix, v.nb, (long long)blockIdx.x);
    __syncthreads();
    const int b = sb;
    const long long o = v.voff[b];
    residual_df_body<RR>(reinterpret_cast<const float2*>(v.A64) + v.moff[b], v.np[b], v.B + o, v.Xdf + o, v.nc[b],
                         v.R + o, (int)(blockIdx.x - v.rows_prefix[b]), IrCheck{});
}

// Final relative residual and capacitance of each structure (one CTA each).
__global__ void batch_finish(BatchView v, double scale)
{
    const int b = blockIdx.x;
    const int n = v.n[b], np = v.np[b], nc = v.nc[b];
    const long long o = v.voff[b];
    const int32_t* cond = v.cond + v.poff[b];
    __shared__ double red[256];
    double worst = 0.0;
    for (int c = 0; c < nc; ++c) {
        double m = 0.0;
        for (int r = threadIdx.x; r < np; r += blockDim.x) m = fmax(m, fabs(v.R[o + r + (size_t)c * np]));
        red[threadIdx.x] = m;
        __syncthreads();
        for (int w = 128; w > 0; w >>= 1) {
            if (threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
            __syncthreads();
        }
        worst = fmax(worst, red[0]);   // |B_c|_inf = 1 for an indicator right-hand side
        __syncthreads();
    }
    if (threadIdx.x == 0) v.resid[b] = worst;
    for (int mk = 0; mk < nc * nc; ++mk) {
        const int m = mk / nc, k = mk % nc;
        double sum = 0.0;
        for (int i = threadIdx.x; i < n; i += blockDim.x)
            if (cond[i] == m) sum += v.X[o + i + (size_t)k * np];
        red[threadIdx.x] = sum;
        __syncthreads();
        for (int w = 128; w > 0; w >>= 1) {
            if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) v.C[v.coff[b] + mk] = scale * red[0];
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_trsv_f64(const double* L, const double* Linv, int np, int nb, double* W, int nrhs,
                            unsigned* sync, int* status, cudaStream_t s)
{
    if (nb != NB || nrhs <= 0) return cudaErrorInvalidValue;
    // Y shares the tail of W's allocation: W holds 2 * np * nrhs entries
    return trsv<double>(L, Linv, np, W, W + (size_t)np * nrhs, nrhs, sync, status, nullptr, s);
}

cudaError_t launch_trsv_f32_guarded(const float* L, const float* Linv, int np, int nb, float* W,
                                    int nrhs, unsigned* sync, int* status, const int* done, cudaStream_t s)
{
    if (nb != NB || nrhs <= 0) return cudaErrorInvalidValue;
    (void)sync;
    float* Y = W + (size_t)np * nrhs;
    unsigned long long* tag = reinterpret_cast<unsigned long long*>(W + 2 * (size_t)np * nrhs);
    // no stale word may carry a live epoch (epochs are never 0)
    cudaError_t ez = cudaMemsetAsync(tag, 0, sizeof(unsigned long long) * (size_t)np * nrhs, s);
    if (ez != cudaSuccess) return ez;
    for (int c0 = 0; c0 < nrhs; c0 += MAXR) {
        const int nr = std::min(MAXR, nrhs - c0);
        float* Wc = W + (size_t)c0 * np;
        float* Yc = Y + (size_t)c0 * np;
        unsigned long long* Tc = tag + (size_t)c0 * np;
        cudaError_t e;
        if (nr <= 4) e = sweep_pair_f32<4>(L, Linv, np, Wc, Yc, Tc, nr, status, done, s);
        else if (nr <= 8) e = sweep_pair_f32<8>(L, Linv, np, Wc, Yc, Tc, nr, status, done, s);
        else e = sweep_pair_f32<16>(L, Linv, np, Wc, Yc, Tc, nr, status, done, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
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

cudaError_t launch_add_f32(const float* W, int np, int nrhs, double* X, float2* Xdf, const int* done,
                           cudaStream_t s)
{
    size_t total = (size_t)np * nrhs;
    add_f32<<<grid_for(total), 256, 0, s>>>(W, total, X, Xdf, done);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_residual(const double* A, int np, const double* Bp, const double* X, int nrhs,
                            double* R, const int* done, cudaStream_t s)
{
    if (np % CT) return cudaErrorInvalidValue;
    for (int c0 = 0; c0 < nrhs; c0 += MAXR) {
        const int nr = std::min(MAXR, nrhs - c0);
        const double* Bc = Bp + (size_t)c0 * np;
        const double* Xc = X + (size_t)c0 * np;
        double* Rc = R + (size_t)c0 * np;
        cudaEvent_t ev = trace_begin(s);
        if (nr <= 4) residual<4><<<np / RT, 256, 0, s>>>(A, np, Bc, Xc, nr, Rc, done);
        else if (nr <= 8) residual<8><<<np / RT, 256, 0, s>>>(A, np, Bc, Xc, nr, Rc, done);
        else residual<16><<<np / RT, 256, 0, s>>>(A, np, Bc, Xc, nr, Rc, done);
        count_launch();
        // the lower triangle of A64 once, B and X read and R written; each
        // lower entry serves two products per right-hand side
        trace_end(GBEM_KERNEL_RESIDUAL, ev, s, 8.0 * ((double)np * (np + CT) / 2 + 3.0 * np * nr),
                  2.0 * (double)np * np * nr);
    }
    return cudaGetLastError();
}

cudaError_t launch_residual_df(const float2* A, int np, const double* Bp, const float2* Xdf, int nrhs,
                               double* R, const int* done, cudaStream_t s, unsigned long long* chk, double* norm,
                               double tol, int* flags)
{
    if (np % CT) return cudaErrorInvalidValue;
    for (int c0 = 0; c0 < nrhs; c0 += MAXR) {
        const int nr = std::min(MAXR, nrhs - c0);
        const double* Bc = Bp + (size_t)c0 * np;
        const float2* Xc = Xdf + (size_t)c0 * np;
        double* Rc = R + (size_t)c0 * np;
        IrCheck ck;
        if (chk) {
            ck.chk = chk;
            ck.col0 = c0;
            ck.ncols = nrhs;
            ck.finalize = c0 + MAXR >= nrhs;
            ck.norm = norm;
            ck.tol = tol;
            ck.flags = flags;
        }
        cudaEvent_t ev = trace_begin(s);
        if (nr <= 4) residual_df<4><<<np / RT, 256, 0, s>>>(A, np, Bc, Xc, nr, Rc, done, ck);
        else if (nr <= 8) residual_df<8><<<np / RT, 256, 0, s>>>(A, np, Bc, Xc, nr, Rc, done, ck);
        else residual_df<16><<<np / RT, 256, 0, s>>>(A, np, Bc, Xc, nr, Rc, done, ck);
        count_launch();
        // the lower triangle of A (float pairs) once, B and X read and R
        // written; each lower entry serves two products per right-hand side
        trace_end(GBEM_KERNEL_RESIDUAL, ev, s, 8.0 * ((double)np * (np + CT) / 2 + 3.0 * np * nr),
                  2.0 * (double)np * np * nr);
    }
    return cudaGetLastError();
}

cudaError_t launch_ir_check(const double* R, const double* Bp, int np, int nrhs, double* norm,
                            double tol, int* flags, cudaStream_t s)
{
    ir_check<<<1, 1024, 0, s>>>(R, Bp, np, nrhs, norm, tol, flags);
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

cudaError_t launch_batch_begin(const BatchView& v, cudaStream_t s)
{
    batch_begin<<<dim3(64, v.nb), 256, 0, s>>>(v);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_batch_iteration(const BatchView& v, size_t vec_total, long long row_blocks, int max_nc,
                                   cudaStream_t s)
{
    const int g = (int)std::min<size_t>(8192, (vec_total + 255) / 256);
    batch_to_f32<<<g, 256, 0, s>>>(v.R, v.W, vec_total);
    count_launch();
    if (max_nc <= 4) trsv_batched<4><<<v.nb, 256, 0, s>>>(v);
    else if (max_nc <= 8) trsv_batched<8><<<v.nb, 256, 0, s>>>(v);
    else trsv_batched<16><<<v.nb, 256, 0, s>>>(v);
    count_launch();
    batch_add<<<g, 256, 0, s>>>(v.W, v.X, v.Xdf, vec_total);
    count_launch();
    if (max_nc <= 4) residual_batched<4><<<(unsigned)row_blocks, 256, 0, s>>>(v);
    else if (max_nc <= 8) residual_batched<8><<<(unsigned)row_blocks, 256, 0, s>>>(v);
    else residual_batched<16><<<(unsigned)row_blocks, 256, 0, s>>>(v);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_batch_finish(const BatchView& v, double scale, cudaStream_t s)
{
    batch_finish<<<v.nb, 256, 0, s>>>(v, scale);
    count_launch();
    return cudaGetLastError();
}
