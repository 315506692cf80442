// Assembly of the Galerkin single-layer matrix (Wu & Li, Sec. 3.4):
//
//   a_ij = 1/(4 pi |I_i| |I_j|) int_{I_i} int_{I_j} 1/|x - y| dy dx
//
// One CTA owns one 32x32 tile of the lower triangle.  Every pair of the tile
// is classified by q = gap / (largest edge of the two panels):
//
//  * near pairs (q below a threshold) are evaluated exactly, in FP64, as a
//    16-term corner sum of a closed-form antiderivative of 1/r.  Parallel
//    panels use F(u,v,w) with d^4F/du^2dv^2 = 1/r (it covers the paper's
//    coplanar case of Eqs. "int1"/"int2" and the offset case for which the
//    paper falls back to 1-D quadrature, Eq. "int3"); perpendicular panels
//    use H(u,v,w) with d^4H/du^2dvdw = 1/r (a closed form of the reduction in
//    Eqs. "int4"/"int5").  Touching and self pairs are the same formula with
//    the 0*log(0) limits taken as 0.
//  * far pairs use an n x n tensor Gauss-Legendre rule on each panel (n^4
//    kernel evaluations), n the smallest order whose calibrated error bound
//    at this q is below the mode's tolerance: FP64 in FP64 mode, FP32 with
//    an FP64 outer sum in mixed mode.
//
// Near pairs are gathered into a per-tile shared-memory list during the
// classification pass and evaluated afterwards by full warps, so the scarce
// FP64 pipe never runs a closed form with most lanes of a warp idle.
#include <cstdio>
#include <type_traits>

#include "gbem_internal.h"
#include "near_field.cuh"

namespace {

__constant__ double c_glx[GBEM_GL_MAX + 1][GBEM_GL_MAX];
__constant__ double c_glw[GBEM_GL_MAX + 1][GBEM_GL_MAX];
__constant__ float c_glxf[GBEM_GL_MAX + 1][GBEM_GL_MAX];
__constant__ float c_glwf[GBEM_GL_MAX + 1][GBEM_GL_MAX];

// Smallest gap ratio q at which the n-point rule is used (index n), per mode.
// FP64 mode targets 1e-11 relative error per entry, mixed mode 3e-7.
__constant__ float c_qmin[2][GBEM_GL_MAX + 1] = {
    {3.0e38f, 3.0e38f, 200.0f, 24.0f, 6.0f, 3.0f, 2.0f},
    {3.0e38f, 700.0f, 16.0f, 3.0f, 1.5f, 1.0f, 0.5f},
};

constexpr double kPi = 3.14159265358979323846;

// ------------------------------------------------------------------ far field

// 1/sqrt(x) in FP64 (near_field.cuh).
__device__ __forceinline__ double rsq(double x) { return rsq64(x); }
// 1/sqrt(x) in FP32: the hardware approximation (PTX rsqrt.approx, relative
// error below 2^-22), flush-to-zero form, one instruction.  The arguments are
// squared distances between quadrature nodes of separated panels, always
// normal numbers, so no subnormal handling is needed.
__device__ __forceinline__ float rsq(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <typename T> __device__ __forceinline__ T glx(int n, int i);
template <typename T> __device__ __forceinline__ T glw(int n, int i);
template <> __device__ __forceinline__ double glx<double>(int n, int i) { return c_glx[n][i]; }
template <> __device__ __forceinline__ double glw<double>(int n, int i) { return c_glw[n][i]; }
template <> __device__ __forceinline__ float glx<float>(int n, int i) { return c_glxf[n][i]; }
template <> __device__ __forceinline__ float glw<float>(int n, int i) { return c_glwf[n][i]; }

// Outer sum of the quadrature: plain FP64 in FP64 mode; in mixed mode a
// compensated (Kahan) FP32 sum, which keeps FP64 instructions -- about 70x
// dearer than FP32 ones here -- out of the far field.
// Far-field entries: double in FP64 mode; in mixed mode an unevaluated float
// pair (hi, lo) formed without any FP64 instruction.
template <typename T> struct FarVal { using type = double; };
template <> struct FarVal<float> { using type = float2; };

template <typename T>
struct OuterSum {
    double s = 0.0;
    __device__ __forceinline__ void add(T v) { s += v; }
    __device__ __forceinline__ double scaled(double f) const { return s * f; }
};
template <>
struct OuterSum<float> {
    float s = 0.f, c = 0.f;   // the sum is s - c
    __device__ __forceinline__ void add(float v)
    {
        const float y = v - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    // (s - c) f as hi + lo: the product's rounding error (exact by FMA) plus
    // the compensation term
    __device__ __forceinline__ float2 scaled(float f) const
    {
        const float hi = __fmul_rn(s, f);
        return make_float2(hi, __fmaf_rn(s, f, -hi) - c * f);
    }
};

// Tensor Gauss-Legendre sum of 1/r over N x N nodes on each panel, without
// the half-extent Jacobians (a_ij = sum / (64 pi)).
//
// Parallel panels: centre offsets (dp, dq) in-plane and w along the normal;
// half extents ai, bi (panel i) and aj, bj (panel j).  The outer loop runs
// over node pairs along p, the inner (unrolled) one over node pairs along q.
template <typename T, int N>
__device__ __noinline__ OuterSum<T> far_par(T dp, T dq, T w, T ai, T bi, T aj, T bj)
{
    T Q[N * N], WQ[N * N];
#pragma unroll
    for (int b = 0; b < N; ++b)
#pragma unroll
        for (int d = 0; d < N; ++d) {
            T t = dq + glx<T>(N, b) * bi - glx<T>(N, d) * bj;
            Q[b * N + d] = t * t + w * w;
            WQ[b * N + d] = glw<T>(N, b) * glw<T>(N, d);
        }
    OuterSum<T> s;
    // low orders (the bulk of the pairs) unrolled whole: nodes and weights
    // become immediate operands
    constexpr int kUnroll = N <= 3 ? N * N : 1;
#pragma unroll kUnroll
    for (int ac = 0; ac < N * N; ++ac) {
        const int a = ac / N, c = ac % N;
        T t = dp + glx<T>(N, a) * ai - glx<T>(N, c) * aj;
        T p = t * t;
        T si = T(0);
#pragma unroll
        for (int k = 0; k < N * N; ++k) si += WQ[k] * rsq(p + Q[k]);
        s.add(glw<T>(N, a) * glw<T>(N, c) * si);
    }
    return s;
}

// Perpendicular panels: shared-axis offset ds with half extents si, sj; the
// offset dv of panel i's centre from panel j's plane (half extent ti of i
// along j's normal) and dw of panel i's plane from panel j's centre (half
// extent tj of j along i's normal).
template <typename T, int N>
__device__ __noinline__ OuterSum<T> far_orth(T ds, T si, T sj, T dv, T ti, T dw, T tj)
{
    T VW[N * N], WVW[N * N];
#pragma unroll
    for (int b = 0; b < N; ++b)
#pragma unroll
        for (int d = 0; d < N; ++d) {
            T tv = dv + glx<T>(N, b) * ti;
            T tw = dw - glx<T>(N, d) * tj;
            VW[b * N + d] = tv * tv + tw * tw;
            WVW[b * N + d] = glw<T>(N, b) * glw<T>(N, d);
        }
    OuterSum<T> s;
    constexpr int kUnroll = N <= 3 ? N * N : 1;
#pragma unroll kUnroll
    for (int ac = 0; ac < N * N; ++ac) {
        const int a = ac / N, c = ac % N;
        T t = ds + glx<T>(N, a) * si - glx<T>(N, c) * sj;
        T p = t * t;
        T acc = T(0);
#pragma unroll
        for (int k = 0; k < N * N; ++k) acc += WVW[k] * rsq(p + VW[k]);
        s.add(glw<T>(N, a) * glw<T>(N, c) * acc);
    }
    return s;
}

// ------------------------------------------------------------------ near field

// ------------------------------------------------------------------ tile kernel

struct TileGeo {
    // FP64 geometry: plane c, extents on the two in-plane axes
    double c[2 * GBEM_TILE], lo0[2 * GBEM_TILE], hi0[2 * GBEM_TILE], lo1[2 * GBEM_TILE],
        hi1[2 * GBEM_TILE];
    // FP32 copies for classification: box extents per global axis
    float blo[3][2 * GBEM_TILE], bhi[3][2 * GBEM_TILE];
    // centres as float hi + lo pairs (mixed far field) and half extents
    float chi[3][2 * GBEM_TILE], clo[3][2 * GBEM_TILE];
    float half[3][2 * GBEM_TILE];  // half extent along each global axis (0 on the normal)
    float lmax[2 * GBEM_TILE];
    float area[2 * GBEM_TILE];
    int axis[2 * GBEM_TILE];
    int valid[2 * GBEM_TILE];
};

__device__ __forceinline__ int ax_p(int k) { return k == 0 ? 1 : 0; }
__device__ __forceinline__ int ax_q(int k) { return k == 2 ? 1 : 2; }

// Exact entry of parallel panels: 16-corner sum of F.
__device__ double near_par(const TileGeo& G, int s, int t)
{
    const double w = G.c[s] - G.c[t];
    double I = 0.0;
#pragma unroll 1
    for (int k = 0; k < 16; ++k) {
        const int al = k & 1, be = (k >> 1) & 1, ga = (k >> 2) & 1, de = (k >> 3) & 1;
        double u = (al ? G.hi0[s] : G.lo0[s]) - (be ? G.hi0[t] : G.lo0[t]);
        double v = (ga ? G.hi1[s] : G.lo1[s]) - (de ? G.hi1[t] : G.lo1[t]);
        double f = F_par(u, v, w);
        I += ((al + be + ga + de) & 1) ? -f : f;
    }
    return I;
}

// Exact entry of perpendicular panels: 16-corner sum of H.  Panel i spans the
// shared axis (p) and j's normal axis (q); panel j spans the shared axis (r)
// and i's normal axis (t).
__device__ double near_orth(const TileGeo& G, int s, int t)
{
    const int ki = G.axis[s], kj = G.axis[t];
    const int sh = 3 - ki - kj;
    const bool i_first = (ax_p(ki) == sh), j_first = (ax_p(kj) == sh);
    const double p0 = i_first ? G.lo0[s] : G.lo1[s], p1 = i_first ? G.hi0[s] : G.hi1[s];
    const double q0 = i_first ? G.lo1[s] : G.lo0[s], q1 = i_first ? G.hi1[s] : G.hi0[s];
    const double r0 = j_first ? G.lo0[t] : G.lo1[t], r1 = j_first ? G.hi0[t] : G.hi1[t];
    const double t0 = j_first ? G.lo1[t] : G.lo0[t], t1 = j_first ? G.hi1[t] : G.hi0[t];
    const double ci = G.c[s], cj = G.c[t];
    double I = 0.0;
#pragma unroll 1
    for (int k = 0; k < 16; ++k) {
        const int al = k & 1, be = (k >> 1) & 1, ga = (k >> 2) & 1, de = (k >> 3) & 1;
        double hv = H_orth((al ? p1 : p0) - (be ? r1 : r0), (ga ? q1 : q0) - cj, ci - (de ? t1 : t0));
        I += ((al + be + ga + de) & 1) ? -hv : hv;
    }
    return I;
}

__device__ __forceinline__ double near_scale(const TileGeo& G, int s, int t)
{
    double ai = (G.hi0[s] - G.lo0[s]) * (G.hi1[s] - G.lo1[s]);
    double aj = (G.hi0[t] - G.lo0[t]) * (G.hi1[t] - G.lo1[t]);
    return 1.0 / (4.0 * kPi * ai * aj);
}

// Far entry of order N for the pair (s, t), T the arithmetic type.
template <typename T, int N>
__device__ typename FarVal<T>::type far_entry(const TileGeo& G, int s, int t)
{
    const int ki = G.axis[s], kj = G.axis[t];
    T d[3];
    if constexpr (sizeof(T) == 8) {
        double ci[3], cj[3];
        ci[ki] = G.c[s];
        ci[ax_p(ki)] = 0.5 * (G.lo0[s] + G.hi0[s]);
        ci[ax_q(ki)] = 0.5 * (G.lo1[s] + G.hi1[s]);
        cj[kj] = G.c[t];
        cj[ax_p(kj)] = 0.5 * (G.lo0[t] + G.hi0[t]);
        cj[ax_q(kj)] = 0.5 * (G.lo1[t] + G.hi1[t]);
#pragma unroll
        for (int e = 0; e < 3; ++e) d[e] = ci[e] - cj[e];
    } else {
        // centre offsets from float (hi, lo) pairs: error about 1 ulp of |d|
#pragma unroll
        for (int e = 0; e < 3; ++e) d[e] = (G.chi[e][s] - G.chi[e][t]) + (G.clo[e][s] - G.clo[e][t]);
    }
    OuterSum<T> sum;
    if (ki == kj) {
        const int p = ax_p(ki), q = ax_q(ki);
        T ai, bi, aj, bj;
        if constexpr (sizeof(T) == 8) {
            ai = 0.5 * (G.hi0[s] - G.lo0[s]);
            bi = 0.5 * (G.hi1[s] - G.lo1[s]);
            aj = 0.5 * (G.hi0[t] - G.lo0[t]);
            bj = 0.5 * (G.hi1[t] - G.lo1[t]);
        } else {
            ai = G.half[p][s];
            bi = G.half[q][s];
            aj = G.half[p][t];
            bj = G.half[q][t];
        }
        if constexpr (N == 1) sum.add(T(4) * rsq(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]));
        else sum = far_par<T, N>(d[p], d[q], d[ki], ai, bi, aj, bj);
    } else {
        const int sh = 3 - ki - kj;
        T hs_i, hv_i, hs_j, hw_j;
        if constexpr (sizeof(T) == 8) {
            const bool i_first = (ax_p(ki) == sh), j_first = (ax_p(kj) == sh);
            hs_i = i_first ? 0.5 * (G.hi0[s] - G.lo0[s]) : 0.5 * (G.hi1[s] - G.lo1[s]);
            hv_i = i_first ? 0.5 * (G.hi1[s] - G.lo1[s]) : 0.5 * (G.hi0[s] - G.lo0[s]);
            hs_j = j_first ? 0.5 * (G.hi0[t] - G.lo0[t]) : 0.5 * (G.hi1[t] - G.lo1[t]);
            hw_j = j_first ? 0.5 * (G.hi1[t] - G.lo1[t]) : 0.5 * (G.hi0[t] - G.lo0[t]);
        } else {
            hs_i = G.half[sh][s];
            hs_j = G.half[sh][t];
            hv_i = G.half[kj][s];
            hw_j = G.half[ki][t];
        }
        if constexpr (N == 1) sum.add(T(4) * rsq(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]));
        else sum = far_orth<T, N>(d[sh], hs_i, hs_j, d[kj], hv_i, d[ki], hw_j);
    }
    // I = (product of half extents) * sum and |I_i||I_j| = 16 * (same product)
    return sum.scaled(T(1.0 / (64.0 * kPi)));
}

constexpr int kThreads = 256;
// mixed mode: gap ratio below which every pair uses the closed form
constexpr float kMixedCfAll = 0.5f;
constexpr int kPairs = GBEM_TILE * GBEM_TILE;
// Pair classes: 0 near parallel, 1 near perpendicular, 2 + 2 (n - 1) + o for
// a far pair of order n = 1..6 (o = 1 if perpendicular).
constexpr int kClasses = 2 + 2 * GBEM_GL_MAX;

__device__ __forceinline__ double near_entry(const TileGeo& G, int cls, int s, int t)
{
    return (cls == 0 ? near_par(G, s, t) : near_orth(G, s, t)) * near_scale(G, s, t);
}

// Far classes only (cls >= 2).
template <typename T>
__device__ typename FarVal<T>::type eval_far(const TileGeo& G, int cls, int s, int t)
{
    switch (cls) {
    case 2: case 3: return far_entry<T, 1>(G, s, t);
    case 4: case 5: return far_entry<T, 2>(G, s, t);
    case 6: case 7: return far_entry<T, 3>(G, s, t);
    case 8: case 9: return far_entry<T, 4>(G, s, t);
    case 10: case 11: return far_entry<T, 5>(G, s, t);
    default: return far_entry<T, 6>(G, s, t);
    }
}

// One 32 x 32 lower tile (linear index b over the lower triangle of tiles).
// Order of the tiles: nt_band > 0: by band over all nt_band tile columns;
// nt_band = 0: row by row.  counts (may be null) receives the pairs of every
// class (kClasses words) and, in word 15, the skipped tiles.
template <bool MIXED>
__device__ __forceinline__ void tile_body(const DevPanels& g, int np, float q_near, double* __restrict__ A64,
                                          float* __restrict__ A32, unsigned long long* __restrict__ counts,
                                          long long b, int nt_band)
{
    using T = typename std::conditional<MIXED, float, double>::type;
    __shared__ TileGeo G;
    __shared__ unsigned short list[kPairs];
    __shared__ unsigned char cls_of[kPairs];
    __shared__ int cls_cnt[kClasses], cls_off[kClasses + 1];
    __shared__ int tile_ij[2];

    const int tid = threadIdx.x;
    if (tid == 0) {
        if (nt_band > 0) {
            // band order: the diagonal tiles first, then the first
            // subdiagonal, ...  Tiles near the diagonal hold the near pairs
            // (FP64 closed forms), so the costly tiles start first and the
            // cheap far-field tiles fill the tail.  Band d starts at
            // d nt - d (d - 1) / 2.
            auto off = [nt_band](long long dd) { return dd * nt_band - dd * (dd - 1) / 2; };
            // a float estimate (an FP64 square root costs microseconds of
            // latency here), corrected by the two loops below
            const float h = 2.0f * nt_band + 1.0f;
            int d = (int)((h - sqrtf(fmaxf(h * h - 8.0f * (float)b, 0.0f))) * 0.5f);
            d = max(0, min(d, nt_band - 1));
            while (d > 0 && off(d) > b) --d;
            while (d + 1 < nt_band && off(d + 1) <= b) ++d;
            // band d, position b - off(d) along it
            tile_ij[1] = (int)(b - off(d));
            tile_ij[0] = tile_ij[1] + d;
        } else {
            // lower-triangular tile coordinates (TI >= TJ) from the linear tile index
            int TI = (int)((sqrtf(8.0f * (float)b + 1.0f) - 1.0f) * 0.5f);
            while ((long long)(TI + 1) * (TI + 2) / 2 <= b) ++TI;
            while ((long long)TI * (TI + 1) / 2 > b) --TI;
            tile_ij[0] = TI;
            tile_ij[1] = (int)(b - (long long)TI * (TI + 1) / 2);
        }
    }
    if (tid < kClasses) cls_cnt[tid] = 0;
    __syncthreads();
    const int TI = tile_ij[0], TJ = tile_ij[1];
    const int n = g.n;
    if (TJ < 0 || TJ > TI || (long long)TI * GBEM_TILE >= (long long)np) {   // not a lower tile: skip, count it
        if (tid == 0 && counts) atomicAdd(&counts[15], 1ull);
        return;
    }

    if (tid < 2 * GBEM_TILE) {
        int slot = tid;
        int idx = (slot < GBEM_TILE) ? TI * GBEM_TILE + slot : TJ * GBEM_TILE + (slot - GBEM_TILE);
        int ok = idx < n;
        G.valid[slot] = ok;
        if (ok) {
            int k = g.axis[idx];
            double c = g.c[idx], l0 = g.lo0[idx], h0 = g.hi0[idx], l1 = g.lo1[idx], h1 = g.hi1[idx];
            G.axis[slot] = k;
            G.c[slot] = c;
            G.lo0[slot] = l0;
            G.hi0[slot] = h0;
            G.lo1[slot] = l1;
            G.hi1[slot] = h1;
            int p = ax_p(k), q = ax_q(k);
            double ctr[3], lo[3], hi[3];
            ctr[k] = c;
            lo[k] = c;
            hi[k] = c;
            ctr[p] = 0.5 * (l0 + h0);
            lo[p] = l0;
            hi[p] = h0;
            ctr[q] = 0.5 * (l1 + h1);
            lo[q] = l1;
            hi[q] = h1;
#pragma unroll
            for (int e = 0; e < 3; ++e) {
                float chi = (float)ctr[e];
                G.chi[e][slot] = chi;
                G.clo[e][slot] = (float)(ctr[e] - (double)chi);
                G.blo[e][slot] = (float)lo[e];
                G.bhi[e][slot] = (float)hi[e];
                G.half[e][slot] = (float)(0.5 * (hi[e] - lo[e]));
            }
            G.lmax[slot] = (float)fmax(h0 - l0, h1 - l1);
            G.area[slot] = (float)((h0 - l0) * (h1 - l1));
        }
    }
    __syncthreads();

    // 1. classify every pair; count the classes
    constexpr int kPer = kPairs / kThreads;
    int my_cls[kPer], my_rank[kPer];
    const int mode = MIXED ? 1 : 0;
    const unsigned lane = tid & 31;
#pragma unroll
    for (int r = 0; r < kPer; ++r) {
        const int e = tid + r * kThreads;
        const int ii = e & (GBEM_TILE - 1), jj = e >> 5;
        const int s = ii, t = GBEM_TILE + jj;
        int cls = -1;
        if (G.valid[s] && G.valid[t] && !(TI == TJ && ii < jj)) {
            float g2 = 0.0f;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                float gd = fmaxf(0.0f, fmaxf(G.blo[d][t] - G.bhi[d][s], G.blo[d][s] - G.bhi[d][t]));
                g2 = fmaf(gd, gd, g2);
            }
            const float L = fmaxf(G.lmax[s], G.lmax[t]);
            const float gap = sqrtf(g2);
            const float q = gap / L;
            // The closed form loses about eps * R^4 / (|I_i| |I_j|) to cancellation
            // between its 16 corner terms (R: largest corner distance); keep it
            // below 2e-12 relative, else use quadrature when an order fits.
            const float R = gap + G.lmax[s] + G.lmax[t];
            const bool cf_ok = (q < q_near) && (R * R * R * R <= 1.8e4f * G.area[s] * G.area[t]);
            // mixed mode: the FP64 closed form below q = 0.5 for every pair,
            // and below q_near only for pairs whose largest edges differ by
            // more than 1.5x (there the FP32 6-point rule can miss its target:
            // 3.1e-6 on the paper's Table 2 partition with a 6x limit; for
            // the others it meets it at a fraction of the closed form's cost,
            // about 5000 FP64 operations a pair on this part)
            const bool mixed_cf =
                q < kMixedCfAll || (q < q_near && fmaxf(G.lmax[s], G.lmax[t]) > 1.5f * fminf(G.lmax[s], G.lmax[t]));
            int order = 0;
            if (MIXED ? !mixed_cf : !cf_ok) {
#pragma unroll
                for (int m = GBEM_GL_MAX; m >= 1; --m)
                    if (q >= c_qmin[mode][m]) order = m;
            }
            const int orth = G.axis[s] != G.axis[t];
            cls = order == 0 ? orth : 2 + 2 * (order - 1) + orth;
        }
        // warp-aggregated rank within the class
        const unsigned peers = __match_any_sync(0xffffffffu, cls);
        const int leader = __ffs(peers) - 1;
        int base = 0;
        if (cls >= 0 && (int)lane == leader) base = atomicAdd(&cls_cnt[cls], __popc(peers));
        base = __shfl_sync(0xffffffffu, base, leader);
        my_cls[r] = cls;
        my_rank[r] = base + __popc(peers & ((1u << lane) - 1u));
        if (cls >= 0) cls_of[e] = (unsigned char)cls;
    }
    __syncthreads();
    // 2. class offsets: near classes first, then far classes by falling order
    if (tid == 0) {
        int acc = 0;
        cls_off[0] = 0;
        cls_off[1] = acc += cls_cnt[0];
        acc += cls_cnt[1];
        for (int c = kClasses - 1; c >= 2; --c) {
            cls_off[c] = acc;
            acc += cls_cnt[c];
        }
        cls_off[kClasses] = acc;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kPer; ++r)
        if (my_cls[r] >= 0) list[cls_off[my_cls[r]] + my_rank[r]] = (unsigned short)(tid + r * kThreads);
    __syncthreads();
    // 3. evaluate in class order: every warp runs one code path but at class
    //    boundaries
    const int total = cls_off[kClasses];
    for (int x = tid; x < total; x += kThreads) {
        const int e = list[x];
        const int ii = e & (GBEM_TILE - 1), jj = e >> 5;
        const int cls = cls_of[e];
        const size_t i = (size_t)TI * GBEM_TILE + ii, j = (size_t)TJ * GBEM_TILE + jj;
        if constexpr (MIXED) {
            // entries kept as unevaluated float pairs (hi + lo) for the
            // compensated FP32 residual; hi is also the factor's copy
            float2 pr;
            if (cls < 2) {
                const double v = near_entry(G, cls, ii, GBEM_TILE + jj);
                const float h = __double2float_rn(v);
                pr = make_float2(h, __double2float_rn(v - (double)h));
            } else {
                pr = eval_far<T>(G, cls, ii, GBEM_TILE + jj);
            }
            reinterpret_cast<float2*>(A64)[i + j * (size_t)np] = pr;
            if (A32) A32[i + j * (size_t)np] = pr.x;
        } else {
            A64[i + j * (size_t)np] = (cls < 2) ? near_entry(G, cls, ii, GBEM_TILE + jj)
                                                : eval_far<T>(G, cls, ii, GBEM_TILE + jj);
        }
    }
    // class counts: near parallel, near perpendicular, then far pairs of
    // order n parallel (2n) and perpendicular (2n + 1)
    if (tid < kClasses && counts && cls_cnt[tid]) atomicAdd(&counts[tid], (unsigned long long)cls_cnt[tid]);
}

// Register caps of 64 (mixed: four CTAs an SM) and 128 (FP64: two): the
// kernel is latency-bound (FP64 closed forms, MUFU, barrier waits), so the
// extra warps pay for the few spilled registers.
template <bool MIXED>
__global__ void __launch_bounds__(kThreads, MIXED ? 4 : 2) assemble_tiles(DevPanels g, int np, float q_near,
                                                           double* __restrict__ A64,
                                                           float* __restrict__ A32,
                                                           unsigned long long* __restrict__ counts)
{
    tile_body<MIXED>(g, np, q_near, A64, A32, counts, blockIdx.x, (g.n + GBEM_TILE - 1) / GBEM_TILE);
}

// Batched assembly: CTA index -> (structure, tile) through the prefix sums of
// the structures' tile counts.
template <bool MIXED>
__global__ void __launch_bounds__(kThreads) assemble_batched(BatchView v, float q_near)
{
    __shared__ int sb;
    if (threadIdx.x == 0) sb = batch_find(v.tile_prefix, v.nb, (long long)blockIdx.x);
    __syncthreads();
    const int b = sb;
    const long long po = v.poff[b];
    DevPanels g;
    g.c = v.c + po;
    g.lo0 = v.lo0 + po;
    g.hi0 = v.hi0 + po;
    g.lo1 = v.lo1 + po;
    g.hi1 = v.hi1 + po;
    g.axis = v.axis + po;
    g.cond = v.cond + po;
    g.n = v.n[b];
    tile_body<MIXED>(g, v.np[b], q_near, v.A64 + v.moff[b], MIXED ? v.A32 + v.moff[b] : nullptr, nullptr,
                     (long long)blockIdx.x - v.tile_prefix[b], 0);
}

// Identity padding of every structure of a batch (rows n..np-1, lower part;
// batches are mixed: float pairs in the FP64 storage and the FP32 copy).
__global__ void pad_batched(BatchView v)
{
    const int b = blockIdx.y;
    const int n = v.n[b], np = v.np[b];
    double* A64 = v.A64 + v.moff[b];
    float* A32 = v.A32 + v.moff[b];
    long long total = (long long)(np - n) * np;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        int r = n + (int)(e % (np - n));
        int c = (int)(e / (np - n));
        if (c > r) continue;
        const float val = (r == c) ? 1.0f : 0.0f;
        reinterpret_cast<float2*>(A64)[r + (size_t)c * np] = make_float2(val, 0.0f);
        A32[r + (size_t)c * np] = val;
    }
}

// Identity in the padding rows (lower part): A[r][c] = (r == c) for r >= n.
// With an FP32 copy (mixed mode) the FP64 storage holds float pairs.
__global__ void pad_identity(double* A64, float* A32, int n, int np)
{
    long long total = (long long)(np - n) * np;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        int r = n + (int)(e % (np - n));
        int c = (int)(e / (np - n));
        if (c > r) continue;
        const double v = (r == c) ? 1.0 : 0.0;
        if (A32) {
            reinterpret_cast<float2*>(A64)[r + (size_t)c * np] = make_float2((float)v, 0.0f);
            A32[r + (size_t)c * np] = (float)v;
        } else {
            A64[r + (size_t)c * np] = v;
        }
    }
}

__global__ void copy_lower(const double* __restrict__ A, double* __restrict__ L, int np)
{
    size_t total = (size_t)np * np;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        size_t r = e % np, c = e / np;
        if (r >= c) L[e] = A[e];
    }
}

}  // namespace

// Gauss-Legendre nodes on [-1,1] from Newton's method on the three-term
// Legendre recurrence (host side, computed once per process).
void gl_nodes(int n, double* x, double* w)
{
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < n; ++i) {
        double z = cos(pi * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = pk;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) {
                // one more evaluation at the converged root for the weight
                p0 = 1.0;
                p1 = z;
                for (int k = 2; k <= n; ++k) {
                    double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                    p0 = p1;
                    p1 = pk;
                }
                dp = n * (z * p1 - p0) / (z * z - 1.0);
                break;
            }
        }
        x[n - 1 - i] = z;
        w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

cudaError_t gl_upload()
{
    double hx[GBEM_GL_MAX + 1][GBEM_GL_MAX] = {}, hw[GBEM_GL_MAX + 1][GBEM_GL_MAX] = {};
    float fx[GBEM_GL_MAX + 1][GBEM_GL_MAX] = {}, fw[GBEM_GL_MAX + 1][GBEM_GL_MAX] = {};
    hx[1][0] = 0.0;
    hw[1][0] = 2.0;
    for (int n = 2; n <= GBEM_GL_MAX; ++n) gl_nodes(n, hx[n], hw[n]);
    for (int n = 1; n <= GBEM_GL_MAX; ++n)
        for (int i = 0; i < n; ++i) {
            fx[n][i] = (float)hx[n][i];
            fw[n][i] = (float)hw[n][i];
        }
    cudaError_t e;
    if ((e = cudaMemcpyToSymbol(c_glx, hx, sizeof(hx))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_glw, hw, sizeof(hw))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_glxf, fx, sizeof(fx))) != cudaSuccess) return e;
    return cudaMemcpyToSymbol(c_glwf, fw, sizeof(fw));
}

cudaError_t launch_assemble(const DevPanels& g, int np, gbem_precision prec, double q_near,
                            double* A64, float* A32, unsigned long long* counts, cudaStream_t s)
{
    if (g.n <= 0) return cudaSuccess;
    const long long nt = (g.n + GBEM_TILE - 1) / GBEM_TILE;
    const long long tiles = nt * (nt + 1) / 2;
    cudaEvent_t ev = trace_begin(s);
    if (prec == GBEM_MIXED)
        assemble_tiles<true><<<(unsigned)tiles, kThreads, 0, s>>>(g, np, (float)q_near, A64, A32, counts);
    else
        assemble_tiles<false><<<(unsigned)tiles, kThreads, 0, s>>>(g, np, (float)q_near, A64, nullptr, counts);
    count_launch();
    // algorithmic bytes: the lower entries written (FP64, or float pairs plus
    // the FP32 copy in mixed mode) and the panels read.  The arithmetic per
    // pair class is known only once the kernel has classified the pairs: it
    // follows from the class counts (gbem_matrix_class_counts).
    const double entries = (double)tiles * GBEM_TILE * GBEM_TILE;
    const double per = prec == GBEM_MIXED ? 12.0 : 8.0;
    trace_end(GBEM_KERNEL_ASSEMBLE, ev, s, entries * per + 45.0 * g.n, 0.0);
    return cudaGetLastError();
}

cudaError_t launch_assemble_batched(const BatchView& v, long long tiles, gbem_precision prec, double q_near,
                                    cudaStream_t s)
{
    if (tiles <= 0) return cudaSuccess;
    if (prec != GBEM_MIXED) return cudaErrorInvalidValue;   // batches are mixed precision
    pad_batched<<<dim3(64, v.nb), 256, 0, s>>>(v);
    count_launch();
    assemble_batched<true><<<(unsigned)tiles, kThreads, 0, s>>>(v, (float)q_near);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_pad(double* A64, float* A32, int n, int np, cudaStream_t s)
{
    if (np == n) return cudaSuccess;
    pad_identity<<<256, 256, 0, s>>>(A64, A32, n, np);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_copy_lower(const double* A, double* L, int np, cudaStream_t s)
{
    copy_lower<<<1024, 256, 0, s>>>(A, L, np);
    count_launch();
    return cudaGetLastError();
}
