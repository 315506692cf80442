// The multi-dielectric system of Wu & Li, Sec. 4, on the device: assembly of
// the per-region equations, LU factorisation with partial pivoting, the solve
// and the charges.
//
// For every region a (a dielectric layer) and every panel I_i of its
// boundary there is one equation
//     (1/2) |I_i| u_i + sum_k Q^a_ik u_k - sum_j U_ij q^a_j = 0,
// U_ij = int int 1/(4 pi |x-y|), Q^a_ik = int int <x-y, n_a(y)>/(4 pi |x-y|^3)
// over I_i x I_k, n_a the outward normal of the region.  Unknowns: u on
// insulating faces and interfaces, q on every panel but insulating faces (on
// an interface the flux of the lower layer; the upper layer's is
// -eps_lower/eps_upper times it).  Known potentials (conductors at 1 V for
// their right-hand side) move to the right-hand sides.
//
// Entries: exact corner sums of closed forms (near_field.cuh) for near
// pairs in FP64, tensor Gauss-Legendre of both kernels at shared nodes for
// far pairs (FP64, or FP32 with FP64 outer sums in mixed mode).  The matrix
// is not symmetric (Sec. 4), so it is factored by a right-looking blocked LU
// with partial pivoting (blocks of 64 columns): the panel is factored by one
// CTA (sub-panels of 8 columns, rank-8 updates between them) or, in FP32, by
// a thread-block cluster holding its rows in distributed shared memory; the
// row interchanges are applied to the other columns as one composed move, a
// triangular solve forms the panel's block row of U, and tiled updates apply
// the panel to the trailing matrix (in FP32 with one panel of lookahead on a
// second stream).  The solve refines against the FP64 system.  Apart from
// the cluster barriers of the panel, no kernel here waits on another CTA.
#include <cooperative_groups.h>
#include <cstdio>

#include "gbem_internal.h"
#include "near_field.cuh"

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int kGl = 6;   // largest Gauss-Legendre order
__constant__ double c_sx[kGl + 1][kGl];
__constant__ double c_sw[kGl + 1][kGl];
__constant__ float c_sxf[kGl + 1][kGl];
__constant__ float c_swf[kGl + 1][kGl];

__device__ __forceinline__ int axp(int k) { return k == 0 ? 1 : 0; }
__device__ __forceinline__ int axq(int k) { return k == 2 ? 1 : 2; }

struct PanelGeo {
    double c, lo0, hi0, lo1, hi1;
    int axis;
};

__device__ __forceinline__ float mufu_rsqrt(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Box extents per global axis of a panel, its gap ratio q = gap / largest
// edge of the pair, and the squared bounding diagonal of the pair.
__device__ __forceinline__ void pair_geometry(const PanelGeo& I, const PanelGeo& K, double* lo_i, double* hi_i,
                                              double* lo_k, double* hi_k, double& q, double& R2)
{
    const int ki = I.axis, kk = K.axis;
    lo_i[ki] = hi_i[ki] = I.c;
    lo_i[axp(ki)] = I.lo0;
    hi_i[axp(ki)] = I.hi0;
    lo_i[axq(ki)] = I.lo1;
    hi_i[axq(ki)] = I.hi1;
    lo_k[kk] = hi_k[kk] = K.c;
    lo_k[axp(kk)] = K.lo0;
    hi_k[axp(kk)] = K.hi0;
    lo_k[axq(kk)] = K.lo1;
    hi_k[axq(kk)] = K.hi1;
    double g2 = 0.0;
    R2 = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double g = fmax(0.0, fmax(lo_k[d] - hi_i[d], lo_i[d] - hi_k[d]));
        g2 += g * g;
        const double e = fmax(hi_i[d], hi_k[d]) - fmin(lo_i[d], lo_k[d]);
        R2 += e * e;
    }
    const double lmax = fmax(fmax(I.hi0 - I.lo0, I.hi1 - I.lo1), fmax(K.hi0 - K.lo0, K.hi1 - K.lo1));
    q = sqrt(g2) / lmax;
}

// How a pair is evaluated: 0 closed forms, else the Gauss-Legendre order.
// FP64 mode: closed forms while their corner sums lose at most about 2e-12
// (eps R^4 / (|I_i| |I_k|), R the pair's bounding diagonal), always below
// q = 3; FP64 Gauss-Legendre for the rest, about 1e-11 relative.  Mixed
// mode: closed forms below q = 1.5, FP32 Gauss-Legendre for the rest, about
// 1e-7 relative.
template <bool MIXED>
__device__ int pair_class(const PanelGeo& I, const PanelGeo& K)
{
    double lo_i[3], hi_i[3], lo_k[3], hi_k[3], q, R2;
    pair_geometry(I, K, lo_i, hi_i, lo_k, hi_k, q, R2);
    if (MIXED) {
        if (q < 1.5) return 0;
        return q >= 40.0 ? 2 : q >= 6.0 ? 3 : q >= 3.0 ? 4 : q >= 2.0 ? 5 : 6;
    }
    const double ai = (I.hi0 - I.lo0) * (I.hi1 - I.lo1), ak = (K.hi0 - K.lo0) * (K.hi1 - K.lo1);
    if (q < 3.0 || (q < 12.0 && R2 * R2 <= 9000.0 * ai * ak)) return 0;
    return q >= 320.0 ? 2 : q >= 40.0 ? 3 : q >= 10.0 ? 4 : q >= 5.0 ? 5 : 6;
}

// U and D (D: the double layer for the normal +e_k of panel k) of one pair
// of class cls (pair_class): FP64 closed forms, FP64 Gauss-Legendre, or in
// mixed mode FP32 Gauss-Legendre (FP64 node offsets, FP32 inner sums, FP64
// outer sums).
template <bool MIXED>
__device__ void pair_UD(const PanelGeo& I, const PanelGeo& K, int cls, double& U, double& D)
{
    const int ki = I.axis, kk = K.axis;
    double lo_i[3], hi_i[3], lo_k[3], hi_k[3], q, R2;
    pair_geometry(I, K, lo_i, hi_i, lo_k, hi_k, q, R2);
    if (cls == 0) {
        double su = 0.0, sd = 0.0;
        if (ki == kk) {
            const double w = I.c - K.c;
#pragma unroll 1
            for (int c = 0; c < 16; ++c) {
                const int al = c & 1, be = (c >> 1) & 1, ga = (c >> 2) & 1, de = (c >> 3) & 1;
                const double u = (al ? I.hi0 : I.lo0) - (be ? K.hi0 : K.lo0);
                const double v = (ga ? I.hi1 : I.lo1) - (de ? K.hi1 : K.lo1);
                double f, p = 0.0;
                if (w != 0.0) FPhi_par(u, v, w, f, p);
                else f = F_par(u, v, w);
                const bool neg = (al + be + ga + de) & 1;
                su += neg ? -f : f;
                sd += neg ? -p : p;
            }
        } else {
            // panel i spans the shared axis (p) and k's normal axis (q);
            // panel k spans the shared axis (r) and i's normal axis (t)
            const int sh = 3 - ki - kk;
            const bool i_first = axp(ki) == sh, k_first = axp(kk) == sh;
            const double p0 = i_first ? I.lo0 : I.lo1, p1 = i_first ? I.hi0 : I.hi1;
            const double q0 = i_first ? I.lo1 : I.lo0, q1 = i_first ? I.hi1 : I.hi0;
            const double r0 = k_first ? K.lo0 : K.lo1, r1 = k_first ? K.hi0 : K.hi1;
            const double t0 = k_first ? K.lo1 : K.lo0, t1 = k_first ? K.hi1 : K.hi0;
#pragma unroll 1
            for (int c = 0; c < 16; ++c) {
                const int al = c & 1, be = (c >> 1) & 1, ga = (c >> 2) & 1, de = (c >> 3) & 1;
                const double u = (al ? p1 : p0) - (be ? r1 : r0);
                const double v = (ga ? q1 : q0) - K.c;
                const double w = I.c - (de ? t1 : t0);
                double h, t;
                HTheta_orth(u, v, w, h, t);
                const bool neg = (al + be + ga + de) & 1;
                su += neg ? -h : h;
                sd += neg ? -t : t;
            }
        }
        U = su * (1.0 / (4.0 * kPi));
        D = sd * (1.0 / (4.0 * kPi));
        return;
    }
    // tensor Gauss-Legendre of 1/r and (x_k - y_k)/r^3 at shared nodes; the
    // order for the double layer's relative error below about 1e-11 (FP64)
    // or 1e-7 (mixed)
    double d0[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) d0[d] = 0.5 * (lo_i[d] + hi_i[d]) - 0.5 * (lo_k[d] + hi_k[d]);
    const double hi_p = 0.5 * (I.hi0 - I.lo0), hi_q = 0.5 * (I.hi1 - I.lo1);
    const double hk_p = 0.5 * (K.hi0 - K.lo0), hk_q = 0.5 * (K.hi1 - K.lo1);
    const int ip = axp(ki), iq = axq(ki), kp = axp(kk), kq = axq(kk);
    double su = 0.0, sd = 0.0;
    const int n = cls;
    if (MIXED) {
        const float fp = (float)hi_p, fq = (float)hi_q, gp = (float)hk_p, gq = (float)hk_q;
#pragma unroll 1
        for (int a = 0; a < n; ++a)
#pragma unroll 1
            for (int b = 0; b < n; ++b) {
                float x[3] = {(float)d0[0], (float)d0[1], (float)d0[2]};
                x[ip] += fp * c_sxf[n][a];
                x[iq] += fq * c_sxf[n][b];
                float tu = 0.0f, td = 0.0f;
#pragma unroll 1
                for (int c = 0; c < n; ++c)
#pragma unroll 1
                    for (int d = 0; d < n; ++d) {
                        float y[3] = {x[0], x[1], x[2]};
                        y[kp] -= gp * c_sxf[n][c];
                        y[kq] -= gq * c_sxf[n][d];
                        const float ri = mufu_rsqrt(y[0] * y[0] + y[1] * y[1] + y[2] * y[2]);
                        const float wcd = c_swf[n][c] * c_swf[n][d];
                        tu = fmaf(wcd, ri, tu);
                        td = fmaf(wcd * y[kk], ri * ri * ri, td);
                    }
                const double wab = c_sw[n][a] * c_sw[n][b];
                su = fma(wab, (double)tu, su);
                sd = fma(wab, (double)td, sd);
            }
        const double f = hi_p * hi_q * hk_p * hk_q * (1.0 / (4.0 * kPi));
        U = su * f;
        D = sd * f;
        return;
    }
#pragma unroll 1
    for (int a = 0; a < n; ++a)
#pragma unroll 1
        for (int b = 0; b < n; ++b) {
            double x[3] = {d0[0], d0[1], d0[2]};
            x[ip] += hi_p * c_sx[n][a];
            x[iq] += hi_q * c_sx[n][b];
            const double wab = c_sw[n][a] * c_sw[n][b];
            double tu = 0.0, td = 0.0;
#pragma unroll 1
            for (int c = 0; c < n; ++c)
#pragma unroll 1
                for (int d = 0; d < n; ++d) {
                    double y[3] = {x[0], x[1], x[2]};
                    y[kp] -= hk_p * c_sx[n][c];
                    y[kq] -= hk_q * c_sx[n][d];
                    const double r2 = y[0] * y[0] + y[1] * y[1] + y[2] * y[2];
                    const double ri = rsq64(r2);
                    const double wcd = c_sw[n][c] * c_sw[n][d];
                    tu = fma(wcd, ri, tu);
                    td = fma(wcd * y[kk], ri * ri * ri, td);
                }
            su = fma(wab, tu, su);
            sd = fma(wab, td, sd);
        }
    const double f = hi_p * hi_q * hk_p * hk_q * (1.0 / (4.0 * kPi));
    U = su * f;
    D = sd * f;
}

// One 32 x 32 tile of one region's pairs (rows: the region's panels I_i,
// columns: its panels I_k) into M0.  Tiles of region a are tile_off[a] .. .
template <bool MIXED>
__global__ void __launch_bounds__(256) stack_assemble(StackView v)
{
    const long long b = blockIdx.x;
    int a = 0;
    while (a + 1 < v.R_layers && v.tile_off[a + 1] <= b) ++a;
    const int r0 = v.reg_off[a], na = v.reg_off[a + 1] - r0;
    const int nt = (na + 31) / 32;
    const long long t = b - v.tile_off[a];
    const int ti = (int)(t % nt), tk = (int)(t / nt);
    __shared__ PanelGeo sg[64];
    __shared__ int sp[64];
    const int tid = threadIdx.x;
    if (tid < 64) {
        const int l = tid < 32 ? ti * 32 + tid : tk * 32 + tid - 32;
        int p = -1;
        if (l < na) {
            p = v.row_panel[r0 + l];
            sg[tid] = PanelGeo{v.c[p], v.lo0[p], v.hi0[p], v.lo1[p], v.hi1[p], (int)v.axis[p]};
        }
        sp[tid] = p;
    }
    __syncthreads();
    // classify the tile's pairs, then evaluate them class by class (closed
    // forms first), so that warps run one kind of evaluation: an FP64 closed
    // form with most lanes of a warp idle would stall the scarce FP64 pipe
    __shared__ unsigned char cls_s[1024];
    __shared__ unsigned short order[1024];
    __shared__ int cnt[8], pos[8];
    if (tid < 8) cnt[tid] = 0;
    __syncthreads();
    for (int e = tid; e < 1024; e += blockDim.x) {
        const int li = e & 31, lk = e >> 5;
        const int c = (sp[li] < 0 || sp[32 + lk] < 0) ? 7 : pair_class<MIXED>(sg[li], sg[32 + lk]);
        cls_s[e] = (unsigned char)c;
        atomicAdd(&cnt[c], 1);
    }
    __syncthreads();
    if (tid == 0) {
        int acc = 0;
        for (int c = 0; c < 8; ++c) {
            pos[c] = acc;
            acc += cnt[c];
        }
    }
    __syncthreads();
    for (int e = tid; e < 1024; e += blockDim.x) order[atomicAdd(&pos[cls_s[e]], 1)] = (unsigned short)e;
    __syncthreads();
    const int total = 1024 - cnt[7];
    const double ea = v.eps[a];
    for (int t = tid; t < total; t += blockDim.x) {
        const int e = order[t];
        const int li = e & 31, lk = e >> 5;
        const int i = sp[li], k = sp[32 + lk];
        const long long row = r0 + ti * 32 + li;
        double U, D;
        pair_UD<MIXED>(sg[li], sg[32 + lk], cls_s[e], U, D);
        const bool own = v.ra[k] == a;
        const double s = own ? (double)v.sign[k] : -(double)v.sign[k];
        double cu = s * D;
        if (i == k) cu += 0.5 * (sg[li].hi0 - sg[li].lo0) * (sg[li].hi1 - sg[li].lo1);
        const double g = own ? 1.0 : -v.eps[v.ra[k]] / ea;
        const size_t ld = (size_t)v.np;
        if (v.ucol[k] >= 0) v.M0[row + (size_t)v.ucol[k] * ld] = cu;
        else if (v.bcol[k] >= 0) atomicAdd(&v.B[row + (size_t)v.bcol[k] * ld], -cu);
        if (v.qcol[k] >= 0) v.M0[row + (size_t)v.qcol[k] * ld] = -U * g;
    }
}

// Rows and columns n_eq .. np-1 of M: the identity.
__global__ void stack_pad(double* M, int n_eq, int np)
{
    for (int r = n_eq + blockIdx.x * blockDim.x + threadIdx.x; r < np; r += gridDim.x * blockDim.x)
        M[(size_t)r + (size_t)r * np] = 1.0;
}

// The FP32 copy that the mixed mode factors.
__global__ void to_f32(const double* __restrict__ A, float* __restrict__ B, size_t count)
{
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x)
        B[e] = (float)A[e];
}


// ------------------------------------------------------------------ LU

constexpr int NB = 64;     // block columns
constexpr int SUB = 8;     // sub-panel columns
constexpr int PT = 512;    // panel threads

// argmax of |M[r, c]| over r in [c, np): the first row of the largest value
// (np if no value compares, i.e. NaN entries).
template <typename T>
__device__ int block_argmax(const T* __restrict__ col, int c, int np, double* sv, int* si)
{
    double best = -1.0;
    int bi = np;
    for (int r = c + threadIdx.x; r < np; r += blockDim.x) {
        const double x = fabs((double)col[r]);
        if (x > best) {
            best = x;
            bi = r;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_down_sync(0xffffffffu, best, o);
        const int oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) {
            best = ob;
            bi = oi;
        }
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        sv[w] = best;
        si[w] = bi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k)
            if (sv[k] > sv[0] || (sv[k] == sv[0] && si[k] < si[0])) {
                sv[0] = sv[k];
                si[0] = si[k];
            }
    }
    __syncthreads();
    const int p = si[0];
    __syncthreads();
    return p;
}

// Factor the panel of columns j0 .. j0+63, rows j0 .. np-1, in place:
// L below the diagonal (unit diagonal implied), U on and above it within the
// panel; ipiv[c] = the row swapped with row c at column c.  A zero pivot
// (or a column without a comparable value) sets *status = GBEM_ERR_NOT_SPD
// and leaves its column unscaled.
template <typename T>
__global__ void __launch_bounds__(PT) lu_panel(T* __restrict__ M, int np, int j0, int* __restrict__ ipiv,
                                               int* status)
{
    __shared__ double sv[PT / 32];
    __shared__ int si[PT / 32];
    __shared__ T urow[NB];
    __shared__ T ublk[SUB][NB];
    const size_t ld = (size_t)np;
    const int tid = threadIdx.x;
    for (int s0 = j0; s0 < j0 + NB; s0 += SUB) {
        for (int c = s0; c < s0 + SUB; ++c) {
            T* col = M + (size_t)c * ld;
            int p = block_argmax(col, c, np, sv, si);
            if (p >= np) {   // no comparable value (NaN entries): keep the row, flag the system
                p = c;
                if (tid == 0) atomicExch(status, (int)GBEM_ERR_NOT_SPD);
            }
            if (tid == 0) ipiv[c] = p;
            // swap rows c and p across the panel's columns
            if (p != c && tid < NB) {
                T* e = M + (size_t)(j0 + tid) * ld;
                const T t = e[c];
                e[c] = e[p];
                e[p] = t;
            }
            __syncthreads();
            const T piv = col[c];
            if (piv == T(0)) {
                if (tid == 0) atomicExch(status, (int)GBEM_ERR_NOT_SPD);
                __syncthreads();
                continue;
            }
            if (tid < s0 + SUB - c - 1) urow[tid] = M[(size_t)c + (size_t)(c + 1 + tid) * ld];
            __syncthreads();
            const T inv = T(1) / piv;
            const int ncol = s0 + SUB - c - 1;
            for (int r = c + 1 + tid; r < np; r += PT) {
                const T l = col[r] * inv;
                col[r] = l;
                for (int k = 0; k < ncol; ++k) {
                    T* e = M + (size_t)(c + 1 + k) * ld + r;
                    *e = fma(-l, urow[k], *e);
                }
            }
            __syncthreads();
        }
        const int rest = j0 + NB - (s0 + SUB);
        if (rest == 0) break;
        // block row of U for the sub-panel: rows s0..s0+7 of the remaining
        // panel columns, L_ss^-1 times them (unit lower 8 x 8)
        if (tid < rest) {
            const int cc = s0 + SUB + tid;
            T x[SUB];
#pragma unroll
            for (int r = 0; r < SUB; ++r) {
                T t = M[(size_t)(s0 + r) + (size_t)cc * ld];
#pragma unroll
                for (int k = 0; k < r; ++k) t = fma(-M[(size_t)(s0 + r) + (size_t)(s0 + k) * ld], x[k], t);
                x[r] = t;
            }
#pragma unroll
            for (int r = 0; r < SUB; ++r) {
                M[(size_t)(s0 + r) + (size_t)cc * ld] = x[r];
                ublk[r][tid] = x[r];
            }
        }
        __syncthreads();
        // rank-8 update of the rows below
        for (int r = s0 + SUB + tid; r < np; r += PT) {
            T l[SUB];
#pragma unroll
            for (int k = 0; k < SUB; ++k) l[k] = M[(size_t)r + (size_t)(s0 + k) * ld];
            for (int j = 0; j < rest; ++j) {
                T* e = M + (size_t)(s0 + SUB + j) * ld + r;
                T t = *e;
#pragma unroll
                for (int k = 0; k < SUB; ++k) t = fma(-l[k], ublk[k][j], t);
                *e = t;
            }
        }
        __syncthreads();
    }
}

// The FP32 panel factorisation across a thread-block cluster: CTA r of the
// cluster holds rows j0 + r*rows .. of the panel's 64 columns in shared
// memory (row-major, rows padded to 65 floats).  Per column every CTA publishes its
// candidate pivot (|value|, row, the row's 64 values) and, if it owns the
// diagonal row, that row, in a slot of its own shared memory; after one
// cluster barrier every CTA reads the slots of all CTAs (distributed shared
// memory), takes the largest candidate (the first row on a tie), swaps rows
// locally and applies the rank-1 update to its rows.  The slots alternate
// between two buffers, so the next column's barrier also orders this
// column's reads before their reuse.  Same results as lu_panel's partial
// pivoting; a zero or incomparable pivot sets *status.
struct PivotSlot {
    float val;
    int row;
    float vals[NB];
};
constexpr int LDA = NB + 1;   // shared row stride: a column's rows fall in distinct banks
constexpr size_t kPanelSmemMax = 220 * 1024;
constexpr size_t panel_cluster_smem(int rows) { return sizeof(float) * (size_t)rows * LDA + 4 * sizeof(PivotSlot); }

__global__ void __launch_bounds__(256) lu_panel_cluster(float* __restrict__ M, int np, int j0, int rows,
                                                       int* __restrict__ ipiv, int* status)
{
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank(), csize = (int)cluster.num_blocks();
    extern __shared__ float psm[];
    float* A = psm;                                                   // rows x LDA
    PivotSlot* cand = reinterpret_cast<PivotSlot*>(psm + (size_t)rows * LDA);  // [2]
    PivotSlot* diag = cand + 2;                                       // [2]: the diagonal row
    __shared__ float pivrow[NB], oldrow[NB];
    __shared__ float wv[8];
    __shared__ int wi[8];
    __shared__ int win_rank, win_row, diag_rank;
    const size_t ld = (size_t)np;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int base = j0 + rank * rows;                                // first global row held here
    const int mine = max(0, min(rows, np - base));                    // rows held
    for (int e = tid; e < mine * NB; e += nt) {
        const int i = e % mine, j = e / mine;
        A[(size_t)i * LDA + j] = M[(size_t)(base + i) + (size_t)(j0 + j) * ld];
    }
    __syncthreads();
    for (int c = 0; c < NB; ++c) {
        const int g = j0 + c, buf = c & 1;
        // local candidate among the held rows >= g
        float best = -1.0f;
        int bi = np;
        for (int i = tid; i < mine; i += nt) {
            const int r = base + i;
            if (r < g) continue;
            const float x = fabsf(A[(size_t)i * LDA + c]);
            if (x > best) {
                best = x;
                bi = r;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float ob = __shfl_down_sync(0xffffffffu, best, o);
            const int oi = __shfl_down_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) {
                best = ob;
                bi = oi;
            }
        }
        if ((tid & 31) == 0) {
            wv[tid >> 5] = best;
            wi[tid >> 5] = bi;
        }
        __syncthreads();
        if (tid == 0) {
            for (int k = 1; k < nt / 32; ++k)
                if (wv[k] > wv[0] || (wv[k] == wv[0] && wi[k] < wi[0])) {
                    wv[0] = wv[k];
                    wi[0] = wi[k];
                }
            cand[buf].val = wv[0];
            cand[buf].row = wi[0];
        }
        __syncthreads();
        const int lrow = wi[0];
        if (tid < NB) {
            cand[buf].vals[tid] = lrow < np ? A[(size_t)(lrow - base) * LDA + tid] : 0.0f;
            if (g >= base && g < base + mine) diag[buf].vals[tid] = A[(size_t)(g - base) * LDA + tid];
        }
        cluster.sync();
        // the winner over the cluster (warp 0, one slot a lane), and the two
        // rows it exchanges
        if (tid < 32) {
            float bv = -1.0f;
            int br = np, bk = tid;
            if (tid < csize) {
                const PivotSlot* o = cluster.map_shared_rank(cand + buf, tid);
                bv = o->val;
                br = o->row;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float ov = __shfl_down_sync(0xffffffffu, bv, o);
                const int orow = __shfl_down_sync(0xffffffffu, br, o);
                const int ok = __shfl_down_sync(0xffffffffu, bk, o);
                if (ov > bv || (ov == bv && orow < br)) {
                    bv = ov;
                    br = orow;
                    bk = ok;
                }
            }
            if (tid == 0) {
                if (br >= np) {   // no comparable value: keep the diagonal row
                    br = g;
                    bk = (g - j0) / rows;
                    if (rank == 0) atomicExch(status, (int)GBEM_ERR_NOT_SPD);
                }
                win_rank = bk;
                win_row = br;
                diag_rank = (g - j0) / rows;
                if (rank == 0) ipiv[g] = br;
            }
        }
        __syncthreads();
        const int w = win_row;
        if (tid < NB) {
            const PivotSlot* ws = cluster.map_shared_rank(cand + buf, win_rank);
            const PivotSlot* ds = cluster.map_shared_rank(diag + buf, diag_rank);
            pivrow[tid] = w == g ? ds->vals[tid] : ws->vals[tid];
            oldrow[tid] = ds->vals[tid];
        }
        __syncthreads();
        if (tid < NB) {
            if (g >= base && g < base + mine) A[(size_t)(g - base) * LDA + tid] = pivrow[tid];
            if (w != g && w >= base && w < base + mine) A[(size_t)(w - base) * LDA + tid] = oldrow[tid];
        }
        __syncthreads();
        const float piv = pivrow[c];
        if (piv == 0.0f) {
            if (rank == 0 && tid == 0) atomicExch(status, (int)GBEM_ERR_NOT_SPD);
        } else {
            const float inv = 1.0f / piv;
            for (int i = tid; i < mine; i += nt) {
                if (base + i <= g) continue;
                float* a = A + (size_t)i * LDA;
                const float l = a[c] * inv;
                a[c] = l;
                for (int j = c + 1; j < NB; ++j) a[j] = fmaf(-l, pivrow[j], a[j]);
            }
        }
        __syncthreads();
    }
    // the next kernel reads the other CTAs' rows only through global memory
    cluster.sync();
    for (int e = tid; e < mine * NB; e += nt) {
        const int i = e % mine, j = e / mine;
        M[(size_t)(base + i) + (size_t)(j0 + j) * ld] = A[(size_t)i * LDA + j];
    }
}

// The panel's 64 interchanges composed into one permutation of the rows they
// touch (at most 128): plan[0] = count, then (destination, source) pairs with
// destination != source.  One warp: rows j0..j0+63 take slots 0..63, every
// other row the slot 64 + (its rank among the other rows by first
// appearance); lane 0 then replays the 64 exchanges on the slots.
__global__ void __launch_bounds__(32) lu_swap_plan(const int* __restrict__ ipiv, int j0, int* __restrict__ plan)
{
    __shared__ int piv[NB], slot[NB], first[NB];
    __shared__ int row[2 * NB], content[2 * NB];
    const int lane = threadIdx.x;
    for (int k = lane; k < NB; k += 32) piv[k] = ipiv[j0 + k];
    __syncwarp();
    // first appearance of each outside row
    for (int k = lane; k < NB; k += 32) {
        int f = k;
        if (piv[k] >= j0 + NB)
            for (int t = 0; t < k; ++t)
                if (piv[t] == piv[k]) {
                    f = t;
                    break;
                }
        first[k] = f;
    }
    __syncwarp();
    for (int k = lane; k < NB; k += 32) {
        const int p = piv[k];
        if (p < j0 + NB) {
            slot[k] = p - j0;
        } else {
            int rnk = 0;   // outside rows first seen before first[k]
            for (int t = 0; t < first[k]; ++t) rnk += (piv[t] >= j0 + NB && first[t] == t) ? 1 : 0;
            slot[k] = NB + rnk;
            if (first[k] == k) {
                row[NB + rnk] = p;
                content[NB + rnk] = p;
            }
        }
    }
    for (int k = lane; k < NB; k += 32) {
        row[k] = j0 + k;
        content[k] = j0 + k;
    }
    __syncwarp();
    if (lane == 0) {
        int n = NB;
        for (int k = 0; k < NB; ++k) {
            const int sp = slot[k];
            n = max(n, sp + 1);
            const int t = content[k];
            content[k] = content[sp];
            content[sp] = t;
        }
        int m = 0;
        for (int t = 0; t < n; ++t)
            if (content[t] != row[t]) {
                plan[1 + 2 * m] = row[t];
                plan[2 + 2 * m] = content[t];
                ++m;
            }
        plan[0] = m;
    }
}

// The panel's interchanges applied to the columns c_lo .. c_hi-1 outside
// skip_lo .. skip_hi-1: each thread gathers the moved rows of its column at
// once, then writes them.
template <typename T>
__global__ void __launch_bounds__(128) lu_swap(T* __restrict__ M, int np, int c_lo, int c_hi, int skip_lo,
                                               int skip_hi, const int* __restrict__ plan)
{
    __shared__ int pl[1 + 4 * NB];
    for (int e = threadIdx.x; e < 1 + 4 * NB; e += blockDim.x) pl[e] = plan[e];
    __syncthreads();
    const int m = pl[0];
    // columns c_lo .. c_hi-1 except skip_lo .. skip_hi-1 (inside the range)
    const int ncols = (c_hi - c_lo) - (skip_hi - skip_lo);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ncols; t += gridDim.x * blockDim.x) {
        const int c = c_lo + t < skip_lo ? c_lo + t : c_lo + t + (skip_hi - skip_lo);
        T* e = M + (size_t)c * np;
        T v[2 * NB];
#pragma unroll 16
        for (int i = 0; i < 2 * NB; ++i)
            if (i < m) v[i] = e[pl[2 + 2 * i]];
#pragma unroll 16
        for (int i = 0; i < 2 * NB; ++i)
            if (i < m) e[pl[1 + 2 * i]] = v[i];
    }
}

// U12 = L11^-1 A12 for 64 columns per CTA from column c_lo on (L11 the
// panel's unit lower block).
template <typename T>
__global__ void __launch_bounds__(NB) lu_trsm(T* __restrict__ M, int np, int j0, int c_lo)
{
    __shared__ T L[NB][NB + 1];
    const size_t ld = (size_t)np;
    const int tid = threadIdx.x;
    for (int e = tid; e < NB * NB; e += NB) {
        const int r = e % NB, c = e / NB;
        L[r][c] = M[(size_t)(j0 + r) + (size_t)(j0 + c) * ld];
    }
    __syncthreads();
    const int cc = c_lo + blockIdx.x * NB + tid;
    T* col = M + (size_t)cc * ld + j0;
    T x[NB];
#pragma unroll
    for (int r = 0; r < NB; ++r) x[r] = col[r];
#pragma unroll
    for (int r = 1; r < NB; ++r) {
        T t = x[r];
#pragma unroll
        for (int k = 0; k < r; ++k) t = fma(-L[r][k], x[k], t);
        x[r] = t;
    }
#pragma unroll
    for (int r = 0; r < NB; ++r) col[r] = x[r];
}

// A22 -= L21 U12 in FP64: one 64 x 64 tile per CTA, 4 x 4 outputs per thread.
constexpr size_t kGemmSmem64 = 2 * sizeof(double) * NB * (NB + 1);
__global__ void __launch_bounds__(256) lu_gemm_f64(double* __restrict__ M, int np, int j0)
{
    extern __shared__ double gsm[];
    double(*Ls)[NB + 1] = reinterpret_cast<double(*)[NB + 1]>(gsm);                  // Ls[k][r] = L21[r][k]
    double(*Us)[NB + 1] = reinterpret_cast<double(*)[NB + 1]>(gsm + NB * (NB + 1));  // Us[k][c] = U12[k][c]
    const size_t ld = (size_t)np;
    const int i0 = j0 + NB + blockIdx.x * NB, c0 = j0 + NB + blockIdx.y * NB;
    const int tid = threadIdx.x;
    for (int e = tid; e < NB * NB; e += 256) {
        const int r = e % NB, k = e / NB;
        Ls[k][r] = M[(size_t)(i0 + r) + (size_t)(j0 + k) * ld];
        Us[r][k] = M[(size_t)(j0 + r) + (size_t)(c0 + k) * ld];
    }
    __syncthreads();
    const int tx = tid & 15, ty = tid >> 4;
    double acc[4][4] = {};
#pragma unroll 4
    for (int k = 0; k < NB; ++k) {
        double a[4], b[4];
#pragma unroll
        for (int x = 0; x < 4; ++x) {
            a[x] = Ls[k][tx + 16 * x];
            b[x] = Us[k][ty + 16 * x];
        }
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < 4; ++y) acc[x][y] = fma(a[x], b[y], acc[x][y]);
    }
#pragma unroll
    for (int y = 0; y < 4; ++y)
#pragma unroll
        for (int x = 0; x < 4; ++x) {
            double* e = M + (size_t)(i0 + tx + 16 * x) + (size_t)(c0 + ty + 16 * y) * ld;
            *e -= acc[x][y];
        }
}

// A22 -= L21 U12 in FP32 for the columns c_lo .. c_hi-1: one 128 x 128 tile
// per CTA, 8 x 8 outputs per thread (rows tx + 16 i, columns ty + 16 j),
// K = 64; the orders are multiples of 64, so edge tiles skip their missing
// half.
constexpr int GT = 128;
constexpr size_t kGemmSmem32 = 2 * sizeof(float) * NB * (GT + 4);
__global__ void __launch_bounds__(256) lu_gemm_f32(float* __restrict__ M, int np, int j0, int c_lo, int c_hi)
{
    extern __shared__ float fsm[];
    float(*Ls)[GT + 4] = reinterpret_cast<float(*)[GT + 4]>(fsm);                   // Ls[k][r]
    float(*Us)[GT + 4] = reinterpret_cast<float(*)[GT + 4]>(fsm + NB * (GT + 4));  // Us[k][c]
    const size_t ld = (size_t)np;
    const int base = j0 + NB;
    const int i0 = base + blockIdx.x * GT, c0 = c_lo + blockIdx.y * GT;
    const int rows = min(GT, np - i0), cols = min(GT, c_hi - c0);
    const int tid = threadIdx.x;
    for (int e = tid; e < NB * GT; e += 256) {
        const int r = e % GT, k = e / GT;
        Ls[k][r] = r < rows ? M[(size_t)(i0 + r) + (size_t)(j0 + k) * ld] : 0.0f;
    }
    for (int e = tid; e < NB * GT; e += 256) {
        const int k = e % NB, c = e / NB;
        Us[k][c] = c < cols ? M[(size_t)(j0 + k) + (size_t)(c0 + c) * ld] : 0.0f;
    }
    __syncthreads();
    const int tx = tid & 15, ty = tid >> 4;
    float acc[8][8] = {};
#pragma unroll 2
    for (int k = 0; k < NB; ++k) {
        float a[8], b[8];
#pragma unroll
        for (int x = 0; x < 8; ++x) {
            a[x] = Ls[k][tx + 16 * x];
            b[x] = Us[k][ty + 16 * x];
        }
#pragma unroll
        for (int x = 0; x < 8; ++x)
#pragma unroll
            for (int y = 0; y < 8; ++y) acc[x][y] = fmaf(a[x], b[y], acc[x][y]);
    }
#pragma unroll
    for (int y = 0; y < 8; ++y) {
        const int c = ty + 16 * y;
        if (c >= cols) continue;
#pragma unroll
        for (int x = 0; x < 8; ++x) {
            const int r = tx + 16 * x;
            if (r < rows) M[(size_t)(i0 + r) + (size_t)(c0 + c) * ld] -= acc[x][y];
        }
    }
}

// ------------------------------------------------------------------ solve

// perm[r] = the original row that ends at row r after ipiv[0..np-1].
__global__ void __launch_bounds__(256) lu_perm(const int* __restrict__ ipiv, int np, int* __restrict__ perm)
{
    extern __shared__ int sperm[];
    for (int r = threadIdx.x; r < np; r += blockDim.x) sperm[r] = r;
    __syncthreads();
    if (threadIdx.x == 0)
        for (int r = 0; r < np; ++r) {
            const int p = ipiv[r];
            const int t = sperm[r];
            sperm[r] = sperm[p];
            sperm[p] = t;
        }
    __syncthreads();
    for (int r = threadIdx.x; r < np; r += blockDim.x) perm[r] = sperm[r];
}

// W[r, m] = R[perm[r], m] in the factor's type.
template <typename T>
__global__ void permute_rhs(const double* __restrict__ R, const int* __restrict__ perm, int np, int nc,
                            T* __restrict__ W)
{
    const long long total = (long long)np * nc;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e % np), m = (int)(e / np);
        W[e] = (T)R[(size_t)perm[r] + (size_t)m * np];
    }
}

// Inverses of the diagonal blocks of the factor, for the sweeps: Inv[2 b]
// = L_bb^-1 (unit lower), Inv[2 b + 1] = U_bb^-1, each 64 x 64 column-major.
// Thread c forms column c of both by substitution.
template <typename T>
__global__ void __launch_bounds__(NB) tri_inverse(const T* __restrict__ M, int np, T* __restrict__ Inv)
{
    __shared__ T Tb[NB][NB + 1];
    const size_t ld = (size_t)np;
    const int j0 = blockIdx.x * NB, c = threadIdx.x;
    for (int e = threadIdx.x; e < NB * NB; e += NB) {
        const int i = e % NB, k = e / NB;
        Tb[i][k] = M[(size_t)(j0 + i) + (size_t)(j0 + k) * ld];
    }
    __syncthreads();
    T* Li = Inv + (size_t)(2 * blockIdx.x) * NB * NB;
    T* Ui = Li + NB * NB;
    T x[NB];
#pragma unroll
    for (int r = 0; r < NB; ++r) {
        T t = r == c ? T(1) : T(0);
#pragma unroll
        for (int k = 0; k < r; ++k) t = fma(-Tb[r][k], x[k], t);
        x[r] = t;
    }
#pragma unroll
    for (int r = 0; r < NB; ++r) Li[(size_t)c * NB + r] = x[r];
#pragma unroll
    for (int r = NB - 1; r >= 0; --r) {
        T t = r == c ? T(1) : T(0);
#pragma unroll
        for (int k = r + 1; k < NB; ++k) t = fma(-Tb[r][k], x[k], t);
        x[r] = t / Tb[r][r];
    }
#pragma unroll
    for (int r = 0; r < NB; ++r) Ui[(size_t)c * NB + r] = x[r];
}

// One step of the forward (LOWER: In = W, Out = Y) or backward sweep (In = Y,
// Out = W) for block b: every CTA forms x_b = T_bb^-1 In_b from the stored
// inverse; CTA 0 writes it to Out_b; every CTA subtracts M[r, block b] x_b
// from the rows of In below (LOWER) or above block b.  In_b is not written
// in this launch, so the CTAs agree on x_b.
template <typename T, bool LOWER, int NR>
__global__ void __launch_bounds__(256) sweep_step(const T* __restrict__ M, const T* __restrict__ Inv, int np, int b,
                                                  int nc, T* __restrict__ In, T* __restrict__ Out)
{
    __shared__ T inv[NB][NB + 1];
    __shared__ T xin[NR][NB];
    __shared__ T xb[NR][NB];
    const size_t ld = (size_t)np;
    const int j0 = b * NB;
    const T* src = Inv + (size_t)(2 * b + (LOWER ? 0 : 1)) * NB * NB;
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) inv[e % NB][e / NB] = src[e];
    const int rlo = LOWER ? j0 + NB : 0, rhi = LOWER ? np : j0;
    for (int m0 = 0; m0 < nc; m0 += NR) {
        const int mn = min(NR, nc - m0);
        __syncthreads();
        for (int e = threadIdx.x; e < NR * NB; e += blockDim.x)
            xin[e / NB][e % NB] = e / NB < mn ? In[(size_t)(m0 + e / NB) * np + j0 + e % NB] : T(0);
        __syncthreads();
        for (int e = threadIdx.x; e < NR * NB; e += blockDim.x) {
            const int m = e / NB, r = e % NB;
            T t = T(0);
#pragma unroll 16
            for (int k = 0; k < NB; ++k) t = fma(inv[r][k], xin[m][k], t);
            xb[m][r] = t;
        }
        __syncthreads();
        if (blockIdx.x == 0)
            for (int e = threadIdx.x; e < mn * NB; e += blockDim.x)
                Out[(size_t)(m0 + e / NB) * np + j0 + e % NB] = xb[e / NB][e % NB];
        for (int r = rlo + blockIdx.x * blockDim.x + threadIdx.x; r < rhi; r += gridDim.x * blockDim.x) {
            T acc[NR] = {};
            const T* row = M + (size_t)r + (size_t)j0 * ld;
#pragma unroll 1
            for (int k0 = 0; k0 < NB; k0 += 16) {
                T l[16];
#pragma unroll
                for (int k = 0; k < 16; ++k) l[k] = row[(size_t)(k0 + k) * ld];
#pragma unroll
                for (int k = 0; k < 16; ++k)
#pragma unroll
                    for (int m = 0; m < NR; ++m) acc[m] = fma(l[k], xb[m][k0 + k], acc[m]);
            }
            for (int m = 0; m < mn; ++m) In[(size_t)(m0 + m) * np + r] -= acc[m];
        }
    }
}

template <typename T, bool LOWER>
void launch_sweep_step(const T* M, const T* Inv, int np, int b, int nc, T* In, T* Out, cudaStream_t s)
{
    const int j0 = b * NB;
    const int rows = LOWER ? np - j0 - NB : j0;
    const int grid = max(1, min(2 * 152, (rows + 255) / 256));
    // at most 16 right-hand sides per pass in FP32, 8 in FP64 (48 KB of
    // static shared memory)
    if (nc <= 4) {
        sweep_step<T, LOWER, 4><<<grid, 256, 0, s>>>(M, Inv, np, b, nc, In, Out);
    } else if constexpr (sizeof(T) == 8) {
        sweep_step<T, LOWER, 8><<<grid, 256, 0, s>>>(M, Inv, np, b, nc, In, Out);
    } else {
        if (nc <= 8) sweep_step<T, LOWER, 8><<<grid, 256, 0, s>>>(M, Inv, np, b, nc, In, Out);
        else sweep_step<T, LOWER, 16><<<grid, 256, 0, s>>>(M, Inv, np, b, nc, In, Out);
    }
    count_launch();
}

// X += W
template <typename T>
__global__ void add_correction(double* __restrict__ X, const T* __restrict__ W, size_t count)
{
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x)
        X[e] += (double)W[e];
}

// Partial products of M0 X in FP64: chunk blockIdx.y of the columns, rows
// blockIdx.x * 128 + threadIdx.x, up to 16 right-hand sides per pass;
// P[(chunk * nc + m) * np + r].
constexpr int kResChunks = 8;
__global__ void __launch_bounds__(128) residual_partial(const double* __restrict__ M0, int n_eq, int np, int nc,
                                                        const double* __restrict__ X, double* __restrict__ P)
{
    const size_t ld = (size_t)np;
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    const int per = (n_eq + kResChunks - 1) / kResChunks;
    const int c_lo = blockIdx.y * per, c_hi = min(n_eq, c_lo + per);
    __shared__ double xs[16][128];
    for (int m0 = 0; m0 < nc; m0 += 16) {
        const int mn = min(16, nc - m0);
        double acc[16] = {};
        for (int cb = c_lo; cb < c_hi; cb += 128) {
            const int cn = min(128, c_hi - cb);
            __syncthreads();
            for (int e = threadIdx.x; e < 16 * 128; e += blockDim.x) {
                const int m = e / 128, c = e % 128;
                xs[m][c] = (m < mn && c < cn) ? X[(size_t)(cb + c) + (size_t)(m0 + m) * ld] : 0.0;
            }
            __syncthreads();
            if (r < n_eq)
                for (int c = 0; c < cn; ++c) {
                    const double a = M0[(size_t)r + (size_t)(cb + c) * ld];
#pragma unroll
                    for (int m = 0; m < 16; ++m) acc[m] = fma(a, xs[m][c], acc[m]);
                }
        }
        if (r < n_eq)
            for (int m = 0; m < mn; ++m) P[((size_t)blockIdx.y * nc + m0 + m) * ld + r] = acc[m];
    }
}

// R = B - sum of the partials (rows < n_eq; 0 below); rnorm[m] = max |R[., m]|,
// bnorm[m] = max |B[., m]| as the bit patterns of non-negative doubles.
__global__ void residual_finish(const double* __restrict__ B, const double* __restrict__ P, int n_eq, int np, int nc,
                                double* __restrict__ R, unsigned long long* rmax, unsigned long long* bmax)
{
    const long long total = (long long)np * nc;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e % np), m = (int)(e / np);
        double t = 0.0;
        if (r < n_eq) {
            t = B[e];
            for (int k = 0; k < kResChunks; ++k) t -= P[((size_t)k * nc + m) * np + r];
            atomicMax(rmax + m, (unsigned long long)__double_as_longlong(fabs(t)));
            atomicMax(bmax + m, (unsigned long long)__double_as_longlong(fabs(B[e])));
        }
        R[e] = t;
    }
}

// C[n][m] = eps0 1e-6 sum over conductor n's panels of eps_a |I_j| q_j (X's
// q rows for right-hand side m); one CTA per (n, m).
__global__ void __launch_bounds__(256) stack_charges(StackView v, const double* __restrict__ X, double eps0)
{
    const int nidx = blockIdx.x, m = blockIdx.y;
    double s = 0.0;
    for (int p = threadIdx.x; p < v.n; p += blockDim.x)
        if (v.cidx[p] == nidx)
            s += v.eps[v.ra[p]] * (v.hi0[p] - v.lo0[p]) * (v.hi1[p] - v.lo1[p]) *
                 X[(size_t)v.qcol[p] + (size_t)m * v.np];
    __shared__ double red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) v.C[(size_t)nidx * v.nc + m] = eps0 * 1e-6 * red[0];
}

// Cluster size for the FP32 panel (16 where the device schedules such
// clusters with the largest shared memory, else 8), 0 if neither.
int panel_cluster_size()
{
    static int dev_sizes[64];
    static bool known[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    if (known[dev]) return dev_sizes[dev];
    int best = 0;
    const size_t smem = kPanelSmemMax;
    if (cudaFuncSetAttribute(lu_panel_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess &&
        cudaFuncSetAttribute(lu_panel_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
        for (int cs : {16, 8}) {
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = cs;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.gridDim = dim3(cs);
            cfg.blockDim = dim3(256);
            cfg.dynamicSmemBytes = smem;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            int n = 0;
            if (cudaOccupancyMaxActiveClusters(&n, lu_panel_cluster, &cfg) == cudaSuccess && n > 0) {
                best = cs;
                break;
            }
        }
    }
    cudaGetLastError();
    dev_sizes[dev] = best;
    known[dev] = true;
    return best;
}

// One panel in FP32 through a cluster when its rows fit the cluster's shared
// memory; false if not (the caller uses lu_panel).
bool panel_f32_cluster(float* M, int np, int j0, const StackView& v, int csize, cudaStream_t s, cudaError_t& err)
{
    if (csize <= 0) return false;
    const int m = np - j0;
    const int rows = (m + csize - 1) / csize;
    const size_t smem = panel_cluster_smem(rows);
    if (smem > kPanelSmemMax) return false;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = csize;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(csize);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    err = cudaLaunchKernelEx(&cfg, lu_panel_cluster, M, np, j0, rows, v.ipiv, v.status);
    count_launch();
    return true;
}

template <typename T>
cudaError_t lu_run(T* M, const StackView& v, cudaStream_t s)
{
    const int np = v.np;
    for (int j0 = 0; j0 < np; j0 += NB) {
        lu_panel<T><<<1, PT, 0, s>>>(M, np, j0, v.ipiv, v.status);
        lu_swap_plan<<<1, 32, 0, s>>>(v.ipiv, j0, v.plan);
        lu_swap<T><<<(np + 127) / 128, 128, 0, s>>>(M, np, 0, np, j0, j0 + NB, v.plan);
        count_launch(3);
        const int nrest = (np - j0 - NB) / NB;
        if (nrest > 0) {
            lu_trsm<T><<<nrest, NB, 0, s>>>(M, np, j0, j0 + NB);
            if constexpr (sizeof(T) == 8) {
                lu_gemm_f64<<<dim3(nrest, nrest), 256, kGemmSmem64, s>>>(M, np, j0);
            } else {
                const int nt = (nrest * NB + GT - 1) / GT;
                lu_gemm_f32<<<dim3(nt, nt), 256, kGemmSmem32, s>>>(M, np, j0, j0 + NB, np);
            }
            count_launch(2);
        }
    }
    return cudaGetLastError();
}

// The FP32 factorisation with one panel of lookahead: after panel k's row
// moves and block row of U, its update of block column k+1 runs first, then
// panel k+1 (cluster kernel, on the side stream) runs beside panel k's
// update of the columns beyond k+1 (main stream); the two touch disjoint
// columns.  Events join the streams before panel k+1's row moves.
cudaError_t lu_run_lookahead(float* M, const StackView& v, int csize, cudaStream_t s, cudaStream_t side,
                             cudaEvent_t ready, cudaEvent_t done)
{
    const int np = v.np;
    cudaError_t e = cudaSuccess;
    if (!panel_f32_cluster(M, np, 0, v, csize, s, e)) {
        lu_panel<float><<<1, PT, 0, s>>>(M, np, 0, v.ipiv, v.status);
        count_launch();
    }
    if (e != cudaSuccess) return e;
    lu_swap_plan<<<1, 32, 0, s>>>(v.ipiv, 0, v.plan);
    count_launch();
    for (int j0 = 0; j0 < np; j0 += NB) {
        const int nrest = (np - j0 - NB) / NB;
        if (nrest == 0) {
            lu_swap<float><<<(np + 127) / 128, 128, 0, s>>>(M, np, 0, np, j0, j0 + NB, v.plan);
            count_launch();
            break;
        }
        // what the next panel needs first: its block column swapped, its
        // block row of U, and this panel's update of it
        const int j1 = j0 + NB, j2 = j0 + 2 * NB;
        lu_swap<float><<<1, 128, 0, s>>>(M, np, j1, j2, j1, j1, v.plan);
        lu_trsm<float><<<1, NB, 0, s>>>(M, np, j0, j1);
        const int nt = (nrest * NB + GT - 1) / GT;
        lu_gemm_f32<<<dim3(nt, 1), 256, kGemmSmem32, s>>>(M, np, j0, j1, j2);
        count_launch(3);
        if ((e = cudaEventRecord(ready, s)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(side, ready, 0)) != cudaSuccess) return e;
        if (!panel_f32_cluster(M, np, j1, v, csize, side, e)) {
            lu_panel<float><<<1, PT, 0, side>>>(M, np, j1, v.ipiv, v.status);
            count_launch();
        }
        if (e != cudaSuccess) return e;
        // the rest beside the next panel: the other columns' row moves (the
        // plan is rewritten only after this, on the side stream), their
        // block row of U and the trailing update
        lu_swap<float><<<(np + 127) / 128, 128, 0, s>>>(M, np, 0, np, j0, j2, v.plan);
        count_launch();
        if (nrest > 1) {
            lu_trsm<float><<<nrest - 1, NB, 0, s>>>(M, np, j0, j2);
            lu_gemm_f32<<<dim3(nt, nrest / 2), 256, kGemmSmem32, s>>>(M, np, j0, j2, np);
            count_launch(2);
        }
        if ((e = cudaEventRecord(ready, s)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(side, ready, 0)) != cudaSuccess) return e;
        lu_swap_plan<<<1, 32, 0, side>>>(v.ipiv, j1, v.plan);
        count_launch();
        if ((e = cudaEventRecord(done, side)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(s, done, 0)) != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t sweeps(const T* M, const StackView& v, T* W, cudaStream_t s)
{
    // forward W -> Y, backward Y -> W
    const int np = v.np, nb = np / NB;
    const T* Inv = static_cast<const T*>(v.Inv);
    T* Y = static_cast<T*>(v.Y);
    for (int b = 0; b < nb; ++b) launch_sweep_step<T, true>(M, Inv, np, b, v.nc, W, Y, s);
    for (int b = nb - 1; b >= 0; --b) launch_sweep_step<T, false>(M, Inv, np, b, v.nc, Y, W, s);
    return cudaGetLastError();
}

}  // namespace

cudaError_t stack_gl_upload(cudaStream_t s)
{
    static double hx[kGl + 1][kGl], hw[kGl + 1][kGl];
    static float fx[kGl + 1][kGl], fw[kGl + 1][kGl];
    static bool ready = false;
    if (!ready) {
        hx[1][0] = 0.0;
        hw[1][0] = 2.0;
        for (int n = 2; n <= kGl; ++n) gl_nodes(n, hx[n], hw[n]);
        for (int n = 1; n <= kGl; ++n)
            for (int i = 0; i < n; ++i) {
                fx[n][i] = (float)hx[n][i];
                fw[n][i] = (float)hw[n][i];
            }
        ready = true;
    }
    cudaError_t e = cudaMemcpyToSymbolAsync(c_sx, hx, sizeof(hx), 0, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(c_sw, hw, sizeof(hw), 0, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(c_sxf, fx, sizeof(fx), 0, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(c_swf, fw, sizeof(fw), 0, cudaMemcpyHostToDevice, s);
    return e;
}

cudaError_t launch_stack_assemble(const StackView& v, long long tiles, bool mixed, cudaStream_t s)
{
    const size_t entries = (size_t)v.np * v.np;
    cudaError_t e = cudaMemsetAsync(v.M0, 0, sizeof(double) * entries, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(v.B, 0, sizeof(double) * (size_t)v.np * v.nc, s);
    if (e != cudaSuccess) return e;
    cudaEvent_t ev = trace_begin(s);
    if (mixed) stack_assemble<true><<<(unsigned)tiles, 256, 0, s>>>(v);
    else stack_assemble<false><<<(unsigned)tiles, 256, 0, s>>>(v);
    count_launch();
    trace_end(GBEM_KERNEL_ASSEMBLE, ev, s, 8.0 * (double)v.n_eq * v.n_eq, 0.0);
    if (v.np > v.n_eq) {
        stack_pad<<<(v.np - v.n_eq + 255) / 256, 256, 0, s>>>(v.M0, v.n_eq, v.np);
        count_launch();
    }
    // the copy the factorisation overwrites
    if (mixed) {
        to_f32<<<1024, 256, 0, s>>>(v.M0, v.M32, entries);
        count_launch();
    } else {
        e = cudaMemcpyAsync(v.M, v.M0, sizeof(double) * entries, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

cudaError_t launch_stack_lu(const StackView& v, bool mixed, cudaStream_t s, cudaStream_t side, cudaEvent_t ready,
                            cudaEvent_t done)
{
    cudaError_t e = mixed ? cudaFuncSetAttribute(lu_gemm_f32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)kGemmSmem32)
                          : cudaFuncSetAttribute(lu_gemm_f64, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)kGemmSmem64);
    if (e != cudaSuccess) return e;
    const size_t perm_smem = sizeof(int) * (size_t)v.np;
    if (perm_smem > 48 * 1024) {
        e = cudaFuncSetAttribute(lu_perm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)perm_smem);
        if (e != cudaSuccess) return e;
    }
    // traced as one span per factorisation: 2 np^3 / 3 flop, the matrix read
    // and written once
    cudaEvent_t ev = trace_begin(s);
    if (mixed) {
        const int csize = panel_cluster_size();
        e = side ? lu_run_lookahead(v.M32, v, csize, s, side, ready, done) : lu_run<float>(v.M32, v, s);
    } else {
        e = lu_run<double>(v.M, v, s);
    }
    if (e == cudaSuccess) {
        if (mixed) tri_inverse<float><<<v.np / NB, NB, 0, s>>>(v.M32, v.np, static_cast<float*>(v.Inv));
        else tri_inverse<double><<<v.np / NB, NB, 0, s>>>(v.M, v.np, static_cast<double*>(v.Inv));
        count_launch();
        e = cudaGetLastError();
    }
    const double n = (double)v.np;
    trace_end(GBEM_KERNEL_FACTOR, ev, s, (mixed ? 8.0 : 16.0) * n * n, 2.0 * n * n * n / 3.0);
    if (e != cudaSuccess) return e;
    lu_perm<<<1, 256, perm_smem, s>>>(v.ipiv, v.np, v.perm);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_stack_correct(const StackView& v, bool mixed, cudaStream_t s)
{
    const size_t count = (size_t)v.np * v.nc;
    cudaEvent_t ev = trace_begin(s);
    cudaError_t e;
    if (mixed) {
        float* W = reinterpret_cast<float*>(v.W);
        permute_rhs<float><<<256, 256, 0, s>>>(v.R, v.perm, v.np, v.nc, W);
        count_launch();
        e = sweeps<float>(v.M32, v, W, s);
        add_correction<float><<<256, 256, 0, s>>>(v.X, W, count);
    } else {
        double* W = reinterpret_cast<double*>(v.W);
        permute_rhs<double><<<256, 256, 0, s>>>(v.R, v.perm, v.np, v.nc, W);
        count_launch();
        e = sweeps<double>(v.M, v, W, s);
        add_correction<double><<<256, 256, 0, s>>>(v.X, W, count);
    }
    count_launch();
    // the two sweeps as one traced span: the factor read once, 2 np^2 nc flop
    const double n = (double)v.np;
    trace_end(GBEM_KERNEL_SWEEP, ev, s, (mixed ? 4.0 : 8.0) * n * n, 2.0 * n * n * v.nc);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_stack_residual(const StackView& v, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(v.norms, 0, sizeof(unsigned long long) * 2 * (size_t)v.nc, s);
    if (e != cudaSuccess) return e;
    cudaEvent_t ev = trace_begin(s);
    residual_partial<<<dim3((v.n_eq + 127) / 128, kResChunks), 128, 0, s>>>(v.M0, v.n_eq, v.np, v.nc, v.X, v.P);
    residual_finish<<<256, 256, 0, s>>>(v.B, v.P, v.n_eq, v.np, v.nc, v.R, v.norms, v.norms + v.nc);
    count_launch(2);
    trace_end(GBEM_KERNEL_RESIDUAL, ev, s, 8.0 * (double)v.n_eq * v.n_eq, 2.0 * (double)v.n_eq * v.n_eq * v.nc);
    return cudaGetLastError();
}

size_t stack_partial_bytes(int np, int nc) { return sizeof(double) * (size_t)kResChunks * np * nc; }

cudaError_t launch_stack_charges(const StackView& v, double eps0, cudaStream_t s)
{
    stack_charges<<<dim3(v.nc, v.nc), 256, 0, s>>>(v, v.X, eps0);
    count_launch();
    return cudaGetLastError();
}
