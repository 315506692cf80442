// Galerkin entries over flat triangles (general conductors), in FP64:
//
//   a_ij = 1/(4 pi |T_i| |T_j|) int_{T_i} int_{T_j} 1/|x - y| dy dx
//
// (Eq. "matrix" of Sec. 3.1 with triangles for panels).  One CTA owns one
// 32x32 tile of the lower triangle; every pair is classified, the tile's
// pairs are sorted by class, and each class is evaluated by full warps:
//
//  * the same triangle: the closed form of the self-integral,
//    (4 |T|^2 / 3) sum_i ln(((l_i + l_j)^2 - l_k^2) / (l_j^2 - (l_i - l_k)^2)) / l_i
//    over the sides (l_i, l_j, l_k) in turn;
//  * triangles sharing a vertex or a side: the exact potential of one
//    triangle (edge-by-edge closed form) integrated over the other with a
//    tanh-sinh rule in both coordinates of its collapsed map (39 x 39
//    points; 25 x 25 in mixed mode), whose sides all lie on the unit
//    square's boundary, where the rule converges fast despite the
//    potential's singular derivatives there;
//  * centroid distance below 3 diameters: the exact potential over the four
//    midpoint children of the other triangle, collapsed Gauss-Legendre of
//    order 8 on each (one order-6 rule in mixed mode);
//  * farther: the collapsed Gauss-Legendre product rule of order 3..6 on
//    both triangles (calibrated to about 1e-11 relative), in FP32 with FP64
//    outer sums in mixed mode (about 1e-7).
// The mixed precision stores each entry as a float pair and its FP32 copy,
// as the rectangle assembly does.
#include <cmath>

#include "gbem_internal.h"
#include "near_field.cuh"

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int kTriTile = 32;
constexpr int kMaxGl = 8;
constexpr int kTsMax = 40;
__constant__ double c_tgx[kMaxGl + 1][kMaxGl];   // Gauss-Legendre nodes on [0, 1]
__constant__ double c_tgw[kMaxGl + 1][kMaxGl];
__constant__ double c_tsx[2][kTsMax];             // tanh-sinh nodes on [0, 1]: step 1/6, 1/4
__constant__ double c_tsw[2][kTsMax];
__constant__ int c_tsn[2];

struct Tri {
    double v[3][3];
};

__device__ __forceinline__ void sub3(const double* a, const double* b, double* c)
{
    c[0] = a[0] - b[0];
    c[1] = a[1] - b[1];
    c[2] = a[2] - b[2];
}
__device__ __forceinline__ void cross3(const double* a, const double* b, double* c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
__device__ __forceinline__ double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

__device__ __forceinline__ double tri_area(const Tri& T)
{
    double e1[3], e2[3], n[3];
    sub3(T.v[1], T.v[0], e1);
    sub3(T.v[2], T.v[0], e2);
    cross3(e1, e2, n);
    return 0.5 * sqrt(dot3(n, n));
}

// Per-edge data of the potential of a triangle: the unit normal, each edge's
// start, unit direction and outward in-plane normal.
struct TriFrame {
    double n[3];
    double p[3][3], l[3][3], u[3][3];
};

__device__ void tri_frame(const Tri& T, TriFrame& F)
{
    double e1[3], e2[3];
    sub3(T.v[1], T.v[0], e1);
    sub3(T.v[2], T.v[0], e2);
    cross3(e1, e2, F.n);
    const double nn = 1.0 / sqrt(dot3(F.n, F.n));
    for (int d = 0; d < 3; ++d) F.n[d] *= nn;
    for (int e = 0; e < 3; ++e) {
        double t[3];
        sub3(T.v[(e + 1) % 3], T.v[e], t);
        const double il = 1.0 / sqrt(dot3(t, t));
        for (int d = 0; d < 3; ++d) {
            F.p[e][d] = T.v[e][d];
            F.l[e][d] = t[d] * il;
        }
        cross3(F.l[e], F.n, F.u[e]);
    }
}

// ln(R + l) with R = sqrt(l^2 + r0sq), the l < 0 branch without cancellation.
__device__ __forceinline__ double lnp(double l, double r0sq, double R) { return l >= 0.0 ? log(R + l) : log(r0sq / (R - l)); }

// int_T 1/|x - y| dy: per edge, with x at height h over its projection rho,
// P0 ln((R+ + l+)/(R- + l-)) - |h| (atan(P0 l+/(R0^2 + |h| R+)) -
// atan(P0 l-/(R0^2 + |h| R-))), l+- the edge ends along the edge from rho,
// P0 the distance of rho from the edge line (positive inside).
__device__ double tri_potential(const TriFrame& F, const double* x)
{
    double xp[3];
    sub3(x, F.p[0], xp);
    const double h = dot3(xp, F.n), ah = fabs(h);
    double s = 0.0;
#pragma unroll 1
    for (int e = 0; e < 3; ++e) {
        double pm[3];
        for (int d = 0; d < 3; ++d) pm[d] = F.p[e][d] - (x[d] - h * F.n[d]);
        const double lm = dot3(pm, F.l[e]);
        const double P0 = dot3(pm, F.u[e]);
        if (P0 == 0.0) continue;
        double qm[3];
        for (int d = 0; d < 3; ++d) qm[d] = F.p[(e + 1) % 3][d] - (x[d] - h * F.n[d]);
        const double lq = dot3(qm, F.l[e]);
        const double r0sq = P0 * P0 + h * h;
        const double Rp = sqrt(lq * lq + r0sq), Rm = sqrt(lm * lm + r0sq);
        s += P0 * (lnp(lq, r0sq, Rp) - lnp(lm, r0sq, Rm));
        if (ah != 0.0) s -= ah * (atan(P0 * lq / (r0sq + ah * Rp)) - atan(P0 * lm / (r0sq + ah * Rm)));
    }
    return s;
}

// The closed form of int_T int_T 1/|x - y|.
__device__ double tri_self(const Tri& T, double area)
{
    double l[3];
    for (int e = 0; e < 3; ++e) {
        double t[3];
        sub3(T.v[(e + 1) % 3], T.v[e], t);
        l[e] = sqrt(dot3(t, t));
    }
    double s = 0.0;
    for (int i = 0; i < 3; ++i) {
        const double a = l[i], b = l[(i + 1) % 3], c = l[(i + 2) % 3];
        s += log(((a + b) * (a + b) - c * c) / (b * b - (a - c) * (a - c))) / a;
    }
    return (4.0 / 3.0) * area * area * s;
}

// int over triangle (a, b, c) of the potential of F, by the collapsed map
// y = a + xi ((b - a) + eta (c - b)) with Gauss-Legendre of order m (ts < 0)
// or tanh-sinh rule ts (0: step 1/6, 1: step 1/4) in both coordinates.
__device__ double outer_rule(const double* a, const double* b, const double* c, const TriFrame& F, int m, int ts)
{
    double ab[3], bc[3], cr[3];
    sub3(b, a, ab);
    sub3(c, b, bc);
    cross3(ab, bc, cr);
    const double j2 = sqrt(dot3(cr, cr));
    const bool t = ts >= 0;
    const int n = t ? c_tsn[ts] : m;
    double s = 0.0;
#pragma unroll 1
    for (int i = 0; i < n; ++i) {
        const double xi = t ? c_tsx[ts][i] : c_tgx[m][i], wx = t ? c_tsw[ts][i] : c_tgw[m][i];
        double row = 0.0;
#pragma unroll 1
        for (int k = 0; k < n; ++k) {
            const double eta = t ? c_tsx[ts][k] : c_tgx[m][k], we = t ? c_tsw[ts][k] : c_tgw[m][k];
            double y[3];
            for (int d = 0; d < 3; ++d) y[d] = a[d] + xi * (ab[d] + eta * bc[d]);
            row += we * tri_potential(F, y);
        }
        s += wx * xi * row;
    }
    return s * j2;
}

__device__ __forceinline__ float mufu_rsqrt(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// The same product rule in FP32 (mixed mode): node offsets from the FP64
// vertex difference, FP32 inner sums, FP64 outer sum; about 1e-7 relative.
__device__ double far_rule_f32(const Tri& A, const Tri& B, int n)
{
    float ab1[3], bc1[3], ab2[3], bc2[3], d0[3];
    double cr[3], e1[3], e2[3];
    for (int d = 0; d < 3; ++d) {
        ab1[d] = (float)(A.v[1][d] - A.v[0][d]);
        bc1[d] = (float)(A.v[2][d] - A.v[1][d]);
        ab2[d] = (float)(B.v[1][d] - B.v[0][d]);
        bc2[d] = (float)(B.v[2][d] - B.v[1][d]);
        d0[d] = (float)(A.v[0][d] - B.v[0][d]);
    }
    sub3(A.v[1], A.v[0], e1);
    sub3(A.v[2], A.v[1], e2);
    cross3(e1, e2, cr);
    const double j1 = sqrt(dot3(cr, cr));
    sub3(B.v[1], B.v[0], e1);
    sub3(B.v[2], B.v[1], e2);
    cross3(e1, e2, cr);
    const double j2 = sqrt(dot3(cr, cr));
    double s = 0.0;
#pragma unroll 1
    for (int i = 0; i < n; ++i)
#pragma unroll 1
        for (int k = 0; k < n; ++k) {
            const float xi = (float)c_tgx[n][i], xk = (float)c_tgx[n][k];
            float x[3];
            for (int d = 0; d < 3; ++d) x[d] = d0[d] + xi * (ab1[d] + xk * bc1[d]);
            float t = 0.0f;
#pragma unroll 1
            for (int p = 0; p < n; ++p) {
                const float xp = (float)c_tgx[n][p], wp = (float)(c_tgw[n][p] * c_tgx[n][p]);
#pragma unroll 1
                for (int q = 0; q < n; ++q) {
                    const float xq = (float)c_tgx[n][q];
                    float r[3];
                    for (int d = 0; d < 3; ++d) r[d] = x[d] - xp * (ab2[d] + xq * bc2[d]);
                    t = fmaf(wp * (float)c_tgw[n][q], mufu_rsqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]), t);
                }
            }
            s += c_tgw[n][i] * c_tgw[n][k] * c_tgx[n][i] * (double)t;
        }
    return s * j1 * j2;
}

// Collapsed Gauss-Legendre product rule of order n on both triangles.
__device__ double far_rule(const Tri& A, const Tri& B, int n)
{
    double ab1[3], bc1[3], ab2[3], bc2[3], cr[3];
    sub3(A.v[1], A.v[0], ab1);
    sub3(A.v[2], A.v[1], bc1);
    sub3(B.v[1], B.v[0], ab2);
    sub3(B.v[2], B.v[1], bc2);
    cross3(ab1, bc1, cr);
    const double j1 = sqrt(dot3(cr, cr));
    cross3(ab2, bc2, cr);
    const double j2 = sqrt(dot3(cr, cr));
    double s = 0.0;
#pragma unroll 1
    for (int i = 0; i < n; ++i)
#pragma unroll 1
        for (int k = 0; k < n; ++k) {
            double x[3];
            for (int d = 0; d < 3; ++d) x[d] = A.v[0][d] + c_tgx[n][i] * (ab1[d] + c_tgx[n][k] * bc1[d]) - B.v[0][d];
            double t = 0.0;
#pragma unroll 1
            for (int p = 0; p < n; ++p)
#pragma unroll 1
                for (int q = 0; q < n; ++q) {
                    double r[3];
                    for (int d = 0; d < 3; ++d) r[d] = x[d] - c_tgx[n][p] * (ab2[d] + c_tgx[n][q] * bc2[d]);
                    t += c_tgw[n][p] * c_tgw[n][q] * c_tgx[n][p] * rsq64(dot3(r, r));
                }
            s += c_tgw[n][i] * c_tgw[n][k] * c_tgx[n][i] * t;
        }
    return s * j1 * j2;
}

__device__ bool share_vertex(const Tri& A, const Tri& B)
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            if (A.v[i][0] == B.v[j][0] && A.v[i][1] == B.v[j][1] && A.v[i][2] == B.v[j][2]) return true;
    return false;
}

// Evaluation class: 0 the same triangle, 1 sharing a vertex, 2 near, else
// the far rule's order.
__device__ int tri_class(const Tri& A, const Tri& B, bool same)
{
    if (same) return 0;
    if (share_vertex(A, B)) return 1;
    double ca[3], cb[3], dmax = 0.0;
    for (int d = 0; d < 3; ++d) {
        ca[d] = (A.v[0][d] + A.v[1][d] + A.v[2][d]) / 3.0;
        cb[d] = (B.v[0][d] + B.v[1][d] + B.v[2][d]) / 3.0;
    }
    for (int i = 0; i < 3; ++i)
        for (int j = i + 1; j < 3; ++j) {
            double t[3];
            sub3(A.v[i], A.v[j], t);
            dmax = fmax(dmax, dot3(t, t));
            sub3(B.v[i], B.v[j], t);
            dmax = fmax(dmax, dot3(t, t));
        }
    double t[3];
    sub3(ca, cb, t);
    const double r = sqrt(dot3(t, t) / dmax);
    if (r < 3.0) return 2;
    return r >= 40.0 ? 3 : r >= 10.0 ? 4 : r >= 4.0 ? 5 : 6;
}

template <bool MIXED>
__device__ double tri_pair(const Tri& A, const Tri& B, int cls, double aa, double ab)
{
    if (cls == 0) return tri_self(A, aa);
    if (cls >= 3) return MIXED ? far_rule_f32(A, B, cls) : far_rule(A, B, cls);
    // the smaller triangle carries the outer rule (the integral is symmetric)
    const Tri& O = aa <= ab ? A : B;
    const Tri& I = aa <= ab ? B : A;
    TriFrame F;
    tri_frame(I, F);
    // mixed mode: the coarser tanh-sinh rule (about 1e-10) and one order-6
    // rule for near pairs (about 1e-8), both far below its FP32 far field
    if (cls == 1) return outer_rule(O.v[0], O.v[1], O.v[2], F, 0, MIXED ? 1 : 0);
    if (MIXED) return outer_rule(O.v[0], O.v[1], O.v[2], F, 6, -1);
    double m01[3], m12[3], m20[3];
    for (int d = 0; d < 3; ++d) {
        m01[d] = 0.5 * (O.v[0][d] + O.v[1][d]);
        m12[d] = 0.5 * (O.v[1][d] + O.v[2][d]);
        m20[d] = 0.5 * (O.v[2][d] + O.v[0][d]);
    }
    return outer_rule(O.v[0], m01, m20, F, 8, -1) + outer_rule(m01, O.v[1], m12, F, 8, -1) +
           outer_rule(m20, m12, O.v[2], F, 8, -1) + outer_rule(m01, m12, m20, F, 8, -1);
}

template <bool MIXED>
__global__ void __launch_bounds__(256) assemble_tri(const double* __restrict__ tri, int n, int np,
                                                     double* __restrict__ A64, float* __restrict__ A32,
                                                     unsigned long long* __restrict__ counts)
{
    const long long b = blockIdx.x;
    int TI = (int)((sqrt(8.0 * (double)b + 1.0) - 1.0) * 0.5);
    while ((long long)TI * (TI + 1) / 2 > b) --TI;
    while ((long long)(TI + 1) * (TI + 2) / 2 <= b) ++TI;
    const int TJ = (int)(b - (long long)TI * (TI + 1) / 2);
    __shared__ Tri st[2 * kTriTile];
    __shared__ double sa[2 * kTriTile];
    __shared__ unsigned char cls_s[kTriTile * kTriTile];
    __shared__ unsigned short order[kTriTile * kTriTile];
    __shared__ int cnt[8], pos[8];
    const int tid = threadIdx.x;
    if (tid < 2 * kTriTile) {
        const int g = tid < kTriTile ? TI * kTriTile + tid : TJ * kTriTile + tid - kTriTile;
        if (g < n) {
            for (int k = 0; k < 3; ++k)
                for (int d = 0; d < 3; ++d) st[tid].v[k][d] = tri[(size_t)g * 9 + 3 * k + d];
            sa[tid] = tri_area(st[tid]);
        }
    }
    if (tid < 8) cnt[tid] = 0;
    __syncthreads();
    for (int e = tid; e < kTriTile * kTriTile; e += blockDim.x) {
        const int li = e & 31, lj = e >> 5;
        const int i = TI * kTriTile + li, j = TJ * kTriTile + lj;
        const int c = (i >= n || j >= n || j > i) ? 7 : tri_class(st[li], st[kTriTile + lj], i == j);
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
    if (counts && tid < 7 && cnt[tid]) atomicAdd(counts + tid, (unsigned long long)cnt[tid]);
    __syncthreads();
    for (int e = tid; e < kTriTile * kTriTile; e += blockDim.x) order[atomicAdd(&pos[cls_s[e]], 1)] = (unsigned short)e;
    __syncthreads();
    const int total = kTriTile * kTriTile - cnt[7];
    for (int t = tid; t < total; t += blockDim.x) {
        const int e = order[t];
        const int li = e & 31, lj = e >> 5;
        const int i = TI * kTriTile + li, j = TJ * kTriTile + lj;
        const double ai = sa[li], aj = sa[kTriTile + lj];
        const double v = tri_pair<MIXED>(st[li], st[kTriTile + lj], cls_s[e], ai, aj) / (4.0 * kPi * ai * aj);
        const size_t at = (size_t)i + (size_t)j * np;
        if constexpr (MIXED) {
            const float h = __double2float_rn(v);
            reinterpret_cast<float2*>(A64)[at] = make_float2(h, __double2float_rn(v - (double)h));
            A32[at] = h;
        } else {
            A64[at] = v;
        }
    }
}

}  // namespace

cudaError_t tri_tables_upload(cudaStream_t s)
{
    static double gx[kMaxGl + 1][kMaxGl], gw[kMaxGl + 1][kMaxGl], tx[2][kTsMax], tw[2][kTsMax];
    static int tn[2] = {0, 0};
    if (tn[0] == 0) {
        for (int m = 2; m <= kMaxGl; ++m) {
            double x[kMaxGl], w[kMaxGl];
            gl_nodes(m, x, w);
            for (int i = 0; i < m; ++i) {
                gx[m][i] = 0.5 * (x[i] + 1.0);
                gw[m][i] = 0.5 * w[i];
            }
        }
        // tanh-sinh on [0, 1], steps 1/6 and 1/4, |t| <= 3.2:
        // x = 1/(1 + exp(-pi sinh t)), each node formed from its nearer end
        const double hp = 0.5 * 3.14159265358979323846;
        for (int r = 0; r < 2; ++r) {
            const double h = r == 0 ? 1.0 / 6.0 : 0.25;
            const int k = (int)(3.2 / h);
            for (int i = -k; i <= k && tn[r] < kTsMax; ++i) {
                const double t = i * h, sh = hp * std::sinh(t), ch = std::cosh(sh);
                const double d = 1.0 / (1.0 + std::exp(2.0 * std::fabs(sh)));
                tx[r][tn[r]] = i < 0 ? d : (i > 0 ? 1.0 - d : 0.5);
                tw[r][tn[r]] = h * 0.5 * hp * std::cosh(t) / (ch * ch);
                ++tn[r];
            }
        }
    }
    cudaError_t e = cudaMemcpyToSymbolAsync(c_tgx, gx, sizeof(gx), 0, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(c_tgw, gw, sizeof(gw), 0, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(c_tsx, tx, sizeof(tx), 0, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(c_tsw, tw, sizeof(tw), 0, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(c_tsn, tn, sizeof(tn), 0, cudaMemcpyHostToDevice, s);
    return e;
}

cudaError_t launch_assemble_tri(const double* tri, int n, int np, gbem_precision prec, double* A64, float* A32,
                                unsigned long long* counts, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    cudaError_t e = tri_tables_upload(s);
    if (e != cudaSuccess) return e;
    const long long nt = (n + kTriTile - 1) / kTriTile;
    const long long tiles = nt * (nt + 1) / 2;
    cudaEvent_t ev = trace_begin(s);
    if (prec == GBEM_MIXED) assemble_tri<true><<<(unsigned)tiles, 256, 0, s>>>(tri, n, np, A64, A32, counts);
    else assemble_tri<false><<<(unsigned)tiles, 256, 0, s>>>(tri, n, np, A64, nullptr, counts);
    count_launch();
    trace_end(GBEM_KERNEL_ASSEMBLE, ev, s, (double)tiles * kTriTile * kTriTile * (prec == GBEM_MIXED ? 12.0 : 8.0),
              0.0);
    return cudaGetLastError();
}
