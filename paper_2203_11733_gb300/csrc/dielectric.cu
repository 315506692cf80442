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
// Entries are FP64: exact corner sums of closed forms (near_field.cuh) for
// near pairs, tensor Gauss-Legendre of both kernels at shared nodes for far
// pairs.  The matrix is not symmetric (Sec. 4), so it is factored by a
// right-looking blocked LU with partial pivoting (blocks of 64 columns): one
// CTA factors the panel (sub-panels of 8 columns, rank-8 updates between
// them), the row interchanges are applied to the other columns, a triangular
// solve forms the panel's block row of U, and a tiled FP64 update applies
// the panel to the trailing matrix.  No kernel here waits on another CTA.
#include <cstdio>

#include "gbem_internal.h"
#include "near_field.cuh"

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int kGl = 6;   // largest Gauss-Legendre order
__constant__ double c_sx[kGl + 1][kGl];
__constant__ double c_sw[kGl + 1][kGl];

__device__ __forceinline__ int axp(int k) { return k == 0 ? 1 : 0; }
__device__ __forceinline__ int axq(int k) { return k == 2 ? 1 : 2; }

struct PanelGeo {
    double c, lo0, hi0, lo1, hi1;
    int axis;
};

// U and D (D: the double layer for the normal +e_k of panel k) of one pair.
__device__ void pair_UD(const PanelGeo& I, const PanelGeo& K, double& U, double& D)
{
    const int ki = I.axis, kk = K.axis;
    double lo_i[3], hi_i[3], lo_k[3], hi_k[3];
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
    double g2 = 0.0, R2 = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double g = fmax(0.0, fmax(lo_k[d] - hi_i[d], lo_i[d] - hi_k[d]));
        g2 += g * g;
        const double e = fmax(hi_i[d], hi_k[d]) - fmin(lo_i[d], lo_k[d]);
        R2 += e * e;
    }
    const double ai = (I.hi0 - I.lo0) * (I.hi1 - I.lo1), ak = (K.hi0 - K.lo0) * (K.hi1 - K.lo1);
    const double lmax = fmax(fmax(I.hi0 - I.lo0, I.hi1 - I.lo1), fmax(K.hi0 - K.lo0, K.hi1 - K.lo1));
    const double q = sqrt(g2) / lmax;
    // closed forms while their corner sums lose at most about 2e-12
    // (eps R^4 / (|I_i| |I_k|), R the pair's bounding diagonal), and always
    // below q = 3, where the quadrature would need more than 6 points
    const bool closed = q < 3.0 || (q < 12.0 && R2 * R2 <= 9000.0 * ai * ak);
    if (closed) {
        double su = 0.0, sd = 0.0;
        if (ki == kk) {
            const double w = I.c - K.c;
#pragma unroll 1
            for (int c = 0; c < 16; ++c) {
                const int al = c & 1, be = (c >> 1) & 1, ga = (c >> 2) & 1, de = (c >> 3) & 1;
                const double u = (al ? I.hi0 : I.lo0) - (be ? K.hi0 : K.lo0);
                const double v = (ga ? I.hi1 : I.lo1) - (de ? K.hi1 : K.lo1);
                const double f = F_par(u, v, w);
                const double p = w != 0.0 ? Phi_par(u, v, w) : 0.0;
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
                const double h = H_orth(u, v, w);
                const double t = Theta_orth(u, v, w);
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
    // order for the double layer's relative error below about 1e-11
    const int n = q >= 320.0 ? 2 : q >= 40.0 ? 3 : q >= 10.0 ? 4 : q >= 5.0 ? 5 : 6;
    double d0[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) d0[d] = 0.5 * (lo_i[d] + hi_i[d]) - 0.5 * (lo_k[d] + hi_k[d]);
    const double hi_p = 0.5 * (I.hi0 - I.lo0), hi_q = 0.5 * (I.hi1 - I.lo1);
    const double hk_p = 0.5 * (K.hi0 - K.lo0), hk_q = 0.5 * (K.hi1 - K.lo1);
    const int ip = axp(ki), iq = axq(ki), kp = axp(kk), kq = axq(kk);
    double su = 0.0, sd = 0.0;
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
// columns: its panels I_k).  Tiles of region a are tile_off[a] .. .
__global__ void __launch_bounds__(256) stack_assemble(StackView v)
{
    const long long b = blockIdx.x;
    int a = 0;
    while (a + 1 < v.R && v.tile_off[a + 1] <= b) ++a;
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
    const double ea = v.eps[a];
    for (int e = tid; e < 1024; e += blockDim.x) {
        const int li = e & 31, lk = e >> 5;
        const int i = sp[li], k = sp[32 + lk];
        if (i < 0 || k < 0) continue;
        const long long row = r0 + ti * 32 + li;
        double U, D;
        pair_UD(sg[li], sg[32 + lk], U, D);
        const bool own = v.ra[k] == a;
        const double s = own ? (double)v.sign[k] : -(double)v.sign[k];
        double cu = s * D;
        if (i == k) cu += 0.5 * (sg[li].hi0 - sg[li].lo0) * (sg[li].hi1 - sg[li].lo1);
        const double g = own ? 1.0 : -v.eps[v.ra[k]] / ea;
        const size_t ld = (size_t)v.np;
        if (v.ucol[k] >= 0) v.M[row + (size_t)v.ucol[k] * ld] = cu;
        else if (v.bcol[k] >= 0) atomicAdd(&v.B[row + (size_t)v.bcol[k] * ld], -cu);
        if (v.qcol[k] >= 0) v.M[row + (size_t)v.qcol[k] * ld] = -U * g;
    }
}

// Rows and columns n_eq .. np-1 of M: the identity.
__global__ void stack_pad(double* M, int n_eq, int np)
{
    for (int r = n_eq + blockIdx.x * blockDim.x + threadIdx.x; r < np; r += gridDim.x * blockDim.x)
        M[(size_t)r + (size_t)r * np] = 1.0;
}

// ------------------------------------------------------------------ LU

constexpr int NB = 64;     // block columns
constexpr int SUB = 8;     // sub-panel columns
constexpr int PT = 512;    // panel threads

// argmax of |M[r, c]| over r in [c, np): the first row of the largest value.
__device__ int block_argmax(const double* __restrict__ col, int c, int np, double* sv, int* si)
{
    double best = -1.0;
    int bi = np;
    for (int r = c + threadIdx.x; r < np; r += blockDim.x) {
        const double x = fabs(col[r]);
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
__global__ void __launch_bounds__(PT) lu_panel(double* __restrict__ M, int np, int j0, int* __restrict__ ipiv,
                                               int* status)
{
    __shared__ double sv[PT / 32];
    __shared__ int si[PT / 32];
    __shared__ double urow[NB];
    __shared__ double ublk[SUB][NB];
    const size_t ld = (size_t)np;
    const int tid = threadIdx.x;
    for (int s0 = j0; s0 < j0 + NB; s0 += SUB) {
        for (int c = s0; c < s0 + SUB; ++c) {
            double* col = M + (size_t)c * ld;
            int p = block_argmax(col, c, np, sv, si);
            if (p >= np) {   // no comparable value (NaN entries): keep the row, flag the system
                p = c;
                if (tid == 0) atomicExch(status, (int)GBEM_ERR_NOT_SPD);
            }
            if (tid == 0) ipiv[c] = p;
            // swap rows c and p across the panel's columns
            if (p != c && tid < NB) {
                double* e = M + (size_t)(j0 + tid) * ld;
                const double t = e[c];
                e[c] = e[p];
                e[p] = t;
            }
            __syncthreads();
            const double piv = col[c];
            if (piv == 0.0) {
                if (tid == 0) atomicExch(status, (int)GBEM_ERR_NOT_SPD);
                __syncthreads();
                continue;
            }
            if (tid < s0 + SUB - c - 1) urow[tid] = M[(size_t)c + (size_t)(c + 1 + tid) * ld];
            __syncthreads();
            const double inv = 1.0 / piv;
            const int ncol = s0 + SUB - c - 1;
            for (int r = c + 1 + tid; r < np; r += PT) {
                const double l = col[r] * inv;
                col[r] = l;
                for (int k = 0; k < ncol; ++k) {
                    double* e = M + (size_t)(c + 1 + k) * ld + r;
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
            double x[SUB];
#pragma unroll
            for (int r = 0; r < SUB; ++r) {
                double t = M[(size_t)(s0 + r) + (size_t)cc * ld];
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
            double l[SUB];
#pragma unroll
            for (int k = 0; k < SUB; ++k) l[k] = M[(size_t)r + (size_t)(s0 + k) * ld];
            for (int j = 0; j < rest; ++j) {
                double* e = M + (size_t)(s0 + SUB + j) * ld + r;
                double t = *e;
#pragma unroll
                for (int k = 0; k < SUB; ++k) t = fma(-l[k], ublk[k][j], t);
                *e = t;
            }
        }
        __syncthreads();
    }
}

// The panel's interchanges applied, in order, to every column outside it.
__global__ void lu_swap(double* __restrict__ M, int np, int j0, const int* __restrict__ ipiv)
{
    __shared__ int piv[NB];
    if (threadIdx.x < NB) piv[threadIdx.x] = ipiv[j0 + threadIdx.x];
    __syncthreads();
    const int ncols = np - NB;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ncols; t += gridDim.x * blockDim.x) {
        const int c = t < j0 ? t : t + NB;
        double* e = M + (size_t)c * np;
        for (int k = 0; k < NB; ++k) {
            const int p = piv[k], r = j0 + k;
            if (p != r) {
                const double x = e[r];
                e[r] = e[p];
                e[p] = x;
            }
        }
    }
}

// U12 = L11^-1 A12 for 64 columns per CTA (L11 the panel's unit lower block).
__global__ void __launch_bounds__(NB) lu_trsm(double* __restrict__ M, int np, int j0)
{
    __shared__ double L[NB][NB + 1];
    const size_t ld = (size_t)np;
    const int tid = threadIdx.x;
    for (int e = tid; e < NB * NB; e += NB) {
        const int r = e % NB, c = e / NB;
        L[r][c] = M[(size_t)(j0 + r) + (size_t)(j0 + c) * ld];
    }
    __syncthreads();
    const int cc = j0 + NB + blockIdx.x * NB + tid;
    double* col = M + (size_t)cc * ld + j0;
    double x[NB];
#pragma unroll
    for (int r = 0; r < NB; ++r) x[r] = col[r];
#pragma unroll
    for (int r = 1; r < NB; ++r) {
        double t = x[r];
#pragma unroll
        for (int k = 0; k < r; ++k) t = fma(-L[r][k], x[k], t);
        x[r] = t;
    }
#pragma unroll
    for (int r = 0; r < NB; ++r) col[r] = x[r];
}

// A22 -= L21 U12, one 64 x 64 tile per CTA, 4 x 4 outputs per thread.
constexpr size_t kGemmSmem = 2 * sizeof(double) * NB * (NB + 1);
__global__ void __launch_bounds__(256) lu_gemm(double* __restrict__ M, int np, int j0)
{
    extern __shared__ double gsm[];
    double(*Ls)[NB + 1] = reinterpret_cast<double(*)[NB + 1]>(gsm);            // Ls[k][r] = L21[r][k]
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

// X[r, m] = B[perm[r], m]
__global__ void permute_rhs(const double* __restrict__ B, const int* __restrict__ perm, int np, int nc,
                            double* __restrict__ X)
{
    const long long total = (long long)np * nc;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e % np), m = (int)(e / np);
        X[e] = B[(size_t)perm[r] + (size_t)m * np];
    }
}

// Diagonal block b of the forward (unit lower) or backward (upper) sweep:
// X_b := T_bb^-1 X_b; thread r owns row r of the block, 16 right-hand sides
// at a time, one barrier per eliminated row.
template <bool LOWER>
__global__ void __launch_bounds__(NB) tri_block(const double* __restrict__ M, int np, int b, int nc,
                                                double* __restrict__ X)
{
    __shared__ double T[NB][NB + 1];
    __shared__ double xs[NB][17];
    const size_t ld = (size_t)np;
    const int j0 = b * NB, r = threadIdx.x;
    for (int e = threadIdx.x; e < NB * NB; e += NB) {
        const int i = e % NB, c = e / NB;
        T[i][c] = M[(size_t)(j0 + i) + (size_t)(j0 + c) * ld];
    }
    for (int m0 = 0; m0 < nc; m0 += 16) {
        const int mn = min(16, nc - m0);
        __syncthreads();
        for (int m = 0; m < mn; ++m) xs[r][m] = X[(size_t)(m0 + m) * np + j0 + r];
        __syncthreads();
        if (LOWER) {
            for (int k = 0; k < NB - 1; ++k) {
                if (r > k)
                    for (int m = 0; m < mn; ++m) xs[r][m] = fma(-T[r][k], xs[k][m], xs[r][m]);
                __syncthreads();
            }
        } else {
            for (int k = NB - 1; k >= 0; --k) {
                if (r == k)
                    for (int m = 0; m < mn; ++m) xs[k][m] = xs[k][m] / T[k][k];
                __syncthreads();
                if (r < k)
                    for (int m = 0; m < mn; ++m) xs[r][m] = fma(-T[r][k], xs[k][m], xs[r][m]);
                __syncthreads();
            }
        }
        for (int m = 0; m < mn; ++m) X[(size_t)(m0 + m) * np + j0 + r] = xs[r][m];
    }
}

// X[r] -= M[r, block b] X_b for the rows below block b (LOWER) or above it.
template <bool LOWER>
__global__ void __launch_bounds__(256) tri_update(const double* __restrict__ M, int np, int b, int nc,
                                                  double* __restrict__ X)
{
    __shared__ double xb[16][NB];
    const size_t ld = (size_t)np;
    const int j0 = b * NB;
    const int rlo = LOWER ? j0 + NB : 0, rhi = LOWER ? np : j0;
    for (int m0 = 0; m0 < nc; m0 += 16) {
        const int mn = min(16, nc - m0);
        __syncthreads();
        for (int e = threadIdx.x; e < mn * NB; e += blockDim.x)
            xb[e / NB][e % NB] = X[(size_t)(m0 + e / NB) * np + j0 + e % NB];
        __syncthreads();
        for (int r = rlo + blockIdx.x * blockDim.x + threadIdx.x; r < rhi; r += gridDim.x * blockDim.x) {
            double acc[16] = {};
            for (int k = 0; k < NB; ++k) {
                const double l = M[(size_t)r + (size_t)(j0 + k) * ld];
#pragma unroll
                for (int m = 0; m < 16; ++m) acc[m] = fma(l, xb[m][k], acc[m]);
            }
            for (int m = 0; m < mn; ++m) X[(size_t)(m0 + m) * np + r] -= acc[m];
        }
    }
}

// R = B - M X over the first n_eq rows; rnorm[m] = max |R[., m]| / max |B[., m]|
// accumulated by atomicMax on the bit patterns of non-negative doubles.
__global__ void __launch_bounds__(256) stack_residual(const double* __restrict__ M, int n_eq, int np, int nc,
                                                      const double* __restrict__ B, const double* __restrict__ X,
                                                      unsigned long long* rmax, unsigned long long* bmax)
{
    const size_t ld = (size_t)np;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n_eq; r += gridDim.x * blockDim.x)
        for (int m = 0; m < nc; ++m) {
            double t = B[(size_t)r + (size_t)m * ld];
            const double b = fabs(t);
            const double* x = X + (size_t)m * ld;
            for (int c = 0; c < n_eq; ++c) t = fma(-M[(size_t)r + (size_t)c * ld], x[c], t);
            atomicMax(rmax + m, (unsigned long long)__double_as_longlong(fabs(t)));
            atomicMax(bmax + m, (unsigned long long)__double_as_longlong(b));
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

}  // namespace

cudaError_t stack_gl_upload(cudaStream_t s)
{
    static double hx[kGl + 1][kGl], hw[kGl + 1][kGl];
    static bool ready = false;
    if (!ready) {
        hx[1][0] = 0.0;
        hw[1][0] = 2.0;
        for (int n = 2; n <= kGl; ++n) gl_nodes(n, hx[n], hw[n]);
        ready = true;
    }
    cudaError_t e = cudaMemcpyToSymbolAsync(c_sx, hx, sizeof(hx), 0, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(c_sw, hw, sizeof(hw), 0, cudaMemcpyHostToDevice, s);
    return e;
}

cudaError_t launch_stack_assemble(const StackView& v, long long tiles, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(v.M, 0, sizeof(double) * (size_t)v.np * v.np, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(v.B, 0, sizeof(double) * (size_t)v.np * v.nc, s);
    if (e != cudaSuccess) return e;
    cudaEvent_t ev = trace_begin(s);
    stack_assemble<<<(unsigned)tiles, 256, 0, s>>>(v);
    count_launch();
    trace_end(GBEM_KERNEL_ASSEMBLE, ev, s, 8.0 * (double)v.n_eq * v.n_eq, 0.0);
    if (v.np > v.n_eq) {
        stack_pad<<<(v.np - v.n_eq + 255) / 256, 256, 0, s>>>(v.M, v.n_eq, v.np);
        count_launch();
    }
    return cudaGetLastError();
}

cudaError_t launch_stack_lu(const StackView& v, cudaStream_t s)
{
    const int np = v.np;
    cudaError_t e = cudaFuncSetAttribute(lu_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGemmSmem);
    if (e != cudaSuccess) return e;
    // traced as one span per factorisation: 2 np^3 / 3 flop, the matrix read
    // and written once
    cudaEvent_t ev = trace_begin(s);
    for (int j0 = 0; j0 < np; j0 += NB) {
        lu_panel<<<1, PT, 0, s>>>(v.M, np, j0, v.ipiv, v.status);
        lu_swap<<<(np + 255) / 256, 256, 0, s>>>(v.M, np, j0, v.ipiv);
        count_launch(2);
        const int nrest = (np - j0 - NB) / NB;
        if (nrest > 0) {
            lu_trsm<<<nrest, NB, 0, s>>>(v.M, np, j0);
            lu_gemm<<<dim3(nrest, nrest), 256, kGemmSmem, s>>>(v.M, np, j0);
            count_launch(2);
        }
    }
    const double n = (double)np;
    trace_end(GBEM_KERNEL_FACTOR, ev, s, 16.0 * n * n, 2.0 * n * n * n / 3.0);
    return cudaGetLastError();
}

cudaError_t launch_stack_solve(const StackView& v, double* X, int* perm, unsigned long long* norms,
                               double eps0, cudaStream_t s)
{
    const int np = v.np, nb = np / NB;
    const size_t perm_smem = sizeof(int) * (size_t)np;
    if (perm_smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(lu_perm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)perm_smem);
        if (e != cudaSuccess) return e;
    }
    lu_perm<<<1, 256, perm_smem, s>>>(v.ipiv, np, perm);
    permute_rhs<<<256, 256, 0, s>>>(v.B, perm, np, v.nc, X);
    count_launch(2);
    const int ug = 2 * 152;
    // the two sweeps as one traced span: the factor read once, 2 np^2 nc flop
    cudaEvent_t ev = trace_begin(s);
    for (int b = 0; b < nb; ++b) {
        tri_block<true><<<1, NB, 0, s>>>(v.M, np, b, v.nc, X);
        count_launch();
        if (b + 1 < nb) {
            tri_update<true><<<ug, 256, 0, s>>>(v.M, np, b, v.nc, X);
            count_launch();
        }
    }
    for (int b = nb - 1; b >= 0; --b) {
        tri_block<false><<<1, NB, 0, s>>>(v.M, np, b, v.nc, X);
        count_launch();
        if (b > 0) {
            tri_update<false><<<ug, 256, 0, s>>>(v.M, np, b, v.nc, X);
            count_launch();
        }
    }
    trace_end(GBEM_KERNEL_SWEEP, ev, s, 8.0 * (double)np * np, 2.0 * (double)np * np * v.nc);
    cudaError_t e = cudaMemsetAsync(norms, 0, sizeof(unsigned long long) * 2 * (size_t)v.nc, s);
    if (e != cudaSuccess) return e;
    stack_charges<<<dim3(v.nc, v.nc), 256, 0, s>>>(v, X, eps0);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_stack_residual(const StackView& v, const double* M0, const double* X,
                                  unsigned long long* norms, cudaStream_t s)
{
    cudaEvent_t ev = trace_begin(s);
    stack_residual<<<(v.n_eq + 255) / 256, 256, 0, s>>>(M0, v.n_eq, v.np, v.nc, v.B, X, norms, norms + v.nc);
    count_launch();
    trace_end(GBEM_KERNEL_RESIDUAL, ev, s, 8.0 * (double)v.n_eq * v.n_eq, 2.0 * (double)v.n_eq * v.n_eq * v.nc);
    return cudaGetLastError();
}
