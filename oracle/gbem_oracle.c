/*
 * FP64 CPU oracle for the Galerkin single-layer matrix of Wu & Li, "GBEM:
 * Galerkin Boundary Element Method for 3-D Capacitance Extraction"
 * (arXiv 2203.11733).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file; only the tests, the package smoke check and the CPU
 * baseline leg of the benchmark use it.  It shares no code, header, table or
 * constant with the CUDA path.
 *
 * What it computes (Sec. 3.1, Eq. "matrix"; Sec. 3.4):
 *     a_ij = 1 / (4 pi |I_i| |I_j|) * int_{I_i} int_{I_j} 1/|x - y| dy dx
 * for axis-aligned rectangular panels I_i, I_j (Sec. 3.3: all conductors are
 * cuboids, so every panel is an axis-aligned rectangle).
 *
 * Method (deliberately different from the GPU path, which uses 4-D corner
 * sums and low-order tensor Gauss-Legendre rules):
 *   - the inner integral over I_j is the exact potential of a uniformly
 *     charged rectangle at the point x (textbook corner formula),
 *   - the outer integral over I_i is a 2-D quadrature: I_i is cut along the
 *     lines where the inner potential is not smooth (the projections of
 *     I_j's edges, or I_j's plane when it is perpendicular); each piece that
 *     touches I_j uses tanh-sinh (double exponential) quadrature with levels
 *     refined until two levels agree, every other piece uses adaptive tensor
 *     Gauss-Legendre (orders 8 and 16 compared, 2x2 subdivision otherwise),
 *   - the outer quadrature runs over the panel with the smaller diagonal
 *     (the integral is symmetric in the two panels),
 *   - pairs whose gap is at least the larger panel diagonal use a direct 4-D
 *     tensor Gauss-Legendre rule (orders 8 and 10 compared beyond three
 *     diagonals, 12 and 16 below), which avoids the cancellation of the
 *     corner formula when the inner panel is small against the distance.
 * Gauss-Legendre nodes are computed here by Newton's method on the Legendre
 * recurrence.
 *
 * Double layer (Sec. 4, the integrals Q_ij of the multi-dielectric system):
 *     d_ij = 1 / (4 pi) * int_{I_i} int_{I_j} (x_k - y_k) / |x - y|^3 dy dx,
 * k the normal axis of I_j, i.e. Q_ij for the normal +e_k of I_j.  Same
 * method: the inner integral is the exact solid-angle function of the
 * rectangle I_j seen from x (corner sum of atan(s t / (w rho))), the outer
 * one the same split tanh-sinh / adaptive Gauss-Legendre quadrature over
 * I_i (never swapped: the kernel is not symmetric), and separated pairs a
 * direct 4-D Gauss-Legendre rule.  Coplanar pairs give 0.
 *
 * Coordinates: a panel has a normal axis k in {0,1,2}, a plane coordinate c,
 * and extents [lo0,hi0] x [lo1,hi1] along the two remaining axes taken in
 * increasing axis order.  geo[5*i .. 5*i+4] = {c, lo0, hi0, lo1, hi1}.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846264338327950288

typedef struct {
    int k;          /* normal axis */
    int a[2];       /* in-plane axes, increasing */
    double c;       /* plane coordinate */
    double lo[3];   /* box extents in global axes (lo[k] == hi[k] == c) */
    double hi[3];
} orc_panel;

static void orc_make_panel(int axis, const double* g, orc_panel* P)
{
    P->k = axis;
    P->a[0] = (axis == 0) ? 1 : 0;
    P->a[1] = (axis == 2) ? 1 : 2;
    P->c = g[0];
    P->lo[axis] = g[0];
    P->hi[axis] = g[0];
    P->lo[P->a[0]] = g[1];
    P->hi[P->a[0]] = g[2];
    P->lo[P->a[1]] = g[3];
    P->hi[P->a[1]] = g[4];
}

static double orc_area(const orc_panel* P)
{
    return (P->hi[P->a[0]] - P->lo[P->a[0]]) * (P->hi[P->a[1]] - P->lo[P->a[1]]);
}

static double orc_diag(const orc_panel* P)
{
    double d0 = P->hi[P->a[0]] - P->lo[P->a[0]];
    double d1 = P->hi[P->a[1]] - P->lo[P->a[1]];
    return sqrt(d0 * d0 + d1 * d1);
}

/* Euclidean distance between two axis-aligned (flat) boxes. */
static double orc_gap(const orc_panel* A, const orc_panel* B)
{
    double s = 0.0;
    for (int d = 0; d < 3; ++d) {
        double g = 0.0;
        if (A->hi[d] < B->lo[d]) g = B->lo[d] - A->hi[d];
        else if (B->hi[d] < A->lo[d]) g = A->lo[d] - B->hi[d];
        s += g * g;
    }
    return sqrt(s);
}

/* ------------------------------------------------------------------ */
/* Inner integral: potential of a unit-density rectangle at a point.   */
/* ------------------------------------------------------------------ */

/* coef * ln(t + sqrt(t^2 + r2)), with the 0 * ln 0 limit taken as 0 and the
 * t < 0 branch written without cancellation. */
static double orc_xlog(double coef, double t, double r2, double rho)
{
    if (coef == 0.0) return 0.0;
    if (t >= 0.0) return coef * log(t + rho);
    return coef * log(r2 / (rho - t));
}

/* K(s,t,w) = s ln(t+rho) + t ln(s+rho) - w atan(s t / (w rho)):
 * d^2 K / ds dt = 1/sqrt(s^2+t^2+w^2). */
static double orc_K(double s, double t, double w)
{
    double rho = sqrt(s * s + t * t + w * w);
    double v = orc_xlog(s, t, s * s + w * w, rho) + orc_xlog(t, s, t * t + w * w, rho);
    if (w != 0.0 && s != 0.0 && t != 0.0) v -= w * atan(s * t / (w * rho));
    return v;
}

/* int_P 1/|x - y| dy */
static double orc_point_potential(const orc_panel* P, const double x[3])
{
    int p = P->a[0], q = P->a[1];
    double w = x[P->k] - P->c;
    double s0 = P->lo[p] - x[p], s1 = P->hi[p] - x[p];
    double t0 = P->lo[q] - x[q], t1 = P->hi[q] - x[q];
    return orc_K(s1, t1, w) - orc_K(s0, t1, w) - orc_K(s1, t0, w) + orc_K(s0, t0, w);
}

/* atan(s t / (w rho)): d^2 / ds dt = w / rho^3 (w != 0). */
static double orc_L(double s, double t, double w)
{
    if (s == 0.0 || t == 0.0) return 0.0;
    double rho = sqrt(s * s + t * t + w * w);
    return atan(s * t / (w * rho));
}

/* int_P (x_k - y_k) / |x - y|^3 dy, k the normal axis of P: the solid angle
 * that P subtends at x, signed by the side of P's plane x lies on; 0 in the
 * plane. */
static double orc_point_dlayer(const orc_panel* P, const double x[3])
{
    int p = P->a[0], q = P->a[1];
    double w = x[P->k] - P->c;
    if (w == 0.0) return 0.0;
    double s0 = P->lo[p] - x[p], s1 = P->hi[p] - x[p];
    double t0 = P->lo[q] - x[q], t1 = P->hi[q] - x[q];
    return orc_L(s1, t1, w) - orc_L(s0, t1, w) - orc_L(s1, t0, w) + orc_L(s0, t0, w);
}

/* ------------------------------------------------------------------ */
/* Gauss-Legendre nodes on [-1,1] by Newton iteration on P_n.          */
/* ------------------------------------------------------------------ */

#define ORC_GL_MAX 24
static double orc_glx[ORC_GL_MAX + 1][ORC_GL_MAX];
static double orc_glw[ORC_GL_MAX + 1][ORC_GL_MAX];
static int orc_gl_ready[ORC_GL_MAX + 1];

static void orc_gl_compute(int n, double* x, double* w)
{
    for (int i = 0; i < n; ++i) {
        /* Chebyshev-like initial guess for the i-th root (descending). */
        double z = cos(ORC_PI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = pk;
            }
            /* p1 = P_n(z), p0 = P_{n-1}(z) */
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-17) break;
        }
        {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = pk;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
        }
        x[i] = -z; /* ascending */
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

static void orc_gl_init(void)
{
    for (int n = 1; n <= ORC_GL_MAX; ++n) {
        if (orc_gl_ready[n]) continue;
        if (n == 1) {
            orc_glx[1][0] = 0.0;
            orc_glw[1][0] = 2.0;
        } else {
            orc_gl_compute(n, orc_glx[n], orc_glw[n]);
        }
        orc_gl_ready[n] = 1;
    }
}

int orc_gl_nodes(int n, double* x, double* w)
{
    if (n < 1 || n > ORC_GL_MAX) return -1;
    orc_gl_init();
    memcpy(x, orc_glx[n], sizeof(double) * n);
    memcpy(w, orc_glw[n], sizeof(double) * n);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Outer quadratures over a sub-rectangle of I_i.                      */
/* ------------------------------------------------------------------ */

typedef struct {
    const orc_panel* Pi;   /* outer panel (gives the plane) */
    const orc_panel* Pj;   /* inner panel */
    int kind;              /* 0: single layer 1/r, 1: double layer */
    double floor;          /* absolute size below which differences count as converged */
} orc_outer;

static double orc_outer_f(const orc_outer* O, double u0, double u1)
{
    double x[3];
    x[O->Pi->k] = O->Pi->c;
    x[O->Pi->a[0]] = u0;
    x[O->Pi->a[1]] = u1;
    return O->kind ? orc_point_dlayer(O->Pj, x) : orc_point_potential(O->Pj, x);
}

static double orc_outer_gl(const orc_outer* O, const double lo[2], const double hi[2], int n)
{
    double m0 = 0.5 * (lo[0] + hi[0]), h0 = 0.5 * (hi[0] - lo[0]);
    double m1 = 0.5 * (lo[1] + hi[1]), h1 = 0.5 * (hi[1] - lo[1]);
    double s = 0.0;
    for (int a = 0; a < n; ++a) {
        double sa = 0.0;
        for (int b = 0; b < n; ++b)
            sa += orc_glw[n][b] * orc_outer_f(O, m0 + h0 * orc_glx[n][a], m1 + h1 * orc_glx[n][b]);
        s += orc_glw[n][a] * sa;
    }
    return s * h0 * h1;
}

/* Adaptive tensor GL on a piece that does not touch the inner panel. */
static double orc_outer_adaptive(const orc_outer* O, const double lo[2], const double hi[2],
                                 int depth, int* nfail)
{
    double i8 = orc_outer_gl(O, lo, hi, 8);
    double i16 = orc_outer_gl(O, lo, hi, 16);
    double diff = fabs(i16 - i8);
    double mag = fmax(fabs(i16), O->floor);
    if (diff <= 1e-14 * mag) return i16;
    /* below 1e-12 the two orders differ by the rounding of the corner sums,
     * not by truncation; subdividing further cannot improve on that */
    if (depth >= 4 && diff <= 1e-12 * mag) return i16;
    if (depth >= 7) {
        ++*nfail;
        return i16;
    }
    double mid0 = 0.5 * (lo[0] + hi[0]), mid1 = 0.5 * (lo[1] + hi[1]);
    double s = 0.0;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            double l2[2] = {a ? mid0 : lo[0], b ? mid1 : lo[1]};
            double h2[2] = {a ? hi[0] : mid0, b ? hi[1] : mid1};
            s += orc_outer_adaptive(O, l2, h2, depth + 1, nfail);
        }
    return s;
}

/* tanh-sinh node/weight on [a,b] at parameter t; the node is formed from the
 * nearer endpoint so that it never rounds onto the far one. */
static void orc_ts_node(double a, double b, double t, double* x, double* w)
{
    const double hp = 0.5 * ORC_PI;
    double s = hp * sinh(t);
    double cs = cosh(s);
    double delta = 1.0 / (1.0 + exp(2.0 * fabs(s))); /* distance to the near end, in units of (b-a) */
    if (t < 0.0) *x = a + (b - a) * delta;
    else if (t > 0.0) *x = b - (b - a) * delta;
    else *x = 0.5 * (a + b);
    *w = 0.5 * (b - a) * hp * cosh(t) / (cs * cs);
}

#define ORC_TS_TMAX 3.5
#define ORC_TS_LMAX 8

/* 2-D tanh-sinh on a piece that touches the inner panel.  Level L uses the
 * step 2^-L in t; successive levels reuse the points already summed. */
static double orc_outer_ts(const orc_outer* O, const double lo[2], const double hi[2], int* nfail)
{
    double total = 0.0, prev = 0.0, est = 0.0;
    for (int L = 2; L <= ORC_TS_LMAX; ++L) {
        double h = 1.0 / (double)(1 << L);
        int kmax = (int)(ORC_TS_TMAX / h);
        for (int ia = -kmax; ia <= kmax; ++ia) {
            double xa, wa;
            orc_ts_node(lo[0], hi[0], ia * h, &xa, &wa);
            if (wa == 0.0) continue;
            double row = 0.0;
            for (int ib = -kmax; ib <= kmax; ++ib) {
                /* points of this level not present in the previous one */
                if (L > 2 && ((ia & 1) == 0) && ((ib & 1) == 0)) continue;
                double xb, wb;
                orc_ts_node(lo[1], hi[1], ib * h, &xb, &wb);
                if (wb == 0.0) continue;
                row += wb * orc_outer_f(O, xa, xb);
            }
            total += wa * row;
        }
        /* the tanh-sinh weights do not depend on h, so the running sum over
         * every point of this level's grid times h^2 is this level's estimate */
        est = total * h * h;
        if (L > 2 && fabs(est - prev) <= 1e-14 * fmax(fabs(est), O->floor)) return est;
        prev = est;
    }
    ++*nfail;
    return est;
}

/* Breakpoints of the inner potential along global axis d, inside (lo,hi). */
static int orc_breaks(const orc_panel* Pj, int d, double lo, double hi, double* out)
{
    double cand[2];
    int nc = 0;
    if (d == Pj->k) {
        cand[nc++] = Pj->c;
    } else {
        cand[nc++] = Pj->lo[d];
        cand[nc++] = Pj->hi[d];
    }
    int n = 0;
    out[n++] = lo;
    for (int i = 0; i < nc; ++i)
        if (cand[i] > lo && cand[i] < hi) {
            int dup = 0;
            for (int j = 0; j < n; ++j)
                if (out[j] == cand[i]) dup = 1;
            if (!dup) out[n++] = cand[i];
        }
    out[n++] = hi;
    /* sort (at most 4 entries) */
    for (int i = 1; i < n; ++i)
        for (int j = i; j > 0 && out[j - 1] > out[j]; --j) {
            double t = out[j];
            out[j] = out[j - 1];
            out[j - 1] = t;
        }
    return n;
}

/* Split-outer method: int_{Pi} [int_{Pj} kernel dy] dx */
static double orc_pair_split_k(const orc_panel* Pi, const orc_panel* Pj, int kind, double floor, int* nfail)
{
    orc_outer O = {Pi, Pj, kind, floor};
    double b0[4], b1[4];
    int p = Pi->a[0], q = Pi->a[1];
    int n0 = orc_breaks(Pj, p, Pi->lo[p], Pi->hi[p], b0);
    int n1 = orc_breaks(Pj, q, Pi->lo[q], Pi->hi[q], b1);
    double s = 0.0;
    for (int a = 0; a + 1 < n0; ++a)
        for (int b = 0; b + 1 < n1; ++b) {
            double lo[2] = {b0[a], b1[b]}, hi[2] = {b0[a + 1], b1[b + 1]};
            /* gap between this piece and Pj */
            orc_panel piece = *Pi;
            piece.lo[p] = lo[0];
            piece.hi[p] = hi[0];
            piece.lo[q] = lo[1];
            piece.hi[q] = hi[1];
            double g = orc_gap(&piece, Pj);
            if (g == 0.0) s += orc_outer_ts(&O, lo, hi, nfail);
            else s += orc_outer_adaptive(&O, lo, hi, 0, nfail);
        }
    return s;
}

static double orc_pair_split(const orc_panel* Pi, const orc_panel* Pj, int* nfail)
{
    return orc_pair_split_k(Pi, Pj, 0, 0.0, nfail);
}

/* Direct 4-D tensor GL of 1/|x-y| (kind 0) or (x_k - y_k)/|x-y|^3, k the
 * normal axis of Pj (kind 1), on two well-separated panels. */
static double orc_pair_gl4_k(const orc_panel* Pi, const orc_panel* Pj, int n, int kind)
{
    int pi0 = Pi->a[0], pi1 = Pi->a[1], pj0 = Pj->a[0], pj1 = Pj->a[1];
    double mi0 = 0.5 * (Pi->lo[pi0] + Pi->hi[pi0]), hi0 = 0.5 * (Pi->hi[pi0] - Pi->lo[pi0]);
    double mi1 = 0.5 * (Pi->lo[pi1] + Pi->hi[pi1]), hi1 = 0.5 * (Pi->hi[pi1] - Pi->lo[pi1]);
    double mj0 = 0.5 * (Pj->lo[pj0] + Pj->hi[pj0]), hj0 = 0.5 * (Pj->hi[pj0] - Pj->lo[pj0]);
    double mj1 = 0.5 * (Pj->lo[pj1] + Pj->hi[pj1]), hj1 = 0.5 * (Pj->hi[pj1] - Pj->lo[pj1]);
    double s = 0.0;
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b) {
            double x[3];
            x[Pi->k] = Pi->c;
            x[pi0] = mi0 + hi0 * orc_glx[n][a];
            x[pi1] = mi1 + hi1 * orc_glx[n][b];
            double wx = orc_glw[n][a] * orc_glw[n][b];
            double sy = 0.0;
            for (int c = 0; c < n; ++c)
                for (int d = 0; d < n; ++d) {
                    double y[3];
                    y[Pj->k] = Pj->c;
                    y[pj0] = mj0 + hj0 * orc_glx[n][c];
                    y[pj1] = mj1 + hj1 * orc_glx[n][d];
                    double dx = x[0] - y[0], dy = x[1] - y[1], dz = x[2] - y[2];
                    double r = sqrt(dx * dx + dy * dy + dz * dz);
                    double f = kind ? (x[Pj->k] - y[Pj->k]) / (r * r * r) : 1.0 / r;
                    sy += orc_glw[n][c] * orc_glw[n][d] * f;
                }
            s += wx * sy;
        }
    return s * hi0 * hi1 * hj0 * hj1;
}

static double orc_pair_gl4(const orc_panel* Pi, const orc_panel* Pj, int n)
{
    return orc_pair_gl4_k(Pi, Pj, n, 0);
}

/* int_{Pi} int_{Pj} (x_k - y_k)/|x-y|^3 dy dx, k = Pj->k (no 1/(4 pi)).
 * Convergence tests are relative to the larger of the value and
 * |Pi||Pj| / (gap + dmax)^2, the size of the integral of 1/|x-y|^2: a pair
 * whose contributions cancel (perpendicular panels placed symmetrically)
 * converges in absolute terms. */
static double orc_pair_dl(const orc_panel* Pi, const orc_panel* Pj, int* nfail)
{
    if (Pi->k == Pj->k && Pi->c == Pj->c) return 0.0;
    double g = orc_gap(Pi, Pj);
    double dmax = fmax(orc_diag(Pi), orc_diag(Pj));
    double floor = orc_area(Pi) * orc_area(Pj) / ((g + dmax) * (g + dmax));
    if (g >= 3.0 * dmax) {
        double i8 = orc_pair_gl4_k(Pi, Pj, 8, 1);
        double i10 = orc_pair_gl4_k(Pi, Pj, 10, 1);
        if (fabs(i10 - i8) <= 5e-14 * fmax(fabs(i10), floor)) return i10;
    } else if (g >= dmax) {
        double i12 = orc_pair_gl4_k(Pi, Pj, 12, 1);
        double i16 = orc_pair_gl4_k(Pi, Pj, 16, 1);
        if (fabs(i16 - i12) <= 5e-14 * fmax(fabs(i16), floor)) return i16;
    }
    return orc_pair_split_k(Pi, Pj, 1, floor, nfail);
}

/* int_{Pi} int_{Pj} 1/|x-y| dy dx  (no 1/(4 pi), no area normalisation).
 * *nfail counts quadratures that stopped before their convergence test. */
static double orc_pair(const orc_panel* Pi, const orc_panel* Pj, int* nfail)
{
    double g = orc_gap(Pi, Pj);
    double dmax = fmax(orc_diag(Pi), orc_diag(Pj));
    /* Separated pairs: direct 4-D rule, two orders compared.  The agreement
     * test allows for the rounding of a sum of up to 16^4 terms. */
    if (g >= 3.0 * dmax) {
        double i8 = orc_pair_gl4(Pi, Pj, 8);
        double i10 = orc_pair_gl4(Pi, Pj, 10);
        if (fabs(i10 - i8) <= 5e-14 * fabs(i10)) return i10;
    } else if (g >= dmax) {
        double i12 = orc_pair_gl4(Pi, Pj, 12);
        double i16 = orc_pair_gl4(Pi, Pj, 16);
        if (fabs(i16 - i12) <= 5e-14 * fabs(i16)) return i16;
    }
    /* The double integral is symmetric in the two panels (Eq. "matrix"; A is
     * symmetric, Sec. 3.2), so the outer quadrature may run over either.  It
     * runs over the one with the smaller diagonal: the exact potential of a
     * panel that is small against its distance cancels between its corners
     * (about eps (R/h)^2), while a large panel's potential at the points of a
     * small one does not, and a small outer domain needs few points. */
    if (orc_diag(Pj) < orc_diag(Pi)) return orc_pair_split(Pj, Pi, nfail);
    return orc_pair_split(Pi, Pj, nfail);
}

/* ------------------------------------------------------------------ */
/* Exported entry points (ctypes).                                     */
/* ------------------------------------------------------------------ */

int orc_version(void) { return 1; }

double orc_rect_potential(int axis, const double* geo, const double* x)
{
    orc_panel P;
    orc_make_panel(axis, geo, &P);
    return orc_point_potential(&P, x);
}

/* Raw double integral of 1/r for one pair; method: 0 auto, 1 force split. */
double orc_pair_integral(int axis_i, const double* geo_i, int axis_j, const double* geo_j,
                         int method, int* nfail)
{
    orc_gl_init();
    orc_panel Pi, Pj;
    orc_make_panel(axis_i, geo_i, &Pi);
    orc_make_panel(axis_j, geo_j, &Pj);
    int nf = 0;
    double r = (method == 1) ? orc_pair_split(&Pi, &Pj, &nf) : orc_pair(&Pi, &Pj, &nf);
    if (nfail) *nfail = nf;
    return r;
}

double orc_rect_dlayer(int axis, const double* geo, const double* x)
{
    orc_panel P;
    orc_make_panel(axis, geo, &P);
    return orc_point_dlayer(&P, x);
}

/* Double-layer entries d_ij = (1/(4 pi)) int int (x_k - y_k)/r^3, k the normal
 * axis of panel j, for m sampled pairs (Sec. 4, Q_ij for the normal +e_k). */
int orc_dl_entries(int n, const int32_t* axis, const double* geo, int64_t m, const int32_t* I,
                   const int32_t* J, double* out, int nthreads)
{
    orc_gl_init();
    int nf_total = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : nf_total)
    for (int64_t t = 0; t < m; ++t) {
        int i = I[t], j = J[t];
        if (i < 0 || j < 0 || i >= n || j >= n) {
            out[t] = NAN;
            continue;
        }
        orc_panel Pi, Pj;
        orc_make_panel(axis[i], geo + 5 * (size_t)i, &Pi);
        orc_make_panel(axis[j], geo + 5 * (size_t)j, &Pj);
        int nf = 0;
        double v = orc_pair_dl(&Pi, &Pj, &nf);
        nf_total += nf;
        out[t] = v / (4.0 * ORC_PI);
    }
    return nf_total;
}

/* Matrix entries a_ij = int int 1/r / (4 pi |I_i| |I_j|) for m sampled pairs. */
int orc_entries(int n, const int32_t* axis, const double* geo, int64_t m, const int32_t* I,
                const int32_t* J, double* out, int nthreads)
{
    orc_gl_init();
    int nf_total = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : nf_total)
    for (int64_t t = 0; t < m; ++t) {
        int i = I[t], j = J[t];
        if (i < 0 || j < 0 || i >= n || j >= n) {
            out[t] = NAN;
            continue;
        }
        orc_panel Pi, Pj;
        orc_make_panel(axis[i], geo + 5 * (size_t)i, &Pi);
        orc_make_panel(axis[j], geo + 5 * (size_t)j, &Pj);
        int nf = 0;
        double v = orc_pair(&Pi, &Pj, &nf);
        nf_total += nf;
        out[t] = v / (4.0 * ORC_PI * orc_area(&Pi) * orc_area(&Pj));
    }
    return nf_total;
}

/* Full symmetric matrix, row-major n x n; the lower triangle is computed and
 * mirrored.  Returns the number of quadratures that did not converge. */
int orc_assemble(int n, const int32_t* axis, const double* geo, double* A, int nthreads)
{
    orc_gl_init();
    int nf_total = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : nf_total)
    for (int i = 0; i < n; ++i) {
        orc_panel Pi;
        orc_make_panel(axis[i], geo + 5 * (size_t)i, &Pi);
        double ai = orc_area(&Pi);
        for (int j = 0; j <= i; ++j) {
            orc_panel Pj;
            orc_make_panel(axis[j], geo + 5 * (size_t)j, &Pj);
            int nf = 0;
            double v = orc_pair(&Pi, &Pj, &nf) / (4.0 * ORC_PI * ai * orc_area(&Pj));
            nf_total += nf;
            A[(size_t)i * n + j] = v;
            A[(size_t)j * n + i] = v;
        }
    }
    return nf_total;
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
