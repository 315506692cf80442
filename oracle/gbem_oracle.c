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
 * Flat triangles (general conductors): the same a_ij over triangles T_i, T_j,
 * with the exact potential of a uniformly charged triangle inside; outside,
 * for triangles that share a vertex (or are the same), a tanh-sinh rule in
 * both coordinates of the collapsed map, refined until two levels agree,
 * else an adaptive collapsed Gauss-Legendre rule (midpoint subdivision);
 * separated pairs by the collapsed rule on both triangles.
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
/* Flat triangles (general conductors).                                */
/* ------------------------------------------------------------------ */

/* Vertices a, b, c; unit normal along (b - a) x (c - a); area. */
typedef struct {
    double v[3][3];
    double n[3];
    double area;
    double diam;
} orc_tri;

static void orc_cross(const double* a, const double* b, double* c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

static double orc_dot(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static void orc_make_tri(const double* p, orc_tri* T)
{
    for (int k = 0; k < 3; ++k)
        for (int d = 0; d < 3; ++d) T->v[k][d] = p[3 * k + d];
    double e1[3], e2[3];
    for (int d = 0; d < 3; ++d) {
        e1[d] = T->v[1][d] - T->v[0][d];
        e2[d] = T->v[2][d] - T->v[0][d];
    }
    orc_cross(e1, e2, T->n);
    double len = sqrt(orc_dot(T->n, T->n));
    T->area = 0.5 * len;
    for (int d = 0; d < 3; ++d) T->n[d] /= len;
    T->diam = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = i + 1; j < 3; ++j) {
            double s = 0.0;
            for (int d = 0; d < 3; ++d) s += (T->v[i][d] - T->v[j][d]) * (T->v[i][d] - T->v[j][d]);
            T->diam = fmax(T->diam, sqrt(s));
        }
}

/* ln(R + l) with R = sqrt(l^2 + r0sq), without cancellation for l < 0. */
static double orc_lnp(double l, double r0sq, double R)
{
    if (l >= 0.0) return log(R + l);
    return log(r0sq / (R - l));
}

/* int_T 1/|x - y| dy: the potential of a uniformly charged flat triangle
 * (the edge-by-edge closed form: for each edge, with x projected to rho in
 * the plane at signed height h, the edge's direction l, its outward in-plane
 * normal u, P0 = (edge start - rho).u, and l+- the edge ends' coordinates
 * along l,  P0 ln((R+ + l+)/(R- + l-)) - |h| [atan(P0 l+/(R0^2 + |h| R+)) -
 * atan(P0 l-/(R0^2 + |h| R-))]). */
static double orc_tri_potential(const orc_tri* T, const double x[3])
{
    double h = 0.0, rho[3];
    for (int d = 0; d < 3; ++d) h += (x[d] - T->v[0][d]) * T->n[d];
    for (int d = 0; d < 3; ++d) rho[d] = x[d] - h * T->n[d];
    const double ah = fabs(h);
    double s = 0.0;
    for (int e = 0; e < 3; ++e) {
        const double* p = T->v[e];
        const double* q = T->v[(e + 1) % 3];
        double l[3], u[3], L = 0.0;
        for (int d = 0; d < 3; ++d) {
            l[d] = q[d] - p[d];
            L += l[d] * l[d];
        }
        L = sqrt(L);
        for (int d = 0; d < 3; ++d) l[d] /= L;
        orc_cross(l, T->n, u);
        double qp[3], pp[3];
        for (int d = 0; d < 3; ++d) {
            qp[d] = q[d] - rho[d];
            pp[d] = p[d] - rho[d];
        }
        const double lp = orc_dot(qp, l), lm = orc_dot(pp, l), P0 = orc_dot(pp, u);
        const double r0sq = P0 * P0 + h * h;
        const double Rp = sqrt(lp * lp + r0sq), Rm = sqrt(lm * lm + r0sq);
        if (P0 != 0.0) {
            s += P0 * (orc_lnp(lp, r0sq, Rp) - orc_lnp(lm, r0sq, Rm));
            if (ah != 0.0) s -= ah * (atan(P0 * lp / (r0sq + ah * Rp)) - atan(P0 * lm / (r0sq + ah * Rm)));
        }
    }
    return s;
}

/* Collapsed Gauss-Legendre rule of order n on triangle (a, b, c) applied to
 * the potential of Tj: y = a + xi ((b - a) + eta (c - b)), dy = 2 |T| xi dxi deta. */
static double orc_tri_outer_gl(const double a[3], const double b[3], const double c[3], const orc_tri* Tj, int n)
{
    double ab[3], bc[3], cr[3];
    for (int d = 0; d < 3; ++d) {
        ab[d] = b[d] - a[d];
        bc[d] = c[d] - b[d];
    }
    orc_cross(ab, bc, cr);
    const double j2 = sqrt(orc_dot(cr, cr));   /* 2 |T| */
    double s = 0.0;
    for (int i = 0; i < n; ++i) {
        const double xi = 0.5 * (orc_glx[n][i] + 1.0);
        double row = 0.0;
        for (int k = 0; k < n; ++k) {
            const double eta = 0.5 * (orc_glx[n][k] + 1.0);
            double y[3];
            for (int d = 0; d < 3; ++d) y[d] = a[d] + xi * (ab[d] + eta * bc[d]);
            row += orc_glw[n][k] * orc_tri_potential(Tj, y);
        }
        s += orc_glw[n][i] * xi * row;
    }
    return 0.25 * j2 * s;
}

/* Adaptive outer quadrature: orders 12 and 16 compared on the triangle,
 * else its four midpoint children. */
static double orc_tri_outer(const double a[3], const double b[3], const double c[3], const orc_tri* Tj,
                            double floor, int depth, int* nfail)
{
    const double i12 = orc_tri_outer_gl(a, b, c, Tj, 12);
    const double i16 = orc_tri_outer_gl(a, b, c, Tj, 16);
    const double diff = fabs(i16 - i12), mag = fmax(fabs(i16), floor);
    if (diff <= 1e-14 * mag || (depth >= 5 && diff <= 1e-12 * mag)) return i16;
    if (depth >= 9) {
        ++*nfail;
        return i16;
    }
    double ab[3], bc[3], ca[3];
    for (int d = 0; d < 3; ++d) {
        ab[d] = 0.5 * (a[d] + b[d]);
        bc[d] = 0.5 * (b[d] + c[d]);
        ca[d] = 0.5 * (c[d] + a[d]);
    }
    return orc_tri_outer(a, ab, ca, Tj, floor, depth + 1, nfail) + orc_tri_outer(ab, b, bc, Tj, floor, depth + 1, nfail) +
           orc_tri_outer(ca, bc, c, Tj, floor, depth + 1, nfail) + orc_tri_outer(ab, bc, ca, Tj, floor, depth + 1, nfail);
}

/* Tanh-sinh rule in both coordinates of the collapsed map of triangle
 * (a, b, c), for an outer integrand whose derivatives are singular on the
 * triangle's sides and corners (the potential of a triangle that shares a
 * vertex, a side or the whole triangle): every side lies on the boundary of
 * the unit square, where the double-exponential rule converges fast.  Level
 * L uses the step 2^-L; levels are refined until two agree. */
static double orc_tri_outer_ts(const double a[3], const double b[3], const double c[3], const orc_tri* Tj,
                               double floor, int* nfail)
{
    double ab[3], bc[3], cr[3];
    for (int d = 0; d < 3; ++d) {
        ab[d] = b[d] - a[d];
        bc[d] = c[d] - b[d];
    }
    orc_cross(ab, bc, cr);
    const double j2 = sqrt(orc_dot(cr, cr));
    double total = 0.0, prev = 0.0, est = 0.0;
    for (int L = 2; L <= ORC_TS_LMAX; ++L) {
        const double h = 1.0 / (double)(1 << L);
        const int kmax = (int)(ORC_TS_TMAX / h);
        for (int ia = -kmax; ia <= kmax; ++ia) {
            double xi, wx;
            orc_ts_node(0.0, 1.0, ia * h, &xi, &wx);
            if (wx == 0.0) continue;
            double row = 0.0;
            for (int ib = -kmax; ib <= kmax; ++ib) {
                if (L > 2 && ((ia & 1) == 0) && ((ib & 1) == 0)) continue;
                double eta, we;
                orc_ts_node(0.0, 1.0, ib * h, &eta, &we);
                if (we == 0.0) continue;
                double y[3];
                for (int d = 0; d < 3; ++d) y[d] = a[d] + xi * (ab[d] + eta * bc[d]);
                row += we * orc_tri_potential(Tj, y);
            }
            total += wx * xi * row;
        }
        est = total * h * h * j2;
        if (L > 2 && fabs(est - prev) <= 1e-14 * fmax(fabs(est), floor)) return est;
        prev = est;
    }
    ++*nfail;
    return est;
}

static int orc_tri_touch(const orc_tri* A, const orc_tri* B)
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            if (A->v[i][0] == B->v[j][0] && A->v[i][1] == B->v[j][1] && A->v[i][2] == B->v[j][2]) return 1;
    return 0;
}

/* int_Ti int_Tj 1/|x - y| (no 1/(4 pi)).  Separated pairs (centroid distance
 * at least three diameters) use the collapsed rule on both triangles, orders
 * 8 and 10 compared; otherwise the adaptive outer quadrature of Tj's exact
 * potential over the smaller triangle (the integral is symmetric). */
static double orc_tri_pair(const orc_tri* Ti, const orc_tri* Tj, int* nfail)
{
    double ci[3], cj[3], dist = 0.0;
    for (int d = 0; d < 3; ++d) {
        ci[d] = (Ti->v[0][d] + Ti->v[1][d] + Ti->v[2][d]) / 3.0;
        cj[d] = (Tj->v[0][d] + Tj->v[1][d] + Tj->v[2][d]) / 3.0;
        dist += (ci[d] - cj[d]) * (ci[d] - cj[d]);
    }
    dist = sqrt(dist);
    const double dmax = fmax(Ti->diam, Tj->diam);
    const orc_tri* O = Ti->area <= Tj->area ? Ti : Tj;
    const orc_tri* I = O == Ti ? Tj : Ti;
    if (dist >= 3.0 * dmax) {
        double r[2];
        for (int t = 0; t < 2; ++t) {
            const int n = t ? 10 : 8;
            double abi[3], bci[3], abj[3], bcj[3], cr[3];
            for (int d = 0; d < 3; ++d) {
                abi[d] = O->v[1][d] - O->v[0][d];
                bci[d] = O->v[2][d] - O->v[1][d];
                abj[d] = I->v[1][d] - I->v[0][d];
                bcj[d] = I->v[2][d] - I->v[1][d];
            }
            orc_cross(abi, bci, cr);
            const double ji = sqrt(orc_dot(cr, cr));
            orc_cross(abj, bcj, cr);
            const double jj = sqrt(orc_dot(cr, cr));
            double s = 0.0;
            for (int a = 0; a < n; ++a)
                for (int b = 0; b < n; ++b) {
                    const double xa = 0.5 * (orc_glx[n][a] + 1.0), eb = 0.5 * (orc_glx[n][b] + 1.0);
                    double x[3];
                    for (int d = 0; d < 3; ++d) x[d] = O->v[0][d] + xa * (abi[d] + eb * bci[d]);
                    double sy = 0.0;
                    for (int c = 0; c < n; ++c)
                        for (int e = 0; e < n; ++e) {
                            const double xc = 0.5 * (orc_glx[n][c] + 1.0), ee = 0.5 * (orc_glx[n][e] + 1.0);
                            double y[3], q = 0.0;
                            for (int d = 0; d < 3; ++d) {
                                y[d] = I->v[0][d] + xc * (abj[d] + ee * bcj[d]) - x[d];
                                q += y[d] * y[d];
                            }
                            sy += orc_glw[n][c] * orc_glw[n][e] * xc / sqrt(q);
                        }
                    s += orc_glw[n][a] * orc_glw[n][b] * xa * sy;
                }
            r[t] = s * ji * jj / 16.0;
        }
        if (fabs(r[1] - r[0]) <= 5e-14 * fabs(r[1])) return r[1];
    }
    const double floor = O->area * I->area / (dist + dmax);
    if (orc_tri_touch(O, I)) return orc_tri_outer_ts(O->v[0], O->v[1], O->v[2], I, floor, nfail);
    return orc_tri_outer(O->v[0], O->v[1], O->v[2], I, floor, 0, nfail);
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

double orc_tri_potential_at(const double* tri, const double* x)
{
    orc_tri T;
    orc_make_tri(tri, &T);
    return orc_tri_potential(&T, x);
}

/* Galerkin entries of flat triangles, a_ij = int int 1/r / (4 pi |T_i| |T_j|),
 * for m sampled pairs (tri: 9 doubles per triangle, its three vertices). */
int orc_tri_entries(int n, const double* tri, int64_t m, const int32_t* I, const int32_t* J, double* out,
                    int nthreads)
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
        orc_tri Ti, Tj;
        orc_make_tri(tri + 9 * (size_t)i, &Ti);
        orc_make_tri(tri + 9 * (size_t)j, &Tj);
        int nf = 0;
        double v = orc_tri_pair(&Ti, &Tj, &nf);
        nf_total += nf;
        out[t] = v / (4.0 * ORC_PI * Ti.area * Tj.area);
    }
    return nf_total;
}
