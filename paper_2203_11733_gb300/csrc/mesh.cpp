// Boundary partition of cuboid conductors into axis-aligned rectangular
// panels (Wu & Li, Sec. 3.1: dOmega = U_j I_j; Sec. 3.3: every conductor is
// built from cuboids, so every panel is an axis-aligned rectangle).
//
// Each box edge is divided on its own; a face is cut on the tensor grid of
// its two edge divisions.  Panels are then ordered by conductor and, inside a
// conductor, by the Morton code of the panel centre, so that a tile of
// consecutive panels is spatially compact (near pairs gather close to the
// diagonal of the matrix, and far tiles see similar distances).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <numeric>
#include <string>
#include <vector>

#include "gbem_internal.h"

void mesh_divide(double lo, double hi, const gbem_mesh_params* p, std::vector<double>& nodes)
{
    nodes.clear();
    const double L = hi - lo;
    const double h = p->h;
    auto uniform = [&]() {
        int n = std::max(1, (int)std::ceil(L / h - 1e-9));
        for (int k = 0; k < n; ++k) nodes.push_back(lo + (L * k) / n);
        nodes.push_back(hi);
    };
    if (p->ratio <= 1.0 || p->h_min <= 0.0 || p->h_min >= h) {
        uniform();
        return;
    }
    std::vector<double> sizes;
    for (double s = p->h_min; s < h; s = s * p->ratio) sizes.push_back(s);
    int m = (int)sizes.size();
    while (m > 0) {
        double tot = 0.0;
        for (int k = 0; k < m; ++k) tot += sizes[k];
        if (2.0 * tot <= L) break;
        --m;
    }
    if (m == 0) {
        uniform();
        return;
    }
    std::vector<double> left{lo}, right{hi};
    double acc = lo;
    for (int k = 0; k < m; ++k) {
        acc = acc + sizes[k];
        left.push_back(acc);
    }
    acc = hi;
    for (int k = 0; k < m; ++k) {
        acc = acc - sizes[k];
        right.push_back(acc);
    }
    std::reverse(right.begin(), right.end());
    const double xl = left.back(), xr = right.front();
    const double M = xr - xl;
    nodes.assign(left.begin(), left.end() - 1);
    if (M > 1e-12 * L) {
        int nmid = std::max(1, (int)std::ceil(M / h - 1e-9));
        for (int k = 0; k < nmid; ++k) nodes.push_back(xl + (M * k) / nmid);
    }
    nodes.insert(nodes.end(), right.begin(), right.end());
}

gbem_status mesh_build_boxes(const gbem_box* boxes, int nbox, const gbem_mesh_params* p,
                             std::vector<int8_t>& axis, std::vector<double>& geo,
                             std::vector<int32_t>& cond_raw, std::string& err)
{
    if (nbox <= 0 || !boxes || !p) {
        err = "gbem_mesh: no boxes";
        return GBEM_ERR_ARG;
    }
    if (!(p->h > 0.0) || !std::isfinite(p->h)) {
        err = "gbem_mesh: h must be positive";
        return GBEM_ERR_ARG;
    }
    for (int b = 0; b < nbox; ++b)
        for (int d = 0; d < 3; ++d)
            if (!(boxes[b].hi[d] > boxes[b].lo[d]) || !std::isfinite(boxes[b].lo[d]) ||
                !std::isfinite(boxes[b].hi[d])) {
                err = "gbem_mesh: box " + std::to_string(b) + " is empty or not finite";
                return GBEM_ERR_MESH;
            }
    // boxes may neither overlap nor touch: touching faces would be interior
    for (int a = 0; a < nbox; ++a)
        for (int b = a + 1; b < nbox; ++b) {
            bool sep = false;
            for (int d = 0; d < 3; ++d)
                if (boxes[a].hi[d] < boxes[b].lo[d] || boxes[b].hi[d] < boxes[a].lo[d]) sep = true;
            if (!sep) {
                err = "gbem_mesh: boxes " + std::to_string(a) + " and " + std::to_string(b) +
                      " overlap or touch";
                return GBEM_ERR_MESH;
            }
        }
    // estimate size first so that a runaway h is refused before allocating
    double est = 0.0;
    std::vector<double> n0, n1;
    for (int b = 0; b < nbox; ++b)
        for (int k = 0; k < 3; ++k) {
            int pa = (k == 0) ? 1 : 0, qa = (k == 2) ? 1 : 2;
            mesh_divide(boxes[b].lo[pa], boxes[b].hi[pa], p, n0);
            mesh_divide(boxes[b].lo[qa], boxes[b].hi[qa], p, n1);
            est += 2.0 * (double)(n0.size() - 1) * (double)(n1.size() - 1);
        }
    if (est > 2.0e6) {
        err = "gbem_mesh: more than 2e6 panels requested";
        return GBEM_ERR_ARG;
    }
    axis.clear();
    geo.clear();
    cond_raw.clear();
    axis.reserve((size_t)est);
    geo.reserve(5 * (size_t)est);
    cond_raw.reserve((size_t)est);
    for (int b = 0; b < nbox; ++b) {
        const gbem_box& B = boxes[b];
        for (int k = 0; k < 3; ++k) {
            int pa = (k == 0) ? 1 : 0, qa = (k == 2) ? 1 : 2;
            mesh_divide(B.lo[pa], B.hi[pa], p, n0);
            mesh_divide(B.lo[qa], B.hi[qa], p, n1);
            for (int side = 0; side < 2; ++side) {
                double plane = side ? B.hi[k] : B.lo[k];
                for (size_t a = 0; a + 1 < n0.size(); ++a)
                    for (size_t c = 0; c + 1 < n1.size(); ++c) {
                        axis.push_back((int8_t)k);
                        geo.push_back(plane);
                        geo.push_back(n0[a]);
                        geo.push_back(n0[a + 1]);
                        geo.push_back(n1[c]);
                        geo.push_back(n1[c + 1]);
                        cond_raw.push_back(B.conductor);
                    }
            }
        }
    }
    return GBEM_OK;
}

static uint64_t spread3(uint64_t x)
{
    x &= 0x1fffff;
    x = (x | x << 32) & 0x1f00000000ffffULL;
    x = (x | x << 16) & 0x1f0000ff0000ffULL;
    x = (x | x << 8) & 0x100f00f00f00f00fULL;
    x = (x | x << 4) & 0x10c30c30c30c30c3ULL;
    x = (x | x << 2) & 0x1249249249249249ULL;
    return x;
}

// Reorder panels by conductor index, then by Morton code of the centre.
void mesh_order(std::vector<int8_t>& axis, std::vector<double>& geo, std::vector<int32_t>& cond)
{
    const size_t n = axis.size();
    if (n == 0) return;
    std::vector<double> ctr(3 * n);
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (size_t i = 0; i < n; ++i) {
        int k = axis[i], pa = (k == 0) ? 1 : 0, qa = (k == 2) ? 1 : 2;
        const double* g = &geo[5 * i];
        ctr[3 * i + k] = g[0];
        ctr[3 * i + pa] = 0.5 * (g[1] + g[2]);
        ctr[3 * i + qa] = 0.5 * (g[3] + g[4]);
        for (int d = 0; d < 3; ++d) {
            lo[d] = std::min(lo[d], ctr[3 * i + d]);
            hi[d] = std::max(hi[d], ctr[3 * i + d]);
        }
    }
    double ext = std::max({hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2], 1e-300});
    std::vector<uint64_t> code(n);
    for (size_t i = 0; i < n; ++i) {
        uint64_t m = 0;
        for (int d = 0; d < 3; ++d) {
            double t = (ctr[3 * i + d] - lo[d]) / ext;
            uint64_t q = (uint64_t)std::min(2097151.0, std::max(0.0, t * 2097151.0));
            m |= spread3(q) << d;
        }
        code[i] = m;
    }
    // sort flat records (conductor, code, original index): the index breaks
    // ties, so the order is that of a stable sort on (conductor, code)
    struct Key {
        int32_t cond;
        uint32_t idx;
        uint64_t code;
    };
    std::vector<Key> keys(n);
    for (size_t i = 0; i < n; ++i) keys[i] = Key{cond[i], (uint32_t)i, code[i]};
    std::sort(keys.begin(), keys.end(), [](const Key& a, const Key& b) {
        if (a.cond != b.cond) return a.cond < b.cond;
        if (a.code != b.code) return a.code < b.code;
        return a.idx < b.idx;
    });
    std::vector<int8_t> ax2(n);
    std::vector<double> g2(5 * n);
    std::vector<int32_t> c2(n);
    for (size_t t = 0; t < n; ++t) {
        const size_t j = keys[t].idx;
        ax2[t] = axis[j];
        c2[t] = cond[j];
        for (int e = 0; e < 5; ++e) g2[5 * t + e] = geo[5 * j + e];
    }
    axis.swap(ax2);
    geo.swap(g2);
    cond.swap(c2);
}

// ---- distance-graded partition (Sec. 3.3)
//
// Every face is split by bisection of its longer edge until each panel I_j
// satisfies the paper's bound for its distance d to the main net:
//     |I_j| <= p4                      if d < p5,
//     |I_j| <= p4 * p3 * (d / p5)^3    otherwise,
// with p4 = p1 for a face that looks toward the main net (the main net lies
// on the outward side of its plane; the main net's own faces and the inner
// faces of a grounded enclosure always do) and p4 = p1 * p2 for a face that
// looks away from it (shielded).  d is the distance between the panel and
// the nearest box of the main net; an optional h_max caps the panel edges.

namespace {

struct GFace {
    int k;         // normal axis
    double plane;  // plane coordinate
    double l0, h0, l1, h1;
    int32_t cond;
    bool toward;   // looks toward the main net
};

double rect_box_distance(int k, double c, double l0, double h0, double l1, double h1, const gbem_box& B)
{
    const int pa = (k == 0) ? 1 : 0, qa = (k == 2) ? 1 : 2;
    double lo[3], hi[3];
    lo[k] = hi[k] = c;
    lo[pa] = l0;
    hi[pa] = h0;
    lo[qa] = l1;
    hi[qa] = h1;
    double d2 = 0.0;
    for (int d = 0; d < 3; ++d) {
        const double g = std::max(0.0, std::max(B.lo[d] - hi[d], lo[d] - B.hi[d]));
        d2 += g * g;
    }
    return std::sqrt(d2);
}

}  // namespace

gbem_status mesh_build_graded(const gbem_box* boxes, int nbox, const gbem_partition_params* p,
                              std::vector<int8_t>& axis, std::vector<double>& geo, std::vector<int32_t>& cond_raw,
                              std::string& err)
{
    if (nbox <= 0 || !boxes || !p) {
        err = "gbem_mesh_graded: no boxes";
        return GBEM_ERR_ARG;
    }
    if (!(p->p1 > 0.0) || !(p->p2 >= 1.0) || !(p->p3 > 0.0) || !(p->p5 > 0.0) || !(p->h_max >= 0.0) ||
        !std::isfinite(p->p1) || !std::isfinite(p->p2) || !std::isfinite(p->p3) || !std::isfinite(p->p5)) {
        err = "gbem_mesh_graded: need p1 > 0, p2 >= 1, p3 > 0, p5 > 0, h_max >= 0";
        return GBEM_ERR_ARG;
    }
    // the same box checks as the uniform mesher (empty, overlapping, touching)
    {
        gbem_mesh_params probe{1e300, 1.0, 0.0};
        std::vector<int8_t> a;
        std::vector<double> g;
        std::vector<int32_t> c;
        gbem_status st = mesh_build_boxes(boxes, nbox, &probe, a, g, c, err);
        if (st != GBEM_OK) return st;
    }
    std::vector<int> mains;
    double mlo[3] = {1e300, 1e300, 1e300}, mhi[3] = {-1e300, -1e300, -1e300};
    for (int b = 0; b < nbox; ++b)
        if (boxes[b].conductor == p->main_conductor) {
            mains.push_back(b);
            for (int d = 0; d < 3; ++d) {
                mlo[d] = std::min(mlo[d], boxes[b].lo[d]);
                mhi[d] = std::max(mhi[d], boxes[b].hi[d]);
            }
        }
    if (mains.empty()) {
        err = "gbem_mesh_graded: no box of the main conductor";
        return GBEM_ERR_ARG;
    }
    std::vector<GFace> faces;
    for (int b = 0; b < nbox; ++b) {
        const gbem_box& B = boxes[b];
        const bool is_main = B.conductor == p->main_conductor;
        for (int k = 0; k < 3; ++k) {
            const int pa = (k == 0) ? 1 : 0, qa = (k == 2) ? 1 : 2;
            for (int side = 0; side < 2; ++side) {
                const double c = side ? B.hi[k] : B.lo[k];
                // outward normal +e_k (side 1) or -e_k (side 0)
                const bool toward = is_main || (side ? mhi[k] > c : mlo[k] < c);
                faces.push_back(GFace{k, c, B.lo[pa], B.hi[pa], B.lo[qa], B.hi[qa], B.conductor, toward});
            }
        }
    }
    if (p->has_enclosure) {
        const double* lo = p->encl_lo;
        const double* hi = p->encl_hi;
        for (int d = 0; d < 3; ++d)
            if (!(hi[d] > lo[d])) {
                err = "gbem_mesh_graded: empty enclosure";
                return GBEM_ERR_MESH;
            }
        for (int b = 0; b < nbox; ++b)
            for (int d = 0; d < 3; ++d)
                if (!(boxes[b].lo[d] > lo[d] && boxes[b].hi[d] < hi[d])) {
                    err = "gbem_mesh_graded: box " + std::to_string(b) + " is not strictly inside the enclosure";
                    return GBEM_ERR_MESH;
                }
        for (int k = 0; k < 3; ++k) {
            const int pa = (k == 0) ? 1 : 0, qa = (k == 2) ? 1 : 2;
            for (int side = 0; side < 2; ++side)
                faces.push_back(GFace{k, side ? hi[k] : lo[k], lo[pa], hi[pa], lo[qa], hi[qa], p->encl_conductor, true});
        }
    }
    axis.clear();
    geo.clear();
    cond_raw.clear();
    struct Piece {
        double l0, h0, l1, h1;
    };
    std::vector<Piece> stack;
    for (const GFace& F : faces) {
        const double p4 = F.toward ? p->p1 : p->p1 * p->p2;
        stack.clear();
        stack.push_back(Piece{F.l0, F.h0, F.l1, F.h1});
        while (!stack.empty()) {
            const Piece r = stack.back();
            stack.pop_back();
            double d = 1e300;
            for (int b : mains) d = std::min(d, rect_box_distance(F.k, F.plane, r.l0, r.h0, r.l1, r.h1, boxes[b]));
            double limit = p4;
            if (d >= p->p5) {
                const double t = d / p->p5;
                limit = p4 * p->p3 * (t * t * t);
            }
            const double e0 = r.h0 - r.l0, e1 = r.h1 - r.l1;
            const bool too_big = e0 * e1 > limit || (p->h_max > 0.0 && std::max(e0, e1) > p->h_max);
            if (!too_big) {
                axis.push_back((int8_t)F.k);
                geo.push_back(F.plane);
                geo.push_back(r.l0);
                geo.push_back(r.h0);
                geo.push_back(r.l1);
                geo.push_back(r.h1);
                cond_raw.push_back(F.cond);
                if (axis.size() > 2000000) {
                    err = "gbem_mesh_graded: more than 2e6 panels requested";
                    return GBEM_ERR_ARG;
                }
                continue;
            }
            // bisect the longer edge (the first on a tie); the second half is
            // pushed first so that the first half is refined first
            if (e0 >= e1) {
                const double m = 0.5 * (r.l0 + r.h0);
                stack.push_back(Piece{m, r.h0, r.l1, r.h1});
                stack.push_back(Piece{r.l0, m, r.l1, r.h1});
            } else {
                const double m = 0.5 * (r.l1 + r.h1);
                stack.push_back(Piece{r.l0, r.h0, m, r.h1});
                stack.push_back(Piece{r.l0, r.h0, r.l1, m});
            }
        }
    }
    return GBEM_OK;
}

// Error-driven refinement (Sec. 3.2, Proposition "error": a net's charge
// error is bounded by C sup_j |I_j| sup_{x in I_j} |dq/dtau|).  With the
// piecewise-constant density of a solve, the tangential derivative on panel j
// is estimated from the panels that share a piece of its boundary (same
// conductor, closed rectangles meeting in a segment of positive length,
// across face edges too) as the largest |q_k - q_j| / |c_k - c_j| (c: panel
// centres); eta_j = |I_j| times that.
// Panels with eta_j >= theta max_k eta_k (when that maximum is positive) are
// bisected across their longer edge (the first in-plane axis on a tie).
// Neighbours are found by a sweep over the panels' boxes sorted along the
// axis of the largest spread.
gbem_status mesh_refine(const std::vector<int8_t>& axis, const std::vector<double>& geo,
                        const std::vector<int32_t>& cond, const double* density, double theta,
                        std::vector<int8_t>& axis_out, std::vector<double>& geo_out,
                        std::vector<int32_t>& cond_out, std::vector<double>& eta, int& n_marked)
{
    const int n = (int)axis.size();
    auto inplane = [](int k, int& p, int& q) {
        p = k == 0 ? 1 : 0;
        q = k == 2 ? 1 : 2;
    };
    // closed boxes and centres
    std::vector<double> lo(3 * (size_t)n), hi(3 * (size_t)n), ctr(3 * (size_t)n), area(n);
    double scale = 0.0;
    for (int i = 0; i < n; ++i) {
        const double* g = &geo[5 * (size_t)i];
        int p, q;
        inplane(axis[i], p, q);
        const int k = axis[i];
        lo[3 * i + k] = hi[3 * i + k] = ctr[3 * i + k] = g[0];
        lo[3 * i + p] = g[1];
        hi[3 * i + p] = g[2];
        ctr[3 * i + p] = 0.5 * (g[1] + g[2]);
        lo[3 * i + q] = g[3];
        hi[3 * i + q] = g[4];
        ctr[3 * i + q] = 0.5 * (g[3] + g[4]);
        area[i] = (g[2] - g[1]) * (g[4] - g[3]);
        for (int e = 0; e < 5; ++e) scale = std::max(scale, std::fabs(g[e]));
    }
    const double tol = 1e-9 * (1.0 + scale);
    // sweep axis: the one with the largest spread of box starts
    int ax = 0;
    double best = -1.0;
    for (int a = 0; a < 3; ++a) {
        double mn = 1e300, mx = -1e300;
        for (int i = 0; i < n; ++i) {
            mn = std::min(mn, lo[3 * i + a]);
            mx = std::max(mx, lo[3 * i + a]);
        }
        if (mx - mn > best) {
            best = mx - mn;
            ax = a;
        }
    }
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::sort(order.begin(), order.end(), [&](int a, int b) { return lo[3 * a + ax] < lo[3 * b + ax]; });
    std::vector<double> grad(n, 0.0);
    for (int u = 0; u < n; ++u) {
        const int j = order[u];
        for (int w = u + 1; w < n; ++w) {
            const int k = order[w];
            if (lo[3 * k + ax] > hi[3 * j + ax] + tol) break;
            if (cond[k] != cond[j]) continue;
            // closed rectangles meeting in a segment of positive length
            bool touch = true;
            double longest = 0.0;
            for (int a = 0; a < 3 && touch; ++a) {
                const double ov = std::min(hi[3 * j + a], hi[3 * k + a]) - std::max(lo[3 * j + a], lo[3 * k + a]);
                touch = ov >= -tol;
                longest = std::max(longest, ov);
            }
            if (!touch || !(longest > tol)) continue;
            double d2 = 0.0;
            for (int a = 0; a < 3; ++a) {
                const double d = ctr[3 * j + a] - ctr[3 * k + a];
                d2 += d * d;
            }
            const double g = std::fabs(density[k] - density[j]) / std::sqrt(d2);
            grad[j] = std::max(grad[j], g);
            grad[k] = std::max(grad[k], g);
        }
    }
    eta.assign(n, 0.0);
    double eta_max = 0.0;
    for (int i = 0; i < n; ++i) {
        eta[i] = area[i] * grad[i];
        eta_max = std::max(eta_max, eta[i]);
    }
    axis_out.clear();
    geo_out.clear();
    cond_out.clear();
    n_marked = 0;
    for (int i = 0; i < n; ++i) {
        const double* g = &geo[5 * (size_t)i];
        const bool mark = eta_max > 0.0 && eta[i] >= theta * eta_max;
        auto push = [&](double l0, double h0, double l1, double h1) {
            axis_out.push_back(axis[i]);
            geo_out.push_back(g[0]);
            geo_out.push_back(l0);
            geo_out.push_back(h0);
            geo_out.push_back(l1);
            geo_out.push_back(h1);
            cond_out.push_back(cond[i]);
        };
        if (!mark) {
            push(g[1], g[2], g[3], g[4]);
            continue;
        }
        ++n_marked;
        if (g[2] - g[1] >= g[4] - g[3]) {
            const double m = 0.5 * (g[1] + g[2]);
            push(g[1], m, g[3], g[4]);
            push(m, g[2], g[3], g[4]);
        } else {
            const double m = 0.5 * (g[3] + g[4]);
            push(g[1], g[2], g[3], m);
            push(g[1], g[2], m, g[4]);
        }
    }
    return GBEM_OK;
}
