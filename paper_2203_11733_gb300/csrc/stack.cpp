// Layered dielectric stacks (Wu & Li, Sec. 4): the host mesher, the layout of
// the per-region system and the gbem_stack_* entry points.  The kernels are
// in dielectric.cu.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include "gbem_internal.h"

struct gbem_stack_s {
    gbem_ctx* ctx = nullptr;
    int n = 0, n_eq = 0, np = 0, nc = 0, R = 0;
    // panels, in mesher order
    std::vector<int8_t> axis, sign;
    std::vector<double> geo;        // 5 per panel
    std::vector<int32_t> kind, cond, ra, rb;
    std::vector<double> eps;
    // layout
    std::vector<int32_t> ucol, qcol, bcol, cidx, row_panel, reg_off, cond_ids;
    std::vector<long long> tile_off;
    // device
    void* meta = nullptr;
    size_t meta_bytes = 0;
    gbem_precision prec = GBEM_FP64;
    void* M0 = nullptr;             // the assembled system (FP64)
    void* Mf = nullptr;             // the copy factored in place (FP64, or FP32 in mixed mode)
    size_t m0_bytes = 0, mf_bytes = 0;
    void* work = nullptr;           // B, X, R, W, Y, Inv, P, C, ipiv, perm, status, norms
    size_t work_bytes = 0;
    StackView v;
    bool assembled = false, factored = false;
    int iters = 0;                  // corrections of the last solve
    cudaStream_t last = nullptr;
    // the mixed factor's lookahead: panels on a second stream (highest
    // priority), joined by two events; created at first use
    cudaStream_t side = nullptr;
    cudaEvent_t ev_ready = nullptr, ev_done = nullptr;
};

namespace {

struct Dev {
    int prev = -1;
    explicit Dev(int d)
    {
        if (d >= 0 && cudaGetDevice(&prev) == cudaSuccess && prev != d) cudaSetDevice(d);
        else prev = -1;
    }
    ~Dev()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

void cells(double lo, double hi, double h, std::vector<double>& out)
{
    gbem_mesh_params p{h, 1.0, 0.0};
    mesh_divide(lo, hi, &p, out);
}

struct Mesher {
    gbem_stack_s* S;
    // the paper's partition (graded): the main net's boxes and parameters
    bool graded = false;
    std::vector<gbem_box> mains;
    double mlo[3] = {0, 0, 0}, mhi[3] = {0, 0, 0};
    double p1 = 0, p2 = 0, p3 = 0, p5 = 0;
    void add(int k, double c, double a0, double b0, double a1, double b1, int kind, int cond, int ra, int rb,
             int sign)
    {
        S->axis.push_back((int8_t)k);
        const double g[5] = {c, a0, b0, a1, b1};
        S->geo.insert(S->geo.end(), g, g + 5);
        S->kind.push_back(kind);
        S->cond.push_back(cond);
        S->ra.push_back(ra);
        S->rb.push_back(rb);
        S->sign.push_back((int8_t)sign);
    }
    double main_distance(int k, double c, double l0, double h0, double l1, double h1) const
    {
        const int pa = k == 0 ? 1 : 0, qa = k == 2 ? 1 : 2;
        double lo[3], hi[3];
        lo[k] = hi[k] = c;
        lo[pa] = l0;
        hi[pa] = h0;
        lo[qa] = l1;
        hi[qa] = h1;
        double best = 1e300;
        for (const gbem_box& B : mains) {
            double d2 = 0.0;
            for (int d = 0; d < 3; ++d) {
                const double g = std::max(0.0, std::max(B.lo[d] - hi[d], lo[d] - B.hi[d]));
                d2 += g * g;
            }
            best = std::min(best, std::sqrt(d2));
        }
        return best;
    }
    // the paper's partition of one face: bisect the longer edge (the first
    // on a tie), first half first, until |I| <= p4 within p5 of the main net
    // and p4 p3 (d/p5)^power beyond, and both edges <= hcap
    void graded_face(int k, double c, double a0, double b0, double a1, double b1, double hcap, double p4, int power,
                     int kind, int cond, int ra, int rb, int sign)
    {
        struct Piece {
            double l0, h0, l1, h1;
        };
        std::vector<Piece> st{Piece{a0, b0, a1, b1}};
        while (!st.empty()) {
            const Piece r = st.back();
            st.pop_back();
            const double d = main_distance(k, c, r.l0, r.h0, r.l1, r.h1);
            double limit = p4;
            if (d >= p5) {
                const double t = d / p5;
                limit = p4 * p3 * (power == 3 ? t * t * t : t * t);
            }
            const double e0 = r.h0 - r.l0, e1 = r.h1 - r.l1;
            if (!(e0 * e1 > limit || (hcap > 0.0 && std::max(e0, e1) > hcap))) {
                add(k, c, r.l0, r.h0, r.l1, r.h1, kind, cond, ra, rb, sign);
                continue;
            }
            if (e0 >= e1) {
                const double m = 0.5 * (r.l0 + r.h0);
                st.push_back(Piece{m, r.h0, r.l1, r.h1});
                st.push_back(Piece{r.l0, m, r.l1, r.h1});
            } else {
                const double m = 0.5 * (r.l1 + r.h1);
                st.push_back(Piece{r.l0, r.h0, m, r.h1});
                st.push_back(Piece{r.l0, r.h0, r.l1, m});
            }
        }
    }
    // the face's panels: the uniform grid, or the paper's partition (rule 3:
    // conductors and the enclosure, 2: interfaces)
    void face(int k, double c, double a0, double b0, double a1, double b1, double h, int power, bool toward, int kind,
              int cond, int ra, int rb, int sign)
    {
        if (graded) graded_face(k, c, a0, b0, a1, b1, h, toward ? p1 : p1 * p2, power, kind, cond, ra, rb, sign);
        else grid(k, c, a0, b0, a1, b1, h, kind, cond, ra, rb, sign);
    }
    // every cell of the tensor grid of [a0,b0] x [a1,b1]
    void grid(int k, double c, double a0, double b0, double a1, double b1, double h, int kind, int cond, int ra,
              int rb, int sign)
    {
        std::vector<double> n0, n1;
        cells(a0, b0, h, n0);
        cells(a1, b1, h, n1);
        for (size_t i = 0; i + 1 < n0.size(); ++i)
            for (size_t j = 0; j + 1 < n1.size(); ++j) add(k, c, n0[i], n0[i + 1], n1[j], n1[j + 1], kind, cond, ra, rb, sign);
    }
};

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

gbem_status stack_build(const gbem_stack* st, const gbem_box* boxes, int nbox, gbem_stack_s* S, std::string& err)
{
    const int R = st->n_layers;
    if (R < 1 || R > GBEM_MAX_LAYERS) return err = "n_layers must be 1 .. GBEM_MAX_LAYERS", GBEM_ERR_ARG;
    for (int d = 0; d < 3; ++d)
        if (!(st->lo[d] < st->hi[d]) || !std::isfinite(st->lo[d]) || !std::isfinite(st->hi[d]))
            return err = "empty enclosure", GBEM_ERR_MESH;
    if (st->z[0] != st->lo[2] || st->z[R] != st->hi[2]) return err = "layer planes must span lo[2] .. hi[2]", GBEM_ERR_ARG;
    for (int a = 0; a < R; ++a) {
        if (!(st->z[a] < st->z[a + 1])) return err = "layer planes must increase", GBEM_ERR_ARG;
        if (!finite_pos(st->eps_r[a])) return err = "eps_r must be positive", GBEM_ERR_ARG;
    }
    for (int f = 0; f < 6; ++f)
        if (st->face_bc[f] < GBEM_FACE_NEUMANN) return err = "bad face condition", GBEM_ERR_ARG;
    if (!finite_pos(st->h) || !(st->h_outer >= 0.0) || !std::isfinite(st->h_outer))
        return err = "cell sizes must be positive", GBEM_ERR_ARG;
    if (nbox < 0 || (nbox > 0 && !boxes)) return err = "boxes", GBEM_ERR_ARG;
    const double h_out = st->h_outer > 0.0 ? st->h_outer : st->h;
    Mesher m{S};
    if (st->graded) {
        if (!(st->p1 > 0.0) || !(st->p2 >= 1.0) || !(st->p3 > 0.0) || !(st->p5 > 0.0) || !std::isfinite(st->p1) ||
            !std::isfinite(st->p2) || !std::isfinite(st->p3) || !std::isfinite(st->p5))
            return err = "graded stacks need p1 > 0, p2 >= 1, p3 > 0, p5 > 0", GBEM_ERR_ARG;
        m.graded = true;
        m.p1 = st->p1;
        m.p2 = st->p2;
        m.p3 = st->p3;
        m.p5 = st->p5;
        for (int d = 0; d < 3; ++d) {
            m.mlo[d] = 1e300;
            m.mhi[d] = -1e300;
        }
        for (int b = 0; b < nbox; ++b)
            if (boxes[b].conductor == st->main_conductor) {
                m.mains.push_back(boxes[b]);
                for (int d = 0; d < 3; ++d) {
                    m.mlo[d] = std::min(m.mlo[d], boxes[b].lo[d]);
                    m.mhi[d] = std::max(m.mhi[d], boxes[b].hi[d]);
                }
            }
        if (m.mains.empty()) return err = "no box of the main conductor", GBEM_ERR_ARG;
    }
    auto layer_of = [&](double zz) {
        for (int a = 0; a < R; ++a)
            if (st->z[a] < zz && zz < st->z[a + 1]) return a;
        return -1;
    };
    for (int b = 0; b < nbox; ++b) {
        const gbem_box& B = boxes[b];
        if (B.conductor < 0) return err = "conductor ids must be >= 0", GBEM_ERR_ARG;
        bool inside = true;
        for (int d = 0; d < 3; ++d) inside = inside && st->lo[d] < B.lo[d] && B.lo[d] < B.hi[d] && B.hi[d] < st->hi[d];
        if (!inside || layer_of(B.lo[2]) < 0 || layer_of(B.hi[2]) < 0)
            return err = "every box must lie strictly inside the enclosure, its bottom and top off the layer planes",
                   GBEM_ERR_MESH;
        for (int c = 0; c < b; ++c) {
            bool apart = false;
            for (int d = 0; d < 3; ++d) apart = apart || boxes[c].hi[d] < B.lo[d] || B.hi[d] < boxes[c].lo[d];
            if (!apart) return err = "boxes must not touch or overlap", GBEM_ERR_MESH;
        }
        for (int k = 0; k < 3; ++k) {
            const int p = k == 0 ? 1 : 0, q = k == 2 ? 1 : 2;
            // the region lies outside the box: its outward normal points into
            // it; a face looks toward the main net when some of the net lies
            // beyond its plane on the conductor's outward side
            const bool is_main = B.conductor == st->main_conductor;
            for (int side = 0; side < 2; ++side) {
                const double plane = side ? B.hi[k] : B.lo[k];
                const bool toward = is_main || (side ? m.mhi[k] > plane : m.mlo[k] < plane);
                const int sign = side ? -1 : 1;
                if (k == 2) {
                    m.face(k, plane, B.lo[p], B.hi[p], B.lo[q], B.hi[q], st->h, 3, toward, 0, B.conductor,
                           layer_of(plane), -1, sign);
                } else {
                    // q == 2: a side face is cut where it crosses a layer plane
                    for (int a = 0; a < R; ++a)
                        if (st->z[a] < B.hi[2] && B.lo[2] < st->z[a + 1])
                            m.face(k, plane, B.lo[p], B.hi[p], std::max(B.lo[2], st->z[a]),
                                   std::min(B.hi[2], st->z[a + 1]), st->h, 3, toward, 0, B.conductor, a, -1, sign);
                }
            }
        }
    }
    for (int k = 0; k < 3; ++k) {
        const int p = k == 0 ? 1 : 0, q = k == 2 ? 1 : 2;
        for (int s = 0; s < 2; ++s) {
            const double plane = s ? st->hi[k] : st->lo[k];
            const int bc = st->face_bc[2 * k + s], sign = s ? 1 : -1;
            if (k == 2) {
                m.face(k, plane, st->lo[p], st->hi[p], st->lo[q], st->hi[q], h_out, 3, true, 1, bc, s ? R - 1 : 0, -1,
                       sign);
            } else {
                // q == 2: the face is cut at every layer plane
                for (int a = 0; a < R; ++a)
                    m.face(k, plane, st->lo[p], st->hi[p], st->z[a], st->z[a + 1], h_out, 3, true, 1, bc, a, -1, sign);
            }
        }
    }
    for (int a = 1; a < R; ++a) {
        // the interface is cut along the footprints of the boxes that cross
        // it; cells inside a footprint are holes
        const double za = st->z[a];
        std::vector<const gbem_box*> holes;
        for (int b = 0; b < nbox; ++b)
            if (boxes[b].lo[2] < za && za < boxes[b].hi[2]) holes.push_back(&boxes[b]);
        std::vector<double> bx{st->lo[0], st->hi[0]}, by{st->lo[1], st->hi[1]};
        for (const gbem_box* B : holes) {
            bx.push_back(B->lo[0]);
            bx.push_back(B->hi[0]);
            by.push_back(B->lo[1]);
            by.push_back(B->hi[1]);
        }
        std::sort(bx.begin(), bx.end());
        bx.erase(std::unique(bx.begin(), bx.end()), bx.end());
        std::sort(by.begin(), by.end());
        by.erase(std::unique(by.begin(), by.end()), by.end());
        for (size_t i = 0; i + 1 < bx.size(); ++i)
            for (size_t j = 0; j + 1 < by.size(); ++j) {
                const double cx = 0.5 * (bx[i] + bx[i + 1]), cy = 0.5 * (by[j] + by[j + 1]);
                bool hole = false;
                for (const gbem_box* B : holes) hole = hole || (B->lo[0] < cx && cx < B->hi[0] && B->lo[1] < cy && cy < B->hi[1]);
                if (hole) continue;
                m.face(2, za, bx[i], bx[i + 1], by[j], by[j + 1], h_out, 2, true, 2, GBEM_PANEL_INTERFACE, a - 1, a, 1);
            }
    }
    S->eps.assign(st->eps_r, st->eps_r + R);
    S->R = R;
    S->n = (int)S->axis.size();
    return GBEM_OK;
}

// Rows: per region, its boundary panels in panel order.  Columns: per panel,
// u (insulating faces, interfaces) then q (all but insulating faces).
gbem_status stack_layout(gbem_stack_s* S, std::string& err)
{
    const int n = S->n, R = S->R;
    S->reg_off.assign(R + 1, 0);
    S->row_panel.clear();
    for (int a = 0; a < R; ++a) {
        S->reg_off[a] = (int32_t)S->row_panel.size();
        for (int i = 0; i < n; ++i)
            if (S->ra[i] == a || S->rb[i] == a) S->row_panel.push_back(i);
    }
    S->reg_off[R] = (int32_t)S->row_panel.size();
    S->ucol.assign(n, -1);
    S->qcol.assign(n, -1);
    int col = 0;
    for (int i = 0; i < n; ++i) {
        if (S->cond[i] == GBEM_FACE_NEUMANN || S->cond[i] == GBEM_PANEL_INTERFACE) S->ucol[i] = col++;
        if (S->cond[i] != GBEM_FACE_NEUMANN) S->qcol[i] = col++;
    }
    S->n_eq = (int)S->row_panel.size();
    if (col != S->n_eq) return err = "the stack's system is not square", GBEM_ERR_MESH;
    std::vector<int32_t> ids;
    for (int i = 0; i < n; ++i)
        if (S->cond[i] >= 0) ids.push_back(S->cond[i]);
    std::sort(ids.begin(), ids.end());
    ids.erase(std::unique(ids.begin(), ids.end()), ids.end());
    if (ids.empty()) return err = "no conductor", GBEM_ERR_MESH;
    S->cond_ids = ids;
    S->nc = (int)ids.size();
    S->bcol.assign(n, -1);
    S->cidx.assign(n, -1);
    for (int i = 0; i < n; ++i)
        if (S->cond[i] >= 0) {
            const int m = (int)(std::lower_bound(ids.begin(), ids.end(), S->cond[i]) - ids.begin());
            S->cidx[i] = m;
            if (S->ucol[i] < 0) S->bcol[i] = m;
        }
    S->tile_off.assign(R + 1, 0);
    for (int a = 0; a < R; ++a) {
        const long long nt = (S->reg_off[a + 1] - S->reg_off[a] + 31) / 32;
        S->tile_off[a + 1] = S->tile_off[a] + nt * nt;
    }
    S->np = (S->n_eq + 63) / 64 * 64;
    return GBEM_OK;
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// One device allocation for the geometry and layout; views into it.
gbem_status stack_upload(gbem_stack_s* S)
{
    gbem_ctx* ctx = S->ctx;
    const size_t n = S->n, R = S->R;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    const size_t o_geo = take(sizeof(double) * 5 * n), o_axis = take(n), o_sign = take(n);
    const size_t o_ra = take(4 * n), o_u = take(4 * n), o_q = take(4 * n), o_b = take(4 * n), o_ci = take(4 * n);
    const size_t o_rows = take(4 * (size_t)S->n_eq), o_reg = take(4 * (R + 1)), o_tile = take(8 * (R + 1));
    const size_t o_eps = take(8 * R);
    std::vector<unsigned char> host(off, 0);
    double* geo = reinterpret_cast<double*>(host.data() + o_geo);
    for (size_t i = 0; i < n; ++i)
        for (int e = 0; e < 5; ++e) geo[e * n + i] = S->geo[5 * i + e];
    std::memcpy(host.data() + o_axis, S->axis.data(), n);
    std::memcpy(host.data() + o_sign, S->sign.data(), n);
    std::memcpy(host.data() + o_ra, S->ra.data(), 4 * n);
    std::memcpy(host.data() + o_u, S->ucol.data(), 4 * n);
    std::memcpy(host.data() + o_q, S->qcol.data(), 4 * n);
    std::memcpy(host.data() + o_b, S->bcol.data(), 4 * n);
    std::memcpy(host.data() + o_ci, S->cidx.data(), 4 * n);
    std::memcpy(host.data() + o_rows, S->row_panel.data(), 4 * (size_t)S->n_eq);
    std::memcpy(host.data() + o_reg, S->reg_off.data(), 4 * (R + 1));
    std::memcpy(host.data() + o_tile, S->tile_off.data(), 8 * (R + 1));
    std::memcpy(host.data() + o_eps, S->eps.data(), 8 * R);
    void* d = ctx_alloc(ctx, off, nullptr);
    if (!d) return ctx_fail(ctx, GBEM_ERR_OOM, "stack geometry");
    S->meta = d;
    S->meta_bytes = off;
    if (cudaMemcpy(d, host.data(), off, cudaMemcpyHostToDevice) != cudaSuccess)
        return ctx_fail(ctx, GBEM_ERR_CUDA, "stack upload");
    unsigned char* b = static_cast<unsigned char*>(d);
    StackView& v = S->v;
    v.n = S->n;
    v.n_eq = S->n_eq;
    v.np = S->np;
    v.nc = S->nc;
    v.R_layers = S->R;
    const double* g = reinterpret_cast<const double*>(b + o_geo);
    v.c = g;
    v.lo0 = g + n;
    v.hi0 = g + 2 * n;
    v.lo1 = g + 3 * n;
    v.hi1 = g + 4 * n;
    v.axis = reinterpret_cast<const int8_t*>(b + o_axis);
    v.sign = reinterpret_cast<const int8_t*>(b + o_sign);
    v.ra = reinterpret_cast<const int32_t*>(b + o_ra);
    v.ucol = reinterpret_cast<const int32_t*>(b + o_u);
    v.qcol = reinterpret_cast<const int32_t*>(b + o_q);
    v.bcol = reinterpret_cast<const int32_t*>(b + o_b);
    v.cidx = reinterpret_cast<const int32_t*>(b + o_ci);
    v.row_panel = reinterpret_cast<const int32_t*>(b + o_rows);
    v.reg_off = reinterpret_cast<const int32_t*>(b + o_reg);
    v.tile_off = reinterpret_cast<const long long*>(b + o_tile);
    v.eps = reinterpret_cast<const double*>(b + o_eps);
    return GBEM_OK;
}

void stack_free(gbem_stack_s* S, cudaStream_t s)
{
    gbem_ctx* ctx = S->ctx;
    if (S->work) ctx_free(ctx, S->work, S->work_bytes, s);
    if (S->Mf) ctx_free(ctx, S->Mf, S->mf_bytes, s);
    if (S->M0) ctx_free(ctx, S->M0, S->m0_bytes, s);
    S->work = S->Mf = S->M0 = nullptr;
}

// The matrices and the solve's buffers for precision `prec` (kept while the
// precision stays the same).
gbem_status stack_alloc(gbem_stack_s* S, gbem_precision prec, cudaStream_t s)
{
    if (S->M0 && S->prec == prec) return GBEM_OK;
    if (S->M0) {
        if (cudaStreamSynchronize(S->last) != cudaSuccess) return ctx_fail(S->ctx, GBEM_ERR_CUDA, "sync");
        stack_free(S, S->last);
    }
    gbem_ctx* ctx = S->ctx;
    const size_t np = S->np, nc = S->nc;
    const bool mixed = prec == GBEM_MIXED;
    S->prec = prec;
    S->m0_bytes = sizeof(double) * np * np;
    S->mf_bytes = (mixed ? sizeof(float) : sizeof(double)) * np * np;
    S->M0 = ctx_alloc(ctx, S->m0_bytes, s);
    if (!S->M0) return ctx_fail(ctx, GBEM_ERR_OOM, "stack matrix");
    S->Mf = ctx_alloc(ctx, S->mf_bytes, s);
    if (!S->Mf) return ctx_fail(ctx, GBEM_ERR_OOM, "stack matrix copy");
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    const size_t vec = 8 * np * nc;
    const size_t o_B = take(vec), o_X = take(vec), o_R = take(vec), o_W = take(vec), o_Y = take(vec);
    const size_t o_inv = take((mixed ? 4 : 8) * np * 2 * 64);
    const size_t o_P = take(stack_partial_bytes((int)np, (int)nc)), o_C = take(8 * nc * nc);
    const size_t o_piv = take(4 * np), o_perm = take(4 * np), o_st = take(4), o_nrm = take(16 * nc);
    const size_t o_plan = take(4 * (1 + 4 * 64));
    S->work = ctx_alloc(ctx, off, s);
    if (!S->work) return ctx_fail(ctx, GBEM_ERR_OOM, "stack work space");
    S->work_bytes = off;
    unsigned char* b = static_cast<unsigned char*>(S->work);
    StackView& v = S->v;
    v.M0 = static_cast<double*>(S->M0);
    v.M = mixed ? nullptr : static_cast<double*>(S->Mf);
    v.M32 = mixed ? static_cast<float*>(S->Mf) : nullptr;
    v.B = reinterpret_cast<double*>(b + o_B);
    v.X = reinterpret_cast<double*>(b + o_X);
    v.R = reinterpret_cast<double*>(b + o_R);
    v.W = b + o_W;
    v.Y = b + o_Y;
    v.Inv = b + o_inv;
    v.P = reinterpret_cast<double*>(b + o_P);
    v.C = reinterpret_cast<double*>(b + o_C);
    v.ipiv = reinterpret_cast<int*>(b + o_piv);
    v.perm = reinterpret_cast<int*>(b + o_perm);
    v.status = reinterpret_cast<int*>(b + o_st);
    v.norms = reinterpret_cast<unsigned long long*>(b + o_nrm);
    v.plan = reinterpret_cast<int*>(b + o_plan);
    return GBEM_OK;
}

bool ok(gbem_ctx* ctx, cudaError_t e, const char* what)
{
    if (e == cudaSuccess) return true;
    ctx_fail(ctx, GBEM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    return false;
}

}  // namespace

gbem_status gbem_stack_mesh(gbem_ctx* ctx, const gbem_stack* stack, const gbem_box* boxes, int nbox,
                            gbem_stack_t** out)
{
    if (!ctx || !stack || !out) return GBEM_ERR_ARG;
    *out = nullptr;
    gbem_stack_s* S = new (std::nothrow) gbem_stack_s();
    if (!S) return GBEM_ERR_OOM;
    S->ctx = ctx;
    std::string err;
    gbem_status st = stack_build(stack, boxes, nbox, S, err);
    if (st == GBEM_OK) st = stack_layout(S, err);
    if (st == GBEM_OK && S->n_eq > 32768) {
        err = "more than 32768 equations";
        st = GBEM_ERR_ARG;
    }
    if (st != GBEM_OK) {
        delete S;
        return ctx_fail(ctx, st, err);
    }
    if (ctx->device >= 0) {
        Dev g(ctx->device);
        st = stack_upload(S);
        if (st != GBEM_OK) {
            gbem_stack_destroy(S);
            return st;
        }
    }
    *out = S;
    return GBEM_OK;
}

gbem_status gbem_stack_info(const gbem_stack_t* S, int* n_panels, int* n_eq, int* n_cond)
{
    if (!S) return GBEM_ERR_ARG;
    if (n_panels) *n_panels = S->n;
    if (n_eq) *n_eq = S->n_eq;
    if (n_cond) *n_cond = S->nc;
    return GBEM_OK;
}

gbem_status gbem_stack_panels(const gbem_stack_t* S, int8_t* axis, double* geo, int32_t* kind, int32_t* cond,
                              int32_t* region_a, int32_t* region_b, int8_t* sign, int32_t* cond_ids)
{
    if (!S) return GBEM_ERR_ARG;
    const size_t n = S->n;
    if (axis) std::memcpy(axis, S->axis.data(), n);
    if (geo) std::memcpy(geo, S->geo.data(), sizeof(double) * 5 * n);
    if (kind) std::memcpy(kind, S->kind.data(), 4 * n);
    if (cond) std::memcpy(cond, S->cond.data(), 4 * n);
    if (region_a) std::memcpy(region_a, S->ra.data(), 4 * n);
    if (region_b) std::memcpy(region_b, S->rb.data(), 4 * n);
    if (sign) std::memcpy(sign, S->sign.data(), n);
    if (cond_ids) std::memcpy(cond_ids, S->cond_ids.data(), 4 * (size_t)S->nc);
    return GBEM_OK;
}

gbem_status gbem_stack_assemble(gbem_stack_t* S, gbem_precision prec, gbem_stream stream)
{
    if (!S) return GBEM_ERR_ARG;
    gbem_ctx* ctx = S->ctx;
    if (ctx->device < 0) return ctx_fail(ctx, GBEM_ERR_NODEV, "context has no device");
    if (prec != GBEM_FP64 && prec != GBEM_MIXED) return ctx_fail(ctx, GBEM_ERR_ARG, "bad precision");
    Dev g(ctx->device);
    TraceScope ts(ctx);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    gbem_status st = stack_alloc(S, prec, s);
    if (st != GBEM_OK) return st;
    S->last = s;
    S->assembled = S->factored = false;
    if (!ok(ctx, stack_gl_upload(s), "quadrature nodes") ||
        !ok(ctx, launch_stack_assemble(S->v, S->tile_off[S->R], prec == GBEM_MIXED, s), "stack assembly"))
        return GBEM_ERR_CUDA;
    S->assembled = true;
    return GBEM_OK;
}

gbem_status gbem_stack_system(gbem_stack_t* S, double* M_host, double* B_host)
{
    if (!S) return GBEM_ERR_ARG;
    gbem_ctx* ctx = S->ctx;
    if (!S->assembled) return ctx_fail(ctx, GBEM_ERR_STATE, "system not assembled");
    Dev g(ctx->device);
    if (!ok(ctx, cudaStreamSynchronize(S->last), "sync")) return GBEM_ERR_CUDA;
    const size_t n = S->n_eq, np = S->np;
    if (M_host) {
        std::vector<double> col(np * n);
        if (!ok(ctx, cudaMemcpy(col.data(), S->v.M0, sizeof(double) * np * n, cudaMemcpyDeviceToHost), "download"))
            return GBEM_ERR_CUDA;
        for (size_t c = 0; c < n; ++c)
            for (size_t r = 0; r < n; ++r) M_host[r * n + c] = col[c * np + r];
    }
    if (B_host) {
        std::vector<double> col(np * S->nc);
        if (!ok(ctx, cudaMemcpy(col.data(), S->v.B, sizeof(double) * np * S->nc, cudaMemcpyDeviceToHost), "download"))
            return GBEM_ERR_CUDA;
        for (size_t m = 0; m < (size_t)S->nc; ++m)
            for (size_t r = 0; r < n; ++r) B_host[r * S->nc + m] = col[m * np + r];
    }
    return GBEM_OK;
}

gbem_status gbem_stack_capacitance(gbem_stack_t* S, gbem_stream stream, double* C_host, double* resid)
{
    if (!S || !C_host) return GBEM_ERR_ARG;
    gbem_ctx* ctx = S->ctx;
    if (ctx->device < 0) return ctx_fail(ctx, GBEM_ERR_NODEV, "context has no device");
    if (!S->assembled) {
        gbem_status st = gbem_stack_assemble(S, GBEM_FP64, stream);
        if (st != GBEM_OK) return st;
    }
    Dev g(ctx->device);
    TraceScope ts(ctx);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (s != S->last) {
        // order this stream after the last one's work on the stack
        cudaEvent_t ev;
        if (!ok(ctx, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "event")) return GBEM_ERR_CUDA;
        cudaEventRecord(ev, S->last);
        cudaStreamWaitEvent(s, ev, 0);
        cudaEventDestroy(ev);
        S->last = s;
    }
    const bool mixed = S->prec == GBEM_MIXED;
    StackView& v = S->v;
    const size_t np = S->np, nc = S->nc;
    if (mixed && !S->side) {
        int least = 0, greatest = 0;
        if (!ok(ctx, cudaDeviceGetStreamPriorityRange(&least, &greatest), "priorities") ||
            !ok(ctx, cudaStreamCreateWithPriority(&S->side, cudaStreamNonBlocking, greatest), "stream") ||
            !ok(ctx, cudaEventCreateWithFlags(&S->ev_ready, cudaEventDisableTiming), "event") ||
            !ok(ctx, cudaEventCreateWithFlags(&S->ev_done, cudaEventDisableTiming), "event"))
            return GBEM_ERR_CUDA;
    }
    if (!S->factored) {
        if (!ok(ctx, cudaMemsetAsync(v.status, 0, sizeof(int), s), "memset") ||
            !ok(ctx, launch_stack_lu(v, mixed, s, mixed ? S->side : nullptr, S->ev_ready, S->ev_done), "LU"))
            return GBEM_ERR_CUDA;
        S->factored = true;
    }
    // X = 0, R = B; corrections X += (LU)^-1 P R, R = B - M0 X until the
    // residual meets the tolerance (one correction in FP64 mode, normally)
    const double tol = ctx->tune.ir_tol > 0.0 ? ctx->tune.ir_tol : 1e-11;
    const int max_iter = ctx->tune.ir_max_iter > 0 ? ctx->tune.ir_max_iter : 10;
    if (!ok(ctx, cudaMemsetAsync(v.X, 0, sizeof(double) * np * nc, s), "memset") ||
        !ok(ctx, cudaMemcpyAsync(v.R, v.B, sizeof(double) * np * nc, cudaMemcpyDeviceToDevice, s), "copy"))
        return GBEM_ERR_CUDA;
    std::vector<unsigned long long> nrm(2 * nc);
    double worst = 0.0;
    int status = 0;
    S->iters = 0;
    for (int it = 0; it < max_iter; ++it) {
        if (!ok(ctx, launch_stack_correct(v, mixed, s), "solve") || !ok(ctx, launch_stack_residual(v, s), "residual") ||
            !ok(ctx, cudaMemcpyAsync(nrm.data(), v.norms, 16 * nc, cudaMemcpyDeviceToHost, s), "d2h") ||
            !ok(ctx, cudaMemcpyAsync(&status, v.status, sizeof(int), cudaMemcpyDeviceToHost, s), "d2h") ||
            !ok(ctx, cudaStreamSynchronize(s), "sync"))
            return GBEM_ERR_CUDA;
        S->iters = it + 1;
        if (status != 0) {
            S->factored = false;
            return ctx_fail(ctx, GBEM_ERR_NOT_SPD, "LU met a zero pivot: the stack's system is singular");
        }
        worst = 0.0;
        for (size_t m = 0; m < nc; ++m) {
            double r, b;
            std::memcpy(&r, &nrm[m], 8);
            std::memcpy(&b, &nrm[nc + m], 8);
            worst = std::max(worst, b > 0.0 ? r / b : r);
        }
        if (!(worst > tol)) break;
    }
    const double eps0 = 8.8541878128e-12;
    if (!ok(ctx, launch_stack_charges(v, eps0, s), "charges") ||
        !ok(ctx, cudaMemcpyAsync(C_host, v.C, sizeof(double) * nc * nc, cudaMemcpyDeviceToHost, s), "d2h") ||
        !ok(ctx, cudaStreamSynchronize(s), "sync"))
        return GBEM_ERR_CUDA;
    if (resid) *resid = worst;
    if (!(worst <= tol)) return ctx_fail(ctx, GBEM_ERR_NOCONV, "refinement missed its tolerance");
    return GBEM_OK;
}

gbem_status gbem_stack_iterations(const gbem_stack_t* S, int* iters)
{
    if (!S || !iters) return GBEM_ERR_ARG;
    *iters = S->iters;
    return GBEM_OK;
}

void gbem_stack_destroy(gbem_stack_t* S)
{
    if (!S) return;
    gbem_ctx* ctx = S->ctx;
    if (ctx->device >= 0 && (S->meta || S->M0 || S->work)) {
        Dev g(ctx->device);
        cudaStreamSynchronize(S->last);
        if (S->side) cudaStreamSynchronize(S->side);
        stack_free(S, S->last);
        if (S->meta) ctx_free(ctx, S->meta, S->meta_bytes, nullptr);
        if (S->ev_ready) cudaEventDestroy(S->ev_ready);
        if (S->ev_done) cudaEventDestroy(S->ev_done);
        if (S->side) cudaStreamDestroy(S->side);
    }
    delete S;
}
