// Host construction of APRIL approximations (A- and F-interval lists), the
// sets' accessors, and a host execution of Algorithm 2 used for measurement.
//
// Construction (paper Sec. 4.1 for what the lists hold, Sec. 6 for how):
//  1. Touched cells.  For every edge, each cell row its closed y-range meets is
//     intersected exactly (rational arithmetic in int64) with the edge to get
//     the x-range of the edge inside that closed row strip; every closed cell
//     of that x-range meets the edge.  For each such cell an exact
//     separating-axis test tells whether the edge also enters the cell's OPEN
//     square ("crossed").  This is the grid traversal of Sec. 6.1 done row by
//     row, with closed cells so that edges along grid lines and through grid
//     corners mark every cell they touch.
//  2. The touched cells are sorted by Hilbert id.  Between two consecutive
//     touched ids lies a gap of untouched cells; consecutive Hilbert cells
//     share an edge, and an untouched cell is either inside the polygon or
//     disjoint from it, so a whole gap is one class and a single
//     point-in-polygon test at its first cell decides it (Sec. 6.2, Alg. 3's
//     observation).  A touched cell that is not crossed is Full when its
//     centre is inside the polygon (it touches the boundary only along its
//     border), otherwise Partial.  Crossed cells are Partial.
//  3. One pass over the sorted ids emits maximal A intervals (all non-empty
//     cells) and F intervals (Full cells).
// Point-in-polygon tests use a crossing count against the edges bucketed by
// the cell row whose centre line they straddle.

#include <algorithm>
#include <atomic>
#include <cfenv>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <thread>

#include "april_internal.h"
#include "geom.h"

namespace april {

static thread_local std::string g_last_error;

april_status fail(april_status code, const std::string &msg) {
    g_last_error = msg;
    return code;
}

namespace {

using namespace april_geom;

struct GridI {
    int64_t ox, oy, h;
    uint32_t order;
    int64_t G;
};

struct Scratch {
    std::vector<uint64_t> keys;      // (hilbert id << 1) | crossed
    std::vector<int64_t> ex0, ey0, ex1, ey1;  // edges, oriented upwards (ey0 < ey1)
    std::vector<uint32_t> row_start, row_edges;
};

struct PolyLists {
    std::vector<uint32_t> A, F;  // st,end pairs
};

// Emits maximal intervals from a stream of increasing [st, end) runs.
struct RunSink {
    std::vector<uint32_t> *out;
    bool open = false;
    uint64_t st = 0, en = 0;
    void add(uint64_t a, uint64_t b) {
        if (open && a == en) {
            en = b;
            return;
        }
        flush();
        open = true;
        st = a;
        en = b;
    }
    void flush() {
        if (open) {
            out->push_back((uint32_t)st);
            out->push_back((uint32_t)en);  // 2^32 wraps to 0 by design
        }
        open = false;
    }
};

april_status build_one(const int32_t *xy, uint64_t nv, const GridI &g, Scratch &sc, PolyLists &out) {
    out.A.clear();
    out.F.clear();
    if (nv < 3) return fail(APRIL_ERR_GEOMETRY, "polygon with fewer than 3 vertices");
    const int64_t h = g.h, G = g.G, ox = g.ox, oy = g.oy;
    int64_t xmn = xy[0], xmx = xy[0], ymn = xy[1], ymx = xy[1];
    for (uint64_t k = 1; k < nv; ++k) {
        xmn = std::min<int64_t>(xmn, xy[2 * k]);
        xmx = std::max<int64_t>(xmx, xy[2 * k]);
        ymn = std::min<int64_t>(ymn, xy[2 * k + 1]);
        ymx = std::max<int64_t>(ymx, xy[2 * k + 1]);
    }
    // window of cells meeting the MBR
    int64_t wi0, wj0, wi1, wj1;
    cell_window(xmn, ymn, xmx, ymx, ox, oy, h, G, wi0, wj0, wi1, wj1);
    if (wi0 > wi1 || wj0 > wj1) return fail(APRIL_ERR_GEOMETRY, "polygon outside the grid");

    // edges, upward
    sc.ex0.resize(nv); sc.ey0.resize(nv); sc.ex1.resize(nv); sc.ey1.resize(nv);
    for (uint64_t k = 0; k < nv; ++k) {
        const uint64_t kn = (k + 1 == nv) ? 0 : k + 1;
        const EdgeUp e = edge_up(xy[2 * k], xy[2 * k + 1], xy[2 * kn], xy[2 * kn + 1]);
        sc.ex0[k] = e.ax; sc.ey0[k] = e.ay; sc.ex1[k] = e.bx; sc.ey1[k] = e.by;
    }

    // 1. touched cells, row by row per edge
    sc.keys.clear();
    for (uint64_t k = 0; k < nv; ++k) {
        const EdgeUp e{sc.ex0[k], sc.ey0[k], sc.ex1[k], sc.ey1[k]};
        int64_t j0, j1;
        edge_rows(e, oy, h, G, j0, j1);
        for (int64_t j = j0; j <= j1; ++j) {
            int64_t i0, i1;
            if (!edge_cells_in_row(e, ox, oy, h, G, j, i0, i1)) continue;
            const int64_t Y0 = oy + j * h;
            for (int64_t i = i0; i <= i1; ++i) {
                const bool crossed = enters_open_square(e.ax, e.ay, e.bx, e.by, ox + i * h, Y0, h);
                const uint64_t d = hilbert_id(g.order, (uint32_t)i, (uint32_t)j);
                sc.keys.push_back((d << 1) | (crossed ? 1u : 0u));
            }
        }
    }
    std::sort(sc.keys.begin(), sc.keys.end());

    // point-in-polygon support: edges bucketed by the rows whose centre line
    // they straddle ((ey0 <= yc < ey1), the half-open crossing rule)
    const int64_t nrows = wj1 - wj0 + 1;
    sc.row_start.assign((size_t)nrows + 1, 0);
    auto row_span = [&](uint64_t k, int64_t &r0, int64_t &r1) {
        centre_rows(EdgeUp{sc.ex0[k], sc.ey0[k], sc.ex1[k], sc.ey1[k]}, oy, h, wj0, wj1, r0, r1);
    };
    for (uint64_t k = 0; k < nv; ++k) {
        int64_t r0, r1;
        row_span(k, r0, r1);
        for (int64_t r = r0; r <= r1; ++r) sc.row_start[(size_t)(r - wj0) + 1]++;
    }
    for (int64_t r = 0; r < nrows; ++r) sc.row_start[(size_t)r + 1] += sc.row_start[(size_t)r];
    sc.row_edges.resize(sc.row_start[(size_t)nrows]);
    {
        std::vector<uint32_t> fill(sc.row_start.begin(), sc.row_start.end() - 1);
        for (uint64_t k = 0; k < nv; ++k) {
            int64_t r0, r1;
            row_span(k, r0, r1);
            for (int64_t r = r0; r <= r1; ++r) sc.row_edges[fill[(size_t)(r - wj0)]++] = (uint32_t)k;
        }
    }
    auto inside = [&](uint32_t i, uint32_t j) -> bool {
        if ((int64_t)i < wi0 || (int64_t)i > wi1 || (int64_t)j < wj0 || (int64_t)j > wj1) return false;
        const int64_t xc = ox + (int64_t)i * h + h / 2, yc = oy + (int64_t)j * h + h / 2;
        const size_t r = (size_t)((int64_t)j - wj0);
        bool in = false;
        for (uint32_t e = sc.row_start[r]; e < sc.row_start[r + 1]; ++e) {
            uint32_t k = sc.row_edges[e];
            if (turn(sc.ex0[k], sc.ey0[k], sc.ex1[k], sc.ey1[k], xc, yc) > 0) in = !in;
        }
        return in;
    };
    auto gap_is_full = [&](uint64_t first) -> bool {
        uint32_t x, y;
        hilbert_cell(g.order, first, x, y);
        return inside(x, y);
    };

    // 2+3. walk touched ids and the gaps between them
    RunSink A{&out.A}, F{&out.F};
    const uint64_t ncells = (uint64_t)G * (uint64_t)G;
    uint64_t next = 0;  // first id not yet classified
    size_t k = 0;
    const size_t nk = sc.keys.size();
    while (k < nk) {
        const uint64_t d = sc.keys[k] >> 1;
        bool crossed = false;
        while (k < nk && (sc.keys[k] >> 1) == d) crossed |= (sc.keys[k++] & 1u) != 0;
        if (d > next) {  // gap [next, d)
            if (gap_is_full(next)) {
                A.add(next, d);
                F.add(next, d);
            }
        }
        A.add(d, d + 1);
        if (!crossed) {
            uint32_t x, y;
            hilbert_cell(g.order, d, x, y);
            if (inside(x, y)) F.add(d, d + 1);
        }
        next = d + 1;
    }
    if (next < ncells && gap_is_full(next)) {
        A.add(next, ncells);
        F.add(next, ncells);
    }
    A.flush();
    F.flush();
    if (out.A.empty()) return fail(APRIL_ERR_GEOMETRY, "polygon meets no cell");
    return APRIL_OK;
}

april_status check_grid(const april_grid *grid, GridI &g) {
    if (!grid) return fail(APRIL_ERR_INVALID_ARG, "grid is NULL");
    if (grid->order < 1 || grid->order > 16) return fail(APRIL_ERR_INVALID_ARG, "grid order must be 1..16");
    if (grid->log2_cell < 1 || grid->log2_cell > 30) return fail(APRIL_ERR_INVALID_ARG, "log2_cell must be 1..30");
    g.ox = grid->ox;
    g.oy = grid->oy;
    g.h = (int64_t)1 << grid->log2_cell;
    g.order = grid->order;
    g.G = (int64_t)1 << grid->order;
    // keep every int64 product in the predicates exact
    const int64_t lim = (int64_t)1 << 26;
    if (g.ox < -lim || g.ox > lim || g.oy < -lim || g.oy > lim || g.h * g.G > lim)
        return fail(APRIL_ERR_INVALID_ARG, "grid outside the supported coordinate range");
    return APRIL_OK;
}

template <class F>
void parallel_for(uint64_t n, uint32_t n_threads, uint64_t chunk, F &&fn) {
    if (n_threads == 0) n_threads = std::max(1u, std::thread::hardware_concurrency());
    n_threads = (uint32_t)std::min<uint64_t>(n_threads, std::max<uint64_t>(1, (n + chunk - 1) / chunk));
    std::atomic<uint64_t> next{0};
    auto worker = [&](uint32_t tid) {
        for (;;) {
            uint64_t b = next.fetch_add(chunk);
            if (b >= n) break;
            uint64_t e = std::min(n, b + chunk);
            fn(tid, b, e);
        }
    };
    if (n_threads <= 1) {
        worker(0);
        return;
    }
    std::vector<std::thread> th;
    th.reserve(n_threads);
    for (uint32_t t = 0; t < n_threads; ++t) th.emplace_back(worker, t);
    for (auto &t : th) t.join();
}

uint32_t resolve_threads(uint32_t n) {
    return n ? n : std::max(1u, std::thread::hardware_concurrency());
}


// Lays out per-entry lists as the device image: each list starts at an even
// interval slot (16-byte aligned), and the entry descriptors point at them.
april_status assemble_lists(april_sets *S, const std::vector<PolyLists> &lists, uint32_t nt) {
    const size_t E = lists.size();
    S->desc.assign(E * 4, 0u);
    uint64_t slot = 0;
    S->a_total = S->f_total = 0;
    for (size_t p = 0; p < E; ++p) {
        uint64_t na = lists[p].A.size() / 2, nf = lists[p].F.size() / 2;
        S->desc[4 * p + 0] = (uint32_t)slot;
        S->desc[4 * p + 1] = (uint32_t)na;
        slot += (na + 1) & ~1ull;
        S->desc[4 * p + 2] = (uint32_t)slot;
        S->desc[4 * p + 3] = (uint32_t)nf;
        slot += (nf + 1) & ~1ull;
        S->a_total += na;
        S->f_total += nf;
        if (slot > 0xFFFFFFF0ull) return fail(APRIL_ERR_INVALID_ARG, "more than 2^32 interval slots in one set");
    }
    S->iv.assign((size_t)slot * 2, 0u);
    parallel_for(E, nt, 256, [&](uint32_t, uint64_t b, uint64_t e) {
        for (uint64_t p = b; p < e; ++p) {
            const auto &L = lists[p];
            if (!L.A.empty()) std::memcpy(&S->iv[2 * (size_t)S->desc[4 * p + 0]], L.A.data(), L.A.size() * 4);
            if (!L.F.empty()) std::memcpy(&S->iv[2 * (size_t)S->desc[4 * p + 2]], L.F.data(), L.F.size() * 4);
        }
    });
    return APRIL_OK;
}

struct Mbr {
    int64_t x0, y0, x1, y1;
};

Mbr poly_mbr(const int32_t *xy, uint64_t nv) {
    Mbr m{xy[0], xy[1], xy[0], xy[1]};
    for (uint64_t k = 1; k < nv; ++k) {
        m.x0 = std::min<int64_t>(m.x0, xy[2 * k]);
        m.y0 = std::min<int64_t>(m.y0, xy[2 * k + 1]);
        m.x1 = std::max<int64_t>(m.x1, xy[2 * k]);
        m.y1 = std::max<int64_t>(m.y1, xy[2 * k + 1]);
    }
    return m;
}

// Closed partition squares [k*side, (k+1)*side] met by the closed range [lo, hi].
inline void part_range(int64_t lo, int64_t hi, int64_t side, int64_t parts, int64_t &k0, int64_t &k1) {
    k0 = std::max<int64_t>(ceil_div(lo, side) - 1, 0);
    k1 = std::min<int64_t>(floor_div(hi, side), parts - 1);
}

}  // namespace

april_status check_grid_params(const april_grid *grid, int64_t &ox, int64_t &oy, int64_t &h, uint32_t &order,
                               int64_t &G) {
    GridI g{};
    const april_status st = check_grid(grid, g);
    if (st) return st;
    ox = g.ox, oy = g.oy, h = g.h, order = g.order, G = g.G;
    return APRIL_OK;
}

}  // namespace april

using namespace april;

extern "C" april_status april_last_error(char *buf, size_t buf_size) {
    if (!buf || buf_size == 0) return APRIL_ERR_INVALID_ARG;
    std::snprintf(buf, buf_size, "%s", g_last_error.c_str());
    return APRIL_OK;
}

extern "C" april_status april_build_sets(const int32_t *xy, const uint64_t *vert_off, uint32_t n_polys,
                                         const april_grid *grid, uint32_t n_threads, april_sets **out) {
    if (!out) return fail(APRIL_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if ((!xy || !vert_off) && n_polys) return fail(APRIL_ERR_INVALID_ARG, "xy/vert_off is NULL");
    GridI g;
    april_status st = check_grid(grid, g);
    if (st) return st;
    for (uint32_t p = 0; p < n_polys; ++p)
        if (vert_off[p + 1] < vert_off[p]) return fail(APRIL_ERR_INVALID_ARG, "vert_off is not monotone");
    try {
        std::vector<PolyLists> lists(n_polys);
        uint32_t nt = resolve_threads(n_threads);
        std::vector<Scratch> scratch(nt);
        std::atomic<int> err{0};
        std::vector<std::string> errmsg(nt);
        parallel_for(n_polys, nt, 64, [&](uint32_t tid, uint64_t b, uint64_t e) {
            for (uint64_t p = b; p < e && !err.load(std::memory_order_relaxed); ++p) {
                april_status s = build_one(xy + 2 * vert_off[p], vert_off[p + 1] - vert_off[p], g, scratch[tid],
                                           lists[p]);
                if (s) {
                    char m[160];
                    std::snprintf(m, sizeof m, "polygon %llu: ", (unsigned long long)p);
                    errmsg[tid] = std::string(m) + g_last_error;
                    int zero = 0;
                    err.compare_exchange_strong(zero, s);
                }
            }
        });
        if (err.load()) {
            for (auto &m : errmsg)
                if (!m.empty()) return fail(err.load(), m);
            return fail(err.load(), "construction failed");
        }
        auto *S = new april_sets();
        S->n = n_polys;
        S->n_entries = n_polys;
        S->order = g.order;
        S->grid_known = true;
        S->grid_ox = g.ox;
        S->grid_oy = g.oy;
        S->grid_log2_cell = grid->log2_cell;
        S->grid_id = april_grid_id(g.ox, g.oy, grid->log2_cell, g.order);
        S->mbr.resize(4 * (size_t)n_polys);
        for (uint32_t p = 0; p < n_polys; ++p) {
            const Mbr m = poly_mbr(xy + 2 * vert_off[p], vert_off[p + 1] - vert_off[p]);
            int32_t *o = &S->mbr[4 * (size_t)p];
            o[0] = (int32_t)m.x0, o[1] = (int32_t)m.y0, o[2] = (int32_t)m.x1, o[3] = (int32_t)m.y1;
        }
        st = assemble_lists(S, lists, nt);
        if (st) {
            delete S;
            return st;
        }
        *out = S;
        return APRIL_OK;
    } catch (const std::bad_alloc &) {
        return fail(APRIL_ERR_NO_MEMORY, "host allocation failed while building sets");
    }
}

extern "C" april_status april_cell_ids(const april_grid *grid, const int64_t *x, const int64_t *y, uint64_t n,
                                       uint64_t *ids) {
    GridI g;
    april_status st = check_grid(grid, g);
    if (st) return st;
    if (n && (!x || !y || !ids)) return fail(APRIL_ERR_INVALID_ARG, "NULL array");
    uint8_t lut[64];
    april_geom::hilbert_lut_build(lut);
    for (uint64_t k = 0; k < n; ++k) {
        const int64_t cx = floor_div(x[k] - g.ox, g.h), cy = floor_div(y[k] - g.oy, g.h);
        ids[k] = cx < 0 || cy < 0 || cx >= g.G || cy >= g.G
                     ? ~0ull
                     : april_geom::hilbert_id_lut(lut, g.order, (uint32_t)cx, (uint32_t)cy);
    }
    return APRIL_OK;
}

extern "C" april_status april_sets_from_lists(uint32_t n, uint32_t order, const uint64_t *a_off,
                                             const uint32_t *a_iv, const uint64_t *f_off, const uint32_t *f_iv,
                                             const int32_t *mbr, april_sets **out) {
    if (!out) return fail(APRIL_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (order < 1 || order > 16) return fail(APRIL_ERR_INVALID_ARG, "grid order must be 1..16");
    if (n && (!a_off || !f_off)) return fail(APRIL_ERR_INVALID_ARG, "NULL offsets");
    const uint64_t ncells = (uint64_t)1 << (2 * order);
    try {
        std::vector<PolyLists> lists(n);
        for (int side = 0; side < 2; ++side) {
            const uint64_t *off = side ? f_off : a_off;
            const uint32_t *iv = side ? f_iv : a_iv;
            if (off[n] > off[0] && !iv) return fail(APRIL_ERR_INVALID_ARG, "NULL interval array");
            for (uint32_t o = 0; o < n; ++o) {
                if (off[o + 1] < off[o]) return fail(APRIL_ERR_INVALID_ARG, "offsets are not monotone");
                uint64_t prev_end = 0;
                auto &L = side ? lists[o].F : lists[o].A;
                for (uint64_t k = off[o]; k < off[o + 1]; ++k) {
                    const uint64_t st = iv[2 * k];
                    const uint64_t en = iv[2 * k + 1] == 0 && ncells == (1ull << 32) ? ncells : iv[2 * k + 1];
                    if (st >= en || en > ncells || (k > off[o] && st < prev_end)) {
                        char m[128];
                        std::snprintf(m, sizeof m, "object %u: intervals must be non-empty, sorted and disjoint", o);
                        return fail(APRIL_ERR_INVALID_ARG, m);
                    }
                    prev_end = en;
                    L.push_back((uint32_t)st);
                    L.push_back((uint32_t)en);
                }
            }
        }
        // an approximation's Full cells are among the cells it meets (Sec.
        // 4.1): every F interval must lie inside one A interval
        for (uint32_t o = 0; o < n; ++o) {
            const auto &Al = lists[o].A, &Fl = lists[o].F;
            size_t a = 0;
            for (size_t f = 0; f < Fl.size(); f += 2) {
                const uint64_t fs = Fl[f], fe = Fl[f + 1] == 0 ? ncells : Fl[f + 1];
                while (a < Al.size() && (Al[a + 1] == 0 ? ncells : Al[a + 1]) < fe) a += 2;
                if (a >= Al.size() || Al[a] > fs) {
                    char m[128];
                    std::snprintf(m, sizeof m, "object %u: an F interval is not inside an A interval", o);
                    return fail(APRIL_ERR_INVALID_ARG, m);
                }
            }
        }
        auto *S = new april_sets();
        S->n = n;
        S->n_entries = n;
        S->order = order;
        if (mbr) S->mbr.assign(mbr, mbr + 4 * (size_t)n);
        april_status st = assemble_lists(S, lists, 0);
        if (st) {
            delete S;
            return st;
        }
        *out = S;
        return APRIL_OK;
    } catch (const std::bad_alloc &) {
        return fail(APRIL_ERR_NO_MEMORY, "host allocation failed while importing lists");
    }
}

extern "C" april_status april_quantize_polygons(const double *xy, const uint64_t *vert_off, uint32_t n_polys,
                                               int32_t *out_xy, uint64_t *out_off) {
    if (n_polys && (!xy || !vert_off || !out_xy || !out_off)) return fail(APRIL_ERR_INVALID_ARG, "NULL argument");
    if (!n_polys) {
        if (out_off) out_off[0] = 0;
        return APRIL_OK;
    }
    if (std::fegetround() != FE_TONEAREST) return fail(APRIL_ERR_INVALID_ARG, "the FPU must round to nearest");
    const double scale = (double)(1 << 24);
    uint64_t o = 0;
    out_off[0] = 0;
    for (uint32_t p = 0; p < n_polys; ++p) {
        if (vert_off[p + 1] < vert_off[p]) return fail(APRIL_ERR_INVALID_ARG, "vert_off is not monotone");
        const uint64_t first = o;
        for (uint64_t k = vert_off[p]; k < vert_off[p + 1]; ++k) {
            int32_t q[2];
            for (int c = 0; c < 2; ++c) {
                const double v = xy[2 * k + c];
                if (!std::isfinite(v)) return fail(APRIL_ERR_INVALID_ARG, "non-finite coordinate");
                // x * 2^24 is exact; nearbyint rounds half to even in the default mode
                const double r = std::nearbyint(std::min(std::max(v * scale, 0.0), scale));
                q[c] = (int32_t)r;
            }
            if (o > first && out_xy[2 * (o - 1)] == q[0] && out_xy[2 * (o - 1) + 1] == q[1]) continue;
            out_xy[2 * o] = q[0];
            out_xy[2 * o + 1] = q[1];
            ++o;
        }
        while (o - first > 1 && out_xy[2 * (o - 1)] == out_xy[2 * first] && out_xy[2 * (o - 1) + 1] == out_xy[2 * first + 1])
            --o;  // a closing vertex equal to the first
        out_off[p + 1] = o;
    }
    return APRIL_OK;
}

extern "C" void april_sets_destroy(april_sets *sets) { delete sets; }

extern "C" april_status april_sets_get_info(const april_sets *S, april_sets_info *info) {
    if (!S || !info) return fail(APRIL_ERR_INVALID_ARG, "NULL argument");
    const april_image_layout L = april_layout(*S);
    info->n_objects = S->n;
    info->order = S->order;
    info->a_intervals = S->a_total;
    info->f_intervals = S->f_total;
    info->iv_slots = S->iv.size() / 2;
    info->device_bytes = L.total;
    info->parts = S->parts;
    info->n_entries = S->n_entries;
    info->packed = S->packed ? 1u : 0u;
    info->reserved = 0;
    info->raw_list_bytes = (uint64_t)S->n_entries * 16 + (uint64_t)S->iv.size() * 4;
    info->packed_list_bytes = S->packed ? (uint64_t)S->pdesc.size() * 4 + (uint64_t)S->anchors.size() * 4 +
                                              (uint64_t)S->gaps.size()
                                        : 0;
    return APRIL_OK;
}

extern "C" april_status april_sets_list(const april_sets *S, uint32_t entry, int which, const uint32_t **iv,
                                        uint32_t *n) {
    if (!S || !iv || !n || (which != 0 && which != 1)) return fail(APRIL_ERR_INVALID_ARG, "bad argument");
    if (entry >= S->n_entries) return fail(APRIL_ERR_OUT_OF_RANGE_ID, "entry out of range");
    uint32_t off = S->desc[4 * (size_t)entry + 2 * which], len = S->desc[4 * (size_t)entry + 2 * which + 1];
    *iv = S->iv.data() + 2 * (size_t)off;
    *n = len;
    return APRIL_OK;
}

extern "C" april_status april_sets_mbrs(const april_sets *S, int32_t *mbr) {
    if (!S || (S->n && !mbr)) return fail(APRIL_ERR_INVALID_ARG, "NULL argument");
    std::copy(S->mbr.begin(), S->mbr.end(), mbr);
    return APRIL_OK;
}

extern "C" april_status april_sets_lengths(const april_sets *S, uint32_t *a_len, uint32_t *f_len) {
    if (!S || (S->n_entries && (!a_len || !f_len))) return fail(APRIL_ERR_INVALID_ARG, "NULL argument");
    for (uint32_t e = 0; e < S->n_entries; ++e) {
        a_len[e] = S->desc[4 * (size_t)e + 1];
        f_len[e] = S->desc[4 * (size_t)e + 3];
    }
    return APRIL_OK;
}

extern "C" april_status april_sets_object_entries(const april_sets *S, uint32_t obj, uint32_t *first,
                                                  uint32_t *count) {
    if (!S || !first || !count) return fail(APRIL_ERR_INVALID_ARG, "NULL argument");
    if (obj >= S->n) return fail(APRIL_ERR_OUT_OF_RANGE_ID, "object id out of range");
    if (S->parts == 0) {
        *first = obj;
        *count = 1;
    } else {
        *first = S->obj_entry[obj];
        *count = S->obj_entry[obj + 1] - S->obj_entry[obj];
    }
    return APRIL_OK;
}

extern "C" april_status april_sets_entry_grid(const april_sets *S, uint32_t entry, uint32_t *pid, april_grid *grid) {
    if (!S || !pid || !grid) return fail(APRIL_ERR_INVALID_ARG, "NULL argument");
    if (entry >= S->n_entries) return fail(APRIL_ERR_OUT_OF_RANGE_ID, "entry out of range");
    if (S->parts == 0) return fail(APRIL_ERR_INVALID_ARG, "sets are not partitioned");
    const uint32_t p = S->entry_pid[entry];
    *pid = p;
    grid->ox = S->part_grid[4 * (size_t)p];
    grid->oy = S->part_grid[4 * (size_t)p + 1];
    grid->log2_cell = (uint32_t)S->part_grid[4 * (size_t)p + 2];
    grid->order = S->order;
    return APRIL_OK;
}

extern "C" april_status april_sets_packed_list(const april_sets *S, uint32_t entry, int which,
                                               const uint32_t **blocks, const uint8_t **gaps, uint32_t *n) {
    if (!S || !blocks || !gaps || !n || (which != 0 && which != 1)) return fail(APRIL_ERR_INVALID_ARG, "bad argument");
    if (!S->packed) return fail(APRIL_ERR_INVALID_ARG, "sets are not compressed");
    if (entry >= S->n_entries) return fail(APRIL_ERR_OUT_OF_RANGE_ID, "entry out of range");
    *blocks = S->anchors.data() + 2 * (size_t)S->pdesc[4 * (size_t)entry + 2 * which];
    *gaps = S->gaps.data();
    *n = S->pdesc[4 * (size_t)entry + 2 * which + 1];
    return APRIL_OK;
}

// Partitioned sets (Sec. 5.2).  The data space [0, 2^24]^2 is split into
// parts x parts equal partitions.  An object is approximated once for every
// partition its (closed) MBR meets, on that partition's own grid of `order`.
// The partition's raster area is the smallest square of power-of-two side
// whose corner is a multiple of its cell side and which covers the MBRs of all
// objects of both inputs that meet the partition (the paper defines it by
// "the MBR of these objects").
extern "C" april_status april_build_partitioned_sets(const int32_t *r_xy, const uint64_t *r_off, uint32_t r_n,
                                                     const int32_t *s_xy, const uint64_t *s_off, uint32_t s_n,
                                                     uint32_t parts, uint32_t order, uint32_t n_threads,
                                                     april_sets **out_r, april_sets **out_s) {
    if (!out_r || !out_s) return fail(APRIL_ERR_INVALID_ARG, "out is NULL");
    *out_r = *out_s = nullptr;
    if ((r_n && (!r_xy || !r_off)) || (s_n && (!s_xy || !s_off))) return fail(APRIL_ERR_INVALID_ARG, "NULL polygons");
    if (parts < 1 || parts > 4096 || (parts & (parts - 1)))
        return fail(APRIL_ERR_INVALID_ARG, "parts must be a power of two in [1, 4096]");
    if (order < 1 || order > 16) return fail(APRIL_ERR_INVALID_ARG, "order must be 1..16");
    const int64_t L = (int64_t)1 << 24, side = L / parts;
    const uint32_t nt = resolve_threads(n_threads);
    try {
        const int32_t *xys[2] = {r_xy, s_xy};
        const uint64_t *offs[2] = {r_off, s_off};
        const uint32_t ns[2] = {r_n, s_n};
        std::vector<Mbr> mbr[2];
        for (int side_i = 0; side_i < 2; ++side_i) {
            mbr[side_i].resize(ns[side_i]);
            for (uint32_t p = 0; p < ns[side_i]; ++p) {
                const uint64_t nv = offs[side_i][p + 1] - offs[side_i][p];
                if (offs[side_i][p + 1] < offs[side_i][p] || nv < 3)
                    return fail(APRIL_ERR_GEOMETRY, "polygon with fewer than 3 vertices");
                Mbr m = poly_mbr(xys[side_i] + 2 * offs[side_i][p], nv);
                if (m.x0 < 0 || m.y0 < 0 || m.x1 > L || m.y1 > L)
                    return fail(APRIL_ERR_GEOMETRY, "polygon outside the data space [0, 2^24]^2");
                mbr[side_i][p] = m;
            }
        }
        // bounds of every partition's members
        const size_t P = (size_t)parts * parts;
        std::vector<int64_t> lo_x(P, INT64_MAX), lo_y(P, INT64_MAX), hi_x(P, INT64_MIN), hi_y(P, INT64_MIN);
        for (int side_i = 0; side_i < 2; ++side_i)
            for (const Mbr &m : mbr[side_i]) {
                int64_t kx0, kx1, ky0, ky1;
                part_range(m.x0, m.x1, side, parts, kx0, kx1);
                part_range(m.y0, m.y1, side, parts, ky0, ky1);
                for (int64_t ky = ky0; ky <= ky1; ++ky)
                    for (int64_t kx = kx0; kx <= kx1; ++kx) {
                        const size_t q = (size_t)(ky * parts + kx);
                        lo_x[q] = std::min(lo_x[q], m.x0);
                        lo_y[q] = std::min(lo_y[q], m.y0);
                        hi_x[q] = std::max(hi_x[q], m.x1);
                        hi_y[q] = std::max(hi_y[q], m.y1);
                    }
            }
        std::vector<int64_t> grid_desc(4 * P, 0);
        std::vector<GridI> grids(P);
        for (size_t q = 0; q < P; ++q) {
            if (lo_x[q] == INT64_MAX) continue;
            for (uint32_t k = order + 1; k < 40; ++k) {
                const int64_t size = (int64_t)1 << k, h = size >> order;
                const int64_t ox = floor_div(lo_x[q], h) * h, oy = floor_div(lo_y[q], h) * h;
                if (ox + size >= hi_x[q] && oy + size >= hi_y[q]) {
                    grids[q] = GridI{ox, oy, h, order, (int64_t)1 << order};
                    grid_desc[4 * q] = ox;
                    grid_desc[4 * q + 1] = oy;
                    grid_desc[4 * q + 2] = (int64_t)(k - order);
                    grid_desc[4 * q + 3] = 1;
                    break;
                }
            }
        }
        april_sets *out[2] = {nullptr, nullptr};
        for (int side_i = 0; side_i < 2; ++side_i) {
            auto *S = new april_sets();
            S->n = ns[side_i];
            S->order = order;
            S->parts = parts;
            S->part_grid = grid_desc;
            S->grid_known = true;
            S->grid_id = april_part_grid_id(grid_desc, order, parts);
            S->obj_ll.resize(2 * (size_t)S->n);
            S->mbr.resize(4 * (size_t)S->n);
            for (uint32_t p = 0; p < S->n; ++p) {
                const Mbr &m = mbr[side_i][p];
                int32_t *o = &S->mbr[4 * (size_t)p];
                o[0] = (int32_t)m.x0, o[1] = (int32_t)m.y0, o[2] = (int32_t)m.x1, o[3] = (int32_t)m.y1;
            }
            S->obj_entry.assign((size_t)S->n + 1, 0u);
            std::vector<uint32_t> ent_obj;
            for (uint32_t p = 0; p < S->n; ++p) {
                const Mbr &m = mbr[side_i][p];
                S->obj_ll[2 * (size_t)p] = (int32_t)m.x0;
                S->obj_ll[2 * (size_t)p + 1] = (int32_t)m.y0;
                int64_t kx0, kx1, ky0, ky1;
                part_range(m.x0, m.x1, side, parts, kx0, kx1);
                part_range(m.y0, m.y1, side, parts, ky0, ky1);
                for (int64_t ky = ky0; ky <= ky1; ++ky)
                    for (int64_t kx = kx0; kx <= kx1; ++kx) {
                        S->entry_pid.push_back((uint32_t)(ky * parts + kx));
                        ent_obj.push_back(p);
                    }
                S->obj_entry[(size_t)p + 1] = (uint32_t)S->entry_pid.size();
            }
            S->n_entries = (uint32_t)S->entry_pid.size();
            std::vector<PolyLists> lists(S->n_entries);
            std::vector<Scratch> scratch(nt);
            std::atomic<int> err{0};
            parallel_for(S->n_entries, nt, 64, [&](uint32_t tid, uint64_t b, uint64_t e) {
                for (uint64_t q = b; q < e && !err.load(std::memory_order_relaxed); ++q) {
                    const uint32_t p = ent_obj[q];
                    const uint64_t o = offs[side_i][p];
                    april_status st = build_one(xys[side_i] + 2 * o, offs[side_i][p + 1] - o,
                                                grids[S->entry_pid[q]], scratch[tid], lists[q]);
                    if (st) {
                        int zero = 0;
                        err.compare_exchange_strong(zero, st);
                    }
                }
            });
            april_status st = err.load() ? (april_status)err.load() : assemble_lists(S, lists, nt);
            if (st) {
                delete S;
                if (out[0]) delete out[0];
                return st;
            }
            out[side_i] = S;
        }
        *out_r = out[0];
        *out_s = out[1];
        return APRIL_OK;
    } catch (const std::bad_alloc &) {
        return fail(APRIL_ERR_NO_MEMORY, "host allocation failed while building partitioned sets");
    }
}

// Compressed lists (Sec. 5.1: delta encoding, decoded while joining).  A list
// of n intervals is the strictly increasing endpoint sequence
// st_0 < end_0 < st_1 < ... (lists are maximal, so end_i < st_{i+1}), cut into
// blocks of 32 endpoints.  Each block has an 8-byte table entry {anchor = its
// first endpoint, offset of its gap block in 64-byte units | wide << 31} and
// a gap block of 32 slots (slot 0 unused) holding the 31 gaps to the
// following endpoints: uint16 slots (64 bytes) when all 31 gaps fit, else
// uint32 slots (128 bytes).  Gaps are taken mod 2^32, so an end stored as 0
// (2^32) decodes back to 0.
extern "C" april_status april_sets_compress(april_sets *S) {
    if (!S) return fail(APRIL_ERR_INVALID_ARG, "sets is NULL");
    if (S->packed) return APRIL_OK;
    try {
        S->pdesc.assign((size_t)S->n_entries * 4, 0u);
        S->anchors.clear();
        S->gaps.clear();
        for (uint32_t e = 0; e < S->n_entries; ++e) {
            for (int which = 0; which < 2; ++which) {
                const uint32_t off = S->desc[4 * (size_t)e + 2 * which], n = S->desc[4 * (size_t)e + 2 * which + 1];
                const uint32_t *v = &S->iv[2 * (size_t)off];  // endpoints v[0 .. 2n)
                const uint32_t ne = 2 * n, nb = (ne + 31) / 32;
                S->pdesc[4 * (size_t)e + 2 * which] = (uint32_t)(S->anchors.size() / 2);
                S->pdesc[4 * (size_t)e + 2 * which + 1] = n;
                for (uint32_t b = 0; b < nb; ++b) {
                    bool wide = false;
                    for (uint32_t k = 1; k < 32 && 32 * b + k < ne; ++k)
                        if ((uint32_t)(v[32 * b + k] - v[32 * b + k - 1]) > 0xFFFFu) wide = true;
                    const size_t base = S->gaps.size();
                    if (base / 64 > 0x7FFFFFF0ull) return fail(APRIL_ERR_INVALID_ARG, "gap stream too large");
                    S->anchors.push_back(v[32 * b]);
                    S->anchors.push_back((uint32_t)(base / 64) | (wide ? 0x80000000u : 0u));
                    S->gaps.resize(base + (wide ? 128 : 64), 0);
                    for (uint32_t k = 1; k < 32 && 32 * b + k < ne; ++k) {
                        const uint32_t g = v[32 * b + k] - v[32 * b + k - 1];
                        if (wide) std::memcpy(&S->gaps[base + 4 * k], &g, 4);
                        else {
                            const uint16_t g16 = (uint16_t)g;
                            std::memcpy(&S->gaps[base + 2 * k], &g16, 2);
                        }
                    }
                }
            }
        }
        S->packed = true;
        return APRIL_OK;
    } catch (const std::bad_alloc &) {
        return fail(APRIL_ERR_NO_MEMORY, "host allocation failed while compressing");
    }
}

namespace {

// IntervalJoin of Algorithm 2 with early exit.  Intervals are [st, end) with
// end stored mod 2^32, so comparisons use last = end - 1.  *used receives the
// number of intervals read on both sides.
bool host_join(const uint32_t *X, uint32_t nx, const uint32_t *Y, uint32_t ny, uint64_t *used) {
    uint32_t i = 0, j = 0;
    while (i < nx && j < ny) {
        uint32_t xs = X[2 * i], xl = X[2 * i + 1] - 1u, ys = Y[2 * j], yl = Y[2 * j + 1] - 1u;
        if (xs <= yl && ys <= xl) {
            *used += (uint64_t)i + 1 + j + 1;
            return true;
        }
        if (xl <= yl) ++i;
        else ++j;
    }
    *used += (uint64_t)std::min(i + 1, nx) + std::min(j + 1, ny);
    return false;
}

// The same join as the GPU kernels read it: each list starts at its first
// interval whose last cell reaches the other list's first start (the merge
// from the front would pass over the intervals before it without a verdict),
// and the merge gallops: once one list has advanced kGallopRun times in a row
// it jumps to its first interval whose last cell reaches the other list's
// current start (the intervals it passes over meet nothing either).  The
// kernels gallop after a window that advanced one list only, so they read at
// least this much.  *used counts the intervals the merge reads plus a binary
// search for every start and jump (bit width of the searched length, in
// probed intervals).
constexpr uint32_t kGallopRun = 16;  // one post of the skip index per 16 intervals

uint32_t lower_bound_last(const uint32_t *L, uint32_t n, uint32_t t) {
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
        const uint32_t mid = lo + (hi - lo) / 2;
        if (L[2 * mid + 1] - 1u < t) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

uint32_t bit_width(uint32_t v) { return v ? 32u - (uint32_t)__builtin_clz(v) : 0u; }

bool host_join_searched(const uint32_t *X, uint32_t nx, const uint32_t *Y, uint32_t ny, uint64_t *used) {
    if (!nx || !ny) return false;
    uint32_t i = lower_bound_last(X, nx, Y[0]), j = lower_bound_last(Y, ny, X[0]);
    *used += bit_width(nx) + bit_width(ny);
    if (i >= nx || j >= ny) return false;
    uint64_t read = 2;   // X[i] and Y[j]
    uint32_t run = 0;    // consecutive advances of the same list
    bool run_x = false;  // ... of X
    for (;;) {
        const uint32_t xs = X[2 * i], xl = X[2 * i + 1] - 1u, ys = Y[2 * j], yl = Y[2 * j + 1] - 1u;
        if (xs <= yl && ys <= xl) {
            *used += read;
            return true;
        }
        const bool adv_x = xl <= yl;
        run = adv_x == run_x ? run + 1 : 1;
        run_x = adv_x;
        if (adv_x) {
            if (++i >= nx) break;
            if (run >= kGallopRun) {
                *used += bit_width(nx - i);
                i += lower_bound_last(X + 2 * (size_t)i, nx - i, ys);
                run = 0;
                if (i >= nx) break;
            }
        } else {
            if (++j >= ny) break;
            if (run >= kGallopRun) {
                *used += bit_width(ny - j);
                j += lower_bound_last(Y + 2 * (size_t)j, ny - j, xs);
                run = 0;
                if (j >= ny) break;
            }
        }
        ++read;
    }
    *used += read;
    return false;
}

}  // namespace

// Entry of object `obj` for partition `pid` (Sec. 5.2 routing), or UINT32_MAX.
static uint32_t find_entry(const april_sets *S, uint32_t obj, uint32_t pid) {
    for (uint32_t e = S->obj_entry[obj]; e < S->obj_entry[obj + 1]; ++e)
        if (S->entry_pid[e] == pid) return e;
    return 0xffffffffu;
}

// The entries a pair (r, s) is evaluated on: the objects themselves on one
// global grid; for partitioned sets (Sec. 5.2) their entries for the
// partition of the lower-left corner of MBR(r) n MBR(s).  An out-of-range id
// or a missing entry gives UINT32_MAX.
static void route_pair(const april_sets *R, const april_sets *S, uint32_t &r, uint32_t &s) {
    if (r >= R->n || s >= S->n) {
        r = s = 0xffffffffu;
        return;
    }
    if (!R->parts) return;
    const int64_t side = ((int64_t)1 << 24) / R->parts;
    const int64_t x = std::max(R->obj_ll[2 * (size_t)r], S->obj_ll[2 * (size_t)s]);
    const int64_t y = std::max(R->obj_ll[2 * (size_t)r + 1], S->obj_ll[2 * (size_t)s + 1]);
    const int64_t P = R->parts;
    const uint32_t pid = (uint32_t)(std::min(y / side, P - 1) * P + std::min(x / side, P - 1));
    r = find_entry(R, r, pid);
    s = find_entry(S, s, pid);
}

extern "C" april_status april_route_pairs(const april_sets *R, const april_sets *S, const uint32_t *pr,
                                          const uint32_t *ps, uint64_t n, uint32_t *er, uint32_t *es) {
    if (!R || !S || (n && (!pr || !ps || !er || !es))) return fail(APRIL_ERR_INVALID_ARG, "NULL argument");
    if (R->parts != S->parts || R->order != S->order) return fail(APRIL_ERR_INVALID_ARG, "R and S use different grids");
    for (uint64_t k = 0; k < n; ++k) {
        uint32_t r = pr[k], s = ps[k];
        route_pair(R, S, r, s);
        er[k] = r;
        es[k] = s;
    }
    return APRIL_OK;
}

// Whether list L (n intervals) holds cell c; *used counts the lookup as the
// triage kernel reads it: a binary search over the list's skip index (one
// post per 16 intervals), then over at most 16 intervals.
static bool host_list_holds(const uint32_t *L, uint32_t n, uint32_t c, uint64_t *used) {
    *used += bit_width(n / 16) + 5;
    const uint32_t i = lower_bound_last(L, n, c);
    return i < n && L[2 * i] <= c;
}

// The triage of the batched kernels: whether the cell under the centre of
// MBR(r) n MBR(s) lies in A(r) and F(s), or in F(r) and A(s) (a true hit).
// *used counts the two MBRs (4 intervals' worth of bytes) and the lookups.
// ro, so: the pairs' objects (their MBRs); the lists' grid: (ox, oy, log2_cell).
static bool host_triage_hit(const april_sets *R, const april_sets *S, uint32_t ro, uint32_t so, int64_t ox,
                            int64_t oy, uint32_t log2_cell, const uint8_t *lut, const uint32_t *Ar, uint32_t nar,
                            const uint32_t *Fr, uint32_t nfr, const uint32_t *As, uint32_t nas, const uint32_t *Fs,
                            uint32_t nfs, uint64_t *used) {
    *used += 4;
    const int32_t *a = &R->mbr[4 * (size_t)ro], *b = &S->mbr[4 * (size_t)so];
    const int64_t x0 = std::max(a[0], b[0]), y0 = std::max(a[1], b[1]), x1 = std::min(a[2], b[2]),
                  y1 = std::min(a[3], b[3]);
    if (x0 > x1 || y0 > y1) return false;
    const int64_t cx = floor_div((x0 + x1) / 2 - ox, (int64_t)1 << log2_cell);
    const int64_t cy = floor_div((y0 + y1) / 2 - oy, (int64_t)1 << log2_cell);
    const int64_t side = (int64_t)1 << R->order;
    if (cx < 0 || cy < 0 || cx >= side || cy >= side) return false;
    const uint32_t c = (uint32_t)hilbert_id_lut(lut, R->order, (uint32_t)cx, (uint32_t)cy);
    if (nfs && nar) {  // the kernel looks both lists up in lockstep
        const bool h1 = host_list_holds(Fs, nfs, c, used), h2 = host_list_holds(Ar, nar, c, used);
        if (h1 && h2) return true;
    }
    if (nfr && nas) {
        const bool h1 = host_list_holds(Fr, nfr, c, used), h2 = host_list_holds(As, nas, c, used);
        if (h1 && h2) return true;
    }
    return false;
}

static april_status host_filter(const april_sets *R, const april_sets *S, const uint32_t *pr, const uint32_t *ps,
                                uint64_t n, uint32_t n_threads, uint8_t *verdict, uint64_t *consumed, bool searched) {
    auto join = searched ? host_join_searched : host_join;
    if (!R || !S || (n && (!pr || !ps || !verdict))) return fail(APRIL_ERR_INVALID_ARG, "NULL argument");
    if (R->parts != S->parts || R->order != S->order) return fail(APRIL_ERR_INVALID_ARG, "R and S use different grids");
    // the batched kernels' triage applies to sets built from polygons on the same grid(s)
    const bool triage = searched && R->grid_known && S->grid_known && R->grid_id == S->grid_id;
    uint8_t lut[64];
    hilbert_lut_build(lut);
    parallel_for(n, resolve_threads(n_threads), 4096, [&](uint32_t, uint64_t b, uint64_t e) {
        for (uint64_t k = b; k < e; ++k) {
            uint32_t r = pr[k], s = ps[k];
            const uint32_t ro = r, so = s;
            uint64_t used = 0;
            uint8_t v;
            route_pair(R, S, r, s);
            if (r >= R->n_entries || s >= S->n_entries) {
                v = APRIL_VERDICT_ERROR;
            } else {
                int64_t gox = R->grid_ox, goy = R->grid_oy;
                uint32_t glc = R->grid_log2_cell;
                bool gok = true;
                if (R->parts) {  // the entry's partition grid
                    const int64_t *pg = &R->part_grid[4 * (size_t)R->entry_pid[r]];
                    gox = pg[0], goy = pg[1], glc = (uint32_t)pg[2], gok = pg[3] != 0;
                }
                const uint32_t *dr = &R->desc[4 * (size_t)r], *ds = &S->desc[4 * (size_t)s];
                const uint32_t *Ar = &R->iv[2 * (size_t)dr[0]], *Fr = &R->iv[2 * (size_t)dr[2]];
                const uint32_t *As = &S->iv[2 * (size_t)ds[0]], *Fs = &S->iv[2 * (size_t)ds[2]];
                if (!searched) {  // Algorithm 2's order: AA, AF, FA
                    if (!join(Ar, dr[1], As, ds[1], &used)) v = APRIL_TRUE_NEGATIVE;
                    else if (join(Ar, dr[1], Fs, ds[3], &used)) v = APRIL_TRUE_HIT;
                    else if (join(Fr, dr[3], As, ds[1], &used)) v = APRIL_TRUE_HIT;
                    else v = APRIL_INCONCLUSIVE;
                } else if (triage && gok && host_triage_hit(R, S, ro, so, gox, goy, glc, lut, Ar, dr[1], Fr, dr[3], As,
                                                           ds[1], Fs, ds[3], &used)) {
                    v = APRIL_TRUE_HIT;  // settled by the triage (an AF or FA overlap)
                } else if (triage) {  // the pairs the triage left: AA, AF, FA, as the kernels join them
                    if (!join(Ar, dr[1], As, ds[1], &used)) v = APRIL_TRUE_NEGATIVE;
                    else if (join(Ar, dr[1], Fs, ds[3], &used)) v = APRIL_TRUE_HIT;
                    else if (join(Fr, dr[3], As, ds[1], &used)) v = APRIL_TRUE_HIT;
                    else v = APRIL_INCONCLUSIVE;
                } else {  // the GPU kernels' order without the triage: AF, AA, FA (same verdicts)
                    if (join(Ar, dr[1], Fs, ds[3], &used)) v = APRIL_TRUE_HIT;
                    else if (!join(Ar, dr[1], As, ds[1], &used)) v = APRIL_TRUE_NEGATIVE;
                    else if (join(Fr, dr[3], As, ds[1], &used)) v = APRIL_TRUE_HIT;
                    else v = APRIL_INCONCLUSIVE;
                }
            }
            verdict[k] = v;
            if (consumed) consumed[k] = used;
        }
    });
    return APRIL_OK;
}

extern "C" april_status april_host_filter(const april_sets *R, const april_sets *S, const uint32_t *pr,
                                          const uint32_t *ps, uint64_t n, uint32_t n_threads, uint8_t *verdict,
                                          uint64_t *consumed) {
    return host_filter(R, S, pr, ps, n, n_threads, verdict, consumed, false);
}

extern "C" april_status april_host_filter_searched(const april_sets *R, const april_sets *S, const uint32_t *pr,
                                                   const uint32_t *ps, uint64_t n, uint32_t n_threads,
                                                   uint8_t *verdict, uint64_t *consumed) {
    return host_filter(R, S, pr, ps, n, n_threads, verdict, consumed, true);
}

namespace {

// One join of a filter variant, sequentially: the merge of Algorithm 2 over
// X and Y, each interval of a side with shift > 0 coarsened as it is read
// (Sec. 5.3); pred 0 looks for an overlap, pred 1 for an X interval that no Y
// interval contains (Sec. 4.3.2).  *used counts the intervals read.
bool host_join_ex(const uint32_t *X, uint32_t nx, uint32_t sx, const uint32_t *Y, uint32_t ny, uint32_t sy, int pred,
                  uint64_t *used) {
    uint32_t i = 0, j = 0;
    auto get = [](const uint32_t *L, uint32_t k, uint32_t sh, uint32_t &st, uint32_t &last) {
        st = L[2 * k] >> sh;
        last = (L[2 * k + 1] - 1u) >> sh;
    };
    while (i < nx && j < ny) {
        uint32_t xs, xl, ys, yl;
        get(X, i, sx, xs, xl);
        get(Y, j, sy, ys, yl);
        if (pred == 0) {
            if (xs <= yl && ys <= xl) {
                *used += (uint64_t)i + 1 + j + 1;
                return true;
            }
        } else if (xl <= yl && ys > xs) {
            *used += (uint64_t)i + 1 + j + 1;
            return true;
        }
        if (xl <= yl) ++i;
        else ++j;
    }
    *used += (uint64_t)std::min(i + 1, nx) + std::min(j + 1, ny);
    return pred == 1 && i < nx;  // containment: X left over once Y ran out
}

}  // namespace

extern "C" april_status april_host_filter_ex(const april_sets *R, const april_sets *S, const uint32_t *pr,
                                             const uint32_t *ps, uint64_t n, int predicate, uint32_t n_threads,
                                             uint8_t *verdict, uint64_t *consumed) {
    if (!R || !S || (n && (!pr || !ps || !verdict))) return fail(APRIL_ERR_INVALID_ARG, "NULL argument");
    if (R->parts || S->parts) return fail(APRIL_ERR_INVALID_ARG, "april_host_filter_ex takes sets on one global grid");
    if (predicate != APRIL_PREDICATE_INTERSECTS && predicate != APRIL_PREDICATE_WITHIN)
        return fail(APRIL_ERR_INVALID_ARG, "unknown predicate");
    if (predicate == APRIL_PREDICATE_WITHIN && R->order != S->order)
        return fail(APRIL_ERR_INVALID_ARG, "the within filter needs both sets on the same grid");
    const uint32_t sx = R->order > S->order ? 2 * (R->order - S->order) : 0;
    const uint32_t sy = S->order > R->order ? 2 * (S->order - R->order) : 0;
    parallel_for(n, resolve_threads(n_threads), 4096, [&](uint32_t, uint64_t b, uint64_t e) {
        for (uint64_t k = b; k < e; ++k) {
            const uint32_t r = pr[k], s = ps[k];
            uint64_t used = 0;
            uint8_t v;
            if (r >= R->n_entries || s >= S->n_entries) {
                v = APRIL_VERDICT_ERROR;
            } else {
                const uint32_t *dr = &R->desc[4 * (size_t)r], *ds = &S->desc[4 * (size_t)s];
                const uint32_t *Ar = &R->iv[2 * (size_t)dr[0]], *Fr = &R->iv[2 * (size_t)dr[2]];
                const uint32_t *As = &S->iv[2 * (size_t)ds[0]], *Fs = &S->iv[2 * (size_t)ds[2]];
                if (!host_join_ex(Ar, dr[1], sx, As, ds[1], sy, 0, &used)) {
                    v = APRIL_TRUE_NEGATIVE;
                } else if (predicate == APRIL_PREDICATE_WITHIN) {
                    v = host_join_ex(Ar, dr[1], 0, Fs, ds[3], 0, 1, &used) ? APRIL_INCONCLUSIVE : APRIL_TRUE_HIT;
                } else if (sx == 0 && sy == 0) {
                    v = (host_join_ex(Ar, dr[1], 0, Fs, ds[3], 0, 0, &used) ||
                         host_join_ex(Fr, dr[3], 0, As, ds[1], 0, 0, &used))
                            ? APRIL_TRUE_HIT
                            : APRIL_INCONCLUSIVE;
                } else if (sx) {
                    v = host_join_ex(Ar, dr[1], sx, Fs, ds[3], 0, 0, &used) ? APRIL_TRUE_HIT : APRIL_INCONCLUSIVE;
                } else {
                    v = host_join_ex(Fr, dr[3], 0, As, ds[1], sy, 0, &used) ? APRIL_TRUE_HIT : APRIL_INCONCLUSIVE;
                }
            }
            verdict[k] = v;
            if (consumed) consumed[k] = used;
        }
    });
    return APRIL_OK;
}
