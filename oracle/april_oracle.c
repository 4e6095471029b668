/*
 * APRIL oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously-correct CPU statement of what the APRIL
 * intermediate filter computes.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may call this code; the product path never
 * does.  It shares no code with the CUDA path or its host-side builder.
 *
 * What it computes (paper, Sec. 4.1 "A- and F-interval lists", Table "APRIL:
 * do two objects intersect in a common cell?", and Algorithm 2 "APRIL join
 * algorithm" read as set operations):
 *
 *   P is a simple polygon taken as a closed region (interior + boundary);
 *   every grid cell c is a closed square.
 *     A(P) = { c : c meets P }          (Full or Partial cells)
 *     F(P) = { c : c is inside P }      (Full cells)
 *   verdict(r,s) = 0 (true negative)  if A(r) n A(s) is empty,
 *                  1 (true hit)       else if A(r) n F(s) or F(r) n A(s) is
 *                                     non-empty,
 *                  2 (inconclusive)   otherwise.
 *
 * The interval lists and the Hilbert order are only an encoding of these cell
 * sets, so the verdict here is computed with no curve at all.  The curve is
 * provided separately (oracle_hilbert_d) so that tests can compare a
 * builder's interval lists with the cell sets computed here.
 *
 * Cell classification, per cell of the polygon's MBR window, with exact
 * integer predicates (vertices are lattice points, the cell side h is an even
 * number of lattice units so cell centres are lattice points too):
 *   cross(c) = some polygon edge meets the OPEN square of c
 *   touch(c) = some polygon edge meets the CLOSED square of c
 *   inside(c)= the centre of c lies inside P (crossing-number test)
 *   class:  cross           -> A only
 *           !cross & inside -> A and F
 *           !cross & touch & !inside -> A only   (contact along the cell border)
 *           otherwise       -> empty
 * Justification: if the open square meets no boundary point it is connected
 * and lies entirely inside or entirely outside the open interior of P, so c
 * is inside P exactly when its centre is; and a cell meets P either through
 * the boundary (touch) or by lying inside.
 *
 * Cost: every edge tests every cell of its own bounding box, and the centre
 * test scans each window row against the edges that straddle that row's
 * centre line.  There is no further blocking or reordering.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define CLS_A 1u
#define CLS_F 2u

static int64_t floordiv(int64_t a, int64_t b) { /* b > 0 */
    int64_t q = a / b;
    if ((a % b) != 0 && (a < 0)) q -= 1;
    return q;
}
static int64_t ceildiv(int64_t a, int64_t b) { /* b > 0 */
    return -floordiv(-a, b);
}
static int64_t imin(int64_t a, int64_t b) { return a < b ? a : b; }
static int64_t imax(int64_t a, int64_t b) { return a > b ? a : b; }

/* Sign of the turn a->b->c. Coordinates are below 2^26 in magnitude. */
static int64_t orient(int64_t ax, int64_t ay, int64_t bx, int64_t by, int64_t cx, int64_t cy) {
    return (bx - ax) * (cy - ay) - (by - ay) * (cx - ax);
}

/* Does the closed segment ab meet the closed box [x0,x1]x[y0,y1]?
 * Separating-axis test: two convex sets are disjoint iff they are strictly
 * separated along an axis of the box or the normal of the segment. */
static int seg_meets_closed_box(int64_t ax, int64_t ay, int64_t bx, int64_t by,
                                int64_t x0, int64_t y0, int64_t x1, int64_t y1) {
    if (imax(ax, bx) < x0 || imin(ax, bx) > x1) return 0;
    if (imax(ay, by) < y0 || imin(ay, by) > y1) return 0;
    int64_t o1 = orient(ax, ay, bx, by, x0, y0);
    int64_t o2 = orient(ax, ay, bx, by, x1, y0);
    int64_t o3 = orient(ax, ay, bx, by, x1, y1);
    int64_t o4 = orient(ax, ay, bx, by, x0, y1);
    if (o1 > 0 && o2 > 0 && o3 > 0 && o4 > 0) return 0;
    if (o1 < 0 && o2 < 0 && o3 < 0 && o4 < 0) return 0;
    return 1;
}

/* Does the closed segment ab meet the OPEN box (x0,x1)x(y0,y1)?
 * An open convex set and a closed one are disjoint iff they are weakly
 * separated (closed half-planes) along one of the same candidate axes. */
static int seg_meets_open_box(int64_t ax, int64_t ay, int64_t bx, int64_t by,
                              int64_t x0, int64_t y0, int64_t x1, int64_t y1) {
    if (imax(ax, bx) <= x0 || imin(ax, bx) >= x1) return 0;
    if (imax(ay, by) <= y0 || imin(ay, by) >= y1) return 0;
    int64_t o1 = orient(ax, ay, bx, by, x0, y0);
    int64_t o2 = orient(ax, ay, bx, by, x1, y0);
    int64_t o3 = orient(ax, ay, bx, by, x1, y1);
    int64_t o4 = orient(ax, ay, bx, by, x0, y1);
    if (o1 >= 0 && o2 >= 0 && o3 >= 0 && o4 >= 0) return 0;
    if (o1 <= 0 && o2 <= 0 && o3 <= 0 && o4 <= 0) return 0;
    return 1;
}

/* Range of cell indices whose closed cells [o+i*h, o+(i+1)*h] meet the closed
 * coordinate range [lo, hi], clamped to [0, G-1]. Returns 0 if empty. */
static int cell_range(int64_t lo, int64_t hi, int64_t o, int64_t h, int64_t G, int64_t *i0, int64_t *i1) {
    int64_t a = ceildiv(lo - o, h) - 1;
    int64_t b = floordiv(hi - o, h);
    a = imax(a, 0);
    b = imin(b, G - 1);
    *i0 = a;
    *i1 = b;
    return a <= b;
}

/* Window of cells that can meet the polygon: the cells meeting its MBR.
 * win = {i0, j0, i1, j1}. Returns the number of cells (0 if none). */
int64_t oracle_window(const int64_t *xy, int64_t nv, int64_t ox, int64_t oy, int64_t h, int64_t G,
                      int64_t *win) {
    if (nv < 3) return 0;
    int64_t xmn = xy[0], xmx = xy[0], ymn = xy[1], ymx = xy[1];
    for (int64_t k = 1; k < nv; k++) {
        xmn = imin(xmn, xy[2 * k]);
        xmx = imax(xmx, xy[2 * k]);
        ymn = imin(ymn, xy[2 * k + 1]);
        ymx = imax(ymx, xy[2 * k + 1]);
    }
    if (!cell_range(xmn, xmx, ox, h, G, &win[0], &win[2])) return 0;
    if (!cell_range(ymn, ymx, oy, h, G, &win[1], &win[3])) return 0;
    return (win[2] - win[0] + 1) * (win[3] - win[1] + 1);
}

/* Classify every cell of the window (row-major, j outer): cls |= CLS_A, CLS_F.
 * Returns 0 on success, -1 if a cell centre lies on an edge that does not
 * cross that cell's open square (impossible for a valid input), -2 on
 * allocation failure. */
int oracle_classify(const int64_t *xy, int64_t nv, int64_t ox, int64_t oy, int64_t h, int64_t G,
                    const int64_t *win, uint8_t *cls) {
    int64_t i0 = win[0], j0 = win[1], i1 = win[2], j1 = win[3];
    int64_t W = i1 - i0 + 1, H = j1 - j0 + 1;
    uint8_t *touch = (uint8_t *)calloc((size_t)(W * H), 1);
    uint8_t *cross = (uint8_t *)calloc((size_t)(W * H), 1);
    int64_t *row_edges = (int64_t *)malloc(sizeof(int64_t) * (size_t)nv);
    if (!touch || !cross || !row_edges) {
        free(touch); free(cross); free(row_edges);
        return -2;
    }
    /* boundary predicates: every edge against every cell of its bounding box */
    for (int64_t k = 0; k < nv; k++) {
        int64_t ax = xy[2 * k], ay = xy[2 * k + 1];
        int64_t kn = (k + 1) % nv;
        int64_t bx = xy[2 * kn], by = xy[2 * kn + 1];
        int64_t ei0, ei1, ej0, ej1;
        if (!cell_range(imin(ax, bx), imax(ax, bx), ox, h, G, &ei0, &ei1)) continue;
        if (!cell_range(imin(ay, by), imax(ay, by), oy, h, G, &ej0, &ej1)) continue;
        for (int64_t j = ej0; j <= ej1; j++) {
            for (int64_t i = ei0; i <= ei1; i++) {
                int64_t cx0 = ox + i * h, cy0 = oy + j * h;
                int64_t cx1 = cx0 + h, cy1 = cy0 + h;
                int64_t idx = (j - j0) * W + (i - i0);
                if (seg_meets_closed_box(ax, ay, bx, by, cx0, cy0, cx1, cy1)) touch[idx] = 1;
                if (seg_meets_open_box(ax, ay, bx, by, cx0, cy0, cx1, cy1)) cross[idx] = 1;
            }
        }
    }
    int rc = 0;
    /* centre-in-polygon by crossing number along the ray to +x */
    for (int64_t j = j0; j <= j1 && rc == 0; j++) {
        int64_t yc = oy + j * h + h / 2;
        int64_t ne = 0;
        for (int64_t k = 0; k < nv; k++) {
            int64_t ay = xy[2 * k + 1];
            int64_t by = xy[2 * ((k + 1) % nv) + 1];
            if ((ay > yc) != (by > yc)) row_edges[ne++] = k;
        }
        for (int64_t i = i0; i <= i1; i++) {
            int64_t idx = (j - j0) * W + (i - i0);
            uint8_t c = 0;
            if (cross[idx]) {
                c = CLS_A;
            } else {
                int64_t xc = ox + i * h + h / 2;
                int inside = 0;
                for (int64_t e = 0; e < ne; e++) {
                    int64_t k = row_edges[e];
                    int64_t kn = (k + 1) % nv;
                    int64_t ax = xy[2 * k], ay = xy[2 * k + 1];
                    int64_t bx = xy[2 * kn], by = xy[2 * kn + 1];
                    if (ay > by) { /* orient the edge upwards */
                        int64_t t;
                        t = ax; ax = bx; bx = t;
                        t = ay; ay = by; by = t;
                    }
                    int64_t o = orient(ax, ay, bx, by, xc, yc);
                    if (o == 0) { rc = -1; break; }
                    if (o > 0) inside ^= 1; /* centre left of an upward edge: crossing to its right */
                }
                if (inside) c = CLS_A | CLS_F;
                else if (touch[idx]) c = CLS_A;
            }
            cls[idx] = c;
        }
    }
    free(touch); free(cross); free(row_edges);
    return rc;
}

typedef struct {
    int64_t win[4];
    uint8_t *cls;
    int64_t id;
} raster_t;

static int make_raster(const int64_t *xy, int64_t nv, int64_t ox, int64_t oy, int64_t h, int64_t G,
                       raster_t *r) {
    int64_t n = oracle_window(xy, nv, ox, oy, h, G, r->win);
    r->cls = NULL;
    if (n <= 0) return -3;
    r->cls = (uint8_t *)malloc((size_t)n);
    if (!r->cls) return -2;
    return oracle_classify(xy, nv, ox, oy, h, G, r->win, r->cls);
}

/* Verdict of one pair from two rasters on the same grid (Algorithm 2 as set
 * operations): scan the common window for A&A, A&F, F&A cells. */
static uint8_t pair_verdict(const raster_t *r, const raster_t *s) {
    int64_t i0 = imax(r->win[0], s->win[0]), i1 = imin(r->win[2], s->win[2]);
    int64_t j0 = imax(r->win[1], s->win[1]), j1 = imin(r->win[3], s->win[3]);
    int aa = 0, af = 0, fa = 0;
    int64_t rw = r->win[2] - r->win[0] + 1, sw = s->win[2] - s->win[0] + 1;
    for (int64_t j = j0; j <= j1; j++) {
        for (int64_t i = i0; i <= i1; i++) {
            uint8_t cr = r->cls[(j - r->win[1]) * rw + (i - r->win[0])];
            uint8_t cs = s->cls[(j - s->win[1]) * sw + (i - s->win[0])];
            if ((cr & CLS_A) && (cs & CLS_A)) aa = 1;
            if ((cr & CLS_A) && (cs & CLS_F)) af = 1;
            if ((cr & CLS_F) && (cs & CLS_A)) fa = 1;
        }
    }
    if (!aa) return 0;
    if (af || fa) return 1;
    return 2;
}

/* Verdicts of candidate pairs (pr[k], ps[k]) on one grid (origin ox,oy; cell
 * side h; G cells per side).  Polygon p of R has vertices
 * rxy[2*roff[p] .. 2*roff[p+1]); same for S.  Rasters are rebuilt per pair,
 * except that the last raster of each side is kept for reuse.
 * Returns 0, or a negative code from the classification. */
int oracle_verdicts(const int64_t *rxy, const int64_t *roff, const int64_t *sxy, const int64_t *soff,
                    const uint32_t *pr, const uint32_t *ps, int64_t npairs,
                    int64_t ox, int64_t oy, int64_t h, int64_t G, uint8_t *out) {
    raster_t rr = {{0, 0, 0, 0}, NULL, -1}, sr = {{0, 0, 0, 0}, NULL, -1};
    int rc = 0;
    for (int64_t k = 0; k < npairs && rc == 0; k++) {
        int64_t r = pr[k], s = ps[k];
        if (rr.id != r) {
            free(rr.cls);
            rr.id = r;
            rc = make_raster(rxy + 2 * roff[r], roff[r + 1] - roff[r], ox, oy, h, G, &rr);
            if (rc) break;
        }
        if (sr.id != s) {
            free(sr.cls);
            sr.id = s;
            rc = make_raster(sxy + 2 * soff[s], soff[s + 1] - soff[s], ox, oy, h, G, &sr);
            if (rc) break;
        }
        out[k] = pair_verdict(&rr, &sr);
    }
    free(rr.cls);
    free(sr.cls);
    return rc;
}

/* Hilbert index of cell (x, y) on a 2^order x 2^order grid.
 *
 * Curve (the paper only says "Hilbert curve", Sec. 3.2): the order-1 curve
 * visits (0,0), (0,1), (1,1), (1,0); the order-k curve is four order-(k-1)
 * curves placed in the quadrants in that same order, the lower-left one
 * reflected in the diagonal x=y and the lower-right one reflected in the
 * anti-diagonal, so that the curve always starts at (0,0) and ends at
 * (2^k - 1, 0).  The loop descends one level per iteration: it adds the
 * quadrant's rank times the quadrant's cell count, then rewrites (x, y) in
 * the quadrant's own frame. */
uint64_t oracle_hilbert_d(int order, uint64_t x, uint64_t y) {
    uint64_t d = 0;
    for (int k = order; k >= 1; k--) {
        uint64_t s = (uint64_t)1 << (k - 1);
        int rx = x >= s, ry = y >= s;
        uint64_t q;
        if (!rx && !ry) q = 0;
        else if (!rx && ry) q = 1;
        else if (rx && ry) q = 2;
        else q = 3;
        d += q * s * s;
        uint64_t lx = x - (rx ? s : 0), ly = y - (ry ? s : 0);
        if (q == 0) {          /* reflected in x = y */
            x = ly; y = lx;
        } else if (q == 3) {   /* reflected in the anti-diagonal */
            x = s - 1 - ly; y = s - 1 - lx;
        } else {
            x = lx; y = ly;
        }
    }
    return d;
}

void oracle_hilbert_many(int order, const int64_t *x, const int64_t *y, int64_t n, uint64_t *d) {
    for (int64_t k = 0; k < n; k++) d[k] = oracle_hilbert_d(order, (uint64_t)x[k], (uint64_t)y[k]);
}

/* ------------------------------------------------------------------------
 * Variants of the filter (paper Sec. 4.3.2 within joins, Sec. 5.3 different
 * granularity), as set operations on rasters.
 *
 * within (pred = 1, one grid):
 *   verdict = 0 if A(r) n A(s) is empty (disjoint: not within),
 *             1 if every cell of A(r) is in F(s) (r lies inside s),
 *             2 otherwise.
 * intersects on two grids of the same data space (pred = 0), the finer one
 * 2^k times finer per axis: let A'(p) be the coarse cells that contain a
 * fine A-cell of the finer polygon p.  With r the finer polygon:
 *   verdict = 0 if A'(r) n A(s) is empty, 1 if A'(r) n F(s) is not empty,
 *             2 otherwise
 * (only the coarse polygon's F-list is used); symmetrically when s is finer.
 * ------------------------------------------------------------------------ */

/* Coarse cell window and bitmap (1 = A') of a polygon rasterised on the fine
 * grid (ox, oy, hf, Gf) and mapped k levels up. */
static int coarse_a(const raster_t *fine, int k, int64_t *cwin, uint8_t **bits) {
    cwin[0] = fine->win[0] >> k;
    cwin[1] = fine->win[1] >> k;
    cwin[2] = fine->win[2] >> k;
    cwin[3] = fine->win[3] >> k;
    int64_t W = cwin[2] - cwin[0] + 1, H = cwin[3] - cwin[1] + 1;
    *bits = (uint8_t *)calloc((size_t)(W * H), 1);
    if (!*bits) return -2;
    int64_t fw = fine->win[2] - fine->win[0] + 1;
    for (int64_t j = fine->win[1]; j <= fine->win[3]; j++)
        for (int64_t i = fine->win[0]; i <= fine->win[2]; i++)
            if (fine->cls[(j - fine->win[1]) * fw + (i - fine->win[0])] & CLS_A)
                (*bits)[((j >> k) - cwin[1]) * W + ((i >> k) - cwin[0])] = 1;
    return 0;
}

static uint8_t cls_at(const raster_t *r, int64_t i, int64_t j) {
    if (i < r->win[0] || i > r->win[2] || j < r->win[1] || j > r->win[3]) return 0;
    return r->cls[(j - r->win[1]) * (r->win[2] - r->win[0] + 1) + (i - r->win[0])];
}

int oracle_verdicts_ex(const int64_t *rxy, const int64_t *roff, const int64_t *sxy, const int64_t *soff,
                       const uint32_t *pr, const uint32_t *ps, int64_t npairs, int64_t ox, int64_t oy,
                       int64_t hr, int64_t Gr, int64_t hs, int64_t Gs, int pred, uint8_t *out) {
    if (hr * Gr != hs * Gs) return -4;
    if (pred == 1 && hr != hs) return -4;
    raster_t rr = {{0, 0, 0, 0}, NULL, -1}, sr = {{0, 0, 0, 0}, NULL, -1};
    int rc = 0;
    for (int64_t k = 0; k < npairs && rc == 0; k++) {
        int64_t r = pr[k], s = ps[k];
        if (rr.id != r) {
            free(rr.cls);
            rr.id = r;
            rc = make_raster(rxy + 2 * roff[r], roff[r + 1] - roff[r], ox, oy, hr, Gr, &rr);
            if (rc) break;
        }
        if (sr.id != s) {
            free(sr.cls);
            sr.id = s;
            rc = make_raster(sxy + 2 * soff[s], soff[s + 1] - soff[s], ox, oy, hs, Gs, &sr);
            if (rc) break;
        }
        uint8_t v = 2;
        if (pred == 1) {
            int aa = 0, all_in = 1;
            int64_t rw = rr.win[2] - rr.win[0] + 1;
            for (int64_t j = rr.win[1]; j <= rr.win[3]; j++)
                for (int64_t i = rr.win[0]; i <= rr.win[2]; i++) {
                    if (!(rr.cls[(j - rr.win[1]) * rw + (i - rr.win[0])] & CLS_A)) continue;
                    uint8_t c = cls_at(&sr, i, j);
                    if (c & CLS_A) aa = 1;
                    if (!(c & CLS_F)) all_in = 0;
                }
            v = !aa ? 0 : (all_in ? 1 : 2);
        } else if (hr == hs) {
            v = pair_verdict(&rr, &sr);
        } else {
            /* the finer polygon's A-cells lifted to the coarse grid */
            const raster_t *fine = hr < hs ? &rr : &sr, *coarse = hr < hs ? &sr : &rr;
            int lv = 0;
            while ((hr < hs ? hr : hs) << lv < (hr < hs ? hs : hr)) lv++;
            int64_t cw[4];
            uint8_t *bits = NULL;
            rc = coarse_a(fine, lv, cw, &bits);
            if (rc == 0) {
                int aa = 0, th = 0;
                int64_t W = cw[2] - cw[0] + 1;
                for (int64_t j = cw[1]; j <= cw[3]; j++)
                    for (int64_t i = cw[0]; i <= cw[2]; i++) {
                        if (!bits[(j - cw[1]) * W + (i - cw[0])]) continue;
                        uint8_t c = cls_at(coarse, i, j);
                        if (c & CLS_A) aa = 1;
                        if (c & CLS_F) th = 1;
                    }
                v = !aa ? 0 : (th ? 1 : 2);
            }
            free(bits);
        }
        out[k] = v;
    }
    free(rr.cls);
    free(sr.cls);
    return rc;
}
