// Exact integer geometry of APRIL construction, shared by the host builder
// (build_sets.cpp) and the GPU builder (build_device.cu) so that both emit
// the same cells: the Hilbert map of Sec. 3.2, the closed-cell predicates of
// the construction (Sec. 4.1 classes, Sec. 6.1 traversal) and the row
// ranges an edge meets.  Coordinates are lattice integers below 2^27 in
// magnitude, so every product here is exact in int64.
#pragma once
#include <cstdint>

#ifdef __CUDACC__
#define APRIL_HD __host__ __device__ __forceinline__
#else
#define APRIL_HD inline
#endif

namespace april_geom {

// ---------------------------------------------------------------- Hilbert
// The curve of Sec. 3.2 (orientation: the order-1 curve visits (0,0), (0,1),
// (1,1), (1,0)).  Walking down the levels, the sub-square the point lies in
// is traversed by the base curve under one of four symmetries of the square:
// identity I=0, transpose T=1 (x<->y), anti-transpose A=2 ((x,y) -> (~y,~x)
// per bit) and the half turn R=3 ((x,y) -> (~x,~y)).  Quadrant 0 of the base
// curve carries T, quadrant 3 carries A, quadrants 1 and 2 the identity.
// The four maps form a Klein group in which composing with T flips bit 0 of
// the code and composing with A flips bit 1.
APRIL_HD void apply_sym(uint32_t s, uint32_t &bx, uint32_t &by) {
    const uint32_t x = bx, y = by;
    switch (s) {
        case 0: break;
        case 1: bx = y; by = x; break;
        case 2: bx = y ^ 1u; by = x ^ 1u; break;
        default: bx = x ^ 1u; by = y ^ 1u; break;
    }
}

APRIL_HD uint64_t hilbert_id(uint32_t order, uint32_t x, uint32_t y) {
    uint32_t s = 0;
    uint64_t d = 0;
    for (int k = (int)order - 1; k >= 0; --k) {
        uint32_t bx = (x >> k) & 1u, by = (y >> k) & 1u;
        apply_sym(s, bx, by);
        const uint32_t digit = (bx << 1) | (bx ^ by);  // (0,0)->0 (0,1)->1 (1,1)->2 (1,0)->3
        d = (d << 2) | digit;
        if (digit == 0) s ^= 1u;
        else if (digit == 3) s ^= 2u;
    }
    return d;
}

APRIL_HD void hilbert_cell(uint32_t order, uint64_t d, uint32_t &x, uint32_t &y) {
    uint32_t s = 0;
    x = y = 0;
    for (int k = (int)order - 1; k >= 0; --k) {
        const uint32_t digit = (uint32_t)(d >> (2 * k)) & 3u;
        uint32_t bx = digit >> 1, by = (digit >> 1) ^ (digit & 1u);
        apply_sym(s, bx, by);  // every symmetry here is its own inverse
        x |= bx << k;
        y |= by << k;
        if (digit == 0) s ^= 1u;
        else if (digit == 3) s ^= 2u;
    }
}

// Two levels of the map at once: entry (s << 4) | (x2 << 2) | y2 of the
// table holds (the two base-4 digits << 2) | the next symmetry, for symmetry
// s and two bits x2, y2 of each coordinate (the higher level in bit 1).
APRIL_HD void hilbert_lut_build(uint8_t *lut) {
    for (uint32_t s = 0; s < 4; ++s)
        for (uint32_t x2 = 0; x2 < 4; ++x2)
            for (uint32_t y2 = 0; y2 < 4; ++y2) {
                uint32_t st = s, d = 0;
                for (int k = 1; k >= 0; --k) {
                    uint32_t bx = (x2 >> k) & 1u, by = (y2 >> k) & 1u;
                    apply_sym(st, bx, by);
                    const uint32_t digit = (bx << 1) | (bx ^ by);
                    d = (d << 2) | digit;
                    if (digit == 0) st ^= 1u;
                    else if (digit == 3) st ^= 2u;
                }
                lut[(s << 4) | (x2 << 2) | y2] = (uint8_t)((d << 2) | st);
            }
}

// hilbert_id by two levels a step through a table from hilbert_lut_build
// (an odd order takes its top level alone, from symmetry 0).
APRIL_HD uint64_t hilbert_id_lut(const uint8_t *lut, uint32_t order, uint32_t x, uint32_t y) {
    uint32_t s = 0;
    uint64_t d = 0;
    int k = (int)order - 2;
    if (order & 1u) {
        const uint32_t bx = (x >> (order - 1)) & 1u, by = (y >> (order - 1)) & 1u;
        const uint32_t digit = (bx << 1) | (bx ^ by);
        d = digit;
        s = digit == 0 ? 1u : digit == 3 ? 2u : 0u;
        k = (int)order - 3;
    }
    for (; k >= 0; k -= 2) {
        const uint32_t e = lut[(s << 4) | (((x >> k) & 3u) << 2) | ((y >> k) & 3u)];
        d = (d << 4) | (e >> 2);
        s = e & 3u;
    }
    return d;
}

// ------------------------------------------------------------- predicates
APRIL_HD int64_t imin(int64_t a, int64_t b) { return a < b ? a : b; }
APRIL_HD int64_t imax(int64_t a, int64_t b) { return a > b ? a : b; }

APRIL_HD int64_t floor_div(int64_t a, int64_t b) {  // b > 0
    const int64_t q = a / b;
    return (a % b != 0 && a < 0) ? q - 1 : q;
}
APRIL_HD int64_t ceil_div(int64_t a, int64_t b) { return -floor_div(-a, b); }

APRIL_HD int64_t turn(int64_t ax, int64_t ay, int64_t bx, int64_t by, int64_t px, int64_t py) {
    return (bx - ax) * (py - ay) - (by - ay) * (px - ax);
}

// Closed segment vs open square (x0,x0+h) x (y0,y0+h): they are disjoint iff
// weakly separated along x, along y, or along the segment's normal.
APRIL_HD bool enters_open_square(int64_t ax, int64_t ay, int64_t bx, int64_t by, int64_t x0, int64_t y0,
                                 int64_t h) {
    const int64_t x1 = x0 + h, y1 = y0 + h;
    if (imax(ax, bx) <= x0 || imin(ax, bx) >= x1) return false;
    if (imax(ay, by) <= y0 || imin(ay, by) >= y1) return false;
    const int64_t t0 = turn(ax, ay, bx, by, x0, y0), t1 = turn(ax, ay, bx, by, x1, y0);
    const int64_t t2 = turn(ax, ay, bx, by, x1, y1), t3 = turn(ax, ay, bx, by, x0, y1);
    const bool pos = t0 >= 0 && t1 >= 0 && t2 >= 0 && t3 >= 0;
    const bool neg = t0 <= 0 && t1 <= 0 && t2 <= 0 && t3 <= 0;
    return !(pos || neg);
}

// An edge oriented upwards (ay < by, or ay == by and ax <= bx).
struct EdgeUp {
    int64_t ax, ay, bx, by;
};

APRIL_HD EdgeUp edge_up(int64_t ax, int64_t ay, int64_t bx, int64_t by) {
    if (ay > by || (ay == by && ax > bx)) return EdgeUp{bx, by, ax, ay};
    return EdgeUp{ax, ay, bx, by};
}

// Cell rows [j0, j1] whose closed strip the edge's closed y-range meets.
APRIL_HD void edge_rows(const EdgeUp &e, int64_t oy, int64_t h, int64_t G, int64_t &j0, int64_t &j1) {
    j0 = imax(ceil_div(e.ay - oy, h) - 1, 0);
    j1 = imin(floor_div(e.by - oy, h), G - 1);
}

// Cells [i0, i1] of row j that the closed edge meets (exact: the edge's
// x-range inside the closed strip, computed in rationals scaled by the
// edge's height); false when the edge misses the strip.
APRIL_HD bool edge_cells_in_row(const EdgeUp &e, int64_t ox, int64_t oy, int64_t h, int64_t G, int64_t j,
                                int64_t &i0, int64_t &i1) {
    const int64_t Y0 = oy + j * h, Y1 = Y0 + h;
    const int64_t den = e.by - e.ay;  // >= 0
    if (den == 0) {
        if (e.ay < Y0 || e.ay > Y1) return false;  // a horizontal edge in this closed strip
        i0 = ceil_div(e.ax - ox, h) - 1;
        i1 = floor_div(e.bx - ox, h);
    } else {
        const int64_t ya = imax(e.ay, Y0), yb = imin(e.by, Y1);
        if (ya > yb) return false;
        const int64_t dx = e.bx - e.ax;
        const int64_t n1 = e.ax * den + (ya - e.ay) * dx;  // x(ya) * den
        const int64_t n2 = e.ax * den + (yb - e.ay) * dx;  // x(yb) * den
        const int64_t lo = imin(n1, n2) - ox * den, hi = imax(n1, n2) - ox * den;
        i0 = ceil_div(lo, den * h) - 1;
        i1 = floor_div(hi, den * h);
    }
    i0 = imax(i0, 0);
    i1 = imin(i1, G - 1);
    return i0 <= i1;
}

// Rows r in [wj0, wj1] whose centre line y = oy + r h + h/2 the edge crosses
// under the half-open rule ey0 <= y < ey1 (point-in-polygon buckets).
APRIL_HD void centre_rows(const EdgeUp &e, int64_t oy, int64_t h, int64_t wj0, int64_t wj1, int64_t &r0,
                          int64_t &r1) {
    r0 = imax(ceil_div(e.ay - oy - h / 2, h), wj0);
    r1 = imin(ceil_div(e.by - oy - h / 2, h) - 1, wj1);
}

// Window of cells meeting the closed MBR [xmn, xmx] x [ymn, ymx].
APRIL_HD void cell_window(int64_t xmn, int64_t ymn, int64_t xmx, int64_t ymx, int64_t ox, int64_t oy, int64_t h,
                          int64_t G, int64_t &wi0, int64_t &wj0, int64_t &wi1, int64_t &wj1) {
    wi0 = imax(ceil_div(xmn - ox, h) - 1, 0);
    wi1 = imin(floor_div(xmx - ox, h), G - 1);
    wj0 = imax(ceil_div(ymn - oy, h) - 1, 0);
    wj1 = imin(floor_div(ymx - oy, h), G - 1);
}

}  // namespace april_geom
