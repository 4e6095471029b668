"""Exact brute-force geometry for tiny inputs, independent of the oracle.

Everything here is written directly from textbook definitions with Python
integers and Fractions:

* closed-segment intersection by orientation tests with the collinear case;
* point-in-or-on-polygon by the winding number plus an on-edge test;
* polygon/polygon intersection of closed simple polygons: their boundaries
  meet, or one contains a vertex of the other;
* convex-polygon / closed-box intersection by the separating-axis theorem;
* area of (convex polygon n box) by Sutherland-Hodgman clipping and the
  shoelace formula, in exact rationals.

A star-shaped polygon is the union of the fan triangles (centre, v_k,
v_{k+1}), which overlap only on their borders, so for a closed cell c:
  c meets P      <=> c meets some fan triangle
  area(c n P)    =  sum over k of area(c n T_k)
and "c is Full" (coverage 100%, paper Sec. 4.1) <=> area(c n P) == area(c).
"""
from __future__ import annotations

from fractions import Fraction


def orient(a, b, c) -> int:
    v = (b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0])
    return (v > 0) - (v < 0)


def _on_seg(a, b, p) -> bool:
    return (orient(a, b, p) == 0 and min(a[0], b[0]) <= p[0] <= max(a[0], b[0])
            and min(a[1], b[1]) <= p[1] <= max(a[1], b[1]))


def segs_intersect(a, b, c, d) -> bool:
    o1, o2, o3, o4 = orient(a, b, c), orient(a, b, d), orient(c, d, a), orient(c, d, b)
    if o1 != o2 and o3 != o4 and o1 * o2 <= 0 and o3 * o4 <= 0:
        if o1 != 0 or o2 != 0:
            return True
    return _on_seg(a, b, c) or _on_seg(a, b, d) or _on_seg(c, d, a) or _on_seg(c, d, b)


def point_in_or_on(p, poly) -> bool:
    n = len(poly)
    wn = 0
    for k in range(n):
        a, b = poly[k], poly[(k + 1) % n]
        if _on_seg(a, b, p):
            return True
        if a[1] <= p[1]:
            if b[1] > p[1] and orient(a, b, p) > 0:
                wn += 1
        else:
            if b[1] <= p[1] and orient(a, b, p) < 0:
                wn -= 1
    return wn != 0


def polygons_intersect(P, Q) -> bool:
    n, m = len(P), len(Q)
    for i in range(n):
        a, b = P[i], P[(i + 1) % n]
        for j in range(m):
            if segs_intersect(a, b, Q[j], Q[(j + 1) % m]):
                return True
    return point_in_or_on(P[0], Q) or point_in_or_on(Q[0], P)


def convex_meets_box(poly, x0, y0, x1, y1) -> bool:
    """Closed convex polygon (CCW or CW) vs closed box, by separating axes."""
    xs = [p[0] for p in poly]
    ys = [p[1] for p in poly]
    if max(xs) < x0 or min(xs) > x1 or max(ys) < y0 or min(ys) > y1:
        return False
    corners = [(x0, y0), (x1, y0), (x1, y1), (x0, y1)]
    n = len(poly)
    for k in range(n):
        a, b = poly[k], poly[(k + 1) % n]
        if a == b:
            continue
        # the polygon lies on one closed side of edge ab; if every corner is
        # strictly on the other side the two are separated
        side = 0
        for q in poly:
            o = orient(a, b, q)
            if o:
                side = o
                break
        if side == 0:
            continue
        if all(orient(a, b, c) == -side for c in corners):
            return False
    return True


def clip_area(poly, x0, y0, x1, y1) -> Fraction:
    """Exact area of (convex polygon n box)."""
    pts = [(Fraction(p[0]), Fraction(p[1])) for p in poly]

    def clip(pts, inside, inter):
        out = []
        n = len(pts)
        for k in range(n):
            cur, nxt = pts[k], pts[(k + 1) % n]
            ci, ni = inside(cur), inside(nxt)
            if ci:
                out.append(cur)
            if ci != ni:
                out.append(inter(cur, nxt))
        return out

    def ix(xv):
        def f(a, b):
            t = (xv - a[0]) / (b[0] - a[0])
            return (Fraction(xv), a[1] + t * (b[1] - a[1]))
        return f

    def iy(yv):
        def f(a, b):
            t = (yv - a[1]) / (b[1] - a[1])
            return (a[0] + t * (b[0] - a[0]), Fraction(yv))
        return f

    for inside, inter in ((lambda p: p[0] >= x0, ix(x0)), (lambda p: p[0] <= x1, ix(x1)),
                          (lambda p: p[1] >= y0, iy(y0)), (lambda p: p[1] <= y1, iy(y1))):
        if not pts:
            return Fraction(0)
        pts = clip(pts, inside, inter)
    if len(pts) < 3:
        return Fraction(0)
    s = Fraction(0)
    for k in range(len(pts)):
        a, b = pts[k], pts[(k + 1) % len(pts)]
        s += a[0] * b[1] - a[1] * b[0]
    return abs(s) / 2


def fan(poly, center):
    n = len(poly)
    return [(tuple(center), tuple(poly[k]), tuple(poly[(k + 1) % n])) for k in range(n)]


def brute_cells(poly, center, ox, oy, h, G):
    """(A, F) cell sets of a star polygon by fan triangles: A = cells meeting
    some triangle, F = cells whose covered area equals h^2."""
    poly = [tuple(int(v) for v in p) for p in poly]
    tris = fan(poly, center)
    xs = [p[0] for p in poly]
    ys = [p[1] for p in poly]
    A, F = set(), set()
    i0 = max((min(xs) - ox) // h - 1, 0)
    i1 = min((max(xs) - ox) // h, G - 1)
    j0 = max((min(ys) - oy) // h - 1, 0)
    j1 = min((max(ys) - oy) // h, G - 1)
    for j in range(j0, j1 + 1):
        for i in range(i0, i1 + 1):
            bx0, by0 = ox + i * h, oy + j * h
            bx1, by1 = bx0 + h, by0 + h
            hit = [t for t in tris if convex_meets_box(t, bx0, by0, bx1, by1)]
            if not hit:
                continue
            A.add((i, j))
            area = sum((clip_area(t, bx0, by0, bx1, by1) for t in hit), Fraction(0))
            if area == h * h:
                F.add((i, j))
    return A, F
