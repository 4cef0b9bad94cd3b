"""Collision detection of Algorithm 1, step 4.1 (DetectCollisions), as brute force.

TEST INFRASTRUCTURE ONLY -- see the package docstring.  These are the
references for the library's device detectors: every proxy is tested against
every obstacle in plain Python loops over IEEE doubles, so a reader can check
each rule by eye.  The arithmetic that decides an integer (which obstacle is
nearest, whether a proxy is active) is written as separate multiplies and
adds in a fixed order, with no fused multiply-add, so that a device
implementation that follows the same order (and rounds each operation to
nearest) takes the same decision bit for bit.

Each function returns the active springs as scenes.Contacts-like arrays
(nodes, w, target, stiffness) with 4 slots (one proxy on one node) or 8
slots (two-sided: slots 0-3 the proxy, slots 4-7 the obstacle point,
negated), matching the penalty energy c/2 ||W x - t||^2 of Eqs. 6-8.

Readings (the paper detects against level sets of its anatomy, Section 5;
these synthetic obstacles stand in for them):
  * sphere: a proxy strictly inside a sphere, not at its centre, is pulled to
    its radial projection on the surface; of several spheres the deepest
    wins, the first one on ties;
  * nearest pair: a side-A node within `gap` of its nearest side-B node
    (first index on ties) gets a spring on x_a - x_b toward the separation
    gap * (x_a - x_b) / |x_a - x_b| (the direction frozen at detection);
  * point-triangle: a side-A node, against the side-B surface triangles that
    were at least `rest_min` away from it in the rest pose, takes the nearest
    triangle (first index on ties); if the closest point q on it is nearer
    than `gap`, the spring acts on d = x_a - q (q = the barycentric
    combination of the triangle's nodes) toward gap * u, frozen at
    detection: u is the unit vector from q to the node, turned to the
    triangle's front side (the side its winding's normal n points to; outward
    for outward-wound faces), or n itself if the node lies on the triangle.
    The node is pushed to distance gap from q on the front side.  For a node
    whose closest point lies on an edge or vertex shared by several
    triangles, u is the same whichever of them is taken.
"""
import math

import numpy as np


def _springs(rows, slots):
    k = len(rows)
    nodes = np.full((k, slots), -1, np.int32)
    w = np.zeros((k, slots))
    t = np.zeros((k, 3))
    c = np.zeros(k)
    for j, (nd, wt, tg, st) in enumerate(rows):
        for a, (ni, wi) in enumerate(zip(nd, wt)):
            if ni >= 0:
                nodes[j, a] = ni
                w[j, a] = wi
        t[j] = tg
        c[j] = st
    return nodes, w, t, c


def sphere_springs(proxies, x, spheres, stiffness):
    """Proxies inside rigid spheres [q] = (cx, cy, cz, r), projected radially
    onto the deepest sphere's surface.  Returns (nodes [k,4], w, target,
    stiffness, active proxy positions in `proxies`)."""
    rows, idx = [], []
    for j, p in enumerate(proxies):
        px, py, pz = (float(v) for v in x[p])
        best, depth = -1, 0.0
        for q, (cx, cy, cz, r) in enumerate(spheres):
            dx, dy, dz = px - float(cx), py - float(cy), pz - float(cz)
            d = math.sqrt((dx * dx + dy * dy) + dz * dz)
            if d < float(r) and d > 1e-12 and float(r) - d > depth:
                best, depth = q, float(r) - d
        if best < 0:
            continue
        cx, cy, cz, r = (float(v) for v in spheres[best])
        dx, dy, dz = px - cx, py - cy, pz - cz
        d = math.sqrt((dx * dx + dy * dy) + dz * dz)
        s = r / d
        rows.append(([int(p)], [1.0], (cx + s * dx, cy + s * dy, cz + s * dz), float(stiffness)))
        idx.append(j)
    return (*_springs(rows, 4), np.asarray(idx, np.int64))


def nearest_pair_springs(side_a, side_b, x, gap, stiffness):
    """Two-sided springs between each side-A node and its nearest side-B node
    closer than gap.  Returns (nodes [k,8], w, target, stiffness, active
    positions in side_a)."""
    rows, idx = [], []
    for j, a in enumerate(side_a):
        ax, ay, az = (float(v) for v in x[a])
        best, bi = 1e300, -1
        for q, b in enumerate(side_b):
            dx, dy, dz = ax - float(x[b, 0]), ay - float(x[b, 1]), az - float(x[b, 2])
            d2 = (dx * dx + dy * dy) + dz * dz
            if d2 < best:
                best, bi = d2, q
        if bi < 0:
            continue
        dist = math.sqrt(best)
        if not (dist < gap) or not (dist > 1e-12):
            continue
        b = int(side_b[bi])
        s = gap / dist
        dx, dy, dz = ax - float(x[b, 0]), ay - float(x[b, 1]), az - float(x[b, 2])
        rows.append(([int(a), -1, -1, -1, b], [1.0, 0.0, 0.0, 0.0, -1.0], (s * dx, s * dy, s * dz),
                     float(stiffness)))
        idx.append(j)
    return (*_springs(rows, 8), np.asarray(idx, np.int64))


def _sub(u, v):
    return (u[0] - v[0], u[1] - v[1], u[2] - v[2])


def _dot(u, v):
    return (u[0] * v[0] + u[1] * v[1]) + u[2] * v[2]


def closest_point_on_triangle(p, a, b, c):
    """Closest point q of the triangle (a, b, c) to p, as (dist^2, (wa, wb, wc), q)
    with q = wa a + wb b + wc c.  If the projection of p on the triangle's
    plane has barycentric coordinates in [0, 1] it is q; otherwise q lies on
    the boundary and is the nearest of the three segment projections (edges
    ab, bc, ca in that order, the first on ties).  A degenerate triangle
    (zero area) is treated through its edges."""
    e0, e1, w = _sub(b, a), _sub(c, a), _sub(p, a)
    d00, d01, d11 = _dot(e0, e0), _dot(e0, e1), _dot(e1, e1)
    d20, d21 = _dot(w, e0), _dot(w, e1)
    den = d00 * d11 - d01 * d01
    if den > 0.0:
        s = (d11 * d20 - d01 * d21) / den
        t = (d00 * d21 - d01 * d20) / den
        if s >= 0.0 and t >= 0.0 and s + t <= 1.0:
            q = (a[0] + s * e0[0] + t * e1[0], a[1] + s * e0[1] + t * e1[1], a[2] + s * e0[2] + t * e1[2])
            r = _sub(p, q)
            return _dot(r, r), (1.0 - s - t, s, t), q
    best, wts, bq = None, None, None
    for (u, v, iu, iv) in ((a, b, 0, 1), (b, c, 1, 2), (c, a, 2, 0)):
        e = _sub(v, u)
        ee = _dot(e, e)
        f = _dot(_sub(p, u), e) / ee if ee > 0.0 else 0.0
        f = 0.0 if f < 0.0 else (1.0 if f > 1.0 else f)
        q = (u[0] + f * e[0], u[1] + f * e[1], u[2] + f * e[2])
        r = _sub(p, q)
        d2 = _dot(r, r)
        if best is None or d2 < best:
            ww = [0.0, 0.0, 0.0]
            ww[iu] = 1.0 - f
            ww[iv] = f
            best, wts, bq = d2, tuple(ww), q
    return best, wts, bq


def _pt(x, i):
    return (float(x[i, 0]), float(x[i, 1]), float(x[i, 2]))


def point_triangle_springs(prox_a, tris_b, x, X, gap, rest_min, stiffness):
    """Side-A proxy nodes against side-B surface triangles [nt, 3] (node ids).
    A pair is a candidate if the node was at least rest_min from the triangle
    in the rest pose X; each node takes its nearest candidate triangle and is
    active if that is nearer than gap.  Returns (nodes [k,8], w, target,
    stiffness, active positions in prox_a, chosen triangle per active node)."""
    rows, idx, which = [], [], []
    rm2 = rest_min * rest_min
    # A triangle whose bounding sphere is farther than gap from the node
    # cannot be active; skipping it (with a relative margin for rounding)
    # leaves the choice unchanged: the nearest candidate is only used if it
    # is nearer than gap.
    tb = np.asarray(tris_b, dtype=np.int64).reshape(-1, 3)
    V = np.asarray(x, dtype=np.float64)[tb]                      # [nt, 3, 3]
    cen = V.mean(axis=1)
    rad = np.sqrt(((V - cen[:, None, :]) ** 2).sum(-1)).max(axis=1)
    for j, a in enumerate(prox_a):
        p, P = _pt(x, a), _pt(X, a)
        best, bi, bw, bq = 1e300, -1, None, None
        dc = np.sqrt(((cen - np.asarray(p)) ** 2).sum(-1))
        near = np.nonzero(dc <= (rad + gap) * (1.0 + 1e-9) + 1e-12)[0]
        for q in near:
            i0, i1, i2 = (int(v) for v in tb[q])
            d2r, _, _ = closest_point_on_triangle(P, _pt(X, i0), _pt(X, i1), _pt(X, i2))
            if d2r < rm2:
                continue
            d2, wts, qp = closest_point_on_triangle(p, _pt(x, i0), _pt(x, i1), _pt(x, i2))
            if d2 < best:
                best, bi, bw, bq = d2, int(q), wts, qp
        if bi < 0 or not (math.sqrt(best) < gap):
            continue
        i0, i1, i2 = (int(v) for v in tris_b[bi])
        A, B, C = _pt(x, i0), _pt(x, i1), _pt(x, i2)
        e0, e1 = _sub(B, A), _sub(C, A)
        n = (e0[1] * e1[2] - e0[2] * e1[1], e0[2] * e1[0] - e0[0] * e1[2], e0[0] * e1[1] - e0[1] * e1[0])
        r = _sub(p, bq)
        if best > 0.0:
            s = gap / math.sqrt(best)
            if _dot(r, n) < 0.0:
                s = -s
            tg = (s * r[0], s * r[1], s * r[2])
        else:
            nn = math.sqrt(_dot(n, n))
            if not (nn > 0.0):
                continue
            s = gap / nn
            tg = (s * n[0], s * n[1], s * n[2])
        rows.append(([int(a), -1, -1, -1, i0, i1, i2], [1.0, 0.0, 0.0, 0.0, -bw[0], -bw[1], -bw[2]], tg,
                     float(stiffness)))
        idx.append(j)
        which.append(bi)
    return (*_springs(rows, 8), np.asarray(idx, np.int64), np.asarray(which, np.int64))
