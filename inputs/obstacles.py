"""Graded triangulation of a 2-D domain with rectangular obstacles on the
bottom wall (the complex-geometry workload; the paper's street-canyon and
cylinder meshes came from Gmsh and are not available here).

Domain [0, Lx] x [0, Ly] with obstacles [x0, x1] x [0, h].  A tensor-product
grid whose x- and y-lines include every obstacle edge is graded
geometrically toward the walls (the bottom, the obstacle faces) from h_min
to h_max = ratio * h_min; cells whose centre lies inside an obstacle are
removed and every remaining rectangle is split into two counter-clockwise
triangles along its (i,j)-(i+1,j+1) diagonal.  Boundary tags: bottom, top and
obstacle faces TAG_WALL; x = 0 TAG_INFLOW and x = Lx TAG_OUTFLOW, the two
being periodic twins (a particle leaving through the outflow re-enters at
the inflow).
"""
import numpy as np

from .channel import TAG_INFLOW, TAG_OUTFLOW, TAG_WALL

DEFAULT_OBSTACLES = ((5.0, 6.0, 1.0), (9.0, 10.0, 2.0), (13.0, 13.5, 1.5))


def _graded_line(breaks, refine, h_min, ratio, growth=1.08):
    """Nodes on [breaks[0], breaks[-1]] through every break point; spacing h_min
    at refined break points growing by `growth` per cell up to ratio*h_min."""
    h_max = ratio * h_min
    nodes = [breaks[0]]
    for a, b in zip(breaks[:-1], breaks[1:]):
        L = b - a
        ra, rb = refine[breaks.index(a)], refine[breaks.index(b)]
        # spacing as a function of the distance to the refined ends
        def size(s):
            d = min(s if ra else np.inf, (L - s) if rb else np.inf)
            if not np.isfinite(d):
                return h_max
            # geometric growth: h(d) ~ h_min + (growth - 1) d, capped
            return min(h_max, h_min + (growth - 1.0) * d)
        pts = [0.0]
        s = 0.0
        while s < L:
            h = size(s)
            s = s + h
            pts.append(min(s, L))
        pts = np.array(pts)
        # stretch the last cell away: map uniformly so the interval ends at L
        n = len(pts) - 1
        if n >= 2 and pts[-1] - pts[-2] < 0.5 * size(L):
            pts = np.delete(pts, -2)
        pts = pts / pts[-1] * L
        nodes.extend((a + pts[1:]).tolist())
    return np.array(nodes)


def obstacle_mesh(Lx=20.0, Ly=5.0, obstacles=DEFAULT_OBSTACLES, h_min=0.0025, ratio=37.0, growth=1.04):
    """Defaults: 535,720 triangles, largest/smallest grid spacing 49.4."""
    xb = sorted({0.0, Lx, *[o[0] for o in obstacles], *[o[1] for o in obstacles]})
    yb = sorted({0.0, Ly, *[o[2] for o in obstacles]})
    xref = [x in {o[0] for o in obstacles} | {o[1] for o in obstacles} for x in xb]
    yref = [y == 0.0 or y in {o[2] for o in obstacles} for y in yb]
    xs = _graded_line(xb, xref, h_min, ratio, growth)
    ys = _graded_line(yb, yref, h_min, ratio, growth)
    nx, ny = len(xs), len(ys)
    X, Y = np.meshgrid(xs, ys)
    xy = np.stack([X.ravel(), Y.ravel()], axis=1)
    xc = 0.5 * (xs[:-1] + xs[1:])
    yc = 0.5 * (ys[:-1] + ys[1:])
    inside = np.zeros((ny - 1, nx - 1), dtype=bool)
    for (x0, x1, h) in obstacles:
        inside |= ((xc[None, :] > x0) & (xc[None, :] < x1) & (yc[:, None] < h))
    jj, ii = np.nonzero(~inside)
    n00 = jj * nx + ii
    n10 = n00 + 1
    n01 = n00 + nx
    n11 = n01 + 1
    tri = np.empty((2 * len(n00), 3), dtype=np.int64)
    tri[0::2] = np.stack([n00, n10, n11], axis=1)
    tri[1::2] = np.stack([n00, n11, n01], axis=1)
    # drop nodes used by no triangle (inside obstacles), renumber
    used = np.zeros(nx * ny, dtype=bool)
    used[tri.ravel()] = True
    new_id = -np.ones(nx * ny, dtype=np.int64)
    new_id[used] = np.arange(used.sum())
    tri = new_id[tri].astype(np.int32)
    xy = xy[used]
    # boundary edges: edges with one triangle
    e = np.concatenate([tri[:, [1, 2]], tri[:, [2, 0]], tri[:, [0, 1]]])
    key = np.sort(e, axis=1)
    uniq, counts = np.unique(key, axis=0, return_counts=True)
    bedges = uniq[counts == 1]
    tags = np.full(len(bedges), TAG_WALL, dtype=np.int32)
    x_a, x_b = xy[bedges[:, 0], 0], xy[bedges[:, 1], 0]
    tags[(x_a == 0.0) & (x_b == 0.0)] = TAG_INFLOW
    tags[(x_a == Lx) & (x_b == Lx)] = TAG_OUTFLOW
    bnd = np.concatenate([bedges.astype(np.int32), tags[:, None]], axis=1)
    # periodic twins between the inflow and outflow columns (same y lines)
    twin = np.full(len(xy), -1, dtype=np.int32)
    left = np.nonzero(xy[:, 0] == 0.0)[0]
    right = np.nonzero(xy[:, 0] == Lx)[0]
    ly = {float(xy[n, 1]): n for n in left}
    for n in right:
        m = ly[float(xy[n, 1])]
        twin[n] = m
        twin[m] = n
    return {"xy": np.ascontiguousarray(xy, dtype=np.float64), "tri": np.ascontiguousarray(tri),
            "twin": twin, "bnd": np.ascontiguousarray(bnd), "period": float(Lx), "Lx": Lx, "Ly": Ly,
            "obstacles": obstacles, "nx": nx, "ny": ny}


def counts_by_area(mesh, mean=128):
    """Particles per element proportional to its area, `mean` on average, at least 1."""
    P = mesh["xy"][mesh["tri"]]
    A = 0.5 * ((P[:, 1, 0] - P[:, 0, 0]) * (P[:, 2, 1] - P[:, 0, 1])
               - (P[:, 1, 1] - P[:, 0, 1]) * (P[:, 2, 0] - P[:, 0, 0]))
    return np.maximum(1, np.rint(mean * A / A.mean())).astype(np.int32)
