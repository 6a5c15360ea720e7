"""Jittered periodic channel mesh, [0, 2*pi] x [-1, 1].

The paper's channel (ch. 4) and canyon/cylinder meshes come from Gmsh and from
data that is not available here; this generator stands in for them with the
per-element particle densities the paper uses (50-500 particles per element).

Layout:
  * node (i, j), i = 0..nx-1 along x, j = 0..ny-1 along y, id n = j*nx + i;
    x_i = 2*pi*i/(nx-1), y_j = -1 + 2*j/(ny-1).  Column i = nx-1 sits exactly
    at x = period and is the periodic twin of column i = 0.
  * jitter (seeded numpy PCG64): interior nodes move by (2u-1)*0.2*spacing in
    both axes; wall nodes (j = 0, ny-1) in x only; the two seam columns in y
    only, with the same draw for both twins (keyed by j); corners are fixed.
  * quad q = j*(nx-1) + i is split along its shorter diagonal (tie: the
    (i,j)-(i+1,j+1) diagonal) into triangles 2q and 2q+1, both counter-clockwise.
  * boundary edges carry a tag: TAG_WALL on y = -1 and y = +1 (wall_tag
    overrides it), TAG_PERIODIC on the two seams, or with inout=True
    TAG_INFLOW at x = 0 and TAG_OUTFLOW at x = period (the twins then pair
    the two ends for the particles, and the mean pressure takes the
    inflow/outflow condition).
"""
import numpy as np

TAG_WALL = 1
TAG_PERIODIC = 2
TAG_INFLOW = 3
TAG_OUTFLOW = 4
TAG_NOSLIP = 5


def channel_mesh(nx, ny, jitter=0.2, seed=1, period=2.0 * np.pi, y0=-1.0, y1=1.0, wall_tag=None, inout=False):
    if nx < 3 or ny < 2:
        raise ValueError("channel_mesh needs nx >= 3 and ny >= 2")
    dx = period / (nx - 1)
    dy = (y1 - y0) / (ny - 1)
    ii, jj = np.meshgrid(np.arange(nx), np.arange(ny))  # [ny, nx]
    x = ii * dx
    y = y0 + jj * dy
    x[:, 0] = 0.0
    x[:, nx - 1] = period
    y[0, :] = y0
    y[ny - 1, :] = y1
    rng = np.random.default_rng(seed)
    # one draw per node and axis, in node-id order, so the mesh depends only on (nx, ny, seed)
    ux = rng.random((ny, nx))
    uy = rng.random((ny, nx))
    jx = (2.0 * ux - 1.0) * jitter * dx
    jy = (2.0 * uy - 1.0) * jitter * dy
    interior = (ii > 0) & (ii < nx - 1) & (jj > 0) & (jj < ny - 1)
    wall = ((jj == 0) | (jj == ny - 1)) & (ii > 0) & (ii < nx - 1)
    seam = ((ii == 0) | (ii == nx - 1)) & (jj > 0) & (jj < ny - 1)
    x = np.where(interior | wall, x + jx, x)
    # the seam twins share the draw of column 0
    jy_seam = np.broadcast_to(jy[:, :1], jy.shape)
    y = np.where(interior, y + jy, y)
    y = np.where(seam, y + jy_seam, y)
    xy = np.stack([x.ravel(), y.ravel()], axis=1).astype(np.float64)

    tri = np.empty((2 * (nx - 1) * (ny - 1), 3), dtype=np.int32)
    for j in range(ny - 1):
        for i in range(nx - 1):
            q = j * (nx - 1) + i
            n00 = j * nx + i
            n10 = n00 + 1
            n01 = n00 + nx
            n11 = n01 + 1
            d1 = np.sum((xy[n00] - xy[n11]) ** 2)
            d2 = np.sum((xy[n10] - xy[n01]) ** 2)
            if d1 <= d2:
                tri[2 * q] = (n00, n10, n11)
                tri[2 * q + 1] = (n00, n11, n01)
            else:
                tri[2 * q] = (n00, n10, n01)
                tri[2 * q + 1] = (n10, n11, n01)

    twin = np.full(nx * ny, -1, dtype=np.int32)
    for j in range(ny):
        twin[j * nx] = j * nx + nx - 1
        twin[j * nx + nx - 1] = j * nx
    wtag = TAG_WALL if wall_tag is None else wall_tag
    bnd = []
    for i in range(nx - 1):
        bnd.append((i, i + 1, wtag))
        top = (ny - 1) * nx
        bnd.append((top + i, top + i + 1, wtag))
    left, right = (TAG_INFLOW, TAG_OUTFLOW) if inout else (TAG_PERIODIC, TAG_PERIODIC)
    for j in range(ny - 1):
        bnd.append((j * nx, (j + 1) * nx, left))
        bnd.append((j * nx + nx - 1, (j + 1) * nx + nx - 1, right))
    bnd = np.asarray(bnd, dtype=np.int32)
    return {
        "xy": np.ascontiguousarray(xy),
        "tri": np.ascontiguousarray(tri),
        "twin": twin,
        "bnd": bnd,
        "period": float(period),
        "nx": nx,
        "ny": ny,
    }


def scalar_slab(mesh, x0=0.5):
    """Initial scalar per element: 1.0 for elements touching the line x = x0
    (min node x <= x0 <= max node x), else 0.0."""
    xs = mesh["xy"][mesh["tri"], 0]
    return ((xs.min(axis=1) <= x0) & (xs.max(axis=1) >= x0)).astype(np.float64)
