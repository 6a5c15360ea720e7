"""Oracle of the elliptic-relaxation solve (TEST INFRASTRUCTURE ONLY).

Eq. elliptic-relaxation-Lagrangian, wp_ij - L^2 lap wp_ij = rhs_ij, with the
lengthscale of Eq. L (anisotropic C_xi of Eq. Cxi), discretised with linear
triangles (sec. 3.2: P1 finite elements) as

    (M + K_L) wp = M rhs,
    M_ab   = sum_e A_e (1 + delta_ab) / 12          (consistent mass)
    K_L,ab = sum_e L2_e A_e grad N_a . grad N_b      (L2_e: mean of nodal L^2)

READINGS (the paper only says "P1 FEM, Jacobi-PCG, warm start"):
  * the term from grad(L^2) is dropped, matching the L^2 lap wp form (ch. 2);
  * reflecting walls are symmetry planes (as the channel centreline, sec.
    4.2.1): off-diagonal components Dirichlet 0 at wall nodes, diagonal
    components natural (Neumann) conditions;
  * no-slip walls take the Dirichlet condition wp_ij = -4.5 eps n_i n_j for
    every component (the section on no-slip wall-boundary conditions), eps of
    eq. dissipation-from-frequency_wall at the node; a node on both kinds of
    wall is a no-slip node;
  * C_xi = 1 + 1.3 n_i n_i for wp_ii, 1 for off-diagonal components, n the
    unit outward normal of the nearest wall edge;
  * periodic twin nodes are one unknown.
The linear system is solved by scipy's sparse direct solver (a library
primitive); the oracle does not iterate.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import NNS  # noqa: F401  (layout constants live in the package)

CL, CETA, CT = 0.134, 72.0, 6.0
KFLOOR = EFLOOR = 1e-12


def wall_normals(mesh):
    """Per node: distance to the nearest wall edge and that edge's unit
    outward normal (nx, ny).  Wall edges are the boundary edges tagged WALL
    or NOSLIP."""
    xy = mesh["xy"]
    bnd = mesh["bnd"]
    walls = bnd[(bnd[:, 2] == 1) | (bnd[:, 2] == 5)]
    a = xy[walls[:, 0]]
    b = xy[walls[:, 1]]
    # outward normal: the wall edge belongs to one triangle; the normal points
    # away from that triangle's third node
    tri = mesh["tri"]
    n_out = np.zeros((len(walls), 2))
    for i, (p, q, _) in enumerate(walls):
        t = np.nonzero(np.sum((tri == p) | (tri == q), axis=1) == 2)[0][0]
        c = [v for v in tri[t] if v != p and v != q][0]
        d = b[i] - a[i]
        nrm = np.array([d[1], -d[0]]) / np.hypot(d[0], d[1])
        if np.dot(xy[c] - a[i], nrm) > 0:
            nrm = -nrm
        n_out[i] = nrm
    dist = np.full(len(xy), np.inf)
    nn = np.zeros((len(xy), 2))
    for i in range(len(walls)):
        d = b[i] - a[i]
        t = np.clip(((xy - a[i]) @ d) / (d @ d), 0.0, 1.0)
        proj = a[i] + t[:, None] * d[None, :]
        di = np.hypot(*(xy - proj).T)
        better = di < dist
        dist[better] = di[better]
        nn[better] = n_out[i]
    return dist, nn


def lengthscale2(S, nu, cxi):
    """L^2 at nodes (Eq. L), S the node statistics [n, 12]."""
    k = np.maximum(0.5 * (S[:, 5] + S[:, 6] + S[:, 7]), KFLOOR)
    om = S[:, 3]
    eps = np.maximum(om * (k + nu * CT * CT * om), EFLOOR)
    L = CL * np.maximum(cxi * k ** 1.5 / eps, CETA * (nu ** 3 / eps) ** 0.25)
    return L * L


def _rep(mesh):
    n = len(mesh["xy"])
    twin = mesh.get("twin")
    rep = np.arange(n)
    if twin is not None:
        t = np.asarray(twin)
        m = t >= 0
        rep[m] = np.minimum(np.arange(n)[m], t[m])
    return rep


def assemble(mesh, L2_node):
    """Sparse (M, K_L) over representative nodes (twins merged)."""
    xy, tri = mesh["xy"], mesh["tri"]
    rep = _rep(mesh)
    n = len(xy)
    rows, cols, mv, kv = [], [], [], []
    for e, t in enumerate(tri):
        P = xy[t]
        twoA = (P[1, 0] - P[0, 0]) * (P[2, 1] - P[0, 1]) - (P[1, 1] - P[0, 1]) * (P[2, 0] - P[0, 0])
        A = 0.5 * twoA
        # shape-function derivatives (sec. 3.4)
        yCA, yBA = P[2, 1] - P[0, 1], P[1, 1] - P[0, 1]
        xCA, xBA = P[2, 0] - P[0, 0], P[1, 0] - P[0, 0]
        dx = np.array([-yCA + yBA, yCA, -yBA]) / twoA
        dy = np.array([xCA - xBA, -xCA, xBA]) / twoA
        L2e = np.mean(L2_node[t])
        for a in range(3):
            for b in range(3):
                rows.append(rep[t[a]])
                cols.append(rep[t[b]])
                mv.append(A * (2.0 if a == b else 1.0) / 12.0)
                kv.append(L2e * A * (dx[a] * dx[b] + dy[a] * dy[b]))
    M = sp.csr_matrix((mv, (rows, cols)), shape=(n, n))
    K = sp.csr_matrix((kv, (rows, cols)), shape=(n, n))
    return M, K


def wall_nodes(mesh, tag=1):
    bnd = mesh["bnd"]
    w = bnd[bnd[:, 2] == tag]
    if len(w) == 0:
        return np.zeros(0, dtype=np.int64)
    return np.unique(np.concatenate([w[:, 0], w[:, 1]]))


def noslip_values(S, nu, nrm):
    """Dirichlet values -4.5 eps n_i n_j [9, n] at every node."""
    k = np.maximum(0.5 * (S[:, 5] + S[:, 6] + S[:, 7]), KFLOOR)
    om = S[:, 3]
    eps = np.maximum(om * (k + nu * CT * CT * om), EFLOOR)
    n3 = np.stack([nrm[:, 0], nrm[:, 1], np.zeros(len(nrm))], axis=1)
    return np.stack([-4.5 * eps * n3[:, i] * n3[:, j] for i in range(3) for j in range(3)])


def _systems(mesh, S, rhs, nu):
    """The nine linear systems of eq. elliptic-relaxation-Lagrangian over the
    representative unknowns: for each component (ij, A, b, idx, rep) with
    the Dirichlet values lifted into b and the fixed rows and columns
    replaced by the identity."""
    n = len(mesh["xy"])
    rep = _rep(mesh)
    is_rep = rep == np.arange(n)
    _, nrm = wall_normals(mesh)
    noslip_rep = np.unique(rep[wall_nodes(mesh, 5)])
    free_rep = np.setdiff1d(np.unique(rep[wall_nodes(mesh, 1)]), noslip_rep)
    gval = noslip_values(S, nu, nrm)
    idx = np.nonzero(is_rep)[0]
    mats = {}  # the three L^2 classes: C_xi of wp_11, of wp_22, and 1
    for ij in range(9):
        i, j = divmod(ij, 3)
        cls = i if (i == j and i < 2) else 2
        if cls not in mats:
            cxi = 1.0 + 1.3 * nrm[:, cls] ** 2 if cls < 2 else np.ones(n)
            mats[cls] = assemble(mesh, lengthscale2(S, nu, cxi))
        M, K = mats[cls]
        A = (M + K).tocsr()
        fixed = noslip_rep if i == j else np.union1d(free_rep, noslip_rep)
        g = np.zeros(n)
        g[noslip_rep] = gval[ij][noslip_rep]
        b = M @ rhs[ij] - A @ g          # lift the Dirichlet values
        b[fixed] = g[fixed]
        mask = np.ones(n)
        mask[fixed] = 0.0
        D = sp.diags(mask)
        A = (D @ A @ D + sp.diags(1.0 - mask)).tocsr()
        yield ij, A[idx][:, idx], b[idx], idx, rep


def solve(mesh, S, rhs, nu):
    """wp [9, n_nodes] from node statistics S [n, 12] and the right-hand side
    rhs [9, n_nodes] (Eq. elliptic-relaxation-Lagrangian at the nodes)."""
    n = len(mesh["xy"])
    out = np.zeros((9, n))
    for ij, A, b, idx, rep in _systems(mesh, S, rhs, nu):
        x = spla.spsolve(A.tocsc(), b)
        full = np.zeros(n)
        full[idx] = x
        out[ij] = full[rep]
    return out


def residual(mesh, S, rhs, nu, wp):
    """Relative residual ||A x - b|| / ||b|| of a given solution wp [9, n]
    in each of the nine systems that solve() solves (a sparse product, no
    solve: usable at sizes where the direct solve is slow)."""
    out = np.zeros(9)
    for ij, A, b, idx, rep in _systems(mesh, S, rhs, nu):
        x = np.asarray(wp[ij], dtype=np.float64)[idx]
        nb = np.linalg.norm(b)
        out[ij] = np.linalg.norm(A @ x - b) / (nb if nb > 0 else 1.0)
    return out
