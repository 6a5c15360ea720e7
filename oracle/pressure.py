"""Oracle of the stabilised mean-pressure projection (TEST INFRASTRUCTURE ONLY).

Sec. 3.2 splits a step into the velocity prediction (eq. velocity-
prediction, the particle step), the projection

    (1/rho) lap(<P>^{n+1} - <P>^n) = (div <U*> - C_p (1/rho) lap <P>^n) / dt
                                                 (eq. pressure-projection-smooth)

and the correction <U>^{n+1} = <U*> - dt grad(<P>^{n+1} - <P>^n) (eq.
velocity-correction), applied to every particle.  rho = 1 (kinematic
pressure).  The equation is discretised with linear triangles (sec. 3.2: P1
finite elements).  Multiplying by N_a and integrating by parts,

    K dP = -(d + C_p (K P^n - G^n)) / dt + G^{n+1} - G^n,
    K_ab = int grad N_a . grad N_b,   d_a = int N_a div <U*>,
    G_a  = int_wall N_a h ds,

h the Neumann data of the pressure at solid walls (eq. wall-pressure-
condition, and in the wall-functions case the advection term of the
equation that follows it).

READINGS (the paper states the equations, not their discretisation):
  * G^n is the wall load the current <P'>^n was made with (0 at the start),
    G^{n+1} that of the statistics of U*; so <P'>^{n+1} satisfies the wall
    condition of the statistics it was made from and the C_p term carries
    the boundary integral of lap <P'>^n;
  * h per wall edge: the element's own gradients of the nodal <u_i u_j> and
    <U_i>, and the mean over the edge's two nodes of lap <U_i> and <U_j>;
    the load on each end is h |edge| / 2 (exact for h constant on the edge);
    WALL and NO-SLIP edges are both stationary solid walls; inflow and
    outflow edges get zero flux;
  * the wall-functions case is the SLM closure;
  * the pure-Neumann system is made solvable by removing the mean of the
    right-hand side over the unknowns, and dP is the zero-mean solution;
  * the correction uses the gradient of dP in the particle's element;
  * the pressure gradient the velocity prediction sees at a node is the mean
    of the gradients of the elements around it (the element-to-node transfer
    of sec. 3.3), periodic twins merged;
  * periodic twin nodes are one unknown;
  * with the street canyon's inflow/outflow condition (the section on the
    canyon's boundary conditions) the inflow and outflow twins are separate
    unknowns with the Dirichlet values dP = Pi L_x - <vv> - <P'>^n
    (inflow) and -<vv> - <P'>^n (outflow), Pi = -Delta P the imposed
    -d<P>/dx and L_x the x-period; the system is then regular (no mean
    removal, no normalisation) and the drift takes the whole gradient of
    the projected field (no separate Pi).
The linear system is solved by scipy's sparse direct solver (one unknown
pinned for the singular system); the oracle does not iterate.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

WALL_TAGS = (1, 5)  # WALL, NO-SLIP


def inout_nodes(mesh):
    """Per node: 1 on an INFLOW edge, 2 on an OUTFLOW edge, else 0."""
    io = np.zeros(len(mesh["xy"]), dtype=np.int64)
    for a, b, tag in mesh["bnd"]:
        if tag in (3, 4):
            io[a] = io[b] = 1 if tag == 3 else 2
    return io


def _rep(mesh, inout=False):
    """Representative node of every node: periodic twins merged (with
    inout=True, except the inflow/outflow pairs)."""
    n = len(mesh["xy"])
    rep = np.arange(n)
    twin = mesh.get("twin")
    if twin is not None:
        t = np.asarray(twin)
        m = t >= 0
        if inout:
            io = inout_nodes(mesh)
            m &= ~((io != 0) & (io[np.maximum(t, 0)] != 0))
        rep[m] = np.minimum(np.arange(n)[m], t[m])
    return rep


def shape_gradients(mesh):
    """Area [n_tri] and the gradients of N_0, N_1, N_2 [n_tri, 2, 3] (x row,
    y row) of every linear triangle."""
    xy, tri = mesh["xy"], mesh["tri"]
    P = xy[tri]                                   # [n_tri, 3, 2]
    x, y = P[:, :, 0], P[:, :, 1]
    twoA = (x[:, 1] - x[:, 0]) * (y[:, 2] - y[:, 0]) - (x[:, 2] - x[:, 0]) * (y[:, 1] - y[:, 0])
    # N_a = (alpha_a + beta_a x + gamma_a y) / 2A, beta_a = y_b - y_c, gamma_a = x_c - x_b
    # for (a, b, c) the cyclic orders of (0, 1, 2)
    gx = np.stack([y[:, 1] - y[:, 2], y[:, 2] - y[:, 0], y[:, 0] - y[:, 1]], axis=1) / twoA[:, None]
    gy = np.stack([x[:, 2] - x[:, 1], x[:, 0] - x[:, 2], x[:, 1] - x[:, 0]], axis=1) / twoA[:, None]
    return 0.5 * twoA, np.stack([gx, gy], axis=1)


def element_gradient(mesh, f):
    """Gradient [n_tri, 2] of the linear interpolant of the nodal field f."""
    _, g = shape_gradients(mesh)
    fv = np.asarray(f)[mesh["tri"]]               # [n_tri, 3]
    return np.einsum("eki,ei->ek", g, fv)


def stiffness(mesh, inout=False):
    """K over the unknowns (twins merged) as a sparse matrix indexed by node
    id (rows and columns of non-representative nodes are empty)."""
    A, g = shape_gradients(mesh)
    rep = _rep(mesh, inout)
    tri = mesh["tri"]
    n = len(mesh["xy"])
    rows, cols, vals = [], [], []
    for a in range(3):
        for b in range(3):
            rows.append(rep[tri[:, a]])
            cols.append(rep[tri[:, b]])
            vals.append(A * (g[:, 0, a] * g[:, 0, b] + g[:, 1, a] * g[:, 1, b]))
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))


def divergence_load(mesh, ns, inout=False):
    """d_a = int N_a div <U> [n_nodes] (on representative nodes), <U>, <V>
    the nodal means of node statistics ns: div is constant on an element and
    int_e N_a = A_e / 3."""
    A, _ = shape_gradients(mesh)
    div = element_gradient(mesh, ns[:, 0])[:, 0] + element_gradient(mesh, ns[:, 1])[:, 1]
    rep = _rep(mesh, inout)
    d = np.zeros(len(mesh["xy"]))
    for a in range(3):
        np.add.at(d, rep[mesh["tri"][:, a]], A * div / 3.0)
    return d


def wall_edges(mesh):
    """Solid wall edges: rows (a, b, element, nx, ny, length) with the unit
    normal pointing out of the domain (away from the element's third node)."""
    xy, tri, bnd = mesh["xy"], mesh["tri"], mesh["bnd"]
    out = []
    for a, b, tag in bnd:
        if tag not in WALL_TAGS:
            continue
        e = int(np.nonzero(np.sum((tri == a) | (tri == b), axis=1) == 2)[0][0])
        c = [v for v in tri[e] if v != a and v != b][0]
        t = xy[b] - xy[a]
        L = float(np.hypot(t[0], t[1]))
        nrm = np.array([t[1], -t[0]]) / L
        if np.dot(xy[c] - xy[a], nrm) > 0:
            nrm = -nrm
        out.append((int(a), int(b), e, nrm[0], nrm[1], L))
    return out


def wall_data(mesh, ns, nd, e, a, b, nu, slm):
    """h = (1/rho) d<P>/dn on a wall edge (a, b) of element e (eq. wall-
    pressure-condition; SLM: minus <U_j> d<U_i>/dx_j n_i as well), as the
    vector (h_x, h_y) to be dotted with the normal."""
    G = {k: element_gradient(mesh, ns[:, i])[e] for k, i in (("U", 0), ("V", 1), ("uu", 5), ("vv", 6), ("uv", 8))}
    lapU = 0.5 * (nd[a, 6] + nd[b, 6])
    lapV = 0.5 * (nd[a, 7] + nd[b, 7])
    # d<u_i u_j>/dx_j for i = x, y
    div_x = G["uu"][0] + G["uv"][1]
    div_y = G["uv"][0] + G["vv"][1]
    hx = nu * lapU - div_x
    hy = nu * lapV - div_y
    if slm:
        U = 0.5 * (ns[a, 0] + ns[b, 0])
        V = 0.5 * (ns[a, 1] + ns[b, 1])
        hx -= U * G["U"][0] + V * G["U"][1]
        hy -= U * G["V"][0] + V * G["V"][1]
    return hx, hy


def wall_load(mesh, ns, nd, nu, slm=False, inout=False):
    """G_a = int_wall N_a h ds [n_nodes] (on representative nodes)."""
    rep = _rep(mesh, inout)
    G = np.zeros(len(mesh["xy"]))
    for a, b, e, nx, ny, L in wall_edges(mesh):
        hx, hy = wall_data(mesh, ns, nd, e, a, b, nu, slm)
        h = hx * nx + hy * ny
        G[rep[a]] += 0.5 * h * L
        G[rep[b]] += 0.5 * h * L
    return G


def nodal_gradient(mesh, f):
    """Per node: the mean of the gradients of the elements around it and,
    for a periodic twin, around its twin [n_nodes, 2]."""
    ge = element_gradient(mesh, f)
    rep = _rep(mesh)
    n = len(mesh["xy"])
    s = np.zeros((n, 2))
    c = np.zeros(n)
    for a in range(3):
        np.add.at(s, rep[mesh["tri"][:, a]], ge)
        np.add.at(c, rep[mesh["tri"][:, a]], 1.0)
    return s[rep] / np.maximum(c[rep], 1.0)[:, None]


def solve_increment(mesh, ns, nd, pres, G_prev, nu, dt, Cp, slm=False, inout=False, Pi=0.0):
    """dP [n_nodes] and G^{n+1} [n_nodes]: zero mean over the unknowns for
    the periodic system; with inout=True the inflow/outflow Dirichlet
    values at those nodes."""
    n = len(mesh["xy"])
    rep = _rep(mesh, inout)
    idx = np.nonzero(rep == np.arange(n))[0]
    K = stiffness(mesh, inout)
    d = divergence_load(mesh, ns, inout)
    G = wall_load(mesh, ns, nd, nu, slm, inout)
    Pn = np.asarray(pres, dtype=np.float64)[rep]
    b = -(d + Cp * (K @ Pn - G_prev)) / dt + G - G_prev
    if not inout:
        b_u = b[idx]
        b_u = b_u - b_u.mean()
        Ku = K[idx][:, idx].tocsc()
        x = np.zeros(len(idx))
        x[1:] = spla.spsolve(Ku[1:, 1:], b_u[1:])   # unknown 0 pinned to 0
        x -= x.mean()
        full = np.zeros(n)
        full[idx] = x
        return full[rep], G
    io = inout_nodes(mesh)
    Lx = float(mesh["period"])
    g = np.where(io == 1, Pi * Lx, 0.0) - ns[:, 6] - np.asarray(pres, dtype=np.float64)
    D = idx[io[idx] != 0]
    F = idx[io[idx] == 0]
    Kc = K.tocsr()
    rhs = b[F] - Kc[F][:, D] @ g[D]
    full = np.zeros(n)
    full[F] = spla.spsolve(Kc[F][:, F].tocsc(), rhs)
    full[D] = g[D]
    G[D] = 0.0
    return full[rep], G


def project(mesh, ns, nd, st, pres, G_prev, nu, dt, Cp, slm=False, inout=False, Pi=0.0):
    """One projection after a predicted step: returns (dP, pres_new, G_new,
    gradP_nodal) and corrects the particle velocities st["u"], st["v"] in
    place (eq. velocity-correction)."""
    dP, G = solve_increment(mesh, ns, nd, pres, G_prev, nu, dt, Cp, slm, inout, Pi)
    ge = element_gradient(mesh, dP)
    el = st["elem"]
    st["u"] = st["u"] - dt * ge[el, 0]
    st["v"] = st["v"] - dt * ge[el, 1]
    pres_new = np.asarray(pres, dtype=np.float64) + dP
    return dP, pres_new, G, nodal_gradient(mesh, pres_new)
