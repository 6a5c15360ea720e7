// Mesh upload: connectivity built on the host once, then copied to the device.
//
// Element-surrounding-element list with tagged boundary neighbours (sec. 3.5)
// and node-surrounding-element lists (sec. 3.3 linked lists), stored as CSR.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <unordered_map>

#include "common.cuh"

namespace pdfgb {

template <typename T>
static pdf_status upload(T** dst, const T* src, size_t n) {
  if (n == 0) { *dst = nullptr; return PDF_OK; }
  cudaError_t e = cudaMalloc((void**)dst, n * sizeof(T));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(mesh)");
  e = cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(mesh)");
  return PDF_OK;
}

static void free_relax(RelaxMesh& r) {
  cudaFree(r.rp); cudaFree(r.ci); cudaFree(r.mval); cudaFree(r.ctb_off); cudaFree(r.ctb_e); cudaFree(r.ctb_k);
  cudaFree(r.wall); cudaFree(r.rep_node); cudaFree(r.node_rep); cudaFree(r.wall_n); cudaFree(r.wall_d);
  cudaFree(r.pw_off); cudaFree(r.pw_e); cudaFree(r.pw_n);
  r = RelaxMesh();
}

// The relaxation system's structure: unknowns (twins merged), CSR pattern,
// consistent mass, per-entry stiffness contributions (element order), wall
// flags and the outward normal of the nearest wall edge at every node.
static pdf_status build_relax(pdf_mesh* m, const std::vector<int32_t>& bnd_wall, const std::vector<int32_t>& wall_tag,
                              const std::vector<double>& dN,
                              const std::vector<int32_t>& nse_off, const std::vector<int32_t>& nse,
                              const std::vector<int32_t>& esup_off, const std::vector<int32_t>& esup) {
  const int32_t nn = m->d.n_nodes, nt = m->d.n_tri;
  const int32_t* T = m->tri.data();
  const double* X = m->xy.data();
  std::vector<int32_t> node_rep(nn), rep_node;
  std::vector<int32_t> rep_of(nn);
  for (int32_t n = 0; n < nn; ++n) rep_of[n] = m->twin[n] >= 0 ? std::min(n, m->twin[n]) : n;
  std::vector<int32_t> idx(nn, -1);
  for (int32_t n = 0; n < nn; ++n)
    if (rep_of[n] == n) { idx[n] = (int32_t)rep_node.size(); rep_node.push_back(n); }
  for (int32_t n = 0; n < nn; ++n) node_rep[n] = idx[rep_of[n]];
  const int32_t nr = (int32_t)rep_node.size();
  // wall unknowns and the nearest wall edge of every node
  std::vector<uint8_t> wall(nr, 0);
  const size_t nw = bnd_wall.size() / 2;
  // 1: free-slip wall node (off-diagonal components 0); 2: no-slip wall node
  // (every component -4.5 eps n_i n_j), which wins where both meet
  for (size_t i = 0; i < nw; ++i) {
    const uint8_t t = wall_tag[i] == PDF_TAG_NOSLIP ? 2 : 1;
    for (int q = 0; q < 2; ++q) {
      uint8_t& w = wall[node_rep[bnd_wall[2 * i + q]]];
      w = std::max(w, t);
    }
  }
  std::vector<double> wn(2 * (size_t)nn, 0.0), wd(nn, 1e300);
  std::vector<double> en(2 * nw);
  for (size_t i = 0; i < nw; ++i) {
    const int32_t a = bnd_wall[2 * i], b = bnd_wall[2 * i + 1];
    const double tx = X[2 * b] - X[2 * a], ty = X[2 * b + 1] - X[2 * a + 1];
    const double len = std::sqrt(tx * tx + ty * ty);
    double nx = ty / len, ny = -tx / len;
    // point away from the element holding the edge
    for (int32_t q = esup_off[a]; q < esup_off[a + 1]; ++q) {
      const int32_t e = esup[q];
      const int32_t* t = T + 3 * e;
      const bool ha = t[0] == a || t[1] == a || t[2] == a, hb = t[0] == b || t[1] == b || t[2] == b;
      if (!(ha && hb)) continue;
      const int32_t c = (t[0] != a && t[0] != b) ? t[0] : ((t[1] != a && t[1] != b) ? t[1] : t[2]);
      if ((X[2 * c] - X[2 * a]) * nx + (X[2 * c + 1] - X[2 * a + 1]) * ny > 0.0) { nx = -nx; ny = -ny; }
      break;
    }
    en[2 * i] = nx; en[2 * i + 1] = ny;
  }
  for (int32_t n = 0; n < nn; ++n) {
    for (size_t i = 0; i < nw; ++i) {
      const int32_t a = bnd_wall[2 * i], b = bnd_wall[2 * i + 1];
      const double ax = X[2 * a], ay = X[2 * a + 1], dx = X[2 * b] - ax, dy = X[2 * b + 1] - ay;
      double t = ((X[2 * n] - ax) * dx + (X[2 * n + 1] - ay) * dy) / (dx * dx + dy * dy);
      t = std::min(1.0, std::max(0.0, t));
      const double px = ax + t * dx - X[2 * n], py = ay + t * dy - X[2 * n + 1];
      const double d = std::sqrt(px * px + py * py);
      if (d < wd[n]) { wd[n] = d; wn[2 * n] = en[2 * i]; wn[2 * n + 1] = en[2 * i + 1]; }
    }
    if (nw == 0) wd[n] = 0.0;
  }
  // CSR pattern: row u holds the unknowns of the elements around its node(s)
  std::vector<int32_t> rp(nr + 1, 0), ci;
  std::vector<std::vector<int32_t>> cols(nr);
  for (int32_t u = 0; u < nr; ++u) {
    const int32_t n = rep_node[u];
    std::vector<int32_t>& c = cols[u];
    for (int32_t i = nse_off[n]; i < nse_off[n + 1]; ++i)
      for (int k = 0; k < 3; ++k) c.push_back(node_rep[T[3 * nse[i] + k]]);
    std::sort(c.begin(), c.end());
    c.erase(std::unique(c.begin(), c.end()), c.end());
    rp[u + 1] = rp[u] + (int32_t)c.size();
  }
  const int64_t nnz = rp[nr];
  ci.reserve(nnz);
  for (int32_t u = 0; u < nr; ++u) ci.insert(ci.end(), cols[u].begin(), cols[u].end());
  std::vector<double> mval(nnz, 0.0);
  std::vector<std::vector<std::pair<int32_t, double>>> ctb(nnz);
  for (int32_t e = 0; e < nt; ++e) {
    const double* d = &dN[6 * (size_t)e];
    const double A = m->area[e];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        const int32_t r = node_rep[T[3 * e + a]], c = node_rep[T[3 * e + b]];
        const int32_t* beg = ci.data() + rp[r];
        const int32_t* end = ci.data() + rp[r + 1];
        const int64_t q = (int64_t)(std::lower_bound(beg, end, c) - ci.data());
        mval[q] += A * (a == b ? 2.0 : 1.0) / 12.0;
        ctb[q].push_back({e, A * (d[a] * d[b] + d[3 + a] * d[3 + b])});
      }
  }
  std::vector<int32_t> ctb_off(nnz + 1, 0), ctb_e;
  std::vector<double> ctb_k;
  for (int64_t q = 0; q < nnz; ++q) {
    ctb_off[q + 1] = ctb_off[q] + (int32_t)ctb[q].size();
    for (auto& pr : ctb[q]) { ctb_e.push_back(pr.first); ctb_k.push_back(pr.second); }
  }
  // structural checks before upload: every row and contribution list is
  // short and inside its array
  for (int32_t u = 0; u < nr; ++u)
    if (rp[u + 1] - rp[u] < 1 || rp[u + 1] - rp[u] > 64) return fail(PDF_EINVAL, "pdf_mesh_create: relaxation row out of range");
  for (int64_t q = 0; q < nnz; ++q) {
    if (ci[q] < 0 || ci[q] >= nr) return fail(PDF_EINVAL, "pdf_mesh_create: relaxation column out of range");
    if (ctb_off[q + 1] - ctb_off[q] < 1 || ctb_off[q + 1] - ctb_off[q] > 64) return fail(PDF_EINVAL, "pdf_mesh_create: relaxation contributions out of range");
  }
  // wall edges at each unknown (elements in order, local edges in order)
  std::vector<std::vector<int32_t>> pwl(nr);
  std::vector<int32_t> pw_e;
  std::vector<double> pw_n;
  for (int32_t e = 0; e < nt; ++e)
    for (int k = 0; k < 3; ++k) {
      const int32_t c = m->nbr[3 * e + k];
      if (c != kNbrWall && c != kNbrNoslip) continue;
      const int32_t a = T[3 * e + (k + 1) % 3], b = T[3 * e + (k + 2) % 3];
      const int32_t id = (int32_t)(pw_e.size() / 3);
      pw_e.insert(pw_e.end(), {e, a, b});
      const double tx = X[2 * b] - X[2 * a], ty = X[2 * b + 1] - X[2 * a + 1];
      const double len = std::sqrt(tx * tx + ty * ty);
      // counter-clockwise element: the outside lies to the right of a -> b
      pw_n.insert(pw_n.end(), {ty / len, -tx / len, len});
      pwl[node_rep[a]].push_back(id);
      pwl[node_rep[b]].push_back(id);
    }
  std::vector<int32_t> pw_off(nr + 1, 0), pw_ue;
  std::vector<double> pw_un;
  for (int32_t u = 0; u < nr; ++u) {
    pw_off[u + 1] = pw_off[u] + (int32_t)pwl[u].size();
    for (int32_t id : pwl[u]) {
      pw_ue.insert(pw_ue.end(), pw_e.begin() + 3 * id, pw_e.begin() + 3 * id + 3);
      pw_un.insert(pw_un.end(), pw_n.begin() + 3 * id, pw_n.begin() + 3 * id + 3);
    }
  }
  m->k_rp = rp;
  m->k_ci = ci;
  m->k_v.assign(nnz, 0.0);
  for (int64_t q = 0; q < nnz; ++q)
    for (int32_t t = ctb_off[q]; t < ctb_off[q + 1]; ++t) m->k_v[q] += ctb_k[t];
  RelaxMesh& R = m->rx;
  R.n_rep = nr;
  R.nnz = nnz;
  m->wall_d = wd;
  m->wall_n = wn;
  pdf_status s;
  if ((s = upload(&R.rp, rp.data(), rp.size())) != PDF_OK || (s = upload(&R.ci, ci.data(), ci.size())) != PDF_OK ||
      (s = upload(&R.mval, mval.data(), mval.size())) != PDF_OK ||
      (s = upload(&R.ctb_off, ctb_off.data(), ctb_off.size())) != PDF_OK ||
      (s = upload(&R.ctb_e, ctb_e.data(), ctb_e.size())) != PDF_OK ||
      (s = upload(&R.ctb_k, ctb_k.data(), ctb_k.size())) != PDF_OK ||
      (s = upload(&R.wall, wall.data(), wall.size())) != PDF_OK ||
      (s = upload(&R.rep_node, rep_node.data(), rep_node.size())) != PDF_OK ||
      (s = upload(&R.node_rep, node_rep.data(), node_rep.size())) != PDF_OK ||
      (s = upload(&R.wall_n, wn.data(), wn.size())) != PDF_OK ||
      (s = upload(&R.wall_d, wd.data(), wd.size())) != PDF_OK ||
      (s = upload(&R.pw_off, pw_off.data(), pw_off.size())) != PDF_OK ||
      (s = upload(&R.pw_e, pw_ue.data(), pw_ue.size())) != PDF_OK ||
      (s = upload(&R.pw_n, pw_un.data(), pw_un.size())) != PDF_OK) {
    free_relax(R);
    return s;
  }
  return PDF_OK;
}

static void free_mesh_dev(MeshDev& d) {
  cudaFree(d.xy); cudaFree(d.tri); cudaFree(d.geo); cudaFree(d.fgeo); cudaFree(d.dN);
  cudaFree(d.nse_off); cudaFree(d.nse); cudaFree(d.esup_off); cudaFree(d.esup); cudaFree(d.nsw_line);
  d = MeshDev();
}

static inline uint64_t edge_key(int32_t a, int32_t b) {
  uint32_t lo = (uint32_t)std::min(a, b), hi = (uint32_t)std::max(a, b);
  return ((uint64_t)hi << 32) | lo;
}

}  // namespace pdfgb

using namespace pdfgb;

extern "C" pdf_status pdf_mesh_create(const double* node_xy, int32_t n_nodes, const int32_t* tri,
                                      int32_t n_tri, const int32_t* twin, const int32_t* bnd_edge,
                                      int32_t n_bnd, double period_x, pdf_mesh** out) {
  if (!out) return fail(PDF_EINVAL, "pdf_mesh_create: out is NULL");
  *out = nullptr;
  if (!node_xy || !tri || n_nodes < 1 || n_tri < 1 || n_bnd < 0 || (n_bnd > 0 && !bnd_edge))
    return fail(PDF_EINVAL, "pdf_mesh_create: bad arguments");
  pdf_mesh* m = new (std::nothrow) pdf_mesh();
  if (!m) return fail(PDF_ENOMEM, "pdf_mesh_create: host allocation");
  m->xy.assign(node_xy, node_xy + 2 * (size_t)n_nodes);
  m->tri.assign(tri, tri + 3 * (size_t)n_tri);
  m->twin.assign(n_nodes, -1);
  if (twin) m->twin.assign(twin, twin + n_nodes);
  for (int32_t i = 0; i < 3 * n_tri; ++i)
    if (m->tri[i] < 0 || m->tri[i] >= n_nodes) { delete m; return fail(PDF_EINVAL, "pdf_mesh_create: node id out of range"); }
  for (int32_t n = 0; n < n_nodes; ++n)
    if (m->twin[n] < -1 || m->twin[n] >= n_nodes) { delete m; return fail(PDF_EINVAL, "pdf_mesh_create: twin out of range"); }

  const double* X = m->xy.data();
  const int32_t* T = m->tri.data();
  m->area.resize(n_tri);
  std::vector<ElemGeo> geo(n_tri);
  std::vector<double> dN(6 * (size_t)n_tri);
  for (int32_t e = 0; e < n_tri; ++e) {
    const double xa = X[2 * T[3 * e]], ya = X[2 * T[3 * e] + 1];
    const double xb = X[2 * T[3 * e + 1]], yb = X[2 * T[3 * e + 1] + 1];
    const double xc = X[2 * T[3 * e + 2]], yc = X[2 * T[3 * e + 2] + 1];
    const double two_a = (xb - xa) * (yc - ya) - (yb - ya) * (xc - xa);
    if (!(two_a > 0.0)) { delete m; return fail(PDF_EINVAL, "pdf_mesh_create: triangle not counter-clockwise or degenerate"); }
    m->area[e] = 0.5 * two_a;
    ElemGeo& g = geo[e];
    std::memset(&g, 0, sizeof(g));
    g.xb = xb; g.yb = yb;
    g.cbx = xc - xb; g.cby = yc - yb;
    g.abx = xa - xb; g.aby = ya - yb;
    g.two_area = two_a;
    // analytic shape-function derivatives of a linear triangle (sec. 3.4)
    const double yCA = yc - ya, yBA = yb - ya, xCA = xc - xa, xBA = xb - xa;
    double* d = &dN[6 * (size_t)e];
    d[0] = (-yCA + yBA) / two_a; d[1] = yCA / two_a; d[2] = -yBA / two_a;
    d[3] = (xCA - xBA) / two_a;  d[4] = -xCA / two_a; d[5] = xBA / two_a;
  }

  // edges: key -> (element, local edge); an interior edge appears twice
  std::unordered_map<uint64_t, std::pair<int32_t, int32_t>> first;
  first.reserve((size_t)n_tri * 2);
  m->nbr.assign(3 * (size_t)n_tri, INT32_MIN);
  m->shift.assign(3 * (size_t)n_tri, 0);
  m->reinj.assign(3 * (size_t)n_tri, 0);
  for (int32_t e = 0; e < n_tri; ++e) {
    for (int k = 0; k < 3; ++k) {
      const int32_t a = T[3 * e + (k + 1) % 3], b = T[3 * e + (k + 2) % 3];
      const uint64_t key = edge_key(a, b);
      auto it = first.find(key);
      if (it == first.end()) {
        first.emplace(key, std::make_pair(e, k));
      } else {
        const int32_t f = it->second.first, kf = it->second.second;
        if (m->nbr[3 * f + kf] != INT32_MIN) { delete m; return fail(PDF_EINVAL, "pdf_mesh_create: edge shared by more than two triangles"); }
        m->nbr[3 * f + kf] = e;
        m->nbr[3 * e + k] = f;
      }
    }
  }
  std::unordered_map<uint64_t, int32_t> tags;
  for (int32_t i = 0; i < n_bnd; ++i) tags[edge_key(bnd_edge[3 * i], bnd_edge[3 * i + 1])] = bnd_edge[3 * i + 2];
  for (int32_t e = 0; e < n_tri; ++e) {
    for (int k = 0; k < 3; ++k) {
      if (m->nbr[3 * e + k] != INT32_MIN) continue;
      const int32_t a = T[3 * e + (k + 1) % 3], b = T[3 * e + (k + 2) % 3];
      auto t = tags.find(edge_key(a, b));
      if (t == tags.end()) { delete m; return fail(PDF_EINVAL, "pdf_mesh_create: untagged boundary edge"); }
      // inflow/outflow edges whose nodes have periodic twins form a periodic
      // pair for the positions; leaving through the outflow re-injects
      int tag = t->second;
      const bool pair = (tag == PDF_TAG_INFLOW || tag == PDF_TAG_OUTFLOW) && m->twin[a] >= 0 && m->twin[b] >= 0;
      if (pair) {
        if (tag == PDF_TAG_OUTFLOW) m->reinj[3 * e + k] = 1;
        tag = PDF_TAG_PERIODIC;
      }
      switch (tag) {
        case PDF_TAG_WALL: m->nbr[3 * e + k] = kNbrWall; break;
        case PDF_TAG_NOSLIP: m->nbr[3 * e + k] = kNbrNoslip; break;
        case PDF_TAG_INFLOW: m->nbr[3 * e + k] = kNbrInflow; break;
        case PDF_TAG_OUTFLOW: m->nbr[3 * e + k] = kNbrOutflow; break;
        case PDF_TAG_PERIODIC: {
          const int32_t ta = m->twin[a], tb = m->twin[b];
          if (ta < 0 || tb < 0) { delete m; return fail(PDF_EINVAL, "pdf_mesh_create: periodic edge without twin nodes"); }
          auto it = first.find(edge_key(ta, tb));
          if (it == first.end() || it->second.first == e) { delete m; return fail(PDF_EINVAL, "pdf_mesh_create: unmatched periodic edge"); }
          m->nbr[3 * e + k] = it->second.first;
          if (period_x > 0.0)
            m->shift[3 * e + k] = (int32_t)std::lround((X[2 * ta] - X[2 * a]) / period_x);
          break;
        }
        default: delete m; return fail(PDF_EINVAL, "pdf_mesh_create: unknown boundary tag");
      }
    }
  }
  for (int32_t e = 0; e < n_tri; ++e)
    for (int k = 0; k < 3; ++k) {
      geo[e].nbr[k] = m->nbr[3 * e + k];
      geo[e].shift[k] = (int8_t)m->shift[3 * e + k];
      if (m->reinj[3 * e + k]) geo[e].reinj |= (uint8_t)(1u << k);
    }
  // no-slip walls: for an element with a node on a no-slip edge, the line of
  // the nearest such edge (from the element's centroid; ties: the first in
  // the order elements, edges, edge ends, elements around the end) with its
  // normal into the fluid
  std::vector<double> nsw_line(4 * (size_t)n_tri, 0.0);
  {
    std::vector<int32_t> esu_off(n_nodes + 1, 0), esu(3 * (size_t)n_tri);
    for (int32_t i = 0; i < 3 * n_tri; ++i) esu_off[T[i] + 1]++;
    for (int32_t n = 0; n < n_nodes; ++n) esu_off[n + 1] += esu_off[n];
    std::vector<int32_t> fill(esu_off.begin(), esu_off.end() - 1);
    for (int32_t e = 0; e < n_tri; ++e)
      for (int k = 0; k < 3; ++k) esu[fill[T[3 * e + k]]++] = e;
    std::vector<double> best(n_tri, INFINITY);
    for (int32_t f = 0; f < n_tri; ++f)
      for (int k = 0; k < 3; ++k) {
        if (m->nbr[3 * f + k] != kNbrNoslip) continue;
        const int32_t a = T[3 * f + (k + 1) % 3], b = T[3 * f + (k + 2) % 3];
        const double xa = X[2 * a], ya = X[2 * a + 1], tx = X[2 * b] - xa, ty = X[2 * b + 1] - ya;
        const double len = std::sqrt(tx * tx + ty * ty);
        const double nx = -ty / len, ny = tx / len;
        const int32_t ends[2] = {a, b};
        for (int q = 0; q < 2; ++q)
          for (int32_t i = esu_off[ends[q]]; i < esu_off[ends[q] + 1]; ++i) {
            const int32_t e = esu[i];
            const int32_t* t = T + 3 * e;
            const double cx = (X[2 * t[0]] + X[2 * t[1]] + X[2 * t[2]]) / 3.0;
            const double cy = (X[2 * t[0] + 1] + X[2 * t[1] + 1] + X[2 * t[2] + 1]) / 3.0;
            double sp = ((cx - xa) * tx + (cy - ya) * ty) / (len * len);
            sp = std::min(1.0, std::max(0.0, sp));
            const double dx = cx - (xa + sp * tx), dy = cy - (ya + sp * ty);
            const double dist = std::sqrt(dx * dx + dy * dy);
            if (dist < best[e]) {
              best[e] = dist;
              geo[e].nsw = 1;
              nsw_line[4 * e] = xa; nsw_line[4 * e + 1] = ya; nsw_line[4 * e + 2] = nx; nsw_line[4 * e + 3] = ny;
            }
          }
      }
  }
  // the fixed-point copy for the FP64-free walk
  std::vector<FxGeo> fgeo(n_tri);
  auto bits = [](double v) { uint64_t b; std::memcpy(&b, &v, 8); return b; };
  for (int32_t e = 0; e < n_tri; ++e) {
    const ElemGeo& g = geo[e];
    FxGeo& f = fgeo[e];
    std::memset(&f, 0, sizeof(f));
    f.xb = fx::d2fix(bits(g.xb), 56);
    f.yb = fx::d2fix(bits(g.yb), 56);
    f.cbx = fx::d2df(bits(g.cbx)); f.cby = fx::d2df(bits(g.cby));
    f.abx = fx::d2df(bits(g.abx)); f.aby = fx::d2df(bits(g.aby));
    f.two_area = fx::d2df(bits(g.two_area));
    for (int k = 0; k < 3; ++k) { f.nbr[k] = g.nbr[k]; f.shift[k] = g.shift[k]; }
    f.reinj = g.reinj;
    f.nsw = g.nsw;
    if (std::fabs(g.xb) >= 63.0 || std::fabs(g.yb) >= 63.0) {
      delete m;
      return fail(PDF_EINVAL, "pdf_mesh_create: node coordinates must lie within |x|, |y| < 63");
    }
  }

  // node -> elements, ascending element ids; merged with the periodic twin
  std::vector<int32_t> esup_off(n_nodes + 1, 0), esup(3 * (size_t)n_tri);
  for (int32_t i = 0; i < 3 * n_tri; ++i) esup_off[T[i] + 1]++;
  std::partial_sum(esup_off.begin(), esup_off.end(), esup_off.begin());
  {
    std::vector<int32_t> fill(esup_off.begin(), esup_off.end() - 1);
    for (int32_t e = 0; e < n_tri; ++e)
      for (int k = 0; k < 3; ++k) esup[fill[T[3 * e + k]]++] = e;
  }
  std::vector<int32_t> nse_off(n_nodes + 1, 0), nse;
  nse.reserve(3 * (size_t)n_tri * 2);
  for (int32_t n = 0; n < n_nodes; ++n) {
    const size_t start = nse.size();
    nse.insert(nse.end(), esup.begin() + esup_off[n], esup.begin() + esup_off[n + 1]);
    if (m->twin[n] >= 0) {
      const int32_t t = m->twin[n];
      nse.insert(nse.end(), esup.begin() + esup_off[t], esup.begin() + esup_off[t + 1]);
    }
    std::sort(nse.begin() + start, nse.end());
    nse_off[n + 1] = (int32_t)nse.size();
  }

  MeshDev& d = m->d;
  d.n_nodes = n_nodes;
  d.n_tri = n_tri;
  d.period = period_x;
  pdf_status s;
  std::vector<int32_t> bnd_wall, wall_tag;
  for (int32_t i = 0; i < n_bnd; ++i)
    if (bnd_edge[3 * i + 2] == PDF_TAG_WALL || bnd_edge[3 * i + 2] == PDF_TAG_NOSLIP) {
      bnd_wall.push_back(bnd_edge[3 * i]);
      bnd_wall.push_back(bnd_edge[3 * i + 1]);
      wall_tag.push_back(bnd_edge[3 * i + 2]);
    }
  if ((s = upload(&d.xy, m->xy.data(), m->xy.size())) != PDF_OK ||
      (s = upload(&d.tri, m->tri.data(), m->tri.size())) != PDF_OK ||
      (s = upload(&d.geo, geo.data(), geo.size())) != PDF_OK ||
      (s = upload(&d.fgeo, fgeo.data(), fgeo.size())) != PDF_OK ||
      (s = upload(&d.dN, dN.data(), dN.size())) != PDF_OK ||
      (s = upload(&d.nse_off, nse_off.data(), nse_off.size())) != PDF_OK ||
      (s = upload(&d.nse, nse.data(), nse.size())) != PDF_OK ||
      (s = upload(&d.esup_off, esup_off.data(), esup_off.size())) != PDF_OK ||
      (s = upload(&d.esup, esup.data(), esup.size())) != PDF_OK ||
      (s = upload(&d.nsw_line, nsw_line.data(), nsw_line.size())) != PDF_OK) {
    free_mesh_dev(d);
    delete m;
    return s;
  }
  if ((s = build_relax(m, bnd_wall, wall_tag, dN, nse_off, nse, esup_off, esup)) != PDF_OK) {
    free_mesh_dev(d);
    delete m;
    return s;
  }
  // host data of the pressure system with inflow/outflow conditions
  m->period = period_x;
  m->dN = dN;
  m->inout.assign(n_nodes, 0);
  for (int32_t i = 0; i < n_bnd; ++i) {
    const int32_t t = bnd_edge[3 * i + 2];
    if (t != PDF_TAG_INFLOW && t != PDF_TAG_OUTFLOW) continue;
    for (int q = 0; q < 2; ++q) m->inout[bnd_edge[3 * i + q]] = t == PDF_TAG_INFLOW ? 1 : 2;
  }
  *out = m;
  return PDF_OK;
}

extern "C" pdf_status pdf_mesh_destroy(pdf_mesh* m) {
  if (!m) return PDF_OK;
  if (m->solver) release_particles(m->solver);
  free_mesh_dev(m->d);
  free_relax(m->rx);
  delete m;
  return PDF_OK;
}

extern "C" pdf_status pdf_mesh_connectivity(const pdf_mesh* m, int32_t* nbr, int32_t* shift) {
  if (!m) return fail(PDF_EINVAL, "pdf_mesh_connectivity: NULL mesh");
  if (nbr) std::memcpy(nbr, m->nbr.data(), m->nbr.size() * sizeof(int32_t));
  if (shift) std::memcpy(shift, m->shift.data(), m->shift.size() * sizeof(int32_t));
  return PDF_OK;
}

extern "C" pdf_status pdf_mesh_wall_distance(const pdf_mesh* m, double* dist, double* normal) {
  if (!m) return fail(PDF_EINVAL, "pdf_mesh_wall_distance: NULL mesh");
  if (dist) std::memcpy(dist, m->wall_d.data(), m->wall_d.size() * sizeof(double));
  if (normal) std::memcpy(normal, m->wall_n.data(), m->wall_n.size() * sizeof(double));
  return PDF_OK;
}

extern "C" pdf_status pdf_mesh_size(const pdf_mesh* m, int32_t* n_nodes, int32_t* n_tri) {
  if (!m) return fail(PDF_EINVAL, "pdf_mesh_size: NULL mesh");
  if (n_nodes) *n_nodes = m->d.n_nodes;
  if (n_tri) *n_tri = m->d.n_tri;
  return PDF_OK;
}
