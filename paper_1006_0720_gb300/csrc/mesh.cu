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

static void free_mesh_dev(MeshDev& d) {
  cudaFree(d.xy); cudaFree(d.tri); cudaFree(d.geo); cudaFree(d.dN);
  cudaFree(d.nse_off); cudaFree(d.nse); cudaFree(d.esup_off); cudaFree(d.esup);
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
      switch (t->second) {
        case PDF_TAG_WALL: m->nbr[3 * e + k] = kNbrWall; break;
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
  if ((s = upload(&d.xy, m->xy.data(), m->xy.size())) != PDF_OK ||
      (s = upload(&d.tri, m->tri.data(), m->tri.size())) != PDF_OK ||
      (s = upload(&d.geo, geo.data(), geo.size())) != PDF_OK ||
      (s = upload(&d.dN, dN.data(), dN.size())) != PDF_OK ||
      (s = upload(&d.nse_off, nse_off.data(), nse_off.size())) != PDF_OK ||
      (s = upload(&d.nse, nse.data(), nse.size())) != PDF_OK ||
      (s = upload(&d.esup_off, esup_off.data(), esup_off.size())) != PDF_OK ||
      (s = upload(&d.esup, esup.data(), esup.size())) != PDF_OK) {
    free_mesh_dev(d);
    delete m;
    return s;
  }
  *out = m;
  return PDF_OK;
}

extern "C" pdf_status pdf_mesh_destroy(pdf_mesh* m) {
  if (!m) return PDF_OK;
  free_mesh_dev(m->d);
  delete m;
  return PDF_OK;
}

extern "C" pdf_status pdf_mesh_connectivity(const pdf_mesh* m, int32_t* nbr, int32_t* shift) {
  if (!m) return fail(PDF_EINVAL, "pdf_mesh_connectivity: NULL mesh");
  if (nbr) std::memcpy(nbr, m->nbr.data(), m->nbr.size() * sizeof(int32_t));
  if (shift) std::memcpy(shift, m->shift.data(), m->shift.size() * sizeof(int32_t));
  return PDF_OK;
}

extern "C" pdf_status pdf_mesh_size(const pdf_mesh* m, int32_t* n_nodes, int32_t* n_tri) {
  if (!m) return fail(PDF_EINVAL, "pdf_mesh_size: NULL mesh");
  if (n_nodes) *n_nodes = m->d.n_nodes;
  if (n_tri) *n_tri = m->d.n_tri;
  return PDF_OK;
}
