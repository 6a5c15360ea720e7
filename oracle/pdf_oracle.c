/*
 * CPU ORACLE for the particle time step of the joint velocity-frequency-scalar
 * PDF method (Bakosi, "PDF modeling of turbulent flows on unstructured grids").
 *
 * TEST INFRASTRUCTURE ONLY.  Plain, slow, single-threaded FP64 C written from
 * the paper, used to check the CUDA library.  Only the tests, the smoke check
 * and the benchmark's CPU-baseline leg may load it.  It shares no code,
 * header, table or helper with the CUDA library.
 *
 * Each function cites the passage it follows.  Readings of places where the
 * paper is silent are marked READING.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared -o liboracle.so pdf_oracle.c -lm
 * (-ffp-contract=off: the FP32 Gaussian transform must round exactly as
 * written so that both implementations draw bit-identical numbers.)
 */
#include <math.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Model constants, Table "Constants for modeling the joint PDF of velocity  */
/* and frequency" (ch. 4, channel modeling specifics).                        */
/* ------------------------------------------------------------------------ */
static const double OR_C1 = 1.85, OR_C2 = 0.63, OR_C3 = 5.0, OR_C4 = 0.25, OR_CT = 6.0,
                    OR_CL = 0.134, OR_CETA = 72.0, OR_CV = 1.4, OR_GAMMA5 = 0.1,
                    OR_COMEGA1 = 0.5, OR_COMEGA2 = 0.73;
/* SLM coefficient, Eq. wall-GandC (sec. 2, wall functions). */
static const double OR_C0_SLM = 3.5;
/* READING (paper silent): floors used in G, C0, b_ij, A_v and L. */
static const double OR_KFLOOR = 1e-12, OR_EFLOOR = 1e-12;

void or_constants(double* c) {
  c[0] = OR_C1; c[1] = OR_C2; c[2] = OR_C3; c[3] = OR_C4; c[4] = OR_CT; c[5] = OR_CL;
  c[6] = OR_CETA; c[7] = OR_CV; c[8] = OR_GAMMA5; c[9] = OR_COMEGA1; c[10] = OR_COMEGA2;
  c[11] = OR_C0_SLM;
}

/* ------------------------------------------------------------------------ */
/* Random numbers.  The paper draws 6 Gaussians per particle per step from   */
/* tables split into per-thread blocks (sec. 3.8).  Here every draw is a     */
/* pure function of (seed, particle id, step, block, purpose): Philox4x32-10 */
/* (Salmon, Moraes, Dror & Shaw, SC'11), then Box-Muller in FP32 with the    */
/* log and sin/cos evaluated as specified below.                             */
/* ------------------------------------------------------------------------ */
void or_philox(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  /* Philox4x32: S-box is the pair of 32x32->64 multiplications with the
   * multipliers 0xD2511F53 and 0xCD9E8D57; the key is bumped by the Weyl
   * constants 0x9E3779B9 and 0xBB67AE85 between rounds; 10 rounds. */
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform in (0,1) from the top 23 bits of a word: (floor(w/2^9) + 1/2) / 2^23.
 * Exact in FP32; smallest value 2^-24, largest 1 - 2^-24. */
float or_u01(uint32_t w) { return ((float)(w >> 9) + 0.5f) * 0x1p-23f; }

/* ln(u) for u in (0, 1], FP32.  u = m 2^e with m in [sqrt(1/2), sqrt(2));
 * ln m = 2 atanh(s), s = (m-1)/(m+1), by its Taylor series
 * 2 s (1 + z/3 + z^2/5 + z^3/7 + z^4/9), z = s^2 (|s| <= 0.1716, remainder
 * below 1e-9 relative); ln 2 is split into a 11-bit head (1420/2048) and a
 * tail so that e*head is exact.  Horner with explicit fused multiply-adds. */
float or_logf(float u) {
  int e;
  float m = frexpf(u, &e); /* m in [0.5, 1) */
  if (m < 0.70710678f) { m = m * 2.0f; e -= 1; }
  float s = (m - 1.0f) / (m + 1.0f);
  float z = s * s;
  float p = fmaf(z, 1.0f / 9.0f, 1.0f / 7.0f);
  p = fmaf(p, z, 1.0f / 5.0f);
  p = fmaf(p, z, 1.0f / 3.0f);
  p = fmaf(p, z, 1.0f);
  float lnm = (2.0f * s) * p;
  const float LN2_HEAD = 1420.0f / 2048.0f;            /* 0.693359375 */
  const float LN2_TAIL = -2.12194440054690582e-4f;     /* ln 2 - head */
  float fe = (float)e;
  return fmaf(fe, LN2_HEAD, fmaf(fe, LN2_TAIL, lnm));
}

/* sin and cos of 2*pi*u for u in (0,1), FP32: t = 4u is split into the
 * nearest quadrant q and a remainder r in [-1/2, 1/2] (both exact), theta =
 * r*pi/2 in [-pi/4, pi/4], then the Taylor series of sin to theta^9 and of
 * cos to theta^10 (remainders below 2e-9), rotated by q quarter turns. */
void or_sincos2pi(float u, float* sn, float* cs) {
  float t = 4.0f * u;
  float q = rintf(t);
  float r = t - q;
  float th = r * 1.57079632679489662f;
  float z = th * th;
  float ps = fmaf(z, 1.0f / 362880.0f, -1.0f / 5040.0f);
  ps = fmaf(ps, z, 1.0f / 120.0f);
  ps = fmaf(ps, z, -1.0f / 6.0f);
  ps = fmaf(ps, z, 1.0f);
  float s = th * ps;
  float pc = fmaf(z, -1.0f / 3628800.0f, 1.0f / 40320.0f);
  pc = fmaf(pc, z, -1.0f / 720.0f);
  pc = fmaf(pc, z, 1.0f / 24.0f);
  pc = fmaf(pc, z, -0.5f);
  float c = fmaf(pc, z, 1.0f);
  int qi = ((int)q) & 3;
  switch (qi) {
    case 0: *sn = s;  *cs = c;  break;
    case 1: *sn = c;  *cs = -s; break;
    case 2: *sn = -s; *cs = -c; break;
    default: *sn = -c; *cs = s; break;
  }
}

/* Box-Muller (1958): two uniforms -> two independent N(0,1). */
static void or_box_muller(float u1, float u2, float* g0, float* g1) {
  float rad = sqrtf(-2.0f * or_logf(u1));
  float sn, cs;
  or_sincos2pi(u2, &sn, &cs);
  *g0 = rad * cs;
  *g1 = rad * sn;
}

/* Four Gaussians from one Philox block, counter (c0, c1, c2, c3). */
void or_gauss4(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, float g[4]) {
  uint32_t ctr[4] = {c0, c1, c2, c3};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t w[4];
  or_philox(ctr, key, w);
  or_box_muller(or_u01(w[0]), or_u01(w[1]), &g[0], &g[1]);
  or_box_muller(or_u01(w[2]), or_u01(w[3]), &g[2], &g[3]);
}

/* Bulk draw for statistical tests: for pid = 0..n-1, the four Gaussians of
 * counter (pid, c1, c2, c3) into out[4*pid .. 4*pid+3]. */
void or_gauss_fill(uint64_t seed, long n, uint32_t c1, uint32_t c2, uint32_t c3, float* out) {
  for (long p = 0; p < n; ++p) or_gauss4(seed, (uint32_t)p, c1, c2, c3, out + 4 * p);
}

/* Counter purposes. */
enum { OR_PURPOSE_STEP = 0, OR_PURPOSE_INIT = 1, OR_PURPOSE_REDIST = 2 };

/* ------------------------------------------------------------------------ */
/* Mesh connectivity (sec. 3.3 linked lists; sec. 3.5 element-surrounding-  */
/* element list with tagged boundary neighbours).                            */
/* ------------------------------------------------------------------------ */
enum { OR_TAG_WALL = 1, OR_TAG_PERIODIC = 2, OR_TAG_INFLOW = 3, OR_TAG_OUTFLOW = 4, OR_TAG_NOSLIP = 5 };
enum { OR_NBR_WALL = -1, OR_NBR_INFLOW = -3, OR_NBR_OUTFLOW = -4, OR_NBR_NOSLIP = -5 };

typedef struct {
  int n_nodes, n_tri;
  double period;
  double* xy;      /* [n_nodes][2] */
  int* tri;        /* [n_tri][3] counter-clockwise A, B, C */
  int* twin;       /* periodic twin node or -1 */
  double* area;    /* A_e */
  int* nbr;        /* [n_tri][3] neighbour across the edge opposite vertex k */
  int* shift;      /* [n_tri][3] periodic shift (multiples of period) of x when crossing */
  int* reinj;      /* [n_tri][3] 1 if crossing this edge leaves through the outflow */
  int* esup_off;   /* node -> elements containing the node (ascending ids) */
  int* esup;
  int* nse_off;    /* node -> elements around the node or its twin (ascending ids) */
  int* nse;
  /* no-slip walls (sec. no-slip wall-boundary conditions): for an element
   * with a node on a no-slip edge, the line of the nearest such edge (a point
   * and the unit normal into the fluid); nsw_flag[e] = 0 elsewhere */
  int* nsw_flag;
  double* nsw;     /* [n_tri][4] x_a, y_a, n_x, n_y */
} or_mesh;

static int cmp_int(const void* a, const void* b) {
  int x = *(const int*)a, y = *(const int*)b;
  return (x > y) - (x < y);
}

static int tri_has(const or_mesh* m, int e, int a) {
  const int* t = m->tri + 3 * e;
  return t[0] == a || t[1] == a || t[2] == a;
}

static int edge_tag(int n_bnd, const int* bnd, int a, int b) {
  for (int i = 0; i < n_bnd; ++i) {
    int p = bnd[3 * i], q = bnd[3 * i + 1];
    if ((p == a && q == b) || (p == b && q == a)) return bnd[3 * i + 2];
  }
  return 0;
}

void or_mesh_free(or_mesh* m) {
  if (!m) return;
  free(m->xy); free(m->tri); free(m->twin); free(m->area); free(m->nbr); free(m->shift); free(m->reinj);
  free(m->esup_off); free(m->esup); free(m->nse_off); free(m->nse);
  free(m->nsw_flag); free(m->nsw);
  free(m);
}

/* Returns NULL on an inconsistent mesh (unlisted boundary edge, clockwise
 * triangle, unmatched periodic edge). */
or_mesh* or_mesh_create(int n_nodes, const double* xy, int n_tri, const int* tri,
                        const int* twin, int n_bnd, const int* bnd, double period) {
  or_mesh* m = (or_mesh*)calloc(1, sizeof(or_mesh));
  m->n_nodes = n_nodes; m->n_tri = n_tri; m->period = period;
  m->xy = (double*)malloc(sizeof(double) * 2 * n_nodes);
  memcpy(m->xy, xy, sizeof(double) * 2 * n_nodes);
  m->tri = (int*)malloc(sizeof(int) * 3 * n_tri);
  memcpy(m->tri, tri, sizeof(int) * 3 * n_tri);
  m->twin = (int*)malloc(sizeof(int) * n_nodes);
  for (int n = 0; n < n_nodes; ++n) m->twin[n] = twin ? twin[n] : -1;
  m->area = (double*)malloc(sizeof(double) * n_tri);
  /* element area A_e = 1/2 (r_B - r_A) x (r_C - r_A) */
  for (int e = 0; e < n_tri; ++e) {
    const int* t = m->tri + 3 * e;
    double xa = xy[2 * t[0]], ya = xy[2 * t[0] + 1];
    double xb = xy[2 * t[1]], yb = xy[2 * t[1] + 1];
    double xc = xy[2 * t[2]], yc = xy[2 * t[2] + 1];
    m->area[e] = 0.5 * ((xb - xa) * (yc - ya) - (yb - ya) * (xc - xa));
    if (!(m->area[e] > 0.0)) { or_mesh_free(m); return NULL; }
  }
  /* elements surrounding points: count, then fill in ascending element order */
  m->esup_off = (int*)calloc(n_nodes + 1, sizeof(int));
  for (int e = 0; e < n_tri; ++e)
    for (int k = 0; k < 3; ++k) m->esup_off[m->tri[3 * e + k] + 1]++;
  for (int n = 0; n < n_nodes; ++n) m->esup_off[n + 1] += m->esup_off[n];
  m->esup = (int*)malloc(sizeof(int) * 3 * n_tri);
  int* fill = (int*)calloc(n_nodes, sizeof(int));
  for (int e = 0; e < n_tri; ++e)
    for (int k = 0; k < 3; ++k) {
      int n = m->tri[3 * e + k];
      m->esup[m->esup_off[n] + fill[n]++] = e;
    }
  free(fill);
  /* merged lists: elements around n and around its periodic twin */
  m->nse_off = (int*)calloc(n_nodes + 1, sizeof(int));
  for (int n = 0; n < n_nodes; ++n) {
    int c = m->esup_off[n + 1] - m->esup_off[n];
    if (m->twin[n] >= 0) c += m->esup_off[m->twin[n] + 1] - m->esup_off[m->twin[n]];
    m->nse_off[n + 1] = m->nse_off[n] + c;
  }
  m->nse = (int*)malloc(sizeof(int) * (m->nse_off[n_nodes] + 1));
  for (int n = 0; n < n_nodes; ++n) {
    int* dst = m->nse + m->nse_off[n];
    int c = 0;
    for (int i = m->esup_off[n]; i < m->esup_off[n + 1]; ++i) dst[c++] = m->esup[i];
    if (m->twin[n] >= 0)
      for (int i = m->esup_off[m->twin[n]]; i < m->esup_off[m->twin[n] + 1]; ++i) dst[c++] = m->esup[i];
    qsort(dst, c, sizeof(int), cmp_int);
  }
  /* element-surrounding-element list; edge k is opposite local vertex k */
  m->nbr = (int*)malloc(sizeof(int) * 3 * n_tri);
  m->shift = (int*)calloc(3 * n_tri, sizeof(int));
  m->reinj = (int*)calloc(3 * n_tri, sizeof(int));
  for (int e = 0; e < n_tri; ++e) {
    for (int k = 0; k < 3; ++k) {
      int a = m->tri[3 * e + (k + 1) % 3], b = m->tri[3 * e + (k + 2) % 3];
      int found = -1;
      for (int i = m->esup_off[a]; i < m->esup_off[a + 1]; ++i) {
        int f = m->esup[i];
        if (f != e && tri_has(m, f, b)) { found = f; break; }
      }
      if (found >= 0) { m->nbr[3 * e + k] = found; continue; }
      int tag = edge_tag(n_bnd, bnd, a, b);
      /* READING (the paper's canyon, ch. 5): inflow and outflow edges whose
       * nodes have periodic twins form a periodic pair for the particles'
       * positions; leaving through the outflow marks the particle as
       * re-entering fluid.  Without twins they are open boundaries. */
      int open_pair = (tag == OR_TAG_INFLOW || tag == OR_TAG_OUTFLOW) && m->twin[a] >= 0 && m->twin[b] >= 0;
      if (tag == OR_TAG_WALL) m->nbr[3 * e + k] = OR_NBR_WALL;
      else if (tag == OR_TAG_NOSLIP) m->nbr[3 * e + k] = OR_NBR_NOSLIP;
      else if (tag == OR_TAG_INFLOW && !open_pair) m->nbr[3 * e + k] = OR_NBR_INFLOW;
      else if (tag == OR_TAG_OUTFLOW && !open_pair) m->nbr[3 * e + k] = OR_NBR_OUTFLOW;
      else if (tag == OR_TAG_PERIODIC || open_pair) {
        if (tag == OR_TAG_OUTFLOW) m->reinj[3 * e + k] = 1;
        int ta = m->twin[a], tb = m->twin[b];
        if (ta < 0 || tb < 0) { or_mesh_free(m); return NULL; }
        for (int i = m->esup_off[ta]; i < m->esup_off[ta + 1]; ++i) {
          int f = m->esup[i];
          if (f != e && tri_has(m, f, tb)) { found = f; break; }
        }
        if (found < 0) { or_mesh_free(m); return NULL; }
        m->nbr[3 * e + k] = found;
        m->shift[3 * e + k] = (int)lround((xy[2 * ta] - xy[2 * a]) / period);
      } else { or_mesh_free(m); return NULL; }
    }
  }
  /* READING: the wall a near-wall particle is measured from is the no-slip
   * edge nearest to its element's centroid among the edges sharing a node
   * with the element (ties: the first found, elements and edges ascending) */
  m->nsw_flag = (int*)calloc(n_tri, sizeof(int));
  m->nsw = (double*)calloc(4 * (size_t)n_tri, sizeof(double));
  double* best = (double*)malloc(sizeof(double) * n_tri);
  for (int e = 0; e < n_tri; ++e) best[e] = INFINITY;
  for (int f = 0; f < n_tri; ++f)
    for (int k = 0; k < 3; ++k) {
      if (m->nbr[3 * f + k] != OR_NBR_NOSLIP) continue;
      int a = m->tri[3 * f + (k + 1) % 3], b = m->tri[3 * f + (k + 2) % 3];
      double xa = xy[2 * a], ya = xy[2 * a + 1], tx = xy[2 * b] - xa, ty = xy[2 * b + 1] - ya;
      double len = sqrt(tx * tx + ty * ty);
      double nx = -ty / len, ny = tx / len;  /* into the fluid: the edge runs a -> b counter-clockwise */
      int ends[2] = {a, b};
      for (int q = 0; q < 2; ++q)
        for (int i = m->esup_off[ends[q]]; i < m->esup_off[ends[q] + 1]; ++i) {
          int e = m->esup[i];
          const int* t = m->tri + 3 * e;
          double cx = (xy[2 * t[0]] + xy[2 * t[1]] + xy[2 * t[2]]) / 3.0;
          double cy = (xy[2 * t[0] + 1] + xy[2 * t[1] + 1] + xy[2 * t[2] + 1]) / 3.0;
          /* distance from the centroid to the segment a-b */
          double s = ((cx - xa) * tx + (cy - ya) * ty) / (len * len);
          if (s < 0.0) s = 0.0;
          if (s > 1.0) s = 1.0;
          double dx = cx - (xa + s * tx), dy = cy - (ya + s * ty);
          double dist = sqrt(dx * dx + dy * dy);
          if (dist < best[e]) {
            best[e] = dist;
            m->nsw_flag[e] = 1;
            m->nsw[4 * e] = xa; m->nsw[4 * e + 1] = ya; m->nsw[4 * e + 2] = nx; m->nsw[4 * e + 3] = ny;
          }
        }
    }
  free(best);
  return m;
}

void or_mesh_noslip(const or_mesh* m, int* flag, double* line) {
  if (flag) memcpy(flag, m->nsw_flag, sizeof(int) * m->n_tri);
  if (line) memcpy(line, m->nsw, sizeof(double) * 4 * m->n_tri);
}

void or_mesh_get(const or_mesh* m, double* area, int* nbr, int* shift) {
  if (area) memcpy(area, m->area, sizeof(double) * m->n_tri);
  if (nbr) memcpy(nbr, m->nbr, sizeof(int) * 3 * m->n_tri);
  if (shift) memcpy(shift, m->shift, sizeof(int) * 3 * m->n_tri);
}

/* ------------------------------------------------------------------------ */
/* Particle tracking, sec. 3.5.                                              */
/* ------------------------------------------------------------------------ */
/* Signed sub-areas of the element test (eq. element-test and the two cross  */
/* products below it): N^A = 1/2 (r_C - r_B) x (r_P - r_B),                   */
/* N^C = 1/2 (r_P - r_B) x (r_A - r_B), N^B = A_e - N^A - N^C.                */
/* READING: the |.| in the printed formulas is dropped (the text calls them   */
/* signed), and a point counts as inside when all three are >= 0.            */
void or_subareas(const or_mesh* m, int e, double px, double py, double N[3]) {
  const int* t = m->tri + 3 * e;
  double xa = m->xy[2 * t[0]], ya = m->xy[2 * t[0] + 1];
  double xb = m->xy[2 * t[1]], yb = m->xy[2 * t[1] + 1];
  double xc = m->xy[2 * t[2]], yc = m->xy[2 * t[2] + 1];
  double NA = 0.5 * ((xc - xb) * (py - yb) - (yc - yb) * (px - xb));
  double NC = 0.5 * ((px - xb) * (ya - yb) - (py - yb) * (xa - xb));
  N[0] = NA;
  N[2] = NC;
  N[1] = m->area[e] - NA - NC;
}

static int or_inside(const double N[3]) { return N[0] >= 0.0 && N[1] >= 0.0 && N[2] >= 0.0; }

/* Tracking status bits (returned per particle). */
enum { OR_TRK_FALLBACK = 1, OR_TRK_BRUTE = 2, OR_TRK_LOST = 4, OR_TRK_EXIT_OUT = 8, OR_TRK_EXIT_IN = 16,
       OR_TRK_REINJECT = 32, OR_TRK_NOSLIP = 64 };

typedef struct { int walk_steps, reflections, crossings_periodic, status; double min_rel; } or_track_info;

/* Neighbour walk from the old host element (sec. 3.5): if the particle is not
 * inside, step to the neighbour across the edge opposite the smallest
 * sub-area (READING: ties go to the lowest local vertex, A < B < C).
 * A periodic edge shifts x by the stored multiple of the period.  A wall
 * edge first triggers the fall-back of the concave-corner figure: the
 * particle is searched among the elements around the current element's
 * nodes; if it is not there it is behind the wall and is reflected across the
 * wall edge line with its wall-normal in-plane velocity reversed (free-slip
 * reflection, as for the channel centreline and the toy problem's walls).
 * After 64 walk steps the search falls back to all elements (lowest id
 * first).  u, v may be NULL (position-only search). */
int or_track(const or_mesh* m, int e0, double* px, double* py, double* u, double* v,
             or_track_info* info) {
  int e = e0, steps = 0;
  double x = *px, y = *py;
  info->walk_steps = 0; info->reflections = 0; info->crossings_periodic = 0; info->status = 0;
  info->min_rel = 0.0;
  for (;;) {
    double N[3];
    or_subareas(m, e, x, y, N);
    if (or_inside(N)) {
      double mn = N[0] < N[1] ? N[0] : N[1];
      if (N[2] < mn) mn = N[2];
      info->min_rel = mn / m->area[e];
      break;
    }
    if (steps >= 64) {
      /* a non-finite position is lost without the search over all elements */
      if (!isfinite(x) || !isfinite(y)) { info->status |= OR_TRK_LOST; break; }
      info->status |= OR_TRK_BRUTE;
      int hit = -1;
      for (int f = 0; f < m->n_tri && hit < 0; ++f) {
        or_subareas(m, f, x, y, N);
        if (or_inside(N)) hit = f;
      }
      if (hit < 0) { info->status |= OR_TRK_LOST; break; }
      e = hit;
      continue;
    }
    int k = 0;
    if (N[1] < N[k]) k = 1;
    if (N[2] < N[k]) k = 2;
    int nb = m->nbr[3 * e + k];
    steps++;
    if (nb >= 0) {
      if (m->shift[3 * e + k] != 0) {
        x += m->shift[3 * e + k] * m->period;
        info->crossings_periodic++;
      }
      if (m->reinj[3 * e + k]) info->status |= OR_TRK_REINJECT;
      e = nb;
      continue;
    }
    if (nb == OR_NBR_OUTFLOW) { info->status |= OR_TRK_EXIT_OUT; break; }
    if (nb == OR_NBR_INFLOW) { info->status |= OR_TRK_EXIT_IN; break; }
    /* wall: fall-back search around the nodes of the current element */
    int hit = -1;
    const int* t = m->tri + 3 * e;
    for (int j = 0; j < 3 && hit < 0; ++j) {
      int n = t[j];
      for (int i = m->esup_off[n]; i < m->esup_off[n + 1] && hit < 0; ++i) {
        int f = m->esup[i];
        double M[3];
        or_subareas(m, f, x, y, M);
        if (or_inside(M)) hit = f;
      }
    }
    if (hit >= 0) { info->status |= OR_TRK_FALLBACK; e = hit; continue; }
    if (info->reflections >= 4) { info->status |= OR_TRK_LOST; break; }
    /* reflect across the line through the wall edge (a -> b); outward normal
     * of a counter-clockwise triangle's edge a->b is (t_y, -t_x)/|t| */
    int a = t[(k + 1) % 3], b = t[(k + 2) % 3];
    double xa = m->xy[2 * a], ya = m->xy[2 * a + 1];
    double tx = m->xy[2 * b] - xa, ty = m->xy[2 * b + 1] - ya;
    double len = sqrt(tx * tx + ty * ty);
    double nx = ty / len, ny = -tx / len;
    double d = (x - xa) * nx + (y - ya) * ny;
    x = x - 2.0 * d * nx;
    y = y - 2.0 * d * ny;
    if (nb == OR_NBR_NOSLIP) {
      /* no-slip wall: the position is reflected, the velocity is reset by the
       * wall condition in or_step */
      info->status |= OR_TRK_NOSLIP;
    } else if (u && v) {
      double un = (*u) * nx + (*v) * ny;
      *u = *u - 2.0 * un * nx;
      *v = *v - 2.0 * un * ny;
    }
    info->reflections++;
  }
  info->walk_steps = steps;
  *px = x; *py = y;
  return e;
}

/* Brute force: first element (lowest id) whose closed triangle holds the point. */
int or_locate_brute(const or_mesh* m, double x, double y) {
  for (int f = 0; f < m->n_tri; ++f) {
    double N[3];
    or_subareas(m, f, x, y, N);
    if (or_inside(N)) return f;
  }
  return -1;
}

/* ------------------------------------------------------------------------ */
/* Particle initialisation, sec. 3.6 (setup phase): an equal number of       */
/* particles (or a given number) uniformly in each element; velocities       */
/* Gaussian, frequencies Gamma with unit mean and variance 1/4, scalar 0.    */
/* Particle ids run element by element.                                      */
/* Draws (purpose INIT, counter (pid, 0, block, 1)):                          */
/*   block 0: words 0,1 -> barycentric (r1, r2), reflected into the triangle */
/*            if r1 + r2 > 1; words 2,3 -> Gaussians g0, g1                   */
/*   block 1: Gaussians g2..g5 (g2 used)                                      */
/*   block 2: four uniforms; omega = -theta * sum ln u_i: Gamma(k=4, theta)   */
/*            (sum of 4 exponentials), theta = 1/4: mean 1, variance 1/4.     */
/* u_profile 1: mean U = 1 - y^2 (channel); 2: uniform U = 1; 0: zero mean.   */
/* ------------------------------------------------------------------------ */
void or_init(const or_mesh* m, const int* count, uint64_t seed, int u_profile, double u_sigma,
             const double* elem_psi0, double* x, double* y, double* u, double* v, double* w,
             double* om, double* ps, int* elem) {
  long p = 0;
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (int e = 0; e < m->n_tri; ++e) {
    const int* t = m->tri + 3 * e;
    double xa = m->xy[2 * t[0]], ya = m->xy[2 * t[0] + 1];
    double xb = m->xy[2 * t[1]], yb = m->xy[2 * t[1] + 1];
    double xc = m->xy[2 * t[2]], yc = m->xy[2 * t[2] + 1];
    for (int j = 0; j < count[e]; ++j, ++p) {
      uint32_t ctr[4] = {(uint32_t)p, 0u, 0u, OR_PURPOSE_INIT};
      uint32_t wd[4];
      or_philox(ctr, key, wd);
      float r1 = or_u01(wd[0]), r2 = or_u01(wd[1]);
      if (r1 + r2 > 1.0f) { r1 = 1.0f - r1; r2 = 1.0f - r2; }
      float g[6];
      or_box_muller(or_u01(wd[2]), or_u01(wd[3]), &g[0], &g[1]);
      or_gauss4(seed, (uint32_t)p, 0u, 1u, OR_PURPOSE_INIT, &g[2]);
      ctr[2] = 2u;
      or_philox(ctr, key, wd);
      float lsum = or_logf(or_u01(wd[0])) + or_logf(or_u01(wd[1]));
      lsum = lsum + or_logf(or_u01(wd[2]));
      lsum = lsum + or_logf(or_u01(wd[3]));
      double R1 = (double)r1, R2 = (double)r2;
      x[p] = xa + R1 * (xb - xa) + R2 * (xc - xa);
      y[p] = ya + R1 * (yb - ya) + R2 * (yc - ya);
      double umean = (u_profile == 1) ? 1.0 - y[p] * y[p] : (u_profile == 2 ? 1.0 : 0.0);
      u[p] = umean + u_sigma * (double)g[0];
      v[p] = u_sigma * (double)g[1];
      w[p] = u_sigma * (double)g[2];
      om[p] = -0.25 * (double)lsum;
      ps[p] = elem_psi0 ? elem_psi0[e] : 0.0;
      elem[p] = e;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Eulerian statistics, sec. 3.3: element pass then node pass.               */
/* Element stats layout (13): N, <U>, <V>, <W>, <omega>, <phi>,              */
/*   <uu>, <vv>, <ww>, <uv>, <uw>, <vw>, <phi'^2>.                           */
/* Node stats layout (12): the same without N.                               */
/* ------------------------------------------------------------------------ */
enum { OR_NES = 13, OR_NNS = 12 };

/* First pass over the particles of each element: means (1/N sums); second
 * pass: central moments about those means with 1/N (sec. 3.3).  Particles
 * are visited in id order.  An empty element gets N = 0 and zeros. */
void or_elem_stats(int n_tri, long n_p, const int* elem, const double* u, const double* v,
                   const double* w, const double* om, const double* ps, double* es) {
  memset(es, 0, sizeof(double) * OR_NES * n_tri);
  for (long p = 0; p < n_p; ++p) {
    double* s = es + OR_NES * elem[p];
    s[0] += 1.0; s[1] += u[p]; s[2] += v[p]; s[3] += w[p]; s[4] += om[p]; s[5] += ps[p];
  }
  for (int e = 0; e < n_tri; ++e) {
    double* s = es + OR_NES * e;
    if (s[0] > 0.0) for (int q = 1; q <= 5; ++q) s[q] /= s[0];
  }
  for (long p = 0; p < n_p; ++p) {
    double* s = es + OR_NES * elem[p];
    double du = u[p] - s[1], dv = v[p] - s[2], dw = w[p] - s[3], dp = ps[p] - s[5];
    s[6] += du * du; s[7] += dv * dv; s[8] += dw * dw;
    s[9] += du * dv; s[10] += du * dw; s[11] += dv * dw; s[12] += dp * dp;
  }
  for (int e = 0; e < n_tri; ++e) {
    double* s = es + OR_NES * e;
    if (s[0] > 0.0) for (int q = 6; q < OR_NES; ++q) s[q] /= s[0];
  }
}

/* ------------------------------------------------------------------------ */
/* Velocity-conditioned scalar mean for the IECM model (eq. IECM), by the    */
/* sort-and-divide binning of the section on conditional statistics and its  */
/* appendix: the particles of an element are sorted by U and divided into    */
/* groups of equal count (up to one), each group sorted by V and divided,    */
/* each subgroup sorted by W and divided; the conditional mean of a particle  */
/* is the scalar mean of its final subgroup.                                  */
/* READINGS: a group of n particles is divided into k = min(n_c, n / m_min)   */
/* parts (at least 1), part j holding sorted positions with floor(k i / n) =  */
/* j (the appendix's bin index, equal counts up to one); m_min = 2 unless     */
/* given ("at least 2 particles should remain in every subgroup"); equal     */
/* velocity components are ordered by particle id; sorts use the stored      */
/* values.                                                                   */
/* ------------------------------------------------------------------------ */
static const double* or_sort_key;  /* component array the comparator reads */
static const int* or_sort_pid;
static int or_cmp_comp(const void* a, const void* b) {
  const long i = *(const long*)a, j = *(const long*)b;
  const double ki = or_sort_key[i], kj = or_sort_key[j];
  if (ki < kj) return -1;
  if (ki > kj) return 1;
  const int pi = or_sort_pid ? or_sort_pid[i] : (int)i, pj = or_sort_pid ? or_sort_pid[j] : (int)j;
  return (pi > pj) - (pi < pj);
}

/* Sorts idx[0..n) by component `level` (0 U, 1 V, 2 W) and divides it;
 * recursion into the parts for the next component; at the last level the
 * parts are the conditioning bins: cond[p] = the bin's scalar mean. */
static void or_iecm_divide(long* idx, long n, int level, const int nc[3], int m_min, const double* comp[3],
                           const int* pid, const double* ps, double* cond) {
  if (level == 3) {
    double s = 0.0;
    for (long i = 0; i < n; ++i) s += ps[idx[i]];
    const double mean = s / (double)n;
    for (long i = 0; i < n; ++i) cond[idx[i]] = mean;
    return;
  }
  or_sort_key = comp[level];
  or_sort_pid = pid;
  qsort(idx, (size_t)n, sizeof(long), or_cmp_comp);
  long k = n / m_min;
  if (k > nc[level]) k = nc[level];
  if (k < 1) k = 1;
  long start = 0;
  for (long j = 0; j < k; ++j) {
    /* part j: positions i with floor(k i / n) == j, i.e. [ceil(j n / k), ceil((j + 1) n / k)) */
    const long end = ((j + 1) * n + k - 1) / k;
    or_iecm_divide(idx + start, end - start, level + 1, nc, m_min, comp, pid, ps, cond);
    start = end;
  }
}

void or_iecm_cond(int n_tri, long n_p, const int* elem, const double* u, const double* v, const double* w,
                  const double* ps, const int* pid, int nu, int nv, int nw, int m_min, double* cond) {
  const int nc[3] = {nu, nv, nw};
  const double* comp[3] = {u, v, w};
  long* cnt = (long*)calloc((size_t)n_tri + 1, sizeof(long));
  long* idx = (long*)malloc(sizeof(long) * (size_t)(n_p > 0 ? n_p : 1));
  for (long p = 0; p < n_p; ++p) cnt[elem[p] + 1]++;
  for (int e = 0; e < n_tri; ++e) cnt[e + 1] += cnt[e];
  long* fill = (long*)malloc(sizeof(long) * ((size_t)n_tri + 1));
  memcpy(fill, cnt, sizeof(long) * ((size_t)n_tri + 1));
  for (long p = 0; p < n_p; ++p) idx[fill[elem[p]]++] = p;  /* particles of each element in index order */
  for (int e = 0; e < n_tri; ++e)
    if (cnt[e + 1] > cnt[e]) or_iecm_divide(idx + cnt[e], cnt[e + 1] - cnt[e], 0, nc, m_min, comp, pid, ps, cond);
  free(fill);
  free(idx);
  free(cnt);
}

/* Second pass (sec. 3.3): node value = average over the non-empty elements
 * surrounding the node (READING: unweighted; a periodic twin pair is one
 * node; a node whose surrounding elements are all empty keeps its previous
 * value, ns holds it on entry).  Returns the number of such nodes. */
int or_node_stats(const or_mesh* m, const double* es, double* ns) {
  int kept = 0;
  for (int n = 0; n < m->n_nodes; ++n) {
    double acc[OR_NNS] = {0};
    int c = 0;
    for (int i = m->nse_off[n]; i < m->nse_off[n + 1]; ++i) {
      const double* s = es + OR_NES * m->nse[i];
      if (s[0] <= 0.0) continue;
      for (int q = 0; q < OR_NNS; ++q) acc[q] += s[q + 1];
      c++;
    }
    if (c == 0) { kept++; continue; }
    for (int q = 0; q < OR_NNS; ++q) ns[OR_NNS * n + q] = acc[q] / c;
  }
  return kept;
}

/* ------------------------------------------------------------------------ */
/* Derivatives, sec. 3.4: the analytic shape-function derivatives of a       */
/* linear triangle (eq. after eq. gradient), constant over the element.      */
/* ------------------------------------------------------------------------ */
void or_shape_derivs(const or_mesh* m, int e, double dNdx[3], double dNdy[3]) {
  const int* t = m->tri + 3 * e;
  double xa = m->xy[2 * t[0]], ya = m->xy[2 * t[0] + 1];
  double xb = m->xy[2 * t[1]], yb = m->xy[2 * t[1] + 1];
  double xc = m->xy[2 * t[2]], yc = m->xy[2 * t[2] + 1];
  double yCA = yc - ya, yBA = yb - ya, xCA = xc - xa, xBA = xb - xa;
  double twoA = 2.0 * m->area[e];
  dNdx[0] = (-yCA + yBA) / twoA; dNdx[1] = yCA / twoA; dNdx[2] = -yBA / twoA;
  dNdy[0] = (xCA - xBA) / twoA;  dNdy[1] = -xCA / twoA; dNdy[2] = xBA / twoA;
}

/* Mean of the frequency given to a particle striking a no-slip wall (eq.
 * frequency-wallstats): <omega> = (1/C_T) d sqrt(2k)/dn along the normal into
 * the fluid, from the element gradient (eq. gradient) of the nodal sqrt(2k) =
 * sqrt(<uu> + <vv> + <ww>).  READING: where that is not positive (no growth
 * of k away from the wall yet) the element average of the nodal <omega> is
 * used.  out[e] = 0 for elements away from no-slip walls. */
void or_noslip_omega(const or_mesh* m, const double* ns, double* out) {
  for (int e = 0; e < m->n_tri; ++e) {
    out[e] = 0.0;
    if (!m->nsw_flag[e]) continue;
    double dNdx[3], dNdy[3];
    or_shape_derivs(m, e, dNdx, dNdy);
    const double nx = m->nsw[4 * e + 2], ny = m->nsw[4 * e + 3];
    double g = 0.0, om = 0.0;
    for (int j = 0; j < 3; ++j) {
      const double* S = ns + OR_NNS * m->tri[3 * e + j];
      double kk = S[5] + S[6] + S[7];
      g += sqrt(kk > 0.0 ? kk : 0.0) * (dNdx[j] * nx + dNdy[j] * ny);
      om += S[3];
    }
    double w = g / OR_CT;
    out[e] = (w > 0.0) ? w : om / 3.0;
  }
}

/* Gradient of nodal fields q[n*stride + off] over each element (eq.
 * gradient), then averaged at nodes over all surrounding elements (twins
 * merged).  gx, gy: node outputs [n_nodes]. */
static void or_node_gradient(const or_mesh* m, const double* q, int stride, int off,
                             double* gx, double* gy) {
  double* ex = (double*)malloc(sizeof(double) * m->n_tri);
  double* ey = (double*)malloc(sizeof(double) * m->n_tri);
  for (int e = 0; e < m->n_tri; ++e) {
    double dNdx[3], dNdy[3];
    or_shape_derivs(m, e, dNdx, dNdy);
    double sx = 0.0, sy = 0.0;
    for (int j = 0; j < 3; ++j) {
      double qj = q[(long)m->tri[3 * e + j] * stride + off];
      sx += dNdx[j] * qj;
      sy += dNdy[j] * qj;
    }
    ex[e] = sx; ey[e] = sy;
  }
  for (int n = 0; n < m->n_nodes; ++n) {
    double sx = 0.0, sy = 0.0;
    int c = m->nse_off[n + 1] - m->nse_off[n];
    for (int i = m->nse_off[n]; i < m->nse_off[n + 1]; ++i) { sx += ex[m->nse[i]]; sy += ey[m->nse[i]]; }
    gx[n] = c ? sx / c : 0.0;
    gy[n] = c ? sy / c : 0.0;
  }
  free(ex); free(ey);
}

/* Node derivative fields (sec. 3.4, two-pass second derivatives):
 *   nd[n][0..5] = dU/dx, dU/dy, dV/dx, dV/dy, dW/dx, dW/dy
 *   nd[n][6..8] = laplacian of <U>, <V>, <W> (gradient of the node-averaged
 *                 gradient, averaged at nodes again)
 *   nd[n][9]    = d<vv>/dy (channel cross-stream mean-momentum balance) */
enum { OR_NND = 10 };
void or_node_derivs(const or_mesh* m, const double* ns, double* nd) {
  int nn = m->n_nodes;
  double* gx = (double*)malloc(sizeof(double) * nn);
  double* gy = (double*)malloc(sizeof(double) * nn);
  double* hx = (double*)malloc(sizeof(double) * nn);
  double* hy = (double*)malloc(sizeof(double) * nn);
  for (int i = 0; i < 3; ++i) {
    or_node_gradient(m, ns, OR_NNS, i, gx, gy);
    for (int n = 0; n < nn; ++n) { nd[OR_NND * n + 2 * i] = gx[n]; nd[OR_NND * n + 2 * i + 1] = gy[n]; }
  }
  for (int i = 0; i < 3; ++i) {
    /* d/dx of dU_i/dx and d/dy of dU_i/dy */
    or_node_gradient(m, nd, OR_NND, 2 * i, gx, gy);
    or_node_gradient(m, nd, OR_NND, 2 * i + 1, hx, hy);
    for (int n = 0; n < nn; ++n) nd[OR_NND * n + 6 + i] = gx[n] + hy[n];
  }
  or_node_gradient(m, ns, OR_NNS, 6, gx, gy);  /* <vv> */
  for (int n = 0; n < nn; ++n) nd[OR_NND * n + 9] = gy[n];
  free(gx); free(gy); free(hx); free(hy);
}

/* ------------------------------------------------------------------------ */
/* Closure at the nodes.                                                      */
/* ------------------------------------------------------------------------ */
enum { OR_CLOSURE_GLM = 0, OR_CLOSURE_SLM = 1 };
enum { OR_TM_TURB = 0, OR_TM_CPHI = 1 };
enum { OR_PRESSURE_NONE = 0, OR_PRESSURE_CHANNEL = 1, OR_PRESSURE_PROJECTION = 2, OR_PRESSURE_PROJECTION_INOUT = 3 };

enum { OR_TM_SOURCE = 2 };
typedef struct {
  double dt, nu, Pi, c_phi;
  int closure, tm_mode, pressure;
  double src_x, src_y, src_r;  /* point source (src_r > 0: particles inside get psi = 1) */
} or_params;
/* micromixing constants of the concentrated-source form (table of constants, ch. 5) */
static const double OR_CS = 0.02, OR_CTT = 0.7;

/* Right-hand side of the elliptic relaxation equation (eq. elliptic-
 * relaxation-Lagrangian): (1-C1)/2 k<omega> delta_ij + k H_ijkl d<U_k>/dx_l
 * with H (eq. H), A_v (eq. after H) and b_ij (eq. bij).  dU[k][l] holds
 * d<U_k>/dx_l with l = 0, 1 (d/dz = 0 in 2-D). */
void or_relax_rhs(const double* S /*12 node stats*/, const double* D /*node derivs*/, double rhs[9]) {
  double R[3][3] = {{S[5], S[8], S[9]}, {S[8], S[6], S[10]}, {S[9], S[10], S[7]}};
  double k = 0.5 * (S[5] + S[6] + S[7]);
  double kg = k > OR_KFLOOR ? k : OR_KFLOOR;
  double om = S[3];
  double dU[3][3] = {{D[0], D[1], 0.0}, {D[2], D[3], 0.0}, {D[4], D[5], 0.0}};
  double detR = R[0][0] * (R[1][1] * R[2][2] - R[1][2] * R[2][1])
              - R[0][1] * (R[1][0] * R[2][2] - R[1][2] * R[2][0])
              + R[0][2] * (R[1][0] * R[2][1] - R[1][1] * R[2][0]);
  double tk = 2.0 * kg / 3.0;
  double Av = OR_CV * detR / (tk * tk * tk);
  if (Av > 1.0) Av = 1.0;
  double b[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) b[i][j] = R[i][j] / (2.0 * kg) - (i == j ? 1.0 / 3.0 : 0.0);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double h = 0.0;
      for (int kk = 0; kk < 3; ++kk)
        for (int l = 0; l < 3; ++l) {
          double H = (OR_C2 * Av + OR_GAMMA5 / 3.0) * (i == kk) * (j == l)
                   - (OR_GAMMA5 / 3.0) * (i == l) * (j == kk)
                   + OR_GAMMA5 * b[i][kk] * (j == l)
                   - OR_GAMMA5 * b[i][l] * (j == kk);
          h += H * dU[kk][l];
        }
      rhs[3 * i + j] = (i == j ? 0.5 * (1.0 - OR_C1) * kg * om : 0.0) + kg * h;
    }
}

/* Node coefficient set (26), the quantities a particle sees (element-
 * averaged afterwards):
 *   0-2  <U_i>
 *   3-8  d<U_i>/dx_j (i = U,V,W; j = x,y)
 *   9-11 a_i = -d<P>/dx_i + 2 nu lap<U_i>   (GLM, eq. Lagrangian-model);
 *             -d<P>/dx_i                   (SLM, eq. Lagrangian-model-wf)
 *   12-20 G_ij: eq. GandC from wp (GLM) or eq. wall-GandC (SLM)
 *   21   sqrt(C0 eps)
 *   22   <omega>
 *   23   S_omega = C_omega2 - C_omega1 P/eps (eq. frequency-source),
 *        P = -<u_i u_j> d<U_i>/dx_j
 *   24   <phi>
 *   25   1/t_m, t_m = max(k/eps, C_T sqrt(nu/eps)) (the turbulence part of
 *        eq. micromixing-timescale-channel), or 2/(C_phi <omega>)
 * eps: eq. dissipation-from-frequency_wall (GLM), eq. dissipation-from-
 * frequency (SLM).  Mean pressure (READING for the periodic channel, sec.
 * 4.2.1): -d<P>/dx = Pi imposed, -d<P>/dy = d<v^2>/dy; with the pressure
 * projection (sec. 3.2): -d<P>/dx_i = Pi delta_i1 - gp_i, gp the nodal
 * gradient of the projected field (NULL: zero); with the inflow/outflow
 * condition of the canyon -d<P>/dx_i = -gp_i.
 * wp: the 9 node values of the elliptic-relaxation tensor, or NULL for the
 * local model (wp = right-hand side, elliptic term dropped). */
void or_node_coeff(const double* S, const double* D, const double* wp_in, const or_params* P,
                   const double* xy, const double* gp, double* c) {
  double k = 0.5 * (S[5] + S[6] + S[7]);
  double kg = k > OR_KFLOOR ? k : OR_KFLOOR;
  double om = S[3];
  double eps = (P->closure == OR_CLOSURE_SLM) ? k * om : om * (k + P->nu * OR_CT * OR_CT * om);
  double eg = eps > OR_EFLOOR ? eps : OR_EFLOOR;
  for (int i = 0; i < 3; ++i) c[i] = S[i];
  for (int i = 0; i < 6; ++i) c[3 + i] = D[i];
  double dpx = 0.0, dpy = 0.0;  /* -d<P>/dx, -d<P>/dy */
  if (P->pressure == OR_PRESSURE_CHANNEL) { dpx = P->Pi; dpy = D[9]; }
  if (P->pressure == OR_PRESSURE_PROJECTION) {
    dpx = P->Pi - (gp ? gp[0] : 0.0);
    dpy = -(gp ? gp[1] : 0.0);
  }
  if (P->pressure == OR_PRESSURE_PROJECTION_INOUT) {  /* the drop comes through the field */
    dpx = -(gp ? gp[0] : 0.0);
    dpy = -(gp ? gp[1] : 0.0);
  }
  if (P->closure == OR_CLOSURE_SLM) {
    c[9] = dpx; c[10] = dpy; c[11] = 0.0;
    double g = -(0.5 + 0.75 * OR_C0_SLM) * om;
    for (int i = 0; i < 9; ++i) c[12 + i] = (i % 4 == 0) ? g : 0.0;
    c[21] = sqrt(OR_C0_SLM * (eps > 0.0 ? eps : 0.0));
  } else {
    c[9] = dpx + 2.0 * P->nu * D[6];
    c[10] = dpy + 2.0 * P->nu * D[7];
    c[11] = 2.0 * P->nu * D[8];
    double wp[9];
    if (wp_in) for (int i = 0; i < 9; ++i) wp[i] = wp_in[i];
    else or_relax_rhs(S, D, wp);
    double R[9] = {S[5], S[8], S[9], S[8], S[6], S[10], S[9], S[10], S[7]};
    double wr = 0.0;
    for (int i = 0; i < 9; ++i) wr += wp[i] * R[i];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) c[12 + 3 * i + j] = (wp[3 * i + j] - (i == j ? 0.5 * eg : 0.0)) / kg;
    double C0 = -2.0 * wr / (3.0 * kg * eg);
    if (C0 < 0.0) C0 = 0.0;  /* READING: realizability needs C0 >= 0 (sec. 2) */
    c[21] = sqrt(C0 * eg);
  }
  c[22] = om;
  double prod = -(S[5] * D[0] + S[8] * D[1] + S[8] * D[2] + S[6] * D[3] + S[9] * D[4] + S[10] * D[5]);
  c[23] = OR_COMEGA2 - OR_COMEGA1 * prod / eg;
  c[24] = S[4];
  if (P->tm_mode == OR_TM_CPHI) {
    c[25] = 0.5 * P->c_phi * om;
  } else {
    double t1 = kg / eg, t2 = OR_CT * sqrt(P->nu / eg);
    double tm = t1 > t2 ? t1 : t2;
    if (P->tm_mode == OR_TM_SOURCE) {
      /* eq. micromixing-timescale-canyon: min(C_s (r0^2/eps)^(1/3) + C_t d/U_c, tm);
       * U_c = |<U>| at the node (READING: floored at 1e-12), d its distance to the source */
      double dx = xy[0] - P->src_x, dy = xy[1] - P->src_y;
      double d = sqrt(dx * dx + dy * dy);
      double uc = sqrt(S[0] * S[0] + S[1] * S[1] + S[2] * S[2]);
      if (uc < 1e-12) uc = 1e-12;
      double ts = OR_CS * cbrt(P->src_r * P->src_r / eg) + OR_CTT * d / uc;
      if (ts < tm) tm = ts;
    }
    c[25] = 1.0 / tm;
  }
}

/* Element-average coefficient rows: the mean of the three nodal values
 * (sec. 3.3: the average of the nodal values is used for all particles in
 * the element; loop (ii) of the table of loop designs).  wp: [9][n_nodes] or
 * NULL; gp: [n_nodes][2] nodal gradient of the projected pressure or NULL. */
enum { OR_NCOEF = 26 };
void or_elem_coeff(const or_mesh* m, const double* ns, const double* nd, const double* wp,
                   const or_params* P, const double* gp, double* rows) {
  double* nc = (double*)malloc(sizeof(double) * OR_NCOEF * m->n_nodes);
  for (int n = 0; n < m->n_nodes; ++n) {
    double w9[9];
    if (wp) for (int i = 0; i < 9; ++i) w9[i] = wp[(long)i * m->n_nodes + n];
    or_node_coeff(ns + OR_NNS * n, nd + OR_NND * n, wp ? w9 : NULL, P, m->xy + 2 * n, gp ? gp + 2 * n : NULL,
                  nc + OR_NCOEF * n);
  }
  for (int e = 0; e < m->n_tri; ++e)
    for (int q = 0; q < OR_NCOEF; ++q) {
      double s = 0.0;
      for (int j = 0; j < 3; ++j) s += nc[OR_NCOEF * m->tri[3 * e + j] + q];
      rows[OR_NCOEF * e + q] = s / 3.0;
    }
  free(nc);
}

/* ------------------------------------------------------------------------ */
/* One particle time step, explicit Euler-Maruyama (sec. 2 summary).         */
/* ------------------------------------------------------------------------ */
/* Gaussians (purpose STEP, counter (pid, step, block, 0)):
 *   block 0 -> g0..g3, block 1 -> g4..g7;
 *   dW_x = g0, dW_y = g1 (position and the d<U_i>/dx_j term, the same dW,
 *   eqs. Lagrangian-position-exact and -velocity-exact), dW'_1..3 = g2, g3,
 *   g4, dW_omega = g5, each times sqrt(dt); g6, g7 unused.
 * Velocity prediction, eq. velocity-prediction; position, eq. Lagrangian-
 * position-exact (SLM: eq. Lagrangian-position-wf, no viscous diffusion),
 * both with time-n values; frequency, eq. frequency-model (READING: the
 * sqrt uses max(omega, 0) and a negative result is reflected, omega -> -omega);
 * scalar, eq. IEM.  Then tracking with wall reflection.
 * rows: element-average coefficients [n_tri][26].  status_out: per-particle
 * tracking status bits (may be NULL); counters: [0] walk steps, [1]
 * reflections, [2] periodic crossings, [3] fallbacks, [4] brute-force,
 * [5] lost, [6] omega reflections, [7] near-face (min sub-area / A_e < 1e-12).
 * pid: the particle id of each entry (NULL: the index), for stepping a
 * subset of particles.  cond: the velocity-conditioned scalar mean of each
 * entry for eq. IECM (NULL: eq. IEM with the element mean). */
/* One particle of or_step (the body of its particle loop); the tracking
 * counts are added to counters[0..7]. */
static void or_step_one(const or_mesh* m, long p, const double* rows, const or_params* P, uint64_t seed,
                        uint32_t step, double sdt, double s2nu, double* x, double* y, double* u, double* v,
                        double* w, double* om, double* ps, int* elem, int* status_out, long* counters,
                        const int* pid, const double* cond, const double* omega_wall) {
  int e = elem[p];
  const double* c = rows + OR_NCOEF * e;
  float g[8];
  uint32_t id = pid ? (uint32_t)pid[p] : (uint32_t)p;
  or_gauss4(seed, id, step, 0u, OR_PURPOSE_STEP, &g[0]);
  or_gauss4(seed, id, step, 1u, OR_PURPOSE_STEP, &g[4]);
  double dWx = sdt * (double)g[0], dWy = sdt * (double)g[1];
  double dWp[3] = {sdt * (double)g[2], sdt * (double)g[3], sdt * (double)g[4]};
  double dWo = sdt * (double)g[5];
  double U[3] = {u[p], v[p], w[p]};
  double Un[3];
  for (int i = 0; i < 3; ++i) {
    double gl = 0.0;
    for (int j = 0; j < 3; ++j) gl += c[12 + 3 * i + j] * (U[j] - c[j]);
    Un[i] = U[i] + c[9 + i] * P->dt
          + s2nu * (c[3 + 2 * i] * dWx + c[4 + 2 * i] * dWy)
          + gl * P->dt
          + c[21] * dWp[i];
  }
  double xn = x[p] + U[0] * P->dt + s2nu * dWx;
  double yn = y[p] + U[1] * P->dt + s2nu * dWy;
  double o = om[p], mo = c[22];
  double on = o - OR_C3 * mo * (o - mo) * P->dt - c[23] * mo * o * P->dt
            + sqrt(2.0 * OR_C3 * OR_C4 * mo * mo * (o > 0.0 ? o : 0.0)) * dWo;
  if (on < 0.0) { on = -on; counters[6]++; }
  /* eq. IEM with the element mean, or eq. IECM with the velocity-conditioned
   * mean of the particle's bin when cond is given */
  double pn = ps[p] - (ps[p] - (cond ? cond[p] : c[24])) * P->dt * c[25];
  /* distances from the no-slip wall before and after the move (sec.
   * no-slip wall-boundary conditions), for particles in elements with a
   * node on such a wall */
  const int near = m->nsw_flag[e];
  double dn = 0.0, d1 = 0.0;
  if (near) {
    const double* L = m->nsw + 4 * e;
    dn = (x[p] - L[0]) * L[2] + (y[p] - L[1]) * L[3];
    d1 = (xn - L[0]) * L[2] + (yn - L[1]) * L[3];
  }
  or_track_info ti;
  int en = or_track(m, e, &xn, &yn, &Un[0], &Un[1], &ti);
  /* wall condition: trajectory (a), behind the wall after the move (the
   * walk reflected the position at a no-slip edge, or d^{n+1} < 0), or
   * trajectory (b), eta < f_w = exp(-d^n d^{n+1} / (nu dt)) (eq. fw,
   * eq. exp-wall-condition); eta is the third word of the step's second
   * random block.  Then U = 0 and omega from a Gamma distribution with
   * the mean of eq. frequency-wallstats and variance C4 <omega>^2 (shape
   * 1/C4 = 4): -<omega>/4 times the sum of the logarithms of the four
   * uniforms of the step's third block. */
  int wall = (ti.status & OR_TRK_NOSLIP) != 0;
  if (near && !wall) {
    if (d1 < 0.0) {
      wall = 1;
    } else {
      uint32_t ctr[4] = {id, step, 1u, OR_PURPOSE_STEP}, key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)}, out[4];
      or_philox(ctr, key, out);
      const double eta = (double)or_u01(out[2]);
      if (eta < exp(-dn * d1 / (P->nu * P->dt))) wall = 1;
    }
  }
  if (wall) {
    Un[0] = Un[1] = Un[2] = 0.0;
    uint32_t ctr[4] = {id, step, 2u, OR_PURPOSE_STEP}, key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)}, out[4];
    or_philox(ctr, key, out);
    float lsum = or_logf(or_u01(out[0])) + or_logf(or_u01(out[1]));
    lsum = lsum + or_logf(or_u01(out[2]));
    lsum = lsum + or_logf(or_u01(out[3]));
    const double mw = omega_wall ? omega_wall[e] : mo;
    on = -0.25 * (mw > 0.0 ? mw : mo) * (double)lsum;
    ti.status |= OR_TRK_NOSLIP;
  }
  counters[0] += ti.walk_steps;
  counters[1] += ti.reflections;
  counters[2] += ti.crossings_periodic;
  if (ti.status & OR_TRK_FALLBACK) counters[3]++;
  if (ti.status & OR_TRK_BRUTE) counters[4]++;
  if (ti.status & OR_TRK_LOST) counters[5]++;
  if (!(ti.status & OR_TRK_LOST) && ti.min_rel < 1e-12) counters[7]++;
  if (status_out) status_out[p] = ti.status | ((ti.min_rel < 1e-12) ? 256 : 0);
  /* READING: fluid re-entering through the inflow carries no scalar */
  if (ti.status & OR_TRK_REINJECT) pn = 0.0;
  /* the concentrated source (ch. 4): particles inside it get psi = 1 */
  if (P->src_r > 0.0 && (xn - P->src_x) * (xn - P->src_x) + (yn - P->src_y) * (yn - P->src_y) <= P->src_r * P->src_r)
    pn = 1.0;
  x[p] = xn; y[p] = yn; u[p] = Un[0]; v[p] = Un[1]; w[p] = Un[2];
  om[p] = on; ps[p] = pn;
  if (!(ti.status & OR_TRK_LOST)) elem[p] = en;
}

void or_step(const or_mesh* m, long n_p, const double* rows, const or_params* P, uint64_t seed,
             uint32_t step, double* x, double* y, double* u, double* v, double* w, double* om,
             double* ps, int* elem, int* status_out, long* counters, const int* pid, const double* cond,
             const double* omega_wall) {
  double sdt = sqrt(P->dt);
  double s2nu = (P->closure == OR_CLOSURE_SLM) ? 0.0 : sqrt(2.0 * P->nu);
  for (int i = 0; i < 8; ++i) counters[i] = 0;
  for (long p = 0; p < n_p; ++p)
    or_step_one(m, p, rows, P, seed, step, sdt, s2nu, x, y, u, v, w, om, ps, elem, status_out, counters, pid,
                cond, omega_wall);
}

/* The same particle loop spread over host threads: the particle-based loop
 * of the paper's loop design (ii) (table of loop designs, sec. 3.9) under
 * OpenMP.  Within a step every particle reads only its own state and its
 * element's coefficients, so the results equal or_step's bit for bit; the
 * threads' counts are summed at the end.  nthreads <= 0: all available.
 * Returns the number of threads used (1 without OpenMP). */
int or_step_threads(const or_mesh* m, long n_p, const double* rows, const or_params* P, uint64_t seed,
                    uint32_t step, double* x, double* y, double* u, double* v, double* w, double* om,
                    double* ps, int* elem, int* status_out, long* counters, const int* pid, const double* cond,
                    const double* omega_wall, int nthreads) {
  double sdt = sqrt(P->dt);
  double s2nu = (P->closure == OR_CLOSURE_SLM) ? 0.0 : sqrt(2.0 * P->nu);
  for (int i = 0; i < 8; ++i) counters[i] = 0;
  int used = 1;
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel num_threads(nthreads)
  {
    long c[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma omp for schedule(static)
    for (long p = 0; p < n_p; ++p)
      or_step_one(m, p, rows, P, seed, step, sdt, s2nu, x, y, u, v, w, om, ps, elem, status_out, c, pid, cond,
                  omega_wall);
#pragma omp critical
    {
      for (int i = 0; i < 8; ++i) counters[i] += c[i];
      used = omp_get_num_threads();
    }
  }
#else
  (void)nthreads;
  for (long p = 0; p < n_p; ++p)
    or_step_one(m, p, rows, P, seed, step, sdt, s2nu, x, y, u, v, w, om, ps, elem, status_out, counters, pid,
                cond, omega_wall);
#endif
  return used;
}

/* ------------------------------------------------------------------------ */
/* Particle redistribution, the more efficient algorithm of App. D (the     */
/* basic idea in App. C, sec. 3.6): the elements sorted by their particle   */
/* count (ascending); for the k-th element of the sorted order with fewer   */
/* than min_npel particles (the critical ones, k = 0, 1, ...) the k-th      */
/* element from the top gives min_npel - n_k of its particles, which take   */
/* the properties (position, U, omega, psi) of the critical element's       */
/* particles in turn (p mod n_k); a particle moved into an empty element    */
/* keeps its properties and is placed uniformly in it.  The counts and the  */
/* element lists are those before any move (the listing regenerates them    */
/* once, at the end).                                                        */
/* READINGS: ties in the sort by element index (a stable sort); "the p-th   */
/* particle of an element" is the one with the p-th smallest particle id;   */
/* the loop stops when the donor from the top would be a critical element   */
/* itself or the same element (k >= n_tri - 1 - k), and a donor gives at    */
/* most all its particles; the uniform point: Philox counter                */
/* (pid, step, 0, purpose REDIST), words 0, 1 as the barycentric (r1, r2)   */
/* of the initialisation.  pid may be NULL (the index).  Returns the number */
/* of particles moved.                                                       */
/* ------------------------------------------------------------------------ */
static const int* g_sort_cnt;
static int cmp_count_index(const void* a, const void* b) {
  const int i = *(const int*)a, j = *(const int*)b;
  if (g_sort_cnt[i] != g_sort_cnt[j]) return g_sort_cnt[i] < g_sort_cnt[j] ? -1 : 1;
  return i < j ? -1 : (i > j ? 1 : 0);
}
static const int* g_sort_pid;
static int cmp_pid(const void* a, const void* b) {
  const long i = *(const long*)a, j = *(const long*)b;
  const long pi = g_sort_pid ? g_sort_pid[i] : i, pj = g_sort_pid ? g_sort_pid[j] : j;
  return pi < pj ? -1 : (pi > pj ? 1 : 0);
}

long or_redistribute(const or_mesh* m, long n, double* x, double* y, double* u, double* v, double* w,
                     double* om, double* ps, int* elem, const int* pid, int min_npel, uint64_t seed,
                     uint32_t step) {
  const int nt = m->n_tri;
  int* cnt = (int*)calloc(nt, sizeof(int));
  for (long p = 0; p < n; ++p) cnt[elem[p]]++;
  long* off = (long*)calloc(nt + 1, sizeof(long));
  for (int e = 0; e < nt; ++e) off[e + 1] = off[e] + cnt[e];
  long* lst = (long*)malloc(sizeof(long) * (n > 0 ? n : 1));
  long* fill = (long*)malloc(sizeof(long) * (nt + 1));
  for (int e = 0; e <= nt; ++e) fill[e] = off[e];
  for (long p = 0; p < n; ++p) lst[fill[elem[p]]++] = p;
  g_sort_pid = pid;
  for (int e = 0; e < nt; ++e) qsort(lst + off[e], (size_t)cnt[e], sizeof(long), cmp_pid);
  int* order = (int*)malloc(sizeof(int) * nt);
  for (int e = 0; e < nt; ++e) order[e] = e;
  g_sort_cnt = cnt;
  qsort(order, (size_t)nt, sizeof(int), cmp_count_index);
  int nce = 0;
  while (nce < nt && cnt[order[nce]] < min_npel) ++nce;
  long moved = 0;
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (int k = 0; k < nce; ++k) {
    if (nt - 1 - k <= k) break;
    const int j = order[k], i = order[nt - 1 - k];
    const int nj = cnt[j], ni = cnt[i];
    int d = min_npel - nj;
    if (d > ni) d = ni;
    for (int q = 0; q < d; ++q) {
      const long pi = lst[off[i] + q];
      if (nj > 0) {
        const long pj = lst[off[j] + q % nj];
        x[pi] = x[pj]; y[pi] = y[pj];
        u[pi] = u[pj]; v[pi] = v[pj]; w[pi] = w[pj];
        om[pi] = om[pj]; ps[pi] = ps[pj];
      } else {
        const uint32_t id = pid ? (uint32_t)pid[pi] : (uint32_t)pi;
        uint32_t ctr[4] = {id, step, 0u, OR_PURPOSE_REDIST}, wd[4];
        or_philox(ctr, key, wd);
        float r1 = or_u01(wd[0]), r2 = or_u01(wd[1]);
        if (r1 + r2 > 1.0f) { r1 = 1.0f - r1; r2 = 1.0f - r2; }
        const int* t = m->tri + 3 * j;
        const double xa = m->xy[2 * t[0]], ya = m->xy[2 * t[0] + 1];
        const double xb = m->xy[2 * t[1]], yb = m->xy[2 * t[1] + 1];
        const double xc = m->xy[2 * t[2]], yc = m->xy[2 * t[2] + 1];
        const double R1 = (double)r1, R2 = (double)r2;
        x[pi] = xa + R1 * (xb - xa) + R2 * (xc - xa);
        y[pi] = ya + R1 * (yb - ya) + R2 * (yc - ya);
      }
      elem[pi] = j;
      ++moved;
    }
  }
  free(cnt); free(off); free(lst); free(fill); free(order);
  return moved;
}

