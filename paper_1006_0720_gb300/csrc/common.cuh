// Internal definitions shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/pdfgb.h"
#include "fx.cuh"

namespace pdfgb {

void set_error(const std::string& msg);
pdf_status fail(pdf_status s, const std::string& msg);
pdf_status cuda_fail(cudaError_t e, const char* what);

#define PDF_CUDA(call)                                          \
  do {                                                          \
    cudaError_t _e = (call);                                    \
    if (_e != cudaSuccess) return ::pdfgb::cuda_fail(_e, #call); \
  } while (0)

#define PDF_LAUNCH_CHECK(name)                                   \
  do {                                                           \
    cudaError_t _e = cudaGetLastError();                         \
    if (_e != cudaSuccess) return ::pdfgb::cuda_fail(_e, name);  \
  } while (0)

constexpr int kNbrWall = -1;
constexpr int kNbrInflow = -3;
constexpr int kNbrOutflow = -4;
constexpr int kNbrNoslip = -5;

// Per-element data the neighbour walk reads: node B, the edge vectors
// C - B and A - B, twice the area, and the three neighbours with their
// periodic shift multipliers.  80 bytes, 16-byte aligned.
struct __align__(16) ElemGeo {
  double xb, yb;    // node B
  double cbx, cby;  // C - B
  double abx, aby;  // A - B
  double two_area;  // 2 A_e
  int32_t nbr[3];   // neighbour across the edge opposite A, B, C
  int8_t shift[3];  // periodic x-shift multipliers for those crossings
  uint8_t reinj;    // bit k: crossing edge k leaves through the outflow
  int32_t nsw;      // 1: a node lies on a no-slip wall (nsw_line holds the wall)
};
static_assert(sizeof(ElemGeo) == 80, "ElemGeo layout");

// The same data for the fixed-point walk: node B in fixed point (56 fraction
// bits), the edge vectors and twice the area as double-floats.
struct __align__(16) FxGeo {
  int64_t xb, yb;
  fx::df cbx, cby, abx, aby, two_area;
  int32_t nbr[3];
  int8_t shift[3];
  uint8_t reinj;
  int32_t nsw;
};
static_assert(sizeof(FxGeo) == 80, "FxGeo layout");

// Fraction bits of the fixed-point particle positions (|x|, |y| < 64).
constexpr int kPosF = 56;

// Coefficient row of the fixed-point kernel (256 B): the element means of
// U, V, W and phi and the scaled coefficients, all as double-floats:
//   c0-5 sqrt(2 nu dt) d<U_i>/dx_j; c6-8 a_i dt; c9-17 G_ij dt;
//   c18 sqrt(C0 eps dt); c19 (C3 + S_w) <w> dt; c20 C3 <w>^2 dt;
//   c21 <w> sqrt(2 C3 C4 dt); c22 dt / t_m; c23-27 unused (zero).
struct __align__(16) FxRow {
  fx::df mean[4];
  fx::df c[28];
};
static_assert(sizeof(FxRow) == 256, "FxRow layout");

// Device-resident mesh.
struct MeshDev {
  int32_t n_nodes = 0, n_tri = 0;
  double period = 0.0;
  double* xy = nullptr;        // [n_nodes][2]
  int32_t* tri = nullptr;      // [n_tri][3]
  ElemGeo* geo = nullptr;      // [n_tri]
  FxGeo* fgeo = nullptr;       // [n_tri]
  double* dN = nullptr;        // [n_tri][6]: dNA/dx dNB/dx dNC/dx dNA/dy dNB/dy dNC/dy
  int32_t* nse_off = nullptr;  // [n_nodes + 1] node -> surrounding elements (twins merged)
  int32_t* nse = nullptr;
  int32_t* esup_off = nullptr; // [n_nodes + 1] node -> elements holding the node
  int32_t* esup = nullptr;
  double* nsw_line = nullptr;  // [n_tri][4] nearest no-slip wall edge: x_a, y_a, normal into the fluid
};

}  // namespace pdfgb

namespace pdfgb {
// The relaxation system over the unknowns (periodic twins merged).
struct RelaxMesh {
  int32_t n_rep = 0;
  int64_t nnz = 0;
  int32_t* rp = nullptr;        // [n_rep + 1] CSR rows
  int32_t* ci = nullptr;        // [nnz] columns (unknown ids)
  double* mval = nullptr;       // [nnz] consistent mass
  int32_t* ctb_off = nullptr;   // [nnz + 1] stiffness contributions per entry
  int32_t* ctb_e = nullptr;     //   element
  double* ctb_k = nullptr;      //   A_e grad N_a . grad N_b
  uint8_t* wall = nullptr;      // [n_rep] 1: free-slip wall node, 2: no-slip wall node
  int32_t* rep_node = nullptr;  // [n_rep] node id of each unknown
  int32_t* node_rep = nullptr;  // [n_nodes] unknown of each node
  double* wall_n = nullptr;     // [n_nodes][2] outward normal of the nearest wall edge
  double* wall_d = nullptr;     // [n_nodes] distance to it
  // wall edges (WALL and NO-SLIP) at each unknown, for the pressure's
  // Neumann load: element, node a, node b; outward normal and length
  int32_t* pw_off = nullptr;    // [n_rep + 1]
  int32_t* pw_e = nullptr;      // [pw_off[n_rep]][3]
  double* pw_n = nullptr;       // [pw_off[n_rep]][3]
};
// Streams, events and staging buffers of pdf_step_host (created at its
// first call): chunks of the caller's arrays are copied by the copy engines
// into two device staging buffers per direction.  At most 7 chunks (at
// least 65,536 particles each): for 15.9M particles with statistics, 5, 7,
// 10 and 14 chunks took 7.2, 7.0, 7.0 and 7.2 ms per call.
constexpr int kHostChunks = 7;
struct HostIo {
  cudaStream_t in = nullptr, out = nullptr;
  cudaEvent_t start = nullptr, done = nullptr;
  cudaEvent_t loaded[kHostChunks] = {}, stepped[kHostChunks] = {};
  cudaEvent_t free_in[2] = {}, free_out[2] = {};
  int64_t cap = 0;                              // particles per staging buffer
  double* stage_in[2] = {nullptr, nullptr};     // [7][cap] FP64
  double* stage_out[2] = {nullptr, nullptr};
  int32_t* stage_ie[2] = {nullptr, nullptr};    // [cap] element ids
  int32_t* stage_oe[2] = {nullptr, nullptr};
};
struct RelaxAmg;
struct RelaxWork {
  int32_t nb = 0;
  // multigrid preconditioner (default) or Jacobi; the hierarchy is built at
  // the first multigrid solve
  bool multigrid = true;
  RelaxAmg* amg = nullptr;
  double *f = nullptr, *L2 = nullptr, *eL2 = nullptr, *aval = nullptr, *diag = nullptr, *g = nullptr;
  double *x = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr;
  double *part = nullptr, *scal = nullptr, *host = nullptr;
  int32_t *ctl = nullptr, *host_ctl = nullptr;  // device control words and their page-locked copy
  // chunks of iterations captured as a CUDA graph on the library's stream
  cudaStream_t cs = nullptr;
  cudaGraphExec_t gx = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  long long graph_launches = 0;
};
void relax_free(RelaxWork& W);
// One linear system of the pressure projection: its unknowns (periodic
// twins merged; with inflow/outflow conditions the inflow and outflow twins
// stay apart and are Dirichlet unknowns), the stiffness matrix K (kval) and
// the matrix the iteration uses (kmask: Dirichlet rows and columns replaced
// by the identity; kmask == kval without them), the wall edges at each
// unknown, the multigrid hierarchy and the captured iteration chunk.
struct Amg;
struct PressSys {
  bool built = false, dirichlet = false, own = false;
  int32_t n = 0;
  int64_t nnz = 0;
  int32_t *rp = nullptr, *ci = nullptr, *rep_node = nullptr, *node_rep = nullptr;
  int32_t *pw_off = nullptr, *pw_e = nullptr;
  double *kval = nullptr, *kmask = nullptr, *pw_n = nullptr;
  int8_t* dir = nullptr;                     // [n] 0 free, 1 inflow, 2 outflow
  double *gw = nullptr, *gw_prev = nullptr;  // wall loads of the new and the current <P'>
  Amg* amg = nullptr;
  cudaGraphExec_t gx = nullptr;
  long long graph_launches = 0;
};
// The pressure projection's work space (allocated on first use); vectors
// are sized for n_nodes unknowns, enough for either system.
struct PressWork {
  PressSys sys[2];             // 0: periodic in x, 1: inflow/outflow conditions
  int32_t last_sys = -1;
  bool persistent = false;     // run the iteration as one persistent cooperative kernel
  int32_t* ctl = nullptr;      // device: done, iterations, max_it, block counters
  int32_t* host_ctl = nullptr; // page-locked copy
  double *b = nullptr, *x = nullptr, *r = nullptr, *z = nullptr;
  double *p = nullptr, *q = nullptr, *part = nullptr, *scal = nullptr, *dP = nullptr, *ge = nullptr;
  float4* gc = nullptr;        // per element -dt grad dP as double-float pairs
  // iteration chunks run as CUDA graphs on the library's own stream
  cudaStream_t cs = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  double* host = nullptr;
};
void press_free(PressWork& W);
// The particle redistribution's work space (allocated on first use).
struct RedistWork {
  int32_t *cnt = nullptr, *k0 = nullptr, *v0 = nullptr, *k1 = nullptr, *v1 = nullptr;
  int32_t *hist = nullptr, *hist_part = nullptr, *dev = nullptr, *host = nullptr;
  int32_t *role = nullptr, *cur = nullptr;
  int64_t* off = nullptr;
};
void redist_free(RedistWork& W);
}  // namespace pdfgb

struct pdf_mesh {
  pdfgb::MeshDev d;
  pdfgb::RelaxMesh rx;
  std::vector<double> wall_d, wall_n;
  // host copies
  std::vector<double> xy;
  std::vector<int32_t> tri, nbr, shift, twin, reinj;
  std::vector<double> area;
  // host copy of the pressure stiffness matrix over the unknowns (the
  // relaxation pattern rp/ci, values sum_e A_e grad N_a . grad N_b)
  std::vector<int32_t> k_rp, k_ci;
  std::vector<double> k_v;
  // x-period, shape-function derivatives [n_tri][6] and, per node, 1 on an
  // INFLOW edge, 2 on an OUTFLOW edge, else 0
  double period = 0.0;
  std::vector<double> dN;
  std::vector<int8_t> inout;
  // statistics-only work space of the mesh-level relaxation solve
  // (pdf_relax_solve), created at its first call
  mutable pdf_particles* solver = nullptr;
};

// Internal coefficient row: 32 doubles (256 B) per element.
//   0-2  <U_i>
//   3-8  sqrt(2 nu dt) d<U_i>/dx_j   (Ux Uy Vx Vy Wx Wy; 0 for SLM)
//   9-11 a_i dt
//   12-20 G_ij dt
//   21   sqrt(C0 eps) sqrt(dt)
//   22   <omega>
//   23   (C3 + S_omega) <omega> dt
//   24   C3 <omega>^2 dt
//   25   <omega> sqrt(2 C3 C4 dt)
//   26   <phi>
//   27   dt / t_m
#define PDFGB_ROW 32

// Particle state in HBM, particle-id order, structure of arrays (8 B per
// value):
//   x, y              64-bit fixed point with kPosF fraction bits: exact
//                     additions and periodic shifts, uniform absolute
//                     resolution 2^-56 over the domain;
//   u, v, w, om, ps   PDF_FP64: double-float pairs (h, l), |l| <= ulp(h)/2,
//                     48 significant bits, the full FP32 exponent range;
//                     PDF_FP32_STATE: FP32 (uf ... psf).
// The public interface reads and writes FP64 in particle-id order; the
// conversions run in pdf_particles_get_state / pdf_particles_set_state.
// Storage order: every `reorder_every` statistics calls the state is
// permuted into the element order of the grouping (so that the particles
// of one element sit together and a warp's row, geometry and state loads
// stay local); pid[i] is the particle id held in slot i (the Philox counter
// and the interface order).
struct pdf_particles {
  const pdf_mesh* mesh = nullptr;
  int64_t n = 0;
  int32_t precision = PDF_FP64;
  uint64_t seed = 0;
  int64_t *x = nullptr, *y = nullptr;
  fx::df *u = nullptr, *v = nullptr, *w = nullptr, *om = nullptr, *ps = nullptr;
  int32_t* elem = nullptr;
  int32_t* pid = nullptr;
  float *uf = nullptr, *vf = nullptr, *wf = nullptr, *omf = nullptr, *psf = nullptr;
  // the other half of each state array for the reordering copy
  int64_t *x2 = nullptr, *y2 = nullptr;
  fx::df *u2 = nullptr, *v2 = nullptr, *w2 = nullptr, *om2 = nullptr, *ps2 = nullptr;
  float *uf2 = nullptr, *vf2 = nullptr, *wf2 = nullptr, *omf2 = nullptr, *psf2 = nullptr;
  int32_t* pid2 = nullptr;
  int32_t reorder_every = 4, since_reorder = 0;
  // IECM (eq. IECM): velocity-conditioned scalar mean per slot, computed by
  // every pdf_estimate_stats while iecm_bins[0] > 0
  fx::df* cond = nullptr;
  float* iecm_scratch_f = nullptr;     // [16 n] working arrays of elements above the shared-memory cap
  int32_t* iecm_scratch_i = nullptr;   // [6 n]
  int32_t iecm_bins[3] = {0, 0, 0}, iecm_min = 2;
  bool have_cond = false;
  double* stage = nullptr;  // [n] FP64 staging for host transfers (allocated on first use)
  float* rows_f32 = nullptr;  // [n_tri][32] coefficient rows in FP32 (same layout as rows)
  // statistics
  double* es = nullptr;    // [n_tri][13]
  double* ns = nullptr;    // [n_nodes][12]
  double* nd = nullptr;    // [n_nodes][10]
  double* eg = nullptr;    // [n_tri][8] element gradients (scratch)
  double* nc = nullptr;    // [n_nodes][26] nodal coefficients (scratch)
  double* rows = nullptr;  // [n_tri][32]
  pdfgb::FxRow* rows_fx = nullptr;  // [n_tri]
  bool have_stats = false;
  // grouping
  int32_t* keys[2] = {nullptr, nullptr};
  int32_t* vals[2] = {nullptr, nullptr};
  int32_t* hist = nullptr;       // [bins][tiles]
  int32_t* hist_part = nullptr;  // scan partials
  int32_t* seg = nullptr;        // [n_tri + 1] segment offsets into the sorted order
  const int32_t* sorted_pid = nullptr;  // storage slot of each sorted position (vals[]), NULL: identity
  int sorted_key_slot = 0;              // keys[] buffer holding the sorted element ids
  int64_t n_tiles = 0;
  int64_t hist_len = 0;
  int32_t n_scan_blocks = 0;
  // counters
  long long* counters = nullptr;  // [16] device
  // elliptic relaxation work space (allocated on first use)
  pdfgb::RelaxWork rx;
  // pressure projection: the nodal field <P'> and its nodal gradient
  // (zero until the first projection), and the solver's work space
  double* pres = nullptr;   // [n_nodes]
  double* gradP = nullptr;  // [n_nodes][2]
  pdfgb::PressWork pw;
  pdfgb::RedistWork rd;
  pdfgb::HostIo hio;
};

namespace pdfgb {
// A handle without particles holding node statistics, derivatives and the
// relaxation work space (the mesh-level solve); the release of any handle
// and of everything it allocated.
pdf_status stats_only_handle(const pdf_mesh* m, pdf_particles** out);
void release_particles(pdf_particles* p);
// Node derivatives (sec. 3.4) from the node statistics in P->ns.
pdf_status node_derivs_from_node_stats(pdf_particles* P, cudaStream_t st);
// The relaxation's nodal right-hand side [9][n_nodes] and L^2 [3][n_nodes]
// for the particle set's current statistics (relax.cu's work space).
pdf_status relax_fields(pdf_particles* P, const pdf_model_params* params, cudaStream_t st, const double** rhs,
                        const double** L2);
// Host-resident state transfers of pdf_step_host (particles.cu): the
// address kernels use for a caller's buffer (NULL for pageable memory);
// the load of particles [beg, beg + cnt) into slots [beg, beg + cnt) (slot =
// particle id; positions outside |x| < 64 counted in *bad) and the store of
// those slots back; the caller's arrays are indexed from io_off (beg for
// the whole arrays, 0 for a staging buffer holding the chunk).
void* state_kernel_view(const void* ptr);
pdf_status host_io_init(pdf_particles* p);
int host_io_blocks();  // grid of each chunk's load and store kernels
pdf_status state_in_range(pdf_particles* p, double* const in[7], const int32_t* ie, int64_t beg, int64_t cnt,
                          unsigned long long* bad, int blocks, cudaStream_t st, int64_t io_off);
pdf_status state_out_range(const pdf_particles* p, double* const out[7], int32_t* oe, int64_t beg, int64_t cnt,
                           int blocks, cudaStream_t st, int64_t io_off);
// The staging buffers of pdf_step_host for chunks of up to cap particles.
pdf_status host_io_stage(pdf_particles* p, int64_t cap);
// Launches through prof_launch are counted and, when timing is enabled,
// bracketed by CUDA events on the launch stream.
void prof_launch(const char* name, cudaStream_t st, void (*launch)(void*), void* ctx);
// Whether per-kernel timing is on; adding launches made by a graph replay
// to the counter; the counter itself.
bool prof_timing();
void prof_count(long long n);
long long prof_launches();
}  // namespace pdfgb

// PDF_KERNEL(name, stream, kernel<<<grid, block, smem, stream>>>(args...));
#define PDF_KERNEL(name, st, ...)                                          \
  do {                                                                     \
    auto _launch = [&]() { __VA_ARGS__; };                                 \
    ::pdfgb::prof_launch(                                                  \
        name, (st), [](void* c) { (*static_cast<decltype(_launch)*>(c))(); }, \
        &_launch);                                                         \
    PDF_LAUNCH_CHECK(name);                                                \
  } while (0)
