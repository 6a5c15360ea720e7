/*
 * pdfgb — the particle time step of the joint velocity-frequency-scalar PDF
 * method on unstructured triangle grids (J. Bakosi, "PDF modeling of
 * turbulent flows on unstructured grids", 2008), as a C-ABI library of
 * hand-written CUDA kernels for one GB300 (sm_103a).
 *
 * Conventions for every entry point:
 *   - Return value: a pdf_status.  Nothing throws or aborts.  On failure
 *     pdf_last_error() returns a message (thread-local, valid until the next
 *     call on the same thread).
 *   - "host" pointers are read (or written) before the call returns.
 *     "device" pointers are caller-owned CUDA global memory on the current
 *     device; they are borrowed for the work enqueued on `stream` and must
 *     stay valid until that work completes.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Work is
 *     enqueued asynchronously; errors raised by the device surface as
 *     PDF_ECUDA at the next call that synchronizes.
 *   - Handles (pdf_mesh, pdf_particles) are library-owned and freed with the
 *     matching *_destroy.  A handle may be used by one thread at a time.
 *   - Particle arrays are structure-of-arrays in particle-id order.
 */
#ifndef PDFGB_H
#define PDFGB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PDF_OK = 0,
  PDF_EINVAL = 1,    /* bad argument: NULL handle, size out of range, inconsistent mesh */
  PDF_ENOMEM = 2,    /* device or host allocation failed */
  PDF_ECUDA = 3,     /* a CUDA runtime call or kernel failed */
  PDF_ELOST = 4,     /* a particle could not be located (counted in pdf_step_info.lost) */
  PDF_ENOTCONV = 5,  /* an iterative solve hit its iteration cap */
  PDF_ENUMERIC = 6,  /* non-finite values found */
  PDF_ESTATE = 7     /* call out of order (e.g. pdf_step before any statistics) */
} pdf_status;

typedef struct pdf_mesh pdf_mesh;
typedef struct pdf_particles pdf_particles;

/* Boundary-edge tags (sec. 3.5: boundary neighbours are tagged).  INFLOW and
 * OUTFLOW edges whose nodes have periodic twins form a periodic pair for the
 * particles' positions (the canyon case of ch. 5 imposes only periodicity on
 * the streamwise positions); a particle leaving through an OUTFLOW edge
 * re-enters as fresh fluid (its scalar is set to 0).  Without twins they are
 * open boundaries and a particle crossing them is reported lost.  WALL is a
 * free-slip reflecting wall.  NOSLIP is a no-slip wall (the section on no-slip
 * wall-boundary conditions): a particle in an element with a node on such a
 * wall gets the wall condition when its move ends behind the wall line
 * (trajectory (a): the position is reflected) or, staying in front of it,
 * with probability f_w = exp(-d^n d^{n+1} / (nu dt)) (eq. fw, trajectory
 * (b); eta = the third word of the step's second Philox block): U = 0 and
 * omega drawn from a Gamma distribution of shape 1/C4 = 4 with the mean of
 * eq. frequency-wallstats (from the third Philox block).  d is measured from
 * the no-slip edge nearest to the element's centroid among those sharing a
 * node with the element.  In the elliptic relaxation NOSLIP nodes take the
 * Dirichlet condition wp_ij = -4.5 eps n_i n_j. */
enum { PDF_TAG_WALL = 1, PDF_TAG_PERIODIC = 2, PDF_TAG_INFLOW = 3, PDF_TAG_OUTFLOW = 4, PDF_TAG_NOSLIP = 5 };

/* Velocity closure.
 * GLM: generalized Langevin model, eq. Lagrangian-model with G_ij and C0 from
 *      the elliptic-relaxation tensor by eq. GandC; eps by eq.
 *      dissipation-from-frequency_wall.
 * SLM: simplified Langevin model with wall functions, eqs.
 *      Lagrangian-position-wf, Lagrangian-model-wf and wall-GandC (C0 = 3.5).
 * FROZEN: the caller supplies the element-average coefficient rows. */
enum { PDF_CLOSURE_GLM = 0, PDF_CLOSURE_SLM = 1, PDF_CLOSURE_FROZEN = 2 };
/* Micromixing time scale: TURB = max(k/eps, C_T sqrt(nu/eps)) (the turbulence
 * part of eq. micromixing-timescale-channel); CPHI = 2/(C_phi <omega>);
 * SOURCE = eq. micromixing-timescale-canyon, min(C_s (r0^2/eps)^(1/3) +
 * C_t d/|<U>|, TURB) with d the node's distance to the source (src_*). */
enum { PDF_TM_TURB = 0, PDF_TM_CPHI = 1, PDF_TM_SOURCE = 2 };
/* Mean pressure gradient in the velocity prediction: NONE (0); CHANNEL,
 * -d<P>/dx = Pi and -d<P>/dy = d<vv>/dy (the channel's cross-stream
 * balance); PROJECTION, -d<P>/dx_i = Pi delta_i1 - d<P'>/dx_i with <P'> the
 * nodal field of pdf_pressure_project (zero until its first call), periodic
 * in x; PROJECTION_INOUT, -d<P>/dx_i = -d<P>/dx_i of the projected field,
 * which carries the imposed drop Pi L_x between the inflow and the outflow
 * through their Dirichlet condition (the street canyon's inflow/outflow
 * condition; see pdf_pressure_project). */
enum { PDF_PRESSURE_NONE = 0, PDF_PRESSURE_CHANNEL = 1, PDF_PRESSURE_PROJECTION = 2,
       PDF_PRESSURE_PROJECTION_INOUT = 3 };
enum { PDF_MIX_IEM = 0, PDF_MIX_IECM = 1 };
/* How the FP64-accurate particle step is computed.  FX (default): no FP64
 * instructions on the fast path -- positions in 64-bit fixed point (exact
 * increments and element tests), velocity, frequency and scalar in
 * double-float FP32 pairs (FMA-exact products, TwoSum additions); particles
 * that move one length unit or more in a step, or whose walk meets a wall,
 * are finished in FP64.  FP64: native FP64 instructions throughout (GB300
 * runs them at ~1/70 of the FP32 rate), on the same stored forms. */
enum { PDF_ARITH_FX = 0, PDF_ARITH_FP64 = 1 };
/* Storage of the particle state on the device.  Positions: 64-bit fixed
 * point with 56 fraction bits (resolution 2^-56, |x|, |y| < 64) in both
 * modes.  PDF_FP64: u, v, w, omega, psi as double-float pairs (48
 * significant bits, relative resolution 2^-48 ~ 3.6e-15, FP32 exponent
 * range).  PDF_FP32_STATE: u, v, w, omega, psi in FP32.  The interface
 * reads and writes FP64 in both modes. */
enum { PDF_FP64 = 0, PDF_FP32_STATE = 1 };

/* Number of element-average coefficients a particle sees (layout below). */
#define PDF_NCOEF 26
/* Element statistics: N, <U>, <V>, <W>, <omega>, <phi>, <uu>, <vv>, <ww>,
 * <uv>, <uw>, <vw>, <phi'^2> (sec. 3.3; central moments with 1/N). */
#define PDF_NES 13
/* Node statistics: the element layout without N. */
#define PDF_NNS 12
/* Node derivatives: dU/dx, dU/dy, dV/dx, dV/dy, dW/dx, dW/dy, lap<U>,
 * lap<V>, lap<W>, d<vv>/dy (sec. 3.4, two-pass second derivatives). */
#define PDF_NND 10

typedef struct {
  double dt;        /* time step */
  double nu;        /* kinematic viscosity */
  double Pi;        /* imposed -d<P>/dx for PDF_PRESSURE_CHANNEL */
  double c_phi;     /* C_phi for PDF_TM_CPHI */
  int32_t closure;  /* PDF_CLOSURE_* */
  int32_t tm_mode;  /* PDF_TM_* */
  int32_t pressure; /* PDF_PRESSURE_* */
  int32_t arith;    /* PDF_ARITH_* */
  /* model constants, table "Constants for modeling the joint PDF of velocity
   * and frequency" (ch. 4), and C0 of eq. wall-GandC */
  double C1, C2, C3, C4, CT, CL, Ceta, Cv, gamma5, Comega1, Comega2, C0_slm;
  /* concentrated scalar source (ch. 4: particles passing through it get
   * psi = 1): centre and radius; src_r = 0 disables it */
  double src_x, src_y, src_r;
  /* micromixing constants C_s, C_t of eq. micromixing-timescale-canyon */
  double Cs, Ct;
  /* micromixing model: PDF_MIX_IEM (eq. IEM, the element mean of <phi>) or
   * PDF_MIX_IECM (eq. IECM, the velocity-conditioned mean of the particle's
   * bin from the last pdf_estimate_stats; needs pdf_particles_set_iecm) */
  int32_t mix;
  int32_t reserved;
} pdf_model_params;

/* Fills the paper's constants and dt = 1e-3, nu = 1e-3, Pi = 2e-3,
 * c_phi = 2, GLM, TURB, CHANNEL, ARITH_FX, no source, C_s = 0.02, C_t = 0.7. */
void pdf_model_params_default(pdf_model_params* p);

typedef struct {
  const int32_t* count;      /* host [n_tri]: particles per element, or NULL to use ppe */
  int32_t ppe;               /* particles per element when count == NULL */
  int32_t u_profile;         /* 0: zero mean velocity; 1: channel profile U = 1 - y^2; 2: U = 1 */
  double u_sigma;            /* standard deviation of each velocity component */
  const double* elem_psi0;   /* host [n_tri]: initial scalar per element, or NULL for 0 */
} pdf_init_params;

/* Per-step counters (filled when pdf_step is given a non-NULL info). */
typedef struct {
  int64_t walk_steps;          /* neighbour-walk steps over all particles */
  int64_t reflections;         /* wall reflections */
  int64_t crossings_periodic;  /* periodic-seam crossings */
  int64_t fallbacks;           /* particles found by the concave-corner fall-back */
  int64_t brute;               /* particles that needed the all-element search */
  int64_t lost;                /* particles not found (state kept, elem unchanged) */
  int64_t omega_reflections;   /* omega < 0 after the Euler-Maruyama step, reflected */
  int64_t near_face;           /* particles within 1e-12 (relative) of an element edge */
} pdf_step_info;

/* ---------------------------------------------------------------- mesh */

/* Builds the element-surrounding-element list with tagged boundary
 * neighbours and the node-surrounding-element lists (sec. 3.3 linked lists,
 * sec. 3.5) on the host and uploads the mesh to the current device.
 *   node_xy  host [n_nodes][2] node coordinates
 *   tri      host [n_tri][3] node ids, counter-clockwise (else PDF_EINVAL)
 *   twin     host [n_nodes] periodic twin node or -1; may be NULL.  Twin
 *            nodes are one node for statistics; edges tagged PERIODIC are
 *            matched to the element holding the twin edge.
 *   bnd_edge host [n_bnd][3] (node a, node b, PDF_TAG_*) for every boundary
 *            edge (an edge with one element).  An untagged boundary edge is
 *            PDF_EINVAL.
 *   period_x the x-period (the shift applied when crossing a PERIODIC edge).
 * Sizes: n_nodes, n_tri >= 1 and < 2^31.  *out receives the handle. */
pdf_status pdf_mesh_create(const double* node_xy, int32_t n_nodes, const int32_t* tri,
                           int32_t n_tri, const int32_t* twin, const int32_t* bnd_edge,
                           int32_t n_bnd, double period_x, pdf_mesh** out);
pdf_status pdf_mesh_destroy(pdf_mesh* m);
/* Host copies of the connectivity (for checking): nbr [n_tri][3] neighbour
 * across the edge opposite local vertex k (>= 0 element, -1 wall, -3 inflow,
 * -4 outflow, -5 no-slip wall); shift [n_tri][3] periodic x-shift
 * multiplier.  Either may be NULL. */
pdf_status pdf_mesh_connectivity(const pdf_mesh* m, int32_t* nbr, int32_t* shift);
pdf_status pdf_mesh_size(const pdf_mesh* m, int32_t* n_nodes, int32_t* n_tri);

/* ---------------------------------------------------------------- particles */

/* Particle initialisation (sec. 3.6): count[e] (or ppe) particles uniform in
 * each element, particle ids element by element; velocity = profile +
 * u_sigma N(0,1) per component; omega ~ Gamma(k=4, theta=1/4) (unit mean,
 * variance 1/4); psi = elem_psi0[e] or 0.  Random numbers: Philox4x32-10
 * keyed by seed, counter (particle id, 0, block, 1).
 * precision: PDF_FP64 or PDF_FP32_STATE (the storage above); anything else
 * is PDF_EINVAL.  Allocates all per-particle and per-mesh device buffers
 * (PDF_ENOMEM if one fails, nothing kept).  The mesh must outlive the
 * particles. */
pdf_status pdf_particles_init(const pdf_mesh* m, const pdf_init_params* ip, uint64_t seed,
                              int32_t precision, void* stream, pdf_particles** out);
pdf_status pdf_particles_destroy(pdf_particles* p);
pdf_status pdf_particles_count(const pdf_particles* p, int64_t* n);
/* Storage order.  Every `every`-th pdf_estimate_stats call (default 4; 0
 * never) copies the state into the element order its grouping computed, so
 * that the particles of one element sit in consecutive slots and the
 * step's coefficient-row and geometry loads, and the statistics' reads,
 * stay local as particles disperse.  The copy needs a second set of state
 * arrays (allocated by pdf_particles_init).  The order is invisible at the
 * interface: particle ids (the random-number counters and the order of
 * pdf_particles_get_state/set_state) move with the particles.  Results
 * depend on it only through the order of the rounded double-float sums of
 * the central moments.  The paper has no counterpart (its particles live
 * in per-element linked lists).  PDF_EINVAL for every < 0. */
pdf_status pdf_particles_set_reorder(pdf_particles* p, int32_t every);
/* IECM conditioning (eq. IECM; the section on conditional statistics and
 * its appendix): while enabled, every pdf_estimate_stats also computes each
 * particle's velocity-conditioned scalar mean by sort-and-divide binning:
 * the particles of an element are sorted by U and divided into nu parts of
 * equal count (up to one), each part sorted by V and divided into nv, each
 * of those sorted by W and divided into nw; a group of n particles is
 * divided into min(n_c, n / m_min) parts (at least one), so every bin keeps
 * m_min particles; equal components are ordered by particle id.  The mean
 * of a particle is its final bin's scalar mean.  nu = nv = nw = 0 disables
 * it.  The first call allocates 8 + 88 bytes per particle (the means and the
 * working arrays of elements with more than 256 particles).  PDF_EINVAL for
 * bins outside [1, 127] (other than all zero) or m_min < 1. */
pdf_status pdf_particles_set_iecm(pdf_particles* p, int32_t nu, int32_t nv, int32_t nw, int32_t m_min);
/* The conditional means of the last pdf_estimate_stats, FP64 [n] in
 * particle-id order (device memory); PDF_ESTATE if there are none. */
pdf_status pdf_iecm_cond(const pdf_particles* p, double* cond, void* stream);

/* Copies the state, converted to FP64, into caller buffers [n] in
 * particle-id order (any pointer may be NULL).  When every given buffer is
 * device, managed or page-locked host memory, one kernel on `stream` writes
 * them all (page-locked memory through its mapping, over the host link, no
 * staging; asynchronous); a pageable host buffer goes through an FP64
 * staging buffer of n doubles that the handle allocates on first use and
 * keeps.  elem: host element id of each particle. */
pdf_status pdf_particles_get_state(const pdf_particles* p, double* x, double* y, double* u,
                                   double* v, double* w, double* om, double* ps, int32_t* elem,
                                   void* stream);
/* Overwrites the state from FP64 caller buffers [n] in particle-id order
 * (all required; device or host memory: one kernel reads them all where
 * they are when none is pageable, else pageable sources go through the
 * staging buffer above), rounding to the stored forms; the slots then
 * follow the particle ids.  Synchronizes `stream`.  A position outside
 * |x|, |y| < 64 is PDF_EINVAL (the state is then undefined).  elem must
 * hold each particle's host element (not checked).  Invalidates the IECM
 * conditioned means until the next pdf_estimate_stats. */
pdf_status pdf_particles_set_state(pdf_particles* p, const double* x, const double* y,
                                   const double* u, const double* v, const double* w,
                                   const double* om, const double* ps, const int32_t* elem,
                                   void* stream);

/* A particle set in a saved byte form, and back: the stored state exactly
 * as it sits in the slots (positions in 64-bit fixed point, velocity,
 * frequency and scalar in the set's storage form, element and particle id
 * of every slot), the statistics of the last pdf_estimate_stats, the IECM
 * conditioned means and settings, the projected pressure field <P'> with
 * its gradient, the reordering interval and counter, and the seed.  A
 * loaded set continues bit for bit where the saved one stood: the same
 * pdf_step / pdf_estimate_stats calls give the same results as on the saved
 * set (the paper's runs restart from saved particle fields; sec. 3.6 and
 * the setup phase of the solver, not a byte format).  Not saved: the
 * relaxation and pressure solvers' work spaces (rebuilt at their next
 * call) and the wall load the current <P'> was projected with (the next
 * pdf_pressure_project starts it from zero, as after pdf_pressure_field).
 * Format (version 1, little-endian, 8-byte aligned sections): an 80-byte
 * header (magic "PDFGBPS\0", version, flags, n, seed, n_tri, n_nodes,
 * precision, reorder interval and counter, IECM bins and minimum), the slot
 * arrays x, y (i64), u, v, w, om, ps (8 B per value for PDF_FP64, 4 B for
 * PDF_FP32_STATE), elem, pid (i32), then the optional sections the flags
 * name (statistics; IECM means; pressure field), then an FNV-1a checksum
 * over the preceding 64-bit words.
 *   size        out: bytes of the saved form of p (pdf_particles_save_size)
 *   buf, cap    host memory (pageable or page-locked) of at least that size;
 *               pdf_particles_save synchronizes `stream`
 * pdf_particles_load checks the magic, version, sizes against the mesh and
 * the buffer, the checksum, that every element id is in range and that the
 * slots' particle ids are a permutation (all on the host, before any device
 * allocation) and returns PDF_EINVAL otherwise; PDF_ENOMEM if the device
 * arrays cannot be allocated.  The new handle is freed with
 * pdf_particles_destroy.  Synchronizes `stream`. */
pdf_status pdf_particles_save_size(const pdf_particles* p, size_t* size);
pdf_status pdf_particles_save(const pdf_particles* p, void* buf, size_t cap, void* stream);
pdf_status pdf_particles_load(const pdf_mesh* m, const void* buf, size_t size, void* stream,
                              pdf_particles** out);

/* ---------------------------------------------------------------- the step */

/* One explicit Euler-Maruyama step of every particle (sec. 2 summary):
 *   velocity prediction, eq. velocity-prediction (SLM: eq. Lagrangian-model-wf);
 *   position, eq. Lagrangian-position-exact with the same dW_j as the
 *     d<U_i>/dx_j term (SLM: eq. Lagrangian-position-wf);
 *   frequency, eq. frequency-model (a negative result is reflected);
 *   scalar, eq. IEM;
 *   then the neighbour walk of sec. 3.5 with periodic seams and reflecting
 *   walls (position mirrored, wall-normal velocity reversed); a particle
 *   that left through an outflow edge gets psi = 0, one inside the source
 *   circle psi = 1.
 * Random numbers: Philox4x32-10 keyed by seed, counter (particle id, step,
 * block, 0), 6 Gaussians per particle (sec. 3.8 draws 6 per particle).
 * Coefficients: for GLM/SLM the element averages of the nodal coefficients
 * computed from the statistics of the last pdf_estimate_stats (sec. 3.3) and,
 * for GLM, from wp; for FROZEN from elem_coeff.
 *   params      host; params->closure selects the model
 *   wp          device [9][n_nodes] elliptic-relaxation tensor at the nodes
 *               (component-major, wp[(3i+j)*n_nodes + n]) or NULL for the
 *               local model (wp = right-hand side of eq. elliptic-relaxation-
 *               Lagrangian); ignored unless GLM
 *   elem_coeff  device [n_tri][PDF_NCOEF] for FROZEN (ignored otherwise):
 *               <U_i>(3), d<U_i>/dx_j (6: Ux Uy Vx Vy Wx Wy), a_i = -d<P>/dx_i
 *               + 2 nu lap<U_i> (3), G_ij row-major (9), sqrt(C0 eps),
 *               <omega>, S_omega, <phi>, 1/t_m
 *   step        the step number (Philox counter word 1)
 *   info        host, may be NULL; when given the call synchronizes `stream`
 *               and fills the counters.  Returns PDF_ELOST if any particle
 *               was lost (the rest of the step is still applied).
 * PDF_ESTATE if GLM/SLM is requested before any pdf_estimate_stats. */
pdf_status pdf_step(pdf_particles* p, const pdf_mesh* m, const pdf_model_params* params,
                    const double* wp, const double* elem_coeff, uint32_t step, void* stream,
                    pdf_step_info* info);
/* pdf_step for a state that lives in host memory: equivalent to
 * pdf_particles_set_state(x ... elem), pdf_step(...) and
 * pdf_particles_get_state(x ... elem) (same results, bit for bit), with the
 * transfers overlapped: the particles are taken in chunks of particle ids
 * (starting on 4 KiB boundaries of the arrays); the copy engines move each
 * chunk's arrays (cudaMemcpyAsync, one call per array and direction) into
 * and out of device staging buffers while the SMs convert and step the
 * previous chunk, so that the host link's two directions and the SMs are
 * busy together.  The staging buffers (two per
 * direction, 60 bytes per particle of a chunk each) are allocated at the
 * first call and kept by the particle set.
 *   x ... ps    page-locked host (or device) [n] FP64, elem [n] int32; read,
 *               then overwritten with the stepped state (in particle-id
 *               order, as pdf_particles_get_state returns it)
 *   other arguments as pdf_step; the counters are always gathered (one
 *               synchronization of `stream` at the end) and filled into
 *               info when given.
 * The particle set keeps the stepped state (slot = particle id) for
 * pdf_estimate_stats.  PDF_EINVAL for pageable host buffers, for positions
 * outside |x|, |y| < 64 and for the IECM mixing model (its conditioned
 * means belong to the device-resident order); PDF_ENOMEM if the staging
 * buffers cannot be allocated; PDF_ELOST if any particle was lost;
 * PDF_ESTATE as pdf_step. */
pdf_status pdf_step_host(pdf_particles* p, const pdf_mesh* m, const pdf_model_params* params, const double* wp,
                         const double* elem_coeff, uint32_t step, double* x, double* y, double* u, double* v,
                         double* w, double* om, double* ps, int32_t* elem, void* stream, pdf_step_info* info);

/* pdf_step_host followed by pdf_estimate_stats, in one call: the same
 * results, bit for bit, as the two calls in sequence, but the statistics of
 * the stepped state start as soon as the last chunk is stepped, while the
 * copy engines still write the last chunks back to the host arrays.
 *   x ... elem  as pdf_step_host (read, then overwritten with the stepped
 *               state)
 *   elem_stats, node_stats, node_derivs  optional copies of the statistics
 *               (NULL for none; device or page-locked host memory, layouts
 *               as pdf_estimate_stats)
 *   other arguments and errors as pdf_step_host; the statistics are kept
 *   for the next step as after pdf_estimate_stats. */
pdf_status pdf_step_host_stats(pdf_particles* p, const pdf_mesh* m, const pdf_model_params* params,
                               const double* wp, const double* elem_coeff, uint32_t step, double* x, double* y,
                               double* u, double* v, double* w, double* om, double* ps, int32_t* elem,
                               double* elem_stats, double* node_stats, double* node_derivs, void* stream,
                               pdf_step_info* info);

/* Particle-in-cell statistics (sec. 3.3) and derivatives (sec. 3.4):
 * groups particles by element (stable radix sort by element id), element
 * means and central moments (two passes, 1/N), node averages over the
 * non-empty surrounding elements (a node with none keeps its previous value),
 * node gradients of the means, second derivatives by the two-pass procedure,
 * and d<vv>/dy.  The library keeps the results for the next pdf_step; the
 * optional outputs receive copies (device or page-locked host memory,
 * layouts PDF_NES / PDF_NNS / PDF_NND per element or node). */
pdf_status pdf_estimate_stats(pdf_particles* p, const pdf_mesh* m, double* elem_stats,
                              double* node_stats, double* node_derivs, void* stream);

/* pdf_estimate_stats for callers that cannot allocate device memory.
 *
 * The paper has no counterpart; this is a service of the library.  Some
 * callers must not call cudaMalloc or cudaFree: a host loop that cannot take
 * the device-wide synchronization those calls may cause, code running where
 * another allocator (an application's memory pool) already owns the device
 * memory budget, or a plugin or callback that is forbidden to allocate.
 * pdf_estimate_stats keeps its grouping scratch in buffers allocated by
 * pdf_particles_init; this variant allocates nothing and instead uses one
 * scratch array of fixed size compiled into the library (about 9.2 MiB, held
 * by every GPU that loads the library until the process exits).
 *
 * Same arguments, results and outputs as pdf_estimate_stats (the statistics
 * are bit-identical to it), with these limits and rules:
 *   - at most PDF_NOALLOC_MAX_PARTICLES particles and PDF_NOALLOC_MAX_ELEMENTS
 *     elements, else PDF_EINVAL with a message naming the limit;
 *   - the first call on each device looks up that device's copy of the
 *     scratch array (with the device current), so make the first call on a
 *     device before any stream capture; the address is kept for the life of
 *     the process, so a device reset (cudaDeviceReset) between calls is not
 *     supported;
 *   - every call shares the one scratch array: calls whose work overlaps on
 *     the GPU (different streams or threads without ordering) race and give
 *     wrong statistics.  The scratch keeps the last call's contents; nothing
 *     in it needs to start at zero. */
#define PDF_NOALLOC_MAX_PARTICLES 524288
#define PDF_NOALLOC_MAX_ELEMENTS 262144
pdf_status pdf_estimate_stats_noalloc(pdf_particles* p, const pdf_mesh* m, double* elem_stats,
                                      double* node_stats, double* node_derivs, void* stream);

/* The element-average coefficient rows [n_tri][PDF_NCOEF] that pdf_step
 * would use for GLM/SLM with this wp (device output). */
pdf_status pdf_elem_coeff(pdf_particles* p, const pdf_mesh* m, const pdf_model_params* params,
                          const double* wp, double* rows, void* stream);

/* ---------------------------------------------------------------- elliptic relaxation */

/* The elliptic-relaxation solve for the tensor wp_ij (eq. elliptic-relaxation-
 * Lagrangian, with eqs. H, A_v, bij, L and Cxi), discretised with linear
 * triangles and solved by preconditioned conjugate gradients in FP64 (sec.
 * 3.2: there Jacobi-preconditioned; here a smoothed-aggregation multigrid
 * V-cycle by default, see pdf_relax_set_solver), all nine components at once:
 *   (M + K_L) wp = M rhs,  M the consistent mass matrix, K_L the stiffness
 *   matrix weighted by the element mean of the nodal L^2.
 * Right-hand side and L from the caller's node statistics (the node
 * derivatives of sec. 3.4 are formed from them, as pdf_estimate_stats
 * does).  Reflecting walls act as symmetry planes: off-diagonal components are 0 on
 * wall nodes, diagonal components have zero normal derivative.  C_xi =
 * 1 + 1.3 n_i n_i for wp_ii with n the outward normal of the nearest wall
 * edge.  Periodic twin nodes share one unknown.
 *   node_stats  device (or page-locked host) [n_nodes][PDF_NNS], the node
 *            layout of pdf_estimate_stats (<U>, <V>, <W>, <omega>, <phi>,
 *            <uu>, <vv>, <ww>, <uv>, <uw>, <vw>, <phi'^2>); read on `stream`
 *   wp       device [9][n_nodes] (component-major, wp[(3i+j)*n_nodes + n]);
 *            in: the initial guess (warm start), out: the solution
 *   rtol     stop a component when ||r|| <= rtol ||b|| (b = M rhs)
 *   max_it   iteration cap; PDF_ENOTCONV if a component is not converged
 *   iters, rel_res  host [9] or NULL: iterations and final ||r||/||b||
 * Multigrid-preconditioned (the default of pdf_relax_set_solver).  The work
 * space (node statistics and derivatives, the CG vectors, the multigrid
 * hierarchy) belongs to the mesh handle and is allocated at the first call
 * (the hierarchy's host set-up then takes about 0.3 s for 80,000 nodes);
 * calls on one mesh must not overlap.  PDF_EINVAL for NULL arguments, rtol
 * <= 0 or max_it < 0; PDF_ENOMEM if the work space cannot be allocated.
 * The call synchronizes `stream` once per 8 iterations (convergence test). */
pdf_status pdf_relax_solve(const pdf_mesh* m, const pdf_model_params* params, const double* node_stats,
                           double* wp, double rtol, int32_t max_it, int32_t* iters, double* rel_res, void* stream);
/* The same solve for the node statistics of a particle set's last
 * pdf_estimate_stats (no copy), with the particle handle's own work space
 * and preconditioner choice (pdf_relax_set_solver).  PDF_ESTATE before the
 * first pdf_estimate_stats; otherwise as pdf_relax_solve. */
pdf_status pdf_relax_solve_particles(pdf_particles* p, const pdf_mesh* m, const pdf_model_params* params,
                                     double* wp, double rtol, int32_t max_it, int32_t* iters, double* rel_res,
                                     void* stream);
/* The preconditioner of pdf_relax_solve_particles: multigrid = 1 (the default) a
 * smoothed-aggregation V-cycle whose prolongations come from the mesh's
 * stiffness matrix (built at the first solve) and whose level matrices are
 * the Galerkin products of the current relaxation matrices (recomputed on
 * the device at every solve; four operators: wp_11, wp_22, wp_33 and the
 * off-diagonal components, each with its own fixed unknowns); multigrid = 0
 * the diagonal (Jacobi) of the paper.  Both converge to the same tolerance;
 * the solve falls back to Jacobi when the hierarchy cannot be built.  The
 * first multigrid solve builds the hierarchy on the host from the mesh's
 * pattern (about 0.3 s for 80,000 nodes); it is kept across switches.
 * Synchronizes the device when the choice changes.  PDF_EINVAL for other
 * values. */
pdf_status pdf_relax_set_solver(pdf_particles* p, int32_t multigrid);
/* The nodal right-hand side rhs [9][n_nodes] and L^2 [3][n_nodes] (C_xi of
 * wp_11, of wp_22, and 1) that pdf_relax_solve_particles uses (device or page-locked
 * host outputs; either may be NULL). */
pdf_status pdf_relax_rhs(pdf_particles* p, const pdf_mesh* m, const pdf_model_params* params, double* rhs,
                         double* L2, void* stream);
/* Host copies of each node's distance to the nearest wall edge [n_nodes] and
 * that edge's unit outward normal [n_nodes][2]; either may be NULL. */
pdf_status pdf_mesh_wall_distance(const pdf_mesh* m, double* dist, double* normal);

/* ---------------------------------------------------------------- particle redistribution */

/* Particle redistribution (the more efficient algorithm of App. D; its idea
 * in App. C and sec. 3.6), typically after pdf_step and before
 * pdf_estimate_stats: the elements are sorted by their particle count
 * (ties by element index); the k-th element with fewer than min_npel
 * particles (k = 0, 1, ...) receives min_npel - n_k particles from the k-th
 * element from the top (at most all of them; it stops where the donor
 * would be a critical element itself).  The moved particles are the
 * donor's lowest particle ids; they copy the position, U, omega and psi of
 * the receiving element's particles in turn (donor particle p copies the
 * receiving element's particle p mod n_k, ordered by particle id), or, into
 * an empty element, keep their values and are placed uniformly in it
 * (Philox4x32-10 keyed by seed, counter (particle id, step, 0, 2); words 0,
 * 1 as the initialisation's barycentric (r1, r2)).  Particle ids (the
 * random streams) stay with the moved particles.
 *   min_npel in [1, 64], else PDF_EINVAL
 *   moved    host or NULL: the number of particles moved
 * Synchronizes `stream`.  The statistics must be estimated again before
 * the next step (PDF_ESTATE otherwise). */
pdf_status pdf_redistribute(pdf_particles* p, const pdf_mesh* m, int32_t min_npel, uint64_t seed, uint32_t step,
                            int32_t* moved, void* stream);

/* ---------------------------------------------------------------- pressure projection */

/* The stabilised pressure projection (sec. 3.2: eqs. velocity-prediction,
 * pressure-projection-smooth, velocity-correction) after a step whose
 * statistics have been estimated (the particles hold U*):
 *   grad^2 dP = (div <U*> - C_p grad^2 <P'>^n) / dt,   dP = <P'>^{n+1} - <P'>^n,
 * with linear triangles, periodic twins one unknown:
 *   K dP = -(d + C_p (K <P'>^n - G^n)) / dt + G^{n+1} - G^n,
 * K the stiffness matrix, d_a = sum_e A_e / 3 div_e <U*>, G the load of the
 * Neumann condition at WALL and NO-SLIP edges (eq. wall-pressure-condition:
 * d<P>/dn = nu lap<U_i> n_i - d<u_i u_j>/dx_j n_i, and with the SLM closure,
 * the wall-functions case, also - <U_j> d<U_i>/dx_j n_i; per edge the
 * element's gradients and the mean of the edge's nodes, load h |edge| / 2 on
 * each end), G^{n+1} from the present statistics and G^n the one stored by
 * the projection that made <P'>^n (0 initially and after pdf_pressure_field
 * sets the field); zero flux at inflow and outflow edges.  Solved in FP64
 * from zero by conjugate gradients preconditioned with one V-cycle of a
 * smoothed-aggregation multigrid of K (built on the host at the first call,
 * once per particle set); the right-hand side has its mean removed
 * (compatibility of the pure-Neumann problem) and dP is normalised to zero
 * mean over the unknowns.  Then every particle's velocity is corrected by
 * -dt grad dP of its element, <P'> += dP, the nodal gradient of <P'>
 * (element gradients averaged over the surrounding elements) is stored for
 * PDF_PRESSURE_PROJECTION steps, and the statistics follow the correction
 * (element means shifted by the same vector, central moments and conditional
 * means unchanged; node statistics and derivatives recomputed).
 *   Cp       the stabilisation constant C_p, a time (the paper suggests 1e-3
 *            in its units).  The pressure mode of this discretisation is
 *            multiplied each step by about 1 - C_p/dt - lambda, lambda in
 *            [0, ~1.2] the ratio of the drift's averaged-gradient Laplacian
 *            to K: C_p/dt near 0.5 damps it, C_p/dt = 1 lets it grow, and
 *            C_p/dt -> 0 leaves the statistical noise undamped.
 *   rtol     stop when ||r|| <= rtol ||b||; PDF_ENOTCONV after max_it
 *   iters, rel_res  host or NULL
 * Synchronizes `stream` once per 8 iterations (once with the persistent
 * solver, see pdf_pressure_set_solver).  PDF_ESTATE without statistics. */
pdf_status pdf_pressure_project(pdf_particles* p, const pdf_mesh* m, const pdf_model_params* params, double Cp,
                                double rtol, int32_t max_it, int32_t* iters, double* rel_res, void* stream);
/* The iteration of pdf_pressure_project runs as separate kernels replayed
 * in CUDA graphs of 8 iterations (persistent = 0, the default) or as one
 * persistent cooperative kernel with grid-wide barriers between its phases
 * (persistent = 1; the separate kernels are used when the device refuses
 * the cooperative launch).  Both compute the same iterates up to the order
 * of the reductions.  PDF_EINVAL for other values. */
pdf_status pdf_pressure_set_solver(pdf_particles* p, int32_t persistent);
/* Copies the pressure field <P'> [n_nodes] (FP64, device or host) in (set,
 * recomputing its nodal gradient and zeroing the stored wall load G^n)
 * and/or out (get); either may be NULL. */
pdf_status pdf_pressure_field(pdf_particles* p, const double* set, double* get, void* stream);

/* ---------------------------------------------------------------- learned warm start */

/* A per-node MLP that proposes the initial guess of pdf_relax_solve.  The
 * paper warm-starts from the previous step (sec. 3.2); the network is an
 * addition, and the FP64 solve it seeds still runs to the same residual.
 * It corrects the local model: where the elliptic term of eq.
 * elliptic-relaxation-Lagrangian vanishes, wp = rhs; the guess is rhs plus
 * the network's estimate of wp - rhs.  Architecture: 11 inputs (the nine
 * rhs_ij, the wall distance over L, log(L^2 / h^2) with L^2 the C_xi = 1
 * length scale and h^2 the mean area of the node's elements) -> 64 -> 64 ->
 * 64 -> 9 outputs (wp_ij - rhs_ij, row-major
 * ij), GELU, standardized inputs and outputs.  Matrix products on the
 * tensor cores from BF16 operands with FP32 accumulation; the standardized
 * input, the weights, each hidden activation and each back-propagated
 * gradient are rounded to BF16 before a product.  Training: mean squared
 * error over the batch and the 9 standardized outputs, Adam (beta 0.9,
 * 0.999, eps 1e-8) on FP32 master parameters.  Deterministic.
 * Parameters, flat FP32 [PDF_MLP_NPARAM]: W0[64][11] b0[64] W1[64][64]
 * b1[64] W2[64][64] b2[64] W3[9][64] b3[9].  Standardization, FP32 [64]:
 * in_mean[16] in_inv_std[16] out_mean[16] out_std[16] (first 11 / 9 used).
 * Feature and target arrays are device FP32: X [n][11], Y [n][9]. */
#define PDF_MLP_NPARAM 9673
typedef struct pdf_mlp pdf_mlp;
/* He-normal weights from Philox (key seed, purpose 3), zero biases, identity
 * standardization; allocates ~12 MB of device memory. */
pdf_status pdf_mlp_create(uint64_t seed, pdf_mlp** out);
pdf_status pdf_mlp_destroy(pdf_mlp* net);
/* Copy parameters / standardization in (set, set_norm) or out (get,
 * get_norm); any pointer may be NULL; host or device memory.  Setting
 * parameters resets the Adam state.  Synchronous. */
pdf_status pdf_mlp_params(pdf_mlp* net, const float* set, float* get, const float* set_norm, float* get_norm);
/* Standardization fitted to n training pairs (means and standard deviations). */
pdf_status pdf_mlp_fit_norm(pdf_mlp* net, const float* X, const float* Y, int64_t n, void* stream);
pdf_status pdf_mlp_forward(const pdf_mlp* net, const float* X, int64_t n, float* Y, void* stream);
/* Loss and gradient [PDF_MLP_NPARAM] (device or host) on n pairs, no update;
 * loss (host, may be NULL; synchronizes). */
pdf_status pdf_mlp_grad(pdf_mlp* net, const float* X, const float* Y, int64_t n, float* grad, float* loss,
                        void* stream);
/* One Adam step with learning rate lr on the n pairs (one batch). */
pdf_status pdf_mlp_train_step(pdf_mlp* net, const float* X, const float* Y, int64_t n, float lr, float* loss,
                              void* stream);
/* A training batch of `batch` rows drawn uniformly (with replacement) from
 * the n pairs (X [n][11], Y [n][9], device FP32) into Xb, Yb (device):
 * row i comes from row floor(w n / 2^32), w word 0 of Philox4x32-10 (key
 * seed, counter (i, step, 0, 4)).  PDF_EINVAL for n outside [1, 2^32). */
pdf_status pdf_mlp_batch(const float* X, const float* Y, int64_t n, uint64_t seed, uint32_t step, int64_t batch,
                         float* Xb, float* Yb, void* stream);
/* Features X [n_nodes][11] of every node from the last statistics (the
 * relaxation's right-hand side and L^2 for params, as pdf_relax_rhs gives
 * them) and, if wp (device [9][n_nodes], a solution) and Y are given, the
 * targets Y [n_nodes][9] = wp - rhs. */
pdf_status pdf_mlp_features(pdf_particles* p, const pdf_mesh* m, const pdf_model_params* params, const double* wp,
                            float* X, float* Y, void* stream);
/* The guess wp = rhs + the network's correction [9][n_nodes] (device FP64)
 * for the current statistics; scratch: device FP32 of at least 20 n_nodes
 * entries. */
pdf_status pdf_mlp_guess(const pdf_mlp* net, pdf_particles* p, const pdf_mesh* m, const pdf_model_params* params,
                         double* wp, float* scratch, void* stream);

/* ---------------------------------------------------------------- random numbers */

/* The library's Gaussian draw, exposed for checking: for i = 0..n-1 the four
 * N(0,1) values of Philox4x32-10 block (key = seed, counter (i, c1, c2, c3))
 * through the FP32 Box-Muller transform.  out: device float [n][4]. */
pdf_status pdf_rng_gauss(uint64_t seed, uint32_t c1, uint32_t c2, uint32_t c3, int64_t n,
                         float* out, void* stream);

/* ---------------------------------------------------------------- measurement */

/* Kernel timing for measurements: while enabled, every kernel the library
 * launches is bracketed by CUDA events on its launch stream.  The paper has
 * no counterpart; it only reports per-stage shares of a time step.
 * pdf_profile_query waits for the recorded events of the named kernel
 * (e.g. "k_step") and returns how many launches were recorded and their
 * summed duration since the last reset. */
pdf_status pdf_profile_enable(int32_t on);
/* Restricts the timing to the kernels named `kernel` (NULL: all kernels),
 * so that a measurement of one kernel does not pay for the events around
 * the others. */
pdf_status pdf_profile_only(const char* kernel);
pdf_status pdf_profile_reset(void);
pdf_status pdf_profile_query(const char* kernel, int64_t* launches, double* total_ms);
/* Number of kernels the library has launched in this process. */
int64_t pdf_kernel_launches(void);

/* ---------------------------------------------------------------- misc */
const char* pdf_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* PDFGB_H */
