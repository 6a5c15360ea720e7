// Saved form of a particle set (pdf_particles_save / pdf_particles_load):
// the stored state exactly as it sits in the slots (fixed-point positions,
// double-float or FP32 values, element and particle id of every slot), the
// statistics of the last pdf_estimate_stats, the IECM conditioned means and
// the projected pressure field, so that a loaded set continues bit for bit
// where the saved one stood.  Little-endian, 8-byte aligned sections:
//
//   header (80 B): magic "PDFGBPS\0", version (u32), flags (u32: 1 stats,
//     2 IECM means, 4 pressure field), n (i64), seed (u64), n_tri, n_nodes,
//     precision, reorder_every, since_reorder (i32), IECM bins (3 x i32),
//     IECM minimum (i32), 12 reserved bytes (zero)
//   x, y            n x i64    fixed point, 56 fraction bits
//   u, v, w, om, ps n x 8 B    double-float pairs (PDF_FP64)
//                   n x 4 B    FP32, each array padded to 8 B (PDF_FP32_STATE)
//   elem, pid       n x i32 each, each padded to 8 B
//   [flags & 1]     element stats [n_tri][13], node stats [n_nodes][12],
//                   node derivatives [n_nodes][10] (f64)
//   [flags & 2]     IECM conditioned mean per slot, n x 8 B (double-float)
//   [flags & 4]     <P'> [n_nodes] and its nodal gradient [n_nodes][2] (f64)
//   checksum (u64): FNV-1a over the preceding 64-bit words
#include <cstring>
#include <vector>

#include "common.cuh"

namespace pdfgb {
pdf_status alloc_state(pdf_particles* P, cudaStream_t st);
}  // namespace pdfgb

using namespace pdfgb;

namespace {

constexpr char kMagic[8] = {'P', 'D', 'F', 'G', 'B', 'P', 'S', '\0'};
constexpr uint32_t kVersion = 1;
enum : uint32_t { kHasStats = 1, kHasCond = 2, kHasPressure = 4 };

struct Header {
  char magic[8];
  uint32_t version, flags;
  int64_t n;
  uint64_t seed;
  int32_t n_tri, n_nodes, precision, reorder_every, since_reorder;
  int32_t iecm_bins[3], iecm_min;
  int32_t reserved[3];
};
static_assert(sizeof(Header) == 80, "saved-form header is 80 bytes");

size_t pad8(size_t b) { return (b + 7) & ~size_t(7); }

// One section of the saved form: a device array and its byte count.
struct Section {
  void* dev;
  size_t bytes;
};

std::vector<Section> sections(const pdf_particles* p, uint32_t flags) {
  const size_t n = (size_t)p->n, nt = (size_t)p->mesh->d.n_tri, nn = (size_t)p->mesh->d.n_nodes;
  std::vector<Section> s = {{p->x, 8 * n}, {p->y, 8 * n}};
  if (p->precision == PDF_FP64) {
    for (void* a : {(void*)p->u, (void*)p->v, (void*)p->w, (void*)p->om, (void*)p->ps}) s.push_back({a, 8 * n});
  } else {
    for (void* a : {(void*)p->uf, (void*)p->vf, (void*)p->wf, (void*)p->omf, (void*)p->psf}) s.push_back({a, 4 * n});
  }
  s.push_back({p->elem, 4 * n});
  s.push_back({p->pid, 4 * n});
  if (flags & kHasStats) {
    s.push_back({p->es, 8 * nt * PDF_NES});
    s.push_back({p->ns, 8 * nn * PDF_NNS});
    s.push_back({p->nd, 8 * nn * PDF_NND});
  }
  if (flags & kHasCond) s.push_back({p->cond, 8 * n});
  if (flags & kHasPressure) {
    s.push_back({p->pres, 8 * nn});
    s.push_back({p->gradP, 16 * nn});
  }
  return s;
}

size_t saved_size(const pdf_particles* p, uint32_t flags) {
  size_t b = sizeof(Header);
  for (const Section& s : sections(p, flags)) b += pad8(s.bytes);
  return b + 8;
}

uint32_t flags_of(const pdf_particles* p) {
  return (p->have_stats ? kHasStats : 0u) | (p->have_cond && p->cond ? kHasCond : 0u) | kHasPressure;
}

uint64_t fnv1a_words(const unsigned char* b, size_t bytes) {
  uint64_t h = 0xcbf29ce484222325ull;
  for (size_t i = 0; i + 8 <= bytes; i += 8) {
    uint64_t w;
    std::memcpy(&w, b + i, 8);
    h = (h ^ w) * 0x100000001b3ull;
  }
  return h;
}

bool host_memory(const void* ptr) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
    cudaGetLastError();
    return true;  // unregistered (pageable) host memory
  }
  return at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeUnregistered;
}

}  // namespace

extern "C" pdf_status pdf_particles_save_size(const pdf_particles* p, size_t* size) {
  if (!p || !size || p->n <= 0) return fail(PDF_EINVAL, "pdf_particles_save_size: NULL argument or a set without particles");
  *size = saved_size(p, flags_of(p));
  return PDF_OK;
}

extern "C" pdf_status pdf_particles_save(const pdf_particles* p, void* buf, size_t cap, void* stream) {
  if (!p || !buf || p->n <= 0) return fail(PDF_EINVAL, "pdf_particles_save: NULL argument or a set without particles");
  if (!host_memory(buf)) return fail(PDF_EINVAL, "pdf_particles_save: buf must be host memory");
  const uint32_t flags = flags_of(p);
  const size_t need = saved_size(p, flags);
  if (cap < need) return fail(PDF_EINVAL, "pdf_particles_save: buffer smaller than pdf_particles_save_size");
  unsigned char* out = static_cast<unsigned char*>(buf);
  Header h;
  std::memset(&h, 0, sizeof(h));
  std::memcpy(h.magic, kMagic, 8);
  h.version = kVersion;
  h.flags = flags;
  h.n = p->n;
  h.n_tri = p->mesh->d.n_tri;
  h.n_nodes = p->mesh->d.n_nodes;
  h.precision = p->precision;
  h.reorder_every = p->reorder_every;
  h.since_reorder = p->since_reorder;
  h.seed = p->seed;
  for (int i = 0; i < 3; ++i) h.iecm_bins[i] = p->iecm_bins[i];
  h.iecm_min = p->iecm_min;
  std::memcpy(out, &h, sizeof(h));
  cudaStream_t st = (cudaStream_t)stream;
  size_t off = sizeof(Header);
  for (const Section& s : sections(p, flags)) {
    PDF_CUDA(cudaMemcpyAsync(out + off, s.dev, s.bytes, cudaMemcpyDeviceToHost, st));
    if (pad8(s.bytes) > s.bytes) std::memset(out + off + s.bytes, 0, pad8(s.bytes) - s.bytes);
    off += pad8(s.bytes);
  }
  PDF_CUDA(cudaStreamSynchronize(st));
  const uint64_t sum = fnv1a_words(out, off);
  std::memcpy(out + off, &sum, 8);
  return PDF_OK;
}

extern "C" pdf_status pdf_particles_load(const pdf_mesh* m, const void* buf, size_t size, void* stream,
                                         pdf_particles** out) {
  if (!out) return fail(PDF_EINVAL, "pdf_particles_load: out is NULL");
  *out = nullptr;
  if (!m || !buf) return fail(PDF_EINVAL, "pdf_particles_load: NULL argument");
  if (!host_memory(buf)) return fail(PDF_EINVAL, "pdf_particles_load: buf must be host memory");
  if (size < sizeof(Header) + 8) return fail(PDF_EINVAL, "pdf_particles_load: buffer too small for a saved set");
  const unsigned char* in = static_cast<const unsigned char*>(buf);
  Header h;
  std::memcpy(&h, in, sizeof(h));
  if (std::memcmp(h.magic, kMagic, 8) != 0) return fail(PDF_EINVAL, "pdf_particles_load: not a saved particle set");
  if (h.version != kVersion)
    return fail(PDF_EINVAL, "pdf_particles_load: saved-form version " + std::to_string(h.version) + " is not " +
                                std::to_string(kVersion));
  if (h.n_tri != m->d.n_tri || h.n_nodes != m->d.n_nodes)
    return fail(PDF_EINVAL, "pdf_particles_load: the set was saved on a mesh of another size");
  if (h.n < 1 || h.n > (int64_t)INT32_MAX || (h.precision != PDF_FP64 && h.precision != PDF_FP32_STATE) ||
      (h.flags & ~uint32_t(kHasStats | kHasCond | kHasPressure)) != 0 || h.reorder_every < 0 || h.since_reorder < 0)
    return fail(PDF_EINVAL, "pdf_particles_load: corrupt header");
  pdf_particles* P = new (std::nothrow) pdf_particles();
  if (!P) return fail(PDF_ENOMEM, "pdf_particles_load: host allocation");
  P->mesh = m;
  P->n = h.n;
  P->precision = h.precision;
  P->seed = h.seed;
  if (saved_size(P, h.flags) != size) {
    delete P;
    return fail(PDF_EINVAL, "pdf_particles_load: size does not match the header");
  }
  uint64_t sum;
  std::memcpy(&sum, in + size - 8, 8);
  if (fnv1a_words(in, size - 8) != sum) {
    delete P;
    return fail(PDF_EINVAL, "pdf_particles_load: checksum mismatch");
  }
  // element ids in range and slot particle ids a permutation: checked on
  // the host before anything reaches the device
  const size_t n = (size_t)h.n;
  const size_t vb = h.precision == PDF_FP64 ? 8 : 4;
  const size_t off_elem = sizeof(Header) + 2 * 8 * n + 5 * pad8(vb * n);
  const size_t off_pid = off_elem + pad8(4 * n);
  {
    std::vector<uint8_t> seen(n, 0);
    for (size_t i = 0; i < n; ++i) {
      int32_t e, q;
      std::memcpy(&e, in + off_elem + 4 * i, 4);
      std::memcpy(&q, in + off_pid + 4 * i, 4);
      if (e < 0 || e >= h.n_tri || q < 0 || (size_t)q >= n || seen[q]) {
        delete P;
        return fail(PDF_EINVAL, "pdf_particles_load: element or particle ids out of range");
      }
      seen[q] = 1;
    }
  }
  cudaStream_t st = (cudaStream_t)stream;
  pdf_status s = alloc_state(P, st);
  if (s == PDF_OK && (h.flags & kHasCond)) {
    cudaError_t e = cudaMalloc((void**)&P->cond, sizeof(fx::df) * n);
    if (e == cudaSuccess) e = cudaMalloc((void**)&P->iecm_scratch_f, sizeof(float) * 16 * n);
    if (e == cudaSuccess) e = cudaMalloc((void**)&P->iecm_scratch_i, sizeof(int32_t) * 6 * n);
    if (e != cudaSuccess) s = fail(PDF_ENOMEM, "pdf_particles_load: cudaMalloc failed");
  }
  if (s != PDF_OK) {
    release_particles(P);
    return s;
  }
  size_t off = sizeof(Header);
  for (const Section& sec : sections(P, h.flags)) {
    const cudaError_t e = cudaMemcpyAsync(sec.dev, in + off, sec.bytes, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
      release_particles(P);
      return cuda_fail(e, "pdf_particles_load: copy to the device");
    }
    off += pad8(sec.bytes);
  }
  const cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    release_particles(P);
    return cuda_fail(e, "pdf_particles_load: copy to the device");
  }
  P->reorder_every = h.reorder_every;
  P->since_reorder = h.since_reorder;
  P->have_stats = (h.flags & kHasStats) != 0;
  for (int i = 0; i < 3; ++i) P->iecm_bins[i] = h.iecm_bins[i];
  P->iecm_min = h.iecm_min;
  P->have_cond = (h.flags & kHasCond) != 0;
  *out = P;
  return PDF_OK;
}
