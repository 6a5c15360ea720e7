// pdf_estimate_stats_noalloc: the statistics entry point for callers that
// must not allocate device memory.  The grouping scratch (radix keys and
// values, tile histograms, scan partials, segment offsets) lives in one
// file-scope device array instead of buffers from cudaMalloc.
#include <mutex>

#include "common.cuh"

namespace pdfgb {
pdf_status estimate_stats_with_buffers(pdf_particles* P, int32_t* keys_a, int32_t* vals_a,
                                       int32_t* keys_b, int32_t* vals_b, int32_t* hist,
                                       int32_t* hist_part, int32_t* seg, cudaStream_t st);
int64_t radix_tiles(int64_t n);
int32_t radix_bins();
int32_t radix_scan_blocks(int64_t hist_len);
}  // namespace pdfgb

using namespace pdfgb;

namespace {

constexpr int64_t kMaxParticles = PDF_NOALLOC_MAX_PARTICLES;  // 2^19
constexpr int64_t kMaxElements = PDF_NOALLOC_MAX_ELEMENTS;    // 2^18
constexpr int64_t kMaxTiles = (kMaxParticles + 4095) / 4096;  // radix tiles of 4096 keys
constexpr int64_t kHistInts = kMaxTiles * 512;
constexpr int64_t kPartInts = 520;  // the digit totals of the scan (512), rounded up
// int32 layout: keys_a | vals_a | keys_b | vals_b | hist | part | seg
constexpr int64_t kScratchInts = 4 * kMaxParticles + kHistInts + kPartInts + (kMaxElements + 1);

// 4 x 2 MiB + 256 KiB + 2 KiB + 1 MiB: every GPU that loads the library
// holds these ~9.2 MiB until the process exits.
static __device__ __align__(256) int32_t g_noalloc_scratch[kScratchInts];

std::mutex g_mu;
// device address of g_noalloc_scratch per device, kept for the life of the
// process (a device reset between calls is not supported)
int32_t* g_scratch_ptr[64] = {nullptr};

}  // namespace

extern "C" pdf_status pdf_estimate_stats_noalloc(pdf_particles* p, const pdf_mesh* m, double* elem_stats,
                                                 double* node_stats, double* node_derivs, void* stream) {
  if (!p || !m || p->mesh != m) return fail(PDF_EINVAL, "pdf_estimate_stats_noalloc: NULL or mismatched handles");
  if (p->n > kMaxParticles)
    return fail(PDF_EINVAL, "pdf_estimate_stats_noalloc: " + std::to_string(p->n) +
                                " particles exceed the limit of " + std::to_string(kMaxParticles));
  if (m->d.n_tri > kMaxElements)
    return fail(PDF_EINVAL, "pdf_estimate_stats_noalloc: " + std::to_string(m->d.n_tri) +
                                " elements exceed the limit of " + std::to_string(kMaxElements));
  if (radix_bins() != 512 || radix_tiles(kMaxParticles) != kMaxTiles ||
      radix_scan_blocks(radix_tiles(p->n) * 512) > kPartInts - 1)
    return fail(PDF_EINVAL, "pdf_estimate_stats_noalloc: scratch layout does not match the grouping kernels");
  int dev = 0;
  PDF_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(PDF_EINVAL, "pdf_estimate_stats_noalloc: device id out of range");
  int32_t* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
      // host code may not use the array's name as an address: ask the runtime
      // for this device's copy (first call on each device, device current)
      void* ptr = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess) return cuda_fail(e, "pdf_estimate_stats_noalloc: cudaGetSymbolAddress");
      g_scratch_ptr[dev] = static_cast<int32_t*>(ptr);
    }
    base = g_scratch_ptr[dev];
  }
  int32_t* keys_a = base;
  int32_t* vals_a = keys_a + kMaxParticles;
  int32_t* keys_b = vals_a + kMaxParticles;
  int32_t* vals_b = keys_b + kMaxParticles;
  int32_t* hist = vals_b + kMaxParticles;
  int32_t* part = hist + kHistInts;
  int32_t* seg = part + kPartInts;
  cudaStream_t st = (cudaStream_t)stream;
  // Nothing in the scratch has to start at zero: every pass writes all the
  // histogram entries, scan partials and key/value slots it later reads.
  pdf_status s = estimate_stats_with_buffers(p, keys_a, vals_a, keys_b, vals_b, hist, part, seg, st);
  if (s != PDF_OK) return s;
  const MeshDev& M = m->d;
  if (elem_stats)
    PDF_CUDA(cudaMemcpyAsync(elem_stats, p->es, sizeof(double) * M.n_tri * PDF_NES, cudaMemcpyDefault, st));
  if (node_stats)
    PDF_CUDA(cudaMemcpyAsync(node_stats, p->ns, sizeof(double) * M.n_nodes * PDF_NNS, cudaMemcpyDefault, st));
  if (node_derivs)
    PDF_CUDA(cudaMemcpyAsync(node_derivs, p->nd, sizeof(double) * M.n_nodes * PDF_NND, cudaMemcpyDefault, st));
  return PDF_OK;
}
