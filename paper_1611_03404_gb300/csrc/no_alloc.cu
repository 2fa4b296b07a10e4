// celeste_elbo_batch_noalloc: ELBO + gradient + Hessian of every source of a bound problem, with the
// kernels' scratch (per-patch tables, per-pixel source moments, per-tile partial sums, per-source
// work flags, counters) held in a fixed device array that this file owns, so that the call itself
// allocates nothing.
//
// Who needs it: callers that may not call cudaMalloc at evaluation time, for example code running
// inside a pre-sized memory arena, a process whose allocator is owned by another framework, or a
// service that must not allocate on its request path.  They pass the bound problem (its inputs),
// theta and the three outputs, all in memory they already hold.
//
// The array is a file-scope __device__ variable: every GPU that loads this library keeps
// NOALLOC_SCRATCH_BYTES of device memory for it until the process exits.  Host code never uses
// the symbol as an address: the device address is obtained with cudaGetSymbolAddress, once per
// device, with that device current, on the first call made on it.
#include <mutex>

#include "celeste_internal.cuh"
#include "kernels.h"
#include "problem.h"

namespace celeste {

constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(8) << 20;   // 8 MiB
constexpr int NOALLOC_MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

static std::mutex g_noalloc_mutex;
static void* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};

static size_t round256(size_t x) { return (x + 255) & ~size_t(255); }

// Layout of the array for one problem: partial sums, flags, tables, source moments, worklists and
// their counts, per-source brightness constants.
struct NoallocLayout {
  size_t partials, flags, ptab, srcmom, wl, wl_count, snc, total;
};
static NoallocLayout noalloc_layout(const celeste_problem* p) {
  NoallocLayout L;
  size_t o = 0;
  L.partials = o;
  o += round256(sizeof(float) * NACC * p->tiles.size());
  L.flags = o;
  o += round256(sizeof(int) * p->S);
  L.ptab = o;
  o += round256(sizeof(float) * TB_FLOATS * p->patches.size());
  L.srcmom = o;
  o += round256(sizeof(float2) * (size_t)p->n_pix);
  L.wl = o;
  o += round256(sizeof(int) * (p->tiles.size() + p->patches.size() + (size_t)p->S));
  L.wl_count = o;
  o += round256(sizeof(int) * WL_INTS);
  L.snc = o;
  o += round256(sizeof(SNConst) * 5 * (size_t)p->S);
  L.total = o;
  return L;
}

// Device address of the array on the current device (looked up once per device).
static int noalloc_base(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return fail(CELESTE_ERR_INVALID_ARG, "device ordinal %d unsupported", dev);
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_noalloc_ptr[dev] = ptr;
  }
  *out = g_noalloc_ptr[dev];
  return CELESTE_OK;
}

}  // namespace celeste

using namespace celeste;

extern "C" int celeste_elbo_batch_noalloc(celeste_problem* p, const double* theta, double* elbo, double* grad,
                                          double* hess, celeste_stream_t stream) {
  if (!p) return fail(CELESTE_ERR_INVALID_ARG, "null problem");
  if (!theta || !elbo || !grad || !hess) return fail(CELESTE_ERR_INVALID_ARG, "theta and all three outputs are required");
  const NoallocLayout NL = noalloc_layout(p);
  if (NL.total > NOALLOC_SCRATCH_BYTES)
    return fail(CELESTE_ERR_INVALID_ARG,
                "problem needs %zu bytes of scratch (%zu tiles, %zu patches, %lld pixels, %d sources); the fixed "
                "array holds %zu bytes",
                NL.total, p->tiles.size(), p->patches.size(), p->n_pix, p->S, NOALLOC_SCRATCH_BYTES);
  if (!p->bound || !p->background_ready)
    return fail(CELESTE_ERR_STATE, "bind the problem and render the background first");
  void* base = nullptr;
  int rc = noalloc_base(&base);
  if (rc != CELESTE_OK) return rc;
  char* b = static_cast<char*>(base);
  ProblemDev D = p->dev;   // inputs from the bound problem, scratch from the fixed array
  D.partials = reinterpret_cast<float*>(b + NL.partials);
  D.flags = reinterpret_cast<int*>(b + NL.flags);
  D.ptab = reinterpret_cast<float*>(b + NL.ptab);
  D.srcmom = reinterpret_cast<float2*>(b + NL.srcmom);
  D.wl = reinterpret_cast<int*>(b + NL.wl);
  D.wl_count = reinterpret_cast<int*>(b + NL.wl_count);
  D.snc = reinterpret_cast<SNConst*>(b + NL.snc);
  cudaStream_t st = (cudaStream_t)stream;
  // The array keeps the previous call's contents: the flags, worklists, brightness constants,
  // tables, source moments and partial sums are fully rewritten below before they are read.  The
  // error words and the pixel counters stay in the bound workspace (a timed-out bulk-copy wait
  // sets the workspace's timeout word, read by celeste_problem_check; the profiling counters count
  // these pixels); the timeout word is cleared first, as in celeste_elbo_batch.
  cudaError_t e = clear_timeout(D, st);
  if (e != cudaSuccess) return cuda_fail(e, "clear timeout word");
  if ((e = launch_set_flags(D, FLAG_FULL, st)) != cudaSuccess) return cuda_fail(e, "set flags");
  if ((e = launch_worklists(D, FLAG_FULL, st)) != cudaSuccess) return cuda_fail(e, "worklists");
  if ((e = launch_tables(D, theta, true, st)) != cudaSuccess) return cuda_fail(e, "tables");
  const int m0 = prof_mark(p, st);
  if ((e = launch_full_kernel(D, st)) != cudaSuccess) return cuda_fail(e, "pixel kernel");
  const int m1 = prof_mark(p, st);
  if (p->prof_on) p->prof_full.push_back({m0, m1});
  if ((e = launch_assemble(D, theta, true, elbo, grad, hess, st)) != cudaSuccess)
    return cuda_fail(e, "assemble kernel");
  prof_count(p, 6);
  return CELESTE_OK;
}
