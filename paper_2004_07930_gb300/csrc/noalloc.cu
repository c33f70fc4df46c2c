// Allocation-free product with A for callers that cannot allocate device
// memory at the time of the call: code running inside a region that
// forbids cudaMalloc/cudaFree (they synchronise the device), callers whose
// device memory is fully reserved by their own allocator, or pipelines that
// must not change the device allocation state after start-up. The matrix
// stays in the context (allocated once by hz_setup); the two [n][s] work
// blocks that hz_apply_A takes from the context workspace live here in a
// file-scope device array instead.
//
// The paper has no counterpart of this entry point; it reuses the kernels
// of hz_apply_A (layout change, split real/imaginary SpMM, layout change).
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/hz.h"
#include "kernels.cuh"

namespace hz {
const DevSplitCsr* ctx_matrix(const hz_ctx* c, int64_t* n);  // hz_api.cu
void set_last_error(const char* msg);                        // hz_api.cu
}  // namespace hz

namespace {

// Scratch of the allocation-free product: two blocks of HZ_NOALLOC_MAX_ENTRIES
// complex values (32 MiB in total), held by every GPU that loads the library
// until the process exits. All calls share it; every call overwrites the
// entries it reads, so nothing has to start at zero.
constexpr int64_t kMaxEntries = HZ_NOALLOC_MAX_ENTRIES;
static __device__ __align__(256) double2 hz_noalloc_scratch[2 * kMaxEntries];

// Host code cannot use the symbol as an address: its device address is
// looked up once per device (with that device current) and cached.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
double2* g_scratch[kMaxDevices] = {};

int scratch_for_current_device(double2** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return HZ_ECUDA;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, hz_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return HZ_ECUDA;
    }
    g_scratch[dev] = (double2*)p;
  }
  *out = g_scratch[dev];
  return HZ_OK;
}

}  // namespace

extern "C" int hz_apply_A_noalloc(hz_ctx* ctx, const double* X, double* Y, int32_t s, void* stream) {
  using namespace hz;
  if (!ctx || !X || !Y || s < 1) {
    set_last_error("hz_apply_A_noalloc: bad argument");
    return HZ_EINVAL;
  }
  int64_t n = 0;
  const DevSplitCsr* A = ctx_matrix(ctx, &n);
  if ((int64_t)s * n > kMaxEntries) {
    set_last_error("hz_apply_A_noalloc: n * s exceeds HZ_NOALLOC_MAX_ENTRIES");
    return HZ_EINVAL;
  }
  double2* scratch = nullptr;
  if (scratch_for_current_device(&scratch) != HZ_OK) {
    set_last_error("hz_apply_A_noalloc: cudaGetSymbolAddress failed");
    return HZ_ECUDA;
  }
  cudaStream_t st = (cudaStream_t)stream;
  double2* B = scratch;                // [n][s] input rows
  double2* R = scratch + kMaxEntries;  // [n][s] product rows
  transpose_to_rows(reinterpret_cast<const double2*>(X), B, n, s, st);
  spmm_split(*A, B, R, nullptr, s, 0, st);
  transpose_from_rows(R, reinterpret_cast<double2*>(Y), n, s, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_last_error(cudaGetErrorString(e));
    return HZ_ECUDA;
  }
  return HZ_OK;
}
