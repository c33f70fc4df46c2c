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

#include "../../include/hz.h"
#include "kernels.cuh"

namespace hz {
const DevSplitCsr* ctx_matrix(const hz_ctx* c, int64_t* n);    // hz_api.cu
void ctx_noalloc(const hz_ctx* c, int* device, void** scratch);  // hz_api.cu
void set_last_error(const char* msg);                          // hz_api.cu
}  // namespace hz

namespace {

// Scratch of the allocation-free product: two blocks of HZ_NOALLOC_MAX_ENTRIES
// complex values (32 MiB in total). All calls share it; every call
// overwrites the entries it reads, so nothing has to start at zero.
constexpr int64_t kMaxEntries = HZ_NOALLOC_MAX_ENTRIES;
static __device__ __align__(256) double2 hz_noalloc_scratch[2 * kMaxEntries];

}  // namespace

namespace hz {
// Device address of the scratch array on the current device. Host code
// cannot use the symbol itself as an address; hz_setup calls this once with
// the context's device current (which loads the array there) and keeps the
// result in the context.
cudaError_t noalloc_scratch_address(void** out) {
  *out = nullptr;
  cudaError_t e = cudaGetSymbolAddress(out, hz_noalloc_scratch);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *out = nullptr;
  }
  return e;
}
}  // namespace hz

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
  int ctx_dev = -1, cur = -1;
  void* scr = nullptr;
  ctx_noalloc(ctx, &ctx_dev, &scr);
  if (cudaGetDevice(&cur) != cudaSuccess) {
    cudaGetLastError();
    set_last_error("hz_apply_A_noalloc: cudaGetDevice failed");
    return HZ_ECUDA;
  }
  if (cur != ctx_dev) {
    set_last_error("hz_apply_A_noalloc: the current device is not the context's device");
    return HZ_EINVAL;
  }
  if (!scr) {
    set_last_error("hz_apply_A_noalloc: the scratch array could not be looked up at setup");
    return HZ_ECUDA;
  }
  cudaStream_t st = (cudaStream_t)stream;
  double2* scratch = (double2*)scr;
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
