// Device kernels of the two-level ORAS preconditioned FGMRES iteration.
//
// Sec. "Domain decomposition preconditioner": each GMRES iteration applies
// A (Eq. eq1) and M^{-1} (Eq. 2lvl): a coarse restriction Z^T, the coarse
// solve, the prolongation Z, a residual with A, the restriction R_i to every
// overlapping subdomain, the local solves A_i^{-1} (multifrontal LDL^T
// factors here, the paper's direct local solver) and the partition-of-unity
// prolongation sum_i R_i^T D_i (Eq. oras). Blocks of right-hand sides are
// stored row-major [n][s] (the s columns of a row contiguous), complex128 as
// double2 (re, im).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>

#include "kernels.cuh"

namespace hz {

std::atomic<long long> g_kernel_launches{0};

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {  // a*b + c
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
__device__ __forceinline__ double2 cfms(double2 a, double2 b, double2 c) {  // c - a*b
  return make_double2(fma(-a.x, b.x, fma(a.y, b.y, c.x)), fma(-a.x, b.y, fma(-a.y, b.x, c.y)));
}
__device__ __forceinline__ double2 conjmul_acc(double2 a, double2 b, double2 c) {  // conj(a)*b + c
  return make_double2(fma(a.x, b.x, fma(a.y, b.y, c.x)), fma(a.x, b.y, fma(-a.y, b.x, c.y)));
}
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }

static inline unsigned grid_for(int64_t work, int block) { return (unsigned)((work + block - 1) / block); }

// ---------------------------------------------------------------------------
// SpMM: Y = (A_re + i A_im) X  or  Y = B - A X   (K1)
// one thread per (row, column); the s threads of a row share the index and
// value loads, the X loads of one nonzero are one contiguous 16 s-byte row.
// ---------------------------------------------------------------------------
__global__ void k_spmm_split(int64_t n, int s, const int64_t* __restrict__ rp_re, const int32_t* __restrict__ col_re,
                             const double* __restrict__ val_re, const int64_t* __restrict__ rp_im,
                             const int32_t* __restrict__ col_im, const double* __restrict__ val_im,
                             const double2* __restrict__ X, double2* __restrict__ Y, const double2* __restrict__ B,
                             int mode) {
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t r = g / s;
  int c = (int)(g - r * s);
  if (r >= n) return;
  double ar = 0.0, ai = 0.0;
  #pragma unroll 4
  for (int64_t p = rp_re[r], pe = rp_re[r + 1]; p < pe; ++p) {
    double a = val_re[p];
    double2 x = X[(int64_t)col_re[p] * s + c];
    ar = fma(a, x.x, ar);
    ai = fma(a, x.y, ai);
  }
  #pragma unroll 4
  for (int64_t p = rp_im[r], pe = rp_im[r + 1]; p < pe; ++p) {
    double b = val_im[p];
    double2 x = X[(int64_t)col_im[p] * s + c];
    ar = fma(-b, x.y, ar);
    ai = fma(b, x.x, ai);
  }
  if (mode == 1) {
    double2 b = B[g];
    Y[g] = make_double2(b.x - ar, b.y - ai);
  } else {
    Y[g] = make_double2(ar, ai);
  }
}

void spmm_split(const DevSplitCsr& A, const double2* X, double2* Y, const double2* B, int s, int mode,
                cudaStream_t st) {
  int64_t work = A.n * s;
  if (work == 0) return;
  { k_spmm_split<<<grid_for(work, 256), 256, 0, st>>>(A.n, s, A.rp_re, A.col_re, A.val_re, A.rp_im, A.col_im,
                                                    A.val_im, X, Y, B, mode); count_launch(); }
}

__global__ void k_spmm_real(int64_t n, int s, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                            const double* __restrict__ val, const double2* __restrict__ X, double2* __restrict__ Y) {
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t r = g / s;
  int c = (int)(g - r * s);
  if (r >= n) return;
  double ar = 0.0, ai = 0.0;
  #pragma unroll 4
  for (int64_t p = rp[r], pe = rp[r + 1]; p < pe; ++p) {
    double a = val[p];
    double2 x = X[(int64_t)col[p] * s + c];
    ar = fma(a, x.x, ar);
    ai = fma(a, x.y, ai);
  }
  Y[g] = make_double2(ar, ai);
}

void spmm_real(int64_t nrows, const int64_t* rp, const int32_t* col, const double* val, const double2* X,
               double2* Y, int s, cudaStream_t st) {
  int64_t work = nrows * s;
  if (work == 0) return;
  { k_spmm_real<<<grid_for(work, 256), 256, 0, st>>>(nrows, s, rp, col, val, X, Y); count_launch(); }
}

// ---------------------------------------------------------------------------
// Restriction R_i (gather, K2) and Boolean partition-of-unity prolongation
// sum_i R_i^T D_i (each dof read from its owning subdomain copy, K3)
// ---------------------------------------------------------------------------
__global__ void k_gather_rows(const int* __restrict__ idx, int64_t nrows, const double2* __restrict__ X,
                              double2* __restrict__ Y, int s) {
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t r = g / s;
  if (r >= nrows) return;
  int c = (int)(g - r * s);
  Y[g] = X[(int64_t)idx[r] * s + c];
}

void gather_rows(const int* idx, int64_t nrows, const double2* X, double2* Y, int s, cudaStream_t st) {
  if (nrows * s == 0) return;
  { k_gather_rows<<<grid_for(nrows * s, 256), 256, 0, st>>>(idx, nrows, X, Y, s); count_launch(); }
}

__global__ void k_scatter_owned(const int* __restrict__ own, int64_t n, const double2* __restrict__ Xsub,
                                const double2* __restrict__ Q, double2* __restrict__ Z, int s) {
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t r = g / s;
  if (r >= n) return;
  int c = (int)(g - r * s);
  double2 v = Xsub[(int64_t)own[r] * s + c];
  if (Q) v = cadd(v, Q[g]);
  Z[g] = v;
}

void scatter_owned(const int* own, int64_t n, const double2* Xsub, const double2* Q, double2* Z, int s,
                   cudaStream_t st) {
  if (n * s == 0) return;
  { k_scatter_owned<<<grid_for(n * s, 256), 256, 0, st>>>(own, n, Xsub, Q, Z, s); count_launch(); }
}

__global__ void k_zero(double2* X, int64_t count) {
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g < count) X[g] = make_double2(0.0, 0.0);
}
void axpy_cols_zero(double2* X, int64_t count, cudaStream_t st) {
  if (count) { k_zero<<<grid_for(count, 256), 256, 0, st>>>(X, count); count_launch(); }
}

// one column c of an [n][s] block: zero it, copy it to another block, or
// extract it as a contiguous vector
__global__ void k_col_zero(double2* X, int64_t n, int s, int c) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) X[i * s + c] = make_double2(0.0, 0.0);
}
__global__ void k_col_copy(const double2* __restrict__ X, double2* __restrict__ Y, int64_t n, int s, int c) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) Y[i * s + c] = X[i * s + c];
}
__global__ void k_col_get(const double2* __restrict__ X, double2* __restrict__ y, int64_t n, int s, int c) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = X[i * s + c];
}
void col_zero(double2* X, int64_t n, int s, int c, cudaStream_t st) {
  if (n) { k_col_zero<<<grid_for(n, 256), 256, 0, st>>>(X, n, s, c); count_launch(); }
}
void col_copy(const double2* X, double2* Y, int64_t n, int s, int c, cudaStream_t st) {
  if (n) { k_col_copy<<<grid_for(n, 256), 256, 0, st>>>(X, Y, n, s, c); count_launch(); }
}
void col_get(const double2* X, double2* y, int64_t n, int s, int c, cudaStream_t st) {
  if (n) { k_col_get<<<grid_for(n, 256), 256, 0, st>>>(X, y, n, s, c); count_launch(); }
}

// ---------------------------------------------------------------------------
// Right-hand sides (K11) and layout changes
// ---------------------------------------------------------------------------
__global__ void k_point_sources(double2* B, const int* __restrict__ idx, const double2* __restrict__ val, int nent) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < nent) B[idx[e]] = cadd(B[idx[e]], val[e]);
}
void scatter_point_sources(double2* B, int64_t n, int s, const int* idx, const double2* val, int nent,
                           cudaStream_t st) {
  (void)n;
  (void)s;
  if (nent) { k_point_sources<<<grid_for(nent, 128), 128, 0, st>>>(B, idx, val, nent); count_launch(); }
}

__global__ void k_to_rows(const double2* __restrict__ F, double2* __restrict__ B, int64_t n, int s) {
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= n * s) return;
  int64_t r = g / s;
  int c = (int)(g - r * s);
  B[g] = F[(int64_t)c * n + r];
}
__global__ void k_from_rows(const double2* __restrict__ B, double2* __restrict__ F, int64_t n, int s) {
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= n * s) return;
  int c = (int)(g / n);
  int64_t r = g - (int64_t)c * n;
  F[g] = B[r * s + c];
}
void transpose_to_rows(const double2* F, double2* B, int64_t n, int s, cudaStream_t st) {
  if (n * s) { k_to_rows<<<grid_for(n * s, 256), 256, 0, st>>>(F, B, n, s); count_launch(); }
}
void transpose_from_rows(const double2* B, double2* F, int64_t n, int s, cudaStream_t st) {
  if (n * s) { k_from_rows<<<grid_for(n * s, 256), 256, 0, st>>>(B, F, n, s); count_launch(); }
}

// debug_bounds: every entry a[i * stride] must lie in [lo, hi); the smallest
// failing check id is kept in *err (initialised to INT_MAX by the caller)
__global__ void k_check_range(const int* __restrict__ a, int64_t count, int stride, int64_t lo, int64_t hi,
                              int* __restrict__ err, int id) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= count) return;
  const int64_t v = a[i * stride];
  if (v < lo || v >= hi) atomicMin(err, id);
}
void check_index_range(const int* a, int64_t count, int stride, int64_t lo, int64_t hi, int* err, int id,
                       cudaStream_t st) {
  if (count > 0 && a) { k_check_range<<<grid_for(count, 256), 256, 0, st>>>(a, count, stride, lo, hi, err, id); count_launch(); }
}

__global__ void k_copy(const double2* __restrict__ X, double2* __restrict__ Y, int64_t count) {
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g < count) Y[g] = X[g];
}
void cast_copy(const double2* X, double2* Y, int64_t count, cudaStream_t st) {
  if (count) { k_copy<<<grid_for(count, 256), 256, 0, st>>>(X, Y, count); count_launch(); }
}

}  // namespace hz
