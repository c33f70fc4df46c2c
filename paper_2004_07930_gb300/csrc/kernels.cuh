// Device kernels of the two-level ORAS / FGMRES hot path (declarations).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace hz {

// Split complex CSR: A = A_re + i A_im, A_im holding only the entries with a
// nonzero imaginary part (Robin faces); both share the row count.
struct DevSplitCsr {
  int64_t n = 0, ncols = 0, nnz_re = 0, nnz_im = 0;
  int64_t* rp_re = nullptr;
  int32_t* col_re = nullptr;
  double* val_re = nullptr;
  int64_t* rp_im = nullptr;
  int32_t* col_im = nullptr;
  double* val_im = nullptr;
  float* val_re_f = nullptr;  // FP32 copies (mixed-form coarse operator only)
  float* val_im_f = nullptr;
};

// Multifrontal factors of a batch of local matrices, grouped by tree height.
// Factor storage per front t: X_t (f x k, column-major) = first k columns of
// [[L11,0],[L21,I]]^{-1}, and 1/D (k); FP64 or FP32 (mixed form).
struct DevMF {
  int64_t nfronts = 0, nsub_rows = 0, rows_total = 0, F_total = 0, amap_total = 0, M_total = 0, D_total = 0;
  int nlevels = 0;
  int max_f = 0;
  int fp32 = 0;
  int* level_ptr_h = nullptr;   // host [nlevels+1]
  int* ftile_ptr_h = nullptr;   // host [nlevels+1] forward tiles per level
  int* btile_ptr_h = nullptr;   // host [nlevels+1] backward tiles per level
  int* level_list = nullptr;    // device [nfronts] front ids ordered by height
  int2* ftiles = nullptr;       // (front, first row) of every forward tile
  int2* btiles = nullptr;       // (front, first pivot) of every backward tile
  int* k = nullptr;             // pivots per front
  int* f = nullptr;             // front order k + m
  int64_t* Foff = nullptr;      // offset of the f x f front workspace (column-major)
  int64_t* Moff = nullptr;      // offset of X_t in M
  int64_t* Doff = nullptr;      // offset of 1/D in Dinv
  int64_t* rowoff = nullptr;    // offset of the front's row list (prefix sum of f)
  int* rows = nullptr;          // [rows_total] flat sub-vector row of each front row
  int* cmap = nullptr;          // [rows_total] parent front position of each update row
  int* child_ptr = nullptr;     // [nfronts+1]
  int* child_idx = nullptr;
  int64_t* amap_ptr = nullptr;  // [nfronts+1]
  int* amap_pos = nullptr;      // front position r + c f of each assembled entry
  int64_t* amap_val = nullptr;  // index into Aval
  double2* Aval = nullptr;      // concatenated local matrix values
  double2* F = nullptr;         // factorisation workspace (freed after setup)
  void* M = nullptr;            // X_t factors (double2 or float2)
  void* Dinv = nullptr;         // 1/D (double2 or float2)
  void* Win = nullptr;          // front vectors [rows_total][s_cap]
  void* Wout = nullptr;
  int s_cap = 0;
  int* gidx = nullptr;          // [nsub_rows] global row of each sub-vector row (R_i)
  int* own = nullptr;           // [n] sub-vector row of the owning copy (D_i Boolean)
  int* perturbed = nullptr;     // device counter
};

// --- sparse products ---
// Y = A X (mode 0) or Y = B - A X (mode 1); X, Y, B row-major [n][s] complex
void spmm_split(const DevSplitCsr& A, const double2* X, double2* Y, const double2* B, int s, int mode,
                cudaStream_t st);
// Y = R X for a real CSR R (rows x cols) on complex blocks
void spmm_real(int64_t nrows, const int64_t* rp, const int32_t* col, const double* val, const double2* X,
               double2* Y, int s, cudaStream_t st);

// --- restriction / prolongation ---
void gather_rows(const int* idx, int64_t nrows, const double2* X, double2* Y, int s, cudaStream_t st);
void scatter_owned(const int* own, int64_t n, const double2* Xsub, const double2* Q, double2* Z, int s,
                   cudaStream_t st);

// --- multifrontal ---
void mf_factor(DevMF& mf, double tau_abs, cudaStream_t st);
void mf_solve(DevMF& mf, void* Xsub, int s, cudaStream_t st);   // Xsub double2 or float2 (mf.fp32)
void gather_rows_f32(const int* idx, int64_t nrows, const double2* X, float2* Y, int s, cudaStream_t st);
void scatter_owned_f32(const int* own, int64_t n, const float2* Xsub, const double2* Q, double2* Z, int s,
                       cudaStream_t st);

// --- Krylov (one Krylov space per column) ---
// Vector-typed arrays hold double2 (fp32 = 0) or float2 (fp32 = 1); the
// Hessenberg data, rotations and norms are FP64 in both cases.
struct DevKrylov {
  int m = 0, s = 0, fp32 = 0;
  int64_t n = 0;
  void* V = nullptr;        // [(m+1)][n][s]
  void* Zk = nullptr;       // [m][n][s]
  void* W = nullptr;        // [n][s]
  double2* H = nullptr;     // [s][(m+1) m] Hessenberg, rotated in place
  double2* hpart = nullptr; // partial dot products [nblk][m+1][s]
  double2* h1 = nullptr;    // [m+1][s]
  double2* h2 = nullptr;    // [m+1][s]
  double* cs = nullptr;     // [s][m] Givens cosines (real)
  double2* sn = nullptr;    // [s][m] Givens sines
  double2* g = nullptr;     // [s][m+1]
  double2* y = nullptr;     // [s][m]
  double* beta = nullptr;   // [s] norms
  double* res = nullptr;    // [s] residual estimates |g_{j+1}|
  double* tol = nullptr;    // [s] absolute stop tolerance per column
  int* kc = nullptr;        // [s] accepted Arnoldi steps
  int* done = nullptr;      // [s]
  int nblk = 0;
};

void column_norms(const void* X, int64_t n, int s, double* out, DevKrylov& K, cudaStream_t st);
void krylov_start(DevKrylov& K, const void* R, cudaStream_t st);  // V0 = R/beta, g = beta e1, flags
void krylov_arnoldi(DevKrylov& K, int j, cudaStream_t st);         // CGS2 of W against V_0..j, H, Givens
void krylov_update(DevKrylov& K, void* X, cudaStream_t st);        // X += Zk y
void axpy_cols_zero(double2* X, int64_t count, cudaStream_t st);

// --- FP32 coarse level (mixed form) ---
void spmm_split_f32(const DevSplitCsr& A, const float2* X, float2* Y, int s, cudaStream_t st);
void gather_rows_ff(const int* idx, int64_t nrows, const float2* X, float2* Y, int s, cudaStream_t st);
void scatter_owned_ff(const int* own, int64_t n, const float2* Xsub, float2* Z, int s, cudaStream_t st);
void cast_d2f(const double2* X, float2* Y, int64_t count, cudaStream_t st);
void cast_f2d(const float2* X, double2* Y, int64_t count, cudaStream_t st);

// --- right-hand sides / layout ---
void scatter_point_sources(double2* B, int64_t n, int s, const int* idx, const double2* val, int nent,
                           cudaStream_t st);
void transpose_to_rows(const double2* F, double2* B, int64_t n, int s, cudaStream_t st);    // [s][n] -> [n][s]
void transpose_from_rows(const double2* B, double2* F, int64_t n, int s, cudaStream_t st);  // [n][s] -> [s][n]
void cast_copy(const double2* X, double2* Y, int64_t count, cudaStream_t st);

}  // namespace hz
