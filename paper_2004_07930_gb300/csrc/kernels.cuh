// Device kernels of the two-level ORAS / FGMRES hot path (declarations).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

namespace hz {

// Kernel launches issued by the library (graph replays add the kernels of
// the replayed graph); read through hz_get_info.
extern std::atomic<long long> g_kernel_launches;
inline void count_launch(long long n = 1) { g_kernel_launches.fetch_add(n, std::memory_order_relaxed); }

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
  float2* val_re_df = nullptr;  // double-float (hi, lo) copies (mixed form, emulated FP64)
  float2* val_im_df = nullptr;
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
  const char* fhalf_h = nullptr;  // host [nlevels]: every forward tile of the level has <= 64 output rows
  const char* bhalf_h = nullptr;  // host [nlevels]: the same for the backward tiles
  int* btile_ptr_h = nullptr;   // host [nlevels+1] backward tiles per level
  int* level_list = nullptr;    // device [nfronts] front ids ordered by height
  int* frb_ptr_h = nullptr;     // host [nlevels+1] forward row blocks per level
  int* brb_ptr_h = nullptr;     // host [nlevels+1] backward row blocks per level
  int64_t* level_row_h = nullptr;  // host [nlevels+1] first front row of each level
  int64_t max_slots = 0;        // partial-result slots of the largest level
  int4* ftiles = nullptr;       // forward tiles (front, first row, first column, slot)
  int4* btiles = nullptr;       // backward tiles (front, first pivot, first row, slot)
  int4* frb = nullptr;          // forward row blocks (front, first row, tiles, first slot)
  int4* brb = nullptr;          // backward row blocks
  int* row_front = nullptr;     // [rows_total] front of each front row
  int* row_local = nullptr;     // [rows_total] position inside its front
  int64_t* cptr = nullptr;      // [rows_total+1] extend-add sources of each front row
  int* cidx = nullptr;          // child update rows, in child order
  int64_t cidx_n = 0;           // entries of cidx
  int64_t ftiles_n = 0, btiles_n = 0;  // tiles of each sweep (all levels)
  void* P = nullptr;            // partial tile results [max_slots][128][s_cap]
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
  double2* Aval = nullptr;      // concatenated local matrix values (freed after the factorisation)
  int64_t aval_n = 0;
  void* F = nullptr;            // factorisation workspace, double2 or float2 (fr32), freed after setup
  int fr32 = 0;                 // factorisation in complex FP32 (mixed form, fine level)
  float factor_ms = 0.f, inverse_ms = 0.f;  // device time of the assembly + LDL^T and of the partitioned inverse
  // factorisation schedule: per level the fronts factored pivot by pivot (f <= FA_SMALL) and the
  // fronts factored by panels; per panel step the trailing-update tiles (front, tile row, tile column)
  int* fa_small = nullptr;
  int* fa_small_ptr_h = nullptr;  // host [nlevels+1]
  int* fa_big = nullptr;
  int* fa_big_ptr_h = nullptr;    // host [nlevels+1]
  int* fa_step_ptr_h = nullptr;   // host [nlevels+1] panel steps of each level (prefix)
  int4* fa_tiles = nullptr;
  int* fa_tile_ptr_h = nullptr;   // host [steps+1]
  int4* fi_tiles = nullptr;       // blocked inverse: update tiles (front, tile row, tile column, panel slot)
  int* fi_tile_ptr_h = nullptr;   // host [steps+1]
  int64_t* fa_pan_off = nullptr;  // [big fronts] offset of each large front's scratch panel (f x FA_NB_H)
  void* fa_pan = nullptr;         // scratch panels, element type of F
  void* M = nullptr;            // X_t factors (double2 or float2), column-major f x k
  void* MT = nullptr;           // X_t^T, column-major k x f (backward sweep)
  void* Dinv = nullptr;         // 1/D (double2 or float2)
  void* Wout = nullptr;         // front vectors [rows_total][s_cap]: y_P and parent updates
  int s_cap = 0;
  int* gidx = nullptr;          // [nsub_rows] global row of each sub-vector row (R_i)
  int* own = nullptr;           // [n] sub-vector row of the owning copy (D_i Boolean)
  int* perturbed = nullptr;     // device counter
  // tensor-core sweeps (complex FP32 form): tiles with at least TC_MIN_ROWS output rows and
  // TC_MIN_K reduction indices run as tcgen05 MMAs (three-term TF32 split, FP32 accumulation in
  // TMEM) when the block has 9-16 columns; the others keep the SIMT kernel
  int tc = 0;                   // packed tensor-core tiles present
  int* fs_ptr_h = nullptr;      // host [nlevels+1] forward SIMT tiles per level (tensor-core mode)
  int* bs_ptr_h = nullptr;      // host [nlevels+1] backward SIMT tiles per level
  int* ftc_ptr_h = nullptr;     // host [nlevels+1] forward tensor-core tiles per level
  int* btc_ptr_h = nullptr;     // host [nlevels+1] backward tensor-core tiles per level
  int4* ftiles_s = nullptr;     // forward tiles left to the SIMT kernel
  int4* btiles_s = nullptr;
  int4* ftiles_tc = nullptr;    // forward tensor-core tiles
  int4* btiles_tc = nullptr;
  int64_t* ftc_off = nullptr;   // byte offset of each tensor-core tile in TC
  int64_t* btc_off = nullptr;
  int64_t ftc_n = 0, btc_n = 0; // tensor-core tiles in each sweep
  unsigned char* TC = nullptr;  // packed factor tiles (per 16-column chunk: Re plane, Im plane)
  int64_t tc_bytes = 0;
  int* tc_err = nullptr;        // device flag: a tensor-core tile gave up waiting on a barrier
  cudaStream_t side = nullptr;  // tensor-core mode: the SIMT tiles of a level run here, beside the tcgen05 tiles
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // persistent sweeps (one launch per direction): tiles in ticket order with slots numbered over all
  // levels, row blocks (front, first row, tiles, first slot), slot -> row block, per-front row-block
  // counts, parent and child counts, and the counters reset before every sweep
  int persistent = 0;
  int pt_nf = 0, pt_nb = 0;     // tiles of the forward / backward sweep
  int prb_nf = 0, prb_nb = 0;   // row blocks with partial tiles
  int4* ptf = nullptr;          // forward tiles, leaves first
  int4* ptb = nullptr;          // backward tiles, roots first
  int* slot_rb_f = nullptr;
  int* slot_rb_b = nullptr;
  int4* prb_f = nullptr;
  int4* prb_b = nullptr;
  int* nrb_f = nullptr;         // [nfronts] row blocks of each front, forward
  int* nrb_b = nullptr;         // [nfronts] backward
  int* parent = nullptr;        // [nfronts] parent front (-1: root)
  int* bdep = nullptr;          // [nfronts] nearest ancestor with pivots (-1: none): backward dependency
  int* nchild = nullptr;        // [nfronts]
  int* cnt = nullptr;           // ticket | row-block counts | front counts | ready children
  int cnt_n = 0;
  int64_t pslots = 0;           // partial slots of the larger sweep
  int* sw_err = nullptr;        // device flag: a persistent sweep gave up waiting
  int sweep_grid = 0;           // resident CTAs of the sweep kernel
};

// fronts of order <= FA_SMALL are factored pivot by pivot, larger ones by panels of FA_NB_H pivots
// with FA_TILE_H x FA_TILE_H trailing-update tiles (FA_NB / FA_TILE in factor.cu)
constexpr int FA_SMALL = 160;
constexpr int FA_NB_H = 32;
constexpr int FA_TILE_H = 64;

// tensor-core tile eligibility (output rows, reduction length) and packing geometry
constexpr int TC_MIN_ROWS = 32;
constexpr int TC_MIN_K = 32;
inline int64_t tc_tile_bytes(int nr, int nk) {  // nr output rows, nk reduction indices
  const int64_t nr8 = (nr + 7) / 8 * 8, nch = (nk + 15) / 16;
  return nch * 2 * nr8 * 64;
}

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
void mf_solve(DevMF& mf, void* Xsub, int s, cudaStream_t st);  // Xsub double2 or float2 (mf.fp32)
bool mf_tc_usable(const DevMF& mf, int s);  // the block width runs the tensor-core sweeps
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
  int* reorth = nullptr;    // [s] second Gram-Schmidt pass needed
  double2* Hraw = nullptr;  // [s][(m+1) m] unrotated Hessenberg (recycling only; may be NULL)
  int nblk = 0;
  // double-float Arnoldi (FP64 Krylov spaces of the mixed form, emulate_fp64): A z arrives in
  // double-float (Wdf); the basis V stays FP64 and is split into FP32 pairs as it is read
  int df = 0;
  float4* Wdf = nullptr;    // [n][s]
  float4* hdf = nullptr;    // [m+1][s] Gram-Schmidt coefficients in double-float
};

// --- double-float products (mixed form, emulated FP64; df.cu) ---
// X [count] complex FP64 -> (re_hi, re_lo, im_hi, im_lo)
void to_df(const double2* X, float4* Y, int64_t count, cudaStream_t st);
// Y = A X (mode 0) or Y = B - A X (mode 1) with X in double-float, A's double-float values;
// with Ydf, A X in double-float instead of Y
void spmm_split_df(const DevSplitCsr& A, const float4* X, double2* Y, const double2* B, int s, int mode,
                   cudaStream_t st, float4* Ydf = nullptr);

// Y = R X for a real CSR R with double-float values, X in double-float, Y in FP64
void spmm_real_df(int64_t nrows, const int64_t* rp, const int32_t* col, const float2* val, const float4* X,
                  double2* Y, int s, cudaStream_t st);

// --- Krylov subspace recycling (option recycle): k vectors U shared by all columns,
// C = A U orthonormal; blocks [n][k] row-major ---
void recycle_dot(const double2* Cb, int k, const double2* W, int s, int64_t n, double2* part, int nblk, double2* out,
                 cudaStream_t st);  // out[a][c] = sum_r conj(C[r][a]) W[r][c]
void recycle_axpy(const double2* Cb, int k, const double2* Y, double2* W, int s, int64_t n, double alpha,
                  cudaStream_t st);  // W[r][c] += alpha sum_a C[r][a] Y[a][c]
void recycle_corr(const double2* Bc, const double2* y, const int* kc, int k, int s, int m, double2* T,
                  cudaStream_t st);  // T[a][c] = sum_{j < kc[c]} Bc[j][a][c] y[c][j]
void recycle_build(const double2* Zk, int64_t vstride, int s, int col, const double2* P, int m, int knew,
                   double2* U, int k, int q0, int64_t n, cudaStream_t st);  // U[r][q0+q] = sum_j Zk_j[r][col] P[j + q m]
void recycle_trsm(double2* W, int64_t n, int k, const double2* R, cudaStream_t st);  // W <- W R^{-1} (R k x k upper, row-major)
void recycle_copy(const double2* src, int sk, int s0, double2* dst, int dk, int d0, int count, int64_t n,
                  cudaStream_t st);  // dst[r][d0 + q] = src[r][s0 + q]

// --- block Krylov (one Krylov space shared by the s columns; FP64, s <= 32) ---
struct DevBlockKrylov {
  int m = 0, s = 0, nblk = 0;
  int64_t n = 0;
  double2* V = nullptr;      // [(m+1)][n][s] orthonormal basis blocks (the per-column form's arrays)
  double2* Zk = nullptr;     // [m][n][s] preconditioned blocks
  double2* W = nullptr;      // [n][s]
  double2* Hd = nullptr;     // block Hessenberg, column-major ((m+1) s) x (m s), rotated in place
  double2* Gr = nullptr;     // rotated right-hand side, column-major ((m+1) s) x s
  double* rc = nullptr;      // Givens cosines [m s][s]
  double2* rsn = nullptr;    // Givens sines [m s][s]
  double2* part = nullptr;   // partial Gram blocks [nblk][m+1][s][s]
  double2* h1 = nullptr;     // [m+1][s][s] first Gram-Schmidt pass
  double2* h2 = nullptr;     // [m+1][s][s] second pass
  double2* gram = nullptr;   // [s][s]
  double2* R = nullptr;      // [s][s] one CholQR factor
  double2* Racc = nullptr;   // [s][s] R2 R1
  double2* Y = nullptr;      // [s][m s] least-squares coefficients
  double* res = nullptr;     // [s] residual estimates
  double* tol = nullptr;     // [s]
  int* done = nullptr;       // [s]
  int* kb = nullptr;         // accepted block steps
  int* deflated = nullptr;   // directions dropped by CholQR in the current cycle
};
void block_krylov_start(DevBlockKrylov& B, double2* R, cudaStream_t st);  // V0 S0 = R (R overwritten), G = [S0; 0]
void block_krylov_arnoldi(DevBlockKrylov& B, int j, cudaStream_t st);     // CGS2 + CholQR2, Hessenberg, Givens
void block_krylov_update(DevBlockKrylov& B, double2* X, cudaStream_t st); // X += Z Y
void block_krylov_attrs();

void column_norms(const void* X, int64_t n, int s, double* out, DevKrylov& K, cudaStream_t st);
void krylov_start(DevKrylov& K, const void* R, cudaStream_t st);  // V0 = R/beta, g = beta e1, flags
void krylov_arnoldi(DevKrylov& K, int j, cudaStream_t st);         // CGS (+selective 2nd pass), H, Givens
void krylov_update(DevKrylov& K, void* X, cudaStream_t st);        // X += Zk y
void axpy_cols_zero(double2* X, int64_t count, cudaStream_t st);

// --- FP32 coarse level (mixed form) ---
void spmm_split_f32(const DevSplitCsr& A, const float2* X, float2* Y, int s, cudaStream_t st,
                    const float2* B = nullptr);  // Y = A X, or B - A X
void spmm_real_f32(int64_t nrows, const int64_t* rp, const int32_t* col, const float* val, const float2* X,
                   float2* Y, int s, cudaStream_t st);
void scatter_owned_fq(const int* own, int64_t n, const float2* Xsub, const float2* Q, double2* Z, int s,
                      cudaStream_t st);
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
// debug_bounds: atomicMin(err, id) if some a[i * stride], i < count, lies outside [lo, hi)
void check_index_range(const int* a, int64_t count, int stride, int64_t lo, int64_t hi, int* err, int id,
                       cudaStream_t st);
// one column c of an [n][s] block
void col_zero(double2* X, int64_t n, int s, int c, cudaStream_t st);
void col_copy(const double2* X, double2* Y, int64_t n, int s, int c, cudaStream_t st);
void col_get(const double2* X, double2* y, int64_t n, int s, int c, cudaStream_t st);  // y [n]
// FWI misfit / adjoint / gradient (fwi.cu); blocks node-major [n][s]
cudaError_t fwi_set_tables(const double* Mhat, const double* Bhat, cudaStream_t st);  // Mhat [20][20], Bhat [4][20][20]
void fwi_residual(int nr, int s, const int* pidx, const double* pw, const double2* U, const double2* d, double2* r,
                  cudaStream_t st);
void fwi_chi(int64_t m, const double2* r, double* chi, cudaStream_t st);
void fwi_adjoint_rhs(int nt, int s, int nr, const int* trow, const int* tptr, const int* tk, const double* tw,
                     const double2* r, double2* B, cudaStream_t st);
void fwi_gradient(int64_t ne, int s, const int* l2g, const double* vol, const double* farea, const double* m,
                  double omega, const double2* U, const double2* L, double* g, cudaStream_t st);

}  // namespace hz
