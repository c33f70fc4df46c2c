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
  for (int64_t p = rp_re[r], pe = rp_re[r + 1]; p < pe; ++p) {
    double a = val_re[p];
    double2 x = X[(int64_t)col_re[p] * s + c];
    ar = fma(a, x.x, ar);
    ai = fma(a, x.y, ai);
  }
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
  k_spmm_split<<<grid_for(work, 256), 256, 0, st>>>(A.n, s, A.rp_re, A.col_re, A.val_re, A.rp_im, A.col_im,
                                                    A.val_im, X, Y, B, mode);
}

__global__ void k_spmm_real(int64_t n, int s, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                            const double* __restrict__ val, const double2* __restrict__ X, double2* __restrict__ Y) {
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t r = g / s;
  int c = (int)(g - r * s);
  if (r >= n) return;
  double ar = 0.0, ai = 0.0;
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
  k_spmm_real<<<grid_for(work, 256), 256, 0, st>>>(nrows, s, rp, col, val, X, Y);
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
  k_gather_rows<<<grid_for(nrows * s, 256), 256, 0, st>>>(idx, nrows, X, Y, s);
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
  k_scatter_owned<<<grid_for(n * s, 256), 256, 0, st>>>(own, n, Xsub, Q, Z, s);
}

// ---------------------------------------------------------------------------
// Krylov: one Arnoldi process per column, CGS2 orthogonalisation (K8),
// Givens QR of the Hessenberg matrix (K10), solution update (K12).
// ---------------------------------------------------------------------------
constexpr int IG = 8;       // basis vectors per dot-product pass
constexpr int KBLOCK = 256;

// part[blk][i0+q][c] = sum over the block's rows of conj(V_{i0+q}[r][c]) W[r][c]
__global__ void k_mdot(const double2* __restrict__ V, int64_t vstride, int i0, int ni, const double2* __restrict__ W,
                       int64_t n, int s, int64_t rows_per_blk, double2* __restrict__ part, int mstride) {
  __shared__ double2 sh[KBLOCK];
  const int nrl = blockDim.x / s;
  const int c = threadIdx.x % s, rl = threadIdx.x / s;
  double2 acc[IG];
#pragma unroll
  for (int q = 0; q < IG; ++q) acc[q] = make_double2(0.0, 0.0);
  const int64_t r0 = blockIdx.x * rows_per_blk;
  const int64_t r1 = min(n, r0 + rows_per_blk);
  if (rl < nrl) {
    for (int64_t r = r0 + rl; r < r1; r += nrl) {
      double2 w = W[r * s + c];
#pragma unroll
      for (int q = 0; q < IG; ++q)
        if (q < ni) acc[q] = conjmul_acc(V[(int64_t)(i0 + q) * vstride + r * s + c], w, acc[q]);
    }
  }
  for (int q = 0; q < ni; ++q) {
    sh[threadIdx.x] = (rl < nrl) ? acc[q] : make_double2(0.0, 0.0);
    __syncthreads();
    if (rl == 0) {
      double2 a = make_double2(0.0, 0.0);
      for (int l = 0; l < nrl; ++l) a = cadd(a, sh[l * s + c]);
      part[((int64_t)blockIdx.x * mstride + i0 + q) * s + c] = a;
    }
    __syncthreads();
  }
}

// out[i][c] = sum over blocks of part[blk][i][c]  (fixed order: deterministic)
__global__ void k_reduce_part(const double2* __restrict__ part, int nblk, int ni, int s, int mstride,
                              double2* __restrict__ out) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= ni * s) return;
  int i = g / s, c = g % s;
  double2 a = make_double2(0.0, 0.0);
  for (int b = 0; b < nblk; ++b) a = cadd(a, part[((int64_t)b * mstride + i) * s + c]);
  out[i * s + c] = a;
}

static void mdot(DevKrylov& K, const double2* V, int64_t vstride, int ni, const double2* W, double2* out,
                 cudaStream_t st) {
  const int s = K.s;
  const int block = (KBLOCK / s) * s;
  const int64_t rpb = (K.n + K.nblk - 1) / K.nblk;
  for (int i0 = 0; i0 < ni; i0 += IG)
    k_mdot<<<K.nblk, block, 0, st>>>(V, vstride, i0, std::min(IG, ni - i0), W, K.n, s, rpb, K.hpart, K.m + 1);
  k_reduce_part<<<grid_for((int64_t)ni * s, 128), 128, 0, st>>>(K.hpart, K.nblk, ni, s, K.m + 1, out);
}

// W[r][c] -= sum_{i<ni} V_i[r][c] h[i][c]
__global__ void k_update(const double2* __restrict__ V, int64_t vstride, int ni, const double2* __restrict__ h,
                         double2* __restrict__ W, int64_t n, int s) {
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= n * s) return;
  int c = (int)(g % s);
  double2 w = W[g];
  for (int i = 0; i < ni; ++i) w = cfms(V[i * vstride + g], h[i * s + c], w);
  W[g] = w;
}

__global__ void k_scale_cols(const double2* __restrict__ X, const double* __restrict__ sc, double2* __restrict__ Y,
                             int64_t n, int s) {
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= n * s) return;
  double a = sc[g % s];
  double2 x = X[g];
  Y[g] = make_double2(a * x.x, a * x.y);
}

__global__ void k_norm_finish(const double2* __restrict__ nrm2, int s, double* __restrict__ out) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < s) out[c] = sqrt(nrm2[c].x);
}

void column_norms(const double2* X, int64_t n, int s, double* out, DevKrylov& K, cudaStream_t st) {
  mdot(K, X, 0, 1, X, K.h2, st);
  k_norm_finish<<<1, 64, 0, st>>>(K.h2, s, out);
}

__global__ void k_start(int s, int m, const double2* __restrict__ nrm2, const double* __restrict__ tol,
                        double2* __restrict__ g, double* __restrict__ beta, int* __restrict__ kc,
                        int* __restrict__ done, double* __restrict__ res) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= s) return;
  double b = sqrt(nrm2[c].x);
  for (int i = 0; i <= m; ++i) g[c * (m + 1) + i] = make_double2(0.0, 0.0);
  g[c * (m + 1)] = make_double2(b, 0.0);
  kc[c] = 0;
  res[c] = b;
  done[c] = (b <= tol[c]) ? 1 : 0;
  beta[c] = b > 0.0 ? 1.0 / b : 0.0;
}

void krylov_start(DevKrylov& K, const double2* R, cudaStream_t st) {
  mdot(K, R, 0, 1, R, K.h2, st);
  k_start<<<1, 64, 0, st>>>(K.s, K.m, K.h2, K.tol, K.g, K.beta, K.kc, K.done, K.res);
  k_scale_cols<<<grid_for(K.n * K.s, 256), 256, 0, st>>>(R, K.beta, K.V, K.n, K.s);
}

// Column j of the Hessenberg matrix, previous Givens rotations, the new one,
// the rotated right-hand side g and the residual estimate |g_{j+1}|.
__global__ void k_arnoldi_finish(int s, int m, int j, const double2* __restrict__ h1, const double2* __restrict__ h2,
                                 const double2* __restrict__ nrm2, double2* __restrict__ H, double* __restrict__ cs,
                                 double2* __restrict__ sn, double2* __restrict__ g, double* __restrict__ beta,
                                 const double* __restrict__ tol, int* __restrict__ kc, int* __restrict__ done,
                                 double* __restrict__ res) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= s) return;
  const double hb = sqrt(nrm2[c].x);
  double hn2 = hb * hb;
  for (int i = 0; i <= j; ++i) hn2 += cabs2(cadd(h1[i * s + c], h2[i * s + c]));
  const bool breakdown = !(hb > 1e-14 * sqrt(hn2));
  beta[c] = breakdown ? 0.0 : 1.0 / hb;
  if (done[c]) return;
  double2* Hc = H + (int64_t)c * (m + 1) * m + (int64_t)j * (m + 1);
  for (int i = 0; i <= j; ++i) Hc[i] = cadd(h1[i * s + c], h2[i * s + c]);
  Hc[j + 1] = make_double2(breakdown ? 0.0 : hb, 0.0);
  double* csc = cs + c * m;
  double2* snc = sn + c * m;
  for (int i = 0; i < j; ++i) {
    double2 a = Hc[i], b = Hc[i + 1];
    double ci = csc[i];
    double2 si = snc[i];
    Hc[i] = cadd(make_double2(ci * a.x, ci * a.y), cmul(si, b));
    Hc[i + 1] = csub(make_double2(ci * b.x, ci * b.y), cmul(make_double2(si.x, -si.y), a));
  }
  double2 a = Hc[j], b = Hc[j + 1];
  double aa = sqrt(cabs2(a)), bb = sqrt(cabs2(b));
  double cj;
  double2 sj;
  if (bb == 0.0) {
    cj = 1.0;
    sj = make_double2(0.0, 0.0);
  } else if (aa == 0.0) {
    cj = 0.0;
    sj = make_double2(b.x / bb, -b.y / bb);  // conj(b)/|b|
  } else {
    double tt = sqrt(aa * aa + bb * bb);
    cj = aa / tt;
    double2 ph = make_double2(a.x / aa, a.y / aa);
    sj = cmul(ph, make_double2(b.x / tt, -b.y / tt));
  }
  csc[j] = cj;
  snc[j] = sj;
  Hc[j] = cadd(make_double2(cj * a.x, cj * a.y), cmul(sj, b));
  Hc[j + 1] = make_double2(0.0, 0.0);
  double2* gc = g + c * (m + 1);
  double2 gj = gc[j];
  gc[j] = make_double2(cj * gj.x, cj * gj.y);
  gc[j + 1] = cmul(make_double2(-sj.x, sj.y), gj);  // -conj(s) g_j
  kc[c] = j + 1;
  double r = sqrt(cabs2(gc[j + 1]));
  res[c] = r;
  if (r <= tol[c] || breakdown) done[c] = 1;
}

void krylov_arnoldi(DevKrylov& K, int j, cudaStream_t st) {
  const int64_t vs = K.n * K.s;
  const unsigned gr = grid_for(vs, 256);
  mdot(K, K.V, vs, j + 1, K.W, K.h1, st);
  k_update<<<gr, 256, 0, st>>>(K.V, vs, j + 1, K.h1, K.W, K.n, K.s);
  mdot(K, K.V, vs, j + 1, K.W, K.h2, st);
  k_update<<<gr, 256, 0, st>>>(K.V, vs, j + 1, K.h2, K.W, K.n, K.s);
  // norm of W into h2 slot j+1 (kept separate from the projection coefficients)
  double2* nrm = K.h2 + (int64_t)(K.m + 1) * K.s - K.s;  // last row of h2 as scratch ([m][s])
  mdot(K, K.W, 0, 1, K.W, nrm, st);
  k_arnoldi_finish<<<1, 64, 0, st>>>(K.s, K.m, j, K.h1, K.h2, nrm, K.H, K.cs, K.sn, K.g, K.beta, K.tol, K.kc, K.done,
                                     K.res);
  k_scale_cols<<<gr, 256, 0, st>>>(K.W, K.beta, K.V + (int64_t)(j + 1) * vs, K.n, K.s);
}

// y = R^{-1} g per column (R = rotated Hessenberg, kc[c] steps)
__global__ void k_ls_solve(int s, int m, const double2* __restrict__ H, const double2* __restrict__ g,
                           const int* __restrict__ kc, double2* __restrict__ y) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= s) return;
  const int k = kc[c];
  const double2* Hc = H + (int64_t)c * (m + 1) * m;
  const double2* gc = g + c * (m + 1);
  double2* yc = y + c * m;
  for (int i = k - 1; i >= 0; --i) {
    double2 v = gc[i];
    for (int l = i + 1; l < k; ++l) v = cfms(Hc[i + l * (m + 1)], yc[l], v);
    double2 d = Hc[i + i * (m + 1)];
    yc[i] = (d.x == 0.0 && d.y == 0.0) ? make_double2(0.0, 0.0) : cdiv(v, d);
  }
}

__global__ void k_sol_update(const double2* __restrict__ Zk, int64_t vstride, const double2* __restrict__ y,
                             const int* __restrict__ kc, double2* __restrict__ X, int64_t n, int s, int m) {
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= n * s) return;
  int c = (int)(g % s);
  double2 x = X[g];
  const int k = kc[c];
  for (int j = 0; j < k; ++j) x = cfma(Zk[j * vstride + g], y[c * m + j], x);
  X[g] = x;
}

void krylov_update(DevKrylov& K, double2* X, cudaStream_t st) {
  k_ls_solve<<<1, 64, 0, st>>>(K.s, K.m, K.H, K.g, K.kc, K.y);
  k_sol_update<<<grid_for(K.n * K.s, 256), 256, 0, st>>>(K.Zk, K.n * K.s, K.y, K.kc, X, K.n, K.s, K.m);
}

__global__ void k_zero(double2* X, int64_t count) {
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g < count) X[g] = make_double2(0.0, 0.0);
}
void axpy_cols_zero(double2* X, int64_t count, cudaStream_t st) {
  if (count) k_zero<<<grid_for(count, 256), 256, 0, st>>>(X, count);
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
  if (nent) k_point_sources<<<grid_for(nent, 128), 128, 0, st>>>(B, idx, val, nent);
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
  if (n * s) k_to_rows<<<grid_for(n * s, 256), 256, 0, st>>>(F, B, n, s);
}
void transpose_from_rows(const double2* B, double2* F, int64_t n, int s, cudaStream_t st) {
  if (n * s) k_from_rows<<<grid_for(n * s, 256), 256, 0, st>>>(B, F, n, s);
}

__global__ void k_copy(const double2* __restrict__ X, double2* __restrict__ Y, int64_t count) {
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g < count) Y[g] = X[g];
}
void cast_copy(const double2* X, double2* Y, int64_t count, cudaStream_t st) {
  if (count) k_copy<<<grid_for(count, 256), 256, 0, st>>>(X, Y, count);
}

}  // namespace hz
