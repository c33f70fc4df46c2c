// Block flexible GMRES building blocks: one Krylov space shared by the s
// right-hand sides of a block (Sec. "Domain decomposition preconditioner":
// GMRES; the block form is the multi-right-hand-side variant the paper's
// multi-source setting calls for, Sec. "Conclusion").
//
// Block Arnoldi with classical Gram-Schmidt applied twice (CGS2) against the
// previous basis blocks, written as tall-skinny products:
//   H_i = V_i^H W  (s x s, i <= j),   W <- W - sum_i V_i H_i      (twice)
// and CholQR2 of the result: W = V_{j+1} R, R = R2 R1 from two Cholesky
// factorisations of the s x s Gram matrix W^H W. A direction whose Cholesky
// pivot falls below 1e-14 of its own Gram entry is dropped (deflated): its
// column of V_{j+1} is zero and its row of R is zero, so duplicated or
// linearly dependent right-hand sides give no division by zero. The block
// Hessenberg matrix is reduced by Givens rotations (s per column, zeroing the
// band of s entries below the diagonal from the bottom up); the rotated
// right-hand side gives each column's residual norm, and the block stops when
// every column has reached its tolerance. All vectors are FP64.
#include <cuda_runtime.h>

#include <algorithm>

#include "kernels.cuh"

namespace hz {

namespace {

__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 zconjmul(double2 a, double2 b) {  // conj(a) b
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double2 zadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 zsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double zabs2(double2 a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ double2 zscale(double a, double2 b) { return make_double2(a * b.x, a * b.y); }
__device__ __forceinline__ double2 zdiv(double2 a, double2 b) {
  const double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

inline unsigned grid_for(int64_t work, int block) { return (unsigned)((work + block - 1) / block); }

constexpr int BG_IG = 4;    // basis blocks per Gram pass
constexpr int BG_TR = 32;   // rows per shared-memory tile
constexpr int BG_THREADS = 256;
constexpr double DEFLATE_REL = 1e-14;

}  // namespace

// part[blk][i0+q][a][b] = sum over the block's rows r of conj(V_{i0+q}[r][a]) W[r][b]
__global__ void __launch_bounds__(BG_THREADS) k_bgram(const double2* __restrict__ Vb, int64_t vstride, int i0, int ni,
                                                      const double2* __restrict__ W, int64_t n, int s,
                                                      int64_t rows_per_blk, double2* __restrict__ part, int mstride) {
  extern __shared__ double2 sm[];
  double2* sW = sm;                       // [BG_TR][s]
  double2* sV = sm + BG_TR * s;           // [BG_IG][BG_TR][s]
  const int ss = s * s;
  const int64_t r0 = blockIdx.x * rows_per_blk;
  const int64_t r1 = min(n, r0 + rows_per_blk);
  constexpr int PPT = 4;  // pairs per thread (s <= 32)
  double2 acc[BG_IG][PPT];
#pragma unroll
  for (int q = 0; q < BG_IG; ++q)
#pragma unroll
    for (int u = 0; u < PPT; ++u) acc[q][u] = make_double2(0.0, 0.0);
  for (int64_t rt = r0; rt < r1; rt += BG_TR) {
    const int nr = (int)((r1 - rt) < BG_TR ? (r1 - rt) : BG_TR);
    for (int e = threadIdx.x; e < nr * s; e += BG_THREADS) {
      sW[e] = W[rt * s + e];
      for (int q = 0; q < ni; ++q) sV[q * BG_TR * s + e] = Vb[(int64_t)(i0 + q) * vstride + rt * s + e];
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < PPT; ++u) {
      const int p = threadIdx.x + u * BG_THREADS;
      if (p >= ss) break;
      const int a = p / s, b = p - a * s;
      for (int r = 0; r < nr; ++r) {
        const double2 w = sW[r * s + b];
#pragma unroll
        for (int q = 0; q < BG_IG; ++q)
          if (q < ni) {
            const double2 v = sV[(q * BG_TR + r) * s + a];
            acc[q][u].x = fma(v.x, w.x, fma(v.y, w.y, acc[q][u].x));
            acc[q][u].y = fma(v.x, w.y, fma(-v.y, w.x, acc[q][u].y));
          }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < PPT; ++u) {
    const int p = threadIdx.x + u * BG_THREADS;
    if (p >= ss) break;
    for (int q = 0; q < ni; ++q) part[((int64_t)blockIdx.x * mstride + i0 + q) * ss + p] = acc[q][u];
  }
}

// out[i][p] = sum over blocks of part[blk][i][p], fixed order
__global__ void k_bgram_reduce(const double2* __restrict__ part, int nblk, int ni, int ss, int mstride,
                               double2* __restrict__ out) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= ni * ss) return;
  const int i = g / ss, p = g - i * ss;
  double2 a = make_double2(0.0, 0.0);
  for (int b = 0; b < nblk; ++b) a = zadd(a, part[((int64_t)b * mstride + i) * ss + p]);
  out[(int64_t)i * ss + p] = a;
}

// W[r][b] -= sum_{i < ni} sum_a V_i[r][a] h[i][a][b]
__global__ void k_bupdate(const double2* __restrict__ Vb, int64_t vstride, int ni, const double2* __restrict__ h,
                          double2* __restrict__ W, int64_t n, int s) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= n * s) return;
  const int64_t r = g / s;
  const int b = (int)(g - r * s);
  double2 w = W[g];
  for (int i = 0; i < ni; ++i) {
    const double2* v = Vb + (int64_t)i * vstride + r * s;
    const double2* hi = h + (int64_t)i * s * s;
    for (int a = 0; a < s; ++a) w = zsub(w, zmul(v[a], hi[a * s + b]));
  }
  W[g] = w;
}

// Cholesky of the Gram matrix G = W^H W (s x s, G[a][b]) with deflation:
// R (upper triangular, R[a][b] row-major) with G ~ R^H R; a pivot below
// DEFLATE_REL of its Gram entry gives a zero row. Accumulates R_acc <- R R_acc
// when `chain` (the second CholQR pass), counts deflated directions.
__global__ void k_bchol(const double2* __restrict__ G, int s, double2* __restrict__ R, double2* __restrict__ Racc,
                        int chain, int* __restrict__ deflated) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int nd = 0;
  for (int a = 0; a < s; ++a)
    for (int b = 0; b < s; ++b) R[a * s + b] = make_double2(0.0, 0.0);
  for (int j = 0; j < s; ++j) {
    double d = G[j * s + j].x;
    for (int k = 0; k < j; ++k) d -= zabs2(R[k * s + j]);
    if (!(d > DEFLATE_REL * G[j * s + j].x) || !(d > 0.0)) {
      ++nd;
      continue;  // row j stays zero
    }
    const double rjj = sqrt(d);
    R[j * s + j] = make_double2(rjj, 0.0);
    for (int l = j + 1; l < s; ++l) {
      double2 v = G[j * s + l];
      for (int k = 0; k < j; ++k) v = zsub(v, zconjmul(R[k * s + j], R[k * s + l]));
      R[j * s + l] = zscale(1.0 / rjj, v);
    }
  }
  if (chain) {  // Racc <- R Racc (both upper triangular)
    double2 T[32 * 32];
    for (int a = 0; a < s; ++a)
      for (int b = 0; b < s; ++b) {
        double2 v = make_double2(0.0, 0.0);
        for (int k = a; k <= b; ++k) v = zadd(v, zmul(R[a * s + k], Racc[k * s + b]));
        T[a * s + b] = v;
      }
    for (int e = 0; e < s * s; ++e) Racc[e] = T[e];
  } else {
    for (int e = 0; e < s * s; ++e) Racc[e] = R[e];
  }
  if (deflated) atomicAdd(deflated, nd);
}

// Vout[r][:] = W[r][:] R^{-1} (x R = w, row by row); zero where R[b][b] = 0
// (W and Vout may be the same block: each thread reads its whole row first)
__global__ void k_btrsm_rows(const double2* W, int64_t n, int s, const double2* __restrict__ R, double2* Vout) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= n) return;
  double2 x[32], w[32];
  for (int b = 0; b < s; ++b) w[b] = W[r * s + b];
  for (int b = 0; b < s; ++b) {
    double2 v = w[b];
    for (int a = 0; a < b; ++a) v = zsub(v, zmul(x[a], R[a * s + b]));
    const double2 d = R[b * s + b];
    x[b] = (d.x == 0.0 && d.y == 0.0) ? make_double2(0.0, 0.0) : zdiv(v, d);
  }
  for (int b = 0; b < s; ++b) Vout[r * s + b] = x[b];
}

// Start of a cycle: G = [S0; 0] from the CholQR2 factor S0 of the residual
// block, residual norms, done flags.
__global__ void k_bstart(int s, int m, const double2* __restrict__ S0, double2* __restrict__ Gr,
                         const double* __restrict__ tol, double* __restrict__ res, int* __restrict__ done,
                         int* __restrict__ kb) {
  const int c = threadIdx.x;
  if (c >= s) return;
  const int ld = (m + 1) * s;
  double nrm = 0.0;
  for (int r = 0; r < ld; ++r) {
    const double2 v = r < s ? S0[r * s + c] : make_double2(0.0, 0.0);
    Gr[(int64_t)c * ld + r] = v;
    nrm += zabs2(v);
  }
  res[c] = sqrt(nrm);
  done[c] = res[c] <= tol[c] ? 1 : 0;
  if (c == 0) *kb = 0;
}

// Givens rotation (c real, s complex) that zeroes b against a:
// [c, s; -conj(s), c] (a, b) = (r, 0)
__device__ __forceinline__ void bgivens(double2 a, double2 b, double& c, double2& sn) {
  const double aa = sqrt(zabs2(a)), bb = sqrt(zabs2(b));
  if (bb == 0.0) {
    c = 1.0;
    sn = make_double2(0.0, 0.0);
  } else if (aa == 0.0) {
    c = 0.0;
    sn = make_double2(b.x / bb, -b.y / bb);
  } else {
    const double t = sqrt(aa * aa + bb * bb);
    c = aa / t;
    sn = zmul(make_double2(a.x / aa, a.y / aa), make_double2(b.x / t, -b.y / t));
  }
}
__device__ __forceinline__ void brot(double c, double2 sn, double2& x1, double2& x2) {
  const double2 y1 = zadd(zscale(c, x1), zmul(sn, x2));
  const double2 y2 = zsub(zscale(c, x2), zmul(make_double2(sn.x, -sn.y), x1));
  x1 = y1;
  x2 = y2;
}

// Block column j of the Hessenberg matrix: coefficients h1 + h2 of the two
// Gram-Schmidt passes above, R below; the previous rotations, the new ones
// (s per column, bottom-up over the band), the rotated right-hand side and
// each column's residual norm. One CTA of s threads (thread c = column j s + c).
__global__ void k_bhess(int s, int m, int j, const double2* __restrict__ h1, const double2* __restrict__ h2,
                        const double2* __restrict__ R, double2* __restrict__ Hd, double* __restrict__ rc,
                        double2* __restrict__ rsn, double2* __restrict__ Gr, const double* __restrict__ tol,
                        double* __restrict__ res, int* __restrict__ done, int* __restrict__ kb) {
  const int c = threadIdx.x;
  const int ld = (m + 1) * s;
  const int J = j * s + c;
  double2* col = Hd + (int64_t)J * ld;
  if (c < s) {
    for (int i = 0; i <= j; ++i)
      for (int a = 0; a < s; ++a) {
        const int64_t e = ((int64_t)i * s + a) * s + c;
        col[i * s + a] = zadd(h1[e], h2[e]);
      }
    for (int a = 0; a < s; ++a) col[(j + 1) * s + a] = R[a * s + c];
    for (int r = (j + 2) * s; r < ld; ++r) col[r] = make_double2(0.0, 0.0);
    // rotations of the previous block columns
    for (int Jp = 0; Jp < j * s; ++Jp)
      for (int l = s; l >= 1; --l) brot(rc[Jp * s + l - 1], rsn[Jp * s + l - 1], col[Jp + l - 1], col[Jp + l]);
  }
  __syncthreads();
  // the new block's columns in order: column c' makes its rotations, the later columns apply them
  for (int cp = 0; cp < s; ++cp) {
    const int Jp = j * s + cp;
    if (c == cp) {
      double2* cc = Hd + (int64_t)Jp * ld;
      for (int l = s; l >= 1; --l) {
        double cs;
        double2 sn;
        bgivens(cc[Jp + l - 1], cc[Jp + l], cs, sn);
        rc[Jp * s + l - 1] = cs;
        rsn[Jp * s + l - 1] = sn;
        brot(cs, sn, cc[Jp + l - 1], cc[Jp + l]);
        cc[Jp + l] = make_double2(0.0, 0.0);
      }
    }
    __syncthreads();
    if (c < s && c > cp)
      for (int l = s; l >= 1; --l) brot(rc[Jp * s + l - 1], rsn[Jp * s + l - 1], col[Jp + l - 1], col[Jp + l]);
    __syncthreads();
  }
  // the right-hand side (thread c = right-hand side c) and the residual estimates
  if (c < s) {
    double2* g = Gr + (int64_t)c * ld;
    for (int cp = 0; cp < s; ++cp) {
      const int Jp = j * s + cp;
      for (int l = s; l >= 1; --l) brot(rc[Jp * s + l - 1], rsn[Jp * s + l - 1], g[Jp + l - 1], g[Jp + l]);
    }
    double nrm = 0.0;
    for (int a = 0; a < s; ++a) nrm += zabs2(g[(j + 1) * s + a]);
    res[c] = sqrt(nrm);
    if (res[c] <= tol[c]) done[c] = 1;
    if (c == 0) *kb = j + 1;
  }
}

// Y = T^{-1} G[0:K] (T the rotated Hessenberg's upper triangle, K = kb s),
// one thread per right-hand side; a zero diagonal (deflated direction)
// gives a zero coefficient
__global__ void k_bls(int s, int m, const double2* __restrict__ Hd, const double2* __restrict__ Gr,
                      const int* __restrict__ kb, double2* __restrict__ Y) {
  const int c = threadIdx.x;
  if (c >= s) return;
  const int ld = (m + 1) * s;
  const int K = *kb * s;
  const double2* g = Gr + (int64_t)c * ld;
  double2* y = Y + (int64_t)c * m * s;
  for (int i = K - 1; i >= 0; --i) {
    double2 v = g[i];
    for (int l = i + 1; l < K; ++l) v = zsub(v, zmul(Hd[(int64_t)l * ld + i], y[l]));
    const double2 d = Hd[(int64_t)i * ld + i];
    y[i] = (sqrt(zabs2(d)) <= 1e-300) ? make_double2(0.0, 0.0) : zdiv(v, d);
  }
}

// X[r][c] += sum_{t < K} Zk_{t / s}[r][t % s] Y[c][t]
__global__ void k_bsol_update(const double2* __restrict__ Zk, int64_t vstride, const double2* __restrict__ Y,
                              const int* __restrict__ kb, double2* __restrict__ X, int64_t n, int s, int m) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= n * s) return;
  const int64_t r = g / s;
  const int c = (int)(g - r * s);
  const int K = *kb * s;
  double2 x = X[g];
  const double2* y = Y + (int64_t)c * m * s;
  for (int t = 0; t < K; ++t) x = zadd(x, zmul(Zk[(int64_t)(t / s) * vstride + r * s + (t % s)], y[t]));
  X[g] = x;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static void bgram(DevBlockKrylov& B, const double2* Vb, int64_t vstride, int ni, const double2* W, double2* out,
                  cudaStream_t st) {
  const int s = B.s;
  const int64_t rpb = (B.n + B.nblk - 1) / B.nblk;
  const size_t shm = sizeof(double2) * (size_t)BG_TR * s * (1 + BG_IG);
  for (int i0 = 0; i0 < ni; i0 += BG_IG)
    { k_bgram<<<B.nblk, BG_THREADS, shm, st>>>(Vb, vstride, i0, std::min(BG_IG, ni - i0), W, B.n, s, rpb, B.part,
                                               B.m + 1); count_launch(); }
  { k_bgram_reduce<<<grid_for((int64_t)ni * s * s, 256), 256, 0, st>>>(B.part, B.nblk, ni, s * s, B.m + 1, out); count_launch(); }
}

// CholQR2: W = Vout Racc (W overwritten by the first pass)
static void cholqr2(DevBlockKrylov& B, double2* W, double2* Vout, cudaStream_t st) {
  const int s = B.s;
  const unsigned gr = grid_for(B.n, 128);
  bgram(B, W, 0, 1, W, B.gram, st);
  { k_bchol<<<1, 1, 0, st>>>(B.gram, s, B.R, B.Racc, 0, B.deflated); count_launch(); }
  { k_btrsm_rows<<<gr, 128, 0, st>>>(W, B.n, s, B.R, W); count_launch(); }
  bgram(B, W, 0, 1, W, B.gram, st);
  { k_bchol<<<1, 1, 0, st>>>(B.gram, s, B.R, B.Racc, 1, nullptr); count_launch(); }
  { k_btrsm_rows<<<gr, 128, 0, st>>>(W, B.n, s, B.R, Vout); count_launch(); }
}

void block_krylov_start(DevBlockKrylov& B, double2* R, cudaStream_t st) {
  cudaMemsetAsync(B.deflated, 0, sizeof(int), st);
  cholqr2(B, R, B.V, st);  // R is overwritten
  { k_bstart<<<1, 32, 0, st>>>(B.s, B.m, B.Racc, B.Gr, B.tol, B.res, B.done, B.kb); count_launch(); }
}

void block_krylov_arnoldi(DevBlockKrylov& B, int j, cudaStream_t st) {
  const int s = B.s;
  const int64_t vs = B.n * s;
  const unsigned gr = grid_for(vs, 256);
  bgram(B, B.V, vs, j + 1, B.W, B.h1, st);
  { k_bupdate<<<gr, 256, 0, st>>>(B.V, vs, j + 1, B.h1, B.W, B.n, s); count_launch(); }
  bgram(B, B.V, vs, j + 1, B.W, B.h2, st);
  { k_bupdate<<<gr, 256, 0, st>>>(B.V, vs, j + 1, B.h2, B.W, B.n, s); count_launch(); }
  cholqr2(B, B.W, B.V + (int64_t)(j + 1) * vs, st);
  { k_bhess<<<1, 32, 0, st>>>(s, B.m, j, B.h1, B.h2, B.Racc, B.Hd, B.rc, B.rsn, B.Gr, B.tol, B.res, B.done, B.kb); count_launch(); }
}

void block_krylov_update(DevBlockKrylov& B, double2* X, cudaStream_t st) {
  { k_bls<<<1, 32, 0, st>>>(B.s, B.m, B.Hd, B.Gr, B.kb, B.Y); count_launch(); }
  { k_bsol_update<<<grid_for(B.n * B.s, 256), 256, 0, st>>>(B.Zk, B.n * B.s, B.Y, B.kb, X, B.n, B.s, B.m); count_launch(); }
}

void block_krylov_attrs() {
  const int shm = (int)(sizeof(double2) * (size_t)BG_TR * 32 * (1 + BG_IG));
  cudaFuncSetAttribute(k_bgram, cudaFuncAttributeMaxDynamicSharedMemorySize, shm);
}

}  // namespace hz
