// Krylov subspace recycling (GCRO-DR style augmentation with deflated
// restarting; Sec. "Conclusion": recycling across sources and frequencies).
//
// The context keeps k vectors U (n x k) and C = A U with orthonormal
// columns, shared by all right-hand sides of a solve. Every restart cycle
// first removes C's share of each column's residual (x += U C^H r,
// r -= C C^H r), runs the Arnoldi process on (I - C C^H) A M^{-1} (each new
// A z is projected against C, the coefficients B_j = C^H A z_j kept), and
// corrects the solution update for them (x -= U sum_j B_j y_j). After the
// cycle the harmonic Ritz vectors of the slowest column's Hessenberg matrix
// with the smallest Ritz values give new directions U_new = Z P, which join
// the kept ones (the oldest dropped beyond k); C = A U is orthonormalised by
// two Cholesky QR passes, U transformed alike. All arithmetic is FP64.
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace hz {

namespace {

inline unsigned grid_for(int64_t work, int block) { return (unsigned)((work + block - 1) / block); }

constexpr int RD_THREADS = 256;
constexpr int RD_TR = 16;  // rows per shared-memory tile

}  // namespace

// part[blk][a][c] = sum over the block's rows of conj(C[r][a]) W[r][c]
__global__ void __launch_bounds__(RD_THREADS) k_rdot(const double2* __restrict__ Cb, int k,
                                                     const double2* __restrict__ W, int s, int64_t n,
                                                     int64_t rows_per_blk, double2* __restrict__ part) {
  __shared__ double2 sC[RD_TR][16];
  __shared__ double2 sW[RD_TR][64];
  const int64_t r0 = blockIdx.x * rows_per_blk;
  const int64_t r1 = min(n, r0 + rows_per_blk);
  const int ks = k * s;
  double2 acc[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) acc[u] = make_double2(0.0, 0.0);
  for (int64_t rt = r0; rt < r1; rt += RD_TR) {
    const int nr = (int)((r1 - rt) < RD_TR ? (r1 - rt) : RD_TR);
    for (int e = threadIdx.x; e < nr * k; e += RD_THREADS) sC[e / k][e % k] = Cb[(rt + e / k) * k + e % k];
    for (int e = threadIdx.x; e < nr * s; e += RD_THREADS) sW[e / s][e % s] = W[(rt + e / s) * s + e % s];
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int p = threadIdx.x + u * RD_THREADS;
      if (p >= ks) break;
      const int a = p / s, c = p - a * s;
      for (int r = 0; r < nr; ++r) {
        const double2 v = sC[r][a], w = sW[r][c];
        acc[u].x = fma(v.x, w.x, fma(v.y, w.y, acc[u].x));
        acc[u].y = fma(v.x, w.y, fma(-v.y, w.x, acc[u].y));
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int p = threadIdx.x + u * RD_THREADS;
    if (p < ks) part[(int64_t)blockIdx.x * ks + p] = acc[u];
  }
}

__global__ void k_rreduce(const double2* __restrict__ part, int nblk, int ks, double2* __restrict__ out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= ks) return;
  double2 a = make_double2(0.0, 0.0);
  for (int b = 0; b < nblk; ++b) {
    const double2 v = part[(int64_t)b * ks + p];
    a.x += v.x;
    a.y += v.y;
  }
  out[p] = a;
}

__global__ void k_raxpy(const double2* __restrict__ Cb, int k, const double2* __restrict__ Y, double2* __restrict__ W,
                        int s, int64_t n, double alpha) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= n * s) return;
  const int64_t r = g / s;
  const int c = (int)(g - r * s);
  double2 w = W[g];
  for (int a = 0; a < k; ++a) {
    const double2 v = Cb[r * k + a], y = Y[a * s + c];
    w.x += alpha * (v.x * y.x - v.y * y.y);
    w.y += alpha * (v.x * y.y + v.y * y.x);
  }
  W[g] = w;
}

__global__ void k_rcorr(const double2* __restrict__ Bc, const double2* __restrict__ y, const int* __restrict__ kc,
                        int k, int s, int m, double2* __restrict__ T) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= k * s) return;
  const int a = p / s, c = p - a * s;
  double2 t = make_double2(0.0, 0.0);
  for (int j = 0; j < kc[c]; ++j) {
    const double2 b = Bc[((int64_t)j * k + a) * s + c], v = y[c * m + j];
    t.x += b.x * v.x - b.y * v.y;
    t.y += b.x * v.y + b.y * v.x;
  }
  T[p] = t;
}

__global__ void k_rbuild(const double2* __restrict__ Zk, int64_t vstride, int s, int col,
                         const double2* __restrict__ P, int m, int knew, double2* __restrict__ U, int k, int q0,
                         int64_t n) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= n * knew) return;
  const int64_t r = g / knew;
  const int q = (int)(g - r * knew);
  double2 u = make_double2(0.0, 0.0);
  for (int j = 0; j < m; ++j) {
    const double2 z = Zk[(int64_t)j * vstride + r * s + col], p = P[j + q * m];
    u.x += z.x * p.x - z.y * p.y;
    u.y += z.x * p.y + z.y * p.x;
  }
  U[r * k + q0 + q] = u;
}

// W[r][:] <- W[r][:] R^{-1} (x R = w; R upper triangular k x k, row-major)
__global__ void k_rtrsm(double2* W, int64_t n, int k, const double2* __restrict__ R) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= n) return;
  double2 x[16];
  for (int b = 0; b < k; ++b) {
    double2 v = W[r * k + b];
    for (int a = 0; a < b; ++a) {
      const double2 ra = R[a * k + b];
      v.x -= x[a].x * ra.x - x[a].y * ra.y;
      v.y -= x[a].x * ra.y + x[a].y * ra.x;
    }
    const double2 d = R[b * k + b];
    const double dd = d.x * d.x + d.y * d.y;
    x[b] = make_double2((v.x * d.x + v.y * d.y) / dd, (v.y * d.x - v.x * d.y) / dd);
  }
  for (int b = 0; b < k; ++b) W[r * k + b] = x[b];
}

// dst[r][d0 + q] = src[r][s0 + q], q < count (row-major blocks of widths sk, dk)
__global__ void k_rcopy(const double2* __restrict__ src, int sk, int s0, double2* __restrict__ dst, int dk, int d0,
                        int count, int64_t n) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= n * count) return;
  const int64_t r = g / count;
  const int q = (int)(g - r * count);
  dst[r * dk + d0 + q] = src[r * sk + s0 + q];
}

void recycle_copy(const double2* src, int sk, int s0, double2* dst, int dk, int d0, int count, int64_t n,
                  cudaStream_t st) {
  if (n * count) { k_rcopy<<<grid_for(n * count, 256), 256, 0, st>>>(src, sk, s0, dst, dk, d0, count, n); count_launch(); }
}

void recycle_dot(const double2* Cb, int k, const double2* W, int s, int64_t n, double2* part, int nblk, double2* out,
                 cudaStream_t st) {
  const int64_t rpb = (n + nblk - 1) / nblk;
  { k_rdot<<<nblk, RD_THREADS, 0, st>>>(Cb, k, W, s, n, rpb, part); count_launch(); }
  { k_rreduce<<<grid_for((int64_t)k * s, 256), 256, 0, st>>>(part, nblk, k * s, out); count_launch(); }
}
void recycle_axpy(const double2* Cb, int k, const double2* Y, double2* W, int s, int64_t n, double alpha,
                  cudaStream_t st) {
  if (n * s) { k_raxpy<<<grid_for(n * s, 256), 256, 0, st>>>(Cb, k, Y, W, s, n, alpha); count_launch(); }
}
void recycle_corr(const double2* Bc, const double2* y, const int* kc, int k, int s, int m, double2* T,
                  cudaStream_t st) {
  { k_rcorr<<<grid_for((int64_t)k * s, 128), 128, 0, st>>>(Bc, y, kc, k, s, m, T); count_launch(); }
}
void recycle_build(const double2* Zk, int64_t vstride, int s, int col, const double2* P, int m, int knew,
                   double2* U, int k, int q0, int64_t n, cudaStream_t st) {
  if (n * knew) { k_rbuild<<<grid_for(n * knew, 256), 256, 0, st>>>(Zk, vstride, s, col, P, m, knew, U, k, q0, n); count_launch(); }
}
void recycle_trsm(double2* W, int64_t n, int k, const double2* R, cudaStream_t st) {
  if (n) { k_rtrsm<<<grid_for(n, 128), 128, 0, st>>>(W, n, k, R); count_launch(); }
}

}  // namespace hz
