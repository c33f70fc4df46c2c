// Batched multifrontal numeric factorisation of the local matrices A_i (the
// paper's direct local solver inside Eq. oras, Sec. "Domain decomposition
// preconditioner"), level by level over the elimination trees of all
// subdomains, and the partitioned inverse that the solve sweeps apply.
//
// Every front F_t (order f = k + m, k pivots) is assembled from the entries
// of A_i and its children's Schur complements (extend-add), then partially
// factored as F_t = L D L^T on its k pivots (complex symmetric, no pivoting,
// static perturbation of tiny pivots); the trailing m x m block becomes the
// Schur complement passed to the parent. The factorisation runs in the
// precision of the front workspace: FP64, or complex FP32 for the fine
// fronts of the mixed form.
//
// Fronts of order f <= FA_SMALL are factored by one CTA each, pivot by
// pivot. Larger fronts go by panels of FA_NB pivots: one CTA per front
// factors the panel's diagonal block in shared memory and solves the rows
// below it (l_r = f_r L_panel^{-T} D^{-1}, one thread per row, the row in
// registers); then the trailing lower triangle takes the update
// F22 -= L21 D L21^T as 64 x 64 tiles spread over all SMs.
//
// Partitioned inverse: the first k columns of the inverse of the unit lower
// trapezoid [[L11, 0], [L21, I]], X_t = [L11^{-1}; -L21 L11^{-1}] (f x k,
// column-major), and 1/D are written to the factor arrays (FP64 or FP32),
// with X_t^T beside X_t for the backward sweep.
#include <cuda_runtime.h>

#include <algorithm>

#include "kernels.cuh"

namespace hz {

namespace {

template <typename T>
struct Cx;
template <>
struct Cx<double2> {
  using R = double;
};
template <>
struct Cx<float2> {
  using R = float;
};

__device__ __forceinline__ double2 mkc(double a, double b, double2) { return make_double2(a, b); }
__device__ __forceinline__ float2 mkc(float a, float b, float2) { return make_float2(a, b); }
template <typename T>
__device__ __forceinline__ T czero() {
  return mkc((typename Cx<T>::R)0, (typename Cx<T>::R)0, T());
}
template <typename T>
__device__ __forceinline__ T cmul(T a, T b) {
  return mkc(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x, T());
}
template <typename T>
__device__ __forceinline__ T csub(T a, T b) {
  return mkc(a.x - b.x, a.y - b.y, T());
}
template <typename T>
__device__ __forceinline__ T cadd(T a, T b) {
  return mkc(a.x + b.x, a.y + b.y, T());
}
template <typename T>
__device__ __forceinline__ T cfms(T a, T b, T c) {  // c - a b
  return mkc(fma(-a.x, b.x, fma(a.y, b.y, c.x)), fma(-a.x, b.y, fma(-a.y, b.x, c.y)), T());
}
template <typename T>
__device__ __forceinline__ T cinv(T b) {
  const auto d = b.x * b.x + b.y * b.y;
  return mkc(b.x / d, -b.y / d, T());
}
template <typename T>
__device__ __forceinline__ double2 to_d(T a) {
  return make_double2((double)a.x, (double)a.y);
}
template <typename V>
__device__ __forceinline__ V from_d2(double2 a);
template <>
__device__ __forceinline__ double2 from_d2<double2>(double2 a) {
  return a;
}
template <>
__device__ __forceinline__ float2 from_d2<float2>(double2 a) {
  return make_float2((float)a.x, (float)a.y);
}

// static perturbation of a tiny pivot: |d| < tau -> d tau / |d| (tau if d = 0)
template <typename T>
__device__ __forceinline__ T perturb(T d, double tau_abs, int* perturbed) {
  const double ad = sqrt((double)d.x * d.x + (double)d.y * d.y);
  if (ad < tau_abs) {
    atomicAdd(perturbed, 1);
    return ad > 0.0 ? mkc((typename Cx<T>::R)(d.x / ad * tau_abs), (typename Cx<T>::R)(d.y / ad * tau_abs), T())
                    : mkc((typename Cx<T>::R)tau_abs, (typename Cx<T>::R)0, T());
  }
  return d;
}

inline unsigned gridn(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

constexpr int FA_NB = 32;     // pivots per panel
constexpr int FA_TILE = 64;   // trailing-update tile
constexpr int FA_THREADS = 256;

// ---------------------------------------------------------------------------
// Assembly (extend-add)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_fa_assemble(const int* __restrict__ list, const int* __restrict__ kk, const int* __restrict__ ff,
                              const int64_t* __restrict__ Foff, const int64_t* __restrict__ rowoff,
                              const int* __restrict__ cmap, const int* __restrict__ child_ptr,
                              const int* __restrict__ child_idx, const int64_t* __restrict__ amap_ptr,
                              const int* __restrict__ amap_pos, const int64_t* __restrict__ amap_val,
                              const double2* __restrict__ Aval, T* __restrict__ F) {
  const int t = list[blockIdx.x];
  const int f = ff[t];
  T* Ft = F + Foff[t];
  const int64_t ff2 = (int64_t)f * f;
  for (int64_t i = threadIdx.x; i < ff2; i += blockDim.x) Ft[i] = czero<T>();
  __syncthreads();
  for (int64_t p = amap_ptr[t] + threadIdx.x; p < amap_ptr[t + 1]; p += blockDim.x) {
    const double2 a = Aval[amap_val[p]];
    Ft[amap_pos[p]] = cadd(Ft[amap_pos[p]], from_d2<T>(a));
  }
  __syncthreads();
  for (int q = child_ptr[t]; q < child_ptr[t + 1]; ++q) {
    const int ch = child_idx[q];
    const int kc = kk[ch], fc = ff[ch], mc = fc - kc;
    const T* Fc = F + Foff[ch];
    const int* cm = cmap + rowoff[ch] + kc;
    const int64_t mm = (int64_t)mc * mc;
    for (int64_t i = threadIdx.x; i < mm; i += blockDim.x) {
      const int a = (int)(i % mc), b = (int)(i / mc);
      if (a < b) continue;
      const int64_t dst = cm[a] + (int64_t)cm[b] * f;
      Ft[dst] = cadd(Ft[dst], Fc[(kc + a) + (int64_t)(kc + b) * fc]);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Small fronts: pivot by pivot, one CTA per front
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_fa_factor(const int* __restrict__ list, const int* __restrict__ kk, const int* __restrict__ ff,
                            const int64_t* __restrict__ Foff, T* __restrict__ F, double tau_abs, int* perturbed) {
  extern __shared__ __align__(16) unsigned char fa_smem[];
  T* col = reinterpret_cast<T*>(fa_smem);
  __shared__ T dinv_s;
  const int t = list[blockIdx.x];
  const int f = ff[t], k = kk[t];
  T* Ft = F + Foff[t];
  for (int j = 0; j < k; ++j) {
    if (threadIdx.x == 0) {
      const T d = perturb(Ft[j + (int64_t)j * f], tau_abs, perturbed);
      Ft[j + (int64_t)j * f] = d;
      dinv_s = cinv(d);
    }
    for (int r = j + 1 + threadIdx.x; r < f; r += blockDim.x) col[r] = Ft[r + (int64_t)j * f];
    __syncthreads();
    const T dinv = dinv_s;
    for (int r = j + 1 + threadIdx.x; r < f; r += blockDim.x) Ft[r + (int64_t)j * f] = cmul(col[r], dinv);
    const int nn = f - j - 1;
    const int64_t nn2 = (int64_t)nn * nn;
    for (int64_t i = threadIdx.x; i < nn2; i += blockDim.x) {
      const int r = j + 1 + (int)(i % nn), c = j + 1 + (int)(i / nn);
      if (r < c) continue;
      const int64_t o = r + (int64_t)c * f;
      Ft[o] = cfms(col[r], cmul(col[c], dinv), Ft[o]);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Large fronts: panel of pivots [p0, p0 + pb), one CTA per front
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(FA_THREADS) k_fa_panel(const int* __restrict__ list, const int* __restrict__ kk,
                                                         const int* __restrict__ ff, const int64_t* __restrict__ Foff,
                                                         T* __restrict__ F, int p0, double tau_abs, int* perturbed) {
  __shared__ T Dg[FA_NB][FA_NB + 1];  // diagonal block: L (strictly lower) and the working entries
  __shared__ T dd[FA_NB], dinv[FA_NB];
  const int t = list[blockIdx.x];
  const int f = ff[t], k = kk[t];
  if (p0 >= k) return;
  const int pb = min(FA_NB, k - p0);
  T* Ft = F + Foff[t];
  const int tid = threadIdx.x;
  for (int e = tid; e < pb * pb; e += FA_THREADS) {
    const int r = e % pb, c = e / pb;
    if (r >= c) Dg[r][c] = Ft[(p0 + r) + (int64_t)(p0 + c) * f];
  }
  __syncthreads();
  for (int j = 0; j < pb; ++j) {
    if (tid == 0) {
      const T d = perturb(Dg[j][j], tau_abs, perturbed);
      dd[j] = d;
      dinv[j] = cinv(d);
    }
    __syncthreads();
    for (int r = j + 1 + tid; r < pb; r += FA_THREADS) Dg[r][j] = cmul(Dg[r][j], dinv[j]);
    __syncthreads();
    const int nn = pb - j - 1;
    for (int e = tid; e < nn * nn; e += FA_THREADS) {
      const int r = j + 1 + e % nn, c = j + 1 + e / nn;
      if (r >= c) Dg[r][c] = cfms(Dg[r][j], cmul(dd[j], Dg[c][j]), Dg[r][c]);
    }
    __syncthreads();
  }
  for (int e = tid; e < pb * pb; e += FA_THREADS) {
    const int r = e % pb, c = e / pb;
    if (r > c) Ft[(p0 + r) + (int64_t)(p0 + c) * f] = Dg[r][c];
    if (r == c) Ft[(p0 + r) + (int64_t)(p0 + c) * f] = dd[r];
  }
  // rows below the panel: l_rj = (f_rj - sum_{c<j} l_rc d_c L_jc) / d_j
  for (int r = p0 + pb + tid; r < f; r += FA_THREADS) {
    T x[FA_NB];
#pragma unroll
    for (int j = 0; j < FA_NB; ++j)
      if (j < pb) x[j] = Ft[r + (int64_t)(p0 + j) * f];
#pragma unroll
    for (int j = 0; j < FA_NB; ++j) {
      if (j >= pb) break;
      T v = x[j];
#pragma unroll
      for (int c = 0; c < FA_NB; ++c) {
        if (c >= j) break;
        v = cfms(x[c], cmul(dd[c], Dg[j][c]), v);
      }
      x[j] = cmul(v, dinv[j]);
    }
#pragma unroll
    for (int j = 0; j < FA_NB; ++j)
      if (j < pb) Ft[r + (int64_t)(p0 + j) * f] = x[j];
  }
}

// Trailing update of the panel [p0, p0 + pb): F[r][c] -= sum_j l_rj d_j l_cj
// for q0 <= c <= r < f, q0 = p0 + pb, on the 64 x 64 tile (ti, tj) of the
// trailing block (tiles with ti >= tj). Each thread owns 4 x 4 entries.
template <typename T>
__global__ void __launch_bounds__(FA_THREADS) k_fa_schur(const int4* __restrict__ tiles, const int* __restrict__ kk,
                                                         const int* __restrict__ ff, const int64_t* __restrict__ Foff,
                                                         T* __restrict__ F, int p0) {
  extern __shared__ __align__(16) unsigned char fa_smem[];
  T(*As)[FA_TILE] = reinterpret_cast<T(*)[FA_TILE]>(fa_smem);                                // [NB][64] l_rj
  T(*Bs)[FA_TILE] = reinterpret_cast<T(*)[FA_TILE]>(fa_smem + sizeof(T) * FA_NB * FA_TILE);  // [NB][64] d_j l_cj
  const int4 tl = tiles[blockIdx.x];
  const int t = tl.x;
  const int f = ff[t], k = kk[t];
  const int pb = min(FA_NB, k - p0);
  const int q0 = p0 + pb;
  const int r0 = q0 + tl.y * FA_TILE, c0 = q0 + tl.z * FA_TILE;
  const T* Ft = F + Foff[t];
  T* Fw = F + Foff[t];
  const int tid = threadIdx.x;
  for (int e = tid; e < FA_NB * FA_TILE; e += FA_THREADS) {
    const int i = e % FA_TILE, j = e / FA_TILE;
    T a = czero<T>(), b = czero<T>();
    if (j < pb) {
      if (r0 + i < f) a = Ft[(r0 + i) + (int64_t)(p0 + j) * f];
      if (c0 + i < f) b = cmul(Ft[(p0 + j) + (int64_t)(p0 + j) * f], Ft[(c0 + i) + (int64_t)(p0 + j) * f]);
    }
    As[j][i] = a;
    Bs[j][i] = b;
  }
  __syncthreads();
  const int tx = tid % 16, ty = tid / 16;
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = czero<T>();
  for (int j = 0; j < pb; ++j) {
    T av[4], bv[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) av[a] = As[j][ty * 4 + a];
#pragma unroll
    for (int b = 0; b < 4; ++b) bv[b] = Bs[j][tx * 4 + b];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        acc[a][b].x = fma(av[a].x, bv[b].x, fma(-av[a].y, bv[b].y, acc[a][b].x));
        acc[a][b].y = fma(av[a].x, bv[b].y, fma(av[a].y, bv[b].x, acc[a][b].y));
      }
  }
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const int c = c0 + tx * 4 + b;
    if (c >= f) continue;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int r = r0 + ty * 4 + a;
      if (r >= f || r < c) continue;
      const int64_t o = r + (int64_t)c * f;
      Fw[o] = csub(Fw[o], acc[a][b]);
    }
  }
}

// ---------------------------------------------------------------------------
// Partitioned inverse, in place on the first k columns of the front:
// L -> X = first k columns of [[L11, 0], [L21, I]]^{-1}; 1/D and X (and X^T)
// to the factor arrays in the storage precision V.
// ---------------------------------------------------------------------------
template <typename T, typename V>
__global__ void k_fa_inverse(const int* __restrict__ list, const int* __restrict__ kk, const int* __restrict__ ff,
                             const int64_t* __restrict__ Foff, const int64_t* __restrict__ Moff,
                             const int64_t* __restrict__ Doff, T* __restrict__ F, V* __restrict__ M,
                             V* __restrict__ MT, V* __restrict__ Dinv) {
  extern __shared__ __align__(16) unsigned char fa_smem[];
  T* col = reinterpret_cast<T*>(fa_smem);
  const int t = list[blockIdx.x];
  const int f = ff[t], k = kk[t];
  T* Ft = F + Foff[t];
  for (int j = threadIdx.x; j < k; j += blockDim.x)
    Dinv[Doff[t] + j] = from_d2<V>(to_d(cinv(Ft[j + (int64_t)j * f])));
  __syncthreads();
  for (int l = 0; l < k; ++l) {
    for (int r = l + 1 + threadIdx.x; r < f; r += blockDim.x) col[r] = Ft[r + (int64_t)l * f];
    __syncthreads();
    // X[r][c] -= L[r][l] X[l][c] for c < l, r > l;  X[r][l] = -L[r][l]
    const int nr = f - l - 1;
    const int64_t work = (int64_t)nr * (l + 1);
    for (int64_t i = threadIdx.x; i < work; i += blockDim.x) {
      const int r = l + 1 + (int)(i % nr), c = (int)(i / nr);
      const int64_t o = r + (int64_t)c * f;
      if (c == l)
        Ft[o] = csub(czero<T>(), col[r]);
      else
        Ft[o] = cfms(col[r], Ft[l + (int64_t)c * f], Ft[o]);
    }
    __syncthreads();
  }
  V* Mt = M + Moff[t];
  V* MTt = MT + Moff[t];
  const int64_t fk = (int64_t)f * k;
  for (int64_t i = threadIdx.x; i < fk; i += blockDim.x) {
    const int r = (int)(i % f), c = (int)(i / f);
    const double2 v = r == c ? make_double2(1.0, 0.0) : (r < c ? make_double2(0.0, 0.0) : to_d(Ft[i]));
    Mt[i] = from_d2<V>(v);
    MTt[c + (int64_t)r * k] = from_d2<V>(v);
  }
}

// ---------------------------------------------------------------------------
// Large fronts: blocked partitioned inverse, in place. X = L~^{-1} E_k with
// L~ = [[L11, 0], [L21, I]] and E_k the first k columns of the identity,
// by row blocks B = [l0, l0 + nb) of the pivot region:
//   X[B, :] <- L~[B, B]^{-1} X[B, :]                  (k_fa_inv_diag)
//   X[r, :] <- X[r, :] - L~[r, B] X[B, :], r > B      (k_fa_inv_update)
// where X starts as E_k. X[r][c] (c < k) shares its storage with L[r][c]:
// the first step copies the panel L[r, B] of the rows below B to a scratch
// panel before the update overwrites it, and the identity entries (the
// diagonal, which keeps d, and the upper triangle) are never stored.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(FA_THREADS) k_fa_inv_diag(const int* __restrict__ list, const int* __restrict__ kk,
                                                            const int* __restrict__ ff,
                                                            const int64_t* __restrict__ Foff, T* __restrict__ F,
                                                            const int64_t* __restrict__ pan_off, T* __restrict__ pan,
                                                            int l0) {
  __shared__ T Lb[FA_NB][FA_NB + 1];
  const int t = list[blockIdx.x];
  const int f = ff[t], k = kk[t];
  if (l0 >= k) return;
  const int nb = min(FA_NB, k - l0);
  T* Ft = F + Foff[t];
  const int tid = threadIdx.x;
  for (int e = tid; e < nb * nb; e += FA_THREADS) {
    const int r = e % nb, c = e / nb;
    if (r > c) Lb[r][c] = Ft[(l0 + r) + (int64_t)(l0 + c) * f];
  }
  // scratch panel: L[r][l0 + j] of the rows below the block, [r - l0 - nb][j]
  T* P = pan + pan_off[blockIdx.x];
  const int below = f - l0 - nb;
  for (int64_t e = tid; e < (int64_t)below * nb; e += FA_THREADS) {
    const int i = (int)(e % below), j = (int)(e / below);
    P[(int64_t)i * FA_NB + j] = Ft[(l0 + nb + i) + (int64_t)(l0 + j) * f];
  }
  __syncthreads();
  // X[B, c] for c < l0 + nb: forward substitution with the unit lower block, one thread per column
  for (int c = tid; c < l0 + nb; c += FA_THREADS) {
    T x[FA_NB];
#pragma unroll
    for (int l = 0; l < FA_NB; ++l) {
      if (l >= nb) break;
      const int gl = l0 + l;
      T v = c < l0 ? Ft[gl + (int64_t)c * f] : (gl == c ? mkc((typename Cx<T>::R)1, (typename Cx<T>::R)0, T())
                                                          : czero<T>());
#pragma unroll
      for (int q = 0; q < FA_NB; ++q) {
        if (q >= l) break;
        v = cfms(Lb[l][q], x[q], v);
      }
      x[l] = v;
    }
#pragma unroll
    for (int l = 0; l < FA_NB; ++l) {
      if (l >= nb) break;
      if (l0 + l > c) Ft[(l0 + l) + (int64_t)c * f] = x[l];
    }
  }
}

// X[r][c] = base - sum_{l in B} L[r][l] X[l][c] on the 64 x 64 tile (ti, tj)
// of rows [l0 + nb, f) x columns [0, l0 + nb); base = X[r][c] for c < l0, 0
// for c in B. X[l][c] for l in B: the stored entry below the diagonal, 1 on
// it, 0 above.
template <typename T>
__global__ void __launch_bounds__(FA_THREADS) k_fa_inv_update(const int4* __restrict__ tiles,
                                                              const int* __restrict__ kk, const int* __restrict__ ff,
                                                              const int64_t* __restrict__ Foff, T* __restrict__ F,
                                                              const int64_t* __restrict__ pan_off,
                                                              const T* __restrict__ pan, int l0) {
  extern __shared__ __align__(16) unsigned char fa_smem[];
  T(*As)[FA_TILE] = reinterpret_cast<T(*)[FA_TILE]>(fa_smem);                                // [NB][64] L[r][l]
  T(*Bs)[FA_TILE] = reinterpret_cast<T(*)[FA_TILE]>(fa_smem + sizeof(T) * FA_NB * FA_TILE);  // [NB][64] X[l][c]
  const int4 tl = tiles[blockIdx.x];
  const int t = tl.x;
  const int f = ff[t], k = kk[t];
  const int nb = min(FA_NB, k - l0);
  const int q0 = l0 + nb;
  const int r0 = q0 + tl.y * FA_TILE, c0 = tl.z * FA_TILE;
  T* Ft = F + Foff[t];
  const T* P = pan + pan_off[tl.w];
  const int tid = threadIdx.x;
  for (int e = tid; e < FA_NB * FA_TILE; e += FA_THREADS) {
    const int i = e % FA_TILE, j = e / FA_TILE;
    T a = czero<T>(), b = czero<T>();
    if (j < nb) {
      if (r0 + i < f) a = P[(int64_t)(r0 + i - q0) * FA_NB + j];
      const int c = c0 + i, l = l0 + j;
      if (c < q0)
        b = l > c ? Ft[l + (int64_t)c * f]
                  : (l == c ? mkc((typename Cx<T>::R)1, (typename Cx<T>::R)0, T()) : czero<T>());
    }
    As[j][i] = a;
    Bs[j][i] = b;
  }
  __syncthreads();
  const int tx = tid % 16, ty = tid / 16;
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = czero<T>();
  for (int j = 0; j < nb; ++j) {
    T av[4], bv[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) av[a] = As[j][ty * 4 + a];
#pragma unroll
    for (int b = 0; b < 4; ++b) bv[b] = Bs[j][tx * 4 + b];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        acc[a][b].x = fma(av[a].x, bv[b].x, fma(-av[a].y, bv[b].y, acc[a][b].x));
        acc[a][b].y = fma(av[a].x, bv[b].y, fma(av[a].y, bv[b].x, acc[a][b].y));
      }
  }
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const int c = c0 + tx * 4 + b;
    if (c >= q0) continue;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int r = r0 + ty * 4 + a;
      if (r >= f) continue;
      const int64_t o = r + (int64_t)c * f;
      const T base = c < l0 ? Ft[o] : czero<T>();
      Ft[o] = csub(base, acc[a][b]);
    }
  }
}

// 1/D and X_t (and X_t^T) to the factor arrays, after the blocked inverse
template <typename T, typename V>
__global__ void k_fa_store(const int* __restrict__ list, const int* __restrict__ kk, const int* __restrict__ ff,
                           const int64_t* __restrict__ Foff, const int64_t* __restrict__ Moff,
                           const int64_t* __restrict__ Doff, const T* __restrict__ F, V* __restrict__ M,
                           V* __restrict__ MT, V* __restrict__ Dinv) {
  const int t = list[blockIdx.x];
  const int f = ff[t], k = kk[t];
  const T* Ft = F + Foff[t];
  for (int j = threadIdx.x; j < k; j += blockDim.x)
    Dinv[Doff[t] + j] = from_d2<V>(to_d(cinv(Ft[j + (int64_t)j * f])));
  V* Mt = M + Moff[t];
  V* MTt = MT + Moff[t];
  const int64_t fk = (int64_t)f * k;
  for (int64_t i = threadIdx.x; i < fk; i += blockDim.x) {
    const int r = (int)(i % f), c = (int)(i / f);
    const double2 v = r == c ? make_double2(1.0, 0.0) : (r < c ? make_double2(0.0, 0.0) : to_d(Ft[i]));
    Mt[i] = from_d2<V>(v);
    MTt[c + (int64_t)r * k] = from_d2<V>(v);
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
template <typename T, typename V>
static void factor_t(DevMF& mf, double tau_abs, cudaStream_t st) {
  T* F = reinterpret_cast<T*>(mf.F);
  cudaEvent_t ev[3];
  for (auto& e : ev) cudaEventCreate(&e);
  cudaEventRecord(ev[0], st);
  const size_t shm = (size_t)std::max(mf.max_f, 1) * sizeof(T);
  const size_t schur_shm = 2 * sizeof(T) * FA_NB * FA_TILE;
  cudaFuncSetAttribute(k_fa_factor<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
  cudaFuncSetAttribute(k_fa_inverse<T, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
  cudaFuncSetAttribute(k_fa_schur<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)schur_shm);
  for (int l = 0; l < mf.nlevels; ++l) {
    const int b = mf.level_ptr_h[l], e = mf.level_ptr_h[l + 1];
    if (e == b) continue;
    { k_fa_assemble<T><<<e - b, 256, 0, st>>>(mf.level_list + b, mf.k, mf.f, mf.Foff, mf.rowoff, mf.cmap,
                                              mf.child_ptr, mf.child_idx, mf.amap_ptr, mf.amap_pos, mf.amap_val,
                                              mf.Aval, F); count_launch(); }
    const int sb = mf.fa_small_ptr_h[l], se = mf.fa_small_ptr_h[l + 1];
    if (se > sb)
      { k_fa_factor<T><<<se - sb, 256, shm, st>>>(mf.fa_small + sb, mf.k, mf.f, mf.Foff, F, tau_abs, mf.perturbed); count_launch(); }
    const int bb = mf.fa_big_ptr_h[l], be = mf.fa_big_ptr_h[l + 1];
    if (be > bb) {
      for (int p = mf.fa_step_ptr_h[l]; p < mf.fa_step_ptr_h[l + 1]; ++p) {
        const int p0 = (p - mf.fa_step_ptr_h[l]) * FA_NB;
        { k_fa_panel<T><<<be - bb, FA_THREADS, 0, st>>>(mf.fa_big + bb, mf.k, mf.f, mf.Foff, F, p0, tau_abs,
                                                        mf.perturbed); count_launch(); }
        const int tb = mf.fa_tile_ptr_h[p], te = mf.fa_tile_ptr_h[p + 1];
        if (te > tb)
          { k_fa_schur<T><<<te - tb, FA_THREADS, schur_shm, st>>>(mf.fa_tiles + tb, mf.k, mf.f, mf.Foff, F, p0); count_launch(); }
      }
    }
  }
  cudaEventRecord(ev[1], st);
  // the inverses only touch the pivot columns: run them after every Schur
  // complement has been consumed by its parent; small fronts one CTA each,
  // large fronts by row blocks (the same steps as their panels)
  cudaFuncSetAttribute(k_fa_inv_update<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)schur_shm);
  T* pan = reinterpret_cast<T*>(mf.fa_pan);
  for (int l = 0; l < mf.nlevels; ++l) {
    const int sb = mf.fa_small_ptr_h[l], se = mf.fa_small_ptr_h[l + 1];
    if (se > sb)
      { k_fa_inverse<T, V><<<se - sb, 256, shm, st>>>(mf.fa_small + sb, mf.k, mf.f, mf.Foff, mf.Moff, mf.Doff, F,
                                                      (V*)mf.M, (V*)mf.MT, (V*)mf.Dinv); count_launch(); }
    const int bb = mf.fa_big_ptr_h[l], be = mf.fa_big_ptr_h[l + 1];
    if (be == bb) continue;
    for (int p = mf.fa_step_ptr_h[l]; p < mf.fa_step_ptr_h[l + 1]; ++p) {
      const int l0 = (p - mf.fa_step_ptr_h[l]) * FA_NB;
      { k_fa_inv_diag<T><<<be - bb, FA_THREADS, 0, st>>>(mf.fa_big + bb, mf.k, mf.f, mf.Foff, F, mf.fa_pan_off + bb,
                                                         pan, l0); count_launch(); }
      const int tb = mf.fi_tile_ptr_h[p], te = mf.fi_tile_ptr_h[p + 1];
      if (te > tb)
        { k_fa_inv_update<T><<<te - tb, FA_THREADS, schur_shm, st>>>(mf.fi_tiles + tb, mf.k, mf.f, mf.Foff, F,
                                                                     mf.fa_pan_off + bb, pan, l0); count_launch(); }
    }
    { k_fa_store<T, V><<<be - bb, 256, 0, st>>>(mf.fa_big + bb, mf.k, mf.f, mf.Foff, mf.Moff, mf.Doff, F, (V*)mf.M,
                                                (V*)mf.MT, (V*)mf.Dinv); count_launch(); }
  }
  cudaEventRecord(ev[2], st);
  cudaEventSynchronize(ev[2]);
  cudaEventElapsedTime(&mf.factor_ms, ev[0], ev[1]);
  cudaEventElapsedTime(&mf.inverse_ms, ev[1], ev[2]);
  for (auto& e : ev) cudaEventDestroy(e);
}

void mf_factor_fronts(DevMF& mf, double tau_abs, cudaStream_t st) {
  if (mf.fr32)
    factor_t<float2, float2>(mf, tau_abs, st);
  else if (mf.fp32)
    factor_t<double2, float2>(mf, tau_abs, st);
  else
    factor_t<double2, double2>(mf, tau_abs, st);
}

}  // namespace hz
