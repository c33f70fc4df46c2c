// Batched multifrontal factorisation and partitioned-inverse solves of the
// local matrices A_i (the paper's direct local solver inside Eq. oras).
//
// Factorisation: every front F_t (order f = k + m, k pivots) is assembled
// from the entries of A_i and its children's Schur complements (extend-add),
// then partially factored as F_t = L D L^T on its k pivots (complex
// symmetric, no pivoting, static perturbation of tiny pivots); the trailing
// m x m block becomes the Schur complement passed to the parent. All fronts
// of one tree height, over all subdomains, are processed by one launch.
//
// Partitioned inverse: the first k columns of the inverse of the unit lower
// trapezoid [[L11, 0], [L21, I]] are stored, X_t = [L11^{-1}; -L21 L11^{-1}]
// (f x k, column-major), with 1/D. The local solve then needs no triangular
// recurrence inside a front:
//   forward  (leaves to root): t = X_t b_P;  y_P = t[0:k] / D;
//                              parent update  w = c_U + t[k:f]
//   backward (root to leaves): x_P = X_t^T [y_P; x_U]
// so that both sweeps are streaming matrix products (forward: one thread per
// factor row; backward: one warp per pivot column) spread over all SMs, in
// FP64 or (mixed form) in FP32.
#include <cuda_runtime.h>

#include <algorithm>

#include "kernels.cuh"

namespace hz {

template <typename R>
struct C2;
template <>
struct C2<double> {
  using T = double2;
};
template <>
struct C2<float> {
  using T = float2;
};

__device__ __forceinline__ double2 mk2(double a, double b) { return make_double2(a, b); }
__device__ __forceinline__ float2 mk2(float a, float b) { return make_float2(a, b); }

template <typename V>
__device__ __forceinline__ V c_fma(V a, V b, V c) {  // a*b + c
  return mk2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
template <typename V>
__device__ __forceinline__ V c_mul(V a, V b) {
  return mk2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename V>
__device__ __forceinline__ V c_add(V a, V b) {
  return mk2(a.x + b.x, a.y + b.y);
}
__device__ __forceinline__ double2 dd(double2 a) { return a; }
__device__ __forceinline__ double2 dd(float2 a) { return make_double2(a.x, a.y); }
template <typename V>
__device__ __forceinline__ V from_d(double2 a);
template <>
__device__ __forceinline__ double2 from_d<double2>(double2 a) {
  return a;
}
template <>
__device__ __forceinline__ float2 from_d<float2>(double2 a) {
  return make_float2((float)a.x, (float)a.y);
}

__device__ __forceinline__ double2 zcdiv(double2 a, double2 b) {
  double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

// ---------------------------------------------------------------------------
// Assembly (extend-add), partial LDL^T, partitioned inverse
// ---------------------------------------------------------------------------
__global__ void k_mf_assemble(const int* __restrict__ list, const int* __restrict__ kk, const int* __restrict__ ff,
                              const int64_t* __restrict__ Foff, const int64_t* __restrict__ rowoff,
                              const int* __restrict__ cmap, const int* __restrict__ child_ptr,
                              const int* __restrict__ child_idx, const int64_t* __restrict__ amap_ptr,
                              const int* __restrict__ amap_pos, const int64_t* __restrict__ amap_val,
                              const double2* __restrict__ Aval, double2* __restrict__ F) {
  const int t = list[blockIdx.x];
  const int f = ff[t];
  double2* Ft = F + Foff[t];
  const int64_t ff2 = (int64_t)f * f;
  for (int64_t i = threadIdx.x; i < ff2; i += blockDim.x) Ft[i] = make_double2(0.0, 0.0);
  __syncthreads();
  for (int64_t p = amap_ptr[t] + threadIdx.x; p < amap_ptr[t + 1]; p += blockDim.x) {
    double2 a = Aval[amap_val[p]];
    double2 v = Ft[amap_pos[p]];
    Ft[amap_pos[p]] = make_double2(v.x + a.x, v.y + a.y);
  }
  __syncthreads();
  for (int q = child_ptr[t]; q < child_ptr[t + 1]; ++q) {
    const int ch = child_idx[q];
    const int kc = kk[ch], fc = ff[ch], mc = fc - kc;
    const double2* Fc = F + Foff[ch];
    const int* cm = cmap + rowoff[ch] + kc;
    const int64_t mm = (int64_t)mc * mc;
    for (int64_t i = threadIdx.x; i < mm; i += blockDim.x) {
      int a = (int)(i % mc), b = (int)(i / mc);
      if (a < b) continue;
      int64_t dst = cm[a] + (int64_t)cm[b] * f;
      double2 s = Fc[(kc + a) + (int64_t)(kc + b) * fc];
      double2 v = Ft[dst];
      Ft[dst] = make_double2(v.x + s.x, v.y + s.y);
    }
    __syncthreads();
  }
}

__global__ void k_mf_factor(const int* __restrict__ list, const int* __restrict__ kk, const int* __restrict__ ff,
                            const int64_t* __restrict__ Foff, double2* __restrict__ F, double tau_abs,
                            int* perturbed) {
  extern __shared__ double2 col[];
  __shared__ double2 dinv_s;
  const int t = list[blockIdx.x];
  const int f = ff[t], k = kk[t];
  double2* Ft = F + Foff[t];
  for (int j = 0; j < k; ++j) {
    if (threadIdx.x == 0) {
      double2 d = Ft[j + (int64_t)j * f];
      double ad = sqrt(d.x * d.x + d.y * d.y);
      if (ad < tau_abs) {
        d = ad > 0.0 ? make_double2(d.x / ad * tau_abs, d.y / ad * tau_abs) : make_double2(tau_abs, 0.0);
        Ft[j + (int64_t)j * f] = d;
        atomicAdd(perturbed, 1);
      }
      dinv_s = zcdiv(make_double2(1.0, 0.0), d);
    }
    for (int r = j + 1 + threadIdx.x; r < f; r += blockDim.x) col[r] = Ft[r + (int64_t)j * f];
    __syncthreads();
    const double2 dinv = dinv_s;
    for (int r = j + 1 + threadIdx.x; r < f; r += blockDim.x) Ft[r + (int64_t)j * f] = c_mul(col[r], dinv);
    const int nn = f - j - 1;
    const int64_t nn2 = (int64_t)nn * nn;
    for (int64_t i = threadIdx.x; i < nn2; i += blockDim.x) {
      int r = j + 1 + (int)(i % nn), c = j + 1 + (int)(i / nn);
      if (r < c) continue;
      int64_t o = r + (int64_t)c * f;
      double2 u = c_mul(col[r], c_mul(col[c], dinv));
      double2 v = Ft[o];
      Ft[o] = make_double2(v.x - u.x, v.y - u.y);
    }
    __syncthreads();
  }
}

// In place on the first k columns: L -> X = first k columns of
// [[L11,0],[L21,I]]^{-1}; stores 1/D and copies X into the compact factor
// array (FP64 or FP32).
template <typename V>
__global__ void k_mf_inverse(const int* __restrict__ list, const int* __restrict__ kk, const int* __restrict__ ff,
                             const int64_t* __restrict__ Foff, const int64_t* __restrict__ Moff,
                             const int64_t* __restrict__ Doff, double2* __restrict__ F, V* __restrict__ M,
                             V* __restrict__ Dinv) {
  extern __shared__ double2 col[];
  const int t = list[blockIdx.x];
  const int f = ff[t], k = kk[t];
  double2* Ft = F + Foff[t];
  for (int j = threadIdx.x; j < k; j += blockDim.x)
    Dinv[Doff[t] + j] = from_d<V>(zcdiv(make_double2(1.0, 0.0), Ft[j + (int64_t)j * f]));
  __syncthreads();
  for (int l = 0; l < k; ++l) {
    for (int r = l + 1 + threadIdx.x; r < f; r += blockDim.x) col[r] = Ft[r + (int64_t)l * f];
    __syncthreads();
    // X[r][c] -= L[r][l] X[l][c] for c < l, r > l;  X[r][l] = -L[r][l]
    const int nr = f - l - 1;
    const int64_t work = (int64_t)nr * (l + 1);
    for (int64_t i = threadIdx.x; i < work; i += blockDim.x) {
      int r = l + 1 + (int)(i % nr), c = (int)(i / nr);
      int64_t o = r + (int64_t)c * f;
      if (c == l) {
        Ft[o] = make_double2(-col[r].x, -col[r].y);
      } else {
        double2 x = Ft[l + (int64_t)c * f];
        double2 u = c_mul(col[r], x);
        double2 v = Ft[o];
        Ft[o] = make_double2(v.x - u.x, v.y - u.y);
      }
    }
    __syncthreads();
  }
  V* Mt = M + Moff[t];
  const int64_t fk = (int64_t)f * k;
  for (int64_t i = threadIdx.x; i < fk; i += blockDim.x) {
    int r = (int)(i % f), c = (int)(i / f);
    double2 v = r == c ? make_double2(1.0, 0.0) : (r < c ? make_double2(0.0, 0.0) : Ft[i]);
    Mt[i] = from_d<V>(v);
  }
}

void mf_factor(DevMF& mf, double tau_abs, cudaStream_t st) {
  size_t shm = (size_t)std::max(mf.max_f, 1) * sizeof(double2);
  cudaFuncSetAttribute(k_mf_factor, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
  cudaFuncSetAttribute(k_mf_inverse<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
  cudaFuncSetAttribute(k_mf_inverse<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
  for (int l = 0; l < mf.nlevels; ++l) {
    int b = mf.level_ptr_h[l], e = mf.level_ptr_h[l + 1];
    if (e == b) continue;
    k_mf_assemble<<<e - b, 256, 0, st>>>(mf.level_list + b, mf.k, mf.f, mf.Foff, mf.rowoff, mf.cmap, mf.child_ptr,
                                         mf.child_idx, mf.amap_ptr, mf.amap_pos, mf.amap_val, mf.Aval, mf.F);
    k_mf_factor<<<e - b, 256, shm, st>>>(mf.level_list + b, mf.k, mf.f, mf.Foff, mf.F, tau_abs, mf.perturbed);
  }
  // the inverses only touch the pivot columns: run them after every Schur
  // complement has been consumed by its parent
  for (int l = 0; l < mf.nlevels; ++l) {
    int b = mf.level_ptr_h[l], e = mf.level_ptr_h[l + 1];
    if (e == b) continue;
    if (mf.fp32)
      k_mf_inverse<float2><<<e - b, 256, shm, st>>>(mf.level_list + b, mf.k, mf.f, mf.Foff, mf.Moff, mf.Doff, mf.F,
                                                    (float2*)mf.M, (float2*)mf.Dinv);
    else
      k_mf_inverse<double2><<<e - b, 256, shm, st>>>(mf.level_list + b, mf.k, mf.f, mf.Foff, mf.Moff, mf.Doff,
                                                     mf.F, (double2*)mf.M, (double2*)mf.Dinv);
  }
}

// ---------------------------------------------------------------------------
// Solve sweeps
// ---------------------------------------------------------------------------
constexpr int FWD_ROWS = 128;  // rows per forward tile: one thread per row
constexpr int BWD_COLS = 8;    // pivots per backward tile: one warp per pivot

// front vector: Win[0:k] = Xsub[pivots], Win[k:f] = 0, plus the children's
// update vectors (Wout[k_c:f_c] of each child) added at their parent rows
template <typename V>
__global__ void k_mf_fvec(const int* __restrict__ list, const int* __restrict__ kk, const int* __restrict__ ff,
                          const int64_t* __restrict__ rowoff, const int* __restrict__ rows,
                          const int* __restrict__ cmap, const int* __restrict__ child_ptr,
                          const int* __restrict__ child_idx, const V* __restrict__ Xsub, V* __restrict__ Win,
                          const V* __restrict__ Wout, int s) {
  const int t = list[blockIdx.x];
  const int f = ff[t], k = kk[t];
  const int* rt = rows + rowoff[t];
  V* fv = Win + rowoff[t] * s;
  for (int i = threadIdx.x; i < f * s; i += blockDim.x) {
    int r = i / s, c = i - r * s;
    fv[i] = r < k ? Xsub[(int64_t)rt[r] * s + c] : mk2((decltype(V::x))0, (decltype(V::x))0);
  }
  __syncthreads();
  for (int q = child_ptr[t]; q < child_ptr[t + 1]; ++q) {
    const int ch = child_idx[q];
    const int kc = kk[ch], mc = ff[ch] - kc;
    const V* wc = Wout + (rowoff[ch] + kc) * s;
    const int* cm = cmap + rowoff[ch] + kc;
    for (int i = threadIdx.x; i < mc * s; i += blockDim.x) {
      int a = i / s, c = i - a * s;
      fv[cm[a] * s + c] = c_add(fv[cm[a] * s + c], wc[i]);
    }
    __syncthreads();
  }
}

// Forward tile: rows [r0, r0 + FWD_ROWS) of t = X_t b_P. One thread per row
// streams its row of X_t (consecutive threads read consecutive addresses of
// the column-major factor) against chunks of b_P staged in shared memory;
// the s right-hand sides are register accumulators, so every factor entry
// is read from HBM once per sweep.
template <typename V, int S>
__global__ void __launch_bounds__(FWD_ROWS) k_mf_fwd(const int2* __restrict__ tiles, const int* __restrict__ kk,
                                                     const int* __restrict__ ff, const int64_t* __restrict__ rowoff,
                                                     const int64_t* __restrict__ Moff, const int64_t* __restrict__ Doff,
                                                     const V* __restrict__ M, const V* __restrict__ Dinv,
                                                     const V* __restrict__ Win, V* __restrict__ Wout, int s) {
  constexpr int KC = (S >= 32) ? 32 : 64;
  __shared__ V bs[KC][S];
  const int2 tile = tiles[blockIdx.x];
  const int t = tile.x, r0 = tile.y;
  const int f = ff[t], k = kk[t];
  const int r = r0 + threadIdx.x;
  const bool active = r < f;
  const V* Mr = M + Moff[t] + r;
  const int64_t ro = rowoff[t];
  const V* bin = Win + ro * s;
  const int kend = (r0 < k) ? min(k, r0 + FWD_ROWS) : k;
  V acc[S];
#pragma unroll
  for (int c = 0; c < S; ++c) acc[c] = mk2((decltype(V::x))0, (decltype(V::x))0);
  for (int k0 = 0; k0 < kend; k0 += KC) {
    const int lmax = min(KC, kend - k0);
    for (int i = threadIdx.x; i < KC * S; i += FWD_ROWS) {
      int l = i / S, c = i % S;
      bs[l][c] = (l < lmax && c < s) ? bin[(k0 + l) * s + c] : mk2((decltype(V::x))0, (decltype(V::x))0);
    }
    __syncthreads();
    if (active) {
#pragma unroll 4
      for (int l = 0; l < lmax; ++l) {
        const V m = Mr[(int64_t)(k0 + l) * f];
#pragma unroll
        for (int c = 0; c < S; ++c) acc[c] = c_fma(m, bs[l][c], acc[c]);
      }
    }
    __syncthreads();
  }
  if (!active) return;
  V* out = Wout + (ro + r) * s;
  if (r < k) {
    const V di = Dinv[Doff[t] + r];
#pragma unroll
    for (int c = 0; c < S; ++c)
      if (c < s) out[c] = c_mul(acc[c], di);
  } else {
    const V* in = bin + (int64_t)r * s;
#pragma unroll
    for (int c = 0; c < S; ++c)
      if (c < s) out[c] = c_add(in[c], acc[c]);
  }
}

// backward: Win[k:f] = x_U gathered from the (final) ancestor pivots
template <typename V>
__global__ void k_mf_bvec(const int* __restrict__ list, const int* __restrict__ kk, const int* __restrict__ ff,
                          const int64_t* __restrict__ rowoff, const int* __restrict__ rows,
                          const V* __restrict__ Xsub, V* __restrict__ Win, int s) {
  const int t = list[blockIdx.x];
  const int f = ff[t], k = kk[t];
  const int* rt = rows + rowoff[t];
  V* fv = Win + rowoff[t] * s;
  for (int i = k * s + threadIdx.x; i < f * s; i += blockDim.x) {
    int r = i / s, c = i - r * s;
    fv[i] = Xsub[(int64_t)rt[r] * s + c];
  }
}

// Backward tile: pivots [j0, j0 + BWD_COLS) of x_P = X_t^T [y_P; x_U]. One
// warp per pivot column j: the lanes stream column j of X_t (contiguous)
// against chunks of the front vector staged in shared memory, then reduce.
template <typename V, int S>
__global__ void __launch_bounds__(32 * BWD_COLS) k_mf_bwd(const int2* __restrict__ tiles, const int* __restrict__ kk,
                                                          const int* __restrict__ ff,
                                                          const int64_t* __restrict__ rowoff,
                                                          const int64_t* __restrict__ Moff, const int* __restrict__ rows,
                                                          const V* __restrict__ M, const V* __restrict__ Win,
                                                          const V* __restrict__ Wout, V* __restrict__ Xsub, int s) {
  constexpr int RC = (S >= 32) ? 32 : 64;
  __shared__ V vs[RC][S + 1];
  const int2 tile = tiles[blockIdx.x];
  const int t = tile.x, j0 = tile.y;
  const int f = ff[t], k = kk[t];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int j = j0 + w;
  const int64_t ro = rowoff[t];
  const V* Mj = M + Moff[t] + (int64_t)j * f;
  V acc[S];
#pragma unroll
  for (int c = 0; c < S; ++c) acc[c] = mk2((decltype(V::x))0, (decltype(V::x))0);
  for (int r0 = j0; r0 < f; r0 += RC) {
    const int lmax = min(RC, f - r0);
    for (int i = threadIdx.x; i < RC * S; i += 32 * BWD_COLS) {
      int l = i / S, c = i % S;
      V v = mk2((decltype(V::x))0, (decltype(V::x))0);
      if (l < lmax && c < s) {
        const int gr = r0 + l;
        v = gr < k ? Wout[(ro + gr) * s + c] : Win[(ro + gr) * s + c];
      }
      vs[l][c] = v;
    }
    __syncthreads();
    if (j < k) {
      for (int l = lane; l < lmax; l += 32) {
        const int gr = r0 + l;
        if (gr < j) continue;  // X_t is zero above the diagonal of its pivot block
        const V m = Mj[gr];
#pragma unroll
        for (int c = 0; c < S; ++c) acc[c] = c_fma(m, vs[l][c], acc[c]);
      }
    }
    __syncthreads();
  }
  if (j >= k) return;
#pragma unroll
  for (int c = 0; c < S; ++c)
    for (int o = 16; o > 0; o >>= 1) {
      acc[c].x += __shfl_xor_sync(0xffffffffu, acc[c].x, o);
      acc[c].y += __shfl_xor_sync(0xffffffffu, acc[c].y, o);
    }
  V* xo = Xsub + (int64_t)rows[ro + j] * s;
#pragma unroll
  for (int c = 0; c < S; ++c)
    if (c < s && c % 32 == lane) xo[c] = acc[c];
}

template <typename V, int S>
static void solve_impl(DevMF& mf, V* Xsub, int s, cudaStream_t st) {
  V* Win = (V*)mf.Win;
  V* Wout = (V*)mf.Wout;
  const V* M = (const V*)mf.M;
  const V* Dv = (const V*)mf.Dinv;
  for (int l = 0; l < mf.nlevels; ++l) {
    int b = mf.level_ptr_h[l], e = mf.level_ptr_h[l + 1];
    if (e == b) continue;
    k_mf_fvec<V><<<e - b, 256, 0, st>>>(mf.level_list + b, mf.k, mf.f, mf.rowoff, mf.rows, mf.cmap, mf.child_ptr,
                                        mf.child_idx, Xsub, Win, Wout, s);
    int tb = mf.ftile_ptr_h[l], te = mf.ftile_ptr_h[l + 1];
    if (te > tb)
      k_mf_fwd<V, S><<<te - tb, FWD_ROWS, 0, st>>>(mf.ftiles + tb, mf.k, mf.f, mf.rowoff, mf.Moff, mf.Doff, M, Dv,
                                                   Win, Wout, s);
  }
  for (int l = mf.nlevels - 1; l >= 0; --l) {
    int b = mf.level_ptr_h[l], e = mf.level_ptr_h[l + 1];
    if (e == b) continue;
    k_mf_bvec<V><<<e - b, 256, 0, st>>>(mf.level_list + b, mf.k, mf.f, mf.rowoff, mf.rows, Xsub, Win, s);
    int tb = mf.btile_ptr_h[l], te = mf.btile_ptr_h[l + 1];
    if (te > tb)
      k_mf_bwd<V, S><<<te - tb, 32 * BWD_COLS, 0, st>>>(mf.btiles + tb, mf.k, mf.f, mf.rowoff, mf.Moff, mf.rows, M,
                                                        Win, Wout, Xsub, s);
  }
}

template <typename V>
static void solve_dispatch(DevMF& mf, V* Xsub, int s, cudaStream_t st) {
  if (s <= 1)
    solve_impl<V, 1>(mf, Xsub, s, st);
  else if (s <= 2)
    solve_impl<V, 2>(mf, Xsub, s, st);
  else if (s <= 4)
    solve_impl<V, 4>(mf, Xsub, s, st);
  else if (s <= 8)
    solve_impl<V, 8>(mf, Xsub, s, st);
  else if (s <= 16)
    solve_impl<V, 16>(mf, Xsub, s, st);
  else if (s <= 32)
    solve_impl<V, 32>(mf, Xsub, s, st);
  else
    solve_impl<V, 64>(mf, Xsub, s, st);
}

void mf_solve(DevMF& mf, void* Xsub, int s, cudaStream_t st) {
  if (mf.fp32)
    solve_dispatch<float2>(mf, (float2*)Xsub, s, st);
  else
    solve_dispatch<double2>(mf, (double2*)Xsub, s, st);
}

// ---------------------------------------------------------------------------
// Restriction / prolongation with the sub-vector in FP32 (mixed form)
// ---------------------------------------------------------------------------
__global__ void k_gather_rows_f32(const int* __restrict__ idx, int64_t nrows, const double2* __restrict__ X,
                                  float2* __restrict__ Y, int s) {
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t r = g / s;
  if (r >= nrows) return;
  int c = (int)(g - r * s);
  double2 v = X[(int64_t)idx[r] * s + c];
  Y[g] = make_float2((float)v.x, (float)v.y);
}

__global__ void k_scatter_owned_f32(const int* __restrict__ own, int64_t n, const float2* __restrict__ Xsub,
                                    const double2* __restrict__ Q, double2* __restrict__ Z, int s) {
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t r = g / s;
  if (r >= n) return;
  int c = (int)(g - r * s);
  float2 v = Xsub[(int64_t)own[r] * s + c];
  double2 o = make_double2(v.x, v.y);
  if (Q) {
    double2 q = Q[g];
    o.x += q.x;
    o.y += q.y;
  }
  Z[g] = o;
}

void gather_rows_f32(const int* idx, int64_t nrows, const double2* X, float2* Y, int s, cudaStream_t st) {
  if (nrows * s == 0) return;
  k_gather_rows_f32<<<(unsigned)((nrows * s + 255) / 256), 256, 0, st>>>(idx, nrows, X, Y, s);
}

void scatter_owned_f32(const int* own, int64_t n, const float2* Xsub, const double2* Q, double2* Z, int s,
                       cudaStream_t st) {
  if (n * s == 0) return;
  k_scatter_owned_f32<<<(unsigned)((n * s + 255) / 256), 256, 0, st>>>(own, n, Xsub, Q, Z, s);
}

}  // namespace hz
