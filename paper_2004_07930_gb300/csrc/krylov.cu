// Flexible GMRES building blocks, one Krylov space per right-hand side
// (Sec. "Domain decomposition preconditioner": GMRES; K8 CGS2 Arnoldi, K10
// Givens least squares, K12 solution update).
//
// The basis vectors are complex blocks [n][s] in FP64 (outer solve) or FP32
// (the inner coarse solve of the mixed form). Dot products accumulate in the
// vector precision inside a CTA and are summed over CTAs in FP64 in a fixed
// order (deterministic); the Hessenberg matrix, the Givens rotations and the
// least-squares solve are FP64 in both cases.
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "df.cuh"
#include "kernels.cuh"

namespace hz {

namespace {

__device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
__device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
template <typename V>
__device__ __forceinline__ V zero() {
  return mk((decltype(V::x))0, (decltype(V::x))0);
}
template <typename V>
__device__ __forceinline__ V from2(double2 a) {
  return mk((decltype(V::x))a.x, (decltype(V::x))a.y);
}
template <typename V>
__device__ __forceinline__ double2 to2(V a) {
  return make_double2((double)a.x, (double)a.y);
}
template <typename V>
__device__ __forceinline__ V cfms(V a, V b, V c) {  // c - a*b
  return mk(fma(-a.x, b.x, fma(a.y, b.y, c.x)), fma(-a.x, b.y, fma(-a.y, b.x, c.y)));
}
template <typename V>
__device__ __forceinline__ V cfma(V a, V b, V c) {  // c + a*b
  return mk(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
template <typename V>
__device__ __forceinline__ V conjmul_acc(V a, V b, V c) {  // c + conj(a)*b
  return mk(fma(a.x, b.x, fma(a.y, b.y, c.x)), fma(a.x, b.y, fma(-a.y, b.x, c.y)));
}
__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 zadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 zsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 zdiv(double2 a, double2 b) {
  double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
__device__ __forceinline__ double zabs2(double2 a) { return a.x * a.x + a.y * a.y; }

inline unsigned grid_for(int64_t work, int block) { return (unsigned)((work + block - 1) / block); }

constexpr int IG = 8;  // basis vectors per dot-product pass
constexpr int KBLOCK = 256;

}  // namespace

// part[blk][i0+q][c] = sum over the block's rows of conj(V_{i0+q}[r][c]) W[r][c]
// (columns with mask[c] == 0 contribute zeros without reading their data)
template <typename V>
__global__ void k_mdot(const V* __restrict__ Vb, int64_t vstride, int i0, int ni, const V* __restrict__ W, int64_t n,
                       int s, int64_t rows_per_blk, double2* __restrict__ part, int mstride,
                       const int* __restrict__ mask) {
  __shared__ double2 sh[KBLOCK];
  const int nrl = blockDim.x / s;
  const int c = threadIdx.x % s, rl = threadIdx.x / s;
  V acc[IG];
#pragma unroll
  for (int q = 0; q < IG; ++q) acc[q] = zero<V>();
  const int64_t r0 = blockIdx.x * rows_per_blk;
  const int64_t r1 = (mask && !mask[c]) ? r0 : min(n, r0 + rows_per_blk);
  for (int64_t r = r0 + rl; r < r1; r += nrl) {
    const V w = W[r * s + c];
#pragma unroll
    for (int q = 0; q < IG; ++q)
      if (q < ni) acc[q] = conjmul_acc(Vb[(int64_t)(i0 + q) * vstride + r * s + c], w, acc[q]);
  }
  for (int q = 0; q < ni; ++q) {
    sh[threadIdx.x] = to2(acc[q]);
    __syncthreads();
    if (rl == 0) {
      double2 a = make_double2(0.0, 0.0);
      for (int l = 0; l < nrl; ++l) a = zadd(a, sh[l * s + c]);
      part[((int64_t)blockIdx.x * mstride + i0 + q) * s + c] = a;
    }
    __syncthreads();
  }
}

// out[i][c] = sum over blocks of part[blk][i][c]: one warp per (i, c), lanes
// stride over the blocks, fixed shuffle tree (deterministic)
__global__ void k_reduce_part(const double2* __restrict__ part, int nblk, int ni, int s, int mstride,
                              double2* __restrict__ out) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= ni * s) return;
  const int i = w / s, c = w % s;
  double2 a = make_double2(0.0, 0.0);
  for (int b = lane; b < nblk; b += 32) a = zadd(a, part[((int64_t)b * mstride + i) * s + c]);
  for (int o = 16; o > 0; o >>= 1) {
    a.x += __shfl_xor_sync(0xffffffffu, a.x, o);
    a.y += __shfl_xor_sync(0xffffffffu, a.y, o);
  }
  if (lane == 0) out[i * s + c] = a;
}

template <typename V>
static void mdot(DevKrylov& K, const V* Vb, int64_t vstride, int ni, const V* W, double2* out, cudaStream_t st,
                 const int* mask = nullptr) {
  const int s = K.s;
  const int block = (KBLOCK / s) * s;
  const int64_t rpb = (K.n + K.nblk - 1) / K.nblk;
  for (int i0 = 0; i0 < ni; i0 += IG)
    { k_mdot<V><<<K.nblk, block, 0, st>>>(Vb, vstride, i0, std::min(IG, ni - i0), W, K.n, s, rpb, K.hpart, K.m + 1,
                                        mask); count_launch(); }
  { k_reduce_part<<<grid_for((int64_t)ni * s * 32, 256), 256, 0, st>>>(K.hpart, K.nblk, ni, s, K.m + 1, out); count_launch(); }
}

// W[r][c] -= sum_{i<ni} V_i[r][c] h[i][c]
template <typename V>
__global__ void k_update(const V* __restrict__ Vb, int64_t vstride, int ni, const double2* __restrict__ h,
                         V* __restrict__ W, int64_t n, int s, const int* __restrict__ mask) {
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= n * s) return;
  int c = (int)(g % s);
  if (mask && !mask[c]) return;
  V w = W[g];
  for (int i = 0; i < ni; ++i) w = cfms(Vb[i * vstride + g], from2<V>(h[i * s + c]), w);
  W[g] = w;
}

template <typename V>
__global__ void k_scale_cols(const V* __restrict__ X, const double* __restrict__ sc, V* __restrict__ Y, int64_t n,
                             int s) {
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= n * s) return;
  const auto a = (decltype(V::x))sc[g % s];
  V x = X[g];
  Y[g] = mk(a * x.x, a * x.y);
}

// Second Gram-Schmidt pass only where the first one cancelled: with w the
// vector before and w' after the first pass, ||w'||^2 = ||w||^2 - sum |h_i|^2;
// reorthogonalise when ||w'||^2 < ||w||^2 / 2 ("twice is enough" criterion).
__global__ void k_reorth_flags(int s, int j, const double2* __restrict__ h1, const double2* __restrict__ w2,
                               int* __restrict__ flags) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= s) return;
  double hh = 0.0;
  for (int i = 0; i <= j; ++i) hh += zabs2(h1[i * s + c]);
  const double ww = w2[c].x;
  flags[c] = (ww - hh < 0.5 * ww) ? 1 : 0;
}

__global__ void k_norm_finish(const double2* __restrict__ nrm2, int s, double* __restrict__ out) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < s) out[c] = sqrt(nrm2[c].x);
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

// Column j of the Hessenberg matrix, the previous Givens rotations, the new
// one, the rotated right-hand side g and the residual estimate |g_{j+1}|.
__global__ void k_arnoldi_finish(int s, int m, int j, const double2* __restrict__ h1, const double2* __restrict__ h2,
                                 const double2* __restrict__ nrm2, double2* __restrict__ H, double* __restrict__ cs,
                                 double2* __restrict__ sn, double2* __restrict__ g, double* __restrict__ beta,
                                 const double* __restrict__ tol, int* __restrict__ kc, int* __restrict__ done,
                                 double* __restrict__ res, double2* __restrict__ Hraw) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= s) return;
  const double hb = sqrt(nrm2[c].x);
  double hn2 = hb * hb;
  for (int i = 0; i <= j; ++i) hn2 += zabs2(zadd(h1[i * s + c], h2[i * s + c]));
  const bool breakdown = !(hb > 1e-14 * sqrt(hn2));
  beta[c] = breakdown ? 0.0 : 1.0 / hb;
  if (done[c]) return;
  double2* Hc = H + (int64_t)c * (m + 1) * m + (int64_t)j * (m + 1);
  for (int i = 0; i <= j; ++i) Hc[i] = zadd(h1[i * s + c], h2[i * s + c]);
  Hc[j + 1] = make_double2(breakdown ? 0.0 : hb, 0.0);
  if (Hraw) {  // the unrotated column (recycling reads it after the cycle)
    double2* Hr = Hraw + (int64_t)c * (m + 1) * m + (int64_t)j * (m + 1);
    for (int i = 0; i <= j + 1; ++i) Hr[i] = Hc[i];
  }
  double* csc = cs + c * m;
  double2* snc = sn + c * m;
  for (int i = 0; i < j; ++i) {
    double2 a = Hc[i], b = Hc[i + 1];
    double ci = csc[i];
    double2 si = snc[i];
    Hc[i] = zadd(make_double2(ci * a.x, ci * a.y), zmul(si, b));
    Hc[i + 1] = zsub(make_double2(ci * b.x, ci * b.y), zmul(make_double2(si.x, -si.y), a));
  }
  double2 a = Hc[j], b = Hc[j + 1];
  double aa = sqrt(zabs2(a)), bb = sqrt(zabs2(b));
  double cj;
  double2 sj;
  if (bb == 0.0) {
    cj = 1.0;
    sj = make_double2(0.0, 0.0);
  } else if (aa == 0.0) {
    cj = 0.0;
    sj = make_double2(b.x / bb, -b.y / bb);
  } else {
    double tt = sqrt(aa * aa + bb * bb);
    cj = aa / tt;
    sj = zmul(make_double2(a.x / aa, a.y / aa), make_double2(b.x / tt, -b.y / tt));
  }
  csc[j] = cj;
  snc[j] = sj;
  Hc[j] = zadd(make_double2(cj * a.x, cj * a.y), zmul(sj, b));
  Hc[j + 1] = make_double2(0.0, 0.0);
  double2* gc = g + c * (m + 1);
  double2 gj = gc[j];
  gc[j] = make_double2(cj * gj.x, cj * gj.y);
  gc[j + 1] = zmul(make_double2(-sj.x, sj.y), gj);
  kc[c] = j + 1;
  double r = sqrt(zabs2(gc[j + 1]));
  res[c] = r;
  if (r <= tol[c] || breakdown) done[c] = 1;
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
    for (int l = i + 1; l < k; ++l) v = zsub(v, zmul(Hc[i + l * (m + 1)], yc[l]));
    double2 d = Hc[i + i * (m + 1)];
    yc[i] = (d.x == 0.0 && d.y == 0.0) ? make_double2(0.0, 0.0) : zdiv(v, d);
  }
}

template <typename V>
__global__ void k_sol_update(const V* __restrict__ Zk, int64_t vstride, const double2* __restrict__ y,
                             const int* __restrict__ kc, V* __restrict__ X, int64_t n, int s, int m) {
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= n * s) return;
  int c = (int)(g % s);
  V x = X[g];
  const int k = kc[c];
  for (int j = 0; j < k; ++j) x = cfma(Zk[j * vstride + g], from2<V>(y[c * m + j]), x);
  X[g] = x;
}

// double-float Gram-Schmidt products (below)
template <typename VB, typename VW>
static void mdot_df(DevKrylov& K, const VB* Vb, int64_t vstride, int ni, const VW* W, double2* out,
                    cudaStream_t st, const int* mask = nullptr);

template <typename V>
static void column_norms_t(const V* X, int64_t n, int s, double* out, DevKrylov& K, cudaStream_t st) {
  if constexpr (std::is_same<V, double2>::value) {
    if (K.df) {
      mdot_df(K, X, 0, 1, X, K.h2, st);
      { k_norm_finish<<<1, 64, 0, st>>>(K.h2, s, out); count_launch(); }
      return;
    }
  }
  mdot<V>(K, X, 0, 1, X, K.h2, st);
  { k_norm_finish<<<1, 64, 0, st>>>(K.h2, s, out); count_launch(); }
}

template <typename V>
static void krylov_start_t(DevKrylov& K, const V* R, cudaStream_t st) {
  if constexpr (std::is_same<V, double2>::value) {
    if (K.df)
      mdot_df(K, R, 0, 1, R, K.h2, st);
    else
      mdot<V>(K, R, 0, 1, R, K.h2, st);
  } else {
    mdot<V>(K, R, 0, 1, R, K.h2, st);
  }
  { k_start<<<1, 64, 0, st>>>(K.s, K.m, K.h2, K.tol, K.g, K.beta, K.kc, K.done, K.res); count_launch(); }
  { k_scale_cols<V><<<grid_for(K.n * K.s, 256), 256, 0, st>>>(R, K.beta, (V*)K.V, K.n, K.s); count_launch(); }
}

template <typename V>
static void krylov_arnoldi_t(DevKrylov& K, int j, cudaStream_t st) {
  const int64_t vs = K.n * K.s;
  const unsigned gr = grid_for(vs, 256);
  V* Vb = (V*)K.V;
  V* W = (V*)K.W;
  double2* nrm = K.h2 + (int64_t)K.m * K.s;  // row m of h2: scratch for |W|^2
  mdot<V>(K, W, 0, 1, W, nrm, st);
  mdot<V>(K, Vb, vs, j + 1, W, K.h1, st);
  { k_update<V><<<gr, 256, 0, st>>>(Vb, vs, j + 1, K.h1, W, K.n, K.s, nullptr); count_launch(); }
  { k_reorth_flags<<<1, 64, 0, st>>>(K.s, j, K.h1, nrm, K.reorth); count_launch(); }
  mdot<V>(K, Vb, vs, j + 1, W, K.h2, st, K.reorth);
  { k_update<V><<<gr, 256, 0, st>>>(Vb, vs, j + 1, K.h2, W, K.n, K.s, K.reorth); count_launch(); }
  mdot<V>(K, W, 0, 1, W, nrm, st);
  { k_arnoldi_finish<<<1, 64, 0, st>>>(K.s, K.m, j, K.h1, K.h2, nrm, K.H, K.cs, K.sn, K.g, K.beta, K.tol, K.kc, K.done,
                                     K.res, K.Hraw); count_launch(); }
  { k_scale_cols<V><<<gr, 256, 0, st>>>(W, K.beta, Vb + (int64_t)(j + 1) * vs, K.n, K.s); count_launch(); }
}

// ---------------------------------------------------------------------------
// Double-float Arnoldi (FP64 Krylov spaces of the mixed form with
// emulate_fp64): the same CGS with selective reorthogonalisation, the
// products and updates in double-float arithmetic (FP32 pairs). The basis
// stays in FP64 (the preconditioner reads it) and is split into FP32 pairs by
// its bit layout as it is read, so that it costs no second copy; W (A z) is a
// double-float block. The partial dot products of each thread are converted
// to FP64 and summed in FP64 in the same fixed order as above; Hessenberg,
// rotations and least squares unchanged.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float4 df_split2(const double2 v) {
  const float2 r = df_split(v.x), i = df_split(v.y);
  return make_float4(r.x, r.y, i.x, i.y);
}
__device__ __forceinline__ float4 as_df(const float4 v) { return v; }
__device__ __forceinline__ float4 as_df(const double2 v) { return df_split2(v); }

// (reh, rel, imh, iml) += conj(v) w
__device__ __forceinline__ void df_conj_mac(float4& a, const float4 v, const float4 w) {
  df_mac(a.x, a.y, v.x, v.y, w.x, w.y);    // re += vr wr
  df_mac(a.x, a.y, v.z, v.w, w.z, w.w);    // re += vi wi
  df_mac(a.z, a.w, v.x, v.y, w.z, w.w);    // im += vr wi
  df_mac(a.z, a.w, -v.z, -v.w, w.x, w.y);  // im -= vi wr
}

// VB, VW: double2 (FP64, split as read) or float4 (double-float)
template <typename VB, typename VW>
__global__ void k_mdot_df(const VB* __restrict__ Vb, int64_t vstride, int i0, int ni,
                          const VW* __restrict__ W, int64_t n, int s, int64_t rows_per_blk,
                          double2* __restrict__ part, int mstride, const int* __restrict__ mask) {
  __shared__ double2 sh[KBLOCK];
  const int nrl = blockDim.x / s;
  const int c = threadIdx.x % s, rl = threadIdx.x / s;
  float4 acc[IG];
#pragma unroll
  for (int q = 0; q < IG; ++q) acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
  const int64_t r0 = blockIdx.x * rows_per_blk;
  const int64_t r1 = (mask && !mask[c]) ? r0 : min(n, r0 + rows_per_blk);
  for (int64_t r = r0 + rl; r < r1; r += nrl) {
    const float4 w = as_df(W[r * s + c]);
#pragma unroll
    for (int q = 0; q < IG; ++q)
      if (q < ni) df_conj_mac(acc[q], as_df(Vb[(int64_t)(i0 + q) * vstride + r * s + c]), w);
  }
  for (int q = 0; q < ni; ++q) {
    sh[threadIdx.x] = make_double2(f2d(acc[q].x) + f2d(acc[q].y), f2d(acc[q].z) + f2d(acc[q].w));
    __syncthreads();
    if (rl == 0) {
      double2 a = make_double2(0.0, 0.0);
      for (int l = 0; l < nrl; ++l) a = zadd(a, sh[l * s + c]);
      part[((int64_t)blockIdx.x * mstride + i0 + q) * s + c] = a;
    }
    __syncthreads();
  }
}

template <typename VB, typename VW>
static void mdot_df(DevKrylov& K, const VB* Vb, int64_t vstride, int ni, const VW* W, double2* out,
                    cudaStream_t st, const int* mask) {
  const int s = K.s;
  const int block = (KBLOCK / s) * s;
  const int64_t rpb = (K.n + K.nblk - 1) / K.nblk;
  for (int i0 = 0; i0 < ni; i0 += IG)
    { k_mdot_df<VB, VW><<<K.nblk, block, 0, st>>>(Vb, vstride, i0, std::min(IG, ni - i0), W, K.n, s, rpb, K.hpart,
                                            K.m + 1, mask); count_launch(); }
  { k_reduce_part<<<grid_for((int64_t)ni * s * 32, 256), 256, 0, st>>>(K.hpart, K.nblk, ni, s, K.m + 1, out); count_launch(); }
}

// h (FP64) -> double-float
__global__ void k_h_df(const double2* __restrict__ h, float4* __restrict__ out, int count) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= count) return;
  const float2 a = df_split(h[g].x), b = df_split(h[g].y);
  out[g] = make_float4(a.x, a.y, b.x, b.y);
}

// W[r][c] -= sum_{i<ni} V_i[r][c] h[i][c], double-float (V in FP64, split as read)
__global__ void k_update_df(const double2* __restrict__ Vb, int64_t vstride, int ni, const float4* __restrict__ h,
                            float4* __restrict__ W, int64_t n, int s, const int* __restrict__ mask) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= n * s) return;
  const int c = (int)(g % s);
  if (mask && !mask[c]) return;
  float4 w = W[g];
  for (int i = 0; i < ni; ++i) {
    const float4 v = df_split2(Vb[i * vstride + g]), hc = h[i * s + c];
    df_mac(w.x, w.y, -v.x, -v.y, hc.x, hc.y);  // re -= vr hr
    df_mac(w.x, w.y, v.z, v.w, hc.z, hc.w);    // re += vi hi
    df_mac(w.z, w.w, -v.x, -v.y, hc.z, hc.w);  // im -= vr hi
    df_mac(w.z, w.w, -v.z, -v.w, hc.x, hc.y);  // im -= vi hr
  }
  df_norm(w.x, w.y);
  df_norm(w.z, w.w);
  W[g] = w;
}

// v = w beta[c] (double-float product, stored in FP64: hi + lo is exact in FP64)
__global__ void k_scale_df(const float4* __restrict__ X, const double* __restrict__ beta, double2* __restrict__ Y,
                           int64_t n, int s) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= n * s) return;
  const float2 b = df_split(beta[g % s]);
  const float4 x = X[g];
  float4 y;
  df_mul(y.x, y.y, x.x, x.y, b.x, b.y);
  df_mul(y.z, y.w, x.z, x.w, b.x, b.y);
  Y[g] = make_double2(f2d(y.x) + f2d(y.y), f2d(y.z) + f2d(y.w));
}

static void krylov_arnoldi_df(DevKrylov& K, int j, cudaStream_t st) {
  const int64_t vs = K.n * K.s;
  const unsigned gr = grid_for(vs, 256);
  double2* nrm = K.h2 + (int64_t)K.m * K.s;
  const int nh = (j + 1) * K.s;
  mdot_df(K, K.Wdf, 0, 1, K.Wdf, nrm, st);
  const double2* Vb = (const double2*)K.V;
  mdot_df(K, Vb, vs, j + 1, K.Wdf, K.h1, st);
  { k_h_df<<<grid_for(nh, 128), 128, 0, st>>>(K.h1, K.hdf, nh); count_launch(); }
  { k_update_df<<<gr, 256, 0, st>>>(Vb, vs, j + 1, K.hdf, K.Wdf, K.n, K.s, nullptr); count_launch(); }
  { k_reorth_flags<<<1, 64, 0, st>>>(K.s, j, K.h1, nrm, K.reorth); count_launch(); }
  mdot_df(K, Vb, vs, j + 1, K.Wdf, K.h2, st, K.reorth);
  { k_h_df<<<grid_for(nh, 128), 128, 0, st>>>(K.h2, K.hdf, nh); count_launch(); }
  { k_update_df<<<gr, 256, 0, st>>>(Vb, vs, j + 1, K.hdf, K.Wdf, K.n, K.s, K.reorth); count_launch(); }
  mdot_df(K, K.Wdf, 0, 1, K.Wdf, nrm, st);
  { k_arnoldi_finish<<<1, 64, 0, st>>>(K.s, K.m, j, K.h1, K.h2, nrm, K.H, K.cs, K.sn, K.g, K.beta, K.tol, K.kc, K.done,
                                     K.res, K.Hraw); count_launch(); }
  { k_scale_df<<<gr, 256, 0, st>>>(K.Wdf, K.beta, (double2*)K.V + (j + 1) * vs, K.n, K.s); count_launch(); }
}

template <typename V>
static void krylov_update_t(DevKrylov& K, V* X, cudaStream_t st) {
  { k_ls_solve<<<1, 64, 0, st>>>(K.s, K.m, K.H, K.g, K.kc, K.y); count_launch(); }
  { k_sol_update<V><<<grid_for(K.n * K.s, 256), 256, 0, st>>>((const V*)K.Zk, K.n * K.s, K.y, K.kc, X, K.n, K.s, K.m); count_launch(); }
}

void column_norms(const void* X, int64_t n, int s, double* out, DevKrylov& K, cudaStream_t st) {
  if (K.fp32)
    column_norms_t<float2>((const float2*)X, n, s, out, K, st);
  else
    column_norms_t<double2>((const double2*)X, n, s, out, K, st);
}
void krylov_start(DevKrylov& K, const void* R, cudaStream_t st) {
  if (K.fp32) {
    krylov_start_t<float2>(K, (const float2*)R, st);
  } else {
    krylov_start_t<double2>(K, (const double2*)R, st);
  }
}
void krylov_arnoldi(DevKrylov& K, int j, cudaStream_t st) {
  if (K.df)
    krylov_arnoldi_df(K, j, st);
  else if (K.fp32)
    krylov_arnoldi_t<float2>(K, j, st);
  else
    krylov_arnoldi_t<double2>(K, j, st);
}
void krylov_update(DevKrylov& K, void* X, cudaStream_t st) {
  if (K.fp32)
    krylov_update_t<float2>(K, (float2*)X, st);
  else
    krylov_update_t<double2>(K, (double2*)X, st);
}

// ---------------------------------------------------------------------------
// FP32 coarse-level helpers (mixed form): SpMM with float values, gathers
// and scatters between FP32 blocks, precision casts
// ---------------------------------------------------------------------------
// Y = A X, or Y = B - A X when B is given (FP32 values and blocks)
__global__ void k_spmm_split_f32(int64_t n, int s, const int64_t* __restrict__ rp_re, const int32_t* __restrict__ col_re,
                                 const float* __restrict__ val_re, const int64_t* __restrict__ rp_im,
                                 const int32_t* __restrict__ col_im, const float* __restrict__ val_im,
                                 const float2* __restrict__ X, float2* __restrict__ Y, const float2* __restrict__ B) {
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t r = g / s;
  int c = (int)(g - r * s);
  if (r >= n) return;
  float ar = 0.f, ai = 0.f;
  #pragma unroll 4
  for (int64_t p = rp_re[r], pe = rp_re[r + 1]; p < pe; ++p) {
    float a = val_re[p];
    float2 x = X[(int64_t)col_re[p] * s + c];
    ar = fmaf(a, x.x, ar);
    ai = fmaf(a, x.y, ai);
  }
  #pragma unroll 4
  for (int64_t p = rp_im[r], pe = rp_im[r + 1]; p < pe; ++p) {
    float b = val_im[p];
    float2 x = X[(int64_t)col_im[p] * s + c];
    ar = fmaf(-b, x.y, ar);
    ai = fmaf(b, x.x, ai);
  }
  if (B) {
    const float2 b = B[g];
    Y[g] = make_float2(b.x - ar, b.y - ai);
  } else {
    Y[g] = make_float2(ar, ai);
  }
}

void spmm_split_f32(const DevSplitCsr& A, const float2* X, float2* Y, int s, cudaStream_t st, const float2* B) {
  int64_t work = A.n * s;
  if (work == 0) return;
  { k_spmm_split_f32<<<grid_for(work, 256), 256, 0, st>>>(A.n, s, A.rp_re, A.col_re, A.val_re_f, A.rp_im, A.col_im,
                                                        A.val_im_f, X, Y, B); count_launch(); }
}

__global__ void k_spmm_real_f32(int64_t n, int s, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                const float* __restrict__ val, const float2* __restrict__ X, float2* __restrict__ Y) {
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t r = g / s;
  int c = (int)(g - r * s);
  if (r >= n) return;
  float ar = 0.f, ai = 0.f;
  #pragma unroll 4
  for (int64_t p = rp[r], pe = rp[r + 1]; p < pe; ++p) {
    float a = val[p];
    float2 x = X[(int64_t)col[p] * s + c];
    ar = fmaf(a, x.x, ar);
    ai = fmaf(a, x.y, ai);
  }
  Y[g] = make_float2(ar, ai);
}

void spmm_real_f32(int64_t nrows, const int64_t* rp, const int32_t* col, const float* val, const float2* X,
                   float2* Y, int s, cudaStream_t st) {
  if (nrows * s) { k_spmm_real_f32<<<grid_for(nrows * s, 256), 256, 0, st>>>(nrows, s, rp, col, val, X, Y); count_launch(); }
}

// z = (FP64) Xsub[owning copy] + (FP64) q  (prolongation of the FP32 local solutions)
__global__ void k_scatter_owned_fq(const int* __restrict__ own, int64_t n, const float2* __restrict__ Xsub,
                                   const float2* __restrict__ Q, double2* __restrict__ Z, int s) {
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t r = g / s;
  if (r >= n) return;
  const float2 v = Xsub[(int64_t)own[r] * s + (g - r * s)];
  const float2 q = Q[g];
  Z[g] = make_double2((double)v.x + (double)q.x, (double)v.y + (double)q.y);
}
void scatter_owned_fq(const int* own, int64_t n, const float2* Xsub, const float2* Q, double2* Z, int s,
                      cudaStream_t st) {
  if (n * s) { k_scatter_owned_fq<<<grid_for(n * s, 256), 256, 0, st>>>(own, n, Xsub, Q, Z, s); count_launch(); }
}

__global__ void k_gather_ff(const int* __restrict__ idx, int64_t nrows, const float2* __restrict__ X,
                            float2* __restrict__ Y, int s) {
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t r = g / s;
  if (r >= nrows) return;
  Y[g] = X[(int64_t)idx[r] * s + (g - r * s)];
}
void gather_rows_ff(const int* idx, int64_t nrows, const float2* X, float2* Y, int s, cudaStream_t st) {
  if (nrows * s) { k_gather_ff<<<grid_for(nrows * s, 256), 256, 0, st>>>(idx, nrows, X, Y, s); count_launch(); }
}

__global__ void k_scatter_ff(const int* __restrict__ own, int64_t n, const float2* __restrict__ Xsub,
                             float2* __restrict__ Z, int s) {
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t r = g / s;
  if (r >= n) return;
  Z[g] = Xsub[(int64_t)own[r] * s + (g - r * s)];
}
void scatter_owned_ff(const int* own, int64_t n, const float2* Xsub, float2* Z, int s, cudaStream_t st) {
  if (n * s) { k_scatter_ff<<<grid_for(n * s, 256), 256, 0, st>>>(own, n, Xsub, Z, s); count_launch(); }
}

__global__ void k_d2f(const double2* __restrict__ X, float2* __restrict__ Y, int64_t count) {
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g < count) Y[g] = make_float2((float)X[g].x, (float)X[g].y);
}
__global__ void k_f2d(const float2* __restrict__ X, double2* __restrict__ Y, int64_t count) {
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g < count) Y[g] = make_double2(X[g].x, X[g].y);
}
void cast_d2f(const double2* X, float2* Y, int64_t count, cudaStream_t st) {
  if (count) { k_d2f<<<grid_for(count, 256), 256, 0, st>>>(X, Y, count); count_launch(); }
}
void cast_f2d(const float2* X, double2* Y, int64_t count, cudaStream_t st) {
  if (count) { k_f2d<<<grid_for(count, 256), 256, 0, st>>>(X, Y, count); count_launch(); }
}

}  // namespace hz
