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
// so that each level of each sweep is two flat launches: fixed-size
// 128 x 256 factor tiles split along the reduction (balanced over all SMs
// whatever the front sizes; the extend-add of the children's update vectors
// is done while staging the input), and a fixed-order sum of the tiles'
// partial results. FP64, or FP32 in the mixed
// form. X_t is stored twice, column-major and transposed, so that both
// sweeps read their factor with unit stride across a warp.
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
                             V* __restrict__ MT, V* __restrict__ Dinv) {
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
  V* MTt = MT + Moff[t];
  const int64_t fk = (int64_t)f * k;
  for (int64_t i = threadIdx.x; i < fk; i += blockDim.x) {
    int r = (int)(i % f), c = (int)(i / f);
    double2 v = r == c ? make_double2(1.0, 0.0) : (r < c ? make_double2(0.0, 0.0) : Ft[i]);
    Mt[i] = from_d<V>(v);
    MTt[c + (int64_t)r * k] = from_d<V>(v);
  }
}

template <typename V>
static void tile_attrs_all();

void mf_factor(DevMF& mf, double tau_abs, cudaStream_t st) {
  if (mf.fp32)
    tile_attrs_all<float2>();
  else
    tile_attrs_all<double2>();
  size_t shm = (size_t)std::max(mf.max_f, 1) * sizeof(double2);
  cudaFuncSetAttribute(k_mf_factor, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
  cudaFuncSetAttribute(k_mf_inverse<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
  cudaFuncSetAttribute(k_mf_inverse<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
  for (int l = 0; l < mf.nlevels; ++l) {
    int b = mf.level_ptr_h[l], e = mf.level_ptr_h[l + 1];
    if (e == b) continue;
    { k_mf_assemble<<<e - b, 256, 0, st>>>(mf.level_list + b, mf.k, mf.f, mf.Foff, mf.rowoff, mf.cmap, mf.child_ptr,
                                         mf.child_idx, mf.amap_ptr, mf.amap_pos, mf.amap_val, mf.Aval, mf.F); count_launch(); }
    { k_mf_factor<<<e - b, 256, shm, st>>>(mf.level_list + b, mf.k, mf.f, mf.Foff, mf.F, tau_abs, mf.perturbed); count_launch(); }
  }
  // the inverses only touch the pivot columns: run them after every Schur
  // complement has been consumed by its parent
  for (int l = 0; l < mf.nlevels; ++l) {
    int b = mf.level_ptr_h[l], e = mf.level_ptr_h[l + 1];
    if (e == b) continue;
    if (mf.fp32)
      { k_mf_inverse<float2><<<e - b, 256, shm, st>>>(mf.level_list + b, mf.k, mf.f, mf.Foff, mf.Moff, mf.Doff, mf.F,
                                                    (float2*)mf.M, (float2*)mf.MT, (float2*)mf.Dinv); count_launch(); }
    else
      { k_mf_inverse<double2><<<e - b, 256, shm, st>>>(mf.level_list + b, mf.k, mf.f, mf.Foff, mf.Moff, mf.Doff,
                                                     mf.F, (double2*)mf.M, (double2*)mf.MT, (double2*)mf.Dinv); count_launch(); }
  }
}

// ---------------------------------------------------------------------------
// Solve sweeps
// ---------------------------------------------------------------------------
constexpr int MF_TILE = 128;  // output rows per tile (MF_TILE_ROWS on the host)
constexpr int MF_TK = 128;    // reduction length per tile (MF_TILE_K on the host)

// One tile: MF_TILE output rows x MF_TK reduction indices of
//   forward : t = X_t b_P      (X_t column-major f x k); b_P at a pivot row
//             is the sub-vector entry plus the children's update vectors
//             that land on it (extend-add, child order)
//   backward: x = X_t^T v      (X_t^T column-major k x f, v = [y_P; x_U]:
//             y_P kept in Wout by the forward sweep, x_U the final values of
//             the ancestors' pivots in the sub-vector)
// A row block covered by one tile (slot < 0) applies the epilogue directly;
// otherwise the tile writes a partial result to its slot of P and the row
// block's partials are summed in a fixed order by k_mf_reduce. Epilogue:
//   forward : rows r < k -> y = t / D (kept in Wout for the backward sweep);
//             rows r >= k -> parent update c_U + t (Wout), c_U = the children's
//             update vectors landing on the row
//   backward: x at the pivot rows of the sub-vector
// Each thread owns R output rows
// (NT apart, so a warp reads 32 consecutive factor entries per column) and
// the s right-hand sides as register accumulators; chunks of the input vector
// are staged in shared memory and read as broadcasts.
__device__ __forceinline__ void cp_async_elem(void* dst_smem, const float2* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_elem(void* dst_smem, const double2* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// columns of the factor tile per asynchronous chunk (two chunks in flight)
template <typename V>
struct TileChunk {
  static constexpr int K = sizeof(V) == 8 ? 16 : 8;
};

template <typename V, int S>
static constexpr size_t tile_smem_bytes() {
  return sizeof(V) * ((size_t)MF_TK * S + 2 * (size_t)TileChunk<V>::K * MF_TILE);
}

// Each thread owns one output row (MF_TILE threads) and keeps the s
// right-hand sides as register accumulators. The tile's input rows are
// staged once in shared memory (read as broadcasts); the factor tile streams
// through a two-chunk shared-memory ring filled by cp.async (a warp copies 32
// consecutive entries of one factor column), so the next chunk's loads are in
// flight while the current one is consumed.
template <typename V, int S, bool FWD>
__global__ void __launch_bounds__(MF_TILE) k_mf_tile(const int4* __restrict__ tiles, const int* __restrict__ kk,
                                                     const int* __restrict__ ff, const int64_t* __restrict__ rowoff,
                                                     const int64_t* __restrict__ Moff, const V* __restrict__ M,
                                                     const int* __restrict__ rows, const int64_t* __restrict__ cptr,
                                                     const int* __restrict__ cidx, const int64_t* __restrict__ Doff,
                                                     const V* __restrict__ Dinv, V* __restrict__ Xsub,
                                                     V* __restrict__ Wout, V* __restrict__ P, int s) {
  constexpr int KCH = TileChunk<V>::K;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V(*bs)[S] = reinterpret_cast<V(*)[S]>(smem_raw);                                       // [MF_TK][S]
  V(*mb)[MF_TILE] = reinterpret_cast<V(*)[MF_TILE]>(smem_raw + sizeof(V) * MF_TK * S);  // [2 KCH][MF_TILE]
  const int4 tile = tiles[blockIdx.x];
  const int t = tile.x, r0 = tile.y, c0 = tile.z, slot = tile.w;
  const int f = ff[t], k = kk[t];
  const int nout = FWD ? f : k;
  const int ld = FWD ? f : k;
  const int kend = FWD ? ((r0 < k) ? min(k, r0 + MF_TILE) : k) : f;
  const int kbeg = FWD ? c0 : max(c0, r0);  // X_t^T is zero left of the diagonal of its pivot block
  const int kstop = min(kend, c0 + MF_TK);
  const V* Mt = M + Moff[t];
  const int64_t ro = rowoff[t];
  const int tid = threadIdx.x;
  const int lmax = max(0, kstop - kbeg);
  const int rr = r0 + tid;
  const bool act = rr < nout;
  const V* mcol = Mt + (act ? rr : 0) + (int64_t)kbeg * ld;
  const int nch = (lmax + KCH - 1) / KCH;
  // chunk 0 in flight while the input rows are staged
  if (nch > 0) {
    const int cn = min(KCH, lmax);
    if (act)
      for (int j = 0; j < cn; ++j) cp_async_elem(&mb[j][tid], mcol + (int64_t)j * ld);
  }
  cp_async_commit();
  for (int l = tid; l < lmax; l += MF_TILE) {
    const int64_t R = ro + kbeg + l;
    const int local = kbeg + l;
    V v[S];
    const V* src = (FWD || local >= k) ? Xsub + (int64_t)rows[R] * s : Wout + R * s;
#pragma unroll
    for (int c = 0; c < S; ++c) v[c] = c < s ? src[c] : mk2((decltype(V::x))0, (decltype(V::x))0);
    if (FWD) {
      const int64_t pe = cptr[R + 1];
      for (int64_t p = cptr[R]; p < pe; ++p) {
        const V* w = Wout + (int64_t)cidx[p] * s;
#pragma unroll
        for (int c = 0; c < S; ++c)
          if (c < s) v[c] = c_add(v[c], w[c]);
      }
    }
#pragma unroll
    for (int c = 0; c < S; ++c) bs[l][c] = v[c];
  }
  V acc[S];
#pragma unroll
  for (int c = 0; c < S; ++c) acc[c] = mk2((decltype(V::x))0, (decltype(V::x))0);
  for (int ch = 0; ch < nch; ++ch) {
    // issue chunk ch + 1 into the other half of the ring, then wait for ch
    if (ch + 1 < nch) {
      const int j0 = (ch + 1) * KCH, cn = min(KCH, lmax - j0);
      const int half = ((ch + 1) & 1) * KCH;
      if (act)
        for (int j = 0; j < cn; ++j) cp_async_elem(&mb[half + j][tid], mcol + (int64_t)(j0 + j) * ld);
    }
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    const int half = (ch & 1) * KCH;
    const int j0 = ch * KCH, cn = min(KCH, lmax - j0);
#pragma unroll 4
    for (int j = 0; j < cn; ++j) {
      const V m = mb[half + j][tid];
#pragma unroll
      for (int c = 0; c < S; ++c) acc[c] = c_fma(m, bs[j0 + j][c], acc[c]);
    }
    __syncthreads();  // the half just read is refilled in the next iteration
  }
  cp_async_wait<0>();
  if (slot >= 0) {
    V* out = P + ((int64_t)slot * MF_TILE + tid) * s;
#pragma unroll
    for (int c = 0; c < S; ++c)
      if (c < s) out[c] = acc[c];
    return;
  }
  if (!act) return;
  const int64_t Rg = ro + rr;
  if (FWD) {
    if (rr < k) {
      const V di = Dinv[Doff[t] + rr];
#pragma unroll
      for (int c = 0; c < S; ++c)
        if (c < s) Wout[Rg * s + c] = c_mul(acc[c], di);
    } else {
      // parent update: the children's update vectors landing on this row,
      // one contiguous row of s values per contribution
      const int64_t pe = cptr[Rg + 1];
      for (int64_t p = cptr[Rg]; p < pe; ++p) {
        const V* w = Wout + (int64_t)cidx[p] * s;
#pragma unroll
        for (int c = 0; c < S; ++c)
          if (c < s) acc[c] = c_add(acc[c], w[c]);
      }
#pragma unroll
      for (int c = 0; c < S; ++c)
        if (c < s) Wout[Rg * s + c] = acc[c];
    }
  } else {
    V* xo = Xsub + (int64_t)rows[Rg] * s;
#pragma unroll
    for (int c = 0; c < S; ++c)
      if (c < s) xo[c] = acc[c];
  }
}

// Row-block epilogue, one thread per (row, column): sum the row block's
// partial tiles in order, then
//   forward : rows r < k -> y = t / D (kept in Wout for the backward sweep);
//             rows r >= k -> parent update c_U + t (Wout), c_U = the children's
//             update vectors landing on the row
//   backward: x at the pivot rows of the sub-vector
template <typename V, bool FWD>
__global__ void k_mf_reduce(const int4* __restrict__ rblocks, int nrb, const int* __restrict__ kk,
                            const int* __restrict__ ff, const int64_t* __restrict__ rowoff,
                            const int64_t* __restrict__ Doff, const int* __restrict__ rows,
                            const int64_t* __restrict__ cptr, const int* __restrict__ cidx,
                            const V* __restrict__ Dinv, V* __restrict__ Wout, const V* __restrict__ P,
                            V* __restrict__ Xsub, int s) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t per = (int64_t)MF_TILE * s;
  if (g >= nrb * per) return;
  const int4 rb = rblocks[g / per];
  const int i = (int)((g % per) / s), c = (int)(g % s);
  const int t = rb.x, r = rb.y + i;
  const int k = kk[t];
  if (r >= (FWD ? ff[t] : k)) return;
  V acc = mk2((decltype(V::x))0, (decltype(V::x))0);
  for (int q = 0; q < rb.z; ++q) acc = c_add(acc, P[((int64_t)(rb.w + q) * MF_TILE + i) * s + c]);
  const int64_t R = rowoff[t] + r;
  if (FWD) {
    if (r < k) {
      Wout[R * s + c] = c_mul(acc, Dinv[Doff[t] + r]);
    } else {
      for (int64_t p = cptr[R]; p < cptr[R + 1]; ++p) acc = c_add(acc, Wout[(int64_t)cidx[p] * s + c]);
      Wout[R * s + c] = acc;
    }
  } else {
    Xsub[(int64_t)rows[R] * s + c] = acc;
  }
}

static inline unsigned blocks_for(int64_t work, int b) { return (unsigned)((work + b - 1) / b); }

template <typename V, int S>
static void solve_impl(DevMF& mf, V* Xsub, int s, cudaStream_t st) {
  const size_t shm = tile_smem_bytes<V, S>();
  V* Wout = (V*)mf.Wout;
  V* P = (V*)mf.P;
  const V* M = (const V*)mf.M;
  const V* MT = (const V*)mf.MT;
  const V* Dv = (const V*)mf.Dinv;
  for (int l = 0; l < mf.nlevels; ++l) {
    const int tb = mf.ftile_ptr_h[l], te = mf.ftile_ptr_h[l + 1];
    if (te > tb)
      { k_mf_tile<V, S, true><<<te - tb, MF_TILE, shm, st>>>(mf.ftiles + tb, mf.k, mf.f, mf.rowoff, mf.Moff, M, mf.rows,
                                                             mf.cptr, mf.cidx, mf.Doff, Dv, Xsub, Wout, P, s); count_launch(); }
    const int rb = mf.frb_ptr_h[l], re = mf.frb_ptr_h[l + 1];
    if (re > rb)
      { k_mf_reduce<V, true><<<blocks_for((int64_t)(re - rb) * MF_TILE * s, 256), 256, 0, st>>>(
          mf.frb + rb, re - rb, mf.k, mf.f, mf.rowoff, mf.Doff, mf.rows, mf.cptr, mf.cidx, Dv, Wout, P, Xsub, s); count_launch(); }
  }
  for (int l = mf.nlevels - 1; l >= 0; --l) {
    const int tb = mf.btile_ptr_h[l], te = mf.btile_ptr_h[l + 1];
    if (te > tb)
      { k_mf_tile<V, S, false><<<te - tb, MF_TILE, shm, st>>>(mf.btiles + tb, mf.k, mf.f, mf.rowoff, mf.Moff, MT,
                                                              mf.rows, mf.cptr, mf.cidx, mf.Doff, Dv, Xsub, Wout, P, s); count_launch(); }
    const int rb = mf.brb_ptr_h[l], re = mf.brb_ptr_h[l + 1];
    if (re > rb)
      { k_mf_reduce<V, false><<<blocks_for((int64_t)(re - rb) * MF_TILE * s, 256), 256, 0, st>>>(
          mf.brb + rb, re - rb, mf.k, mf.f, mf.rowoff, mf.Doff, mf.rows, mf.cptr, mf.cidx, Dv, Wout, P, Xsub, s); count_launch(); }
  }
}

// Opt the tile kernels into their dynamic shared memory once, outside any
// stream capture (called from the factorisation).
template <typename V, int S>
static void tile_attrs() {
  const int shm = (int)tile_smem_bytes<V, S>();
  cudaFuncSetAttribute(k_mf_tile<V, S, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, shm);
  cudaFuncSetAttribute(k_mf_tile<V, S, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, shm);
}

#define HZ_TILE_WIDTHS(X) X(1) X(2) X(4) X(8) X(16) X(32) X(64)

template <typename V>
static void tile_attrs_all() {
#define HZ_ATTR(S) tile_attrs<V, S>();
  HZ_TILE_WIDTHS(HZ_ATTR)
#undef HZ_ATTR
}

template <typename V>
static void solve_dispatch(DevMF& mf, V* Xsub, int s, cudaStream_t st) {
#define HZ_CASE(S)                       \
  if (s <= S) {                          \
    solve_impl<V, S>(mf, Xsub, s, st);   \
    return;                              \
  }
  HZ_TILE_WIDTHS(HZ_CASE)
#undef HZ_CASE
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
  { k_gather_rows_f32<<<(unsigned)((nrows * s + 255) / 256), 256, 0, st>>>(idx, nrows, X, Y, s); count_launch(); }
}

void scatter_owned_f32(const int* own, int64_t n, const float2* Xsub, const double2* Q, double2* Z, int s,
                       cudaStream_t st) {
  if (n * s == 0) return;
  { k_scatter_owned_f32<<<(unsigned)((n * s + 255) / 256), 256, 0, st>>>(own, n, Xsub, Q, Z, s); count_launch(); }
}

}  // namespace hz
