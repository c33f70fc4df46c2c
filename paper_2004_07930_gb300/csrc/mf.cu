// Partitioned-inverse solves of the local matrices A_i (the paper's direct
// local solver inside Eq. oras); the factorisation is in factor.cu.
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
#include <type_traits>

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

template <typename V>
static void tile_attrs_all();
static void tc_pack_all(DevMF& mf, cudaStream_t st);
void mf_factor_fronts(DevMF& mf, double tau_abs, cudaStream_t st);  // factor.cu

// Numeric factorisation and partitioned inverse (factor.cu), then the
// sweep kernels' attributes and the tensor-core tile packing.
void mf_factor(DevMF& mf, double tau_abs, cudaStream_t st) {
  if (mf.fp32)
    tile_attrs_all<float2>();
  else
    tile_attrs_all<double2>();
  mf_factor_fronts(mf, tau_abs, st);
  // tensor-core tiles: pack their factor blocks from X_t (forward) and X_t^T (backward)
  if (mf.tc && mf.fp32) tc_pack_all(mf, st);
}

bool mf_tc_usable(const DevMF& mf, int s) { return mf.tc && mf.fp32 && s > 8 && s <= 16; }

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
template <typename V, int S>
static constexpr size_t tile_smem_bytes() {
  return sizeof(V) * (size_t)MF_TK * S;  // the staged input rows
}

// loads of data that other CTAs of the same launch write (persistent sweeps):
// through L2 only, so that no stale line of this SM's L1 is read
template <bool CG, typename V>
__device__ __forceinline__ V ldv(const V* p) {
  if constexpr (CG)
    return __ldcg(p);
  else
    return *p;
}

// One tile. TPR threads share each output row (MF_TILE x TPR threads), each
// keeping S/TPR of the right-hand sides as register accumulators, so that a
// tile's serial work per thread (and its latency) shrinks with TPR while the
// accumulation order of every column stays the same. The tile's input rows
// are staged once in shared memory (read as broadcasts); each thread streams
// its row of the factor tile straight from global memory (the TPR threads of
// a row read the same entry, a warp 32/TPR consecutive entries of one factor
// column per load), the next MF_UNROLL columns in flight while the current
// ones are used (the first batch while the input rows are staged), so the only
// barrier is the one after the staging and the small shared-memory footprint
// leaves room for several CTAs per SM. A tile with slot >= 0 writes its
// partial result to P; the others apply the epilogue.
constexpr int MF_UNROLL = 8;
// threads per output row for a block width S in the short launches (a level
// with fewer than MF_SHORT_LEVEL tiles, where one tile's latency bounds the
// launch); levels with more tiles, and the persistent sweep, keep one thread
// per row
template <int S>
__host__ __device__ constexpr int tile_tpr() {
  return S >= 16 ? 4 : (S >= 8 ? 2 : 1);
}
constexpr int MF_SHORT_LEVEL = 1536;
// a long level whose tiles all have at most MF_HALF output rows (the leaf
// fronts' pivot rows in the backward sweep, for instance) runs half-height
// tiles: MF_HALF rows, tile_tpr_half threads per row, no idle threads
constexpr int MF_HALF = 64;
template <int S>
__host__ __device__ constexpr int tile_tpr_half() {
  return S >= 2 ? 2 : 1;
}
// complex FP32 tiles of up to 16 columns: 1024 resident threads per SM with
// several threads per row (64 registers per thread), 6 half-height tiles of
// 128 threads (85 registers), 5 blocks of 128 with one thread per row (102)
template <typename V, int S, int TPR, int ROWS>
__host__ __device__ constexpr int tile_min_blocks() {
  return (sizeof(V) == 8 && S <= 16) ? (ROWS < MF_TILE ? 6 : (TPR > 1 ? 1024 / (MF_TILE * TPR) : 5)) : 1;
}
// Programmatic dependent launch (sm_90 and later): a kernel launched with
// programmatic stream serialisation may start while its predecessor in the
// stream is finishing; pdl_wait() blocks until the predecessor has completed
// and its writes are visible, pdl_trigger() lets the successor be scheduled.
// Both are no-ops for kernels launched without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename V, int S, bool FWD, bool CG, int TPR, int ROWS>
__device__ __forceinline__ void sweep_tile(const int4 tile, const int* __restrict__ kk, const int* __restrict__ ff,
                                           const int64_t* __restrict__ rowoff, const int64_t* __restrict__ Moff,
                                           const V* __restrict__ M, const int* __restrict__ rows,
                                           const int64_t* __restrict__ cptr, const int* __restrict__ cidx,
                                           const int64_t* __restrict__ Doff, const V* __restrict__ Dinv, V* Xsub,
                                           V* Wout, V* P, int s, unsigned char* smem_raw) {
  static_assert(S % TPR == 0, "columns split evenly over the threads of a row");
  static_assert(ROWS <= MF_TILE, "a tile computes at most MF_TILE output rows");
  constexpr int CPT = S / TPR;  // columns per thread
  V(*bs)[S] = reinterpret_cast<V(*)[S]>(smem_raw);  // [MF_TK][S]
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
  const int row = tid / TPR, cb = (tid % TPR) * CPT;  // output row of the tile, first column
  const int lmax = max(0, kstop - kbeg);
  const int rr = r0 + row;
  const bool act = rr < nout;
  const V* mcol = Mt + (act ? rr : 0) + (int64_t)kbeg * ld;
  // the first factor columns are read while the input rows are staged
  V m0[MF_UNROLL];
#pragma unroll
  for (int u = 0; u < MF_UNROLL; ++u)
    m0[u] = (act && u < lmax) ? __ldg(mcol + (int64_t)u * ld) : mk2((decltype(V::x))0, (decltype(V::x))0);
  // everything above reads set-up data only; the input rows come from the previous launches
  pdl_wait();
  for (int l = row; l < lmax; l += ROWS) {
    const int64_t R = ro + kbeg + l;
    const int local = kbeg + l;
    V v[CPT];
    const V* src = (FWD || local >= k) ? Xsub + (int64_t)rows[R] * s : Wout + R * s;
#pragma unroll
    for (int q = 0; q < CPT; ++q)
      v[q] = cb + q < s ? ldv<CG>(src + cb + q) : mk2((decltype(V::x))0, (decltype(V::x))0);
    if (FWD) {
      const int64_t pe = cptr[R + 1];
      for (int64_t p = cptr[R]; p < pe; ++p) {
        const V* w = Wout + (int64_t)cidx[p] * s;
#pragma unroll
        for (int q = 0; q < CPT; ++q)
          if (cb + q < s) v[q] = c_add(v[q], ldv<CG>(w + cb + q));
      }
    }
#pragma unroll
    for (int q = 0; q < CPT; ++q) bs[l][cb + q] = v[q];
  }
  __syncthreads();
  V acc[CPT];
#pragma unroll
  for (int q = 0; q < CPT; ++q) acc[q] = mk2((decltype(V::x))0, (decltype(V::x))0);
  if (act) {
    // software pipeline: the next MF_UNROLL factor columns are in flight while the current ones are used
    int j = 0;
    while (j < lmax) {
      const int jn = j + MF_UNROLL;
      V m1[MF_UNROLL];
#pragma unroll
      for (int u = 0; u < MF_UNROLL; ++u)
        m1[u] = jn + u < lmax ? __ldg(mcol + (int64_t)(jn + u) * ld) : mk2((decltype(V::x))0, (decltype(V::x))0);
#pragma unroll
      for (int u = 0; u < MF_UNROLL; ++u)
        if (j + u < lmax)
#pragma unroll
          for (int q = 0; q < CPT; ++q) acc[q] = c_fma(m0[u], bs[j + u][cb + q], acc[q]);
#pragma unroll
      for (int u = 0; u < MF_UNROLL; ++u) m0[u] = m1[u];
      j = jn;
    }
  }
  if (slot >= 0) {
    V* out = P + ((int64_t)slot * MF_TILE + row) * s;
#pragma unroll
    for (int q = 0; q < CPT; ++q)
      if (cb + q < s) out[cb + q] = acc[q];
    return;
  }
  if (!act) return;
  const int64_t Rg = ro + rr;
  if (FWD) {
    if (rr < k) {
      const V di = Dinv[Doff[t] + rr];
#pragma unroll
      for (int q = 0; q < CPT; ++q)
        if (cb + q < s) Wout[Rg * s + cb + q] = c_mul(acc[q], di);
    } else {
      // parent update: the children's update vectors landing on this row,
      // one contiguous row of s values per contribution
      const int64_t pe = cptr[Rg + 1];
      for (int64_t p = cptr[Rg]; p < pe; ++p) {
        const V* w = Wout + (int64_t)cidx[p] * s;
#pragma unroll
        for (int q = 0; q < CPT; ++q)
          if (cb + q < s) acc[q] = c_add(acc[q], ldv<CG>(w + cb + q));
      }
#pragma unroll
      for (int q = 0; q < CPT; ++q)
        if (cb + q < s) Wout[Rg * s + cb + q] = acc[q];
    }
  } else {
    V* xo = Xsub + (int64_t)rows[Rg] * s;
#pragma unroll
    for (int q = 0; q < CPT; ++q)
      if (cb + q < s) xo[cb + q] = acc[q];
  }
}

template <typename V, int S, bool FWD, int TPR, int ROWS>
__global__ void __launch_bounds__(ROWS * TPR, tile_min_blocks<V, S, TPR, ROWS>()) k_mf_tile(const int4* __restrict__ tiles, const int* __restrict__ kk,
                                                     const int* __restrict__ ff, const int64_t* __restrict__ rowoff,
                                                     const int64_t* __restrict__ Moff, const V* __restrict__ M,
                                                     const int* __restrict__ rows, const int64_t* __restrict__ cptr,
                                                     const int* __restrict__ cidx, const int64_t* __restrict__ Doff,
                                                     const V* __restrict__ Dinv, V* __restrict__ Xsub,
                                                     V* __restrict__ Wout, V* __restrict__ P, int s) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pdl_trigger();
  sweep_tile<V, S, FWD, false, TPR, ROWS>(tiles[blockIdx.x], kk, ff, rowoff, Moff, M, rows, cptr, cidx, Doff, Dinv, Xsub, Wout,
                               P, s, smem_raw);
}

// Epilogue of a split row block (rb = front, first row, tiles, first slot):
// sum its partial tiles in slot order, then
//   forward : rows r < k -> y = t / D (kept in Wout for the backward sweep);
//             rows r >= k -> parent update c_U + t (Wout), c_U = the children's
//             update vectors landing on the row
//   backward: x at the pivot rows of the sub-vector
// (i, c) = (row of the block, column); CG: partials and update vectors
// written by other CTAs of the same launch are read through L2
template <typename V, bool FWD, bool CG>
__device__ __forceinline__ void rb_epilogue(const int4 rb, int i, int c, const int* __restrict__ kk,
                                            const int* __restrict__ ff, const int64_t* __restrict__ rowoff,
                                            const int64_t* __restrict__ Doff, const int* __restrict__ rows,
                                            const int64_t* __restrict__ cptr, const int* __restrict__ cidx,
                                            const V* __restrict__ Dinv, V* Wout, const V* P, V* Xsub, int s) {
  const int t = rb.x, r = rb.y + i;
  const int k = kk[t];
  if (r >= (FWD ? ff[t] : k)) return;
  V acc = mk2((decltype(V::x))0, (decltype(V::x))0);
  for (int q = 0; q < rb.z; ++q) acc = c_add(acc, ldv<CG>(P + ((int64_t)(rb.w + q) * MF_TILE + i) * s + c));
  const int64_t R = rowoff[t] + r;
  if (FWD) {
    if (r < k) {
      Wout[R * s + c] = c_mul(acc, Dinv[Doff[t] + r]);
    } else {
      for (int64_t p = cptr[R]; p < cptr[R + 1]; ++p) acc = c_add(acc, ldv<CG>(Wout + (int64_t)cidx[p] * s + c));
      Wout[R * s + c] = acc;
    }
  } else {
    Xsub[(int64_t)rows[R] * s + c] = acc;
  }
}

// Row-block epilogues of one level, one thread per (row, column).
template <typename V, bool FWD>
__global__ void k_mf_reduce(const int4* __restrict__ rblocks, int nrb, const int* __restrict__ kk,
                            const int* __restrict__ ff, const int64_t* __restrict__ rowoff,
                            const int64_t* __restrict__ Doff, const int* __restrict__ rows,
                            const int64_t* __restrict__ cptr, const int* __restrict__ cidx,
                            const V* __restrict__ Dinv, V* __restrict__ Wout, const V* __restrict__ P,
                            V* __restrict__ Xsub, int s) {
  pdl_trigger();
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t per = (int64_t)MF_TILE * s;
  if (g >= nrb * per) return;
  const int i = (int)((g % per) / s), c = (int)(g % s);
  pdl_wait();
  rb_epilogue<V, FWD, false>(rblocks[g / per], i, c, kk, ff, rowoff, Doff, rows, cptr, cidx, Dinv, Wout, P, Xsub, s);
}

// ---------------------------------------------------------------------------
// Persistent sweeps: one launch per sweep direction over every level.
//
// Resident CTAs take the tiles in level order through a ticket counter (the
// forward sweep from the leaves up, the backward sweep from the roots down).
// Before its tile, a CTA waits until the front's inputs are final: forward,
// every child front with rows has finished (its parent-update rows written);
// backward, the nearest ancestor with pivots has finished (so all the
// ancestors' pivots are final in the sub-vector; `parent` is that ancestor
// in the backward launch). A split row block's partial tiles count themselves in; the
// last one sums the partials in slot order (so the result does not depend
// on which tile comes last) and applies the epilogue. A front has finished
// when all its row blocks have, and then (forward) it counts itself into its
// parent. Every dependency has a smaller ticket, and a ticket is only taken
// by a running CTA, so the smallest unfinished ticket can always proceed.
// Waits are bounded by the global timer; a timeout sets *err and the CTA
// stops taking tiles (the sweep's result is then invalid and reported).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t sw_clock_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ int sw_load(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
// wait until *p >= target; false after about two seconds
__device__ __forceinline__ bool sw_wait(const int* p, int target) {
  if (sw_load(p) >= target) return true;
  const uint64_t t0 = sw_clock_ns();
  while (sw_load(p) < target) {
    __nanosleep(200);
    if (sw_clock_ns() - t0 > 2000000000ull) return false;
  }
  return true;
}

template <typename V, int S, bool FWD>
__global__ void __launch_bounds__(MF_TILE) k_mf_sweep(
    const int4* __restrict__ tiles, int ntiles, const int* __restrict__ slot_rb, const int4* __restrict__ rblocks,
    const int* __restrict__ front_nrb, const int* __restrict__ parent, const int* __restrict__ nchild,
    int* __restrict__ cnt, int nrb_total, int nfronts, int* __restrict__ err, const int* __restrict__ kk,
    const int* __restrict__ ff, const int64_t* __restrict__ rowoff, const int64_t* __restrict__ Moff,
    const V* __restrict__ M, const int* __restrict__ rows, const int64_t* __restrict__ cptr,
    const int* __restrict__ cidx, const int64_t* __restrict__ Doff, const V* __restrict__ Dinv, V* Xsub, V* Wout,
    V* P, int s) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_tile, s_flag;
  int* ticket = cnt;
  int* rb_cnt = cnt + 1;
  int* front_done = rb_cnt + nrb_total;
  int* child_ready = front_done + nfronts;
  const int tid = threadIdx.x;
  while (true) {
    if (tid == 0) {
      int tk = atomicAdd(ticket, 1);
      const int4 tl = tk < ntiles ? tiles[tk] : make_int4(0, 0, 0, 0);
      bool ok = true;
      if (tk < ntiles) {
        const int g = tl.x;
        if (FWD) {
          ok = sw_wait(child_ready + g, nchild[g]);
        } else if (parent[g] >= 0) {
          ok = sw_wait(front_done + parent[g], front_nrb[parent[g]]);
        }
        if (!ok) {
          atomicExch(err, 1);
          tk = ntiles;
        }
      }
      s_tile = tk;
    }
    __syncthreads();
    const int tk = s_tile;
    if (tk >= ntiles) break;
    const int4 tile = tiles[tk];
    sweep_tile<V, S, FWD, true, 1, MF_TILE>(tile, kk, ff, rowoff, Moff, M, rows, cptr, cidx, Doff, Dinv, Xsub, Wout, P, s,
                                smem_raw);
    __syncthreads();  // every write of the tile is issued
    const int g = tile.x;
    if (tid == 0) {
      int fin = 1;  // the tile finished its row block
      if (tile.w >= 0) {
        __threadfence();
        const int rb = slot_rb[tile.w];
        fin = atomicAdd(rb_cnt + rb, 1) == rblocks[rb].z - 1 ? 2 : 0;  // 2: last partial, sum the row block
        if (fin == 2) __threadfence();
        s_flag = fin == 2 ? rb : -1;
      } else {
        s_flag = -1;
      }
      if (fin == 1) {
        __threadfence();
        if (atomicAdd(front_done + g, 1) == front_nrb[g] - 1 && FWD && parent[g] >= 0) {
          __threadfence();
          atomicAdd(child_ready + parent[g], 1);
        }
      }
    }
    __syncthreads();
    const int rbl = s_flag;
    if (rbl >= 0) {
      const int4 rb = rblocks[rbl];
      for (int e = tid; e < MF_TILE * s; e += MF_TILE)
        rb_epilogue<V, FWD, true>(rb, e / s, e % s, kk, ff, rowoff, Doff, rows, cptr, cidx, Dinv, Wout, P, Xsub,
                                  s);
      __syncthreads();
      if (tid == 0) {
        __threadfence();
        if (atomicAdd(front_done + g, 1) == front_nrb[g] - 1 && FWD && parent[g] >= 0) {
          __threadfence();
          atomicAdd(child_ready + parent[g], 1);
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Tensor-core tiles (complex FP32 form): the same tile product on tcgen05,
// with FP32 accuracy from a three-term TF32 split (Markidis et al. 2018:
// a = a_hi + a_lo with a_hi = a rounded to TF32, a_lo = a - a_hi also in
// TF32; a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi, the dropped a_lo b_lo being
// ~2^-22 relative).
//
// The tile's factor block is packed once, after the factorisation, as
// 16-column chunks; each chunk holds a real and an imaginary plane of
// nr8 = roundup(rows, 8) rows x 16 reduction indices in FP32, in the
// K-major layout of 8-row x 16-byte core matrices (a row group's 4 core
// matrices are adjacent, row groups 512 bytes apart), reduction indices past
// the tile's end zero. A chunk is two contiguous copies (cp.async.bulk) into
// a ring of shared-memory stages; once it has landed, the CTA truncates it
// in place to its TF32 high part and writes the low part beside it. The input
// rows are staged once per tile as N x 128 operands, N = 2S, in high and low
// parts: B1 = [Re b | Im b] and B2 = [-Im b | Re b], so that
//   D = Re(M) B1^T + Im(M) B2^T = [Re(M b) | Im(M b)]
// accumulates in TMEM (128 lanes = output rows, N columns, FP32). Thread 0
// issues the MMAs (M = 128, N = 2S, K = 8 per instruction, 6 per 8 reduction
// indices) and commits them to the ring's barriers. Every wait is bounded by
// the global timer; a timeout sets *err, skips the epilogue, and the CTA
// waits (bounded again) for its copies in flight and its MMAs before it
// frees its TMEM and exits. Rows past the tile's end hold stale shared
// memory; their outputs are never written.
// ---------------------------------------------------------------------------
constexpr int TC_PLANE = 8192;              // one plane of a 128-row chunk in shared memory
constexpr int TC_STAGE = 2 * TC_PLANE;      // a chunk (real + imaginary plane)
constexpr int TC_SBO_A = 4 * 128;           // row-group stride of a 16-column chunk
constexpr int TC_SBO_B = (MF_TK / 4) * 128; // row-group stride of an N x 128 operand

__device__ __forceinline__ uint32_t tc_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
// shared-memory matrix descriptor: no swizzle, K-major, descriptor version 1
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}
__device__ __forceinline__ uint64_t tc_clock_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// wait for phase `parity` of an mbarrier, giving up after about half a second
__device__ __forceinline__ bool tc_wait(uint32_t bar, uint32_t parity) {
  uint32_t done = 0;
  const uint64_t t0 = tc_clock_ns();
  while (!done) {
    asm volatile(
        "{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (!done && tc_clock_ns() - t0 > 500000000ull) return false;
  }
  return true;
}
// TF32 value of x by truncation of the 13 low mantissa bits: the high part
// of the split, exactly representable in TF32, with x - hi exact in FP32
__device__ __forceinline__ float tc_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }
// byte offset of element (row, col) in a K-major core-matrix tile whose row
// groups are sbo bytes apart
__device__ __forceinline__ int tc_off(int row, int col, int sbo) {
  return (row >> 3) * sbo + (col >> 2) * 128 + (row & 7) * 16 + (col & 3) * 4;
}

// tile geometry shared by the packer and the kernel
struct TcGeom {
  int t, r0, slot, f, k, nout, ld, kbeg, kstop, nr, nr8, nk, nch;
};
template <bool FWD>
__device__ __forceinline__ TcGeom tc_geom(int4 tile, const int* kk, const int* ff) {
  TcGeom g;
  g.t = tile.x;
  g.r0 = tile.y;
  g.slot = tile.w;
  g.f = ff[g.t];
  g.k = kk[g.t];
  g.nout = FWD ? g.f : g.k;
  g.ld = FWD ? g.f : g.k;
  const int kend = FWD ? ((g.r0 < g.k) ? min(g.k, g.r0 + MF_TILE) : g.k) : g.f;
  g.kbeg = FWD ? tile.z : max(tile.z, g.r0);
  g.kstop = min(kend, tile.z + MF_TK);
  g.nr = min(MF_TILE, g.nout - g.r0);
  g.nr8 = (g.nr + 7) & ~7;
  g.nk = g.kstop - g.kbeg;
  g.nch = (g.nk + 15) / 16;
  return g;
}

// Pack the factor blocks of the tensor-core tiles (after k_mf_inverse), FP32.
template <bool FWD>
__global__ void k_tc_pack(const int4* __restrict__ tiles, const int64_t* __restrict__ off, const int* __restrict__ kk,
                          const int* __restrict__ ff, const int64_t* __restrict__ Moff, const float2* __restrict__ M,
                          unsigned char* __restrict__ TC) {
  const TcGeom g = tc_geom<FWD>(tiles[blockIdx.x], kk, ff);
  const float2* Mt = M + Moff[g.t];
  unsigned char* base = TC + off[blockIdx.x];
  const int plane = g.nr8 * 64;
  const int64_t total = (int64_t)g.nch * 16 * g.nr8;
  for (int64_t i = threadIdx.x; i < total; i += blockDim.x) {
    const int m = (int)(i % g.nr8);
    const int kc = (int)((i / g.nr8) % 16);
    const int q = (int)(i / ((int64_t)g.nr8 * 16));
    const int col = g.kbeg + q * 16 + kc;
    float2 v = make_float2(0.f, 0.f);
    if (m < g.nr && col < g.kstop) v = Mt[(g.r0 + m) + (int64_t)col * g.ld];
    unsigned char* ch = base + (int64_t)q * 2 * plane;
    const int o = tc_off(m, kc, TC_SBO_A);
    *reinterpret_cast<float*>(ch + o) = v.x;
    *reinterpret_cast<float*>(ch + plane + o) = v.y;
  }
}

static void tc_pack_all(DevMF& mf, cudaStream_t st) {
  if (mf.ftc_n)
    { k_tc_pack<true><<<(unsigned)mf.ftc_n, 256, 0, st>>>(mf.ftiles_tc, mf.ftc_off, mf.k, mf.f, mf.Moff,
                                                         (const float2*)mf.M, mf.TC); count_launch(); }
  if (mf.btc_n)
    { k_tc_pack<false><<<(unsigned)mf.btc_n, 256, 0, st>>>(mf.btiles_tc, mf.btc_off, mf.k, mf.f, mf.Moff,
                                                          (const float2*)mf.MT, mf.TC); count_launch(); }
}

// shared memory of the tensor-core tile (96 KB, two CTAs per SM): the input
// operand B = [Re b | Im b] (N x 128) in high and low parts, a ring of
// TC_NRAW raw factor chunks and one working chunk (high part | low part)
// that the MMAs read
constexpr int TC_NRAW = 2;
template <int S>
static constexpr size_t tc_smem_bytes() {
  return 2 * (size_t)(2 * S) * MF_TK * 4 + (size_t)TC_NRAW * TC_STAGE + 2 * (size_t)TC_STAGE;
}

__device__ __forceinline__ void tc_mma(uint32_t taddr, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(taddr),
      "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

// Complex product on real MMAs: D1 = Re(M) B and D2 = Im(M) B accumulate in
// two TMEM blocks of N = 2S columns; the epilogue forms
//   Re(M b) = D1[:, 0:S] - D2[:, S:2S],  Im(M b) = D1[:, S:2S] + D2[:, 0:S].
// Chunk pipeline (128 threads): thread 0 keeps TC_NRAW raw chunks in flight;
// every thread waits for chunk q and for the MMAs of chunk q - 1 (which read
// the working buffer), splits the raw chunk into its high and low parts in
// the working buffer, and after a CTA barrier (which also frees the raw stage
// for the copy of chunk q + TC_NRAW) thread 0 issues the six MMAs per 8
// reduction indices and commits them to the working buffer's barrier.
template <int S, bool FWD>
__global__ void __launch_bounds__(MF_TILE) k_mf_tile_tc(
    const int4* __restrict__ tiles, const int64_t* __restrict__ tcoff, const unsigned char* __restrict__ TC,
    const int* __restrict__ kk, const int* __restrict__ ff, const int64_t* __restrict__ rowoff,
    const int* __restrict__ rows, const int64_t* __restrict__ cptr, const int* __restrict__ cidx,
    const int64_t* __restrict__ Doff, const float2* __restrict__ Dinv, float2* __restrict__ Xsub,
    float2* __restrict__ Wout, float2* __restrict__ P, int s, int* __restrict__ err) {
  static_assert(S == 16, "tensor-core tiles are built for blocks of 16 columns");
  constexpr int N = 2 * S;
  constexpr int BT = N * MF_TK * 4;
  constexpr uint32_t NCOL = 2 * N;  // D1 and D2
  extern __shared__ __align__(1024) unsigned char smem_tc[];
  unsigned char* sBh = smem_tc;
  unsigned char* sBl = smem_tc + BT;
  unsigned char* raw = smem_tc + 2 * BT;            // TC_NRAW x TC_STAGE
  unsigned char* wh = raw + TC_NRAW * TC_STAGE;     // working chunk, high part (real plane, imaginary plane)
  unsigned char* wl = wh + TC_STAGE;                // low part
  __shared__ __align__(8) uint64_t full[TC_NRAW], freeb, done;
  __shared__ uint32_t tslot;
  __shared__ int s_ok;
  const int tid = threadIdx.x, warp = tid >> 5;
  const TcGeom g = tc_geom<FWD>(tiles[blockIdx.x], kk, ff);
  const unsigned char* src = TC + tcoff[blockIdx.x];
  const uint32_t plane = (uint32_t)g.nr8 * 64, cbytes = 2 * plane;
  if (tid == 0) {
    for (int i = 0; i < TC_NRAW; ++i) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem(&full[i])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem(&freeb)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem(&done)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_ok = 1;
  }
  __syncthreads();
  int issued = 0;  // thread 0: chunks whose copies were issued
  auto load_chunk = [&](int q) {  // thread 0: chunk q into raw stage q % TC_NRAW
    const uint32_t bar = tc_smem(&full[q % TC_NRAW]);
    const uint32_t dst = tc_smem(raw + (q % TC_NRAW) * TC_STAGE);
    const unsigned char* c = src + (int64_t)q * cbytes;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(cbytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(c), "r"(plane), "r"(bar)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     dst + TC_PLANE),
                 "l"(c + plane), "r"(plane), "r"(bar)
                 : "memory");
    issued = q + 1;
  };
  if (tid == 0)
    for (int q = 0; q < min(TC_NRAW, g.nch); ++q) load_chunk(q);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_smem(&tslot)),
                 "r"(NCOL));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  // input rows -> high and low parts of B = [Re | Im], zero past the tile's reduction end
  const int64_t ro = rowoff[g.t];
  if (tid < g.nch * 16) {
    const int l = tid;
    float2 v[S];
#pragma unroll
    for (int c = 0; c < S; ++c) v[c] = make_float2(0.f, 0.f);
    if (l < g.nk) {
      const int64_t R = ro + g.kbeg + l;
      const int local = g.kbeg + l;
      const float2* xs = (FWD || local >= g.k) ? Xsub + (int64_t)rows[R] * s : Wout + R * s;
#pragma unroll
      for (int c = 0; c < S; ++c)
        if (c < s) v[c] = xs[c];
      if (FWD) {
        const int64_t pe = cptr[R + 1];
        for (int64_t p = cptr[R]; p < pe; ++p) {
          const float2* w = Wout + (int64_t)cidx[p] * s;
#pragma unroll
          for (int c = 0; c < S; ++c)
            if (c < s) v[c] = make_float2(v[c].x + w[c].x, v[c].y + w[c].y);
        }
      }
    }
#pragma unroll
    for (int c = 0; c < S; ++c) {
      const float reh = tc_hi(v[c].x), imh = tc_hi(v[c].y);
      const int o0 = tc_off(c, l, TC_SBO_B), o1 = tc_off(S + c, l, TC_SBO_B);
      *reinterpret_cast<float*>(sBh + o0) = reh;
      *reinterpret_cast<float*>(sBh + o1) = imh;
      *reinterpret_cast<float*>(sBl + o0) = tc_hi(v[c].x - reh);
      *reinterpret_cast<float*>(sBl + o1) = tc_hi(v[c].y - imh);
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // B: generic writes, async-proxy reads
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t taddr = tslot;
  // kind::tf32: D f32, A and B tf32, both K-major, N = 2S, M = 128
  constexpr uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
  const int per_plane = g.nr8 * 16;  // floats of one plane of a chunk
  for (int q = 0; q < g.nch; ++q) {
    const int r = q % TC_NRAW;
    bool okq = tc_wait(tc_smem(&full[r]), (q / TC_NRAW) & 1);
    if (okq && q >= 1) okq = tc_wait(tc_smem(&freeb), (q - 1) & 1);  // MMAs of chunk q - 1 done
    if (!okq) s_ok = 0;
    if (okq)
      for (int i = tid; i < 2 * per_plane; i += MF_TILE) {
        const int pl = i >= per_plane, e = i - pl * per_plane;
        const float x = *(reinterpret_cast<const float*>(raw + r * TC_STAGE + pl * TC_PLANE) + e);
        const float h = tc_hi(x);
        *(reinterpret_cast<float*>(wh + pl * TC_PLANE) + e) = h;
        *(reinterpret_cast<float*>(wl + pl * TC_PLANE) + e) = tc_hi(x - h);
      }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (!s_ok) break;
    if (tid == 0) {
      // every thread has read raw stage r: it takes the copy of chunk q + TC_NRAW
      if (q + TC_NRAW < g.nch) load_chunk(q + TC_NRAW);
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t aReH = tc_smem(wh), aImH = aReH + TC_PLANE, aReL = tc_smem(wl), aImL = aReL + TC_PLANE;
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const uint32_t kb = (uint32_t)(q * 4 + 2 * j) * 128;
        const uint64_t dReH = tc_desc(aReH + j * 256, 128, TC_SBO_A), dImH = tc_desc(aImH + j * 256, 128, TC_SBO_A);
        const uint64_t dReL = tc_desc(aReL + j * 256, 128, TC_SBO_A), dImL = tc_desc(aImL + j * 256, 128, TC_SBO_A);
        const uint64_t dbh = tc_desc(tc_smem(sBh) + kb, 128, TC_SBO_B), dbl = tc_desc(tc_smem(sBl) + kb, 128, TC_SBO_B);
        const uint32_t first = (q > 0 || j > 0) ? 1u : 0u;
        tc_mma(taddr, dReH, dbh, idesc, first);
        tc_mma(taddr, dReH, dbl, idesc, 1u);
        tc_mma(taddr, dReL, dbh, idesc, 1u);
        tc_mma(taddr + N, dImH, dbh, idesc, first);
        tc_mma(taddr + N, dImH, dbl, idesc, 1u);
        tc_mma(taddr + N, dImL, dbh, idesc, 1u);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       tc_smem(&freeb))
                   : "memory");
    }
  }
  // `done` arrives once every MMA issued so far has completed
  if (tid == 0)
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(tc_smem(&done))
                 : "memory");
  const bool fin = tc_wait(tc_smem(&done), 0);
  if (!fin) s_ok = 0;
  __syncthreads();
  const bool ok = s_ok != 0;
  if (!ok && tid == 0) {
    atomicExch(err, 1);
    // copies still in flight must land before the CTA's shared memory is released (bounded waits;
    // a stage whose chunk was already consumed passes at once)
    for (int q = max(0, issued - TC_NRAW); q < issued; ++q) tc_wait(tc_smem(&full[q % TC_NRAW]), (q / TC_NRAW) & 1);
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok) {
    const int m = tid;  // TMEM lane = output row of the tile
    const bool act = m < g.nr;
    const int rr = g.r0 + m;
    const int64_t Rg = ro + rr;
    const uint32_t lane_base = taddr + ((uint32_t)(warp * 32) << 16);
    uint32_t d1r[16], d1i[16], d2r[16], d2i[16];
#define HZ_TMEM_LD16(dst, col)                                                                                      \
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];" \
               : "=r"(dst[0]), "=r"(dst[1]), "=r"(dst[2]), "=r"(dst[3]), "=r"(dst[4]), "=r"(dst[5]), "=r"(dst[6]),     \
                 "=r"(dst[7]), "=r"(dst[8]), "=r"(dst[9]), "=r"(dst[10]), "=r"(dst[11]), "=r"(dst[12]), "=r"(dst[13]), \
                 "=r"(dst[14]), "=r"(dst[15])                                                                       \
               : "r"(lane_base + (col)))
    HZ_TMEM_LD16(d1r, 0);
    HZ_TMEM_LD16(d1i, S);
    HZ_TMEM_LD16(d2r, N);
    HZ_TMEM_LD16(d2i, N + S);
#undef HZ_TMEM_LD16
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    if (act) {
#pragma unroll
      for (int c = 0; c < S; ++c) {
        if (c >= s) break;
        // Re(M b) = Re M Re b - Im M Im b,  Im(M b) = Re M Im b + Im M Re b
        float2 a = make_float2(__uint_as_float(d1r[c]) - __uint_as_float(d2i[c]),
                               __uint_as_float(d1i[c]) + __uint_as_float(d2r[c]));
        if (g.slot >= 0) {
          P[((int64_t)g.slot * MF_TILE + m) * s + c] = a;
        } else if (FWD) {
          if (rr < g.k) {
            Wout[Rg * s + c] = c_mul(a, Dinv[Doff[g.t] + rr]);
          } else {
            const int64_t pe = cptr[Rg + 1];
            for (int64_t p = cptr[Rg]; p < pe; ++p) a = c_add(a, Wout[(int64_t)cidx[p] * s + c]);
            Wout[Rg * s + c] = a;
          }
        } else {
          Xsub[(int64_t)rows[Rg] * s + c] = a;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(NCOL));
}

static inline unsigned blocks_for(int64_t work, int b) { return (unsigned)((work + b - 1) / b); }

template <typename V, int S>
static constexpr bool tc_width() {
  return std::is_same<V, float2>::value && S == 16;
}

template <typename V, int S, bool FWD>
static void tc_launch(DevMF& mf, int l, V* Xsub, int s, cudaStream_t st) {
  if constexpr (tc_width<V, S>()) {
    const int* ptr = FWD ? mf.ftc_ptr_h : mf.btc_ptr_h;
    const int tb = ptr[l], te = ptr[l + 1];
    if (te > tb) {
      k_mf_tile_tc<S, FWD><<<te - tb, MF_TILE, tc_smem_bytes<S>(), st>>>(
          (FWD ? mf.ftiles_tc : mf.btiles_tc) + tb, (FWD ? mf.ftc_off : mf.btc_off) + tb, mf.TC, mf.k, mf.f,
          mf.rowoff, mf.rows, mf.cptr, mf.cidx, mf.Doff, (const float2*)mf.Dinv, (float2*)Xsub, (float2*)mf.Wout,
          (float2*)mf.P, s, mf.tc_err);
      count_launch();
    }
  }
}

// resident CTAs of k_mf_sweep<V, S, *> (set with the kernels' attributes, outside any capture)
static int g_sweep_grid[2][7];
template <typename V, int S>
static int& sweep_grid() {
  constexpr int vi = sizeof(V) == 8 ? 0 : 1;
  constexpr int si = S == 1 ? 0 : S == 2 ? 1 : S == 4 ? 2 : S == 8 ? 3 : S == 16 ? 4 : S == 32 ? 5 : 6;
  return g_sweep_grid[vi][si];
}

template <typename V, int S>
static void sweep_persistent(DevMF& mf, V* Xsub, int s, cudaStream_t st) {
  const size_t shm = tile_smem_bytes<V, S>();
  const int grid = sweep_grid<V, S>();
  V* Wout = (V*)mf.Wout;
  V* P = (V*)mf.P;
  const V* Dv = (const V*)mf.Dinv;
  cudaMemsetAsync(mf.cnt, 0, (size_t)mf.cnt_n * sizeof(int), st);
  if (mf.pt_nf > 0)
    { k_mf_sweep<V, S, true><<<std::min(grid, mf.pt_nf), MF_TILE, shm, st>>>(
        mf.ptf, mf.pt_nf, mf.slot_rb_f, mf.prb_f, mf.nrb_f, mf.parent, mf.nchild, mf.cnt, mf.prb_nf,
        (int)mf.nfronts, mf.sw_err, mf.k, mf.f, mf.rowoff, mf.Moff, (const V*)mf.M, mf.rows, mf.cptr, mf.cidx,
        mf.Doff, Dv, Xsub, Wout, P, s); count_launch(); }
  cudaMemsetAsync(mf.cnt, 0, (size_t)mf.cnt_n * sizeof(int), st);
  if (mf.pt_nb > 0)
    { k_mf_sweep<V, S, false><<<std::min(grid, mf.pt_nb), MF_TILE, shm, st>>>(
        mf.ptb, mf.pt_nb, mf.slot_rb_b, mf.prb_b, mf.nrb_b, mf.bdep, mf.nchild, mf.cnt, mf.prb_nb,
        (int)mf.nfronts, mf.sw_err, mf.k, mf.f, mf.rowoff, mf.Moff, (const V*)mf.MT, mf.rows, mf.cptr, mf.cidx,
        mf.Doff, Dv, Xsub, Wout, P, s); count_launch(); }
}

// Launch with programmatic stream serialisation when `pdl` (the sweep's
// tile and reduce launches: the next level's CTAs are scheduled while the
// previous launch drains and read their factor columns before pdl_wait()).
template <typename... P, typename... A>
static void launch_k(bool pdl, void (*k)(P...), unsigned grid, unsigned block, size_t shm, cudaStream_t st,
                     A&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = shm;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  cudaLaunchKernelEx(&cfg, k, std::forward<A>(args)...);
  count_launch();
}

// One level's SIMT tiles: several threads per output row when the level has
// few tiles (latency-bound); on long levels half-height tiles when every tile
// has at most MF_HALF output rows, else one thread per row.
template <typename V, int S, bool FWD>
static void launch_tiles(bool pdl, int ntiles, bool half, size_t shm, cudaStream_t st, const int4* tiles,
                         const DevMF& mf, const V* M, const V* Dv, V* Xsub, V* Wout, V* P, int s) {
  constexpr int TPR = tile_tpr<S>();
  constexpr int TPH = tile_tpr_half<S>();
  if (half && ntiles >= MF_SHORT_LEVEL)
    launch_k(pdl, k_mf_tile<V, S, FWD, TPH, MF_HALF>, ntiles, MF_HALF * TPH, shm, st, tiles, (const int*)mf.k,
             (const int*)mf.f, (const int64_t*)mf.rowoff, (const int64_t*)mf.Moff, M, (const int*)mf.rows,
             (const int64_t*)mf.cptr, (const int*)mf.cidx, (const int64_t*)mf.Doff, Dv, Xsub, Wout, P, s);
  else if (TPR > 1 && ntiles < MF_SHORT_LEVEL)
    launch_k(pdl, k_mf_tile<V, S, FWD, TPR, MF_TILE>, ntiles, MF_TILE * TPR, shm, st, tiles, (const int*)mf.k,
             (const int*)mf.f, (const int64_t*)mf.rowoff, (const int64_t*)mf.Moff, M, (const int*)mf.rows,
             (const int64_t*)mf.cptr, (const int*)mf.cidx, (const int64_t*)mf.Doff, Dv, Xsub, Wout, P, s);
  else
    launch_k(pdl, k_mf_tile<V, S, FWD, 1, MF_TILE>, ntiles, MF_TILE, shm, st, tiles, (const int*)mf.k, (const int*)mf.f,
             (const int64_t*)mf.rowoff, (const int64_t*)mf.Moff, M, (const int*)mf.rows, (const int64_t*)mf.cptr,
             (const int*)mf.cidx, (const int64_t*)mf.Doff, Dv, Xsub, Wout, P, s);
}

template <typename V, int S>
static void solve_impl(DevMF& mf, V* Xsub, int s, cudaStream_t st) {
  const size_t shm = tile_smem_bytes<V, S>();
  V* Wout = (V*)mf.Wout;
  V* P = (V*)mf.P;
  const V* M = (const V*)mf.M;
  const V* MT = (const V*)mf.MT;
  const V* Dv = (const V*)mf.Dinv;
  // with the tensor cores on, each level's tiles are split between the
  // tcgen05 kernel and the SIMT kernel (the tiles the SIMT kernel keeps are
  // the small ones); both write the same partial slots and epilogues
  const bool tc = tc_width<V, S>() && mf.tc;
  if (!tc && mf.persistent && sweep_grid<V, S>() > 0) {
    sweep_persistent<V, S>(mf, Xsub, s, st);
    return;
  }
  const int* fptr = tc ? mf.fs_ptr_h : mf.ftile_ptr_h;
  const int* bptr = tc ? mf.bs_ptr_h : mf.btile_ptr_h;
  const int4* ftl = tc ? mf.ftiles_s : mf.ftiles;
  const int4* btl = tc ? mf.btiles_s : mf.btiles;
  // tensor-core mode: a level's SIMT tiles run on the side stream, concurrently with its tcgen05 tiles
  // (they write disjoint outputs and partial slots); the level's reduce waits for both
  const bool fork = tc && mf.side;
  // programmatic dependent launches between the levels (not with the tensor-core fork/join)
  const bool pdl = !tc;
  auto fork_begin = [&]() {
    if (!fork) return st;
    cudaEventRecord(mf.ev_fork, st);
    cudaStreamWaitEvent(mf.side, mf.ev_fork, 0);
    return mf.side;
  };
  auto fork_end = [&]() {
    if (!fork) return;
    cudaEventRecord(mf.ev_join, mf.side);
    cudaStreamWaitEvent(st, mf.ev_join, 0);
  };
  for (int l = 0; l < mf.nlevels; ++l) {
    const int tb = fptr[l], te = fptr[l + 1];
    cudaStream_t ss = fork_begin();
    if (te > tb)
      launch_tiles<V, S, true>(pdl, te - tb, mf.fhalf_h[l] != 0, shm, ss, ftl + tb, mf, M, Dv, Xsub, Wout, P, s);
    if (tc) tc_launch<V, S, true>(mf, l, Xsub, s, st);
    fork_end();
    const int rb = mf.frb_ptr_h[l], re = mf.frb_ptr_h[l + 1];
    if (re > rb)
      launch_k(pdl, k_mf_reduce<V, true>, blocks_for((int64_t)(re - rb) * MF_TILE * s, 256), 256, 0, st,
               (const int4*)(mf.frb + rb), re - rb, (const int*)mf.k, (const int*)mf.f, (const int64_t*)mf.rowoff,
               (const int64_t*)mf.Doff, (const int*)mf.rows, (const int64_t*)mf.cptr, (const int*)mf.cidx, Dv, Wout,
               (const V*)P, Xsub, s);
  }
  for (int l = mf.nlevels - 1; l >= 0; --l) {
    const int tb = bptr[l], te = bptr[l + 1];
    cudaStream_t ss = fork_begin();
    if (te > tb)
      launch_tiles<V, S, false>(pdl, te - tb, mf.bhalf_h[l] != 0, shm, ss, btl + tb, mf, MT, Dv, Xsub, Wout, P, s);
    if (tc) tc_launch<V, S, false>(mf, l, Xsub, s, st);
    fork_end();
    const int rb = mf.brb_ptr_h[l], re = mf.brb_ptr_h[l + 1];
    if (re > rb)
      launch_k(pdl, k_mf_reduce<V, false>, blocks_for((int64_t)(re - rb) * MF_TILE * s, 256), 256, 0, st,
               (const int4*)(mf.brb + rb), re - rb, (const int*)mf.k, (const int*)mf.f, (const int64_t*)mf.rowoff,
               (const int64_t*)mf.Doff, (const int*)mf.rows, (const int64_t*)mf.cptr, (const int*)mf.cidx, Dv, Wout,
               (const V*)P, Xsub, s);
  }
}

// Opt the tile kernels into their dynamic shared memory once, outside any
// stream capture (called from the factorisation).
template <typename V, int S>
static void tile_attrs() {
  const int shm = (int)tile_smem_bytes<V, S>();
  cudaFuncSetAttribute(k_mf_tile<V, S, true, 1, MF_TILE>, cudaFuncAttributeMaxDynamicSharedMemorySize, shm);
  cudaFuncSetAttribute(k_mf_tile<V, S, false, 1, MF_TILE>, cudaFuncAttributeMaxDynamicSharedMemorySize, shm);
  cudaFuncSetAttribute(k_mf_tile<V, S, true, tile_tpr<S>(), MF_TILE>, cudaFuncAttributeMaxDynamicSharedMemorySize, shm);
  cudaFuncSetAttribute(k_mf_tile<V, S, false, tile_tpr<S>(), MF_TILE>, cudaFuncAttributeMaxDynamicSharedMemorySize, shm);
  cudaFuncSetAttribute(k_mf_tile<V, S, true, tile_tpr_half<S>(), MF_HALF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       shm);
  cudaFuncSetAttribute(k_mf_tile<V, S, false, tile_tpr_half<S>(), MF_HALF>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, shm);
  cudaFuncSetAttribute(k_mf_sweep<V, S, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, shm);
  cudaFuncSetAttribute(k_mf_sweep<V, S, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, shm);
  {
    // resident CTAs per SM of the persistent sweep (the smaller of the two directions) x SMs
    int dev = 0, sms = 0, a = 0, b = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_mf_sweep<V, S, true>, MF_TILE, shm);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_mf_sweep<V, S, false>, MF_TILE, shm);
    sweep_grid<V, S>() = std::max(0, std::min(a, b)) * sms;
    cudaGetLastError();
  }
  if constexpr (tc_width<V, S>()) {
    const int tshm = (int)tc_smem_bytes<S>();
    cudaFuncSetAttribute(k_mf_tile_tc<S, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, tshm);
    cudaFuncSetAttribute(k_mf_tile_tc<S, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, tshm);
  }
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
