// Double-float ("float-float") arithmetic for the FP64 parts of the mixed
// form: the outer product with A (Eq. eq1) and the coarse product with E.
//
// GB300 issues 64 FP32 fused multiply-adds for every FP64 one, so an FP64
// product with A is bound by the FP64 pipe at any block width. Here a double
// is carried as an unevaluated sum hi + lo of two FP32 numbers (|lo| below
// one ulp of hi, about 47-48 significant bits), after Dekker (1971): the product
// of two such numbers keeps hi*hi exactly through one fused multiply-add
// (TwoProduct) plus the two cross terms, and every partial sum is added with
// Knuth's error-free TwoSum; the rounding errors of the low parts are summed
// in FP32. The relative error of a row sum of m terms is about m * 2^-48
// of sum |a_ij x_j| (FP64: m * 2^-53), far below what the residual test of
// FGMRES needs. All operations use the _rn intrinsics so that the compiler
// cannot contract a product and a sum into one FMA (which would break the
// error-free transformations). Magnitudes from about 2^-103 (1e-31) to 2^128
// keep the full precision; smaller ones are carried with FP32 precision, like
// the mixed form's FP32 local solves.
//
// Layouts: a complex FP64 block [n][s] double2 becomes [n][s] float4
// (re_hi, re_lo, im_hi, im_lo), 16 bytes per entry like the FP64 block; the
// real values of a split CSR matrix become float2 (hi, lo) per nonzero.
#include <cuda_runtime.h>

#include "df.cuh"
#include "kernels.cuh"

namespace hz {

namespace {
inline unsigned grid_for(int64_t work, int block) { return (unsigned)((work + block - 1) / block); }
}  // namespace

__global__ void k_to_df(const double2* __restrict__ X, float4* __restrict__ Y, int64_t count) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= count) return;
  const double2 x = X[g];
  const float2 r = df_split(x.x), i = df_split(x.y);
  Y[g] = make_float4(r.x, r.y, i.x, i.y);
}

// Y = (A_re + i A_im) X or Y = B - A X, X in double-float; one thread per
// (row, column), the s threads of a row share the index and value loads.
// With Ydf the product A X is written in double-float instead (renormalised).
__global__ void k_spmm_df(int64_t n, int s, const int64_t* __restrict__ rp_re, const int32_t* __restrict__ col_re,
                          const float2* __restrict__ val_re, const int64_t* __restrict__ rp_im,
                          const int32_t* __restrict__ col_im, const float2* __restrict__ val_im,
                          const float4* __restrict__ X, double2* __restrict__ Y, const double2* __restrict__ B,
                          int mode, float4* __restrict__ Ydf) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t r = g / s;
  const int c = (int)(g - r * s);
  if (r >= n) return;
  float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
#pragma unroll 4
  for (int64_t p = rp_re[r], pe = rp_re[r + 1]; p < pe; ++p) {
    const float2 a = val_re[p];
    const float4 x = X[(int64_t)col_re[p] * s + c];
    df_mac(rh, rl, a.x, a.y, x.x, x.y);
    df_mac(ih, il, a.x, a.y, x.z, x.w);
  }
#pragma unroll 4
  for (int64_t p = rp_im[r], pe = rp_im[r + 1]; p < pe; ++p) {
    const float2 b = val_im[p];
    const float4 x = X[(int64_t)col_im[p] * s + c];
    df_mac(rh, rl, -b.x, -b.y, x.z, x.w);  // re -= b im(x)
    df_mac(ih, il, b.x, b.y, x.x, x.y);    // im += b re(x)
  }
  if (Ydf) {
    df_norm(rh, rl);
    df_norm(ih, il);
    Ydf[g] = make_float4(rh, rl, ih, il);
    return;
  }
  const double ar = f2d(rh) + f2d(rl), ai = f2d(ih) + f2d(il);
  if (mode == 1) {
    const double2 b = B[g];
    Y[g] = make_double2(b.x - ar, b.y - ai);
  } else {
    Y[g] = make_double2(ar, ai);
  }
}

// Y = R X for a real CSR R (the coarse restriction Z^T and prolongation Z),
// X in double-float, Y in FP64
__global__ void k_spmm_real_df(int64_t n, int s, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                               const float2* __restrict__ val, const float4* __restrict__ X, double2* __restrict__ Y) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t r = g / s;
  const int c = (int)(g - r * s);
  if (r >= n) return;
  float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
#pragma unroll 4
  for (int64_t p = rp[r], pe = rp[r + 1]; p < pe; ++p) {
    const float2 a = val[p];
    const float4 x = X[(int64_t)col[p] * s + c];
    df_mac(rh, rl, a.x, a.y, x.x, x.y);
    df_mac(ih, il, a.x, a.y, x.z, x.w);
  }
  Y[g] = make_double2(f2d(rh) + f2d(rl), f2d(ih) + f2d(il));
}

void spmm_real_df(int64_t nrows, const int64_t* rp, const int32_t* col, const float2* val, const float4* X,
                  double2* Y, int s, cudaStream_t st) {
  const int64_t work = nrows * s;
  if (work == 0) return;
  { k_spmm_real_df<<<grid_for(work, 256), 256, 0, st>>>(nrows, s, rp, col, val, X, Y); count_launch(); }
}

void to_df(const double2* X, float4* Y, int64_t count, cudaStream_t st) {
  if (count) { k_to_df<<<grid_for(count, 256), 256, 0, st>>>(X, Y, count); count_launch(); }
}

void spmm_split_df(const DevSplitCsr& A, const float4* X, double2* Y, const double2* B, int s, int mode,
                   cudaStream_t st, float4* Ydf) {
  const int64_t work = A.n * s;
  if (work == 0) return;
  { k_spmm_df<<<grid_for(work, 256), 256, 0, st>>>(A.n, s, A.rp_re, A.col_re, A.val_re_df, A.rp_im, A.col_im,
                                                  A.val_im_df, X, Y, B, mode, Ydf); count_launch(); }
}

}  // namespace hz
