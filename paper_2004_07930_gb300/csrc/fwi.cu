// Full-waveform-inversion misfit and gradient kernels (adjoint-state method).
//
// The paper's solver is the forward engine of frequency-domain FWI
// (Sec. "Introduction"); it prints no gradient. With receivers sampled by the
// P3 interpolation P, chi = 1/2 sum_s |P u_s - d_s|^2, A u_s = F_s and, A
// being complex symmetric, the adjoint states A lambda_s = P^T conj(r_s),
// r_s = P u_s - d_s, the gradient with respect to the squared slowness m_e of
// element e is
//   g_e = -Re sum_s lambda_e^T (dA/dm_e) u_e,
//   dA/dm_e = -omega^2 M_e - (i omega / (2 sqrt(m_e))) sum_{Robin f of e} B_f,
// on the element's non-Dirichlet dofs, with M_e = |T| Mhat and
// B_f = |f| Bhat_c (Mhat, Bhat_c the geometry-free P3 tables).
// Blocks are node-major [n][s] like the solver's workspaces.
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace hz {

__constant__ double c_Mhat[20 * 20];
__constant__ double c_Bhat[4 * 20 * 20];

// r[q][k] = sum_i w[k][i] U[idx[k][i]][q] - d[q][k]; one thread per (k, q).
__global__ void k_fwi_residual(int nr, int s, const int* __restrict__ pidx, const double* __restrict__ pw,
                               const double2* __restrict__ U, const double2* __restrict__ d,
                               double2* __restrict__ r) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nr * s) return;
  const int k = t / s, q = t % s;
  double2 acc = make_double2(0.0, 0.0);
  for (int i = 0; i < 20; ++i) {
    const int j = pidx[k * 20 + i];
    if (j < 0) continue;
    const double w = pw[k * 20 + i];
    const double2 u = U[(int64_t)j * s + q];
    acc.x += w * u.x;
    acc.y += w * u.y;
  }
  const double2 dv = d ? d[(int64_t)q * nr + k] : make_double2(0.0, 0.0);
  r[(int64_t)q * nr + k] = make_double2(acc.x - dv.x, acc.y - dv.y);
}

// chi += 1/2 sum |r|^2 over m values; one block of 256 threads, fixed order.
__global__ void k_fwi_chi(int64_t m, const double2* __restrict__ r, double* __restrict__ chi) {
  __shared__ double sh[256];
  double a = 0.0;
  for (int64_t i = threadIdx.x; i < m; i += 256) a += r[i].x * r[i].x + r[i].y * r[i].y;
  sh[threadIdx.x] = a;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *chi += 0.5 * sh[0];
}

// B[dof][q] = sum over the receivers k in row dof of P^T of w conj(r[q][k]).
// Rows of P^T in CSR (tptr / tk / tw) over the touched dofs trow.
__global__ void k_fwi_adjoint_rhs(int nt, int s, int nr, const int* __restrict__ trow, const int* __restrict__ tptr,
                                  const int* __restrict__ tk, const double* __restrict__ tw,
                                  const double2* __restrict__ r, double2* __restrict__ B) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt * s) return;
  const int a = t / s, q = t % s;
  double2 acc = make_double2(0.0, 0.0);
  for (int p = tptr[a]; p < tptr[a + 1]; ++p) {
    const double2 v = r[(int64_t)q * nr + tk[p]];
    acc.x += tw[p] * v.x;
    acc.y -= tw[p] * v.y;
  }
  B[(int64_t)trow[a] * s + q] = acc;
}

// One thread per element; g[e] -= the contribution of the s columns of this block.
__global__ void k_fwi_gradient(int64_t ne, int s, const int* __restrict__ l2g, const double* __restrict__ vol,
                               const double* __restrict__ farea, const double* __restrict__ m, double omega,
                               const double2* __restrict__ U, const double2* __restrict__ L,
                               double* __restrict__ g) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= ne) return;
  int dof[20];
  for (int i = 0; i < 20; ++i) dof[i] = l2g[e * 20 + i];
  double fa[4];
  bool any_face = false;
  for (int c = 0; c < 4; ++c) {
    fa[c] = farea[e * 4 + c];
    any_face |= fa[c] != 0.0;
  }
  const double mass = -omega * omega * vol[e];
  const double rob = -omega / (2.0 * sqrt(m[e]));  // coefficient of i
  double acc = 0.0;
  for (int q = 0; q < s; ++q) {
    double2 u[20];
    for (int j = 0; j < 20; ++j) u[j] = dof[j] >= 0 ? U[(int64_t)dof[j] * s + q] : make_double2(0.0, 0.0);
    // tm = lambda^T Mhat u, tb = lambda^T (sum_c fa_c Bhat_c) u
    double2 tm = make_double2(0.0, 0.0), tb = make_double2(0.0, 0.0);
    for (int i = 0; i < 20; ++i) {
      if (dof[i] < 0) continue;
      const double2 l = L[(int64_t)dof[i] * s + q];
      double2 mu = make_double2(0.0, 0.0), bu = make_double2(0.0, 0.0);
      for (int j = 0; j < 20; ++j) {
        const double w = c_Mhat[i * 20 + j];
        mu.x += w * u[j].x;
        mu.y += w * u[j].y;
      }
      if (any_face)
        for (int j = 0; j < 20; ++j) {
          double bw = 0.0;
          for (int c = 0; c < 4; ++c) bw += fa[c] * c_Bhat[(c * 20 + i) * 20 + j];
          bu.x += bw * u[j].x;
          bu.y += bw * u[j].y;
        }
      tm.x += l.x * mu.x - l.y * mu.y;
      tb.y += l.x * bu.y + l.y * bu.x;
    }
    // Re(mass tm + i rob tb) = mass Re(tm) - rob Im(tb)
    acc += mass * tm.x - rob * tb.y;
  }
  g[e] -= acc;
}

cudaError_t fwi_set_tables(const double* Mhat, const double* Bhat, cudaStream_t st) {
  cudaError_t e = cudaMemcpyToSymbolAsync(c_Mhat, Mhat, sizeof(double) * 400, 0, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbolAsync(c_Bhat, Bhat, sizeof(double) * 1600, 0, cudaMemcpyHostToDevice, st);
}

void fwi_residual(int nr, int s, const int* pidx, const double* pw, const double2* U, const double2* d, double2* r,
                  cudaStream_t st) {
  if (nr * s == 0) return;
  k_fwi_residual<<<(nr * s + 255) / 256, 256, 0, st>>>(nr, s, pidx, pw, U, d, r);
  count_launch();
}

void fwi_chi(int64_t m, const double2* r, double* chi, cudaStream_t st) {
  k_fwi_chi<<<1, 256, 0, st>>>(m, r, chi);
  count_launch();
}

void fwi_adjoint_rhs(int nt, int s, int nr, const int* trow, const int* tptr, const int* tk, const double* tw,
                     const double2* r, double2* B, cudaStream_t st) {
  if (nt * s == 0) return;
  k_fwi_adjoint_rhs<<<(nt * s + 255) / 256, 256, 0, st>>>(nt, s, nr, trow, tptr, tk, tw, r, B);
  count_launch();
}

void fwi_gradient(int64_t ne, int s, const int* l2g, const double* vol, const double* farea, const double* m,
                  double omega, const double2* U, const double2* L, double* g, cudaStream_t st) {
  if (ne == 0) return;
  k_fwi_gradient<<<(unsigned)((ne + 127) / 128), 128, 0, st>>>(ne, s, l2g, vol, farea, m, omega, U, L, g);
  count_launch();
}

}  // namespace hz
