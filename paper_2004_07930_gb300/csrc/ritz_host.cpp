// Harmonic Ritz vectors of one FGMRES cycle, for Krylov subspace recycling
// (GCRO-DR, deflated restarting; Sec. "Conclusion": recycling across sources
// and frequencies).
//
// Given the cycle's (m+1) x m Hessenberg matrix Hbar (Hm on top, h = Hbar[m][m-1]
// below), the harmonic Ritz values theta and vectors p of A M^{-1} with
// respect to the preconditioned Krylov space satisfy
//     (Hm + h^2 f e_m^T) p = theta p,   Hm^H f = e_m,
// the matrix on the left being upper Hessenberg (only its last column
// changes). Its eigenpairs come from the shifted QR iteration (Wilkinson
// shifts, Givens rotations, deflation at negligible subdiagonals) and the
// eigenvectors of the triangular Schur factor by back substitution. The k
// vectors with the smallest |theta| span the directions FGMRES converges on
// slowest; they are the ones kept.
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

namespace hz {

using zc = std::complex<double>;

namespace {

// complex Givens rotation zeroing b: [c, s; -conj(s), c] [a; b] = [r; 0], c real
void givens(zc a, zc b, double& c, zc& s) {
  const double aa = std::abs(a), bb = std::abs(b);
  if (bb == 0.0) {
    c = 1.0;
    s = 0.0;
  } else if (aa == 0.0) {
    c = 0.0;
    s = std::conj(b) / bb;
  } else {
    const double t = std::hypot(aa, bb);
    c = aa / t;
    s = (a / aa) * std::conj(b) / t;
  }
}

// solve A x = b (n x n, row-major) by Gaussian elimination with partial pivoting; false if singular
bool solve_dense(std::vector<zc> A, std::vector<zc>& b, int n) {
  for (int j = 0; j < n; ++j) {
    int p = j;
    for (int i = j + 1; i < n; ++i)
      if (std::abs(A[i * n + j]) > std::abs(A[p * n + j])) p = i;
    if (std::abs(A[p * n + j]) == 0.0) return false;
    if (p != j) {
      for (int c = 0; c < n; ++c) std::swap(A[j * n + c], A[p * n + c]);
      std::swap(b[j], b[p]);
    }
    for (int i = j + 1; i < n; ++i) {
      const zc l = A[i * n + j] / A[j * n + j];
      if (l == 0.0) continue;
      for (int c = j; c < n; ++c) A[i * n + c] -= l * A[j * n + c];
      b[i] -= l * b[j];
    }
  }
  for (int j = n - 1; j >= 0; --j) {
    zc v = b[j];
    for (int c = j + 1; c < n; ++c) v -= A[j * n + c] * b[c];
    b[j] = v / A[j * n + j];
  }
  return true;
}

}  // namespace

// Schur decomposition of an upper Hessenberg matrix T (n x n, row-major, in
// place): T <- Q^H T Q upper triangular, Q accumulated (row-major). False if
// the iteration does not converge.
bool hessenberg_schur(std::vector<zc>& T, std::vector<zc>& Q, int n) {
  Q.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) Q[i * n + i] = 1.0;
  const double eps = 1e-15;
  int hi = n - 1, iter = 0;
  while (hi > 0) {
    if (++iter > 100 * n) return false;
    // lowest negligible subdiagonal in the active window
    int lo = hi;
    while (lo > 0) {
      const double s = std::abs(T[lo * n + lo]) + std::abs(T[(lo - 1) * n + lo - 1]);
      if (std::abs(T[lo * n + lo - 1]) <= eps * (s > 0 ? s : 1.0)) {
        T[lo * n + lo - 1] = 0.0;
        break;
      }
      --lo;
    }
    if (lo == hi) {  // a 1 x 1 block has converged
      --hi;
      iter = 0;
      continue;
    }
    // Wilkinson shift: the eigenvalue of the trailing 2 x 2 block closer to its last entry
    const zc a = T[(hi - 1) * n + hi - 1], b = T[(hi - 1) * n + hi], c = T[hi * n + hi - 1], d = T[hi * n + hi];
    const zc tr = a + d, det = a * d - b * c;
    const zc disc = std::sqrt(tr * tr - 4.0 * det);
    const zc l1 = 0.5 * (tr + disc), l2 = 0.5 * (tr - disc);
    zc mu = std::abs(l1 - d) < std::abs(l2 - d) ? l1 : l2;
    if (iter % 11 == 10) mu += std::abs(T[hi * n + hi - 1]);  // exceptional shift
    // one implicit single-shift QR sweep over rows/columns lo..hi
    zc x = T[lo * n + lo] - mu, y = T[(lo + 1) * n + lo];
    for (int k = lo; k < hi; ++k) {
      double cs;
      zc sn;
      givens(x, y, cs, sn);
      // rows k, k+1 from the left: G
      for (int j = std::max(lo, k - 1); j < n; ++j) {
        const zc t1 = T[k * n + j], t2 = T[(k + 1) * n + j];
        T[k * n + j] = cs * t1 + sn * t2;
        T[(k + 1) * n + j] = -std::conj(sn) * t1 + cs * t2;
      }
      // columns k, k+1 from the right: G^H
      for (int i = 0; i <= std::min(hi, k + 2); ++i) {
        const zc t1 = T[i * n + k], t2 = T[i * n + k + 1];
        T[i * n + k] = cs * t1 + std::conj(sn) * t2;
        T[i * n + k + 1] = -sn * t1 + cs * t2;
      }
      for (int i = 0; i < n; ++i) {
        const zc q1 = Q[i * n + k], q2 = Q[i * n + k + 1];
        Q[i * n + k] = cs * q1 + std::conj(sn) * q2;
        Q[i * n + k + 1] = -sn * q1 + cs * q2;
      }
      if (k < hi - 1) {
        x = T[(k + 1) * n + k];
        y = T[(k + 2) * n + k];
      }
    }
  }
  return true;
}

// Harmonic Ritz vectors: Hbar column-major (m+1) x m (entry (i, j) at i + j (m+1)).
// On success P (m x k, column-major) holds the k eigenvectors with the smallest
// |theta| (unit 2-norm) and theta their values, ascending in |theta|.
bool harmonic_ritz(const std::vector<zc>& Hbar, int m, int k, std::vector<zc>& P, std::vector<zc>& theta) {
  if (m < 1 || k < 1 || k > m) return false;
  const int ld = m + 1;
  std::vector<zc> Hm((size_t)m * m);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) Hm[i * m + j] = Hbar[i + (size_t)j * ld];
  const zc h = Hbar[m + (size_t)(m - 1) * ld];
  // f = Hm^{-H} e_m
  std::vector<zc> HmH((size_t)m * m), f(m, 0.0);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) HmH[i * m + j] = std::conj(Hm[j * m + i]);
  f[m - 1] = 1.0;
  if (!solve_dense(HmH, f, m)) return false;
  std::vector<zc> T = Hm;
  const zc h2 = h * std::conj(h);
  for (int i = 0; i < m; ++i) T[i * m + m - 1] += h2 * f[i];
  std::vector<zc> Q;
  if (!hessenberg_schur(T, Q, m)) return false;
  // eigenvectors of the triangular T, then y -> Q y
  std::vector<int> order(m);
  for (int i = 0; i < m; ++i) order[i] = i;
  std::sort(order.begin(), order.end(),
            [&](int a, int b) { return std::abs(T[a * m + a]) < std::abs(T[b * m + b]); });
  P.assign((size_t)m * k, 0.0);
  theta.assign(k, 0.0);
  for (int q = 0; q < k; ++q) {
    const int e = order[q];
    const zc lam = T[e * m + e];
    std::vector<zc> y(m, 0.0);
    y[e] = 1.0;
    for (int j = e - 1; j >= 0; --j) {
      zc v = 0.0;
      for (int l = j + 1; l <= e; ++l) v += T[j * m + l] * y[l];
      zc dd = T[j * m + j] - lam;
      if (std::abs(dd) < 1e-14 * (std::abs(lam) + 1e-300)) dd = 1e-14 * (std::abs(lam) + 1e-300);
      y[j] = -v / dd;
    }
    double nrm = 0.0;
    std::vector<zc> p(m, 0.0);
    for (int i = 0; i < m; ++i) {
      for (int j = 0; j <= e; ++j) p[i] += Q[i * m + j] * y[j];
      nrm += std::norm(p[i]);
    }
    nrm = std::sqrt(nrm);
    if (!(nrm > 0.0) || !std::isfinite(nrm)) return false;
    for (int i = 0; i < m; ++i) P[i + (size_t)q * m] = p[i] / nrm;
    theta[q] = lam;
  }
  return true;
}

}  // namespace hz

// Host-only entry for the CPU tests of the routine above (not part of the
// public ABI): Hbar column-major (m+1) x m as interleaved doubles; P (m x k,
// column-major) and theta (k) as interleaved doubles. Returns 0 on success.
extern "C" int hz_internal_harmonic_ritz(const double* Hbar, int m, int k, double* P, double* theta) {
  std::vector<hz::zc> H((size_t)(m + 1) * m), Pv, th;
  for (size_t i = 0; i < H.size(); ++i) H[i] = hz::zc(Hbar[2 * i], Hbar[2 * i + 1]);
  if (!hz::harmonic_ritz(H, m, k, Pv, th)) return 1;
  for (size_t i = 0; i < Pv.size(); ++i) {
    P[2 * i] = Pv[i].real();
    P[2 * i + 1] = Pv[i].imag();
  }
  for (int q = 0; q < k; ++q) {
    theta[2 * q] = th[q].real();
    theta[2 * q + 1] = th[q].imag();
  }
  return 0;
}
