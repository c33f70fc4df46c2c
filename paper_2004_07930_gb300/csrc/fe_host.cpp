// P3 finite elements on tetrahedra: reference tables by exact integration,
// dof numbering, element geometry and the generic CSR assembler.
//
// Sec. "Tetrahedral finite element method": Lagrange elements of order 3 on
// a tet mesh; Eq. eqh written as A u = b (Eq. eq1). Reading of the sign
// convention: A = sum_e (K_e - omega^2 m_e M_e) - i omega sum_{Robin f}
// sqrt(m_e) B_f, the weak form of -Lap u - k^2 u = s with d_n u - i k u = g.
//
// The reference integrals are computed exactly from the barycentric
// monomial rule int_T lambda^beta = |T| 3! beta! / (|beta| + 3)! (and its
// 2D analogue on faces), with each basis function expanded as a polynomial
// in the four barycentric coordinates.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <numeric>

#include "host.h"

namespace hz {

const int P3_ALPHA[NLOC][4] = {
    {3, 0, 0, 0}, {0, 3, 0, 0}, {0, 0, 3, 0}, {0, 0, 0, 3},
    // edges (0,1),(0,2),(0,3),(1,2),(1,3),(2,3): node near first, node near second
    {2, 1, 0, 0}, {1, 2, 0, 0}, {2, 0, 1, 0}, {1, 0, 2, 0}, {2, 0, 0, 1}, {1, 0, 0, 2},
    {0, 2, 1, 0}, {0, 1, 2, 0}, {0, 2, 0, 1}, {0, 1, 0, 2}, {0, 0, 2, 1}, {0, 0, 1, 2},
    // faces opposite vertex 0,1,2,3
    {0, 1, 1, 1}, {1, 0, 1, 1}, {1, 1, 0, 1}, {1, 1, 1, 0}};

static const int EDGE_V[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};

namespace {

// Dense polynomial in (l0,l1,l2,l3), each exponent 0..6.
constexpr int PD = 7;
constexpr int PSIZE = PD * PD * PD * PD;
using Poly = std::array<double, PSIZE>;

inline int pidx(int a, int b, int c, int d) { return a + PD * (b + PD * (c + PD * d)); }

Poly poly_one() {
  Poly p{};
  p[0] = 1.0;
  return p;
}

// p * (c1 * l_var + c0)
Poly poly_mul_linear(const Poly& p, int var, double c1, double c0) {
  Poly r{};
  for (int d = 0; d < PD; ++d)
    for (int c = 0; c < PD; ++c)
      for (int b = 0; b < PD; ++b)
        for (int a = 0; a < PD; ++a) {
          double v = p[pidx(a, b, c, d)];
          if (v == 0.0) continue;
          r[pidx(a, b, c, d)] += c0 * v;
          int e[4] = {a, b, c, d};
          e[var] += 1;
          if (e[var] < PD) r[pidx(e[0], e[1], e[2], e[3])] += c1 * v;
        }
  return r;
}

Poly poly_mul(const Poly& p, const Poly& q) {
  Poly r{};
  std::vector<std::pair<int, double>> qn;
  for (int i = 0; i < PSIZE; ++i)
    if (q[i] != 0.0) qn.push_back({i, q[i]});
  for (int d = 0; d < PD; ++d)
    for (int c = 0; c < PD; ++c)
      for (int b = 0; b < PD; ++b)
        for (int a = 0; a < PD; ++a) {
          double v = p[pidx(a, b, c, d)];
          if (v == 0.0) continue;
          for (auto& t : qn) {
            int i = t.first;
            int qa = i % PD, qb = (i / PD) % PD, qc = (i / (PD * PD)) % PD, qd = i / (PD * PD * PD);
            if (a + qa >= PD || b + qb >= PD || c + qc >= PD || d + qd >= PD) continue;
            r[pidx(a + qa, b + qb, c + qc, d + qd)] += v * t.second;
          }
        }
  return r;
}

Poly poly_diff(const Poly& p, int var) {
  Poly r{};
  for (int d = 0; d < PD; ++d)
    for (int c = 0; c < PD; ++c)
      for (int b = 0; b < PD; ++b)
        for (int a = 0; a < PD; ++a) {
          int e[4] = {a, b, c, d};
          if (e[var] == 0) continue;
          double v = p[pidx(a, b, c, d)] * e[var];
          e[var] -= 1;
          r[pidx(e[0], e[1], e[2], e[3])] += v;
        }
  return r;
}

double fact(int n) {
  double f = 1.0;
  for (int i = 2; i <= n; ++i) f *= i;
  return f;
}

// int over the simplex of dimension `dim` (3: tet, 2: face with var `skip` = 0)
double poly_integral(const Poly& p, int dim, int skip) {
  double s = 0.0;
  for (int d = 0; d < PD; ++d)
    for (int c = 0; c < PD; ++c)
      for (int b = 0; b < PD; ++b)
        for (int a = 0; a < PD; ++a) {
          double v = p[pidx(a, b, c, d)];
          if (v == 0.0) continue;
          int e[4] = {a, b, c, d};
          if (skip >= 0 && e[skip] != 0) continue;  // lambda_skip = 0 on that face
          s += v * fact(dim) * fact(a) * fact(b) * fact(c) * fact(d) / fact(a + b + c + d + dim);
        }
  return s;
}

Poly basis_poly(int i) {
  Poly p = poly_one();
  for (int a = 0; a < 4; ++a)
    for (int j = 0; j < P3_ALPHA[i][a]; ++j) p = poly_mul_linear(p, a, 3.0 / (j + 1), -double(j) / (j + 1));
  return p;
}

P3Tables build_tables() {
  P3Tables t;
  std::vector<Poly> phi(NLOC);
  std::vector<std::array<Poly, 4>> dphi(NLOC);
  for (int i = 0; i < NLOC; ++i) {
    phi[i] = basis_poly(i);
    for (int a = 0; a < 4; ++a) dphi[i][a] = poly_diff(phi[i], a);
  }
  for (int i = 0; i < NLOC; ++i)
    for (int j = 0; j <= i; ++j) {
      Poly pp = poly_mul(phi[i], phi[j]);
      t.M[i][j] = t.M[j][i] = poly_integral(pp, 3, -1);
      for (int c = 0; c < 4; ++c) t.B[c][i][j] = t.B[c][j][i] = poly_integral(pp, 2, c);
    }
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b)
      for (int i = 0; i < NLOC; ++i)
        for (int j = 0; j < NLOC; ++j) t.S[a][b][i][j] = poly_integral(poly_mul(dphi[i][a], dphi[j][b]), 3, -1);
  for (int c = 0; c < 4; ++c) {
    int q = 0;
    for (int i = 0; i < NLOC; ++i)
      if (P3_ALPHA[i][c] == 0) t.face_nodes[c][q++] = i;
  }
  return t;
}

}  // namespace

const P3Tables& p3_tables() {
  static const P3Tables t = build_tables();
  return t;
}

void p3_basis(const double lam[4], double phi[NLOC]) {
  for (int i = 0; i < NLOC; ++i) {
    double v = 1.0;
    for (int a = 0; a < 4; ++a)
      for (int j = 0; j < P3_ALPHA[i][a]; ++j) v *= (3.0 * lam[a] - j) / (j + 1);
    phi[i] = v;
  }
}

ElemGeom elem_geom(const double* P) {
  double J[3][3];  // columns P1-P0, P2-P0, P3-P0: J[r][c]
  for (int c = 0; c < 3; ++c)
    for (int r = 0; r < 3; ++r) J[r][c] = P[3 * (c + 1) + r] - P[r];
  double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
               J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
  if (det == 0.0) throw HzError{1, "degenerate tetrahedron"};
  double inv[3][3];
  inv[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
  inv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
  inv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
  inv[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
  inv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
  inv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
  inv[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
  inv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
  inv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
  double g[4][3];
  for (int d = 0; d < 3; ++d) {
    g[1][d] = inv[0][d];
    g[2][d] = inv[1][d];
    g[3][d] = inv[2][d];
    g[0][d] = -(g[1][d] + g[2][d] + g[3][d]);
  }
  ElemGeom eg;
  eg.vol = std::fabs(det) / 6.0;
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) eg.G[a][b] = g[a][0] * g[b][0] + g[a][1] * g[b][1] + g[a][2] * g[b][2];
  return eg;
}

double face_area(const double* P, int c) {
  int o[3], q = 0;
  for (int a = 0; a < 4; ++a)
    if (a != c) o[q++] = a;
  double u[3], v[3];
  for (int d = 0; d < 3; ++d) {
    u[d] = P[3 * o[1] + d] - P[3 * o[0] + d];
    v[d] = P[3 * o[2] + d] - P[3 * o[0] + d];
  }
  double cx = u[1] * v[2] - u[2] * v[1], cy = u[2] * v[0] - u[0] * v[2], cz = u[0] * v[1] - u[1] * v[0];
  return 0.5 * std::sqrt(cx * cx + cy * cy + cz * cz);
}

// ---------------------------------------------------------------------------
// Mesh adjacency and boundary tags
// ---------------------------------------------------------------------------
namespace {
struct FaceKey {
  int32_t v[3];
  int64_t e;
  int8_t c;
  bool operator<(const FaceKey& o) const {
    if (v[0] != o.v[0]) return v[0] < o.v[0];
    if (v[1] != o.v[1]) return v[1] < o.v[1];
    if (v[2] != o.v[2]) return v[2] < o.v[2];
    return e < o.e;
  }
  bool same(const FaceKey& o) const { return v[0] == o.v[0] && v[1] == o.v[1] && v[2] == o.v[2]; }
};
inline void sort3(int32_t* v) {
  if (v[0] > v[1]) std::swap(v[0], v[1]);
  if (v[1] > v[2]) std::swap(v[1], v[2]);
  if (v[0] > v[1]) std::swap(v[0], v[1]);
}
}  // namespace

void mesh_build_adjacency(Mesh& m) {
  const int64_t ne = m.ne;
  for (int64_t i = 0; i < 4 * ne; ++i)
    if (m.tets[i] < 0 || m.tets[i] >= m.nv) throw HzError{1, "tet vertex index out of range"};
  std::vector<FaceKey> f(4 * ne);
  for (int64_t e = 0; e < ne; ++e)
    for (int c = 0; c < 4; ++c) {
      FaceKey& k = f[4 * e + c];
      int q = 0;
      for (int a = 0; a < 4; ++a)
        if (a != c) k.v[q++] = m.tets[4 * e + a];
      sort3(k.v);
      k.e = e;
      k.c = (int8_t)c;
    }
  std::sort(f.begin(), f.end());
  m.nbr.assign(4 * ne, -1);
  m.ftag.assign(4 * ne, -1);
  std::vector<FaceKey> ext;
  for (size_t i = 0; i < f.size();) {
    size_t j = i + 1;
    while (j < f.size() && f[j].same(f[i])) ++j;
    if (j - i == 2) {
      m.nbr[4 * f[i].e + f[i].c] = f[i + 1].e;
      m.nbr[4 * f[i + 1].e + f[i + 1].c] = f[i].e;
    } else if (j - i == 1) {
      ext.push_back(f[i]);
    } else {
      throw HzError{1, "non-manifold face shared by more than two tetrahedra"};
    }
    i = j;
  }
  const int64_t nbf = (int64_t)m.btag.size();
  for (int64_t b = 0; b < nbf; ++b) {
    FaceKey k;
    for (int d = 0; d < 3; ++d) k.v[d] = m.bfaces[3 * b + d];
    sort3(k.v);
    k.e = -1;
    auto it = std::lower_bound(ext.begin(), ext.end(), k);
    if (it == ext.end() || !it->same(k)) throw HzError{1, "listed boundary face is not an exterior face"};
    if (m.btag[b] != 0 && m.btag[b] != 1) throw HzError{1, "boundary tag must be 0 (Robin) or 1 (Dirichlet)"};
    m.ftag[4 * it->e + it->c] = (int8_t)m.btag[b];
  }
}

// ---------------------------------------------------------------------------
// P3 dof numbering
// ---------------------------------------------------------------------------
Space p3_space(const Mesh& m) {
  const int64_t ne = m.ne, nv = m.nv;
  Space sp;
  // vertices in use
  std::vector<int64_t> vid(nv, -1);
  int64_t nvu = 0;
  for (int64_t i = 0; i < 4 * ne; ++i)
    if (vid[m.tets[i]] < 0) vid[m.tets[i]] = 0;
  for (int64_t v = 0; v < nv; ++v)
    if (vid[v] == 0) vid[v] = nvu++;
  // edges
  std::vector<int64_t> ekeys(6 * ne);
  for (int64_t e = 0; e < ne; ++e)
    for (int q = 0; q < 6; ++q) {
      int64_t a = m.tets[4 * e + EDGE_V[q][0]], b = m.tets[4 * e + EDGE_V[q][1]];
      ekeys[6 * e + q] = std::min(a, b) * nv + std::max(a, b);
    }
  std::vector<int64_t> eu(ekeys);
  std::sort(eu.begin(), eu.end());
  eu.erase(std::unique(eu.begin(), eu.end()), eu.end());
  // faces
  struct F3 {
    int32_t v[3];
    bool operator<(const F3& o) const {
      return v[0] != o.v[0] ? v[0] < o.v[0] : (v[1] != o.v[1] ? v[1] < o.v[1] : v[2] < o.v[2]);
    }
    bool operator==(const F3& o) const { return v[0] == o.v[0] && v[1] == o.v[1] && v[2] == o.v[2]; }
  };
  std::vector<F3> fk(4 * ne);
  for (int64_t e = 0; e < ne; ++e)
    for (int c = 0; c < 4; ++c) {
      int q = 0;
      for (int a = 0; a < 4; ++a)
        if (a != c) fk[4 * e + c].v[q++] = m.tets[4 * e + a];
      sort3(fk[4 * e + c].v);
    }
  std::vector<F3> fu(fk);
  std::sort(fu.begin(), fu.end());
  fu.erase(std::unique(fu.begin(), fu.end()), fu.end());
  const int64_t nE = (int64_t)eu.size(), nF = (int64_t)fu.size();
  const int64_t n = nvu + 2 * nE + nF;
  std::vector<int64_t> l2g(NLOC * ne);
  for (int64_t e = 0; e < ne; ++e) {
    const int32_t* t = &m.tets[4 * e];
    for (int a = 0; a < 4; ++a) l2g[NLOC * e + a] = vid[t[a]];
    for (int q = 0; q < 6; ++q) {
      int64_t a = t[EDGE_V[q][0]], b = t[EDGE_V[q][1]];
      int64_t id = std::lower_bound(eu.begin(), eu.end(), ekeys[6 * e + q]) - eu.begin();
      // local node 4+2q is near EDGE_V[q][0]; global first dof is near the lower vertex id
      bool first_is_lo = a < b;
      l2g[NLOC * e + 4 + 2 * q] = nvu + 2 * id + (first_is_lo ? 0 : 1);
      l2g[NLOC * e + 5 + 2 * q] = nvu + 2 * id + (first_is_lo ? 1 : 0);
    }
    for (int c = 0; c < 4; ++c) {
      int64_t id = std::lower_bound(fu.begin(), fu.end(), fk[4 * e + c]) - fu.begin();
      l2g[NLOC * e + 16 + c] = nvu + 2 * nE + id;
    }
  }
  // coordinates in the provisional numbering
  std::vector<double> X(3 * n, 0.0);
  for (int64_t e = 0; e < ne; ++e) {
    const int32_t* t = &m.tets[4 * e];
    for (int i = 0; i < NLOC; ++i) {
      int64_t g = l2g[NLOC * e + i];
      for (int d = 0; d < 3; ++d) {
        double s = 0.0;
        for (int a = 0; a < 4; ++a) s += P3_ALPHA[i][a] * m.xyz[3 * t[a] + d];
        X[3 * g + d] = s / 3.0;
      }
    }
  }
  // spatial order: slowest axis = largest extent
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int64_t g = 0; g < n; ++g)
    for (int d = 0; d < 3; ++d) {
      lo[d] = std::min(lo[d], X[3 * g + d]);
      hi[d] = std::max(hi[d], X[3 * g + d]);
    }
  int ax[3] = {0, 1, 2};
  std::stable_sort(ax, ax + 3, [&](int a, int b) { return (hi[a] - lo[a]) > (hi[b] - lo[b]); });
  double ext = std::max({hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2], 1e-300});
  std::vector<std::array<int64_t, 3>> key(n);
  for (int64_t g = 0; g < n; ++g)
    for (int q = 0; q < 3; ++q) key[g][q] = std::llround((X[3 * g + ax[q]] - lo[ax[q]]) / (1e-7 * ext));
  std::vector<int64_t> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return key[a] < key[b]; });
  std::vector<int64_t> newid(n);
  for (int64_t i = 0; i < n; ++i) newid[order[i]] = i;
  sp.n = n;
  sp.l2g.resize(NLOC * ne);
  for (int64_t i = 0; i < NLOC * ne; ++i) sp.l2g[i] = newid[l2g[i]];
  sp.coords.resize(3 * n);
  for (int64_t g = 0; g < n; ++g)
    for (int d = 0; d < 3; ++d) sp.coords[3 * newid[g] + d] = X[3 * g + d];
  // Dirichlet dofs: the 10 nodes of every Dirichlet face
  const P3Tables& T = p3_tables();
  sp.dirichlet.assign(n, 0);
  for (int64_t e = 0; e < ne; ++e)
    for (int c = 0; c < 4; ++c)
      if (m.ftag.size() && m.ftag[4 * e + c] == 1)
        for (int q = 0; q < 10; ++q) sp.dirichlet[sp.l2g[NLOC * e + T.face_nodes[c][q]]] = 1;
  return sp;
}

// ---------------------------------------------------------------------------
// Generic assembler (row-parallel, deterministic)
// ---------------------------------------------------------------------------
CsrC assemble(const AssemblyInput& in) {
  const Space& sp = *in.space;
  const Mesh& m = *in.mesh;
  const int64_t nel = (int64_t)in.elems.size();
  const int64_t nl = in.nloc;
  const P3Tables& T = p3_tables();
  // row -> (element slot, local node)
  std::vector<int64_t> cnt(nl + 1, 0);
  for (int64_t q = 0; q < nel; ++q) {
    int64_t e = in.elems[q];
    for (int i = 0; i < NLOC; ++i) {
      int64_t r = in.g2l[sp.l2g[NLOC * e + i]];
      if (r < 0) throw HzError{4, "assembler: element dof outside the local set"};
      cnt[r + 1]++;
    }
  }
  for (int64_t r = 0; r < nl; ++r) cnt[r + 1] += cnt[r];
  std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
  std::vector<int64_t> rel(cnt[nl]);
  for (int64_t q = 0; q < nel; ++q) {
    int64_t e = in.elems[q];
    for (int i = 0; i < NLOC; ++i) {
      int64_t r = in.g2l[sp.l2g[NLOC * e + i]];
      rel[fill[r]++] = q * NLOC + i;
    }
  }
  auto is_dir = [&](int64_t r) { return !in.dir_local.empty() && in.dir_local[r]; };
  // pattern
  CsrC A;
  A.nrows = A.ncols = nl;
  A.rowptr.assign(nl + 1, 0);
  std::vector<int64_t> rlen(nl, 0);
#pragma omp parallel
  {
    std::vector<int32_t> buf;
#pragma omp for schedule(dynamic, 512)
    for (int64_t r = 0; r < nl; ++r) {
      if (is_dir(r)) {
        rlen[r] = 1;
        continue;
      }
      buf.clear();
      for (int64_t p = cnt[r]; p < cnt[r + 1]; ++p) {
        int64_t e = in.elems[rel[p] / NLOC];
        for (int j = 0; j < NLOC; ++j) {
          int64_t c = in.g2l[sp.l2g[NLOC * e + j]];
          if (!is_dir(c)) buf.push_back((int32_t)c);
        }
      }
      std::sort(buf.begin(), buf.end());
      rlen[r] = std::unique(buf.begin(), buf.end()) - buf.begin();
    }
  }
  for (int64_t r = 0; r < nl; ++r) A.rowptr[r + 1] = A.rowptr[r] + rlen[r];
  A.col.resize(A.rowptr[nl]);
  A.val.assign(A.rowptr[nl], cplx(0.0, 0.0));
#pragma omp parallel
  {
    std::vector<int32_t> buf;
#pragma omp for schedule(dynamic, 512)
    for (int64_t r = 0; r < nl; ++r) {
      int64_t o = A.rowptr[r];
      if (is_dir(r)) {
        A.col[o] = (int32_t)r;
        A.val[o] = 1.0;
        continue;
      }
      buf.clear();
      for (int64_t p = cnt[r]; p < cnt[r + 1]; ++p) {
        int64_t e = in.elems[rel[p] / NLOC];
        for (int j = 0; j < NLOC; ++j) {
          int64_t c = in.g2l[sp.l2g[NLOC * e + j]];
          if (!is_dir(c)) buf.push_back((int32_t)c);
        }
      }
      std::sort(buf.begin(), buf.end());
      buf.erase(std::unique(buf.begin(), buf.end()), buf.end());
      std::copy(buf.begin(), buf.end(), A.col.begin() + o);
      const int32_t* cb = &A.col[o];
      const int64_t len = (int64_t)buf.size();
      for (int64_t p = cnt[r]; p < cnt[r + 1]; ++p) {
        const int64_t q = rel[p] / NLOC;
        const int li = (int)(rel[p] % NLOC);
        const int64_t e = in.elems[q];
        cplx row[NLOC];
        if (in.elem_mats) {
          for (int j = 0; j < NLOC; ++j) row[j] = (*in.elem_mats)[(q * NLOC + li) * NLOC + j];
        } else {
          const int32_t* t = &m.tets[4 * e];
          double P[12];
          for (int a = 0; a < 4; ++a)
            for (int d = 0; d < 3; ++d) P[3 * a + d] = m.xyz[3 * t[a] + d];
          ElemGeom g = elem_geom(P);
          const double me = in.mvals[e];
          const double k2 = in.omega * in.omega * me;
          for (int j = 0; j < NLOC; ++j) {
            double k = 0.0;
            for (int a = 0; a < 4; ++a)
              for (int b = 0; b < 4; ++b) k += g.G[a][b] * T.S[a][b][li][j];
            row[j] = cplx(g.vol * (k - k2 * T.M[li][j]), 0.0);
          }
          if (!in.robin_face.empty())
            for (int c = 0; c < 4; ++c)
              if (in.robin_face[4 * e + c]) {
                const double s = -in.omega * std::sqrt(me) * face_area(P, c);
                for (int j = 0; j < NLOC; ++j) row[j] += cplx(0.0, s * T.B[c][li][j]);
              }
        }
        for (int j = 0; j < NLOC; ++j) {
          int64_t c = in.g2l[sp.l2g[NLOC * e + j]];
          if (is_dir(c)) continue;
          int64_t pos = std::lower_bound(cb, cb + len, (int32_t)c) - cb;
          A.val[o + pos] += row[j];
        }
      }
    }
  }
  return A;
}

void split_re_im(const CsrC& A, CsrR& re, CsrR& im) {
  const int64_t n = A.nrows;
  re.nrows = im.nrows = n;
  re.ncols = im.ncols = A.ncols;
  re.rowptr = A.rowptr;
  re.col = A.col;
  re.val.resize(A.val.size());
  for (size_t i = 0; i < A.val.size(); ++i) re.val[i] = A.val[i].real();
  im.rowptr.assign(n + 1, 0);
  im.col.clear();
  im.val.clear();
  for (int64_t r = 0; r < n; ++r) {
    for (int64_t p = A.rowptr[r]; p < A.rowptr[r + 1]; ++p)
      if (A.val[p].imag() != 0.0) {
        im.col.push_back(A.col[p]);
        im.val.push_back(A.val[p].imag());
      }
    im.rowptr[r + 1] = (int64_t)im.col.size();
  }
}

}  // namespace hz
