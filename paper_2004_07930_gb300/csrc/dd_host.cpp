// Domain decomposition setup: overlapping subdomains, partition of unity,
// local Robin matrices, the coarse space and the nested-dissection symbolic
// analysis of every local matrix.
//
// Sec. "Domain decomposition preconditioner", Eq. oras: subdomains Gamma_i
// of an overlapping decomposition, Boolean restrictions R_i, diagonal
// partition of unity D_i and local operators A_i with absorbing conditions
// on the interfaces. Eq. 2lvl: coarse space on a coarse mesh Gamma_H with
// E = Z^T A Z. Readings (the paper names neither the overlap rule nor the
// partition of unity): overlap = the subdomain's elements plus every
// element sharing a vertex with them; D_i = Boolean ownership by the lowest
// subdomain whose own elements carry the dof; A_i keeps the physical
// Dirichlet rows.
#include <algorithm>
#include <cmath>
#include <functional>
#include <numeric>

#include "dd_host.h"

namespace hz {

// ---------------------------------------------------------------------------
// Overlapping subdomains and local matrices
// ---------------------------------------------------------------------------
std::vector<Subdomain> build_subdomains(const Mesh& m, const Space& sp, const std::vector<int32_t>& part,
                                        int nparts, const std::vector<double>& mvals, double omega, int layers) {
  const int64_t ne = m.ne, n = sp.n;
  std::vector<int32_t> owner(n, nparts);
  for (int64_t e = 0; e < ne; ++e)
    for (int i = 0; i < NLOC; ++i) {
      int64_t g = sp.l2g[NLOC * e + i];
      owner[g] = std::min(owner[g], part[e]);
    }
  std::vector<Subdomain> subs(nparts);
  std::vector<int64_t> g2l(n, -1);
  std::vector<uint8_t> vmark(m.nv), inset(ne);
  for (int i = 0; i < nparts; ++i) {
    Subdomain& S = subs[i];
    // each layer adds every element sharing a vertex with the current set
    for (int64_t e = 0; e < ne; ++e) inset[e] = part[e] == i;
    for (int layer = 0; layer < layers; ++layer) {
      std::fill(vmark.begin(), vmark.end(), 0);
      for (int64_t e = 0; e < ne; ++e)
        if (inset[e])
          for (int a = 0; a < 4; ++a) vmark[m.tets[4 * e + a]] = 1;
      for (int64_t e = 0; e < ne; ++e) {
        bool hit = false;
        for (int a = 0; a < 4; ++a) hit |= vmark[m.tets[4 * e + a]] != 0;
        inset[e] = hit;
      }
    }
    for (int64_t e = 0; e < ne; ++e)
      if (inset[e]) S.elems.push_back(e);
    if (S.elems.empty()) throw HzError{1, "empty subdomain in the partition"};
    for (int64_t e : S.elems)
      for (int q = 0; q < NLOC; ++q) S.dofs.push_back(sp.l2g[NLOC * e + q]);
    std::sort(S.dofs.begin(), S.dofs.end());
    S.dofs.erase(std::unique(S.dofs.begin(), S.dofs.end()), S.dofs.end());
    const int64_t nl = (int64_t)S.dofs.size();
    for (int64_t l = 0; l < nl; ++l) g2l[S.dofs[l]] = l;
    S.owned.resize(nl);
    for (int64_t l = 0; l < nl; ++l) S.owned[l] = owner[S.dofs[l]] == i;
    AssemblyInput in;
    in.space = &sp;
    in.mesh = &m;
    in.elems = S.elems;
    in.mvals = mvals;
    in.omega = omega;
    in.robin_face.assign(4 * ne, 0);
    for (int64_t e : S.elems)
      for (int c = 0; c < 4; ++c) {
        int64_t nb = m.nbr[4 * e + c];
        if (nb >= 0)
          in.robin_face[4 * e + c] = inset[nb] ? 0 : 1;  // interface: absorbing
        else
          in.robin_face[4 * e + c] = m.ftag[4 * e + c] == 0 ? 1 : 0;
      }
    in.g2l = g2l;
    in.nloc = nl;
    in.dir_local.resize(nl);
    for (int64_t l = 0; l < nl; ++l) in.dir_local[l] = sp.dirichlet[S.dofs[l]];
    S.A = assemble(in);
    for (int64_t l = 0; l < nl; ++l) g2l[S.dofs[l]] = -1;
  }
  return subs;
}

CsrC assemble_global(const Mesh& m, const Space& sp, const std::vector<double>& mvals, double omega) {
  AssemblyInput in;
  in.space = &sp;
  in.mesh = &m;
  in.elems.resize(m.ne);
  std::iota(in.elems.begin(), in.elems.end(), 0);
  in.mvals = mvals;
  in.omega = omega;
  in.robin_face.assign(4 * m.ne, 0);
  for (int64_t i = 0; i < 4 * m.ne; ++i) in.robin_face[i] = (m.nbr[i] < 0 && m.ftag[i] == 0) ? 1 : 0;
  in.g2l.resize(sp.n);
  std::iota(in.g2l.begin(), in.g2l.end(), 0);
  in.nloc = sp.n;
  in.dir_local = sp.dirichlet;
  return assemble(in);
}

// ---------------------------------------------------------------------------
// Point location in a tet mesh (uniform bins)
// ---------------------------------------------------------------------------
struct Locator {
  const Mesh* m;
  double lo[3], h[3];
  int nb[3];
  std::vector<int64_t> ptr, lst;
  explicit Locator(const Mesh& mesh) : m(&mesh) {
    for (int d = 0; d < 3; ++d) {
      lo[d] = 1e300;
      double hi = -1e300;
      for (int64_t v = 0; v < mesh.nv; ++v) {
        lo[d] = std::min(lo[d], mesh.xyz[3 * v + d]);
        hi = std::max(hi, mesh.xyz[3 * v + d]);
      }
      double ext = std::max(hi - lo[d], 1e-300);
      nb[d] = std::max(1, (int)std::cbrt((double)mesh.ne) );
      h[d] = ext / nb[d] * (1 + 1e-12);
    }
    std::vector<std::vector<int64_t>> bins((size_t)nb[0] * nb[1] * nb[2]);
    for (int64_t e = 0; e < mesh.ne; ++e) {
      int b0[3], b1[3];
      for (int d = 0; d < 3; ++d) {
        double a = 1e300, b = -1e300;
        for (int q = 0; q < 4; ++q) {
          double x = mesh.xyz[3 * mesh.tets[4 * e + q] + d];
          a = std::min(a, x);
          b = std::max(b, x);
        }
        double eps = 1e-9 * h[d];
        b0[d] = std::max(0, std::min(nb[d] - 1, (int)std::floor((a - eps - lo[d]) / h[d])));
        b1[d] = std::max(0, std::min(nb[d] - 1, (int)std::floor((b + eps - lo[d]) / h[d])));
      }
      for (int k = b0[2]; k <= b1[2]; ++k)
        for (int j = b0[1]; j <= b1[1]; ++j)
          for (int i = b0[0]; i <= b1[0]; ++i) bins[i + (size_t)nb[0] * (j + (size_t)nb[1] * k)].push_back(e);
    }
    ptr.assign(bins.size() + 1, 0);
    for (size_t b = 0; b < bins.size(); ++b) ptr[b + 1] = ptr[b] + bins[b].size();
    lst.reserve(ptr.back());
    for (auto& v : bins) lst.insert(lst.end(), v.begin(), v.end());
  }
  static bool bary(const double* P, const double* x, double lam[4]) {
    double J[3][3], r[3];
    for (int c = 0; c < 3; ++c)
      for (int d = 0; d < 3; ++d) J[d][c] = P[3 * (c + 1) + d] - P[d];
    for (int d = 0; d < 3; ++d) r[d] = x[d] - P[d];
    double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                 J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    if (det == 0.0) return false;
    // Cramer's rule
    double s[3];
    for (int c = 0; c < 3; ++c) {
      double M[3][3];
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) M[a][b] = (b == c) ? r[a] : J[a][b];
      s[c] = (M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) - M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
              M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0])) /
             det;
    }
    lam[1] = s[0];
    lam[2] = s[1];
    lam[3] = s[2];
    lam[0] = 1.0 - s[0] - s[1] - s[2];
    return true;
  }
  // lowest element index containing x (barycentrics >= -tol), or -1
  int64_t locate(const double* x, double lam_out[4], double tol = 1e-9) const {
    int b[3];
    for (int d = 0; d < 3; ++d) b[d] = std::max(0, std::min(nb[d] - 1, (int)std::floor((x[d] - lo[d]) / h[d])));
    size_t bi = b[0] + (size_t)nb[0] * (b[1] + (size_t)nb[1] * b[2]);
    int64_t best = -1;
    for (int64_t p = ptr[bi]; p < ptr[bi + 1]; ++p) {
      int64_t e = lst[p];
      if (best >= 0 && e >= best) continue;
      double P[12], lam[4];
      for (int q = 0; q < 4; ++q)
        for (int d = 0; d < 3; ++d) P[3 * q + d] = m->xyz[3 * m->tets[4 * e + q] + d];
      if (!bary(P, x, lam)) continue;
      if (std::min({lam[0], lam[1], lam[2], lam[3]}) >= -tol) {
        best = e;
        std::copy(lam, lam + 4, lam_out);
      }
    }
    return best;
  }
};

void locate_points(const Mesh& m, const double* x, int64_t np, int64_t* elem, double* lam) {
  Locator loc(m);
  for (int64_t i = 0; i < np; ++i) elem[i] = loc.locate(x + 3 * i, lam + 4 * i);
}

// ---------------------------------------------------------------------------
// Coarse space (nested coarse mesh)
// ---------------------------------------------------------------------------
CoarseSpace build_coarse(const Mesh& fm, const Space& fs, const std::vector<double>& mvals_f,
                         const std::vector<int32_t>& part_f, double omega, Mesh& cm) {
  CoarseSpace C;
  mesh_build_adjacency(cm);
  C.space = p3_space(cm);
  const Space& cs = C.space;
  const int64_t nef = fm.ne, nec = cm.ne;
  Locator loc(cm);
  // fine element -> containing coarse element (all four vertices inside)
  C.parent.assign(nef, -1);
  std::vector<int64_t> bad(1, 0);
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < nef; ++e) {
    double x[3] = {0, 0, 0}, lam[4];
    for (int q = 0; q < 4; ++q)
      for (int d = 0; d < 3; ++d) x[d] += 0.25 * fm.xyz[3 * fm.tets[4 * e + q] + d];
    int64_t E = loc.locate(x, lam);
    if (E < 0) {
#pragma omp atomic
      bad[0]++;
      continue;
    }
    double P[12];
    for (int q = 0; q < 4; ++q)
      for (int d = 0; d < 3; ++d) P[3 * q + d] = cm.xyz[3 * cm.tets[4 * E + q] + d];
    for (int q = 0; q < 4; ++q) {
      Locator::bary(P, &fm.xyz[3 * fm.tets[4 * e + q]], lam);
      if (std::min({lam[0], lam[1], lam[2], lam[3]}) < -1e-9) {
#pragma omp atomic
        bad[0]++;
      }
    }
    C.parent[e] = E;
  }
  if (bad[0]) throw HzError{1, "coarse mesh is not nested in the fine mesh"};
  // Z rows: coarse basis at each fine dof, evaluated in its element's parent
  const int64_t n = fs.n;
  std::vector<int64_t> first_elem(n, -1), first_loc(n, -1);
  for (int64_t e = 0; e < nef; ++e)
    for (int i = 0; i < NLOC; ++i) {
      int64_t g = fs.l2g[NLOC * e + i];
      if (first_elem[g] < 0) {
        first_elem[g] = e;
        first_loc[g] = i;
      }
    }
  std::vector<std::vector<std::pair<int32_t, double>>> rows(n);
#pragma omp parallel for schedule(static)
  for (int64_t g = 0; g < n; ++g) {
    int64_t E = C.parent[first_elem[g]];
    double P[12], lam[4], phi[NLOC];
    for (int q = 0; q < 4; ++q)
      for (int d = 0; d < 3; ++d) P[3 * q + d] = cm.xyz[3 * cm.tets[4 * E + q] + d];
    Locator::bary(P, &fs.coords[3 * g], lam);
    p3_basis(lam, phi);
    for (int J = 0; J < NLOC; ++J) {
      int64_t G = cs.l2g[NLOC * E + J];
      if (cs.dirichlet[G] || std::fabs(phi[J]) <= 1e-14) continue;
      rows[g].push_back({(int32_t)G, phi[J]});
    }
    std::sort(rows[g].begin(), rows[g].end());
  }
  CsrR& Z = C.Z;
  Z.nrows = n;
  Z.ncols = cs.n;
  Z.rowptr.assign(n + 1, 0);
  for (int64_t g = 0; g < n; ++g) Z.rowptr[g + 1] = Z.rowptr[g] + rows[g].size();
  Z.col.resize(Z.rowptr[n]);
  Z.val.resize(Z.rowptr[n]);
  for (int64_t g = 0; g < n; ++g)
    for (size_t q = 0; q < rows[g].size(); ++q) {
      Z.col[Z.rowptr[g] + q] = rows[g][q].first;
      Z.val[Z.rowptr[g] + q] = rows[g][q].second;
    }
  // Z^T
  CsrR& ZT = C.ZT;
  ZT.nrows = cs.n;
  ZT.ncols = n;
  ZT.rowptr.assign(cs.n + 1, 0);
  for (int64_t p = 0; p < Z.rowptr[n]; ++p) ZT.rowptr[Z.col[p] + 1]++;
  for (int64_t r = 0; r < cs.n; ++r) ZT.rowptr[r + 1] += ZT.rowptr[r];
  ZT.col.resize(Z.rowptr[n]);
  ZT.val.resize(Z.rowptr[n]);
  {
    std::vector<int64_t> f(ZT.rowptr.begin(), ZT.rowptr.end() - 1);
    for (int64_t g = 0; g < n; ++g)
      for (int64_t p = Z.rowptr[g]; p < Z.rowptr[g + 1]; ++p) {
        int64_t q = f[Z.col[p]]++;
        ZT.col[q] = (int32_t)g;
        ZT.val[q] = Z.val[p];
      }
  }
  // children per coarse element
  std::vector<std::vector<int64_t>> kids(nec);
  for (int64_t e = 0; e < nef; ++e) kids[C.parent[e]].push_back(e);
  // coarse partition and coarse squared slowness
  C.part.assign(nec, 0);
  C.mvals.assign(nec, 0.0);
  const P3Tables& T = p3_tables();
  for (int64_t E = 0; E < nec; ++E) {
    if (kids[E].empty()) throw HzError{1, "coarse element without fine elements"};
    double x[3] = {0, 0, 0};
    for (int q = 0; q < 4; ++q)
      for (int d = 0; d < 3; ++d) x[d] += 0.25 * cm.xyz[3 * cm.tets[4 * E + q] + d];
    int32_t best = INT32_MAX;
    double ms = 0.0, vs = 0.0;
    for (int64_t e : kids[E]) {
      double P[12], lam[4];
      for (int q = 0; q < 4; ++q)
        for (int d = 0; d < 3; ++d) P[3 * q + d] = fm.xyz[3 * fm.tets[4 * e + q] + d];
      if (Locator::bary(P, x, lam) && std::min({lam[0], lam[1], lam[2], lam[3]}) >= -1e-9)
        best = std::min(best, part_f[e]);
      double vol = elem_geom(P).vol;
      ms += vol * mvals_f[e];
      vs += vol;
    }
    if (best == INT32_MAX) throw HzError{1, "coarse centroid not located in its fine elements"};
    C.part[E] = best;
    C.mvals[E] = ms / vs;
  }
  // Galerkin coarse element matrices: sum over children of Z_e^T C_e Z_e
  std::vector<cplx> emat((size_t)nec * NLOC * NLOC, cplx(0, 0));
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t E = 0; E < nec; ++E) {
    double PE[12];
    for (int q = 0; q < 4; ++q)
      for (int d = 0; d < 3; ++d) PE[3 * q + d] = cm.xyz[3 * cm.tets[4 * E + q] + d];
    cplx* out = &emat[(size_t)E * NLOC * NLOC];
    for (int64_t e : kids[E]) {
      double P[12];
      for (int q = 0; q < 4; ++q)
        for (int d = 0; d < 3; ++d) P[3 * q + d] = fm.xyz[3 * fm.tets[4 * e + q] + d];
      ElemGeom g = elem_geom(P);
      const double me = mvals_f[e];
      cplx Ce[NLOC][NLOC];
      for (int i = 0; i < NLOC; ++i)
        for (int j = 0; j < NLOC; ++j) {
          double k = 0.0;
          for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) k += g.G[a][b] * T.S[a][b][i][j];
          Ce[i][j] = cplx(g.vol * (k - omega * omega * me * T.M[i][j]), 0.0);
        }
      for (int c = 0; c < 4; ++c)
        if (fm.nbr[4 * e + c] < 0 && fm.ftag[4 * e + c] == 0) {
          double s = -omega * std::sqrt(me) * face_area(P, c);
          for (int i = 0; i < NLOC; ++i)
            for (int j = 0; j < NLOC; ++j) Ce[i][j] += cplx(0.0, s * T.B[c][i][j]);
        }
      // Z_e[i][J] = coarse basis J at fine local node i
      double Ze[NLOC][NLOC];
      for (int i = 0; i < NLOC; ++i) {
        double x[3], lam[4];
        for (int d = 0; d < 3; ++d) {
          double s = 0.0;
          for (int a = 0; a < 4; ++a) s += P3_ALPHA[i][a] * P[3 * a + d];
          x[d] = s / 3.0;
        }
        Locator::bary(PE, x, lam);
        p3_basis(lam, Ze[i]);
      }
      // Fine Dirichlet rows/cols of A are identity: the kept coarse basis
      // vanishes on the Dirichlet plane, so they add nothing to E; the
      // coarse Dirichlet dofs get identity rows in the coarse assembly.
      cplx tmp[NLOC][NLOC];
      for (int i = 0; i < NLOC; ++i)
        for (int J = 0; J < NLOC; ++J) {
          cplx s(0, 0);
          for (int j = 0; j < NLOC; ++j)
            if (!fs.dirichlet[fs.l2g[NLOC * e + j]]) s += Ce[i][j] * Ze[j][J];
          tmp[i][J] = fs.dirichlet[fs.l2g[NLOC * e + i]] ? cplx(0, 0) : s;
        }
      for (int I = 0; I < NLOC; ++I)
        for (int J = 0; J < NLOC; ++J) {
          cplx s(0, 0);
          for (int i = 0; i < NLOC; ++i)
            if (!fs.dirichlet[fs.l2g[NLOC * e + i]]) s += Ze[i][I] * tmp[i][J];
          out[I * NLOC + J] += s;
        }
    }
  }
  AssemblyInput in;
  in.space = &cs;
  in.mesh = &cm;
  in.elems.resize(nec);
  std::iota(in.elems.begin(), in.elems.end(), 0);
  in.elem_mats = &emat;
  in.g2l.resize(cs.n);
  std::iota(in.g2l.begin(), in.g2l.end(), 0);
  in.nloc = cs.n;
  in.dir_local = cs.dirichlet;
  C.E = assemble(in);
  return C;
}

// ---------------------------------------------------------------------------
// Nested dissection with coordinate plane separators
// ---------------------------------------------------------------------------
FrontTree nd_symbolic(const CsrC& A, const std::vector<double>& X, int leaf) {
  const int64_t n = A.nrows;
  FrontTree T;
  T.n = n;
  std::vector<int32_t> mark(n, -1);
  int32_t epoch = 0;
  std::vector<std::vector<int32_t>> piv_lists;
  // returns front id (ids are created in postorder)
  std::function<int32_t(std::vector<int32_t>&)> build = [&](std::vector<int32_t>& S) -> int32_t {
    std::vector<int32_t> kids;
    std::vector<int32_t> sep;
    if ((int64_t)S.size() > leaf) {
      double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
      for (int32_t v : S)
        for (int d = 0; d < 3; ++d) {
          lo[d] = std::min(lo[d], X[3 * v + d]);
          hi[d] = std::max(hi[d], X[3 * v + d]);
        }
      int order[3] = {0, 1, 2};
      std::stable_sort(order, order + 3, [&](int a, int b) { return hi[a] - lo[a] > hi[b] - lo[b]; });
      bool split = false;
      for (int oi = 0; oi < 3 && !split; ++oi) {
        const int ax = order[oi];
        if (hi[ax] - lo[ax] <= 0) break;
        const double tol = 1e-9 * (hi[ax] - lo[ax]);
        std::vector<int32_t> s2(S);
        std::stable_sort(s2.begin(), s2.end(), [&](int32_t a, int32_t b) { return X[3 * a + ax] < X[3 * b + ax]; });
        std::vector<double> vals;
        for (int32_t v : s2) {
          double c = X[3 * v + ax];
          if (vals.empty() || c > vals.back() + tol) vals.push_back(c);
        }
        if (vals.size() < 2) continue;
        const double med = X[3 * s2[s2.size() / 2] + ax];
        size_t mi = std::lower_bound(vals.begin(), vals.end(), med - tol) - vals.begin();
        ++epoch;
        for (int32_t v : S) mark[v] = epoch;
        int64_t best_sz = -1;
        double best_c = 0, best_dist = 0;
        for (long q = (long)mi - 3; q <= (long)mi + 3; ++q) {
          if (q < 1 || q >= (long)vals.size()) continue;
          const double c = vals[q] - tol;
          int64_t sz = 0;
          for (int32_t v : S) {
            if (X[3 * v + ax] < c) continue;
            for (int64_t p = A.rowptr[v]; p < A.rowptr[v + 1]; ++p) {
              int32_t u = A.col[p];
              if (mark[u] == epoch && X[3 * u + ax] < c) {
                ++sz;
                break;
              }
            }
          }
          double dist = std::fabs((double)q - (double)mi);
          if (best_sz < 0 || sz < best_sz || (sz == best_sz && dist < best_dist)) {
            best_sz = sz;
            best_c = c;
            best_dist = dist;
          }
        }
        if (best_sz < 0) continue;
        std::vector<int32_t> L, R;
        for (int32_t v : S) {
          if (X[3 * v + ax] < best_c) {
            L.push_back(v);
            continue;
          }
          bool is_sep = false;
          for (int64_t p = A.rowptr[v]; p < A.rowptr[v + 1] && !is_sep; ++p) {
            int32_t u = A.col[p];
            is_sep = mark[u] == epoch && X[3 * u + ax] < best_c;
          }
          (is_sep ? sep : R).push_back(v);
        }
        if (L.empty() || R.empty()) {
          sep.clear();
          continue;
        }
        split = true;
        kids.push_back(build(L));
        kids.push_back(build(R));
      }
      if (!split) sep = S;
    } else {
      sep = S;
    }
    std::sort(sep.begin(), sep.end());
    int32_t id = (int32_t)piv_lists.size();
    piv_lists.push_back(sep);
    T.children.push_back(kids);
    return id;
  };
  std::vector<int32_t> all(n);
  std::iota(all.begin(), all.end(), 0);
  int32_t root = build(all);
  (void)root;
  const int32_t nf = (int32_t)piv_lists.size();
  T.k.resize(nf);
  T.m.resize(nf);
  T.parent.assign(nf, -1);
  T.height.assign(nf, 0);
  T.piv_begin.resize(nf);
  T.perm.resize(n);
  T.pos.resize(n);
  int64_t p = 0;
  for (int32_t t = 0; t < nf; ++t) {
    T.piv_begin[t] = p;
    T.k[t] = (int32_t)piv_lists[t].size();
    for (int32_t v : piv_lists[t]) {
      T.perm[p] = v;
      T.pos[v] = (int32_t)p;
      ++p;
    }
    for (int32_t c : T.children[t]) {
      T.parent[c] = t;
      T.height[t] = std::max(T.height[t], T.height[c] + 1);
    }
  }
  // update rows: neighbours of the pivots and the children's update rows
  // that are eliminated after this front, ascending elimination position
  std::vector<std::vector<int32_t>> U(nf);
  for (int32_t t = 0; t < nf; ++t) {
    const int64_t last = T.piv_begin[t] + T.k[t] - 1;
    std::vector<int32_t> s;
    for (int64_t q = T.piv_begin[t]; q <= last; ++q) {
      int32_t v = T.perm[q];
      for (int64_t e = A.rowptr[v]; e < A.rowptr[v + 1]; ++e)
        if (T.pos[A.col[e]] > last) s.push_back(T.pos[A.col[e]]);
    }
    for (int32_t c : T.children[t])
      for (int32_t u : U[c])
        if (u > last) s.push_back(u);
    std::sort(s.begin(), s.end());
    s.erase(std::unique(s.begin(), s.end()), s.end());
    U[t] = s;
    T.m[t] = (int32_t)s.size();
  }
  T.upd_ptr.assign(nf + 1, 0);
  for (int32_t t = 0; t < nf; ++t) T.upd_ptr[t + 1] = T.upd_ptr[t] + T.m[t];
  T.upd.resize(T.upd_ptr[nf]);
  for (int32_t t = 0; t < nf; ++t)
    for (int32_t q = 0; q < T.m[t]; ++q) T.upd[T.upd_ptr[t] + q] = T.perm[U[t][q]];
  return T;
}

}  // namespace hz
