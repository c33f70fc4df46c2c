// Host-side setup structures of the Helmholtz / two-level ORAS library.
//
// Everything here runs once per (mesh, frequency) on the CPU: P3 dof
// numbering, element matrices, CSR assembly, overlapping subdomains, the
// coarse space and the nested-dissection symbolic analysis of the local
// matrices. The per-iteration work runs in the CUDA kernels.
#pragma once

#include <complex>
#include <cstdint>
#include <string>
#include <vector>

namespace hz {

using cplx = std::complex<double>;

struct HzError {
  int code;
  std::string msg;
};

// ---------------------------------------------------------------------------
// Tet mesh with boundary faces
// ---------------------------------------------------------------------------
struct Mesh {
  int64_t nv = 0, ne = 0;
  std::vector<double> xyz;        // [nv][3]
  std::vector<int32_t> tets;      // [ne][4]
  std::vector<int32_t> bfaces;    // [nbf][3]
  std::vector<int32_t> btag;      // [nbf] 0 = Robin, 1 = Dirichlet
  // derived
  std::vector<int64_t> nbr;       // [ne][4] element across face c (opposite local vertex c), -1 outside
  std::vector<int8_t> ftag;       // [ne][4] -1 interior/unlisted, 0 Robin, 1 Dirichlet
};

void mesh_build_adjacency(Mesh& m);  // throws HzError

// ---------------------------------------------------------------------------
// P3 space
// ---------------------------------------------------------------------------
constexpr int NLOC = 20;

// local node c-th multi-index: vertices 0..3, edge nodes 4..15, face nodes 16..19
extern const int P3_ALPHA[NLOC][4];

struct P3Tables {
  double M[NLOC][NLOC];                 // int phi_i phi_j / |T|
  double S[4][4][NLOC][NLOC];           // int d_a phi_i d_b phi_j / |T|
  double B[4][NLOC][NLOC];              // int_{face c} phi_i phi_j / |f|
  int face_nodes[4][10];
};
const P3Tables& p3_tables();
void p3_basis(const double lam[4], double phi[NLOC]);

struct Space {
  int64_t n = 0;
  std::vector<int64_t> l2g;       // [ne][20] global dof (final, spatially sorted order)
  std::vector<double> coords;     // [n][3]
  std::vector<uint8_t> dirichlet; // [n]
};

// numbering: vertices, edges, faces, then a stable spatial sort
Space p3_space(const Mesh& m);

struct ElemGeom {
  double vol;        // |T|
  double G[4][4];    // grad lambda_a . grad lambda_b
};
ElemGeom elem_geom(const double* P /*[4][3]*/);
double face_area(const double* P, int c);

// ---------------------------------------------------------------------------
// CSR
// ---------------------------------------------------------------------------
struct CsrC {             // complex CSR
  int64_t nrows = 0, ncols = 0;
  std::vector<int64_t> rowptr;
  std::vector<int32_t> col;
  std::vector<cplx> val;
};
struct CsrR {             // real CSR
  int64_t nrows = 0, ncols = 0;
  std::vector<int64_t> rowptr;
  std::vector<int32_t> col;
  std::vector<double> val;
};

// Element contribution source for the generic assembler.
struct AssemblyInput {
  const Space* space = nullptr;
  const Mesh* mesh = nullptr;
  std::vector<int64_t> elems;          // elements to assemble
  std::vector<double> mvals;           // squared slowness per element (indexed by mesh element)
  double omega = 0.0;
  std::vector<int8_t> robin_face;      // [ne][4] 1 -> add -i w sqrt(m) B_f on that face
  std::vector<int64_t> g2l;            // global dof -> row index (-1 absent), size space->n
  int64_t nloc = 0;
  std::vector<uint8_t> dir_local;      // [nloc] identity rows/cols
  // optional override of element matrices (complex, [elems.size()][20][20]) and element dof map
  const std::vector<cplx>* elem_mats = nullptr;
};
CsrC assemble(const AssemblyInput& in);
void split_re_im(const CsrC& A, CsrR& re, CsrR& im);  // im keeps rows with nonzero imaginary part

// ---------------------------------------------------------------------------
// Domain decomposition
// ---------------------------------------------------------------------------
struct Subdomain {
  std::vector<int64_t> elems;     // overlapping element set
  std::vector<int64_t> dofs;      // global dofs, ascending
  std::vector<uint8_t> owned;     // D_i (Boolean)
  CsrC A;                         // local Robin matrix
};

struct FrontTree {               // symbolic multifrontal structure of one local matrix
  int64_t n = 0;
  std::vector<int32_t> perm;      // elimination position -> local row
  std::vector<int32_t> pos;       // local row -> elimination position
  // per front
  std::vector<int32_t> k, m, parent, height;
  std::vector<int64_t> piv_begin; // pivots are perm[piv_begin .. piv_begin + k)
  std::vector<int64_t> upd_ptr;   // update rows (local rows) in upd[upd_ptr[t] .. upd_ptr[t+1])
  std::vector<int32_t> upd;
  std::vector<std::vector<int32_t>> children;
};
FrontTree nd_symbolic(const CsrC& A, const std::vector<double>& coords /*[n][3]*/, int leaf);

struct Level {                   // one level (fine or coarse) of the preconditioner
  Space space;
  std::vector<Subdomain> subs;
  std::vector<FrontTree> trees;
};

}  // namespace hz
