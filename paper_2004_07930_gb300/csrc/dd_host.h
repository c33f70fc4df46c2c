// Domain-decomposition and coarse-space setup (host).
#pragma once

#include "host.h"

namespace hz {

struct CoarseSpace {
  Space space;                  // coarse P3 space (coarse Dirichlet dofs get identity rows)
  CsrR Z, ZT;                   // fine <- coarse interpolation and its transpose
  CsrC E;                       // Galerkin coarse operator Z^T A Z
  std::vector<int64_t> parent;  // fine element -> coarse element
  std::vector<int32_t> part;    // coarse element -> subdomain
  std::vector<double> mvals;    // coarse squared slowness
};

CsrC assemble_global(const Mesh& m, const Space& sp, const std::vector<double>& mvals, double omega);
std::vector<Subdomain> build_subdomains(const Mesh& m, const Space& sp, const std::vector<int32_t>& part,
                                        int nparts, const std::vector<double>& mvals, double omega,
                                        int layers = 1);  // overlap: element layers grown by vertex sharing
CoarseSpace build_coarse(const Mesh& fm, const Space& fs, const std::vector<double>& mvals_f,
                         const std::vector<int32_t>& part_f, double omega, Mesh& cm);
void locate_points(const Mesh& m, const double* x, int64_t np, int64_t* elem, double* lam);

}  // namespace hz
