// dg_varcoef.cuh -- variable advection and reaction fields (Sec. 4.2, and
// any affine b with a cubic c) added to a system the row kernels wrote with
// b = 0 and c = 0.
//
// The fields come from a table chosen per mesh (dg_mesh_set_fields):
//   b_d(x) = b0[d] + sum_e bx[d][e] x_e,   c(x) = sum_k c[k] m_k(x),
// m_k the graded monomials of total degree <= 3 in the order of DG_SRC_POLY
// (2D: the first 10).  The paper's test problem is b0 = (1, 1, 1), bx = I,
// c = 3 + prod_d x_d.
//
// The terms of Eq. (2.4) and Eq. (2.5) that carry b and c:
//   volume  sum_q W [ (b(x_q) . grad phi_j) phi_i + c(x_q) phi_j phi_i ],
//   faces   at every face point where row r's element is inflow,
//           b(x) . n_r < 0 with n_r out of r (b . n = 0 is outflow), except on
//           Neumann faces:
//             A_rr += -(b . n_r) phi^r_j phi^r_i,  A_r,nb += (b . n_r) phi^nb_j phi^r_i,
//   load    sum_q W (b . grad u + c u)(x_q) phi_i on the volume points and
//           -(b . n_r) g phi_i at the inflow points of Dirichlet boundary
//           faces (g = u).
// One warp per element row (dg_varcoef.cu): each lane stages one point of a
// chunk of 32 (its basis values U, its weighted field row V, its load term R)
// in shared memory, then 25 lanes contract the chunk into register tiles of
// the block, as the row kernels do.
#pragma once

#include "dg_internal.h"

namespace dg {

struct VcFields {
  double b0[3], bx[3][3], c[20];
  float b0f[3], bxf[3][3], cf[20];
  void round_copies() {
    for (int d = 0; d < 3; ++d) {
      b0f[d] = (float)b0[d];
      for (int e = 0; e < 3; ++e) bxf[d][e] = (float)bx[d][e];
    }
    for (int k = 0; k < 20; ++k) cf[k] = (float)c[k];
  }
};

// the fields of the paper's 3D test problem (Sec. 4.2), in dimension dim:
// b_d = 1 + x_d, c = 3 + prod_d x_d (graded monomial 4 in 2D, 15 in 3D)
inline VcFields vc_sec42_fields(int dim) {
  VcFields f{};
  for (int d = 0; d < 3; ++d) {
    f.b0[d] = d < dim ? 1.0 : 0.0;
    for (int e = 0; e < 3; ++e) f.bx[d][e] = d == e && d < dim ? 1.0 : 0.0;
  }
  f.c[0] = 3.0;
  f.c[dim == 2 ? 4 : 15] = 1.0;
  f.round_copies();
  return f;
}

// The b and c terms of every row of the mesh, added to vals (and rhs, may be
// null) in T = double (fp32 false) or float; one launch per degree group.
// Returns the number of launches.
int launch_varcoef(const DevMesh& m, const VcFields& f, bool fp32, void* vals, void* rhs, int sm_count,
                   cudaStream_t st);

}  // namespace dg
