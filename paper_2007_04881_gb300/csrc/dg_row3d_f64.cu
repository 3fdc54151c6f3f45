// dg_row3d_f64.cu -- 3D row kernels (double contractions), degrees 1..4.
#include "dg_launch.cuh"

namespace dg {

int launch_row3d_f64(const DevMesh& m, int mode, double* vals, double* rhs, int sm_count, const LaunchOpts& lo, Tracer* tr) {
  int n = 0;
  n += launch_row_p<3, 1, double>(m, mode, vals, rhs, sm_count, lo, tr);
  n += launch_row_p<3, 2, double>(m, mode, vals, rhs, sm_count, lo, tr);
  n += launch_row_p<3, 3, double>(m, mode, vals, rhs, sm_count, lo, tr);
  n += launch_row_p<3, 4, double>(m, mode, vals, rhs, sm_count, lo, tr);
  return n;
}

}  // namespace dg
