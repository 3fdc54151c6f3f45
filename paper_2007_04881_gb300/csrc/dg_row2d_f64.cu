// dg_row2d_f64.cu -- 2D row kernels (double contractions), degrees 1..6.
#include "dg_launch.cuh"

namespace dg {

int launch_row2d_f64(const DevMesh& m, int mode, double* vals, double* rhs, int sm_count, const LaunchOpts& lo, Tracer* tr) {
  int n = 0;
  n += launch_row_p<2, 1, double>(m, mode, vals, rhs, sm_count, lo, tr);
  n += launch_row_p<2, 2, double>(m, mode, vals, rhs, sm_count, lo, tr);
  n += launch_row_p<2, 3, double>(m, mode, vals, rhs, sm_count, lo, tr);
  n += launch_row_p<2, 4, double>(m, mode, vals, rhs, sm_count, lo, tr);
  n += launch_row_p<2, 5, double>(m, mode, vals, rhs, sm_count, lo, tr);
  n += launch_row_p<2, 6, double>(m, mode, vals, rhs, sm_count, lo, tr);
  return n;
}

}  // namespace dg
