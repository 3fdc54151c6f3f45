// dg_row2d_f32.cu -- 2D row kernels (float contractions), degrees 1..6.
#include "dg_launch.cuh"

namespace dg {

int launch_row2d_f32(const DevMesh& m, int mode, float* vals, float* rhs, int sm_count, const LaunchOpts& lo, Tracer* tr) {
  int n = 0;
  n += launch_row_p<2, 1, float>(m, mode, vals, rhs, sm_count, lo, tr);
  n += launch_row_p<2, 2, float>(m, mode, vals, rhs, sm_count, lo, tr);
  n += launch_row_p<2, 3, float>(m, mode, vals, rhs, sm_count, lo, tr);
  n += launch_row_p<2, 4, float>(m, mode, vals, rhs, sm_count, lo, tr);
  n += launch_row_p<2, 5, float>(m, mode, vals, rhs, sm_count, lo, tr);
  n += launch_row_p<2, 6, float>(m, mode, vals, rhs, sm_count, lo, tr);
  return n;
}

}  // namespace dg
