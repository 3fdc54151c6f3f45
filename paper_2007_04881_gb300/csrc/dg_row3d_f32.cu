// dg_row3d_f32.cu -- 3D row kernels (float contractions), degrees 1..4.
#include "dg_launch.cuh"

namespace dg {

int launch_row3d_f32(const DevMesh& m, int mode, float* vals, float* rhs, int sm_count, const LaunchOpts& lo0, Tracer* tr) {
  LaunchOpts lo = lo0;
  iface_setup<3, float>(m, mode, lo, tr);
  int n = 0;
  n += launch_row_p<3, 1, float>(m, mode, vals, rhs, sm_count, lo, tr);
  n += launch_row_p<3, 2, float>(m, mode, vals, rhs, sm_count, lo, tr);
  n += launch_row_p<3, 3, float>(m, mode, vals, rhs, sm_count, lo, tr);
  n += launch_row_p<3, 4, float>(m, mode, vals, rhs, sm_count, lo, tr);
  n += launch_iface_all<3, float>(m, vals, sm_count, lo, tr);
  return n;
}

}  // namespace dg
