// dg_row3d_tf32.cu -- 3D row kernels with 3xTF32 tensor-core contractions, degrees 1..4.
#include "dg_launch.cuh"
#include "dg_mma.cuh"

namespace dg {

int launch_row3d_tf32(const DevMesh& m, int mode, float* vals, float* rhs, int sm_count, const LaunchOpts& lo, Tracer* tr) {
  int n = 0;
  n += launch_row_mma_p<3, 1, kMmaTf32>(m, mode, vals, rhs, sm_count, lo, tr);
  n += launch_row_mma_p<3, 2, kMmaTf32>(m, mode, vals, rhs, sm_count, lo, tr);
  n += launch_row_mma_p<3, 3, kMmaTf32>(m, mode, vals, rhs, sm_count, lo, tr);
  n += launch_row_mma_p<3, 4, kMmaTf32>(m, mode, vals, rhs, sm_count, lo, tr);
  return n;
}

}  // namespace dg
