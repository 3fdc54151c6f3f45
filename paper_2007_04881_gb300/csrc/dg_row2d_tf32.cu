// dg_row2d_tf32.cu -- 2D row kernels with 3xTF32 tensor-core contractions, degrees 1..6.
#include "dg_launch.cuh"
#include "dg_mma.cuh"

namespace dg {

int launch_row2d_tf32(const DevMesh& m, int mode, float* vals, float* rhs, int sm_count, const LaunchOpts& lo, Tracer* tr) {
  int n = 0;
  n += launch_row_mma_p<2, 1, kMmaTf32>(m, mode, vals, rhs, sm_count, lo, tr);
  n += launch_row_mma_p<2, 2, kMmaTf32>(m, mode, vals, rhs, sm_count, lo, tr);
  n += launch_row_mma_p<2, 3, kMmaTf32>(m, mode, vals, rhs, sm_count, lo, tr);
  n += launch_row_mma_p<2, 4, kMmaTf32>(m, mode, vals, rhs, sm_count, lo, tr);
  n += launch_row_mma_p<2, 5, kMmaTf32>(m, mode, vals, rhs, sm_count, lo, tr);
  n += launch_row_mma_p<2, 6, kMmaTf32>(m, mode, vals, rhs, sm_count, lo, tr);
  return n;
}

}  // namespace dg
