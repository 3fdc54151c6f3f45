// dg_varcoef_f32.cu -- the variable-coefficient kernels in FP32 (geometry
// records, field table and basis in FP32, FP32 accumulation).
#include "dg_varcoef_kernel.cuh"

namespace dg {

int launch_varcoef_f32(const DevMesh& m, const VcFields& f, float* vals, float* rhs, int sm_count, cudaStream_t st) {
  return launch_varcoef_t<float>(m, f, vals, rhs, sm_count, st);
}

}  // namespace dg
