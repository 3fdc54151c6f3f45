// dg_varcoef.cu -- launch of the variable-coefficient terms (dg_varcoef.cuh)
// in the contraction type of the pass.
#include "dg_varcoef_kernel.cuh"

namespace dg {

int launch_varcoef(const DevMesh& m, const VcFields& f, bool fp32, void* vals, void* rhs, int sm_count,
                   cudaStream_t st) {
  if (m.ne <= 0) return 0;
  if (fp32)
    return launch_varcoef_f32(m, f, static_cast<float*>(vals), static_cast<float*>(rhs), sm_count, st);
  return launch_varcoef_f64(m, f, static_cast<double*>(vals), static_cast<double*>(rhs), sm_count, st);
}

}  // namespace dg
