// dg_varcoef_f64.cu -- the variable-coefficient kernels in FP64.
#include "dg_varcoef_kernel.cuh"

namespace dg {

int launch_varcoef_f64(const DevMesh& m, const VcFields& f, double* vals, double* rhs, int sm_count, cudaStream_t st) {
  return launch_varcoef_t<double>(m, f, vals, rhs, sm_count, st);
}

}  // namespace dg
