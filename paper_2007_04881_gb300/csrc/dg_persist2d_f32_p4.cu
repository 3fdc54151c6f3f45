// dg_persist2d_f32_p4.cu -- the FP32 persistent pass over 2D meshes of degree <= 4.
#include "dg_persist.cuh"

namespace dg {

int launch_persist2d_f32_p4(const DevMesh& m, float* vals, float* rhs, const PersistArgs& a, int sm_count,
                            cudaStream_t st) {
  return launch_persist_pmax<2, float, 4>(m, vals, rhs, a, sm_count, st);
}

}  // namespace dg
