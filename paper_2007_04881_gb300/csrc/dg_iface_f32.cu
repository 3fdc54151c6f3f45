// dg_iface_f32.cu -- interface kernels (float contractions): the two
// off-diagonal blocks of every interface, grouped by the larger degree of
// the pair (Sec. 3.1).
#include "dg_launch.cuh"

namespace dg {

int launch_iface_f32(const DevMesh& m, float* vals, int sm_count, cudaStream_t st, Tracer* tr) {
  int n = 0;
  if (m.dim == 2) {
    n += launch_iface_p<2, 1, float>(m, vals, sm_count, st, tr);
    n += launch_iface_p<2, 2, float>(m, vals, sm_count, st, tr);
    n += launch_iface_p<2, 3, float>(m, vals, sm_count, st, tr);
    n += launch_iface_p<2, 4, float>(m, vals, sm_count, st, tr);
    n += launch_iface_p<2, 5, float>(m, vals, sm_count, st, tr);
    n += launch_iface_p<2, 6, float>(m, vals, sm_count, st, tr);
  } else {
    n += launch_iface_p<3, 1, float>(m, vals, sm_count, st, tr);
    n += launch_iface_p<3, 2, float>(m, vals, sm_count, st, tr);
    n += launch_iface_p<3, 3, float>(m, vals, sm_count, st, tr);
    n += launch_iface_p<3, 4, float>(m, vals, sm_count, st, tr);
  }
  return n;
}

}  // namespace dg
