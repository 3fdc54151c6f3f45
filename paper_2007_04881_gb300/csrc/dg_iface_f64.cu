// dg_iface_f64.cu -- interface kernels (double contractions): the two
// off-diagonal blocks of every interface, grouped by the larger degree of
// the pair (Sec. 3.1).
#include "dg_launch.cuh"

namespace dg {

int launch_iface_f64(const DevMesh& m, double* vals, int sm_count, cudaStream_t st, Tracer* tr) {
  int n = 0;
  if (m.dim == 2) {
    n += launch_iface_p<2, 1, double>(m, vals, sm_count, st, tr);
    n += launch_iface_p<2, 2, double>(m, vals, sm_count, st, tr);
    n += launch_iface_p<2, 3, double>(m, vals, sm_count, st, tr);
    n += launch_iface_p<2, 4, double>(m, vals, sm_count, st, tr);
    n += launch_iface_p<2, 5, double>(m, vals, sm_count, st, tr);
    n += launch_iface_p<2, 6, double>(m, vals, sm_count, st, tr);
  } else {
    n += launch_iface_p<3, 1, double>(m, vals, sm_count, st, tr);
    n += launch_iface_p<3, 2, double>(m, vals, sm_count, st, tr);
    n += launch_iface_p<3, 3, double>(m, vals, sm_count, st, tr);
    n += launch_iface_p<3, 4, double>(m, vals, sm_count, st, tr);
  }
  return n;
}

}  // namespace dg
