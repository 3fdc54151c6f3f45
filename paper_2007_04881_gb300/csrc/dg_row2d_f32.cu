// dg_row2d_f32.cu -- 2D row kernels (float contractions), degrees 1..6.
#include "dg_launch.cuh"

namespace dg {

int launch_row2d_f32(const DevMesh& m, int mode, float* vals, float* rhs, int sm_count, const LaunchOpts& lo0, Tracer* tr) {
  LaunchOpts lo = lo0;
  iface_setup<2, float>(m, mode, lo, tr);
  int n = 0;
  n += launch_row_p<2, 1, float>(m, mode, vals, rhs, sm_count, lo, tr);
  n += launch_row_p<2, 2, float>(m, mode, vals, rhs, sm_count, lo, tr);
  n += launch_row_p<2, 3, float>(m, mode, vals, rhs, sm_count, lo, tr);
  n += launch_row_p<2, 4, float>(m, mode, vals, rhs, sm_count, lo, tr);
  n += launch_row_p<2, 5, float>(m, mode, vals, rhs, sm_count, lo, tr);
  n += launch_row_p<2, 6, float>(m, mode, vals, rhs, sm_count, lo, tr);
  n += launch_iface_all<2, float>(m, vals, sm_count, lo, tr);
  return n;
}

namespace {
// variants 0 .. tile_variants - 1 of the row kernel; 3 = the persistent
// pass's tiles
template <int D, int P, typename T>
int tm_of(int v) {
  if (v == 3) return tile_tm<D, P, T>(3);
  return v < tile_variants<D, P, T>() ? tile_tm<D, P, T>(v) : 0;
}
template <int D, typename T>
int tm_dim(int p, int v) {
  switch (p) {
    case 1: return tm_of<D, 1, T>(v);
    case 2: return tm_of<D, 2, T>(v);
    case 3: return tm_of<D, 3, T>(v);
    case 4: return tm_of<D, 4, T>(v);
    case 5: if constexpr (D == 2) return tm_of<D, 5, T>(v); return 0;
    case 6: if constexpr (D == 2) return tm_of<D, 6, T>(v); return 0;
    default: return 0;
  }
}
}  // namespace

// the tensor-core forms have one contraction layout per degree
int row_tile_tm(int dim, int p, int prec, int v) {
  if (prec == 0) return dim == 2 ? tm_dim<2, double>(p, v) : tm_dim<3, double>(p, v);
  if (prec == 1) return dim == 2 ? tm_dim<2, float>(p, v) : tm_dim<3, float>(p, v);
  return v == 0 ? -1 : 0;
}

}  // namespace dg
