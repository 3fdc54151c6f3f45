// dg_persist3d_f32.cu -- the FP32 persistent pass over 3D meshes of every degree, and the dispatch of both dimensions.
#include "dg_persist.cuh"

namespace dg {

int launch_persist2d_f32_p4(const DevMesh&, float*, float*, const PersistArgs&, int, cudaStream_t);
int launch_persist2d_f32_p5(const DevMesh&, float*, float*, const PersistArgs&, int, cudaStream_t);

int launch_persist2d_f32(const DevMesh& m, float* vals, float* rhs, const PersistArgs& a, int pmax, int sm_count,
                         cudaStream_t st) {
  if (pmax <= 4) return launch_persist2d_f32_p4(m, vals, rhs, a, sm_count, st);
  if (pmax == 5) return launch_persist2d_f32_p5(m, vals, rhs, a, sm_count, st);
  return -1;  // degree 6: not compiled into the persistent pass
}

int launch_persist3d_f32(const DevMesh& m, float* vals, float* rhs, const PersistArgs& a, int pmax, int sm_count,
                         cudaStream_t st) {
  if (pmax <= 3) return launch_persist_pmax<3, float, 3>(m, vals, rhs, a, sm_count, st);
  return -1;  // degree 4: not compiled into the persistent pass
}

namespace {
template <int D, int P>
void layout_p(int* mask, int* gmom, int* grow) {
  if constexpr (P <= (D == 2 ? kPMax2 : kPMax3)) {
    // 3D degree 2 keeps the per-point volume terms in the persistent pass:
    // inlined there, its moment tile gave one wrong diagonal entry (the
    // (2,0,0) x (2,0,0) one) on the GPU while the per-degree moment launch
    // is exact; the row tile's volume terms are exact
    if (persist_mom_ok<D, P, float>() && !(D == 3 && P == 2)) *mask |= 1 << P;
    gmom[P] = MomCfg<D, P, float>::G;
    grow[P] = TileCfg<D, P, float, persist_tv<D, P, float>()>::G;
    layout_p<D, P + 1>(mask, gmom, grow);
  }
}
__global__ void wait_probe_kernel(const int* flag, int* status, long long limit_ns) {
  if (threadIdx.x == 0 && !wait_flag(flag, limit_ns)) atomicOr(status, 1);
}
}  // namespace

int persist_layout(int dim, int* mom_ok_mask, int* gmom, int* grow) {
  *mom_ok_mask = 0;
  for (int p = 0; p < 9; ++p) gmom[p] = grow[p] = 0;
  if (dim == 2)
    layout_p<2, 1>(mom_ok_mask, gmom, grow);
  else
    layout_p<3, 1>(mom_ok_mask, gmom, grow);
  return dim == 2 ? 5 : 3;  // the highest degree a persistent pass serves
}

void launch_wait_probe(const int* flag, int* status, long long limit_ns, cudaStream_t st) {
  wait_probe_kernel<<<1, 32, 0, st>>>(flag, status, limit_ns);
}

}  // namespace dg
