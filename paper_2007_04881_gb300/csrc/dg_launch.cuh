// dg_launch.cuh -- launch helpers for the templated element / interface
// kernels: one persistent launch per polynomial degree (the degree grouping of
// Sec. 3.1), grid sized to the number of co-resident CTAs.
#pragma once

#include <cstdio>

#include "dg_device.cuh"

namespace dg {

template <typename K>
inline int resident_grid(K kernel, size_t smem, int sm_count, int want_blocks) {
  static_assert(sizeof(K) > 0, "");
  int occ = 0;
  if (smem > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, kWarps * 32, smem);
  if (occ < 1) occ = 1;
  int g = occ * sm_count;
  return want_blocks < g ? want_blocks : g;
}

template <int D, int P, typename T>
inline int launch_elem_p(const DevMesh& m, int mode, T* vals, T* rhs, int sm_count, cudaStream_t st, Tracer* tr) {
  const int count = m.elem_pstart[P + 1] - m.elem_pstart[P];
  if (count <= 0) return 0;
  constexpr int G = TileCfg<D, P>::G;
  const int ntiles = (count + G - 1) / G;
  static_assert(ElemSmem<D, P, T>::total(kWarps) <= 227 * 1024, "element kernel shared memory exceeds 227 KB");
  const size_t smem = ElemSmem<D, P, T>::total(kWarps);
  auto k = elem_kernel<D, P, T>;
  const int grid = resident_grid(k, smem, sm_count, (ntiles + kWarps - 1) / kWarps);
  if (tr && tr->on) {
    char name[48];
    snprintf(name, sizeof name, "elem%dd_p%d_%s", D, P, sizeof(T) == 8 ? "f64" : "f32");
    tr->begin(name, 0, P, sizeof(T), st);
  }
  k<<<grid, kWarps * 32, smem, st>>>(m, mode, vals, rhs);
  if (tr && tr->on) tr->end(st);
  return 1;
}

template <int D, int PM, typename T>
inline int launch_iface_p(const DevMesh& m, T* vals, int sm_count, cudaStream_t st, Tracer* tr) {
  const int count = m.if_pstart[PM + 1] - m.if_pstart[PM];
  if (count <= 0) return 0;
  static_assert(IfaceSmem<D, PM, T>::total(kWarps) <= 227 * 1024, "interface kernel shared memory exceeds 227 KB");
  const size_t smem = IfaceSmem<D, PM, T>::total(kWarps);
  auto k = iface_kernel<D, PM, T>;
  const int grid = resident_grid(k, smem, sm_count, (count + kWarps - 1) / kWarps);
  if (tr && tr->on) {
    char name[48];
    snprintf(name, sizeof name, "iface%dd_p%d_%s", D, PM, sizeof(T) == 8 ? "f64" : "f32");
    tr->begin(name, 1, PM, sizeof(T), st);
  }
  k<<<grid, kWarps * 32, smem, st>>>(m, vals);
  if (tr && tr->on) tr->end(st);
  return 1;
}

}  // namespace dg
