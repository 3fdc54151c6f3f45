// dg_launch.cuh -- launch helper for the templated row kernel: one
// persistent launch per polynomial degree (the degree grouping of Sec. 3.1),
// grid sized to the number of co-resident CTAs.
#pragma once

#include <cstdio>

#include "dg_device.cuh"
#include "dg_iface.cuh"
#include "dg_moment.cuh"

namespace dg {

template <typename K>
inline int resident_grid(K kernel, size_t smem, int sm_count, int want_blocks, int occ_cap = 0) {
  int occ = 0;
  if (smem > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, kWarps * 32, smem);
  if (occ_cap > 0 && occ > occ_cap) occ = occ_cap;
  if (occ < 1) occ = 1;
  int g = occ * sm_count;
  return want_blocks < g ? want_blocks : g;
}

// The row-kernel launch of one degree group with tile variant V (kind: the
// tracer's accounting kind, 0 whole rows, 4 off-diagonal blocks next to the
// moment launch).
template <int D, int P, typename T, int V>
int launch_row_tile(const DevMesh& m, int mode, T* vals, T* rhs, int sm_count, const LaunchOpts& lo, Tracer* tr,
                    int kind) {
  const int count = m.elem_pstart[P + 1] - m.elem_pstart[P];
  cudaStream_t st = lo.pst[P];
  if (tr && tr->on) {
    char name[48];
    snprintf(name, sizeof name, "row%dd_p%d_%s", D, P, sizeof(T) == 8 ? "f64" : "f32");
    // the lane kernel's own launch with the interface kernel on: its rows
    // less the interface launch's blocks (kind 6); next to a moment launch it
    // is the off-diagonal launch (kind 4)
    const bool lane_if = TileCfg<D, P, T, V>::TPE == 1 && ((lo.imask >> P) & 1) && kind == 0;
    tr->begin(name, lane_if ? 6 : kind, P, sizeof(T), st);
  }
  if constexpr (TileCfg<D, P, T, V>::TPE == 1) {
    // a few lanes per element, no staging; the blocks of interfaces whose
    // larger degree is in imask come from the interface launch, and when
    // that leaves none (no neighbour degree above P outside imask) only the
    // diagonal part is launched
    if ((lo.imask >> P) & 1) {
      mode |= lo.imask << kModeMaskShift;
      if (!(lo.present & ~lo.imask & ~((2 << P) - 1))) mode |= kModeDiagOnly;
    }
    if (mode & kModeDiagOnly) {
      auto k = row_lane_kernel<D, P, T, 1>;
      const int grid = resident_grid(k, 0, sm_count, lane_blocks<D, P, T>(count, 1), lo.occ_cap);
      k<<<grid, kWarps * 32, 0, st>>>(m, mode, vals, rhs);
    } else {
      auto k = row_lane_kernel<D, P, T, 2>;
      const int grid = resident_grid(k, 0, sm_count, lane_blocks<D, P, T>(count, 2), lo.occ_cap);
      k<<<grid, kWarps * 32, 0, st>>>(m, mode, vals, rhs);
    }
  } else {
    using SM = RowSmem<D, P, T, V>;
    constexpr int G = TileCfg<D, P, T, V>::G;
    static_assert(SM::total(kWarps, nbasis(D, D == 2 ? kPMax2 : kPMax3)) <= 227 * 1024,
                  "row kernel shared memory exceeds 227 KB");
    const int ntiles = (count + G - 1) / G;
    const size_t smem = SM::total(kWarps, m.nmax);
    auto k = row_kernel<D, P, T, V>;
    const int grid = resident_grid(k, smem, sm_count, (ntiles + kWarps - 1) / kWarps, lo.occ_cap);
    k<<<grid, kWarps * 32, smem, st>>>(m, mode, vals, rhs);
  }
  if (tr && tr->on) tr->end(st);
  return 1;
}

// Tile variants beyond the default, compiled in their own translation units
// (dg_row*_tiles*.cu) so that the build runs them in parallel.
#define DG_ROW_TILE_VARIANTS(X)                                                                               \
  X(2, 3, float, 1) X(2, 4, float, 1) X(2, 4, float, 2) X(2, 5, float, 1) X(2, 5, float, 2) X(2, 6, float, 1) \
  X(3, 2, float, 1) X(3, 3, float, 1) X(3, 3, float, 2)
#define DG_EXTERN_ROW_TILE(D, P, T, V) \
  extern template int launch_row_tile<D, P, T, V>(const DevMesh&, int, T*, T*, int, const LaunchOpts&, Tracer*, int);
DG_ROW_TILE_VARIANTS(DG_EXTERN_ROW_TILE)

template <int D, int P, typename T>
inline int launch_row_range(const DevMesh& m, int mode, T* vals, T* rhs, int sm_count, const LaunchOpts& lo,
                            Tracer* tr);

// the row-kernel launch in the tile variant lo.tile[P]
template <int D, int P, typename T>
inline int launch_row_variant(const DevMesh& m, int mode, T* vals, T* rhs, int sm_count, const LaunchOpts& lo,
                              Tracer* tr, int kind) {
  constexpr int NV = tile_variants<D, P, T>();
  const int v = lo.tile[P] < NV ? lo.tile[P] : 0;
  if constexpr (NV > 2)
    if (v == 2) return launch_row_tile<D, P, T, 2>(m, mode, vals, rhs, sm_count, lo, tr, kind);
  if constexpr (NV > 1)
    if (v == 1) return launch_row_tile<D, P, T, 1>(m, mode, vals, rhs, sm_count, lo, tr, kind);
  return launch_row_tile<D, P, T, 0>(m, mode, vals, rhs, sm_count, lo, tr, kind);
}

// One degree group: in lo.split[P] parts of equal element count, each a copy
// of the mesh view whose range [elem_pstart[P], elem_pstart[P+1]) is the
// part's (every kernel takes its elements from that range), on its own stream.
template <int D, int P, typename T>
inline int launch_row_p(const DevMesh& m, int mode, T* vals, T* rhs, int sm_count, const LaunchOpts& lo, Tracer* tr) {
  const int count = m.elem_pstart[P + 1] - m.elem_pstart[P];
  if (count <= 0) return 0;
  int parts = lo.split[P] < 1 ? 1 : lo.split[P] > kMaxSplit ? kMaxSplit : lo.split[P];
  if (parts > count) parts = count;  // no empty part
  if (parts == 1) return launch_row_range<D, P, T>(m, mode, vals, rhs, sm_count, lo, tr);
  int n = 0;
  const int base = m.elem_pstart[P];
  for (int i = 0; i < parts; ++i) {
    DevMesh mp = m;
    mp.elem_pstart[P] = base + (int)((int64_t)count * i / parts);
    mp.elem_pstart[P + 1] = base + (int)((int64_t)count * (i + 1) / parts);
    if (mp.elem_pstart[P + 1] <= mp.elem_pstart[P]) continue;
    LaunchOpts lp = lo;
    if (lo.part[P][i]) lp.pst[P] = lo.part[P][i];
    if (tr) tr->scale = (double)(mp.elem_pstart[P + 1] - mp.elem_pstart[P]) / count;
    n += launch_row_range<D, P, T>(mp, mode, vals, rhs, sm_count, lp, tr);
  }
  if (tr) tr->scale = 1.0;
  return n;
}

template <int D, int P, typename T>
inline int launch_row_range(const DevMesh& m, int mode, T* vals, T* rhs, int sm_count, const LaunchOpts& lo,
                            Tracer* tr) {
  const int count = m.elem_pstart[P + 1] - m.elem_pstart[P];
  if (count <= 0) return 0;
  cudaStream_t st = lo.pst[P];
  const char* tn = sizeof(T) == 8 ? "f64" : "f32";
  int n = 0, kind = 0;
  // every degree the moment path serves takes it, the lane kernel's degree 2
  // (2D FP32) included: its off-diagonal blocks come from the interface launch
  if constexpr (moment_volume_ok<D, P, T>()) {
    // the moment path needs the linearisation tables of the rule set
    if (lo.vol_moments && m.rt.lin32 && m.rt.lin64 && (mode & (kModeVol | kModeFace | kModeRhs))) {
      // volume and own-face terms through the moments (the diagonal block and
      // the load vector complete), then the off-diagonal blocks by the row
      // kernel, which no longer reads what the moment launch writes
      using MC = MomCfg<D, P, T>;
      static_assert(MC::total <= 227 * 1024, "moment kernel shared memory exceeds 227 KB");
      if (tr && tr->on) {
        char name[48];
        snprintf(name, sizeof name, "row%dd_vol_p%d_%s", D, P, tn);
        tr->begin(name, 3, P, sizeof(T), st);
      }
      auto k = vol_moment_kernel<D, P, T>;
      const int ngroups = (count + MC::G - 1) / MC::G;
      const int grid = resident_grid(k, MC::total, sm_count, (ngroups + kWarps - 1) / kWarps, lo.occ_cap);
      const int xm = lo.vol_exact ? kModeExactMom : 0;
      k<<<grid, kWarps * 32, MC::total, st>>>(
          m, (mode & (kModeVol | kModeFace | kModeRhs | kModeAccum)) | xm | kModeMomFace, vals, rhs);
      if (tr && tr->on) tr->end(st);
      ++n;
      if (!(mode & kModeFace)) return n;
      // the off-diagonal blocks: those of interfaces whose larger degree is in
      // imask come from the interface launch (launch_iface_all), the rest
      // (neighbours of a higher degree outside imask) from here
      if ((lo.imask >> P) & 1 && !(lo.present & ~lo.imask & ~((2 << P) - 1))) return n;
      mode = kModeFace | kModeSkipVol | kModeOffDiag | (lo.imask << kModeMaskShift);
      kind = 4;
    }
  }
  return n + launch_row_variant<D, P, T>(m, mode, vals, rhs, sm_count, lo, tr, kind);
}

// whether the interface kernel serves degree P: the FP32 degrees of the
// moment path, whose moment launch completes the diagonal blocks (a pass off
// the moment path leaves every block to the row and lane kernels)
template <int D, int P, typename T>
__host__ __device__ constexpr bool iface_rows() {
  return sizeof(T) == 4 && moment_volume_ok<D, P, T>();
}

// lo.present and lo.imask of one pass (interfaces by the interface kernel:
// FP32, moment path, face terms requested)
template <int D, typename T>
inline void iface_setup(const DevMesh& m, int mode, LaunchOpts& lo, Tracer* tr) {
  lo.present = m.pmask;  // the neighbours' degrees count: ghost elements of a partition
  lo.imask = 0;
  if (sizeof(T) == 4 && lo.iface && lo.vol_moments && m.rt.lin32 && m.rt.lin64 && (mode & kModeFace)) {
    if (iface_rows<D, 1, T>()) lo.imask |= 1 << 1;
    if (iface_rows<D, 2, T>()) lo.imask |= 1 << 2;
    if (iface_rows<D, 3, T>()) lo.imask |= 1 << 3;
    if (iface_rows<D, 4, T>()) lo.imask |= 1 << 4;
    if (D == 2 && iface_rows<D, 5, T>()) lo.imask |= 1 << 5;
    if (D == 2 && iface_rows<D, 6, T>()) lo.imask |= 1 << 6;
  }
  if (tr) tr->imask = lo.imask;
}

// The interface launches of larger degree P: if_perm[if_pstart[P] ..
// if_pstart[P + 1]) in lo.split[P] contiguous parts on the group's streams.
template <int D, int P, typename T>
inline int launch_iface_p(const DevMesh& m, T* vals, int sm_count, const LaunchOpts& lo, Tracer* tr) {
  if constexpr (!iface_rows<D, P, T>()) {
    return 0;
  } else {
    if (!((lo.imask >> P) & 1)) return 0;
    const int b = m.if_pstart[P], count = m.if_pstart[P + 1] - b;
    if (count <= 0) return 0;
    using Cfg = IfaceCfg<D, P, T>;
    static_assert(Cfg::total(kWarps) <= 227 * 1024, "interface kernel shared memory exceeds 227 KB");
    int parts = lo.split[P] < 1 ? 1 : lo.split[P] > kMaxSplit ? kMaxSplit : lo.split[P];
    if (parts > count) parts = count;
    auto k = iface_kernel<D, P, T>;
    const size_t smem = Cfg::total(kWarps);
    int n = 0;
    for (int i = 0; i < parts; ++i) {
      const int i0 = b + (int)((int64_t)count * i / parts), i1 = b + (int)((int64_t)count * (i + 1) / parts);
      cudaStream_t st = lo.part[P][i] ? lo.part[P][i] : lo.pst[P];
      if (tr && tr->on) {
        char name[48];
        snprintf(name, sizeof name, "row%dd_iface_p%d_f32", D, P);
        tr->scale = (double)(i1 - i0) / count;
        tr->begin(name, 5, P, sizeof(T), st);
        tr->scale = 1.0;
      }
      const int ntiles = (i1 - i0 + Cfg::G - 1) / Cfg::G;
      const int grid = resident_grid(k, smem, sm_count, (ntiles + kWarps - 1) / kWarps, lo.occ_cap);
      k<<<grid, kWarps * 32, smem, st>>>(m, lo.imask, i0, i1, vals);
      if (tr && tr->on) tr->end(st);
      ++n;
    }
    return n;
  }
}

template <int D, typename T>
inline int launch_iface_all(const DevMesh& m, T* vals, int sm_count, const LaunchOpts& lo, Tracer* tr) {
  if (!lo.imask) return 0;
  int n = 0;
  n += launch_iface_p<D, 1, T>(m, vals, sm_count, lo, tr);
  n += launch_iface_p<D, 2, T>(m, vals, sm_count, lo, tr);
  n += launch_iface_p<D, 3, T>(m, vals, sm_count, lo, tr);
  n += launch_iface_p<D, 4, T>(m, vals, sm_count, lo, tr);
  if constexpr (D == 2) {
    n += launch_iface_p<D, 5, T>(m, vals, sm_count, lo, tr);
    n += launch_iface_p<D, 6, T>(m, vals, sm_count, lo, tr);
  }
  return n;
}

}  // namespace dg
