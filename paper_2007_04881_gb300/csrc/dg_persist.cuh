// dg_persist.cuh -- the persistent pass: one launch over a work list.
//
// The per-degree launches of the row pass (Sec. 3.1 groups elements by
// degree, one launch per group) leave the GPU to balance the groups, and on
// the moment path each group is two launches in a row (the moment kernel
// writes the diagonal blocks and the volume load vector, the faces-only row
// kernel adds to them).  The persistent pass instead launches one kernel
// with as many CTAs as fit on the GPU at once; each warp takes the next item
// of a work list (an atomic counter) until the list is done.  An item is one
// tile of one degree group: a moment tile (the volume terms of G elements)
// or a row tile (the faces, off-diagonal blocks and, off the moment path,
// the volume terms of G elements).  The host orders the list: every moment
// tile first, then the row tiles, each part by estimated work, largest
// first.  A row tile that adds to an element's diagonal block waits for the
// element's flag, set by its moment tile; since every moment tile is taken
// before any row tile and runs without waiting, each wait ends once a
// running warp finishes, and the wait is bounded (WaitCtl) all the same.
// Every element is computed by the same tile code as in the per-degree
// launches, so results do not depend on the list's order; with tiles of the
// same shape they are bitwise equal to them.
#pragma once

#include "dg_launch.cuh"

namespace dg {

// tile variant of degree P in the persistent pass
template <int D, int P, typename T>
__host__ __device__ constexpr int persist_tv() {
  return 3;
}
// whether degree P can take the moment path in the persistent pass (the
// degrees that take it in the per-degree launches)
template <int D, int P, typename T>
__host__ __device__ constexpr bool persist_mom_ok() {
  return TileCfg<D, P, T>::TPE != 1 && moment_volume_ok<D, P, T>();
}

template <int D, typename T>
struct PersistHead {
  static constexpr int NMAXC = nbasis(D, D == 2 ? kPMax2 : kPMax3);
  static constexpr int NLIN = MomCfg<D, 2, T>::NLIN;
  // volume rules of degrees 1..pmax (the packed global table), basis scales,
  // linearisation tables, then the basis exponents (int [NMAXC][3])
  __host__ __device__ static constexpr size_t bytes(int nrule_vals) {
    return align_up(sizeof(T) * ((size_t)nrule_vals + NMAXC + NLIN), 16) + align_up(sizeof(int) * 3 * NMAXC, 16);
  }
};

template <int D, typename T, int P, int PMAX>
__device__ __forceinline__ void persist_item(const DevMesh& m, T* vals, T* rhs, const PersistArgs& a, int4 w,
                                             const T* rules, const T* ctab, const T* lin, const int* alf,
                                             unsigned char* wb, const WaitCtl* wc) {
  if constexpr (P <= PMAX) {
    if (w.y == P) {
      const T* rule = rules + (size_t)m.rt.vol_off[P] * (D + 1);
      const bool mom = (a.mom_mask >> P) & 1;
      if constexpr (persist_mom_ok<D, P, T>()) {
        if (w.x == 1) {
          mom_tile<D, P, T>(m, (a.mode & (kModeVol | kModeRhs)) | a.exact, vals, rhs, w.z, lin, rule, ctab, alf,
                            reinterpret_cast<T*>(wb), wc);
          return;
        }
      }
      const int mode = mom ? (a.mode & ~kModeVol) | kModeSkipVol | ((a.mode & kModeVol) ? kModeAccum : 0) : a.mode;
      row_tile<D, P, T, persist_tv<D, P, T>()>(m, mode, vals, rhs, w.z, rule, ctab, wb, wc);
      return;
    }
    persist_item<D, T, P + 1, PMAX>(m, vals, rhs, a, w, rules, ctab, lin, alf, wb, wc);
  }
}

template <int D, typename T, int PMAX>
__global__ void __launch_bounds__(kWarps * 32)
    persist_kernel(const DevMesh m, T* __restrict__ vals, T* __restrict__ rhs, const PersistArgs a) {
  using H = PersistHead<D, T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nrule = (m.rt.vol_off[PMAX] + m.rt.vol_n[PMAX]) * (D + 1);
  T* rules = reinterpret_cast<T*>(smem_raw);
  T* ctab = rules + nrule;
  T* lin = ctab + H::NMAXC;
  int* alf = reinterpret_cast<int*>(smem_raw + align_up(sizeof(T) * ((size_t)nrule + H::NMAXC + H::NLIN), 16));
  const T* grule = pick<T>(m.rt.vol64, m.rt.vol32);
  for (int i = threadIdx.x; i < nrule; i += blockDim.x) rules[i] = grule[i];
  fill_ctab<D, T>(ctab, H::NMAXC);
  if (a.mom_mask) {
    const T* glin = pick<T>(m.rt.lin64, m.rt.lin32);
    for (int i = threadIdx.x; i < H::NLIN; i += blockDim.x) lin[i] = glin[i];
  }
  for (int i = threadIdx.x; i < H::NMAXC; i += blockDim.x) {
    int al[3] = {0, 0, 0};
    basis_alpha<D>(i, al);
    alf[3 * i] = al[0];
    alf[3 * i + 1] = al[1];
    alf[3 * i + 2] = al[2];
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* wb = smem_raw + H::bytes(nrule) + (size_t)warp * a.warp_bytes;
  const WaitCtl wc{a.vdone, a.status, a.limit_ns};
  for (;;) {
    int it = 0;
    if (lane == 0) it = atomicAdd(a.queue, 1);
    it = __shfl_sync(0xffffffffu, it, 0);
    if (it >= a.nitems) break;
    const int4 w = a.items[it];
    __syncwarp();
    persist_item<D, T, 1, PMAX>(m, vals, rhs, a, w, rules, ctab, lin, alf, wb, &wc);
  }
}

// shared memory per warp: the largest tile of degrees 1..pmax present
template <int D, typename T, int P, int PMAX>
inline size_t persist_warp_bytes(const DevMesh& m, int mom_mask) {
  if constexpr (P > PMAX) {
    return 0;
  } else {
    size_t b = 0;
    if (m.elem_pstart[P + 1] > m.elem_pstart[P]) {
      using SM = RowSmem<D, P, T, persist_tv<D, P, T>()>;
      b = SM::warp_bytes(SM::vs(m.nmax));
      if constexpr (persist_mom_ok<D, P, T>()) {
        if ((mom_mask >> P) & 1) {
          using MC = MomCfg<D, P, T>;
          const size_t mb = align_up(sizeof(T) * (size_t)MC::G * MC::PER_ELEM, 16);
          b = b > mb ? b : mb;
        }
      }
    }
    const size_t r = persist_warp_bytes<D, T, P + 1, PMAX>(m, mom_mask);
    return b > r ? b : r;
  }
}

// Launch the persistent pass on st (the queue and flags already zeroed).
// Returns the number of launches (1), or -1 when the shared memory does not
// fit.
template <int D, typename T, int PMAX>
inline int launch_persist_pmax(const DevMesh& m, T* vals, T* rhs, PersistArgs a, int sm_count, cudaStream_t st) {
  const size_t wbytes = align_up(persist_warp_bytes<D, T, 1, PMAX>(m, a.mom_mask), 16);
  const int nrule = (m.rt.vol_off[PMAX] + m.rt.vol_n[PMAX]) * (D + 1);
  const size_t smem = PersistHead<D, T>::bytes(nrule) + kWarps * wbytes;
  if (smem > 227 * 1024) return -1;
  a.warp_bytes = (int)wbytes;
  auto k = persist_kernel<D, T, PMAX>;
  const int grid = resident_grid(k, smem, sm_count, (a.nitems + kWarps - 1) / kWarps, 0);
  k<<<grid, kWarps * 32, smem, st>>>(m, vals, rhs, a);
  return 1;
}

}  // namespace dg
