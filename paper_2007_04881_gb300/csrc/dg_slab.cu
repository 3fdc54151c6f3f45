// dg_slab.cu -- space-time slab systems (Sec. 2.3) expanded from the spatial
// blocks.  With the orthonormal Legendre basis T_k of the slab's interval the
// prism block of elements (r, s) is
//   A[(k, j), (l, m)] = [k = l] B[j, m] + [r = s] D_kl M[j, m],
// B the spatial block of Eq. (2.4), M the spatial mass matrix and D the time
// part (the derivative and the jump at t0).  These kernels only move and
// scale values: one warp per element row, its lanes along each block's
// entries, so every store of a block is contiguous and coalesced.  The slab
// matrix is several times the spatial one (25x at p = 4 in PQ), so the
// expansion is bound by its HBM writes.
#include "dg_slab.cuh"

namespace dg {

namespace {

constexpr int kSlabThreads = 256;

// one warp per element row, grid-strided over the rows largest first; the
// time matrix and the dof decode tables of degrees 1..pmax in shared memory
template <typename T>
__global__ void __launch_bounds__(kSlabThreads) slab_matrix_kernel(SlabPattern sp, SlabTimes<T> tt, int pmax,
                                                                   const T* __restrict__ B, const T* __restrict__ M,
                                                                   T* __restrict__ vals) {
  __shared__ T sD[kSlabKMax * kSlabKMax];
  __shared__ SlabDecode dec;
  for (int i = threadIdx.x; i < kSlabKMax * kSlabKMax; i += blockDim.x) sD[i] = tt.D[i / kSlabKMax][i % kSlabKMax];
  slab_decode_tables(sp.dim, sp.space, pmax, dec, threadIdx.x, blockDim.x);
  __syncthreads();
  const int nwarps = gridDim.x * (kSlabThreads / 32);
  for (int w = blockIdx.x * (kSlabThreads / 32) + (threadIdx.x >> 5); w < sp.ne; w += nwarps) {
    const int r = sp.order ? sp.order[sp.ne - 1 - w] : w;
    slab_matrix_row<T>(sp, sD, dec, B, M, vals, r, threadIdx.x & 31, 32);
  }
}

template <typename T>
__global__ void __launch_bounds__(kSlabThreads) slab_rhs_kernel(SlabPattern sp, SlabTimes<T> tt,
                                                                const T* __restrict__ l, const T* __restrict__ M,
                                                                const T* __restrict__ u_prev, T* __restrict__ rhs) {
  const int nwarps = gridDim.x * (kSlabThreads / 32);
  for (int r = blockIdx.x * (kSlabThreads / 32) + (threadIdx.x >> 5); r < sp.ne; r += nwarps)
    slab_rhs_row<T>(sp, tt, l, M, u_prev, rhs, r, threadIdx.x & 31, 32);
}

template <typename T>
__global__ void __launch_bounds__(kSlabThreads) slab_trace_kernel(SlabPattern sp, SlabTimes<T> tt,
                                                                  const T* __restrict__ U, T* __restrict__ u_end) {
  const int nwarps = gridDim.x * (kSlabThreads / 32);
  for (int r = blockIdx.x * (kSlabThreads / 32) + (threadIdx.x >> 5); r < sp.ne; r += nwarps)
    slab_trace_row<T>(sp, tt, U, u_end, r, threadIdx.x & 31, 32);
}

template <typename T>
SlabTimes<T> cast_times(const SlabTimes<double>& t) {
  SlabTimes<T> o;
  for (int k = 0; k < kSlabKMax; ++k) {
    for (int l = 0; l < kSlabKMax; ++l) o.D[k][l] = T(t.D[k][l]);
    o.at0[k] = T(t.at0[k]);
    o.at1[k] = T(t.at1[k]);
  }
  o.sqrt_tau = T(t.sqrt_tau);
  return o;
}

// warps: one per element, grid-strided; at most 16 CTAs of 8 warps per SM
int slab_grid(int ne, int sm_count) {
  const int want = (ne + kSlabThreads / 32 - 1) / (kSlabThreads / 32);
  const int cap = 16 * (sm_count > 0 ? sm_count : 1);
  return want < cap ? want : cap;
}

}  // namespace

int launch_slab_matrix(const SlabPattern& sp, const SlabTimes<double>& tt, bool fp32, const void* B, const void* M,
                       void* vals, int pmax, int sm_count, cudaStream_t st) {
  if (sp.ne <= 0) return 0;
  const int grid = slab_grid(sp.ne, sm_count);
  if (fp32)
    slab_matrix_kernel<float><<<grid, kSlabThreads, 0, st>>>(sp, cast_times<float>(tt), pmax,
                                                             static_cast<const float*>(B),
                                                             static_cast<const float*>(M), static_cast<float*>(vals));
  else
    slab_matrix_kernel<double><<<grid, kSlabThreads, 0, st>>>(sp, tt, pmax, static_cast<const double*>(B),
                                                              static_cast<const double*>(M),
                                                              static_cast<double*>(vals));
  return 1;
}

int launch_slab_rhs(const SlabPattern& sp, const SlabTimes<double>& tt, bool fp32, const void* l, const void* M,
                    const void* u_prev, void* rhs, int sm_count, cudaStream_t st) {
  if (sp.ne <= 0) return 0;
  const int grid = slab_grid(sp.ne, sm_count);
  if (fp32)
    slab_rhs_kernel<float><<<grid, kSlabThreads, 0, st>>>(sp, cast_times<float>(tt), static_cast<const float*>(l),
                                                          static_cast<const float*>(M),
                                                          static_cast<const float*>(u_prev), static_cast<float*>(rhs));
  else
    slab_rhs_kernel<double><<<grid, kSlabThreads, 0, st>>>(sp, tt, static_cast<const double*>(l),
                                                           static_cast<const double*>(M),
                                                           static_cast<const double*>(u_prev),
                                                           static_cast<double*>(rhs));
  return 1;
}

int launch_slab_trace(const SlabPattern& sp, const SlabTimes<double>& tt, bool fp32, const void* U, void* u_end,
                      int sm_count, cudaStream_t st) {
  if (sp.ne <= 0) return 0;
  const int grid = slab_grid(sp.ne, sm_count);
  if (fp32)
    slab_trace_kernel<float><<<grid, kSlabThreads, 0, st>>>(sp, cast_times<float>(tt), static_cast<const float*>(U),
                                                            static_cast<float*>(u_end));
  else
    slab_trace_kernel<double><<<grid, kSlabThreads, 0, st>>>(sp, tt, static_cast<const double*>(U),
                                                             static_cast<double*>(u_end));
  return 1;
}

}  // namespace dg
