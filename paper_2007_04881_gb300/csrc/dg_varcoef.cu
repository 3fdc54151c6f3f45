// dg_varcoef.cu -- kernels of the variable-coefficient terms (Sec. 4.2): one
// warp per element row, grid-strided, its lanes along the entries of each
// block of the row (the row bodies are in dg_varcoef.cuh).  The row kernels
// have already written every block and the load vector with b = 0, c = 0;
// these launches add the b and c terms in place, each entry by its one lane.
#include "dg_varcoef.cuh"

namespace dg {

namespace {

constexpr int kVcThreads = 128;

template <int D>
__global__ void __launch_bounds__(kVcThreads) varcoef_matrix_kernel(VcView v, double* __restrict__ vals) {
  const int nwarps = gridDim.x * (kVcThreads / 32);
  for (int r = blockIdx.x * (kVcThreads / 32) + (threadIdx.x >> 5); r < v.ne; r += nwarps)
    vc_matrix_row<D>(v, vals, r, threadIdx.x & 31, 32);
}

template <int D>
__global__ void __launch_bounds__(kVcThreads) varcoef_rhs_kernel(VcView v, double* __restrict__ rhs) {
  const int nwarps = gridDim.x * (kVcThreads / 32);
  for (int r = blockIdx.x * (kVcThreads / 32) + (threadIdx.x >> 5); r < v.ne; r += nwarps)
    vc_rhs_row<D>(v, rhs, r, threadIdx.x & 31, 32);
}

int vc_grid(int ne, int sm_count) {
  const int want = (ne + kVcThreads / 32 - 1) / (kVcThreads / 32);
  const int cap = 16 * (sm_count > 0 ? sm_count : 1);
  return want < cap ? want : cap;
}

}  // namespace

int launch_varcoef(const VcView& v, int dim, double* vals, double* rhs, int sm_count, cudaStream_t st) {
  if (v.ne <= 0) return 0;
  const int grid = vc_grid(v.ne, sm_count);
  int n = 0;
  if (vals) {
    if (dim == 2)
      varcoef_matrix_kernel<2><<<grid, kVcThreads, 0, st>>>(v, vals);
    else
      varcoef_matrix_kernel<3><<<grid, kVcThreads, 0, st>>>(v, vals);
    ++n;
  }
  if (rhs) {
    if (dim == 2)
      varcoef_rhs_kernel<2><<<grid, kVcThreads, 0, st>>>(v, rhs);
    else
      varcoef_rhs_kernel<3><<<grid, kVcThreads, 0, st>>>(v, rhs);
    ++n;
  }
  return n;
}

}  // namespace dg
