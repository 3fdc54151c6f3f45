// Host build of the slab kernels' row bodies (paper_2007_04881_gb300/csrc/
// dg_slab.cuh), for the CPU test of their arithmetic against the slab oracle
// (tests/test_slab_rows_cpu.py).  Each row is run lane by lane as one warp of
// the kernels would run it.  Test infrastructure: nothing in the library
// calls this.
#include "dg_slab.cuh"

using namespace dg;

namespace {
SlabPattern pattern(int dim, int ne, int space, const int* p, const int* row_ptr, const int* col, const int* diag_blk,
                    const int64_t* blk_off, const int64_t* dof_off, const int64_t* sblk_off, const int64_t* sdof_off) {
  SlabPattern sp;
  sp.dim = dim;
  sp.ne = ne;
  sp.space = space;
  sp.p = p;
  sp.row_ptr = row_ptr;
  sp.col = col;
  sp.diag_blk = diag_blk;
  sp.blk_off = blk_off;
  sp.dof_off = dof_off;
  sp.sblk_off = sblk_off;
  sp.sdof_off = sdof_off;
  return sp;
}
constexpr int kLanes = 32;
}  // namespace

extern "C" {
void host_slab_matrix(int dim, int ne, int space, const int* p, const int* row_ptr, const int* col,
                      const int* diag_blk, const int64_t* blk_off, const int64_t* dof_off, const int64_t* sblk_off,
                      const int64_t* sdof_off, double t0, double t1, const double* B, const double* M, double* vals) {
  const SlabPattern sp = pattern(dim, ne, space, p, row_ptr, col, diag_blk, blk_off, dof_off, sblk_off, sdof_off);
  const SlabTimes<double> tt = slab_time_data(t0, t1);
  // the kernel's shared tables, built by the same code, one thread
  static SlabDecode dec;
  int pmax = 1;
  for (int e = 0; e < ne; ++e) pmax = p[e] > pmax ? p[e] : pmax;
  slab_decode_tables(dim, space, pmax, dec, 0, 1);
  double D[kSlabKMax * kSlabKMax];
  for (int i = 0; i < kSlabKMax * kSlabKMax; ++i) D[i] = tt.D[i / kSlabKMax][i % kSlabKMax];
  for (int r = 0; r < ne; ++r)
    for (int lane = 0; lane < kLanes; ++lane) slab_matrix_row<double>(sp, D, dec, B, M, vals, r, lane, kLanes);
}

void host_slab_rhs(int dim, int ne, int space, const int* p, const int* row_ptr, const int* col, const int* diag_blk,
                   const int64_t* blk_off, const int64_t* dof_off, const int64_t* sblk_off, const int64_t* sdof_off,
                   double t0, double t1, const double* l, const double* M, const double* u_prev, double* rhs) {
  const SlabPattern sp = pattern(dim, ne, space, p, row_ptr, col, diag_blk, blk_off, dof_off, sblk_off, sdof_off);
  const SlabTimes<double> tt = slab_time_data(t0, t1);
  for (int r = 0; r < ne; ++r)
    for (int lane = 0; lane < kLanes; ++lane) slab_rhs_row<double>(sp, tt, l, M, u_prev, rhs, r, lane, kLanes);
}

void host_slab_trace(int dim, int ne, int space, const int* p, const int* row_ptr, const int* col,
                     const int* diag_blk, const int64_t* blk_off, const int64_t* dof_off, const int64_t* sblk_off,
                     const int64_t* sdof_off, double t0, double t1, const double* U, double* u_end) {
  const SlabPattern sp = pattern(dim, ne, space, p, row_ptr, col, diag_blk, blk_off, dof_off, sblk_off, sdof_off);
  const SlabTimes<double> tt = slab_time_data(t0, t1);
  for (int r = 0; r < ne; ++r)
    for (int lane = 0; lane < kLanes; ++lane) slab_trace_row<double>(sp, tt, U, u_end, r, lane, kLanes);
}
}
