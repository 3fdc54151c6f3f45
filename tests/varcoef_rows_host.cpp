// Host build of the variable-coefficient row bodies (paper_2007_04881_gb300/
// csrc/dg_varcoef.cuh), for the CPU test of their arithmetic against the
// oracle (tests/test_varcoef_rows_cpu.py).  Each row is run lane by lane as
// one warp of the kernels would run it.  Test infrastructure: nothing in the
// library calls this.
#include "dg_varcoef.cuh"

using namespace dg;

namespace {
template <int D>
void run(const int* ints, const int* p, const int* eptr, const double* eg, const double* sg, const double* fs,
         const double* fsc, const int* f_e0, const int* f_e1, const int* f_nq, const int* hf_ptr, const int* hf_face,
         const int8_t* hf_side, const int* if_fptr, const int* row_ptr, const int* col, const int* blk_if,
         const int64_t* blk_off, const int64_t* dof_off, const double* vol_rule, const double* face_rule,
         const int* offs, double* vals, double* rhs) {
  VcView v;
  v.ne = ints[0];
  v.nf = ints[1];
  v.nsub = ints[2];
  v.source = ints[3];
  v.p = p;
  v.eptr = eptr;
  v.eg = eg;
  v.sg = sg;
  v.fs = fs;
  v.fsc = fsc;
  v.f_e0 = f_e0;
  v.f_e1 = f_e1;
  v.f_nq = f_nq;
  v.hf_ptr = hf_ptr;
  v.hf_face = hf_face;
  v.hf_side = hf_side;
  v.if_fptr = if_fptr;
  v.row_ptr = row_ptr;
  v.col = col;
  v.blk_if = blk_if;
  v.blk_off = blk_off;
  v.dof_off = dof_off;
  v.vol_rule = vol_rule;
  v.face_rule = face_rule;
  for (int k = 0; k < 8; ++k) {
    v.vol_off[k] = offs[k];
    v.vol_n[k] = offs[8 + k];
  }
  for (int k = 0; k < 10; ++k) {
    v.face_off[k] = offs[16 + k];
    v.face_n[k] = offs[26 + k];
  }
  for (int r = 0; r < v.ne; ++r)
    for (int lane = 0; lane < 32; ++lane) {
      vc_matrix_row<D>(v, vals, r, lane, 32);
      vc_rhs_row<D>(v, rhs, r, lane, 32);
    }
}
}  // namespace

// ints: ne, nf, nsub, source; arrays as VcView; offs: vol_off[8], vol_n[8],
// face_off[10], face_n[10]
#define VC_ARGS                                                                                                    \
  const int *ints, const int *p, const int *eptr, const double *eg, const double *sg, const double *fs,           \
      const double *fsc, const int *f_e0, const int *f_e1, const int *f_nq, const int *hf_ptr, const int *hf_face, \
      const int8_t *hf_side, const int *if_fptr, const int *row_ptr, const int *col, const int *blk_if,           \
      const int64_t *blk_off, const int64_t *dof_off, const double *vol_rule, const double *face_rule,            \
      const int *offs, double *vals, double *rhs
#define VC_PASS                                                                                                \
  ints, p, eptr, eg, sg, fs, fsc, f_e0, f_e1, f_nq, hf_ptr, hf_face, hf_side, if_fptr, row_ptr, col, blk_if, \
      blk_off, dof_off, vol_rule, face_rule, offs, vals, rhs

extern "C" {
void host_varcoef_2d(VC_ARGS) { run<2>(VC_PASS); }
void host_varcoef_3d(VC_ARGS) { run<3>(VC_PASS); }
}
