// dg_internal.h -- device-side mesh view and launch helpers shared by the
// host code (dg_host.cu) and the kernels (dg_geom.cu, dg_elem*.cu,
// dg_iface.cu).  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <functional>
#include <string>
#include <vector>

#include <cuda_runtime.h>

namespace dg {

constexpr int kPMax2 = 6;  // highest degree with compiled kernels in 2D
constexpr int kPMax3 = 4;  // ... in 3D
constexpr int kPMaxLin = 6;  // Legendre linearisation tables: degrees 0..6, products to 12
constexpr int kWarps = 4;  // warps per CTA of the element / interface kernels

// values per sub-simplex in bounding-box coordinates xi = 2(x-lo)/L - 1:
//   2D triangle: xi0(2), e1(2), e2(2), |J|          -> 7
//   3D tetrahedron: xi0(3), e1(3), e2(3), e3(3), |J| -> 13
__host__ __device__ constexpr int sub_vals(int dim) { return dim == 2 ? 7 : 13; }
// values per face side (side s frame of element e_s):
//   2D: xi(v0)(2), xi(v1)-xi(v0)(2), n'(2)              -> 6
//   3D: xi(v0)(3), xi(v1)-xi(v0)(3), xi(v2)-xi(v0)(3), n'(3) -> 12
// with n'_d = 2 n_d / L_d, n the unit normal pointing out of e0.
__host__ __device__ constexpr int side_vals(int dim) { return dim == 2 ? 6 : 12; }
// values per element record: lo, L, 1/L (dim each) and R
__host__ __device__ constexpr int elem_vals(int dim) { return 3 * dim + 1; }
// values per half-face record (face f seen from side s, element e_s), one
// contiguous record per half face in the element's half-face order:
//   [0, FV)      side s's values (side_vals layout), normal part times sgn_s
//   [FV, 2 FV)   the other side's values (zero on the boundary), normal part
//                times sgn_s
//   2 FV: J, 2 FV + 1: sigma, 2 FV + 2: sgn_s b . n0, 2 FV + 3: nq (points
//   per direction), negated on a boundary face
// with sgn_0 = +1, sgn_1 = -1, so every normal in the record points out of
// e_s.  2D 16 values, 3D 28 padded to 32 (one or two 64-byte lines in FP32).
__host__ __device__ constexpr int hf_rec_vals(int dim) { return dim == 2 ? 16 : 32; }

__host__ __device__ constexpr int nbasis(int dim, int p) {
  return dim == 2 ? (p + 1) * (p + 2) / 2 : (p + 1) * (p + 2) * (p + 3) / 6;
}

// Reference-rule tables (host-built once per context, FP64 + FP32 copies).
//   volume rule of degree p: (p+2)^d collapsed points (r, s[, t], w)
//   face rule with n points per direction: 2D n Gauss points (t, w);
//   3D n^2 collapsed triangle points (r, s, w)
struct RuleTables {
  const double* vol64 = nullptr;  // packed, [point][d+1]
  const float* vol32 = nullptr;
  int vol_off[8] = {0};  // offset (in points) of degree p's rule
  int vol_n[8] = {0};    // points of degree p's rule
  const double* face64 = nullptr;
  const float* face32 = nullptr;
  int face_off[10] = {0};  // offset (in points) of the n-point rule
  int face_n[10] = {0};    // points of the n-point rule
  // Legendre linearisation coefficients [3][kPMaxLin+1][kPMaxLin+1][2 kPMaxLin+1]:
  // P_a P_b, P'_a P_b and P'_a P'_b expanded in P_c
  const double* lin64 = nullptr;
  const float* lin32 = nullptr;
};

// Problem data (constant over the mesh).
struct Problem {
  double b[3];
  double c;
  int source;
  double poly[20];
  double c_sigma;
  // Neumann sides (bit 2d + s: x_d = dlo[d] for s = 0, dhi[d] for s = 1)
  // and the bounding box of the vertices they refer to
  int neumann;
  double dlo[3], dhi[3];
  // the same constants rounded to FP32, for the FP32 kernels: on a part whose
  // FP64 rate is 1/64 of FP32 a per-point conversion occupies the FP64 pipe
  float bf[3], cf, polyf[20], c_sigmaf;
  void round_copies() {
    for (int d = 0; d < 3; ++d) bf[d] = (float)b[d];
    cf = (float)c;
    for (int k = 0; k < 20; ++k) polyf[k] = (float)poly[k];
    c_sigmaf = (float)c_sigma;
  }
};

// a problem constant in the contraction type T (FP64 value or its FP32 copy)
template <typename T>
__host__ __device__ __forceinline__ T pb_val(double v64, float v32) {
  if constexpr (sizeof(T) == 4)
    return v32;
  else
    return v64;
}

// Everything a kernel needs, by device pointer.  Passed by value.
struct DevMesh {
  int dim, nv, ne, nsub, nf, ni, nhf;
  const double* X[3];
  // 2D: vertex loops; 3D: tetrahedra (4 vertex ids each)
  const int* eptr;
  const int* eidx;
  // unique vertex list per element (2D: the loop itself)
  const int* uvptr;
  const int* uvidx;
  const int* sub_elem;  // element of each sub-simplex
  const int* sub_loc;   // 2D: loop position of the triangle's first vertex; 3D: unused
  const int* p;         // [ne]
  const double* a;      // [ne]
  // element geometry (FP64)
  double* lo;   // [dim][ne]
  double* L;    // [dim][ne]
  double* cen;  // [dim][ne]
  double* vol;  // [ne]
  double* h;    // [ne]
  double* pen;  // [ne] a_k p_k^2 / h_k
  // per-element records in the contraction precision, SoA [k][ne]:
  // lo[D], L[D], 1/L[D], R = 1/sqrt(prod_d L_d)
  double* eg64;
  float* eg32;
  // reduced-precision geometry (the FP32 and tensor-core forms).  xs2: every
  // vertex coordinate as an unevaluated float pair hi + lo, [dim][nv].  gx32,
  // SoA [k][ne]: the box's lower corner as pairs (hi[D], lo[D]), the low
  // parts of its extent L (the high parts are eg32's L), and a_k p_k^2 / h_k.
  // Null where only the FP64 kernels run.
  float2* xs2;
  float* gx32;
  // sub-simplex data, SoA [k][nsub]
  double* sg64;
  float* sg32;
  // faces
  const int* f_e0;
  const int* f_e1;  // -1 on the boundary
  const int* f_v;   // [nf][dim] vertex ids in e0's order (2D: along e0's CCW loop; 3D: e0's tetrahedron)
  const int8_t* f_flip;  // 3D: 1 if (v1-v0) x (v2-v0) points into e0
  double* fs64;     // [2][side_vals][nf] (FP64 only: the variable-coefficient path)
  double* fsc64;  // [3][nf]: J (2D |F|, 3D 2|F|), sigma, b.n
  int* f_nq;  // points per direction on the face: max(p0, p1) + 1
  const int* f_hf;  // [2][nf] half-face index of face f on side s (-1: none)
  // half-face records (hf_rec_vals layout), [nhf][hf_rec_vals], written by
  // the face geometry kernels
  double* hfr64;
  float* hfr32;
  // element -> faces (half faces), fixed order
  const int* hf_ptr;   // [ne+1]
  const int* hf_face;  // [nhf]
  const int8_t* hf_side;
  const int* hf_qoff;  // [nhf] first face point of the half face within its element
  const int* e_nqf;    // [ne] face points of the element
  // interfaces
  const int* if_e0;
  const int* if_e1;
  const int* if_fptr;  // [ni+1] faces of interface i (consecutive in face order)
  const int* if_slot01;
  const int* if_slot10;
  // per interface position k of if_perm, two int4: {e0, e1, e0's half face of
  // the first face, faces}, {slot01, slot10, p[e0] | p[e1] << 8, 0}; the
  // interface kernel's parameters in one coalesced load (built at upload)
  const int4* if_rec;
  // BSR
  const int* row_ptr;  // [ne+1]
  const int* col;      // [nnzb]
  const int* blk_if;   // [nnzb] interface of an off-diagonal block, -1 on the diagonal
  // [nnzb] per off-diagonal block (r, k): k, the first of the interface's
  // half faces in r's half-face list, the interface's faces, p_k (diagonal
  // blocks: -1, 0, 0, 0)
  const int4* blk_rec;
  const int64_t* blk_off;
  const int* diag_blk;
  const int64_t* dof_off;
  int nmax;   // largest basis size in the mesh
  int pmask;  // bit p: an element of degree p in the mesh (a neighbour's, too, in a partition)
  // work lists
  const int* elem_perm;  // elements grouped by degree, each group cost-descending
  int elem_pstart[9];    // group of degree p: elem_perm[elem_pstart[p] .. elem_pstart[p+1])
  const int* if_perm;    // interfaces grouped by max degree
  int if_pstart[9];
  Problem pb;
  RuleTables rt;
  // learned volume rules (2D): per element 28 points (xi, eta) and physical
  // weights, used where lq_ok[e] != 0; null when none are installed
  const int* lq_ok;
  const double* lq64;  // [ne][84]
  const float* lq32;
  // the context's status word (bit 0 a bounded wait ran out, bit 1 an index
  // range failed a DG_CHECK_BOUNDS check) and the output sizes it checks
  int* status;
  int64_t nvals, ndofs;
};

// mode bits of the element kernel
enum : int {
  kModeVol = 1,    // volume integrals into the diagonal block
  kModeFace = 2,   // own-face integrals into the diagonal block
  kModeRhs = 4,    // load vector
  kModeAccum = 8,  // add to the diagonal block instead of overwriting it
  kModeSkipVol = 16,  // volume terms done by the moment kernel: faces only, load vector added
  kModeExactMom = 32,  // moment launch: volume moments exact (2D: Green's theorem along the edges; 3D: the divergence theorem on the boundary triangles)
  // moment launch: the own-face terms too, the diagonal block's through face
  // moments (with kModeFace) and the boundary load terms per point (with
  // kModeRhs), so that the block row's only other writer is the row kernel's
  // off-diagonal launch (kModeOffDiag)
  kModeMomFace = 64,
  kModeOffDiag = 128,  // row kernel: the off-diagonal blocks only (diagonal block and load vector untouched)
};
// with kModeOffDiag (row kernel) and in the lane kernel, bits
// kModeMaskShift + q: the interfaces whose larger degree is q are assembled
// by the interface kernel (the row skips their blocks)
constexpr int kModeMaskShift = 8;
// lane kernel: the diagonal block and the load vector only (every
// off-diagonal block of the rows comes from the interface kernel)
constexpr int kModeDiagOnly = 1 << 20;

// Optional per-launch timing: CUDA events recorded on the launch stream
// around each kernel, with the kernel's label and its algorithmic flop and
// byte counts (host-computed per launch group).
struct LaunchRec {
  char name[48];
  double flops;   // algorithmic (the quadrature formulation's count)
  double xflops;  // executed (differs for the moment form of the volume terms)
  double bytes;
  cudaEvent_t ev0, ev1;
};

constexpr int kKinds = 4;
constexpr int kNoCounts = 99;  // Tracer::begin kind of a launch with no algorithmic counts
struct Tracer {
  bool on = false;
  LaunchRec* recs = nullptr;  // capacity cap, filled from n
  int cap = 0;
  int n = 0;
  // per launch-group algorithmic counts, indexed [kind][p]; kind 0 = row
  // kernel of degree p (volume and faces), 1 = its faces-only launch next to
  // the moment kernel, 2 = the moment volume kernel, 3 = the moment kernel
  // with the own-face terms; words = values written + read, scaled by
  // sizeof(T).  Kinds 4 (the row kernel's off-diagonal launch: the blocks of
  // degree-p rows whose neighbour degree is not in imask) and 5 (the
  // interface launch of larger degree p: interfaces with both degrees in
  // imask) take their counts from offd, and so does kind 6 (the lane kernel
  // of degree p with the interface kernel on: kind 0 less the blocks of
  // interfaces whose larger degree is in imask).
  const double* flops = nullptr;   // [kKinds][9]
  const double* words = nullptr;   // [kKinds][9]
  const double* xflops = nullptr;  // [2][9]: flops the kind-2 and kind-3 launches execute
  const double* offd = nullptr;    // [2][9][9]: interface-term flops, words of degree-p rows by neighbour degree
  int imask = 0;
  // share of its degree group's counts the next begin() records (a group
  // launched as several parts)
  double scale = 1.0;
  void begin(const char* name, int kind, int p, size_t tsize, cudaStream_t st);
  // a launch with its counts given directly
  void begin_counts(const char* name, double fl, double xfl, double by, cudaStream_t st);
  void end(cudaStream_t st);
  static void record(cudaEvent_t ev, cudaStream_t st);
};

// Executed-operation tables of the moment launch by degree (dg_host.cu).
struct MomentOps {
  double pt[9] = {0}, map[9] = {0}, fpt[9] = {0}, bnd[9] = {0}, mapf[9] = {0};
};
void moment_op_tables(int dim, MomentOps& o);

// Launchers (defined in the kernel translation units).  Each returns the
// number of kernel launches issued.
// wmask: bit 0 writes the FP64 copies of the sub-simplex / face records,
// bit 1 the FP32 copies (element records are always written in both).
// wmask == 2 on a mesh with xs2 / gx32 takes the reduced-precision kernels
// instead: FP32 records only, with no FP64 arithmetic beyond splitting the
// coordinates; the FP64 element arrays and records keep their last values.
// Returns the number of launches.
int launch_geometry(const DevMesh& m, cudaStream_t st, Tracer* tr = nullptr, int wmask = 3);
// Launch shape of the row kernels: cap on co-resident CTAs per SM (0: the
// occupancy limit) and the stream of each degree's launch (index p).
constexpr int kMaxSplit = 4;  // parts of one degree group
struct LaunchOpts {
  int occ_cap = 0;
  bool vol_moments = true;  // volume blocks through Legendre-product moments where supported
  bool vol_exact = false;   // those moments exact, from the element's boundary (edges / triangles)
  int tile[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};  // register-tile variant of each degree's row kernel
  cudaStream_t pst[9] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  // each degree group as split[p] (1..kMaxSplit) contiguous parts of equal
  // element count, part i on stream part[p][i] (part[p][0] = pst[p]): the
  // parts' moment-then-rows chains run side by side
  int split[9] = {1, 1, 1, 1, 1, 1, 1, 1, 1};
  cudaStream_t part[9][kMaxSplit] = {};
  bool iface = true;  // interfaces between two off-diagonal rows by the interface kernel (FP32)
  // set by the launchers: the degrees in the mesh (neighbours included) and
  // the degrees whose block rows leave their off-diagonal blocks to the
  // interface kernel
  int present = 0, imask = 0;
};

// Edge TM of the register tiles of tile variant v of the (dim, p) row kernel
// in precision prec (DG_PREC_*); 0 when there is no such variant.  v = 3 is
// the persistent pass's tile.
int row_tile_tm(int dim, int p, int prec, int v);

int launch_row2d_f64(const DevMesh& m, int mode, double* vals, double* rhs, int sm_count, const LaunchOpts& lo, Tracer* tr);
int launch_row2d_f32(const DevMesh& m, int mode, float* vals, float* rhs, int sm_count, const LaunchOpts& lo, Tracer* tr);
int launch_row3d_f64(const DevMesh& m, int mode, double* vals, double* rhs, int sm_count, const LaunchOpts& lo, Tracer* tr);
int launch_row3d_f32(const DevMesh& m, int mode, float* vals, float* rhs, int sm_count, const LaunchOpts& lo, Tracer* tr);
// tensor-core forms (split-BF16 and 3xTF32 contractions)
int launch_row2d_bf16(const DevMesh& m, int mode, float* vals, float* rhs, int sm_count, const LaunchOpts& lo, Tracer* tr);
int launch_row2d_tf32(const DevMesh& m, int mode, float* vals, float* rhs, int sm_count, const LaunchOpts& lo, Tracer* tr);
int launch_row3d_bf16(const DevMesh& m, int mode, float* vals, float* rhs, int sm_count, const LaunchOpts& lo, Tracer* tr);
int launch_row3d_tf32(const DevMesh& m, int mode, float* vals, float* rhs, int sm_count, const LaunchOpts& lo, Tracer* tr);

// The persistent pass (dg_persist.cuh): one launch in which every warp
// takes tiles from a work list until it is done.
struct PersistArgs {
  const int4* items;   // x: kind (0 row tile, 1 moment tile), y: degree, z: tile index
  int nitems;
  int* queue;          // next item; zero before the launch
  int* vdone;          // [ne] moment-tile flags; zero before the launch
  int* status;         // bit 0: a bounded wait ran out
  long long limit_ns;  // bound of one wait
  int mode;            // assembly mode of the pass (kModeVol | kModeFace | kModeRhs)
  int mom_mask;        // bit p: degree p takes the moment path
  int exact;           // kModeExactMom for the moment tiles (volume path 2), else 0
  int warp_bytes;      // shared memory per warp (set by the launcher)
};
// FP32 persistent passes: the launch (1, or -1 when the shared memory does
// not fit), the degrees that can take the moment path, and the elements per
// tile of each kind (gmom[p], grow[p], 9 entries each).
int launch_persist2d_f32(const DevMesh& m, float* vals, float* rhs, const PersistArgs& a, int pmax, int sm_count,
                         cudaStream_t st);
int launch_persist3d_f32(const DevMesh& m, float* vals, float* rhs, const PersistArgs& a, int pmax, int sm_count,
                         cudaStream_t st);
int persist_layout(int dim, int* mom_ok_mask, int* gmom, int* grow);
// a one-warp launch of the persistent pass's bounded wait on flag; a wait
// that runs out sets bit 0 of *status
void launch_wait_probe(const int* flag, int* status, long long limit_ns, cudaStream_t st);

// The block-sparse pattern built on the device (dg_pattern.cu): the same
// arrays as the host pass plan_mesh, in device memory the caller's alloc
// provides, plus host copies of what the host keeps.
struct DevPattern {
  int *sub_elem = nullptr, *f_e0 = nullptr, *f_e1 = nullptr, *f_v = nullptr, *f_nq = nullptr, *f_hf = nullptr;
  int8_t *f_flip = nullptr, *hf_side = nullptr;
  int *hf_ptr = nullptr, *hf_face = nullptr, *hf_qoff = nullptr, *e_nqf = nullptr;
  int *if_e0 = nullptr, *if_e1 = nullptr, *if_fptr = nullptr, *slot01 = nullptr, *slot10 = nullptr;
  int *row_ptr = nullptr, *col = nullptr, *blk_if = nullptr, *diag_blk = nullptr;
  int64_t *blk_off = nullptr, *dof_off = nullptr;
  int4* blk_rec = nullptr;
  const int *uvptr = nullptr, *uvidx = nullptr;
  int *elem_perm = nullptr, *if_perm = nullptr;
  int nsub = 0, nf = 0, nint = 0, ni = 0, nhf = 0, nnzb = 0;
  int64_t nvals = 0, ndofs = 0, nqvol = 0, nqface = 0;
  int elem_pstart[9] = {0}, if_pstart[9] = {0};
  double flops[kKinds][9] = {{0}}, words[kKinds][9] = {{0}}, mom_exec[2][9] = {{0}}, mom_pt[9] = {0};
  double offd[2][9][9] = {{{0}}};
  std::vector<int> h_row_ptr, h_col, h_e_nqf, h_nvq, h_perm;
  std::vector<int64_t> h_blk_off, h_dof_off;
};

// learned quadrature (dg_learned.cu)
void lq_prepare(const DevMesh& m, double* mom, double* mmom, void* feat, int* elig, cudaStream_t st);
void lq_gn(const DevMesh& m, const double* mom, const double* mmom, const int* elig, const float* init, int iters,
           double* rule, float* resid, int* ok, int sm_count, cudaStream_t st);
void lq_install(const DevMesh& m, const double* rule, const int* ok, double* lq64, float* lq32, int* lq_ok,
                cudaStream_t st);
void lq_targets(int ne, const double* rule, const double* mmom, float* tgt, cudaStream_t st);

}  // namespace dg
#include "../../include/dg.h"
namespace dg {
int build_pattern_device(const dg_mesh_desc* d, const int* eptr, const int* eidx, const int* p, const double* const* X,
                         const std::function<void*(size_t)>& alloc, cudaStream_t st, DevPattern* P, std::string* msg);
// the interface records dm.if_rec[2 * ni] from the topology arrays (stream st)
void launch_iface_recs(const DevMesh& dm, int4* rec, cudaStream_t st);

// Host: collapsed reference rule on the d-simplex with n Gauss points per
// direction, packed as [point][d+1] = (coordinates, weight); d = 1 gives the
// n-point Gauss-Legendre rule on [0,1].
}  // namespace dg
#include <vector>
namespace dg {
void reference_rule(int dim, int n, std::vector<double>& pts);
}  // namespace dg

// shared by the host translation units
struct dg_ctx;
cudaStream_t dg_ctx_stream(dg_ctx* ctx);
int dg_fail_msg(int code, const char* msg);
