// dg_host.cu -- host side of libdg: contexts, mesh upload (validation, face
// and interface derivation, block-sparse pattern, work lists), reference
// quadrature tables, and the C ABI declared in include/dg.h.
//
// The sparsity pattern is built before any quadrature, with one block per
// element pair however many faces the pair shares: the "Approach 2" idea of
// Sec. 3.4 (precomputed pattern, values written in place).  Unlike the
// paper's atomics, every block has exactly one writer per launch, so the
// result is bitwise reproducible.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <chrono>
#include <climits>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/dg.h"
#include "dg_internal.h"
#include "dg_slab.cuh"
#include "dg_varcoef.cuh"

#include <nvtx3/nvToolsExt.h>

using namespace dg;

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define DG_CUDA_TRY(expr)                                                                   \
  do {                                                                                      \
    cudaError_t _e = (expr);                                                                \
    if (_e != cudaSuccess)                                                                  \
      return fail(_e == cudaErrorMemoryAllocation ? DG_ERR_OOM : DG_ERR_CUDA, "%s: %s", #expr, \
                  cudaGetErrorString(_e));                                                  \
  } while (0)

// ---------------------------------------------------------------------------
// reference quadrature (Gauss-Legendre by Newton's method, collapsed rules)
// ---------------------------------------------------------------------------

// n-point Gauss-Legendre rule on [0,1].  Newton's method on P_n, started
// from Tricomi's asymptotic approximation of the roots.
void gauss_legendre01(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  const double pi = 3.14159265358979323846;
  for (int i = 1; i <= n; ++i) {
    double t = (1.0 - 1.0 / (8.0 * n * n) + 1.0 / (8.0 * n * n * n)) * std::cos(pi * (4.0 * i - 1.0) / (4.0 * n + 2.0));
    double dp = 1.0;
    for (int iter = 0; iter < 64; ++iter) {
      // P_n(t) and P_n'(t)
      double pm = 1.0, pc = t;
      for (int k = 2; k <= n; ++k) {
        const double pn = ((2.0 * k - 1.0) * t * pc - (k - 1.0) * pm) / k;
        pm = pc;
        pc = pn;
      }
      if (n == 1) {
        pm = 1.0;
        pc = t;
      }
      dp = n * (t * pc - pm) / (t * t - 1.0);
      const double step = pc / dp;
      t -= step;
      if (std::fabs(step) <= 1e-16 * std::fabs(t) + 1e-300) break;
    }
    // recompute the derivative at the converged root for the weight
    double pm = 1.0, pc = t;
    for (int k = 2; k <= n; ++k) {
      const double pn = ((2.0 * k - 1.0) * t * pc - (k - 1.0) * pm) / k;
      pm = pc;
      pc = pn;
    }
    if (n == 1) {
      pm = 1.0;
      pc = t;
    }
    dp = n * (t * pc - pm) / (t * t - 1.0);
    const double wt = 2.0 / ((1.0 - t * t) * dp * dp);
    x[i - 1] = 0.5 * (1.0 - t);  // roots come out descending in t; store ascending
    w[i - 1] = 0.5 * wt;
  }
}

// Collapsed rules.  Triangle: (r, s) = (a(1-b), b), weight w_a w_b (1-b).
// Tetrahedron: (r, s, t) = (a(1-b)(1-c), b(1-c), c), weight w_a w_b w_c (1-b)(1-c)^2.
void simplex_rule(int dim, int n, std::vector<double>& pts /* [q][dim+1] */) {
  std::vector<double> g, gw;
  gauss_legendre01(n, g, gw);
  pts.clear();
  if (dim == 1) {
    for (int i = 0; i < n; ++i) {
      pts.push_back(g[i]);
      pts.push_back(gw[i]);
    }
  } else if (dim == 2) {
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        const double a = g[i], b = g[j];
        pts.push_back(a * (1.0 - b));
        pts.push_back(b);
        pts.push_back(gw[i] * gw[j] * (1.0 - b));
      }
  } else {
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j)
        for (int k = 0; k < n; ++k) {
          const double a = g[i], b = g[j], c = g[k];
          pts.push_back(a * (1.0 - b) * (1.0 - c));
          pts.push_back(b * (1.0 - c));
          pts.push_back(c);
          pts.push_back(gw[i] * gw[j] * gw[k] * (1.0 - b) * (1.0 - c) * (1.0 - c));
        }
  }
}

struct DevBuf {
  std::vector<void*> ptrs;
  ~DevBuf() {
    for (void* p : ptrs) cudaFree(p);
  }
  template <typename T>
  cudaError_t alloc(T** out, size_t n) {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T));
    if (e == cudaSuccess) {
      ptrs.push_back(p);
      *out = static_cast<T*>(p);
    }
    return e;
  }
};

}  // namespace

int dg_fail_msg(int code, const char* msg) { return fail(code, "%s", msg); }
cudaStream_t dg_ctx_stream(dg_ctx* ctx);

namespace dg {
void reference_rule(int dim, int n, std::vector<double>& pts) { simplex_rule(dim, n, pts); }
int fail_na_impl(int code, const char* msg) { return fail(code, "%s", msg); }
}  // namespace dg

// Forked streams and events for concurrent per-degree launches (created on
// first use).  The context has one set for its direct launches; every graph
// captures through a set of its own, so that a recorded pass does not depend
// on what the context's streams did before it.
struct SideStreams {
  static constexpr int kN = 8;
  cudaStream_t side[kN] = {};
  cudaEvent_t fork = nullptr, join[kN] = {};
  cudaError_t ensure() {
    if (fork) return cudaSuccess;
    cudaError_t e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    for (int i = 0; i < kN && e == cudaSuccess; ++i) {
      e = cudaStreamCreateWithFlags(&side[i], cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join[i], cudaEventDisableTiming);
    }
    return e;
  }
  ~SideStreams() {
    for (int i = 0; i < kN; ++i) {
      if (side[i]) cudaStreamDestroy(side[i]);
      if (join[i]) cudaEventDestroy(join[i]);
    }
    if (fork) cudaEventDestroy(fork);
  }
};

struct dg_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int sm_count = 0;
  int last_launches = 0;
  DevBuf bufs;
  RuleTables rt[4];  // indexed by dim (2, 3)
  Tracer tracer;
  bool vol_moments = true;  // volume blocks through Legendre-product moments
  bool vol_exact = false;   // those moments exact (2D: Green's theorem along the edges; 3D: the divergence theorem on the boundary triangles)
  int tiles[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};  // row-kernel tile variants of untuned passes
  int splits[9] = {1, 1, 1, 1, 1, 1, 1, 1, 1};  // parts of each degree group in untuned concurrent passes
  int* status_dev = nullptr;  // bit 0: a bounded device wait ran out; bit 1: a DG_CHECK_BOUNDS check failed (read and cleared by dg_sync)
  long long wait_ns = 2000000000LL;  // bound of one device wait
  bool persist = false;  // untuned per-step passes and untuned graphs take the persistent pass
  bool pattern_device = false;  // dg_mesh_upload builds the block pattern on the device
  bool nvtx = false;  // NVTX ranges around the calls and their stages (dg_set_nvtx)
  std::vector<LaunchRec> recs;
  SideStreams streams;  // the direct launches' forked streams
  ~dg_ctx() {
    if (status_dev) cudaFree(status_dev);
    for (auto& r : recs) {
      cudaEventDestroy(r.ev0);
      cudaEventDestroy(r.ev1);
    }
  }
};

// An NVTX range over a call or a stage (host markers for a profiler's
// timeline; no effect without a tool attached, none at all when off).
struct NvtxRange {
  bool on;
  NvtxRange(const dg_ctx* ctx, const char* name) : on(ctx && ctx->nvtx) {
    if (on) nvtxRangePushA(name);
  }
  ~NvtxRange() {
    if (on) nvtxRangePop();
  }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// the context's volume path: 0 per-point, 1 quadrature moments, 2 exact 2D moments
static int ctx_vol_path(const dg_ctx* ctx) { return !ctx->vol_moments ? 0 : ctx->vol_exact ? 2 : 1; }

// The per-pass geometry of a precision argument that may carry DG_GEOM_FP64:
// the launch_geometry mask (1: FP64 records; 2: the reduced-precision
// kernels, FP32 records; 3: the FP64 kernels writing the FP64 records and
// their FP32 roundings).  Strips the flag from *prec; -1 for an unknown value.
static int pass_geometry(int* prec) {
  const int flags = *prec & ~0xF, base = *prec & 0xF;
  if ((flags & ~DG_GEOM_FP64) || base < DG_PREC_FP64 || base > DG_PREC_TF32X3) return -1;
  *prec = base;
  if (base == DG_PREC_FP64) return 1;
  return (flags & DG_GEOM_FP64) ? 3 : 2;
}

struct dg_graph {
  cudaStream_t stream = nullptr;  // capture stream
  SideStreams streams;            // forked streams of the captured pass
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int occ_cap = 0;
  int concurrent = 0;
  int vol_path = 1;
  int tiles[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};  // tile variant per degree
  int tile_tm[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};  // its tile edge (0: no group of that degree)
  int split[9] = {1, 1, 1, 1, 1, 1, 1, 1, 1};  // parts per degree group (concurrent shape)
  int trials = 0;  // passes the autotuner timed
  int persist = 0;  // 1: the row work is the persistent pass
  float tuned_ms = 0.f;
  int launches = 0;
  int ntrace = 0;  // timing events recorded inside the graph (tracing on at capture)
  ~dg_graph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (stream) cudaStreamDestroy(stream);
  }
};

namespace dg {
void Tracer::begin(const char* name, int kind, int p, size_t tsize, cudaStream_t st) {
  if (!on || n >= cap) return;
  LaunchRec& r = recs[n];
  snprintf(r.name, sizeof r.name, "%s", name);
  r.flops = ((kind < kKinds && flops) ? flops[kind * 9 + p] : 0.0) * scale;
  r.bytes = ((kind < kKinds && words) ? words[kind * 9 + p] * (double)tsize : 0.0) * scale;
  if (kind == 6) {
    // the lane kernel's rows less the blocks the interface kernel writes
    double fl = flops ? flops[p] : 0.0, wd = words ? words[p] : 0.0;
    for (int q = 1; q <= 8 && offd; ++q)
      if ((imask >> std::max(p, q)) & 1) {
        fl -= offd[p * 9 + q];
        wd -= offd[81 + p * 9 + q];
      }
    r.flops = fl * scale;
    r.bytes = wd * (double)tsize * scale;
  }
  if ((kind == 4 || kind == 5) && offd) {
    // kind 4: blocks of degree-p rows whose interface's larger degree is not
    // in imask; kind 5: interfaces of larger degree p, the blocks of their
    // rows in imask
    double fl = 0.0, wd = 0.0;
    for (int q = 1; q <= 8; ++q) {
      if (kind == 4 && !((imask >> std::max(p, q)) & 1)) {
        fl += offd[p * 9 + q];
        wd += offd[81 + p * 9 + q];
      }
      if (kind == 5 && q <= p) {
        if ((imask >> p) & 1) {
          fl += offd[p * 9 + q];
          wd += offd[81 + p * 9 + q];
        }
        if (q < p && ((imask >> q) & 1)) {
          fl += offd[q * 9 + p];
          wd += offd[81 + q * 9 + p];
        }
      }
    }
    r.flops = fl * scale;
    r.bytes = wd * (double)tsize * scale;
  }
  r.xflops = ((kind == 2 || kind == 3) && xflops) ? xflops[(kind - 2) * 9 + p] * scale : r.flops;
  record(r.ev0, st);
}
void Tracer::begin_counts(const char* name, double fl, double xfl, double by, cudaStream_t st) {
  if (!on || n >= cap) return;
  LaunchRec& r = recs[n];
  snprintf(r.name, sizeof r.name, "%s", name);
  r.flops = fl;
  r.xflops = xfl;
  r.bytes = by;
  record(r.ev0, st);
}
void Tracer::end(cudaStream_t st) {
  if (!on || n >= cap) return;
  record(recs[n].ev1, st);
  ++n;
}
// FMA-equivalent operations the moment launch executes, by degree pp
// (q = 2 pp, nmom moments c + d (+ e) <= q, nn basis functions):
//   pt   per volume point: 2 d (q - 1) for the Legendre values to degree q,
//        q + 1 weighted values, one update per moment (in 3D also the
//        (q+1)(q+2)/2 partial products), nn d for the load vector;
//   map  per element: 3 per moment combination of every block entry (in 3D
//        also 3 per (c, d) pair), 3 d per exponent pair and degree for the
//        coefficient tables;
//   fpt  per own-face point: 3 d (q - 1) for the Legendre values and
//        derivatives, d + 2 weights, 2 per degree c (in 3D 3, and 4 per
//        (c, d) pair), 2 per moment;
//   bnd  per boundary-face point: 3 (pp + 1) + 3 nn for the load terms;
//   mapf per element: the face moments' share of the combination (2D: one
//        more FMA per stage-one term; 3D: 2 per moment combination).
void moment_op_tables(int dim, MomentOps& o) {
  o = MomentOps{};
  for (int pp = 1; pp <= 8; ++pp) {
    const int q = 2 * pp, nn = nbasis(dim, pp);
    const double nmom = dim == 2 ? (q + 1) * (q + 2) / 2.0 : (q + 1) * (q + 2) * (q + 3) / 6.0;
    const double npair = dim == 3 ? (q + 1) * (q + 2) / 2.0 : 0.0;
    o.pt[pp] = 2.0 * dim * (q - 1) + (q + 1) + nmom + npair + nn * dim;
    o.fpt[pp] = 3.0 * dim * (q - 1) + (dim + 2) + (dim == 2 ? 2.0 : 3.0) * (q + 1) + 4.0 * npair + 2.0 * nmom;
    o.bnd[pp] = 3.0 * (pp + 1) + 3.0 * nn;
    std::vector<std::array<int, 3>> al;
    for (int k = 0; k <= pp; ++k)
      for (int l = 0; l <= (dim == 3 ? k : 0); ++l)
        for (int j = 0; j <= k - l; ++j) al.push_back({k - j - l, j, l});
    double ops = 3.0 * dim * (pp + 1) * (pp + 1) * (q + 1), opf = 0.0;
    for (const auto& a : al)
      for (const auto& b : al) {
        const double cx = a[0] + b[0] + 1, cy = a[1] + b[1] + 1, cz = dim == 3 ? a[2] + b[2] + 1 : 1;
        ops += dim == 2 ? 3.0 * cx * cy : 3.0 * cx * cy * cz + 3.0 * cx * cy;
        if (dim == 3) opf += 2.0 * cx * cy * cz;
      }
    if (dim == 2)
      for (int c = 0; c <= q; ++c)
        for (int b = 0; b <= pp; ++b)
          for (int bp = 0; bp <= pp; ++bp) opf += std::min(b + bp, q - c) + 1;
    o.map[pp] = ops;
    o.mapf[pp] = opf;
  }
}

// Inside a stream capture the record becomes an external event node, so the
// event is stamped on every replay of the graph and stays timeable.
void Tracer::record(cudaEvent_t ev, cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(st, &cs);
  if (cs == cudaStreamCaptureStatusActive)
    cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal);
  else
    cudaEventRecord(ev, st);
}
}  // namespace dg

struct dg_mesh {
  dg_ctx* ctx = nullptr;
  DevBuf bufs;
  DevMesh dm{};
  // advection and reaction fields of dg_assemble_varcoef (dg_mesh_set_fields;
  // default the Sec. 4.2 fields)
  VcFields fields{};
  bool fields_set = false;
  dg_bsr_info info{};
  std::vector<int> row_ptr, col;
  std::vector<int64_t> blk_off, dof_off;
  const void* vol_vals = nullptr;  // vals last written by dg_assemble_volume
  // library-owned buffers of the host-memory path
  void* h_vals = nullptr;
  void* h_rhs = nullptr;
  int h_prec = -1;
  // pipelined host entry points (dg_assemble_host_submit / _wait): two device
  // slots for the system, a copy stream, and per slot the events of its pass
  // (computed, on the context's stream) and of its copy back (done)
  void* hp_vals[2] = {nullptr, nullptr};
  void* hp_rhs[2] = {nullptr, nullptr};
  int hp_prec = -1;
  cudaStream_t hp_copy = nullptr;
  cudaEvent_t hp_computed[2] = {nullptr, nullptr}, hp_done[2] = {nullptr, nullptr};
  long long hp_next = 0;
  // launch shape per precision, recorded by dg_graph_create's autotuner and
  // used by the per-step entry points (dg_assemble_step, dg_assemble_host)
  // (kept with the context's volume-path setting it was tuned under)
  int shape_set[4] = {0, 0, 0, 0}, shape_occ[4] = {0, 0, 0, 0}, shape_conc[4] = {0, 0, 0, 0};
  int shape_path[4] = {-1, -1, -1, -1}, shape_vm[4] = {0, 0, 0, 0};
  int shape_tile[4][9] = {{0}};  // tuned tile variant per degree
  int shape_persist[4] = {0, 0, 0, 0};  // tuned: the persistent pass
  int shape_split[4][9] = {{0}};  // tuned parts per degree group (0 = 1)
  double* X[3] = {nullptr, nullptr, nullptr};
  double* a = nullptr;
  double flops[kKinds][9] = {{0}}, words[kKinds][9] = {{0}};
  double mom_exec[2][9] = {{0}}, mom_pt[9] = {0};
  double offd[2][9][9] = {{{0}}};
  std::vector<int> batch_elem_off;  // element offset of each batch member (empty: one mesh)
  // partition meshes: local -> global element and vertex ids, owned flags
  std::vector<int> part_elem, part_vert;
  std::vector<int8_t> owned_h;  // empty: every element owned
  // host copies used to rebuild the work list when volume rules change
  std::vector<int> p_h, nvq_h, nqf_h;
  std::vector<double> vfma_h;  // algorithmic FMAs per volume point of each element
  std::vector<int> perm_fan;  // the sub-simplex-rule work list
  std::vector<int> perm_h;    // the current work list (host copy of perm_dev)
  double pattern_ms = 0.0, upload_ms = 0.0;  // wall time of the pattern build and of the whole upload
  bool pattern_on_device = false;
  // persistent pass: queue word, pad and the elements' moment flags
  // (zeroed before each launch), the work list of tiles and what it was built for
  int* pk_sync = nullptr;
  // one work list per moment mask, kept for the mesh's life (recorded graphs
  // hold their list's address); retired lists were built for an earlier
  // element work list (learned rules installed or cleared)
  struct PkList {
    int key;
    int4* items;
    int n;
  };
  std::vector<PkList> pk_lists, pk_retired;
  // learned quadrature (2D)
  double *lq_mom = nullptr, *lq_mmom = nullptr, *lq_rule = nullptr, *lq64 = nullptr;
  float *lq32 = nullptr, *lq_resid = nullptr, *lq_out = nullptr;
  int *lq_elig = nullptr, *lq_ok = nullptr, *lq_okm = nullptr;
  void* lq_feat = nullptr;
  int* perm_dev = nullptr;  // device work list (owned by bufs)
  // space-time slabs, per space (DG_SPACE_P, DG_SPACE_PQ): block and dof
  // offsets on the host and the device (owned by bufs), and the scratch of
  // the spatial pass: blocks B, mass matrix M (diagonal blocks' places),
  // load vector l, and the zero diffusion of the mass pass
  std::vector<int64_t> slab_blk_h[2], slab_dof_h[2];
  int64_t* slab_blk[2] = {nullptr, nullptr};
  int64_t* slab_dof[2] = {nullptr, nullptr};
  double *slab_B = nullptr, *slab_M = nullptr, *slab_l = nullptr, *slab_zero_a = nullptr;
  ~dg_mesh() {
    if (h_vals) cudaFree(h_vals);
    if (h_rhs) cudaFree(h_rhs);
    if (hp_copy) cudaStreamSynchronize(hp_copy);
    for (int i = 0; i < 2; ++i) {
      if (hp_vals[i]) cudaFree(hp_vals[i]);
      if (hp_rhs[i]) cudaFree(hp_rhs[i]);
      if (hp_computed[i]) cudaEventDestroy(hp_computed[i]);
      if (hp_done[i]) cudaEventDestroy(hp_done[i]);
    }
    if (hp_copy) cudaStreamDestroy(hp_copy);
    void* q[] = {lq_mom, lq_mmom, lq_rule, lq64, lq32, lq_resid, lq_elig, lq_ok, lq_okm, lq_feat, lq_out, pk_sync};
    for (void* x : q)
      if (x) cudaFree(x);
    for (auto& l : pk_lists) cudaFree(l.items);
    for (auto& l : pk_retired) cudaFree(l.items);
  }
};

static void trace_reset(dg_ctx* ctx, const dg_mesh* mesh) {
  ctx->tracer.n = 0;
  ctx->tracer.flops = &mesh->flops[0][0];
  ctx->tracer.words = &mesh->words[0][0];
  ctx->tracer.xflops = &mesh->mom_exec[0][0];
  ctx->tracer.offd = &mesh->offd[0][0][0];
}

namespace {

int build_rule_tables(dg_ctx* ctx) {
  for (int dim = 2; dim <= 3; ++dim) {
    RuleTables& rt = ctx->rt[dim];
    const int pmax = dim == 2 ? kPMax2 : kPMax3;
    std::vector<double> vol, face, pts;
    for (int p = 1; p <= pmax; ++p) {
      simplex_rule(dim, p + 2, pts);
      rt.vol_off[p] = (int)(vol.size() / (dim + 1));
      rt.vol_n[p] = (int)(pts.size() / (dim + 1));
      vol.insert(vol.end(), pts.begin(), pts.end());
    }
    for (int n = 1; n <= pmax + 1; ++n) {
      simplex_rule(dim - 1, n, pts);
      rt.face_off[n] = (int)(face.size() / dim);
      rt.face_n[n] = (int)(pts.size() / dim);
      face.insert(face.end(), pts.begin(), pts.end());
    }
    double *v64, *f64;
    float *v32, *f32;
    DG_CUDA_TRY(ctx->bufs.alloc(&v64, vol.size()));
    DG_CUDA_TRY(ctx->bufs.alloc(&v32, vol.size()));
    DG_CUDA_TRY(ctx->bufs.alloc(&f64, face.size()));
    DG_CUDA_TRY(ctx->bufs.alloc(&f32, face.size()));
    std::vector<float> vf(vol.begin(), vol.end()), ff(face.begin(), face.end());
    DG_CUDA_TRY(cudaMemcpy(v64, vol.data(), vol.size() * 8, cudaMemcpyHostToDevice));
    DG_CUDA_TRY(cudaMemcpy(v32, vf.data(), vf.size() * 4, cudaMemcpyHostToDevice));
    DG_CUDA_TRY(cudaMemcpy(f64, face.data(), face.size() * 8, cudaMemcpyHostToDevice));
    DG_CUDA_TRY(cudaMemcpy(f32, ff.data(), ff.size() * 4, cudaMemcpyHostToDevice));
    rt.vol64 = v64;
    rt.vol32 = v32;
    rt.face64 = f64;
    rt.face32 = f32;
  }
  // Legendre linearisation: P_a P_b, P'_a P_b, P'_a P'_b = sum_c coef P_c,
  // coef = (2c + 1)/2 int_{-1}^{1} (product) P_c, by Gauss-Legendre with
  // enough points for degree 4 kPMaxLin (exact)
  {
    constexpr int PL = kPMaxLin + 1, CL = 2 * kPMaxLin + 1;
    std::vector<double> gx, gw;
    gauss_legendre01(2 * kPMaxLin + 2, gx, gw);
    const int ng = (int)gx.size();
    std::vector<double> Pv((size_t)ng * (CL + 1)), dPv((size_t)ng * (CL + 1));
    for (int g = 0; g < ng; ++g) {
      const double t = 2.0 * gx[g] - 1.0;
      double* P = &Pv[(size_t)g * (CL + 1)];
      double* dP = &dPv[(size_t)g * (CL + 1)];
      P[0] = 1.0;
      dP[0] = 0.0;
      P[1] = t;
      dP[1] = 1.0;
      for (int k = 1; k < CL; ++k) {
        P[k + 1] = ((2 * k + 1) * t * P[k] - k * P[k - 1]) / (k + 1);
        dP[k + 1] = dP[k - 1] + (2 * k + 1) * P[k];
      }
    }
    std::vector<double> lin((size_t)3 * PL * PL * CL, 0.0);
    for (int a = 0; a < PL; ++a)
      for (int b = 0; b < PL; ++b)
        for (int c = 0; c < CL; ++c) {
          double s0 = 0, s1 = 0, s2 = 0;
          for (int g = 0; g < ng; ++g) {
            const double* P = &Pv[(size_t)g * (CL + 1)];
            const double* dP = &dPv[(size_t)g * (CL + 1)];
            const double w = 2.0 * gw[g] * P[c];
            s0 += w * P[a] * P[b];
            s1 += w * dP[a] * P[b];
            s2 += w * dP[a] * dP[b];
          }
          const double nc = 0.5 * (2 * c + 1);
          lin[(size_t)(a * PL + b) * CL + c] = nc * s0;
          lin[(size_t)PL * PL * CL + (a * PL + b) * CL + c] = nc * s1;
          lin[(size_t)2 * PL * PL * CL + (a * PL + b) * CL + c] = nc * s2;
        }
    double* l64;
    float* l32;
    DG_CUDA_TRY(ctx->bufs.alloc(&l64, lin.size()));
    DG_CUDA_TRY(ctx->bufs.alloc(&l32, lin.size()));
    std::vector<float> lf(lin.begin(), lin.end());
    DG_CUDA_TRY(cudaMemcpy(l64, lin.data(), lin.size() * 8, cudaMemcpyHostToDevice));
    DG_CUDA_TRY(cudaMemcpy(l32, lf.data(), lf.size() * 4, cudaMemcpyHostToDevice));
    for (int dim = 2; dim <= 3; ++dim) {
      ctx->rt[dim].lin64 = l64;
      ctx->rt[dim].lin32 = l32;
    }
  }
  return DG_OK;
}

template <typename T>
int upload(DevBuf& b, const T** out, const std::vector<T>& v) {
  T* p;
  DG_CUDA_TRY(b.alloc(&p, v.size()));
  if (!v.empty()) DG_CUDA_TRY(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  *out = p;
  return DG_OK;
}

struct HalfFace {
  int key[3];
  int elem;
  int v[3];   // vertices in the element's order (2D: v[0] -> v[1] along its CCW loop)
  bool flip;  // 3D: (v1-v0) x (v2-v0) points into the element
};

bool key_less(const HalfFace& a, const HalfFace& b) {
  for (int i = 0; i < 3; ++i)
    if (a.key[i] != b.key[i]) return a.key[i] < b.key[i];
  return a.elem < b.elem;
}

bool key_eq(const HalfFace& a, const HalfFace& b) {
  return a.key[0] == b.key[0] && a.key[1] == b.key[1] && a.key[2] == b.key[2];
}

struct FaceRec {
  int e0, e1;
  int v[3];
  int key[3];
  bool flip;
};

// Stable LSD radix sort of (key, idx) pairs by key: 11-bit digits (2048
// buckets, whose write positions stay in cache), as many passes as the
// largest key has digits.
void radix_sort_u64(std::vector<uint64_t>& key, std::vector<uint32_t>& idx) {
  const size_t n = key.size();
  if (n < 2) return;
  uint64_t kmax = 0;
  for (size_t i = 0; i < n; ++i) kmax = std::max(kmax, key[i]);
  std::vector<uint64_t> k2(n);
  std::vector<uint32_t> i2(n);
  constexpr int kBits = 11;
  constexpr uint64_t kMask = (1u << kBits) - 1;
  std::vector<size_t> cnt(kMask + 1);
  for (int shift = 0; shift < 64 && (kmax >> shift) != 0; shift += kBits) {
    std::fill(cnt.begin(), cnt.end(), 0);
    for (size_t i = 0; i < n; ++i) ++cnt[(key[i] >> shift) & kMask];
    size_t sum = 0;
    for (size_t& c : cnt) {
      const size_t t = c;
      c = sum;
      sum += t;
    }
    for (size_t i = 0; i < n; ++i) {
      const size_t at = cnt[(key[i] >> shift) & kMask]++;
      k2[at] = key[i];
      i2[at] = idx[i];
    }
    key.swap(k2);
    idx.swap(i2);
  }
}

}  // namespace

struct Plan {
  std::vector<int> sub_elem, if_e0, if_e1, if_fptr, row_ptr, col, diag_blk, slot01, slot10, blk_if;
  std::vector<int64_t> blk_off, dof_off;
  std::vector<FaceRec> F;
  std::vector<int> f_e0, f_e1, f_v, f_nq, hf_ptr, hf_face, hf_qoff, e_nqf, uvptr, uvidx, elem_perm, if_perm;
  std::vector<int8_t> hf_side, f_flip;
  std::vector<int> f_hf;     // [2][nf] half-face index of each face side (-1: none)
  std::vector<int> blk_rec;  // [nnzb][4]: k, first half face of the interface in the row, faces, p_k
  int elem_pstart[9] = {0}, if_pstart[9] = {0};
  int nsub = 0, nf = 0, nint = 0, ni = 0, nhf = 0;
  int64_t nqvol = 0, nqface = 0;
  // algorithmic flops / words per launch group [kind][p] (kind 0: row
  // kernel of degree p, whole block rows and load vector)
  double flops[kKinds][9] = {{0}}, words[kKinds][9] = {{0}};
  double mom_exec[2][9] = {{0}};  // moment form: executed flops of the volume launch (without, with the own faces), by degree
  double mom_pt[9] = {0};    // moment form: executed flops per volume point, by degree
  double offd[2][9][9] = {{{0}}};  // interface terms of degree-p rows by neighbour degree: flops, words
};

extern "C" {

const char* dg_last_error(void) { return g_err.c_str(); }

int dg_create(dg_ctx** out, int device, void* stream) {
  if (!out) return fail(DG_ERR_ARG, "dg_create: null output pointer");
  *out = nullptr;
  int ndev = 0;
  DG_CUDA_TRY(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return fail(DG_ERR_ARG, "dg_create: device %d out of range (%d devices)", device, ndev);
  DG_CUDA_TRY(cudaSetDevice(device));
  dg_ctx* ctx = new (std::nothrow) dg_ctx();
  if (!ctx) return fail(DG_ERR_OOM, "dg_create: out of host memory");
  ctx->device = device;
  ctx->stream = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) {
    delete ctx;
    return fail(DG_ERR_CUDA, "dg_create: %s", cudaGetErrorString(e));
  }
  int rc = build_rule_tables(ctx);
  if (rc != DG_OK) {
    delete ctx;
    return rc;
  }
  if (cudaMalloc(&ctx->status_dev, sizeof(int)) != cudaSuccess ||
      cudaMemset(ctx->status_dev, 0, sizeof(int)) != cudaSuccess) {
    delete ctx;
    return fail(DG_ERR_OOM, "dg_create: status word");
  }
  *out = ctx;
  return DG_OK;
}

void dg_destroy(dg_ctx* ctx) { delete ctx; }

int dg_mesh_free(dg_mesh* mesh) {
  delete mesh;
  return DG_OK;
}

// owned == nullptr: every element is assembled.  Otherwise only elements
// with owned[e] != 0 get block rows, load-vector entries and work-list
// entries; the others (the halo of a partition) only supply geometry.
// The descriptor's arguments and per-element scalars (the checks that need
// no faces): sizes, pointers, problem data, elem_ptr, degrees, a, vertex ids.
static int check_desc(const dg_mesh_desc* d) {
  if (!d) return fail(DG_ERR_ARG, "null mesh descriptor");
  const int dim = d->dim;
  if (dim != 2 && dim != 3) return fail(DG_ERR_ARG, "dim must be 2 or 3 (got %d)", dim);
  if (d->nv <= 0 || d->ne <= 0) return fail(DG_ERR_ARG, "nv and ne must be positive");
  if (!d->x || !d->y || (dim == 3 && !d->z) || !d->elem_ptr || !d->elem_idx || !d->p || !d->a)
    return fail(DG_ERR_ARG, "dg_mesh_upload: null array in descriptor");
  if (d->source < 0 || d->source > 2) return fail(DG_ERR_ARG, "unknown source %d", d->source);
  if (!(d->c_sigma > 0.0)) return fail(DG_ERR_MESH, "C_sigma must be positive");
  if (!(d->c >= 0.0)) return fail(DG_ERR_MESH, "c must be >= 0");
  if (d->neumann < 0 || d->neumann >= (1 << (2 * dim)))
    return fail(DG_ERR_ARG, "neumann mask 0x%x names a side past dimension %d", (unsigned)d->neumann, dim);
  const int nv = d->nv, ne = d->ne;
  const int pmax = dim == 2 ? kPMax2 : kPMax3;
  if (d->elem_ptr[0] != 0) return fail(DG_ERR_MESH, "elem_ptr[0] must be 0");
  for (int e = 0; e < ne; ++e) {
    const int cnt = d->elem_ptr[e + 1] - d->elem_ptr[e];
    if (cnt < (dim == 2 ? 3 : 1)) return fail(DG_ERR_MESH, "element %d has %d entries", e, cnt);
    if (d->p[e] < 1 || d->p[e] > pmax) return fail(DG_ERR_MESH, "element %d: p = %d outside 1..%d", e, d->p[e], pmax);
    if (!(d->a[e] > 0.0) || !std::isfinite(d->a[e])) return fail(DG_ERR_MESH, "element %d: a must be > 0", e);
  }
  const int nidx = d->elem_ptr[ne] * (dim == 2 ? 1 : 4);
  for (int i = 0; i < nidx; ++i)
    if (d->elem_idx[i] < 0 || d->elem_idx[i] >= nv) return fail(DG_ERR_MESH, "vertex index %d out of range", d->elem_idx[i]);
  return DG_OK;
}

static int plan_mesh(const dg_mesh_desc* d, Plan& P, const int8_t* owned = nullptr) {
  if (int rc = check_desc(d)) return rc;
  const int dim = d->dim, nv = d->nv, ne = d->ne;
  const double* X[3] = {d->x, d->y, dim == 3 ? d->z : nullptr};

  // --- geometric validity (host, FP64)
  if (dim == 2) {
    for (int e = 0; e < ne; ++e) {
      const int b = d->elem_ptr[e], k = d->elem_ptr[e + 1] - b;
      double A = 0, cx = 0, cy = 0;
      for (int i = 0; i < k; ++i) {
        const int v0 = d->elem_idx[b + i], v1 = d->elem_idx[b + (i + 1) % k];
        const double cr = X[0][v0] * X[1][v1] - X[0][v1] * X[1][v0];
        A += 0.5 * cr;
        cx += (X[0][v0] + X[0][v1]) * cr;
        cy += (X[1][v0] + X[1][v1]) * cr;
      }
      if (!(A > 0.0)) return fail(DG_ERR_MESH, "element %d: loop is not counter-clockwise (area %g)", e, A);
      cx /= 6 * A;
      cy /= 6 * A;
      for (int i = 0; i < k; ++i) {
        const int v0 = d->elem_idx[b + i], v1 = d->elem_idx[b + (i + 1) % k];
        const double tri = (X[0][v0] - cx) * (X[1][v1] - cy) - (X[1][v0] - cy) * (X[0][v1] - cx);
        if (!(tri > 0.0)) return fail(DG_ERR_MESH, "element %d: fan triangle %d has non-positive area", e, i);
      }
    }
  } else {
    const int nt = d->elem_ptr[ne];
    for (int t = 0; t < nt; ++t) {
      const int* tv = d->elem_idx + 4 * t;
      double u[3], v[3], w[3];
      for (int q = 0; q < 3; ++q) {
        u[q] = X[q][tv[1]] - X[q][tv[0]];
        v[q] = X[q][tv[2]] - X[q][tv[0]];
        w[q] = X[q][tv[3]] - X[q][tv[0]];
      }
      const double det = u[0] * (v[1] * w[2] - v[2] * w[1]) - u[1] * (v[0] * w[2] - v[2] * w[0]) +
                         u[2] * (v[0] * w[1] - v[1] * w[0]);
      if (!(std::fabs(det) > 0.0)) return fail(DG_ERR_MESH, "tetrahedron %d has zero volume", t);
    }
  }

  // --- faces
  std::vector<HalfFace> H;
  std::vector<int>& sub_elem = P.sub_elem;
  if (dim == 2) {
    H.reserve(d->elem_ptr[ne]);
    sub_elem.resize(d->elem_ptr[ne]);
    for (int e = 0; e < ne; ++e) {
      const int b = d->elem_ptr[e], k = d->elem_ptr[e + 1] - b;
      for (int i = 0; i < k; ++i) {
        HalfFace h{};
        const int v0 = d->elem_idx[b + i], v1 = d->elem_idx[b + (i + 1) % k];
        if (v0 == v1) return fail(DG_ERR_MESH, "element %d: repeated vertex in loop", e);
        h.key[0] = std::min(v0, v1);
        h.key[1] = std::max(v0, v1);
        h.key[2] = -1;
        h.elem = e;
        h.v[0] = v0;
        h.v[1] = v1;
        h.v[2] = -1;
        H.push_back(h);
        sub_elem[b + i] = e;
      }
    }
  } else {
    const int nt = d->elem_ptr[ne];
    H.reserve((size_t)4 * nt);
    sub_elem.resize(nt);
    for (int e = 0; e < ne; ++e)
      for (int t = d->elem_ptr[e]; t < d->elem_ptr[e + 1]; ++t) {
        sub_elem[t] = e;
        const int* tv = d->elem_idx + 4 * t;
        for (int o = 0; o < 4; ++o) {
          HalfFace h{};
          int c = 0;
          for (int i = 0; i < 4; ++i)
            if (i != o) h.v[c++] = tv[i];
          // orient (v0, v1, v2) so that (v1-v0) x (v2-v0) points away from tv[o]
          double u[3], v[3], w[3];
          for (int q = 0; q < 3; ++q) {
            u[q] = X[q][h.v[1]] - X[q][h.v[0]];
            v[q] = X[q][h.v[2]] - X[q][h.v[0]];
            w[q] = X[q][tv[o]] - X[q][h.v[0]];
          }
          const double cr[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]};
          // keep the tetrahedron's vertex order (the face rule is applied in
          // this order); record whether the right-hand normal points inward
          h.flip = cr[0] * w[0] + cr[1] * w[1] + cr[2] * w[2] > 0.0;
          int kk[3] = {h.v[0], h.v[1], h.v[2]};
          std::sort(kk, kk + 3);
          for (int q = 0; q < 3; ++q) h.key[q] = kk[q];
          h.elem = e;
          H.push_back(h);
        }
      }
  }
  // Order the half faces by (key, element).  They were generated element by
  // element, so a stable sort by the key alone gives that order: a radix sort
  // of the sorted vertex ids as one number in base nv (below 2^64 for
  // nv < 2^21), else a comparison sort.
  std::vector<uint32_t> ord(H.size());
  std::iota(ord.begin(), ord.end(), 0u);
  if (dim == 2 || nv < (1 << 21)) {
    std::vector<uint64_t> hk(H.size());
    const uint64_t base = (uint64_t)nv;
    for (size_t i = 0; i < H.size(); ++i)
      hk[i] = dim == 2 ? (uint64_t)H[i].key[0] * base + (uint64_t)H[i].key[1]
                       : ((uint64_t)H[i].key[0] * base + (uint64_t)H[i].key[1]) * base + (uint64_t)H[i].key[2];
    radix_sort_u64(hk, ord);
  } else {
    std::stable_sort(ord.begin(), ord.end(), [&](uint32_t a, uint32_t b) { return key_less(H[a], H[b]); });
  }
  std::vector<FaceRec>& F = P.F;
  F.reserve(H.size() / 2 + 1);
  for (size_t i = 0; i < H.size();) {
    const HalfFace& h0 = H[ord[i]];
    size_t j = i + 1;
    while (j < H.size() && key_eq(h0, H[ord[j]])) ++j;
    const size_t cnt = j - i;
    if (cnt > 2) return fail(DG_ERR_MESH, "a face is shared by %zu element pieces (non-manifold)", cnt);
    const HalfFace* h1 = cnt == 2 ? &H[ord[i + 1]] : nullptr;
    if (h1 && h0.elem == h1->elem) {
      if (dim == 2) return fail(DG_ERR_MESH, "element %d traverses an edge twice", h0.elem);
      // interior to one 3D element: not a face
    } else {
      FaceRec f{};
      f.e0 = h0.elem;
      f.e1 = h1 ? h1->elem : -1;
      for (int q = 0; q < 3; ++q) {
        f.v[q] = h0.v[q];
        f.key[q] = h0.key[q];
      }
      f.flip = h0.flip;
      if (dim == 2 && h1 && !(h0.v[0] == h1->v[1] && h0.v[1] == h1->v[0]))
        return fail(DG_ERR_MESH, "elements %d and %d traverse their common edge in the same direction", f.e0, f.e1);
      F.push_back(f);
    }
    i = j;
  }
  std::vector<uint32_t>().swap(ord);
  // Face order: interior faces first, then by (e0, e1, key).  F is in key
  // order, so a stable sort by (boundary, e0, e1) gives it.
  {
    std::vector<uint64_t> fk(F.size());
    std::vector<uint32_t> fo(F.size());
    const uint64_t base = (uint64_t)ne + 1;  // e0 < ne, e1 + 1 <= ne
    for (size_t i = 0; i < F.size(); ++i) {
      fk[i] = ((uint64_t)(F[i].e1 < 0) * base + (uint64_t)F[i].e0) * base + (uint64_t)(F[i].e1 + 1);
      fo[i] = (uint32_t)i;
    }
    radix_sort_u64(fk, fo);
    std::vector<FaceRec> Fs(F.size());
    for (size_t i = 0; i < F.size(); ++i) Fs[i] = F[fo[i]];
    F.swap(Fs);
  }
  const int nf = (int)F.size();
  int nint = 0;
  while (nint < nf && F[nint].e1 >= 0) ++nint;

  // --- interfaces
  std::vector<int>&if_e0 = P.if_e0, &if_e1 = P.if_e1, &if_fptr = P.if_fptr;
  for (int f = 0; f < nint;) {
    int g = f + 1;
    while (g < nint && F[g].e0 == F[f].e0 && F[g].e1 == F[f].e1) ++g;
    if_e0.push_back(F[f].e0);
    if_e1.push_back(F[f].e1);
    if_fptr.push_back(f);
    f = g;
  }
  if_fptr.push_back(nint);
  const int ni = (int)if_e0.size();

  // --- block-sparse pattern
  std::vector<int> nb(ne);
  for (int e = 0; e < ne; ++e) nb[e] = nbasis(dim, d->p[e]);
  // rows: the element and every element it shares an interface with,
  // ascending; a halo element (not owned) has no block row
  Plan* m = &P;
  std::vector<int>& diag_blk = P.diag_blk;
  diag_blk.assign(ne, -1);
  auto own = [&](int e) { return owned == nullptr || owned[e] != 0; };
  {
    std::vector<int> deg(ne, 0);
    for (int i = 0; i < ni; ++i) {
      ++deg[if_e0[i]];
      ++deg[if_e1[i]];
    }
    m->row_ptr.assign(ne + 1, 0);
    for (int e = 0; e < ne; ++e) m->row_ptr[e + 1] = m->row_ptr[e] + (own(e) ? deg[e] + 1 : 0);
    m->col.resize(m->row_ptr[ne]);
    std::vector<int> fill(ne, 0);
    for (int e = 0; e < ne; ++e)
      if (own(e)) m->col[m->row_ptr[e] + fill[e]++] = e;
    for (int i = 0; i < ni; ++i) {
      const int a = if_e0[i], b = if_e1[i];
      if (own(a)) m->col[m->row_ptr[a] + fill[a]++] = b;
      if (own(b)) m->col[m->row_ptr[b] + fill[b]++] = a;
    }
    for (int e = 0; e < ne; ++e) std::sort(m->col.begin() + m->row_ptr[e], m->col.begin() + m->row_ptr[e + 1]);
  }
  m->blk_off.assign(m->row_ptr[ne] + 1, 0);
  for (int e = 0; e < ne; ++e)
    for (int idx = m->row_ptr[e]; idx < m->row_ptr[e + 1]; ++idx) {
      const int c = m->col[idx];
      m->blk_off[idx + 1] = m->blk_off[idx] + (int64_t)nb[e] * nb[c];
      if (c == e) diag_blk[e] = idx;
    }
  auto slot = [&](int r, int c) {
    const int* b = m->col.data() + m->row_ptr[r];
    const int* en = m->col.data() + m->row_ptr[r + 1];
    return (int)(std::lower_bound(b, en, c) - m->col.data());
  };
  std::vector<int>&slot01 = P.slot01, &slot10 = P.slot10;
  slot01.assign(ni, 0);
  slot10.assign(ni, 0);
  P.blk_if.assign(m->row_ptr[ne], -1);
  for (int i = 0; i < ni; ++i) {
    slot01[i] = own(if_e0[i]) ? slot(if_e0[i], if_e1[i]) : -1;
    slot10[i] = own(if_e1[i]) ? slot(if_e1[i], if_e0[i]) : -1;
    if (slot01[i] >= 0) P.blk_if[slot01[i]] = i;
    if (slot10[i] >= 0) P.blk_if[slot10[i]] = i;
  }
  m->dof_off.assign(ne + 1, 0);
  for (int e = 0; e < ne; ++e) m->dof_off[e + 1] = m->dof_off[e] + (own(e) ? nb[e] : 0);

  // --- half faces (element -> faces, global face order) and face points
  std::vector<int>&f_e0 = P.f_e0, &f_e1 = P.f_e1, &f_v = P.f_v, &f_nq = P.f_nq;
  P.f_flip.assign(nf, 0);
  f_e0.assign(nf, 0);
  f_e1.assign(nf, 0);
  f_v.assign((size_t)dim * nf, 0);
  f_nq.assign(nf, 0);
  std::vector<int> hf_cnt(ne + 1, 0);
  int64_t nqface = 0;
  for (int f = 0; f < nf; ++f) {
    f_e0[f] = F[f].e0;
    f_e1[f] = F[f].e1;
    for (int q = 0; q < dim; ++q) f_v[(size_t)dim * f + q] = F[f].v[q];
    P.f_flip[f] = F[f].flip ? 1 : 0;
    const int pm = F[f].e1 >= 0 ? std::max(d->p[F[f].e0], d->p[F[f].e1]) : d->p[F[f].e0];
    f_nq[f] = pm + 1;
    nqface += dim == 2 ? f_nq[f] : f_nq[f] * f_nq[f];
    hf_cnt[F[f].e0 + 1]++;
    if (F[f].e1 >= 0) hf_cnt[F[f].e1 + 1]++;
  }
  std::vector<int>& hf_ptr = P.hf_ptr;
  hf_ptr.assign(ne + 1, 0);
  for (int e = 0; e < ne; ++e) hf_ptr[e + 1] = hf_ptr[e] + hf_cnt[e + 1];
  const int nhf = hf_ptr[ne];
  std::vector<int>&hf_face = P.hf_face, &hf_qoff = P.hf_qoff, &e_nqf = P.e_nqf;
  hf_face.assign(nhf, 0);
  hf_qoff.assign(nhf, 0);
  e_nqf.assign(ne, 0);
  std::vector<int> fill(ne, 0);
  std::vector<int8_t>& hf_side = P.hf_side;
  hf_side.assign(nhf, 0);
  P.f_hf.assign((size_t)2 * nf, -1);
  for (int f = 0; f < nf; ++f)
    for (int s = 0; s < 2; ++s) {
      const int e = s == 0 ? F[f].e0 : F[f].e1;
      if (e < 0) continue;
      const int k = hf_ptr[e] + fill[e]++;
      hf_face[k] = f;
      hf_side[k] = (int8_t)s;
      hf_qoff[k] = e_nqf[e];
      P.f_hf[(size_t)s * nf + f] = k;
      e_nqf[e] += dim == 2 ? f_nq[f] : f_nq[f] * f_nq[f];
    }
  // off-diagonal block records: an interface's faces are consecutive in the
  // global face order, hence in the row element's half-face list
  P.blk_rec.assign((size_t)4 * m->row_ptr[ne], 0);
  for (int e = 0; e < ne; ++e)
    for (int bk = m->row_ptr[e]; bk < m->row_ptr[e + 1]; ++bk) {
      int* r = &P.blk_rec[(size_t)4 * bk];
      const int it = P.blk_if[bk];
      if (it < 0) {
        r[0] = -1;
        continue;
      }
      const int f0 = if_fptr[it];
      const int hf0 = P.f_hf[(size_t)(if_e0[it] == e ? 0 : 1) * nf + f0];
      r[0] = m->col[bk];
      r[1] = hf0;
      r[2] = if_fptr[it + 1] - f0;
      r[3] = d->p[m->col[bk]];
    }

  // --- unique vertices per element, sub-simplex counts
  std::vector<int>&uvptr = P.uvptr, &uvidx = P.uvidx;
  uvptr.assign(ne + 1, 0);
  if (dim == 2) {
    uvptr.assign(d->elem_ptr, d->elem_ptr + ne + 1);
    uvidx.assign(d->elem_idx, d->elem_idx + d->elem_ptr[ne]);
  } else {
    // each element's distinct vertex ids, ascending: a stamp per vertex marks
    // the ones already taken, then the short list is sorted
    std::vector<int> tmp, stamp(nv, -1);
    uvidx.reserve((size_t)d->elem_ptr[ne]);
    for (int e = 0; e < ne; ++e) {
      tmp.clear();
      for (int i = 4 * d->elem_ptr[e]; i < 4 * d->elem_ptr[e + 1]; ++i) {
        const int v = d->elem_idx[i];
        if (stamp[v] != e) {
          stamp[v] = e;
          tmp.push_back(v);
        }
      }
      std::sort(tmp.begin(), tmp.end());
      uvidx.insert(uvidx.end(), tmp.begin(), tmp.end());
      uvptr[e + 1] = (int)uvidx.size();
    }
  }
  const int nsub = d->elem_ptr[ne];
  int64_t nqvol = 0;
  std::vector<int64_t> cost(ne);
  for (int e = 0; e < ne; ++e) {
    int qt = 1;
    for (int q = 0; q < dim; ++q) qt *= d->p[e] + 2;
    const int64_t nvq = (int64_t)(d->elem_ptr[e + 1] - d->elem_ptr[e]) * qt;
    if (own(e)) nqvol += nvq;
    cost[e] = nvq + e_nqf[e];
  }

  // --- work lists: elements by degree (cost-descending), interfaces by max degree
  std::vector<int>& elem_perm = P.elem_perm;
  elem_perm.clear();
  for (int e = 0; e < ne; ++e)
    if (own(e)) elem_perm.push_back(e);
  std::stable_sort(elem_perm.begin(), elem_perm.end(), [&](int x, int y) {
    if (d->p[x] != d->p[y]) return d->p[x] < d->p[y];
    return cost[x] > cost[y];
  });
  for (int p = 0; p <= 8; ++p) {
    P.elem_pstart[p] = (int)(std::lower_bound(elem_perm.begin(), elem_perm.end(), p,
                                               [&](int e, int pv) { return d->p[e] < pv; }) -
                              elem_perm.begin());
  }
  std::vector<int>& if_perm = P.if_perm;
  if_perm.assign(ni, 0);
  std::vector<int> if_pm(ni), if_np(ni);
  for (int i = 0; i < ni; ++i) {
    if_pm[i] = std::max(d->p[if_e0[i]], d->p[if_e1[i]]);
    if_np[i] = (if_fptr[i + 1] - if_fptr[i]) * (dim == 2 ? (if_pm[i] + 1) : (if_pm[i] + 1) * (if_pm[i] + 1));
  }
  std::iota(if_perm.begin(), if_perm.end(), 0);
  std::stable_sort(if_perm.begin(), if_perm.end(), [&](int x, int y) {
    if (if_pm[x] != if_pm[y]) return if_pm[x] < if_pm[y];
    return if_np[x] > if_np[y];
  });
  for (int p = 0; p <= 8; ++p)
    P.if_pstart[p] = (int)(std::lower_bound(if_perm.begin(), if_perm.end(), p,
                                             [&](int i, int pv) { return if_pm[i] < pv; }) -
                            if_perm.begin());

  // Algorithmic work (FMA = 2 flops), per quadrature point, element of n
  // dofs in dimension d: volume d n(n+1)/2 (symmetric diffusion) +
  // [b or c != 0](n^2 + n(d+1)) + basis n d^2 + 5 d p; own interior-face
  // point 3 n^2 + [b != 0] n^2/2 + basis; boundary-face point 3 n^2 +
  // [b != 0] n^2 + basis; load vector n per volume point and 2n per boundary
  // point.  Off-diagonal block (e, k): 3 n_e n_k + [b != 0] n_e n_k / 2 per
  // interface point (each side's basis is counted once, with its own faces).
  {
    const bool advb = d->b[0] != 0.0 || d->b[1] != 0.0 || (dim == 3 && d->b[2] != 0.0);
    const bool adv = advb || d->c != 0.0;
    const int SV = sub_vals(dim), FV = side_vals(dim);
    for (int e = 0; e < ne; ++e) {
      if (!own(e)) continue;
      const int pe = d->p[e];
      const double n = nb[e];
      const double basis = n * dim * dim + 5.0 * dim * pe;
      int qt = 1;
      for (int q = 0; q < dim; ++q) qt *= pe + 2;
      const double nvq = (double)(d->elem_ptr[e + 1] - d->elem_ptr[e]) * qt;
      double fma = nvq * (dim * n * (n + 1) / 2 + (adv ? n * n + n * (dim + 1) : 0.0) + basis + n);
      double w = n * n + n + (double)(d->elem_ptr[e + 1] - d->elem_ptr[e]) * SV + 2 * dim + 2;
      for (int k = hf_ptr[e]; k < hf_ptr[e + 1]; ++k) {
        const int f = hf_face[k];
        const double qf = dim == 2 ? f_nq[f] : (double)f_nq[f] * f_nq[f];
        const bool bnd = F[f].e1 < 0;
        fma += qf * (3 * n * n + (advb ? (bnd ? n * n : n * n / 2) : 0.0) + basis + (bnd ? 2 * n : 0.0));
        w += FV + 3;
      }
      P.flops[0][pe] += 2.0 * fma;
      P.words[0][pe] += w;
      P.flops[3][pe] += 2.0 * fma;
      P.words[3][pe] += w;
    }
    for (int i = 0; i < ni; ++i) {
      for (int side = 0; side < 2; ++side) {
        const int e = side == 0 ? if_e0[i] : if_e1[i], k = side == 0 ? if_e1[i] : if_e0[i];
        if (!own(e)) continue;
        const double ne_ = nb[e], nk = nb[k];
        double fma = 0.0, w = ne_ * nk;
        for (int f = if_fptr[i]; f < if_fptr[i + 1]; ++f) {
          const double qf = dim == 2 ? f_nq[f] : (double)f_nq[f] * f_nq[f];
          fma += qf * (3 * ne_ * nk + (advb ? ne_ * nk / 2 : 0.0));
          w += 2 * FV + 3;
        }
        P.flops[0][d->p[e]] += 2.0 * fma;
        P.words[0][d->p[e]] += w;
        P.offd[0][d->p[e]][d->p[k]] += 2.0 * fma;
        P.offd[1][d->p[e]][d->p[k]] += w;
      }
    }
    // The launches of the moment path.  Without the own faces, the volume
    // launch (kind 2) is credited with the volume terms' algorithmic work
    // above (the quadrature sums it evaluates) and the row kernel's
    // faces-only launch beside it (kind 1) with the rest; with them, the
    // moment launch (kind 3) takes the element's volume and own-face terms
    // and the off-diagonal launch (kind 4) the interface terms.  What the
    // moment form executes instead is mom_exec (moment_op_tables).  It is
    // reported as the "row_pass_executed" record beside "row_pass".
    MomentOps ops;
    moment_op_tables(dim, ops);
    for (int e = 0; e < ne; ++e) {
      if (!own(e)) continue;
      const int pe = d->p[e];
      const double n = nb[e];
      int qt = 1;
      for (int q = 0; q < dim; ++q) qt *= pe + 2;
      const double nvq = (double)(d->elem_ptr[e + 1] - d->elem_ptr[e]) * qt;
      const double vol_direct = nvq * (dim * n * (n + 1) / 2 + (adv ? n * n + n * (dim + 1) : 0.0) +
                                       n * dim * dim + 5.0 * dim * pe + n);
      const double vol_words = n * n + n + (double)(d->elem_ptr[e + 1] - d->elem_ptr[e]) * SV + 2 * dim + 2;
      double nfq = 0.0, nbq = 0.0;  // own-face points, boundary-face points
      for (int k = hf_ptr[e]; k < hf_ptr[e + 1]; ++k) {
        const int f = hf_face[k];
        const double qf = dim == 2 ? f_nq[f] : (double)f_nq[f] * f_nq[f];
        nfq += qf;
        if (F[f].e1 < 0) nbq += qf;
      }
      P.flops[1][pe] -= 2.0 * vol_direct;
      P.words[1][pe] -= vol_words;
      P.flops[2][pe] += 2.0 * vol_direct;
      P.words[2][pe] += vol_words;
      const double vx = nvq * ops.pt[pe] + ops.map[pe];
      P.mom_exec[0][pe] += 2.0 * vx;
      P.mom_exec[1][pe] += 2.0 * (vx + nfq * ops.fpt[pe] + nbq * ops.bnd[pe] + ops.mapf[pe]);
    }
    for (int pp = 0; pp <= 8; ++pp) {
      P.flops[1][pp] += P.flops[0][pp];
      P.words[1][pp] += P.words[0][pp];
      P.mom_pt[pp] = 2.0 * ops.pt[pp];
    }
  }
  P.nsub = nsub;
  P.nf = nf;
  P.nint = nint;
  P.ni = ni;
  P.nhf = nhf;
  P.nqvol = nqvol;
  P.nqface = nqface;
  return DG_OK;
}

static void fill_info(const dg_mesh_desc* d, const Plan& P, dg_bsr_info& I) {
  I.ne = d->ne;
  I.nnzb = P.row_ptr[d->ne];
  I.nvals = P.blk_off[I.nnzb];
  I.ndofs = P.dof_off[d->ne];
  I.nfaces = P.nf;
  I.ninterfaces = P.ni;
  I.nbfaces = P.nf - P.nint;
  I.nsub = P.nsub;
  I.nqvol = P.nqvol;
  I.nqface = P.nqface;
}

int dg_mesh_check(const dg_mesh_desc* d, dg_bsr_info* info, int* row_ptr, int* col, int64_t* blk_off) {
  Plan P;
  int rc = plan_mesh(d, P);
  if (rc != DG_OK) return rc;
  dg_bsr_info I{};
  fill_info(d, P, I);
  if (info) *info = I;
  if (row_ptr) std::copy(P.row_ptr.begin(), P.row_ptr.end(), row_ptr);
  if (col) std::copy(P.col.begin(), P.col.end(), col);
  if (blk_off) std::copy(P.blk_off.begin(), P.blk_off.end(), blk_off);
  return DG_OK;
}

}  // extern "C"

// The geometry records of a mesh (device, written by the geometry kernels).
static int alloc_records(dg_mesh* m, int dim, int ne, int nv, int nsub, int nf, int nhf) {
  DevMesh& dm = m->dm;
  DevBuf& B = m->bufs;
  int rc = DG_OK;
  auto alloc_d = [&](double** p, size_t n) {
    if (rc == DG_OK && B.alloc(p, n) != cudaSuccess) rc = fail(DG_ERR_OOM, "device allocation failed");
  };
  auto alloc_f = [&](float** p, size_t n) {
    if (rc == DG_OK && B.alloc(p, n) != cudaSuccess) rc = fail(DG_ERR_OOM, "device allocation failed");
  };
  alloc_d(&dm.lo, (size_t)dim * ne);
  alloc_d(&dm.L, (size_t)dim * ne);
  alloc_d(&dm.cen, (size_t)dim * ne);
  alloc_d(&dm.vol, ne);
  alloc_d(&dm.h, ne);
  alloc_d(&dm.pen, ne);
  alloc_d(&dm.eg64, (size_t)elem_vals(dim) * ne);
  alloc_f(&dm.eg32, (size_t)elem_vals(dim) * ne);
  if (rc == DG_OK && B.alloc(&dm.xs2, (size_t)dim * nv) != cudaSuccess) rc = fail(DG_ERR_OOM, "device allocation failed");
  alloc_f(&dm.gx32, (size_t)elem_vals(dim) * ne);
  alloc_d(&dm.sg64, (size_t)sub_vals(dim) * nsub);
  alloc_f(&dm.sg32, (size_t)sub_vals(dim) * nsub);
  alloc_d(&dm.fs64, (size_t)2 * side_vals(dim) * nf);
  alloc_d(&dm.fsc64, (size_t)3 * nf);
  alloc_d(&dm.hfr64, (size_t)hf_rec_vals(dim) * nhf);
  alloc_f(&dm.hfr32, (size_t)hf_rec_vals(dim) * nhf);
  // the interface records (the topology and degrees are in place on both
  // upload paths by now)
  dm.if_rec = nullptr;
  if (rc == DG_OK && dm.ni > 0) {
    int4* rec = nullptr;
    if (B.alloc(&rec, (size_t)2 * dm.ni) != cudaSuccess) return fail(DG_ERR_OOM, "device allocation failed");
    launch_iface_recs(dm, rec, m->ctx->stream);
    if (cudaGetLastError() != cudaSuccess) return fail(DG_ERR_CUDA, "interface records: launch failed");
    dm.if_rec = rec;
  }
  return rc;
}

// bounding box of a descriptor's vertices (the sides the Neumann bits name)
static void vertex_box(const dg_mesh_desc* d, double* lo, double* hi) {
  const double* X[3] = {d->x, d->y, d->z};
  for (int q = 0; q < 3; ++q) {
    lo[q] = hi[q] = 0.0;
    if (q >= d->dim) continue;
    lo[q] = hi[q] = X[q][0];
    for (int v = 1; v < d->nv; ++v) {
      lo[q] = std::min(lo[q], X[q][v]);
      hi[q] = std::max(hi[q], X[q][v]);
    }
  }
}

// the problem data and the context's rule tables; box (lo[3], hi[3]) the
// vertex box the Neumann sides refer to, null = the descriptor's own
static void set_problem(dg_mesh* m, const dg_ctx* ctx, const dg_mesh_desc* d, const double* box = nullptr) {
  DevMesh& dm = m->dm;
  for (int q = 0; q < 3; ++q) dm.pb.b[q] = d->b[q];
  if (d->dim == 2) dm.pb.b[2] = 0.0;
  dm.pb.c = d->c;
  dm.pb.source = d->source;
  for (int q = 0; q < 20; ++q) dm.pb.poly[q] = d->poly[q];
  dm.pb.c_sigma = d->c_sigma;
  dm.pb.neumann = d->neumann;
  vertex_box(d, dm.pb.dlo, dm.pb.dhi);
  if (box)
    for (int q = 0; q < 3; ++q) {
      dm.pb.dlo[q] = box[q];
      dm.pb.dhi[q] = box[3 + q];
    }
  dm.pb.round_copies();
  dm.rt = ctx->rt[d->dim];
}

// algorithmic FMAs per volume point of each element (the accounting of the
// learned rules' work lists)
static void set_vfma(dg_mesh* m, const dg_mesh_desc* d) {
  const int dim = d->dim, ne = d->ne;
  const bool adv = d->b[0] != 0.0 || d->b[1] != 0.0 || (dim == 3 && d->b[2] != 0.0) || d->c != 0.0;
  m->vfma_h.resize(ne);
  for (int e = 0; e < ne; ++e) {
    const double n = nbasis(dim, d->p[e]);
    m->vfma_h[e] = dim * n * (n + 1) / 2 + (adv ? n * n + n * (dim + 1) : 0.0) + n * dim * dim + 5.0 * dim * d->p[e] + n;
  }
}

static int upload_impl(dg_ctx* ctx, const dg_mesh_desc* d, const int8_t* owned, dg_mesh** out,
                       const double* box = nullptr) {
  if (!ctx || !d || !out) return fail(DG_ERR_ARG, "dg_mesh_upload: null argument");
  *out = nullptr;
  const auto t_start = std::chrono::steady_clock::now();
  Plan P;
  int prc;
  {
    NvtxRange nv_plan(ctx, "pattern (host)");
    prc = plan_mesh(d, P, owned);
  }
  if (prc != DG_OK) return prc;
  const double plan_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
  const int dim = d->dim, nv = d->nv, ne = d->ne;
  const int nidx = d->elem_ptr[ne] * (dim == 2 ? 1 : 4);
  const double* X[3] = {d->x, d->y, dim == 3 ? d->z : nullptr};
  const int nsub = P.nsub, nf = P.nf, ni = P.ni, nhf = P.nhf;
  dg_mesh* m = new (std::nothrow) dg_mesh();
  if (!m) return fail(DG_ERR_OOM, "out of host memory");
  m->ctx = ctx;
  m->row_ptr = P.row_ptr;
  m->col = P.col;
  std::memcpy(m->flops, P.flops, sizeof P.flops);
  std::memcpy(m->words, P.words, sizeof P.words);
  std::memcpy(m->mom_exec, P.mom_exec, sizeof P.mom_exec);
  std::memcpy(m->mom_pt, P.mom_pt, sizeof P.mom_pt);
  std::memcpy(m->offd, P.offd, sizeof P.offd);
  m->blk_off = P.blk_off;
  m->dof_off = P.dof_off;
  DevMesh& dm = m->dm;
  for (int p = 0; p <= 8; ++p) {
    dm.elem_pstart[p] = P.elem_pstart[p];
    dm.if_pstart[p] = P.if_pstart[p];
  }
  auto& sub_elem = P.sub_elem;
  auto &uvptr = P.uvptr, &uvidx = P.uvidx;
  auto &f_e0 = P.f_e0, &f_e1 = P.f_e1, &f_v = P.f_v, &f_nq = P.f_nq;
  auto &hf_ptr = P.hf_ptr, &hf_face = P.hf_face, &hf_qoff = P.hf_qoff, &e_nqf = P.e_nqf;
  auto& hf_side = P.hf_side;
  auto &if_e0 = P.if_e0, &if_e1 = P.if_e1, &if_fptr = P.if_fptr, &slot01 = P.slot01, &slot10 = P.slot10;
  auto& diag_blk = P.diag_blk;
  auto &elem_perm = P.elem_perm, &if_perm = P.if_perm;
  // --- upload
  dm.dim = dim;
  dm.nv = nv;
  dm.ne = ne;
  dm.nsub = nsub;
  dm.nf = nf;
  dm.ni = ni;
  dm.nhf = nhf;
  DevBuf& B = m->bufs;
  int rc = DG_OK;
  auto up_i = [&](const int** dst, const std::vector<int>& v) {
    if (rc == DG_OK) rc = upload(B, dst, v);
  };
  for (int q = 0; q < 3; ++q) {
    dm.X[q] = nullptr;
    if (q < dim) {
      std::vector<double> v(X[q], X[q] + nv);
      const double* p = nullptr;
      if (rc == DG_OK) rc = upload(B, &p, v);
      dm.X[q] = p;
      m->X[q] = const_cast<double*>(p);
    }
  }
  std::vector<int> eptr(d->elem_ptr, d->elem_ptr + ne + 1), eidx(d->elem_idx, d->elem_idx + nidx);
  up_i(&dm.eptr, eptr);
  up_i(&dm.eidx, eidx);
  up_i(&dm.uvptr, uvptr);
  up_i(&dm.uvidx, uvidx);
  up_i(&dm.sub_elem, sub_elem);
  dm.sub_loc = nullptr;
  std::vector<int> pv(d->p, d->p + ne);
  up_i(&dm.p, pv);
  {
    std::vector<double> av(d->a, d->a + ne);
    if (rc == DG_OK) rc = upload(B, &dm.a, av);
    m->a = const_cast<double*>(dm.a);
  }
  up_i(&dm.f_e0, f_e0);
  up_i(&dm.f_e1, f_e1);
  up_i(&dm.f_v, f_v);
  if (rc == DG_OK) rc = upload(B, &dm.f_flip, P.f_flip);
  {
    const int* p = nullptr;
    up_i(&p, f_nq);
    dm.f_nq = const_cast<int*>(p);
  }
  up_i(&dm.hf_ptr, hf_ptr);
  up_i(&dm.hf_face, hf_face);
  if (rc == DG_OK) rc = upload(B, &dm.hf_side, hf_side);
  up_i(&dm.hf_qoff, hf_qoff);
  up_i(&dm.f_hf, P.f_hf);
  {
    const int* p = nullptr;
    up_i(&p, P.blk_rec);
    dm.blk_rec = reinterpret_cast<const int4*>(p);
  }
  up_i(&dm.e_nqf, e_nqf);
  up_i(&dm.if_e0, if_e0);
  up_i(&dm.if_e1, if_e1);
  up_i(&dm.if_fptr, if_fptr);
  up_i(&dm.if_slot01, slot01);
  up_i(&dm.if_slot10, slot10);
  if (rc == DG_OK) rc = upload(B, &dm.blk_off, m->blk_off);
  up_i(&dm.row_ptr, P.row_ptr);
  up_i(&dm.col, P.col);
  up_i(&dm.blk_if, P.blk_if);
  dm.nmax = 0;
  dm.pmask = 0;
  for (int e = 0; e < ne; ++e) {
    dm.nmax = std::max(dm.nmax, nbasis(dim, d->p[e]));
    dm.pmask |= 1 << d->p[e];
  }
  up_i(&dm.diag_blk, diag_blk);
  if (rc == DG_OK) rc = upload(B, &dm.dof_off, m->dof_off);
  up_i(&dm.elem_perm, elem_perm);
  up_i(&dm.if_perm, if_perm);
  if (rc != DG_OK) {
    delete m;
    return rc;
  }
  rc = alloc_records(m, dim, ne, nv, nsub, nf, nhf);
  if (rc != DG_OK) {
    delete m;
    return rc;
  }
  set_problem(m, ctx, d, box);

  fill_info(d, P, m->info);
  m->p_h.assign(d->p, d->p + ne);
  m->nqf_h = e_nqf;
  m->nvq_h.resize(ne);
  for (int e = 0; e < ne; ++e) {
    int qt = 1;
    for (int q = 0; q < dim; ++q) qt *= d->p[e] + 2;
    m->nvq_h[e] = (d->elem_ptr[e + 1] - d->elem_ptr[e]) * qt;
  }
  set_vfma(m, d);
  m->perm_fan = elem_perm;
  m->perm_h = elem_perm;
  m->perm_dev = const_cast<int*>(dm.elem_perm);
  if (owned) m->owned_h.assign(owned, owned + ne);
  dm.lq_ok = nullptr;
  dm.lq64 = nullptr;
  dm.lq32 = nullptr;
  dm.status = ctx->status_dev;
  dm.nvals = m->info.nvals;
  dm.ndofs = m->info.ndofs;

  cudaSetDevice(ctx->device);
  {
    NvtxRange nv_geo(ctx, "geometry");
    launch_geometry(dm, ctx->stream);
  }
  cudaError_t ce = cudaGetLastError();
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(ctx->stream);
  if (ce != cudaSuccess) {
    delete m;
    return fail(DG_ERR_CUDA, "geometry kernels: %s", cudaGetErrorString(ce));
  }
  m->pattern_ms = plan_ms;
  m->upload_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
  *out = m;
  return DG_OK;
}

// dg_mesh_upload with the block pattern built on the device
// (dg_pattern.cu): the descriptor's scalar checks on the host, the inputs
// uploaded, then faces, interfaces, block rows, half-face lists, work lists
// and the accounting by kernels; the geometry kernels follow as on the host
// path.  The arrays equal the host plan's bit for bit.
static int upload_impl_device(dg_ctx* ctx, const dg_mesh_desc* d, dg_mesh** out) {
  if (!ctx || !d || !out) return fail(DG_ERR_ARG, "dg_mesh_upload: null argument");
  *out = nullptr;
  const auto t_start = std::chrono::steady_clock::now();
  if (int rc = check_desc(d)) return rc;
  const int dim = d->dim, nv = d->nv, ne = d->ne;
  const int nidx = d->elem_ptr[ne] * (dim == 2 ? 1 : 4);
  dg_mesh* m = new (std::nothrow) dg_mesh();
  if (!m) return fail(DG_ERR_OOM, "out of host memory");
  m->ctx = ctx;
  DevMesh& dm = m->dm;
  DevBuf& B = m->bufs;
  int rc = DG_OK;
  cudaSetDevice(ctx->device);
  for (int q = 0; q < 3; ++q) {
    dm.X[q] = nullptr;
    if (q < dim) {
      const double* src = q == 0 ? d->x : q == 1 ? d->y : d->z;
      std::vector<double> v(src, src + nv);
      const double* p = nullptr;
      if (rc == DG_OK) rc = upload(B, &p, v);
      dm.X[q] = p;
      m->X[q] = const_cast<double*>(p);
    }
  }
  {
    std::vector<int> eptr(d->elem_ptr, d->elem_ptr + ne + 1), eidx(d->elem_idx, d->elem_idx + nidx), pv(d->p, d->p + ne);
    if (rc == DG_OK) rc = upload(B, &dm.eptr, eptr);
    if (rc == DG_OK) rc = upload(B, &dm.eidx, eidx);
    if (rc == DG_OK) rc = upload(B, &dm.p, pv);
    std::vector<double> av(d->a, d->a + ne);
    if (rc == DG_OK) rc = upload(B, &dm.a, av);
    m->a = const_cast<double*>(dm.a);
  }
  if (rc != DG_OK) {
    delete m;
    return rc;
  }
  const auto t_pat = std::chrono::steady_clock::now();
  DevPattern P;
  std::string msg;
  auto alloc = [&](size_t bytes) -> void* {
    char* q = nullptr;
    return B.alloc(&q, bytes) == cudaSuccess ? static_cast<void*>(q) : nullptr;
  };
  {
    NvtxRange nv_pat(ctx, "pattern (device)");
    rc = build_pattern_device(d, dm.eptr, dm.eidx, dm.p, dm.X, alloc, ctx->stream, &P, &msg);
  }
  if (rc != DG_OK) {
    delete m;
    return fail(rc, "dg_mesh_upload (device pattern): %s", msg.empty() ? "allocation failed" : msg.c_str());
  }
  m->pattern_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_pat).count();
  m->pattern_on_device = true;
  dm.dim = dim;
  dm.nv = nv;
  dm.ne = ne;
  dm.nsub = P.nsub;
  dm.nf = P.nf;
  dm.ni = P.ni;
  dm.nhf = P.nhf;
  dm.uvptr = P.uvptr;
  dm.uvidx = P.uvidx;
  dm.sub_elem = P.sub_elem;
  dm.sub_loc = nullptr;
  dm.f_e0 = P.f_e0;
  dm.f_e1 = P.f_e1;
  dm.f_v = P.f_v;
  dm.f_flip = P.f_flip;
  dm.f_nq = P.f_nq;
  dm.f_hf = P.f_hf;
  dm.hf_ptr = P.hf_ptr;
  dm.hf_face = P.hf_face;
  dm.hf_side = P.hf_side;
  dm.hf_qoff = P.hf_qoff;
  dm.e_nqf = P.e_nqf;
  dm.if_e0 = P.if_e0;
  dm.if_e1 = P.if_e1;
  dm.if_fptr = P.if_fptr;
  dm.if_slot01 = P.slot01;
  dm.if_slot10 = P.slot10;
  dm.row_ptr = P.row_ptr;
  dm.col = P.col;
  dm.blk_if = P.blk_if;
  dm.blk_off = P.blk_off;
  dm.diag_blk = P.diag_blk;
  dm.dof_off = P.dof_off;
  dm.blk_rec = P.blk_rec;
  dm.elem_perm = P.elem_perm;
  dm.if_perm = P.if_perm;
  for (int q = 0; q <= 8; ++q) {
    dm.elem_pstart[q] = P.elem_pstart[q];
    dm.if_pstart[q] = P.if_pstart[q];
  }
  dm.nmax = 0;
  dm.pmask = 0;
  for (int e = 0; e < ne; ++e) {
    dm.nmax = std::max(dm.nmax, nbasis(dim, d->p[e]));
    dm.pmask |= 1 << d->p[e];
  }
  m->row_ptr = std::move(P.h_row_ptr);
  m->col = std::move(P.h_col);
  m->blk_off = std::move(P.h_blk_off);
  m->dof_off = std::move(P.h_dof_off);
  std::memcpy(m->flops, P.flops, sizeof P.flops);
  std::memcpy(m->words, P.words, sizeof P.words);
  std::memcpy(m->mom_exec, P.mom_exec, sizeof P.mom_exec);
  std::memcpy(m->mom_pt, P.mom_pt, sizeof P.mom_pt);
  std::memcpy(m->offd, P.offd, sizeof P.offd);
  rc = alloc_records(m, dim, ne, nv, P.nsub, P.nf, P.nhf);
  if (rc != DG_OK) {
    delete m;
    return rc;
  }
  set_problem(m, ctx, d);
  m->info.ne = ne;
  m->info.nnzb = P.nnzb;
  m->info.nvals = P.nvals;
  m->info.ndofs = P.ndofs;
  m->info.nfaces = P.nf;
  m->info.ninterfaces = P.ni;
  m->info.nbfaces = P.nf - P.nint;
  m->info.nsub = P.nsub;
  m->info.nqvol = P.nqvol;
  m->info.nqface = P.nqface;
  m->p_h.assign(d->p, d->p + ne);
  m->nqf_h = P.h_e_nqf;
  m->nvq_h = P.h_nvq;
  set_vfma(m, d);
  m->perm_fan = P.h_perm;
  m->perm_h = P.h_perm;
  m->perm_dev = P.elem_perm;
  dm.lq_ok = nullptr;
  dm.lq64 = nullptr;
  dm.lq32 = nullptr;
  dm.status = ctx->status_dev;
  dm.nvals = m->info.nvals;
  dm.ndofs = m->info.ndofs;
  {
    NvtxRange nv_geo(ctx, "geometry");
    launch_geometry(dm, ctx->stream);
  }
  cudaError_t ce = cudaGetLastError();
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(ctx->stream);
  if (ce != cudaSuccess) {
    delete m;
    return fail(DG_ERR_CUDA, "geometry kernels: %s", cudaGetErrorString(ce));
  }
  m->upload_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
  *out = m;
  return DG_OK;
}

extern "C" {

int dg_mesh_upload(dg_ctx* ctx, const dg_mesh_desc* d, dg_mesh** out) {
  NvtxRange nv_(ctx, "dg_mesh_upload");
  if (ctx && ctx->pattern_device) return upload_impl_device(ctx, d, out);
  return upload_impl(ctx, d, nullptr, out);
}

int dg_mesh_array(const dg_mesh* mesh, const char* name, void* host, int64_t cap_bytes, int64_t* bytes) {
  if (!mesh || !name) return fail(DG_ERR_ARG, "dg_mesh_array: null argument");
  const DevMesh& m = mesh->dm;
  const int ne = m.ne, nf = m.nf, ni = m.ni, nhf = m.nhf, nnzb = mesh->info.nnzb, dim = m.dim;
  struct A {
    const char* n;
    const void* p;
    int64_t b;
  };
  const int nuv = dim == 2 ? mesh->info.nsub : (int)0;
  int nuv3 = 0;
  if (dim == 3) cudaMemcpy(&nuv3, m.uvptr + ne, sizeof(int), cudaMemcpyDeviceToHost);
  const A tab[] = {
      {"row_ptr", m.row_ptr, 4LL * (ne + 1)},    {"col", m.col, 4LL * nnzb},
      {"blk_off", m.blk_off, 8LL * (nnzb + 1)},  {"dof_off", m.dof_off, 8LL * (ne + 1)},
      {"blk_if", m.blk_if, 4LL * nnzb},          {"diag_blk", m.diag_blk, 4LL * ne},
      {"blk_rec", m.blk_rec, 16LL * nnzb},       {"f_e0", m.f_e0, 4LL * nf},
      {"f_e1", m.f_e1, 4LL * nf},                {"f_v", m.f_v, 4LL * dim * nf},
      {"f_flip", m.f_flip, 1LL * nf},            {"f_nq", m.f_nq, 4LL * nf},
      {"f_hf", m.f_hf, 8LL * nf},                {"hf_ptr", m.hf_ptr, 4LL * (ne + 1)},
      {"hf_face", m.hf_face, 4LL * nhf},         {"hf_side", m.hf_side, 1LL * nhf},
      {"hf_qoff", m.hf_qoff, 4LL * nhf},         {"e_nqf", m.e_nqf, 4LL * ne},
      {"if_e0", m.if_e0, 4LL * ni},              {"if_e1", m.if_e1, 4LL * ni},
      {"if_fptr", m.if_fptr, 4LL * (ni + 1)},    {"if_slot01", m.if_slot01, 4LL * ni},
      {"if_slot10", m.if_slot10, 4LL * ni},      {"elem_perm", m.elem_perm, 4LL * ne},
      {"if_perm", m.if_perm, 4LL * ni},          {"sub_elem", m.sub_elem, 4LL * mesh->info.nsub},
      {"uvptr", m.uvptr, 4LL * (ne + 1)},        {"uvidx", m.uvidx, 4LL * (dim == 2 ? nuv : nuv3)},
      {"elem_pstart", nullptr, 4LL * 9},         {"if_pstart", nullptr, 4LL * 9},
  };
  for (const A& a : tab) {
    if (std::strcmp(a.n, name) != 0) continue;
    if (bytes) *bytes = a.b;
    if (!host) return DG_OK;
    if (cap_bytes < a.b) return fail(DG_ERR_ARG, "dg_mesh_array: %s needs %lld bytes", name, (long long)a.b);
    if (!a.p) {
      std::memcpy(host, std::strcmp(name, "elem_pstart") == 0 ? m.elem_pstart : m.if_pstart, 36);
      return DG_OK;
    }
    DG_CUDA_TRY(cudaMemcpy(host, a.p, a.b, cudaMemcpyDeviceToHost));
    return DG_OK;
  }
  return fail(DG_ERR_ARG, "dg_mesh_array: unknown array %s", name);
}

int dg_set_pattern_device(dg_ctx* ctx, int on) {
  if (!ctx) return fail(DG_ERR_ARG, "dg_set_pattern_device: null context");
  ctx->pattern_device = on != 0;
  return DG_OK;
}

int dg_mesh_timings(const dg_mesh* mesh, double* pattern_ms, double* upload_ms, int* on_device) {
  if (!mesh) return fail(DG_ERR_ARG, "dg_mesh_timings: null mesh");
  if (pattern_ms) *pattern_ms = mesh->pattern_ms;
  if (upload_ms) *upload_ms = mesh->upload_ms;
  if (on_device) *on_device = mesh->pattern_on_device ? 1 : 0;
  return DG_OK;
}

int dg_bsr_layout(const dg_mesh* mesh, dg_bsr_info* out) {
  if (!mesh || !out) return fail(DG_ERR_ARG, "dg_bsr_layout: null argument");
  *out = mesh->info;
  return DG_OK;
}

int dg_bsr_pattern(const dg_mesh* mesh, int* row_ptr, int* col, int64_t* blk_off, int64_t* dof_off) {
  if (!mesh) return fail(DG_ERR_ARG, "dg_bsr_pattern: null mesh");
  if (row_ptr) std::copy(mesh->row_ptr.begin(), mesh->row_ptr.end(), row_ptr);
  if (col) std::copy(mesh->col.begin(), mesh->col.end(), col);
  if (blk_off) std::copy(mesh->blk_off.begin(), mesh->blk_off.end(), blk_off);
  if (dof_off) std::copy(mesh->dof_off.begin(), mesh->dof_off.end(), dof_off);
  return DG_OK;
}

int dg_geometry(dg_ctx* ctx, dg_mesh* mesh) {
  NvtxRange nv_(ctx, "dg_geometry");
  if (!ctx || !mesh) return fail(DG_ERR_ARG, "dg_geometry: null argument");
  trace_reset(ctx, mesh);
  ctx->last_launches = launch_geometry(mesh->dm, ctx->stream, &ctx->tracer);
  DG_CUDA_TRY(cudaGetLastError());
  return DG_OK;
}

int dg_mesh_update(dg_ctx* ctx, dg_mesh* mesh, const double* x, const double* y, const double* z, const double* a) {
  NvtxRange nv_(ctx, "dg_mesh_update");
  if (!ctx || !mesh) return fail(DG_ERR_ARG, "dg_mesh_update: null argument");
  const int nv = mesh->dm.nv, ne = mesh->dm.ne;
  const double* src[3] = {x, y, z};
  for (int q = 0; q < mesh->dm.dim; ++q)
    if (src[q]) DG_CUDA_TRY(cudaMemcpyAsync(mesh->X[q], src[q], sizeof(double) * nv, cudaMemcpyHostToDevice, ctx->stream));
  if (a) DG_CUDA_TRY(cudaMemcpyAsync(mesh->a, a, sizeof(double) * ne, cudaMemcpyHostToDevice, ctx->stream));
  return dg_geometry(ctx, mesh);
}

// The row-kernel launches of one pass over m in precision prec; returns the
// number of launches.
static int dispatch_rows(const DevMesh& m, int prec, int mode, void* vals, void* rhs, int sm_count,
                         const LaunchOpts& lo, Tracer* tr) {
  if (prec == DG_PREC_FP64) {
    double* v = static_cast<double*>(vals);
    double* r = static_cast<double*>(rhs);
    return m.dim == 2 ? launch_row2d_f64(m, mode, v, r, sm_count, lo, tr) : launch_row3d_f64(m, mode, v, r, sm_count, lo, tr);
  }
  float* v = static_cast<float*>(vals);
  float* r = static_cast<float*>(rhs);
  if (prec == DG_PREC_FP32)
    return m.dim == 2 ? launch_row2d_f32(m, mode, v, r, sm_count, lo, tr) : launch_row3d_f32(m, mode, v, r, sm_count, lo, tr);
  if (prec == DG_PREC_BF16X3)
    return m.dim == 2 ? launch_row2d_bf16(m, mode, v, r, sm_count, lo, tr) : launch_row3d_bf16(m, mode, v, r, sm_count, lo, tr);
  return m.dim == 2 ? launch_row2d_tf32(m, mode, v, r, sm_count, lo, tr) : launch_row3d_tf32(m, mode, v, r, sm_count, lo, tr);
}

// Issue the row kernels of one assembly pass on stream st.  concurrent:
// the per-degree launches go to forked side streams and join back into st.
// vpath: volume path (0 per-point contraction, 1 moments, 2 exact 2D moments), -1 the context's
// setting; meshes with learned rules installed take the per-point path
// unless a path is given (their elements have only 28 points each)
static int run_assembly(dg_ctx* ctx, const dg_mesh* mesh, int prec, int mode, void* vals, void* rhs, bool iface,
                        bool reset = true, cudaStream_t st = nullptr, bool use_ctx_stream = true, int occ_cap = 0,
                        bool concurrent = false, int vpath = -1, SideStreams* ss = nullptr,
                        const int* tiles = nullptr, const int* splits = nullptr) {
  if (!ctx || !mesh) return fail(DG_ERR_ARG, "null context or mesh");
  if (prec < DG_PREC_FP64 || prec > DG_PREC_TF32X3) return fail(DG_ERR_ARG, "unknown precision %d", prec);
  if ((mode & (kModeVol | kModeFace)) && !vals) return fail(DG_ERR_ARG, "vals is null");
  if ((mode & kModeRhs) && !rhs) return fail(DG_ERR_ARG, "rhs is null");
  if (use_ctx_stream) st = ctx->stream;
  const DevMesh& m = mesh->dm;
  Tracer* tr = &ctx->tracer;
  if (reset) trace_reset(ctx, mesh);
  (void)iface;
  LaunchOpts lo;
  lo.occ_cap = occ_cap;
  lo.vol_moments = vpath >= 0 ? vpath >= 1 : ctx->vol_moments && !mesh->dm.lq_ok;
  lo.vol_exact = lo.vol_moments && (vpath >= 0 ? vpath == 2 : ctx->vol_exact);
  for (int p = 0; p < 9; ++p) {
    lo.pst[p] = st;
    lo.tile[p] = tiles ? tiles[p] : ctx->tiles[p];
  }
  if (!ss) ss = &ctx->streams;
  if (concurrent) {
    DG_CUDA_TRY(ss->ensure());
    DG_CUDA_TRY(cudaEventRecord(ss->fork, st));
    for (int i = 0; i < SideStreams::kN; ++i) DG_CUDA_TRY(cudaStreamWaitEvent(ss->side[i], ss->fork, 0));
    // highest degrees (longest launches) first, each part of a split group
    // on a stream of its own
    int k = 0;
    for (int p = 7; p >= 1; --p) {
      const int parts = splits ? std::max(1, std::min(kMaxSplit, splits[p])) : ctx->splits[p];
      lo.split[p] = parts;
      lo.pst[p] = ss->side[k % SideStreams::kN];
      for (int i = 0; i < parts; ++i) lo.part[p][i] = ss->side[(k + i) % SideStreams::kN];
      if (m.elem_pstart[p + 1] > m.elem_pstart[p]) k += parts;
    }
    lo.pst[8] = lo.pst[0] = ss->side[0];
  }
  const int n = dispatch_rows(m, prec, mode, vals, rhs, ctx->sm_count, lo, tr);
  if (concurrent) {
    for (int i = 0; i < SideStreams::kN; ++i) {
      DG_CUDA_TRY(cudaEventRecord(ss->join[i], ss->side[i]));
      DG_CUDA_TRY(cudaStreamWaitEvent(st, ss->join[i], 0));
    }
  }
  ctx->last_launches = reset ? n : ctx->last_launches + n;
  DG_CUDA_TRY(cudaGetLastError());
  return DG_OK;
}

int dg_assemble_volume(dg_ctx* ctx, const dg_mesh* mesh, int prec, void* vals) {
  NvtxRange nv_(ctx, "dg_assemble_volume");
  int rc = run_assembly(ctx, mesh, prec, kModeVol, vals, nullptr, false);
  if (rc == DG_OK) const_cast<dg_mesh*>(mesh)->vol_vals = vals;
  return rc;
}

int dg_assemble_faces(dg_ctx* ctx, const dg_mesh* mesh, int prec, void* vals) {
  NvtxRange nv_(ctx, "dg_assemble_faces");
  if (!mesh || mesh->vol_vals != vals || !vals)
    return fail(DG_ERR_ORDER, "dg_assemble_faces: call dg_assemble_volume on the same vals first");
  int rc = run_assembly(ctx, mesh, prec, kModeFace | kModeAccum, vals, nullptr, true);
  if (rc == DG_OK) const_cast<dg_mesh*>(mesh)->vol_vals = nullptr;
  return rc;
}

int dg_assemble_rhs(dg_ctx* ctx, const dg_mesh* mesh, int prec, void* rhs) {
  NvtxRange nv_(ctx, "dg_assemble_rhs");
  return run_assembly(ctx, mesh, prec, kModeRhs, nullptr, rhs, false);
}

int dg_assemble(dg_ctx* ctx, const dg_mesh* mesh, int prec, void* vals, void* rhs) {
  NvtxRange nv_(ctx, "dg_assemble");
  const int mode = kModeVol | kModeFace | (rhs ? kModeRhs : 0);
  return run_assembly(ctx, mesh, prec, mode, vals, rhs, true);
}

// The per-step launch shape: the autotuned one where dg_graph_create has
// tuned this precision on this mesh, else concurrent degree groups when the
// mesh has more than one.
static bool persist_ok(const dg_ctx* ctx, const dg_mesh* mesh, int prec, int vpath, int* mom_mask);

static void step_shape(const dg_ctx* ctx, const dg_mesh* mesh, int prec, int* occ, bool* conc, int* path,
                       const int** tiles, bool* persist = nullptr, const int** splits = nullptr) {
  *tiles = ctx->tiles;
  if (splits) *splits = ctx->splits;
  if (persist) *persist = false;
  if (mesh->shape_set[prec] && mesh->shape_vm[prec] == ctx_vol_path(ctx)) {
    *occ = mesh->shape_occ[prec];
    *conc = mesh->shape_conc[prec] != 0;
    *path = mesh->shape_path[prec];
    *tiles = mesh->shape_tile[prec];
    if (splits) *splits = mesh->shape_split[prec];
    if (persist) *persist = mesh->shape_persist[prec] != 0;
    return;
  }
  int groups = 0;
  for (int q = 1; q + 1 < 9; ++q) groups += mesh->dm.elem_pstart[q + 1] > mesh->dm.elem_pstart[q];
  for (int q = 1; q + 1 < 9; ++q) groups += ctx->splits[q] > 1 ? 1 : 0;
  *occ = 0;
  *conc = groups > 1;
  *path = -1;
  int mask = 0;
  if (persist && ctx->persist) *persist = persist_ok(ctx, mesh, prec, -1, &mask);
}

static int issue_persist_step(dg_ctx* ctx, dg_mesh* mesh, int prec, int mode, void* vals, void* rhs, int vpath);

int dg_assemble_host(dg_ctx* ctx, dg_mesh* mesh, int prec, const double* x, const double* y, const double* z,
                     const double* a, void* vals_host, void* rhs_host) {
  NvtxRange nv_(ctx, "dg_assemble_host");
  if (!ctx || !mesh || !vals_host) return fail(DG_ERR_ARG, "dg_assemble_host: null argument");
  const int gmask = pass_geometry(&prec);
  if (gmask < 0) return fail(DG_ERR_ARG, "unknown precision %d", prec);
  const size_t es = prec == DG_PREC_FP64 ? 8 : 4;
  if (mesh->h_prec != prec) {
    if (mesh->h_vals) cudaFree(mesh->h_vals);
    if (mesh->h_rhs) cudaFree(mesh->h_rhs);
    mesh->h_vals = mesh->h_rhs = nullptr;
    DG_CUDA_TRY(cudaMalloc(&mesh->h_vals, es * std::max<int64_t>(mesh->info.nvals, 1)));
    DG_CUDA_TRY(cudaMalloc(&mesh->h_rhs, es * std::max<int64_t>(mesh->info.ndofs, 1)));
    mesh->h_prec = prec;
  }
  const int nv = mesh->dm.nv, ne = mesh->dm.ne;
  const double* src[3] = {x, y, z};
  for (int q = 0; q < mesh->dm.dim; ++q)
    if (src[q]) DG_CUDA_TRY(cudaMemcpyAsync(mesh->X[q], src[q], sizeof(double) * nv, cudaMemcpyHostToDevice, ctx->stream));
  if (a) DG_CUDA_TRY(cudaMemcpyAsync(mesh->a, a, sizeof(double) * ne, cudaMemcpyHostToDevice, ctx->stream));
  // geometry records only in the precision this pass consumes
  trace_reset(ctx, mesh);
  ctx->last_launches = launch_geometry(mesh->dm, ctx->stream, &ctx->tracer, gmask);
  DG_CUDA_TRY(cudaGetLastError());
  int occ = 0, path = -1;
  bool conc = false;
  const int* tiles = nullptr;
  bool persist = false;
  const int* splits = nullptr;
  step_shape(ctx, mesh, prec, &occ, &conc, &path, &tiles, &persist, &splits);
  const int mode = kModeVol | kModeFace | (rhs_host ? kModeRhs : 0);
  int rc = persist ? issue_persist_step(ctx, mesh, prec, mode, mesh->h_vals, rhs_host ? mesh->h_rhs : nullptr, path)
                   : run_assembly(ctx, mesh, prec, mode, mesh->h_vals, rhs_host ? mesh->h_rhs : nullptr, true, false,
                                  nullptr, true, occ, conc, path, nullptr, tiles, splits);
  if (rc != DG_OK) return rc;
  // one copy each: several parts on parallel streams measured no faster
  DG_CUDA_TRY(cudaMemcpyAsync(vals_host, mesh->h_vals, es * mesh->info.nvals, cudaMemcpyDeviceToHost, ctx->stream));
  if (rhs_host)
    DG_CUDA_TRY(cudaMemcpyAsync(rhs_host, mesh->h_rhs, es * mesh->info.ndofs, cudaMemcpyDeviceToHost, ctx->stream));
  DG_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return DG_OK;
}

int dg_assemble_host_submit(dg_ctx* ctx, dg_mesh* mesh, int prec, const double* x, const double* y,
                            const double* z, const double* a, void* vals_host, void* rhs_host, long long* ticket) {
  NvtxRange nv_(ctx, "dg_assemble_host_submit");
  if (!ctx || !mesh || !vals_host || !ticket) return fail(DG_ERR_ARG, "dg_assemble_host_submit: null argument");
  const int gmask = pass_geometry(&prec);
  if (gmask < 0) return fail(DG_ERR_ARG, "unknown precision %d", prec);
  const size_t es = prec == DG_PREC_FP64 ? 8 : 4;
  if (!mesh->hp_copy) {
    DG_CUDA_TRY(cudaStreamCreateWithFlags(&mesh->hp_copy, cudaStreamNonBlocking));
    for (int i = 0; i < 2; ++i) {
      DG_CUDA_TRY(cudaEventCreateWithFlags(&mesh->hp_computed[i], cudaEventDisableTiming));
      DG_CUDA_TRY(cudaEventCreateWithFlags(&mesh->hp_done[i], cudaEventDisableTiming));
    }
  }
  if (mesh->hp_prec != prec) {
    // a change of precision: every submitted copy ends before the slots go
    DG_CUDA_TRY(cudaStreamSynchronize(mesh->hp_copy));
    DG_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    for (int i = 0; i < 2; ++i) {
      if (mesh->hp_vals[i]) cudaFree(mesh->hp_vals[i]);
      if (mesh->hp_rhs[i]) cudaFree(mesh->hp_rhs[i]);
      mesh->hp_vals[i] = mesh->hp_rhs[i] = nullptr;
    }
    mesh->hp_prec = -1;
    for (int i = 0; i < 2; ++i) {
      DG_CUDA_TRY(cudaMalloc(&mesh->hp_vals[i], es * std::max<int64_t>(mesh->info.nvals, 1)));
      DG_CUDA_TRY(cudaMalloc(&mesh->hp_rhs[i], es * std::max<int64_t>(mesh->info.ndofs, 1)));
    }
    mesh->hp_prec = prec;
  }
  const int slot = (int)(mesh->hp_next & 1);
  void* dv = mesh->hp_vals[slot];
  void* dr = rhs_host ? mesh->hp_rhs[slot] : nullptr;
  // the slot's previous copy back ends before this pass overwrites it (an
  // event never recorded is already complete)
  DG_CUDA_TRY(cudaStreamWaitEvent(ctx->stream, mesh->hp_done[slot], 0));
  const int nv = mesh->dm.nv, ne = mesh->dm.ne;
  const double* src[3] = {x, y, z};
  for (int q = 0; q < mesh->dm.dim; ++q)
    if (src[q]) DG_CUDA_TRY(cudaMemcpyAsync(mesh->X[q], src[q], sizeof(double) * nv, cudaMemcpyHostToDevice, ctx->stream));
  if (a) DG_CUDA_TRY(cudaMemcpyAsync(mesh->a, a, sizeof(double) * ne, cudaMemcpyHostToDevice, ctx->stream));
  trace_reset(ctx, mesh);
  ctx->last_launches = launch_geometry(mesh->dm, ctx->stream, &ctx->tracer, gmask);
  DG_CUDA_TRY(cudaGetLastError());
  int occ = 0, path = -1;
  bool conc = false;
  const int* tiles = nullptr;
  bool persist = false;
  const int* splits = nullptr;
  step_shape(ctx, mesh, prec, &occ, &conc, &path, &tiles, &persist, &splits);
  const int mode = kModeVol | kModeFace | (rhs_host ? kModeRhs : 0);
  int rc = persist ? issue_persist_step(ctx, mesh, prec, mode, dv, dr, path)
                   : run_assembly(ctx, mesh, prec, mode, dv, dr, true, false, nullptr, true, occ, conc, path, nullptr,
                                  tiles, splits);
  if (rc != DG_OK) return rc;
  // the copy back on the mesh's copy stream, after this pass: the next
  // submit's pass runs beside it
  DG_CUDA_TRY(cudaEventRecord(mesh->hp_computed[slot], ctx->stream));
  DG_CUDA_TRY(cudaStreamWaitEvent(mesh->hp_copy, mesh->hp_computed[slot], 0));
  DG_CUDA_TRY(cudaMemcpyAsync(vals_host, dv, es * mesh->info.nvals, cudaMemcpyDeviceToHost, mesh->hp_copy));
  if (rhs_host)
    DG_CUDA_TRY(cudaMemcpyAsync(rhs_host, dr, es * mesh->info.ndofs, cudaMemcpyDeviceToHost, mesh->hp_copy));
  DG_CUDA_TRY(cudaEventRecord(mesh->hp_done[slot], mesh->hp_copy));
  *ticket = mesh->hp_next++;
  return DG_OK;
}

int dg_assemble_host_wait(dg_ctx* ctx, dg_mesh* mesh, long long ticket) {
  NvtxRange nv_(ctx, "dg_assemble_host_wait");
  if (!ctx || !mesh) return fail(DG_ERR_ARG, "dg_assemble_host_wait: null argument");
  if (ticket < 0 || ticket >= mesh->hp_next)
    return fail(DG_ERR_ARG, "dg_assemble_host_wait: ticket %lld was not submitted on this mesh", ticket);
  // the slot's event holds this ticket's copy or a later one on the same copy
  // stream; either way this ticket's copy has ended once it completes
  DG_CUDA_TRY(cudaEventSynchronize(mesh->hp_done[ticket & 1]));
  return DG_OK;
}

int dg_assemble_step(dg_ctx* ctx, dg_mesh* mesh, int prec, void* vals, void* rhs) {
  NvtxRange nv_(ctx, "dg_assemble_step");
  if (!ctx || !mesh) return fail(DG_ERR_ARG, "dg_assemble_step: null argument");
  const int gmask = pass_geometry(&prec);
  if (gmask < 0) return fail(DG_ERR_ARG, "unknown precision %d", prec);
  // geometry records only in the precision this pass consumes
  trace_reset(ctx, mesh);
  ctx->last_launches = launch_geometry(mesh->dm, ctx->stream, &ctx->tracer, gmask);
  DG_CUDA_TRY(cudaGetLastError());
  int occ = 0, path = -1;
  bool conc = false;
  const int* tiles = nullptr;
  bool persist = false;
  const int* splits = nullptr;
  step_shape(ctx, mesh, prec, &occ, &conc, &path, &tiles, &persist, &splits);
  const int mode = kModeVol | kModeFace | (rhs ? kModeRhs : 0);
  if (persist) return issue_persist_step(ctx, mesh, prec, mode, vals, rhs, path);
  return run_assembly(ctx, mesh, prec, mode, vals, rhs, true, false, nullptr, true, occ, conc, path, nullptr, tiles,
                      splits);
}

// ---------------------------------------------------------------------------
// Space-time slabs (Sec. 2.3): prisms kappa x (t0, t1], the slab system
// expanded from the spatial blocks by the slab kernels (dg_slab.cu).
// ---------------------------------------------------------------------------

int dg_slab_offsets(int dim, int ne, const int* row_ptr, const int* col, const int* p, int space, int64_t* blk_off,
                    int64_t* dof_off) {
  if (dim != 2 && dim != 3) return fail(DG_ERR_ARG, "dg_slab_offsets: dim %d", dim);
  if (space != DG_SPACE_P && space != DG_SPACE_PQ) return fail(DG_ERR_ARG, "dg_slab_offsets: space %d", space);
  if (ne < 0) return fail(DG_ERR_ARG, "dg_slab_offsets: ne %d", ne);
  if (ne > 0 && (!p || (blk_off && (!row_ptr || !col)))) return fail(DG_ERR_ARG, "dg_slab_offsets: null array");
  const int pmax = dim == 2 ? kPMax2 : kPMax3;
  for (int e = 0; e < ne; ++e)
    if (p[e] < 1 || p[e] > pmax) return fail(DG_ERR_ARG, "dg_slab_offsets: element %d: p = %d outside 1..%d", e, p[e], pmax);
  if (dof_off) {
    dof_off[0] = 0;
    for (int e = 0; e < ne; ++e) dof_off[e + 1] = dof_off[e] + slab_count(dim, p[e], space);
  }
  if (blk_off) {
    blk_off[0] = 0;
    if (ne > 0 && row_ptr[0] != 0) return fail(DG_ERR_ARG, "dg_slab_offsets: row_ptr[0] must be 0");
    for (int r = 0; r < ne; ++r) {
      if (row_ptr[r + 1] < row_ptr[r]) return fail(DG_ERR_ARG, "dg_slab_offsets: row_ptr decreases at %d", r);
      const int64_t nr = slab_count(dim, p[r], space);
      for (int b = row_ptr[r]; b < row_ptr[r + 1]; ++b) {
        const int c = col[b];
        if (c < 0 || c >= ne) return fail(DG_ERR_ARG, "dg_slab_offsets: column %d out of range", c);
        blk_off[b + 1] = blk_off[b] + nr * slab_count(dim, p[c], space);
      }
    }
  }
  return DG_OK;
}

// Host offsets of the slab layout (computed once per space) and, with a
// context, their device copies and the spatial scratch.
static int slab_prepare(dg_ctx* ctx, dg_mesh* mesh, int space, const char* who) {
  if (!mesh->part_elem.empty()) return fail(DG_ERR_ARG, "%s: partition meshes are not supported", who);
  if (space != DG_SPACE_P && space != DG_SPACE_PQ) return fail(DG_ERR_ARG, "%s: space %d", who, space);
  const int ne = mesh->dm.ne;
  const size_t nnzb = mesh->col.size();
  if (mesh->slab_dof_h[space].empty()) {
    std::vector<int64_t> bo(nnzb + 1), dofs((size_t)ne + 1);
    const int rc = dg_slab_offsets(mesh->dm.dim, ne, mesh->row_ptr.data(), mesh->col.data(), mesh->p_h.data(), space,
                                   bo.data(), dofs.data());
    if (rc != DG_OK) return rc;
    mesh->slab_blk_h[space] = std::move(bo);
    mesh->slab_dof_h[space] = std::move(dofs);
  }
  if (!ctx) return DG_OK;
  if (!mesh->slab_blk[space]) {
    int64_t *bo = nullptr, *dofs = nullptr;
    DG_CUDA_TRY(mesh->bufs.alloc(&bo, nnzb + 1));
    DG_CUDA_TRY(mesh->bufs.alloc(&dofs, (size_t)ne + 1));
    DG_CUDA_TRY(cudaMemcpy(bo, mesh->slab_blk_h[space].data(), (nnzb + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
    DG_CUDA_TRY(cudaMemcpy(dofs, mesh->slab_dof_h[space].data(), ((size_t)ne + 1) * sizeof(int64_t),
                           cudaMemcpyHostToDevice));
    mesh->slab_blk[space] = bo;
    mesh->slab_dof[space] = dofs;
  }
  if (!mesh->slab_B) {
    double *B = nullptr, *M = nullptr, *l = nullptr, *a0 = nullptr;
    DG_CUDA_TRY(mesh->bufs.alloc(&B, (size_t)mesh->info.nvals));
    DG_CUDA_TRY(mesh->bufs.alloc(&M, (size_t)mesh->info.nvals));
    DG_CUDA_TRY(mesh->bufs.alloc(&l, (size_t)mesh->info.ndofs));
    DG_CUDA_TRY(mesh->bufs.alloc(&a0, (size_t)ne));
    DG_CUDA_TRY(cudaMemset(a0, 0, std::max<size_t>(ne, 1) * sizeof(double)));
    mesh->slab_B = B;
    mesh->slab_M = M;
    mesh->slab_l = l;
    mesh->slab_zero_a = a0;
  }
  return DG_OK;
}

static SlabPattern slab_pattern(const dg_mesh* mesh, int space) {
  const DevMesh& m = mesh->dm;
  SlabPattern sp;
  sp.dim = m.dim;
  sp.ne = m.ne;
  sp.space = space;
  sp.p = m.p;
  sp.row_ptr = m.row_ptr;
  sp.col = m.col;
  sp.diag_blk = m.diag_blk;
  sp.blk_off = m.blk_off;
  sp.dof_off = m.dof_off;
  sp.sblk_off = mesh->slab_blk[space];
  sp.sdof_off = mesh->slab_dof[space];
  sp.order = m.elem_perm;
  return sp;
}

int dg_slab_layout(const dg_mesh* mesh, int space, int64_t* nvals, int64_t* ndofs) {
  if (!mesh) return fail(DG_ERR_ARG, "dg_slab_layout: null mesh");
  dg_mesh* m = const_cast<dg_mesh*>(mesh);  // caches the host offsets
  const int rc = slab_prepare(nullptr, m, space, "dg_slab_layout");
  if (rc != DG_OK) return rc;
  if (nvals) *nvals = m->slab_blk_h[space].back();
  if (ndofs) *ndofs = m->slab_dof_h[space].back();
  return DG_OK;
}

static int slab_check(dg_ctx* ctx, dg_mesh* mesh, int prec, int space, double t0, double t1, void* vals,
                      const char* who) {
  if (!ctx || !mesh || !vals) return fail(DG_ERR_ARG, "%s: null argument", who);
  if (prec != DG_PREC_FP64 && prec != DG_PREC_FP32)
    return fail(DG_ERR_ARG, "%s: precision %d (DG_PREC_FP64 or DG_PREC_FP32)", who, prec);
  if (!std::isfinite(t0) || !std::isfinite(t1) || !(t1 > t0)) return fail(DG_ERR_ARG, "%s: the slab needs finite t0 < t1", who);
  return slab_prepare(ctx, mesh, space, who);
}

// One slab step on stream st: the spatial pass (B, l) and the mass pass (M),
// each with its degree groups on forked streams (ss), then the expansion and
// the load vector.  Everything allocated beforehand (slab_prepare), so the
// step can be captured.
static int issue_slab(dg_ctx* ctx, dg_mesh* mesh, int prec, int space, double t0, double t1, const void* u_prev,
                      void* vals, void* rhs, cudaStream_t st, SideStreams* ss) {
  int occ = 0, path = -1;
  bool conc = false;
  const int* tiles = nullptr;
  const int* splits = nullptr;
  step_shape(ctx, mesh, prec, &occ, &conc, &path, &tiles, nullptr, &splits);
  // B and l: the spatial pass
  int rc = run_assembly(ctx, mesh, prec, kModeVol | kModeFace | (rhs ? kModeRhs : 0), mesh->slab_B,
                        rhs ? mesh->slab_l : nullptr, true, true, st, false, occ, true, path, ss, tiles, splits);
  if (rc != DG_OK) return rc;
  int n = ctx->last_launches;
  // M: the volume pass of the same rules with a = 0, b = 0, c = 1
  DevMesh mm = mesh->dm;
  for (int d = 0; d < 3; ++d) mm.pb.b[d] = 0.0;
  mm.pb.c = 1.0;
  mm.pb.round_copies();
  mm.a = mesh->slab_zero_a;
  LaunchOpts lo;
  lo.vol_moments = path >= 0 ? path >= 1 : ctx->vol_moments && !mesh->dm.lq_ok;
  lo.vol_exact = lo.vol_moments && (path >= 0 ? path == 2 : ctx->vol_exact);
  DG_CUDA_TRY(ss->ensure());
  DG_CUDA_TRY(cudaEventRecord(ss->fork, st));
  for (int i = 0; i < 4; ++i) DG_CUDA_TRY(cudaStreamWaitEvent(ss->side[i], ss->fork, 0));
  for (int p = 0; p < 9; ++p) {
    lo.pst[p] = ss->side[(8 - p) % 4];
    lo.tile[p] = tiles ? tiles[p] : 0;
  }
  n += dispatch_rows(mm, prec, kModeVol, mesh->slab_M, nullptr, ctx->sm_count, lo, &ctx->tracer);
  for (int i = 0; i < 4; ++i) {
    DG_CUDA_TRY(cudaEventRecord(ss->join[i], ss->side[i]));
    DG_CUDA_TRY(cudaStreamWaitEvent(st, ss->join[i], 0));
  }
  DG_CUDA_TRY(cudaGetLastError());
  const SlabPattern sp = slab_pattern(mesh, space);
  const SlabTimes<double> tt = slab_time_data(t0, t1);
  const bool fp32 = prec == DG_PREC_FP32;
  // per-launch timing records (no algorithmic flop or byte counts: kind kNoCounts)
  Tracer* tr = &ctx->tracer;
  tr->begin(fp32 ? "slab_matrix_f32" : "slab_matrix_f64", kNoCounts, 0, fp32 ? 4 : 8, st);
  int pmax = 1;
  for (int q = 1; q <= 7; ++q)
    if (mesh->dm.elem_pstart[q + 1] > mesh->dm.elem_pstart[q]) pmax = q;
  n += launch_slab_matrix(sp, tt, fp32, mesh->slab_B, mesh->slab_M, vals, pmax, ctx->sm_count, st);
  tr->end(st);
  if (rhs) {
    tr->begin(fp32 ? "slab_rhs_f32" : "slab_rhs_f64", kNoCounts, 0, fp32 ? 4 : 8, st);
    n += launch_slab_rhs(sp, tt, fp32, mesh->slab_l, mesh->slab_M, u_prev, rhs, ctx->sm_count, st);
    tr->end(st);
  }
  DG_CUDA_TRY(cudaGetLastError());
  ctx->last_launches = n;
  return DG_OK;
}

int dg_assemble_slab(dg_ctx* ctx, dg_mesh* mesh, int prec, int space, double t0, double t1, const void* u_prev,
                     void* vals, void* rhs) {
  NvtxRange nv_(ctx, "dg_assemble_slab");
  int rc = slab_check(ctx, mesh, prec, space, t0, t1, vals, "dg_assemble_slab");
  if (rc != DG_OK) return rc;
  return issue_slab(ctx, mesh, prec, space, t0, t1, u_prev, vals, rhs, ctx->stream, &ctx->streams);
}

int dg_slab_graph_create(dg_ctx* ctx, dg_mesh* mesh, int prec, int space, double t0, double t1, const void* u_prev,
                         void* vals, void* rhs, dg_graph** out) {
  NvtxRange nv_(ctx, "dg_slab_graph_create");
  if (!out) return fail(DG_ERR_ARG, "dg_slab_graph_create: null output");
  *out = nullptr;
  int rc = slab_check(ctx, mesh, prec, space, t0, t1, vals, "dg_slab_graph_create");
  if (rc != DG_OK) return rc;
  dg_graph* g = new (std::nothrow) dg_graph();
  if (!g) return fail(DG_ERR_OOM, "out of host memory");
  if (cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking) != cudaSuccess || g->streams.ensure() != cudaSuccess) {
    delete g;
    return fail(DG_ERR_CUDA, "dg_slab_graph_create: stream creation failed");
  }
  trace_reset(ctx, mesh);
  if (cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    delete g;
    return fail(DG_ERR_CUDA, "dg_slab_graph_create: begin capture failed");
  }
  rc = issue_slab(ctx, mesh, prec, space, t0, t1, u_prev, vals, rhs, g->stream, &g->streams);
  cudaError_t ce = cudaStreamEndCapture(g->stream, &g->graph);
  g->ntrace = ctx->tracer.on ? ctx->tracer.n : 0;
  if (rc == DG_OK && ce != cudaSuccess) rc = fail(DG_ERR_CUDA, "dg_slab_graph_create: capture: %s", cudaGetErrorString(ce));
  if (rc == DG_OK && cudaGraphInstantiate(&g->exec, g->graph, 0) != cudaSuccess)
    rc = fail(DG_ERR_CUDA, "dg_slab_graph_create: instantiate failed");
  if (rc != DG_OK) {
    delete g;
    return rc;
  }
  g->launches = ctx->last_launches;
  *out = g;
  return DG_OK;
}

int dg_slab_trace(dg_ctx* ctx, const dg_mesh* mesh, int prec, int space, double t0, double t1, const void* U,
                  void* u_end) {
  if (!ctx || !mesh || !U || !u_end) return fail(DG_ERR_ARG, "dg_slab_trace: null argument");
  if (prec != DG_PREC_FP64 && prec != DG_PREC_FP32)
    return fail(DG_ERR_ARG, "dg_slab_trace: precision %d (DG_PREC_FP64 or DG_PREC_FP32)", prec);
  if (!std::isfinite(t0) || !std::isfinite(t1) || !(t1 > t0))
    return fail(DG_ERR_ARG, "dg_slab_trace: the slab needs finite t0 < t1");
  dg_mesh* m = const_cast<dg_mesh*>(mesh);  // caches the offsets and scratch
  const int rc = slab_prepare(ctx, m, space, "dg_slab_trace");
  if (rc != DG_OK) return rc;
  ctx->last_launches = launch_slab_trace(slab_pattern(m, space), slab_time_data(t0, t1), prec == DG_PREC_FP32, U, u_end,
                                         ctx->sm_count, ctx->stream);
  DG_CUDA_TRY(cudaGetLastError());
  return DG_OK;
}

// ---------------------------------------------------------------------------
// Variable advection and reaction (Sec. 4.2 fields, or an affine b and a
// cubic c from a table) at every point, added by the variable-coefficient
// kernels (dg_varcoef_kernel.cuh) to a row pass without b and c.
// ---------------------------------------------------------------------------

int dg_mesh_set_fields(dg_mesh* mesh, const dg_fields* f) {
  if (!mesh) return fail(DG_ERR_ARG, "dg_mesh_set_fields: null mesh");
  if (!f) {
    mesh->fields_set = false;
    return DG_OK;
  }
  VcFields v{};
  for (int d = 0; d < 3; ++d) {
    v.b0[d] = f->b0[d];
    for (int e = 0; e < 3; ++e) v.bx[d][e] = f->bx[d][e];
  }
  for (int k = 0; k < 20; ++k) v.c[k] = f->c[k];
  for (int k = 0; k < 3; ++k)
    if (!std::isfinite(v.b0[k]) || !std::isfinite(v.bx[k][0]) || !std::isfinite(v.bx[k][1]) || !std::isfinite(v.bx[k][2]))
      return fail(DG_ERR_ARG, "dg_mesh_set_fields: non-finite b coefficient");
  for (int k = 0; k < 20; ++k)
    if (!std::isfinite(v.c[k])) return fail(DG_ERR_ARG, "dg_mesh_set_fields: non-finite c coefficient");
  // the third coordinate does not exist in 2D
  if (mesh->dm.dim == 2) {
    v.b0[2] = 0.0;
    for (int e = 0; e < 3; ++e) v.bx[2][e] = v.bx[e][2] = 0.0;
    for (int k = 10; k < 20; ++k) v.c[k] = 0.0;
  }
  v.round_copies();
  mesh->fields = v;
  mesh->fields_set = true;
  return DG_OK;
}

int dg_assemble_varcoef_form(dg_ctx* ctx, dg_mesh* mesh, int prec, void* vals, void* rhs) {
  NvtxRange nv_(ctx, "dg_assemble_varcoef_form");
  if (!ctx || !mesh || !vals) return fail(DG_ERR_ARG, "dg_assemble_varcoef: null argument");
  if (prec != DG_PREC_FP64 && prec != DG_PREC_FP32)
    return fail(DG_ERR_ARG, "dg_assemble_varcoef: precision %d (DG_PREC_FP64 or DG_PREC_FP32)", prec);
  const DevMesh& m = mesh->dm;
  if (!mesh->part_elem.empty()) return fail(DG_ERR_ARG, "dg_assemble_varcoef: partition meshes are not supported");
  if (m.pb.b[0] != 0.0 || m.pb.b[1] != 0.0 || m.pb.b[2] != 0.0 || m.pb.c != 0.0)
    return fail(DG_ERR_ARG, "dg_assemble_varcoef: upload the mesh with b = 0 and c = 0 (the call supplies b(x), c(x))");
  if (m.lq_ok) return fail(DG_ERR_ARG, "dg_assemble_varcoef: learned volume rules are installed");
  // every term without b and c: the row kernels
  int rc = run_assembly(ctx, mesh, prec, kModeVol | kModeFace | (rhs ? kModeRhs : 0), vals, rhs, true);
  if (rc != DG_OK) return rc;
  int n = ctx->last_launches;
  const VcFields f = mesh->fields_set ? mesh->fields : vc_sec42_fields(m.dim);
  Tracer* tr = &ctx->tracer;
  const bool fp32 = prec == DG_PREC_FP32;
  tr->begin(fp32 ? "varcoef_terms_f32" : "varcoef_terms_f64", kNoCounts, 0, fp32 ? 4 : 8, ctx->stream);
  n += launch_varcoef(m, f, fp32, vals, rhs, ctx->sm_count, ctx->stream);
  tr->end(ctx->stream);
  DG_CUDA_TRY(cudaGetLastError());
  ctx->last_launches = n;
  return DG_OK;
}

int dg_assemble_varcoef(dg_ctx* ctx, dg_mesh* mesh, void* vals, void* rhs) {
  return dg_assemble_varcoef_form(ctx, mesh, DG_PREC_FP64, vals, rhs);
}

int dg_batch_upload(dg_ctx* ctx, const dg_mesh_desc* const* descs, int n, dg_mesh** out) {
  NvtxRange nv_(ctx, "dg_batch_upload");
  if (!ctx || !descs || n <= 0 || !out) return fail(DG_ERR_ARG, "dg_batch_upload: bad argument");
  *out = nullptr;
  const dg_mesh_desc* d0 = descs[0];
  if (!d0) return fail(DG_ERR_ARG, "dg_batch_upload: null descriptor 0");
  const int dim = d0->dim;
  int64_t nv = 0, ne = 0, nidx = 0;
  for (int k = 0; k < n; ++k) {
    const dg_mesh_desc* d = descs[k];
    if (!d || d->dim != dim) return fail(DG_ERR_ARG, "dg_batch_upload: descriptor %d null or of another dimension", k);
    if (d->c != d0->c || d->source != d0->source || d->c_sigma != d0->c_sigma || d->b[0] != d0->b[0] ||
        d->b[1] != d0->b[1] || d->b[2] != d0->b[2] || std::memcmp(d->poly, d0->poly, sizeof d->poly) != 0 ||
        d->neumann != d0->neumann)
      return fail(DG_ERR_ARG, "dg_batch_upload: descriptor %d has different problem data", k);
    if (d->nv <= 0 || d->ne <= 0 || !d->elem_ptr || !d->elem_idx || !d->x || !d->y || (dim == 3 && !d->z))
      return fail(DG_ERR_ARG, "dg_batch_upload: descriptor %d is empty", k);
    if (d->neumann != 0) {
      // the sides are those of each member's vertex box; the union keeps them
      // only where every member spans the same box
      double lo0[3], hi0[3], lo[3], hi[3];
      vertex_box(d0, lo0, hi0);
      vertex_box(d, lo, hi);
      for (int q = 0; q < dim; ++q)
        if (lo[q] != lo0[q] || hi[q] != hi0[q])
          return fail(DG_ERR_ARG, "dg_batch_upload: descriptor %d with Neumann sides spans another box than descriptor 0", k);
    }
    nv += d->nv;
    ne += d->ne;
    nidx += (int64_t)d->elem_ptr[d->ne] * (dim == 2 ? 1 : 4);
  }
  if (nv > INT32_MAX || ne > INT32_MAX || nidx > INT32_MAX) return fail(DG_ERR_ARG, "dg_batch_upload: batch too large");
  // disjoint union: vertex ids and element pointers shifted per mesh
  std::vector<double> X[3];
  std::vector<int> eptr(1, 0), eidx;
  std::vector<int8_t> p;
  std::vector<double> a;
  std::vector<int> elem_off(1, 0);
  for (int q = 0; q < dim; ++q) X[q].reserve(nv);
  eidx.reserve(nidx);
  int voff = 0;
  for (int k = 0; k < n; ++k) {
    const dg_mesh_desc* d = descs[k];
    const double* src[3] = {d->x, d->y, d->z};
    for (int q = 0; q < dim; ++q) {
      if (!src[q]) return fail(DG_ERR_ARG, "dg_batch_upload: descriptor %d lacks coordinates", k);
      X[q].insert(X[q].end(), src[q], src[q] + d->nv);
    }
    const int nk = d->elem_ptr[d->ne] * (dim == 2 ? 1 : 4);
    for (int i = 0; i < nk; ++i) {
      const int v = d->elem_idx[i];
      if (v < 0 || v >= d->nv) return fail(DG_ERR_MESH, "dg_batch_upload: mesh %d vertex index out of range", k);
      eidx.push_back(v + voff);
    }
    const int base = eptr.back();
    for (int e = 0; e < d->ne; ++e) eptr.push_back(base + d->elem_ptr[e + 1]);
    p.insert(p.end(), d->p, d->p + d->ne);
    a.insert(a.end(), d->a, d->a + d->ne);
    voff += d->nv;
    elem_off.push_back(elem_off.back() + d->ne);
  }
  dg_mesh_desc u = *d0;
  u.nv = (int)nv;
  u.x = X[0].data();
  u.y = X[1].data();
  u.z = dim == 3 ? X[2].data() : nullptr;
  u.ne = (int)ne;
  u.elem_ptr = eptr.data();
  u.elem_idx = eidx.data();
  u.p = p.data();
  u.a = a.data();
  int rc = dg_mesh_upload(ctx, &u, out);
  if (rc != DG_OK) return rc;
  (*out)->batch_elem_off = elem_off;
  return DG_OK;
}

// ---------------------------------------------------------------------------
// Partitions (Sec. 4.2: elements split across GPUs, cut faces computed by both
// owners, no communication during assembly).
// ---------------------------------------------------------------------------

}  // extern "C"

namespace {

// Hilbert index of (x, y) on an n x n grid, n a power of two: the classic
// quadrant rotate-and-reflect construction.
uint64_t hilbert2(uint32_t x, uint32_t y, uint32_t n) {
  uint64_t d = 0;
  for (uint32_t s = n / 2; s > 0; s /= 2) {
    const uint32_t rx = (x & s) ? 1u : 0u, ry = (y & s) ? 1u : 0u;
    d += (uint64_t)s * s * ((3u * rx) ^ ry);
    if (ry == 0) {
      if (rx == 1) {
        x = n - 1 - x;
        y = n - 1 - y;
      }
      std::swap(x, y);
    }
  }
  return d;
}

// Morton (Z-order) index of three 21-bit coordinates
uint64_t morton3(uint32_t x, uint32_t y, uint32_t z) {
  uint64_t d = 0;
  for (int b = 20; b >= 0; --b)
    d = (d << 3) | ((uint64_t)((x >> b) & 1u) << 2) | ((uint64_t)((y >> b) & 1u) << 1) | ((z >> b) & 1u);
  return d;
}

int check_desc_arrays(const dg_mesh_desc* d, const char* who) {
  if (!d) return fail(DG_ERR_ARG, "%s: null descriptor", who);
  if (d->dim != 2 && d->dim != 3) return fail(DG_ERR_ARG, "%s: dim must be 2 or 3", who);
  if (d->nv <= 0 || d->ne <= 0) return fail(DG_ERR_ARG, "%s: nv and ne must be positive", who);
  if (!d->x || !d->y || (d->dim == 3 && !d->z) || !d->elem_ptr || !d->elem_idx || !d->p || !d->a)
    return fail(DG_ERR_ARG, "%s: null array in descriptor", who);
  if (d->elem_ptr[0] != 0) return fail(DG_ERR_MESH, "%s: elem_ptr[0] must be 0", who);
  for (int e = 0; e < d->ne; ++e)
    if (d->elem_ptr[e + 1] <= d->elem_ptr[e]) return fail(DG_ERR_MESH, "%s: element %d is empty", who, e);
  const int64_t nidx = (int64_t)d->elem_ptr[d->ne] * (d->dim == 2 ? 1 : 4);
  for (int64_t i = 0; i < nidx; ++i)
    if (d->elem_idx[i] < 0 || d->elem_idx[i] >= d->nv) return fail(DG_ERR_MESH, "%s: vertex index out of range", who);
  return DG_OK;
}

// The local mesh of one part: its owned elements plus every element sharing
// a face with one of them (the halo), in increasing global element order;
// vertices renumbered in increasing global order.  Both orders are kept so
// that faces, interfaces and neighbour slots come out in the same relative
// order as in the whole mesh, which makes each owned block row bitwise equal
// to the whole mesh's.
struct PartMesh {
  dg_mesh_desc d{};
  std::vector<double> X[3];
  std::vector<int> eptr, eidx, elem_global, vert_global;
  std::vector<int8_t> p, owned;
  std::vector<double> a;
  int nowned = 0;
};

void half_face_keys(const dg_mesh_desc* d, int e, std::vector<std::array<int, 3>>& out) {
  const int b = d->elem_ptr[e], k = d->elem_ptr[e + 1] - b;
  if (d->dim == 2) {
    for (int i = 0; i < k; ++i) {
      const int v0 = d->elem_idx[b + i], v1 = d->elem_idx[b + (i + 1) % k];
      out.push_back({std::min(v0, v1), std::max(v0, v1), -1});
    }
  } else {
    for (int t = b; t < b + k; ++t) {
      const int* tv = d->elem_idx + 4 * t;
      for (int o = 0; o < 4; ++o) {
        std::array<int, 3> kk{};
        int c = 0;
        for (int i = 0; i < 4; ++i)
          if (i != o) kk[c++] = tv[i];
        std::sort(kk.begin(), kk.end());
        out.push_back(kk);
      }
    }
  }
}

int build_part(const dg_mesh_desc* d, const int* part, int my_part, PartMesh& L, const char* who) {
  int rc = check_desc_arrays(d, who);
  if (rc != DG_OK) return rc;
  if (!part) return fail(DG_ERR_ARG, "%s: null part array", who);
  const int ne = d->ne, dim = d->dim;
  std::vector<std::array<int, 3>> own_keys, keys;
  std::vector<int8_t> sel(ne, 0);  // 0 outside, 1 halo, 2 owned
  for (int e = 0; e < ne; ++e) {
    if (part[e] < 0) return fail(DG_ERR_ARG, "%s: part[%d] = %d is negative", who, e, part[e]);
    if (part[e] == my_part) {
      sel[e] = 2;
      half_face_keys(d, e, own_keys);
    }
  }
  if (own_keys.empty()) return fail(DG_ERR_ARG, "%s: part %d owns no element", who, my_part);
  std::sort(own_keys.begin(), own_keys.end());
  own_keys.erase(std::unique(own_keys.begin(), own_keys.end()), own_keys.end());
  for (int e = 0; e < ne; ++e) {
    if (sel[e]) continue;
    keys.clear();
    half_face_keys(d, e, keys);
    for (const auto& k : keys)
      if (std::binary_search(own_keys.begin(), own_keys.end(), k)) {
        sel[e] = 1;
        break;
      }
  }
  std::vector<int> vmap(d->nv, -1);
  for (int e = 0; e < ne; ++e) {
    if (!sel[e]) continue;
    const int64_t b = (int64_t)d->elem_ptr[e] * (dim == 2 ? 1 : 4), en = (int64_t)d->elem_ptr[e + 1] * (dim == 2 ? 1 : 4);
    for (int64_t i = b; i < en; ++i) vmap[d->elem_idx[i]] = 0;
  }
  const double* Xg[3] = {d->x, d->y, d->z};
  for (int v = 0; v < d->nv; ++v)
    if (vmap[v] == 0) {
      vmap[v] = (int)L.vert_global.size();
      L.vert_global.push_back(v);
      for (int q = 0; q < dim; ++q) L.X[q].push_back(Xg[q][v]);
    }
  L.eptr.assign(1, 0);
  for (int e = 0; e < ne; ++e) {
    if (!sel[e]) continue;
    const int64_t b = (int64_t)d->elem_ptr[e] * (dim == 2 ? 1 : 4), en = (int64_t)d->elem_ptr[e + 1] * (dim == 2 ? 1 : 4);
    for (int64_t i = b; i < en; ++i) L.eidx.push_back(vmap[d->elem_idx[i]]);
    L.eptr.push_back(L.eptr.back() + d->elem_ptr[e + 1] - d->elem_ptr[e]);
    L.elem_global.push_back(e);
    L.owned.push_back(sel[e] == 2 ? 1 : 0);
    L.nowned += sel[e] == 2;
    L.p.push_back(d->p[e]);
    L.a.push_back(d->a[e]);
  }
  L.d = *d;
  L.d.nv = (int)L.vert_global.size();
  L.d.x = L.X[0].data();
  L.d.y = L.X[1].data();
  L.d.z = dim == 3 ? L.X[2].data() : nullptr;
  L.d.ne = (int)L.elem_global.size();
  L.d.elem_ptr = L.eptr.data();
  L.d.elem_idx = L.eidx.data();
  L.d.p = L.p.data();
  L.d.a = L.a.data();
  return DG_OK;
}

}  // namespace

extern "C" {

int dg_partition(const dg_mesh_desc* d, int nparts, int* part) {
  int rc = check_desc_arrays(d, "dg_partition");
  if (rc != DG_OK) return rc;
  if (!part) return fail(DG_ERR_ARG, "dg_partition: null output");
  const int ne = d->ne, dim = d->dim;
  if (nparts < 1 || nparts > ne) return fail(DG_ERR_ARG, "dg_partition: nparts = %d outside 1..%d", nparts, ne);
  for (int e = 0; e < ne; ++e)
    if (d->p[e] < 1 || d->p[e] > (dim == 2 ? kPMax2 : kPMax3))
      return fail(DG_ERR_MESH, "dg_partition: element %d has degree %d", e, d->p[e]);
  const double* X[3] = {d->x, d->y, d->z};
  double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  for (int q = 0; q < dim; ++q) {
    lo[q] = *std::min_element(X[q], X[q] + d->nv);
    hi[q] = *std::max_element(X[q], X[q] + d->nv);
  }
  const uint32_t grid = dim == 2 ? (1u << 16) : (1u << 21);
  std::vector<uint64_t> key(ne);
  std::vector<double> w(ne);
  for (int e = 0; e < ne; ++e) {
    const int64_t b = (int64_t)d->elem_ptr[e] * (dim == 2 ? 1 : 4), en = (int64_t)d->elem_ptr[e + 1] * (dim == 2 ? 1 : 4);
    uint32_t c[3] = {0, 0, 0};
    for (int q = 0; q < dim; ++q) {
      double s = 0;
      for (int64_t i = b; i < en; ++i) s += X[q][d->elem_idx[i]];
      s /= (double)(en - b);
      const double t = hi[q] > lo[q] ? (s - lo[q]) / (hi[q] - lo[q]) : 0.0;
      c[q] = (uint32_t)std::min<double>(grid - 1, std::max(0.0, std::floor(t * grid)));
    }
    key[e] = dim == 2 ? hilbert2(c[0], c[1], grid) : morton3(c[0], c[1], c[2]);
    // cost ~ volume points x n^2 (the volume contraction)
    int qt = 1;
    for (int q = 0; q < dim; ++q) qt *= d->p[e] + 2;
    const double n = nbasis(dim, d->p[e]);
    w[e] = (double)(d->elem_ptr[e + 1] - d->elem_ptr[e]) * qt * n * n;
  }
  std::vector<int> order(ne);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return key[x] < key[y]; });
  double total = 0;
  for (int e : order) total += w[e];
  double before = 0;
  for (int e : order) {
    const int k = (int)std::floor((before + 0.5 * w[e]) * nparts / total);
    part[e] = std::min(nparts - 1, std::max(0, k));
    before += w[e];
  }
  return DG_OK;
}

int dg_part_check(const dg_mesh_desc* d, const int* part, int my_part, dg_bsr_info* info, int* nowned, int* row_ptr,
                  int* col, int64_t* blk_off, int* elem_global, int8_t* owned) {
  PartMesh L;
  int rc = build_part(d, part, my_part, L, "dg_part_check");
  if (rc != DG_OK) return rc;
  Plan P;
  rc = plan_mesh(&L.d, P, L.owned.data());
  if (rc != DG_OK) return rc;
  dg_bsr_info I{};
  fill_info(&L.d, P, I);
  if (info) *info = I;
  if (nowned) *nowned = L.nowned;
  if (row_ptr) std::copy(P.row_ptr.begin(), P.row_ptr.end(), row_ptr);
  if (col) std::copy(P.col.begin(), P.col.end(), col);
  if (blk_off) std::copy(P.blk_off.begin(), P.blk_off.end(), blk_off);
  if (elem_global) std::copy(L.elem_global.begin(), L.elem_global.end(), elem_global);
  if (owned) std::copy(L.owned.begin(), L.owned.end(), owned);
  return DG_OK;
}

int dg_mesh_upload_part(dg_ctx* ctx, const dg_mesh_desc* d, const int* part, int my_part, dg_mesh** out) {
  NvtxRange nv_(ctx, "dg_mesh_upload_part");
  if (!ctx || !out) return fail(DG_ERR_ARG, "dg_mesh_upload_part: null argument");
  *out = nullptr;
  PartMesh L;
  int rc = build_part(d, part, my_part, L, "dg_mesh_upload_part");
  if (rc != DG_OK) return rc;
  // the Neumann sides are those of the whole mesh's vertex box
  double box[6];
  vertex_box(d, box, box + 3);
  rc = upload_impl(ctx, &L.d, L.owned.data(), out, box);
  if (rc != DG_OK) return rc;
  (*out)->part_elem = L.elem_global;
  (*out)->part_vert = L.vert_global;
  return DG_OK;
}

int dg_part_map(const dg_mesh* mesh, int* nowned, int* nvlocal, int* elem_global, int8_t* owned, int* vert_global) {
  if (!mesh) return fail(DG_ERR_ARG, "dg_part_map: null mesh");
  if (mesh->part_elem.empty()) return fail(DG_ERR_ARG, "dg_part_map: not a partition mesh");
  if (nowned) *nowned = (int)std::count(mesh->owned_h.begin(), mesh->owned_h.end(), (int8_t)1);
  if (nvlocal) *nvlocal = (int)mesh->part_vert.size();
  if (elem_global) std::copy(mesh->part_elem.begin(), mesh->part_elem.end(), elem_global);
  if (owned) std::copy(mesh->owned_h.begin(), mesh->owned_h.end(), owned);
  if (vert_global) std::copy(mesh->part_vert.begin(), mesh->part_vert.end(), vert_global);
  return DG_OK;
}

int dg_batch_offsets(const dg_mesh* mesh, int* nmesh, int* elem_off, int64_t* val_off, int64_t* dof_off) {
  if (!mesh) return fail(DG_ERR_ARG, "dg_batch_offsets: null mesh");
  const std::vector<int>& eo = mesh->batch_elem_off;
  const int n = eo.empty() ? 1 : (int)eo.size() - 1;
  if (nmesh) *nmesh = n;
  for (int k = 0; k <= n; ++k) {
    const int e = eo.empty() ? (k == 0 ? 0 : mesh->dm.ne) : eo[k];
    if (elem_off) elem_off[k] = e;
    if (val_off) val_off[k] = mesh->blk_off[mesh->row_ptr[e]];
    if (dof_off) dof_off[k] = mesh->dof_off[e];
  }
  return DG_OK;
}

// ---------------------------------------------------------------------------
// The persistent pass (dg_persist.cuh): one launch over a work list of tiles.
// ---------------------------------------------------------------------------

// whether the persistent pass serves this mesh and precision; *mom_mask gets
// the degrees that take the moment path on volume path vpath
static bool persist_ok(const dg_ctx* ctx, const dg_mesh* mesh, int prec, int vpath, int* mom_mask) {
  if (prec != DG_PREC_FP32) return false;
  int ok_mask = 0, gm[9], gr[9];
  const int pserve = persist_layout(mesh->dm.dim, &ok_mask, gm, gr);
  int present = 0, pmax = 0;
  for (int p = 1; p <= 7; ++p)
    if (mesh->dm.elem_pstart[p + 1] > mesh->dm.elem_pstart[p]) {
      present |= 1 << p;
      pmax = p;
    }
  if (pmax > pserve || present == 0) return false;
  const bool moments = vpath >= 0 ? vpath >= 1 : ctx->vol_moments && !mesh->dm.lq_ok;
  *mom_mask = moments && mesh->dm.rt.lin32 ? ok_mask & present : 0;
  return true;
}

// The work list for mom_mask: every moment tile, then every row tile, each
// part by estimated work (points times n^2 over the tile's elements),
// largest first.  Built on the host and uploaded (synchronous); cached.
static const dg_mesh::PkList* persist_list(const dg_mesh* mesh, int key) {
  for (const auto& l : mesh->pk_lists)
    if (l.key == key) return &l;
  return nullptr;
}

static int persist_items(dg_ctx* ctx, dg_mesh* mesh, int mom_mask) {
  const int key = mom_mask;
  if (persist_list(mesh, key)) return DG_OK;
  int ok_mask = 0, gm[9], gr[9];
  persist_layout(mesh->dm.dim, &ok_mask, gm, gr);
  const int dim = mesh->dm.dim, ne = mesh->dm.ne;
  struct Item {
    double cost;
    int kind, p, tile;
  };
  std::vector<Item> mom, row;
  const bool lrn = mesh->dm.lq_ok != nullptr;
  std::vector<int> okh;
  if (lrn) {
    okh.resize(ne);
    DG_CUDA_TRY(cudaMemcpy(okh.data(), mesh->dm.lq_ok, sizeof(int) * ne, cudaMemcpyDeviceToHost));
  }
  for (int p = 1; p <= 7; ++p) {
    const int b = mesh->dm.elem_pstart[p], cnt = mesh->dm.elem_pstart[p + 1] - b;
    if (cnt <= 0) continue;
    const double n2 = (double)nbasis(dim, p) * nbasis(dim, p);
    const bool mp = (mom_mask >> p) & 1;
    auto cost_of = [&](int lo, int hi, int kind) {
      double c = 0.0;
      for (int i = lo; i < hi && i < cnt; ++i) {
        const int e = mesh->perm_h[b + i];
        const double nvq = lrn && okh[e] ? 28.0 : (double)mesh->nvq_h[e];
        c += kind == 1 ? nvq * n2 / 8.0 : ((mp ? 0.0 : nvq) + mesh->nqf_h[e]) * n2;
      }
      return c;
    };
    if (mp)
      for (int t = 0; t * gm[p] < cnt; ++t) mom.push_back({cost_of(t * gm[p], (t + 1) * gm[p], 1), 1, p, t});
    for (int t = 0; t * gr[p] < cnt; ++t) row.push_back({cost_of(t * gr[p], (t + 1) * gr[p], 0), 0, p, t});
  }
  auto by_cost = [](const Item& x, const Item& y) {
    if (x.cost != y.cost) return x.cost > y.cost;
    if (x.p != y.p) return x.p > y.p;
    return x.tile < y.tile;
  };
  std::sort(mom.begin(), mom.end(), by_cost);
  std::sort(row.begin(), row.end(), by_cost);
  std::vector<int4> items;
  items.reserve(mom.size() + row.size());
  for (const auto& it : mom) items.push_back(make_int4(it.kind, it.p, it.tile, 0));
  for (const auto& it : row) items.push_back(make_int4(it.kind, it.p, it.tile, 0));
  if (!mesh->pk_sync && cudaMalloc(&mesh->pk_sync, sizeof(int) * (2 + (size_t)ne)) != cudaSuccess)
    return fail(DG_ERR_OOM, "persistent pass: flags");
  int4* dev = nullptr;
  if (cudaMalloc(&dev, sizeof(int4) * std::max<size_t>(items.size(), 1)) != cudaSuccess)
    return fail(DG_ERR_OOM, "persistent pass: work list");
  if (cudaMemcpy(dev, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(dev);
    return fail(DG_ERR_CUDA, "persistent pass: work list upload");
  }
  mesh->pk_lists.push_back({key, dev, (int)items.size()});
  (void)ctx;
  return DG_OK;
}

// Issue the persistent pass's row work on st (the work list must exist:
// persist_items before any capture).
static int issue_persist_rows(dg_ctx* ctx, dg_mesh* mesh, int prec, int mode, void* vals, void* rhs, cudaStream_t st,
                              int vpath) {
  int mom_mask = 0;
  if (!persist_ok(ctx, mesh, prec, vpath, &mom_mask)) return fail(DG_ERR_ARG, "the persistent pass does not serve this mesh");
  const dg_mesh::PkList* list = persist_list(mesh, mom_mask);
  if (!list) return fail(DG_ERR_ARG, "persistent pass: work list not built");
  const int ne = mesh->dm.ne;
  DG_CUDA_TRY(cudaMemsetAsync(mesh->pk_sync, 0, sizeof(int) * (2 + (size_t)ne), st));
  PersistArgs a{};
  a.items = list->items;
  a.nitems = list->n;
  a.queue = mesh->pk_sync;
  a.vdone = mesh->pk_sync + 2;
  a.status = ctx->status_dev;
  a.limit_ns = ctx->wait_ns;
  a.mode = mode;
  a.mom_mask = mom_mask;
  const bool exact = vpath >= 0 ? vpath == 2 : ctx->vol_exact;
  a.exact = exact ? kModeExactMom : 0;
  int pmax = 0;
  for (int p = 1; p <= 7; ++p)
    if (mesh->dm.elem_pstart[p + 1] > mesh->dm.elem_pstart[p]) pmax = p;
  float* v = static_cast<float*>(vals);
  float* r = static_cast<float*>(rhs);
  Tracer* tr = &ctx->tracer;
  if (tr->on) {
    // the whole pass's algorithmic work; executed: the moment form where taken
    double fl = 0.0, xfl = 0.0, by = 0.0;
    for (int p = 1; p <= 8; ++p) {
      fl += mesh->flops[0][p];
      by += mesh->words[0][p] * sizeof(float);
      xfl += ((mom_mask >> p) & 1) ? mesh->mom_exec[0][p] + mesh->flops[1][p] : mesh->flops[0][p];
    }
    tr->begin_counts(mesh->dm.dim == 2 ? "row_persist2d_f32" : "row_persist3d_f32", fl, xfl, by, st);
  }
  const int n = mesh->dm.dim == 2 ? launch_persist2d_f32(mesh->dm, v, r, a, pmax, ctx->sm_count, st)
                                  : launch_persist3d_f32(mesh->dm, v, r, a, pmax, ctx->sm_count, st);
  if (tr->on) tr->end(st);
  if (n < 0) return fail(DG_ERR_ARG, "persistent pass: shared memory does not fit");
  DG_CUDA_TRY(cudaGetLastError());
  return DG_OK;
}

// The persistent pass's row work on the context stream (the per-step entry
// points), the work list built first if needed.
static int issue_persist_step(dg_ctx* ctx, dg_mesh* mesh, int prec, int mode, void* vals, void* rhs, int vpath) {
  int mask = 0;
  if (!persist_ok(ctx, mesh, prec, vpath, &mask)) return fail(DG_ERR_ARG, "the persistent pass does not serve this mesh");
  int rc = persist_items(ctx, mesh, mask);
  if (rc != DG_OK) return rc;
  rc = issue_persist_rows(ctx, mesh, prec, mode, vals, rhs, ctx->stream, vpath);
  if (rc == DG_OK) ctx->last_launches += 1;
  return rc;
}

// One whole pass (geometry + row kernels) on stream st with a launch shape.
static int issue_pass(dg_ctx* ctx, dg_mesh* mesh, int prec, int gmask, void* vals, void* rhs, cudaStream_t st,
                      int occ_cap, bool concurrent, int vpath, SideStreams* ss, const int* tiles, bool persist = false,
                      const int* splits = nullptr) {
  int n = launch_geometry(mesh->dm, st, nullptr, gmask);
  DG_CUDA_TRY(cudaGetLastError());
  const int mode = kModeVol | kModeFace | (rhs ? kModeRhs : 0);
  if (persist) {
    trace_reset(ctx, mesh);
    int rc = issue_persist_rows(ctx, mesh, prec, mode, vals, rhs, st, vpath);
    if (rc != DG_OK) return rc;
    ctx->last_launches = n + 1;
    return DG_OK;
  }
  int rc = run_assembly(ctx, mesh, prec, mode, vals, rhs, true, true, st, false, occ_cap, concurrent, vpath, ss, tiles,
                        splits);
  if (rc != DG_OK) return rc;
  ctx->last_launches += n;
  return DG_OK;
}

int dg_graph_create(dg_ctx* ctx, dg_mesh* mesh, int prec, void* vals, void* rhs, int autotune, dg_graph** out) {
  NvtxRange nv_(ctx, "dg_graph_create");
  if (!ctx || !mesh || !vals || !out) return fail(DG_ERR_ARG, "dg_graph_create: null argument");
  const int gmask = pass_geometry(&prec);
  if (gmask < 0) return fail(DG_ERR_ARG, "unknown precision %d", prec);
  *out = nullptr;
  dg_graph* g = new (std::nothrow) dg_graph();
  if (!g) return fail(DG_ERR_OOM, "out of host memory");
  auto bail = [&](int rc) {
    delete g;
    return rc;
  };
  if (cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking) != cudaSuccess || g->streams.ensure() != cudaSuccess)
    return bail(fail(DG_ERR_CUDA, "dg_graph_create: stream creation failed"));
  const bool was_on = ctx->tracer.on;
  ctx->tracer.on = false;
  // autotuner: time each candidate launch shape (best of 3 after a warm-up):
  // residency cap x serial / concurrent degree groups x volume path (the
  // moment path only where the context allows it and the form has it)
  const int mpath = ctx->vol_exact ? 2 : 1;  // the context's moment path
  const int def_path = ctx->vol_moments && !mesh->dm.lq_ok ? mpath : 0;
  int best_occ = 0, best_conc = 0, best_path = def_path;
  int best_tiles[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  int best_persist = 0;
  int best_split[9] = {1, 1, 1, 1, 1, 1, 1, 1, 1};
  float best = 1e30f;
  if (autotune) {
    const int occs[3] = {0, 1, 2};
    const int npath = ctx->vol_moments && (prec == DG_PREC_FP32 || prec == DG_PREC_FP64) ? 2 : 1;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // L2 is flushed (a 256 MiB write, outside the timed span) before every
    // timed pass: a recorded pass is replayed with its inputs out of cache
    // (the solver runs between assemblies), and a shape that wins with the
    // previous pass's data still in L2 can lose without it.  Without room for
    // the buffer the passes are timed back to back.
    constexpr size_t kFlushBytes = size_t(256) << 20;
    void* flush = nullptr;
    if (cudaMalloc(&flush, kFlushBytes) != cudaSuccess) {
      flush = nullptr;
      cudaGetLastError();
    }
    // one candidate: best of 3 timed passes after a warm-up pass
    auto time_shape = [&](int occ, int conc, int vpath, const int* tiles, float* out, bool persist = false,
                          const int* splits = nullptr) -> int {
      float t = 1e30f;
      for (int rep = 0; rep < 4; ++rep) {
        if (flush) cudaMemsetAsync(flush, rep & 0xff, kFlushBytes, g->stream);
        cudaEventRecord(e0, g->stream);
        int rc = issue_pass(ctx, mesh, prec, gmask, vals, rhs, g->stream, occ, conc != 0, vpath, &g->streams, tiles,
                            persist, splits ? splits : best_split);
        if (rc != DG_OK) return rc;
        cudaEventRecord(e1, g->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) return fail(DG_ERR_CUDA, "dg_graph_create: tuning pass failed");
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < t) t = ms;
      }
      ++g->trials;
      *out = t;
      return DG_OK;
    };
    int rc = DG_OK;
    // launch shape: residency cap x serial / concurrent degree groups x volume path
    for (int pi = 0; rc == DG_OK && pi < npath; ++pi)
      for (int conc = 0; rc == DG_OK && conc < 2; ++conc)
        for (int oi = 0; rc == DG_OK && oi < 3; ++oi) {
          const int vpath = npath == 2 ? (pi == 0 ? mpath : 0) : 0;
          float t = 0.f;
          rc = time_shape(occs[oi], conc, vpath, best_tiles, &t);
          if (rc == DG_OK && t < best) {
            best = t;
            best_occ = occs[oi];
            best_conc = conc;
            best_path = vpath;
          }
        }
    // tiles: for each degree present, each other register-tile variant of
    // its row kernel against the best so far (one pass of coordinate descent)
    for (int p = 1; rc == DG_OK && p <= 7; ++p) {
      if (mesh->dm.elem_pstart[p + 1] <= mesh->dm.elem_pstart[p]) continue;
      for (int v = 1; rc == DG_OK && v < 3 && row_tile_tm(mesh->dm.dim, p, prec, v) > 0; ++v) {
        int cand[9];
        std::copy(best_tiles, best_tiles + 9, cand);
        cand[p] = v;
        float t = 0.f;
        rc = time_shape(best_occ, best_conc, best_path, cand, &t);
        if (rc == DG_OK && t < best) {
          best = t;
          best_tiles[p] = v;
        }
      }
    }
    // degree groups in parts (concurrent shape): for each degree present,
    // from the highest, 2..kMaxSplit parts against the best so far, so that
    // the long moment-then-rows chains of the big groups run side by side
    for (int p = 7; rc == DG_OK && p >= 1; --p) {
      if (mesh->dm.elem_pstart[p + 1] <= mesh->dm.elem_pstart[p]) continue;
      for (int s = 2; rc == DG_OK && s <= kMaxSplit; ++s) {
        int cand[9];
        std::copy(best_split, best_split + 9, cand);
        cand[p] = s;
        float t = 0.f;
        rc = time_shape(best_occ, 1, best_path, best_tiles, &t, false, cand);
        if (rc == DG_OK && t < best) {
          best = t;
          best_conc = 1;
          best_split[p] = s;
        }
      }
    }
    // the persistent pass (its own tiles), on each volume path tried above
    for (int pi = 0; rc == DG_OK && pi < npath; ++pi) {
      const int vpath = npath == 2 ? (pi == 0 ? mpath : 0) : def_path;
      int mask = 0;
      if (!persist_ok(ctx, mesh, prec, vpath, &mask)) continue;
      rc = persist_items(ctx, mesh, mask);
      float t = 0.f;
      if (rc == DG_OK) rc = time_shape(0, 0, vpath, best_tiles, &t, true);
      if (rc == DG_OK && t < best) {
        best = t;
        best_path = vpath;
        best_persist = 1;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (flush) cudaFree(flush);
    if (rc != DG_OK) {
      ctx->tracer.on = was_on;
      return bail(rc);
    }
  }
  if (!autotune && ctx->persist) {
    int mask = 0;
    if (persist_ok(ctx, mesh, prec, best_path, &mask)) best_persist = 1;
  }
  if (best_persist) {
    // the work list of the recorded path, built before the capture
    int mask = 0;
    persist_ok(ctx, mesh, prec, best_path, &mask);
    const int rc = persist_items(ctx, mesh, mask);
    if (rc != DG_OK) {
      ctx->tracer.on = was_on;
      return bail(rc);
    }
  }
  g->occ_cap = best_occ;
  g->concurrent = best_conc;
  g->vol_path = best_path;
  g->persist = best_persist;
  g->tuned_ms = autotune ? best : 0.f;
  for (int p = 0; p < 9; ++p) {
    g->tiles[p] = best_tiles[p];
    g->split[p] = autotune ? (best_conc ? best_split[p] : 1) : ctx->splits[p];
    const bool present = p >= 1 && p <= 7 && mesh->dm.elem_pstart[p + 1] > mesh->dm.elem_pstart[p];
    g->tile_tm[p] = present ? row_tile_tm(mesh->dm.dim, p, prec, best_persist ? 3 : best_tiles[p]) : 0;
  }
  if (autotune) {
    mesh->shape_set[prec] = 1;
    mesh->shape_occ[prec] = best_occ;
    mesh->shape_conc[prec] = best_conc;
    mesh->shape_path[prec] = best_path;
    mesh->shape_vm[prec] = ctx_vol_path(ctx);
    std::copy(best_tiles, best_tiles + 9, mesh->shape_tile[prec]);
    std::copy(g->split, g->split + 9, mesh->shape_split[prec]);
    mesh->shape_persist[prec] = best_persist;
  }
  // with timing enabled the per-launch events are recorded into the graph
  ctx->tracer.on = was_on;
  trace_reset(ctx, mesh);
  if (cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeRelaxed) != cudaSuccess)
    return bail(fail(DG_ERR_CUDA, "dg_graph_create: begin capture failed"));
  int rc = DG_OK;
  {
    const int gl = launch_geometry(mesh->dm, g->stream, &ctx->tracer, gmask);
    const int mode = kModeVol | kModeFace | (rhs ? kModeRhs : 0);
    if (g->persist) {
      rc = issue_persist_rows(ctx, mesh, prec, mode, vals, rhs, g->stream, g->vol_path);
      ctx->last_launches = 1;
    } else {
      rc = run_assembly(ctx, mesh, prec, mode, vals, rhs, true, false, g->stream, false, g->occ_cap,
                        g->concurrent != 0, g->vol_path, &g->streams, g->tiles, g->split);
    }
    ctx->last_launches += gl;
  }
  cudaError_t ce = cudaStreamEndCapture(g->stream, &g->graph);
  g->ntrace = ctx->tracer.on ? ctx->tracer.n : 0;
  if (rc != DG_OK) return bail(rc);
  if (ce != cudaSuccess) return bail(fail(DG_ERR_CUDA, "dg_graph_create: capture failed: %s", cudaGetErrorString(ce)));
  ce = cudaGraphInstantiate(&g->exec, g->graph, 0);
  if (ce != cudaSuccess) return bail(fail(DG_ERR_CUDA, "dg_graph_create: instantiate: %s", cudaGetErrorString(ce)));
  g->launches = ctx->last_launches;
  *out = g;
  return DG_OK;
}

// Many independent meshes in one call: each member's whole pass (geometry
// in the pass's precision, then its row kernels in its own tuned launch
// shape) on one of the context's forked side streams, round robin, joined
// back into the context stream.  use_graph records the lot as one CUDA
// graph, launches it and frees it.
int dg_assemble_batch(dg_ctx* ctx, dg_mesh* const* meshes, int nmesh, int prec, void* const* vals,
                      void* const* rhs, int use_graph) {
  NvtxRange nv_(ctx, "dg_assemble_batch");
  if (!ctx || !meshes || !vals || nmesh <= 0) return fail(DG_ERR_ARG, "dg_assemble_batch: bad argument");
  int base = prec;
  const int gmask = pass_geometry(&base);
  if (gmask < 0) return fail(DG_ERR_ARG, "unknown precision %d", prec);
  for (int k = 0; k < nmesh; ++k)
    if (!meshes[k] || !vals[k]) return fail(DG_ERR_ARG, "dg_assemble_batch: member %d has a null mesh or vals", k);
  SideStreams& ss = ctx->streams;
  DG_CUDA_TRY(ss.ensure());
  cudaStream_t st = ctx->stream;
  cudaStream_t cap = nullptr;
  if (use_graph) {
    DG_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
      cudaStreamDestroy(cap);
      return fail(DG_ERR_CUDA, "dg_assemble_batch: begin capture failed");
    }
    st = cap;
  }
  int rc = DG_OK, launches = 0;
  if (cudaEventRecord(ss.fork, st) != cudaSuccess) rc = fail(DG_ERR_CUDA, "dg_assemble_batch: fork failed");
  for (int i = 0; rc == DG_OK && i < 4; ++i)
    if (cudaStreamWaitEvent(ss.side[i], ss.fork, 0) != cudaSuccess) rc = fail(DG_ERR_CUDA, "dg_assemble_batch: fork failed");
  for (int k = 0; rc == DG_OK && k < nmesh; ++k) {
    dg_mesh* mesh = meshes[k];
    cudaStream_t br = ss.side[k % 4];
    launches += launch_geometry(mesh->dm, br, nullptr, gmask);
    int occ = 0, path = -1;
    bool conc = false;
    const int* tiles = nullptr;
    step_shape(ctx, mesh, base, &occ, &conc, &path, &tiles);
    const int mode = kModeVol | kModeFace | (rhs && rhs[k] ? kModeRhs : 0);
    // a member's degree groups stay on its branch stream (serial): the
    // members themselves are the concurrency
    rc = run_assembly(ctx, mesh, base, mode, vals[k], rhs ? rhs[k] : nullptr, true, true, br, false, occ, false, path,
                      nullptr, tiles);
    launches += ctx->last_launches;
  }
  for (int i = 0; rc == DG_OK && i < 4; ++i) {
    if (cudaEventRecord(ss.join[i], ss.side[i]) != cudaSuccess || cudaStreamWaitEvent(st, ss.join[i], 0) != cudaSuccess)
      rc = fail(DG_ERR_CUDA, "dg_assemble_batch: join failed");
  }
  if (use_graph) {
    cudaGraph_t graph = nullptr;
    cudaError_t ce = cudaStreamEndCapture(cap, &graph);
    cudaGraphExec_t exec = nullptr;
    if (rc == DG_OK && ce != cudaSuccess) rc = fail(DG_ERR_CUDA, "dg_assemble_batch: capture failed: %s", cudaGetErrorString(ce));
    if (rc == DG_OK && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess)
      rc = fail(DG_ERR_CUDA, "dg_assemble_batch: instantiate failed");
    if (rc == DG_OK && cudaGraphLaunch(exec, ctx->stream) != cudaSuccess) rc = fail(DG_ERR_CUDA, "dg_assemble_batch: launch failed");
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cap);
  }
  if (rc != DG_OK) return rc;
  ctx->last_launches = launches;
  DG_CUDA_TRY(cudaGetLastError());
  return DG_OK;
}

int dg_graph_launch(dg_ctx* ctx, dg_graph* g) {
  NvtxRange nv_(ctx, "dg_graph_launch");
  if (!ctx || !g) return fail(DG_ERR_ARG, "dg_graph_launch: null argument");
  DG_CUDA_TRY(cudaGraphLaunch(g->exec, ctx->stream));
  ctx->last_launches = g->launches;
  ctx->tracer.n = g->ntrace;  // the graph's own timing events, if any
  return DG_OK;
}

int dg_graph_info(const dg_graph* g, int* occ_cap, int* concurrent, float* tuned_ms, int* launches, int* vol_path) {
  if (!g) return fail(DG_ERR_ARG, "dg_graph_info: null graph");
  if (vol_path) *vol_path = g->vol_path;
  if (occ_cap) *occ_cap = g->occ_cap;
  if (concurrent) *concurrent = g->concurrent;
  if (tuned_ms) *tuned_ms = g->tuned_ms;
  if (launches) *launches = g->launches;
  return DG_OK;
}

int dg_graph_tiles(const dg_graph* g, int* tile_tm, int* trials, int* persistent) {
  if (!g) return fail(DG_ERR_ARG, "dg_graph_tiles: null graph");
  if (tile_tm) std::copy(g->tile_tm, g->tile_tm + 9, tile_tm);
  if (trials) *trials = g->trials;
  if (persistent) *persistent = g->persist;
  return DG_OK;
}

int dg_graph_splits(const dg_graph* g, int* split) {
  if (!g || !split) return fail(DG_ERR_ARG, "dg_graph_splits: null argument");
  for (int p = 0; p < 9; ++p) split[p] = g->concurrent && !g->persist ? g->split[p] : 1;
  return DG_OK;
}

int dg_graph_free(dg_graph* g) {
  delete g;
  return DG_OK;
}

// ---------------------------------------------------------------------------
// learned quadrature
// ---------------------------------------------------------------------------

int dg_quad_prepare(dg_ctx* ctx, dg_mesh* mesh) {
  NvtxRange nv_(ctx, "dg_quad_prepare");
  if (!ctx || !mesh) return fail(DG_ERR_ARG, "dg_quad_prepare: null argument");
  if (mesh->dm.dim != 2) return fail(DG_ERR_ARG, "dg_quad_prepare: learned rules are 2D only");
  const int ne = mesh->dm.ne;
  if (!mesh->lq_mom) {
    struct {
      void** p;
      size_t bytes;
    } a[] = {{(void**)&mesh->lq_mom, 28 * 8}, {(void**)&mesh->lq_mmom, 28 * 8}, {(void**)&mesh->lq_rule, 84 * 8},
             {(void**)&mesh->lq64, 84 * 8},   {(void**)&mesh->lq32, 84 * 4},   {(void**)&mesh->lq_resid, 4},
             {(void**)&mesh->lq_elig, 4},     {(void**)&mesh->lq_ok, 4},       {(void**)&mesh->lq_okm, 4},
             {(void**)&mesh->lq_feat, 24 * 2}};
    for (auto& x : a)
      if (cudaMalloc(x.p, x.bytes * (size_t)ne) != cudaSuccess) return fail(DG_ERR_OOM, "dg_quad_prepare: buffers");
    DG_CUDA_TRY(cudaMemsetAsync(mesh->lq_okm, 0, sizeof(int) * ne, ctx->stream));
  }
  // the fit reads the FP64 element records, which the reduced-precision
  // geometry of an FP32 step leaves untouched: bring them up to date
  launch_geometry(mesh->dm, ctx->stream, nullptr, 1);
  lq_prepare(mesh->dm, mesh->lq_mom, mesh->lq_mmom, mesh->lq_feat, mesh->lq_elig, ctx->stream);
  DG_CUDA_TRY(cudaGetLastError());
  return DG_OK;
}

int dg_quad_buffers(const dg_mesh* mesh, const void** feat, const double** rules, const float** resid,
                    const int** ok, const double** moments) {
  if (!mesh || !mesh->lq_mom) return fail(DG_ERR_ARG, "dg_quad_buffers: call dg_quad_prepare first");
  if (feat) *feat = mesh->lq_feat;
  if (rules) *rules = mesh->lq_rule;
  if (resid) *resid = mesh->lq_resid;
  if (ok) *ok = mesh->lq_ok;
  if (moments) *moments = mesh->lq_mom;
  return DG_OK;
}

// rebuild the degree-grouped, cost-descending work list for the current rules
static int rebuild_worklist(dg_ctx* ctx, dg_mesh* mesh, const std::vector<int>& learned) {
  const int ne = mesh->dm.ne;
  std::vector<int64_t> cost(ne);
  for (int e = 0; e < ne; ++e) cost[e] = (learned.empty() || !learned[e] ? mesh->nvq_h[e] : 28) + mesh->nqf_h[e];
  std::vector<int> perm;
  for (int e = 0; e < ne; ++e)
    if (mesh->owned_h.empty() || mesh->owned_h[e]) perm.push_back(e);
  std::stable_sort(perm.begin(), perm.end(), [&](int x, int y) {
    if (mesh->p_h[x] != mesh->p_h[y]) return mesh->p_h[x] < mesh->p_h[y];
    return cost[x] > cost[y];
  });
  DG_CUDA_TRY(cudaMemcpyAsync(mesh->perm_dev, perm.data(), sizeof(int) * perm.size(), cudaMemcpyHostToDevice,
                              ctx->stream));
  mesh->perm_h = perm;
  // the persistent pass's tiles follow the work list: new lists from now on
  mesh->pk_retired.insert(mesh->pk_retired.end(), mesh->pk_lists.begin(), mesh->pk_lists.end());
  mesh->pk_lists.clear();
  DG_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return DG_OK;
}

int dg_quad_fit(dg_ctx* ctx, dg_mesh* mesh, const float* init, int iters, int install, dg_quad_stats* stats) {
  NvtxRange nv_(ctx, "dg_quad_fit");
  if (!ctx || !mesh || iters < 0) return fail(DG_ERR_ARG, "dg_quad_fit: bad argument");
  if (!mesh->lq_mom) return fail(DG_ERR_ARG, "dg_quad_fit: call dg_quad_prepare first");
  const int ne = mesh->dm.ne;
  lq_gn(mesh->dm, mesh->lq_mom, mesh->lq_mmom, mesh->lq_elig, init, iters, mesh->lq_rule, mesh->lq_resid, mesh->lq_ok,
        ctx->sm_count, ctx->stream);
  DG_CUDA_TRY(cudaGetLastError());
  if (install) {
    lq_install(mesh->dm, mesh->lq_rule, mesh->lq_ok, mesh->lq64, mesh->lq32, mesh->lq_okm, ctx->stream);
    DG_CUDA_TRY(cudaGetLastError());
  }
  if (stats || install) {
    std::vector<int> ok(ne), elig(ne);
    std::vector<float> res(ne);
    DG_CUDA_TRY(cudaMemcpyAsync(ok.data(), mesh->lq_ok, sizeof(int) * ne, cudaMemcpyDeviceToHost, ctx->stream));
    DG_CUDA_TRY(cudaMemcpyAsync(elig.data(), mesh->lq_elig, sizeof(int) * ne, cudaMemcpyDeviceToHost, ctx->stream));
    DG_CUDA_TRY(cudaMemcpyAsync(res.data(), mesh->lq_resid, sizeof(float) * ne, cudaMemcpyDeviceToHost, ctx->stream));
    DG_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    if (stats) {
      dg_quad_stats st{};
      st.elements = ne;
      float mx = 0.f;
      for (int e = 0; e < ne; ++e) {
        st.eligible += elig[e];
        st.accepted += ok[e];
        if (ok[e]) mx = std::max(mx, res[e]);
      }
      st.max_accepted_residual = mx;
      *stats = st;
    }
    if (install) {
      int rc = rebuild_worklist(ctx, mesh, ok);
      if (rc != DG_OK) return rc;
      mesh->dm.lq_ok = mesh->lq_okm;
      mesh->dm.lq64 = mesh->lq64;
      mesh->dm.lq32 = mesh->lq32;
      // algorithmic volume work of learned elements: 28 points instead of the sub-triangle rule
      for (int e = 0; e < ne; ++e)
        if (ok[e] && (mesh->owned_h.empty() || mesh->owned_h[e])) {
          mesh->flops[0][mesh->p_h[e]] -= 2.0 * (mesh->nvq_h[e] - 28) * mesh->vfma_h[e];
          mesh->flops[2][mesh->p_h[e]] -= 2.0 * (mesh->nvq_h[e] - 28) * mesh->vfma_h[e];
          mesh->flops[3][mesh->p_h[e]] -= 2.0 * (mesh->nvq_h[e] - 28) * mesh->vfma_h[e];
          for (int k = 0; k < 2; ++k) mesh->mom_exec[k][mesh->p_h[e]] -= (mesh->nvq_h[e] - 28) * mesh->mom_pt[mesh->p_h[e]];
        }
    }
  }
  return DG_OK;
}

int dg_quad_learn(dg_ctx* ctx, dg_mesh* mesh, dg_mlp* net, int iters, dg_quad_stats* stats) {
  NvtxRange nv_(ctx, "dg_quad_learn");
  if (!ctx || !mesh || iters < 0) return fail(DG_ERR_ARG, "dg_quad_learn: bad argument");
  int rc = dg_quad_prepare(ctx, mesh);
  if (rc != DG_OK) return rc;
  const float* init = nullptr;
  if (net) {
    if (!mesh->lq_out && cudaMalloc(&mesh->lq_out, sizeof(float) * 84 * (size_t)mesh->dm.ne) != cudaSuccess)
      return fail(DG_ERR_OOM, "dg_quad_learn: proposal buffer");
    rc = dg_mlp_forward(ctx, net, mesh->lq_feat, mesh->dm.ne, mesh->lq_out);
    if (rc != DG_OK) return rc;
    init = mesh->lq_out;
  }
  return dg_quad_fit(ctx, mesh, init, iters, 1, stats);
}

int dg_quad_targets(dg_ctx* ctx, dg_mesh* mesh, float* targets) {
  if (!ctx || !mesh || !targets || !mesh->lq_rule) return fail(DG_ERR_ARG, "dg_quad_targets: bad argument");
  lq_targets(mesh->dm.ne, mesh->lq_rule, mesh->lq_mmom, targets, ctx->stream);
  DG_CUDA_TRY(cudaGetLastError());
  return DG_OK;
}

int dg_quad_clear(dg_ctx* ctx, dg_mesh* mesh) {
  if (!ctx || !mesh) return fail(DG_ERR_ARG, "dg_quad_clear: null argument");
  if (mesh->dm.lq_ok) {
    std::vector<int> ok(mesh->dm.ne, 0);
    std::vector<int> okd(mesh->dm.ne);
    DG_CUDA_TRY(cudaMemcpy(okd.data(), mesh->lq_okm, sizeof(int) * mesh->dm.ne, cudaMemcpyDeviceToHost));
    for (int e = 0; e < mesh->dm.ne; ++e)
      if (okd[e] && (mesh->owned_h.empty() || mesh->owned_h[e])) {
        mesh->flops[0][mesh->p_h[e]] += 2.0 * (mesh->nvq_h[e] - 28) * mesh->vfma_h[e];
        mesh->flops[2][mesh->p_h[e]] += 2.0 * (mesh->nvq_h[e] - 28) * mesh->vfma_h[e];
        mesh->flops[3][mesh->p_h[e]] += 2.0 * (mesh->nvq_h[e] - 28) * mesh->vfma_h[e];
        for (int k = 0; k < 2; ++k) mesh->mom_exec[k][mesh->p_h[e]] += (mesh->nvq_h[e] - 28) * mesh->mom_pt[mesh->p_h[e]];
      }
    int rc = rebuild_worklist(ctx, mesh, ok);
    if (rc != DG_OK) return rc;
  }
  mesh->dm.lq_ok = nullptr;
  mesh->dm.lq64 = nullptr;
  mesh->dm.lq32 = nullptr;
  return DG_OK;
}

int dg_set_timing(dg_ctx* ctx, int enable) {
  if (!ctx) return fail(DG_ERR_ARG, "dg_set_timing: null context");
  if (enable && ctx->recs.empty()) {
    ctx->recs.resize(64);
    for (auto& r : ctx->recs) {
      DG_CUDA_TRY(cudaEventCreate(&r.ev0));
      DG_CUDA_TRY(cudaEventCreate(&r.ev1));
    }
  }
  ctx->tracer.on = enable != 0;
  ctx->tracer.recs = ctx->recs.data();
  ctx->tracer.cap = (int)ctx->recs.size();
  ctx->tracer.n = 0;
  return DG_OK;
}

int dg_kernel_stats(dg_ctx* ctx, dg_kernel_stat* out, int cap) {
  if (!ctx) return fail(DG_ERR_ARG, "dg_kernel_stats: null context");
  DG_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  const int n = ctx->tracer.on ? ctx->tracer.n : 0;
  for (int i = 0; i < n && i < cap && out; ++i) {
    const LaunchRec& r = ctx->recs[i];
    std::memcpy(out[i].name, r.name, sizeof out[i].name);
    float ms = 0.f;
    DG_CUDA_TRY(cudaEventElapsedTime(&ms, r.ev0, r.ev1));
    out[i].ms = ms;
    out[i].flops = r.flops;
    out[i].bytes = r.bytes;
  }
  // one more record, "row_pass": from the first row-kernel start to the last
  // row-kernel end (the per-degree launches may overlap on forked streams)
  int nrow = 0;
  float t0 = 1e30f, t1 = -1e30f;
  double fl = 0.0, by = 0.0;
  for (int i = 0; i < n; ++i) {
    const LaunchRec& r = ctx->recs[i];
    if (std::strncmp(r.name, "row", 3) != 0) continue;
    float a = 0.f, b = 0.f;
    DG_CUDA_TRY(cudaEventElapsedTime(&a, ctx->recs[0].ev0, r.ev0));
    DG_CUDA_TRY(cudaEventElapsedTime(&b, ctx->recs[0].ev0, r.ev1));
    t0 = std::min(t0, a);
    t1 = std::max(t1, b);
    fl += r.flops;
    by += r.bytes;
    ++nrow;
  }
  if (nrow > 0 && n < cap && out) {
    std::snprintf(out[n].name, sizeof out[n].name, "row_pass");
    out[n].ms = t1 - t0;
    out[n].flops = fl;
    out[n].bytes = by;
    if (n + 1 < cap) {
      // the same span with the flops the launches executed (the moment form
      // of the volume terms executes fewer than the quadrature sums it forms)
      double xf = 0.0;
      for (int i = 0; i < n; ++i)
        if (std::strncmp(ctx->recs[i].name, "row", 3) == 0) xf += ctx->recs[i].xflops;
      std::snprintf(out[n + 1].name, sizeof out[n + 1].name, "row_pass_executed");
      out[n + 1].ms = t1 - t0;
      out[n + 1].flops = xf;
      out[n + 1].bytes = by;
      return n + 2;
    }
    return n + 1;
  }
  return n;
}

int dg_set_tile_variants(dg_ctx* ctx, const int* variants) {
  if (!ctx) return fail(DG_ERR_ARG, "dg_set_tile_variants: null context");
  for (int p = 0; p < 9; ++p) {
    const int v = variants ? variants[p] : 0;
    if (v < 0 || v > 2) return fail(DG_ERR_ARG, "dg_set_tile_variants: variant %d of degree %d outside 0..2", v, p);
  }
  for (int p = 0; p < 9; ++p) ctx->tiles[p] = variants ? variants[p] : 0;
  return DG_OK;
}

int dg_set_nvtx(dg_ctx* ctx, int on) {
  if (!ctx) return fail(DG_ERR_ARG, "dg_set_nvtx: null context");
  ctx->nvtx = on != 0;
  return DG_OK;
}

int dg_set_group_split(dg_ctx* ctx, const int* split) {
  if (!ctx) return fail(DG_ERR_ARG, "dg_set_group_split: null context");
  for (int p = 0; p < 9; ++p) {
    const int v = split ? split[p] : 1;
    if (v < 1 || v > kMaxSplit)
      return fail(DG_ERR_ARG, "dg_set_group_split: %d parts for degree %d outside 1..%d", v, p, kMaxSplit);
  }
  for (int p = 0; p < 9; ++p) ctx->splits[p] = split ? split[p] : 1;
  return DG_OK;
}

int dg_set_volume_path(dg_ctx* ctx, int path) {
  if (!ctx || path < 0 || path > 2) return fail(DG_ERR_ARG, "dg_set_volume_path: bad argument");
  ctx->vol_moments = path >= 1;
  ctx->vol_exact = path == 2;
  return DG_OK;
}

int dg_sync(dg_ctx* ctx) {
  if (!ctx) return fail(DG_ERR_ARG, "dg_sync: null context");
  DG_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  DG_CUDA_TRY(cudaGetLastError());
  int st = 0;
  DG_CUDA_TRY(cudaMemcpy(&st, ctx->status_dev, sizeof(int), cudaMemcpyDeviceToHost));
  if (st) {
    DG_CUDA_TRY(cudaMemset(ctx->status_dev, 0, sizeof(int)));
    if (st & 2)
      return fail(DG_ERR_BOUNDS, "a kernel found an output range outside its array and skipped it (status 0x%x)", st);
    return fail(DG_ERR_TIMEOUT, "a bounded device wait ran out (status 0x%x); the pass's results are incomplete", st);
  }
  return DG_OK;
}

int dg_set_persistent(dg_ctx* ctx, int on) {
  if (!ctx) return fail(DG_ERR_ARG, "dg_set_persistent: null context");
  ctx->persist = on != 0;
  return DG_OK;
}

int dg_set_wait_limit(dg_ctx* ctx, double seconds) {
  if (!ctx || !(seconds > 0.0) || seconds > 60.0) return fail(DG_ERR_ARG, "dg_set_wait_limit: seconds outside (0, 60]");
  ctx->wait_ns = (long long)(seconds * 1e9);
  return DG_OK;
}

int dg_wait_probe(dg_ctx* ctx, const int* flag, double seconds) {
  if (!ctx || !flag || !(seconds > 0.0) || seconds > 60.0) return fail(DG_ERR_ARG, "dg_wait_probe: bad argument");
  launch_wait_probe(flag, ctx->status_dev, (long long)(seconds * 1e9), ctx->stream);
  DG_CUDA_TRY(cudaGetLastError());
  return DG_OK;
}

int dg_last_launch_count(const dg_ctx* ctx) { return ctx ? ctx->last_launches : 0; }

}  // extern "C"

cudaStream_t dg_ctx_stream(dg_ctx* ctx) { return ctx->stream; }

extern "C" {

}  // extern "C"
