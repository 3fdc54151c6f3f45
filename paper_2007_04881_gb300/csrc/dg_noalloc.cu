// dg_noalloc.cu -- an entry point that allocates nothing on the device.
//
// Some callers cannot call cudaMalloc: code running inside another
// framework's memory pool or under a fixed memory budget, processes that
// must not grow their footprint after start-up, and hosts that forbid
// device allocation once captured workloads are set up.  dg_volume_noalloc
// serves them: the caller passes its own device buffers for every input and
// output, and the intermediate records of the pass (element and sub-triangle
// geometry, the identity work lists, the reference rules) live in one
// file-scope device array, g_noalloc_scratch, of kNoallocScratchBytes.
// Every GPU that loads the library holds this array until the process exits.
//
// The pass is the library's own: the geometry kernels write the element and
// sub-triangle records into the array, then the degree-p row kernel, in
// volume-only mode, reads them and writes the blocks.
//
// The host cannot read the caller's device index lists without a copy and a
// wait, so the pass never indexes with them directly: a first kernel checks
// them (elem_ptr a non-decreasing list from 0 to nsub with at least three
// vertices per loop, every vertex id in 0..nv-1), a second writes the copies
// the pass reads into the array: the caller's lists when they are valid,
// otherwise a stand-in mesh of the same sizes (three vertices per loop, the
// rest to the last one, vertex 0 for a bad id), so that every index the
// later kernels form stays inside their buffers.  The check's verdict goes to
// the caller's status word.
#include <mutex>
#include <vector>

#include "../../include/dg.h"
#include "dg_internal.h"

namespace dg {

namespace {

constexpr size_t kNoallocScratchBytes = 16u << 20;  // 16 MiB
constexpr int kNoallocMaxElems = 16384;
constexpr int kNoallocMaxSub = 131072;
constexpr int kMaxDevices = 64;
// the reference rules take the first kNoallocRuleBytes of the array, the
// per-call records the rest
constexpr size_t kNoallocRuleBytes = 64u << 10;

// The scratch array.  Host code must not take its address: the host-side
// name is only a stand-in for the device symbol; its device address comes
// from cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

struct NoallocDev {
  unsigned char* base = nullptr;  // device address of g_noalloc_scratch
  int sm_count = 0;
  RuleTables rt;  // 2D reference rules, inside the array
};
NoallocDev g_dev[kMaxDevices];
std::mutex g_mu;

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

// Layout of the array: rule tables first (written once per device at
// set-up), then the per-call records.
struct Carve {
  size_t off = 0;
  template <typename T>
  size_t take(size_t n) {
    const size_t o = off;
    off = up256(off + n * sizeof(T));
    return o;
  }
};

int fail_na(int code, const char* msg);

// Once per device, with that device current: resolve the array's device
// address and write the reference rules into it.
int noalloc_setup(int device, NoallocDev** out) {
  std::lock_guard<std::mutex> lk(g_mu);
  NoallocDev& d = g_dev[device];
  if (!d.base) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return fail_na(DG_ERR_CUDA, cudaGetErrorString(e));
    if (cudaDeviceGetAttribute(&d.sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
      return fail_na(DG_ERR_CUDA, "device attribute query failed");
    // rules: volume rules p = 1..kPMax2 ((p+2)^2 points), edge rules n = 1..kPMax2+1
    std::vector<double> vol, face, pts;
    RuleTables rt;
    for (int p = 1; p <= kPMax2; ++p) {
      reference_rule(2, p + 2, pts);
      rt.vol_off[p] = (int)(vol.size() / 3);
      rt.vol_n[p] = (int)(pts.size() / 3);
      vol.insert(vol.end(), pts.begin(), pts.end());
    }
    for (int n = 1; n <= kPMax2 + 1; ++n) {
      reference_rule(1, n, pts);
      rt.face_off[n] = (int)(face.size() / 2);
      rt.face_n[n] = (int)(pts.size() / 2);
      face.insert(face.end(), pts.begin(), pts.end());
    }
    std::vector<float> vf(vol.begin(), vol.end()), ff(face.begin(), face.end());
    unsigned char* b = static_cast<unsigned char*>(ptr);
    Carve c;
    const size_t o_v64 = c.take<double>(vol.size()), o_v32 = c.take<float>(vol.size());
    const size_t o_f64 = c.take<double>(face.size()), o_f32 = c.take<float>(face.size());
    if (c.off > kNoallocRuleBytes) return fail_na(DG_ERR_CUDA, "reference rules exceed their region of the array");
    if (cudaMemcpy(b + o_v64, vol.data(), vol.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b + o_v32, vf.data(), vf.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b + o_f64, face.data(), face.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b + o_f32, ff.data(), ff.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess)
      return fail_na(DG_ERR_CUDA, "writing the reference rules failed");
    rt.vol64 = reinterpret_cast<const double*>(b + o_v64);
    rt.vol32 = reinterpret_cast<const float*>(b + o_v32);
    rt.face64 = reinterpret_cast<const double*>(b + o_f64);
    rt.face32 = reinterpret_cast<const float*>(b + o_f32);
    d.rt = rt;
    d.base = b;
  }
  *out = &d;
  return DG_OK;
}

// The check of the caller's lists: err (in the array, zeroed before) gets
// bit 0 for a bad elem_ptr, bit 1 for a vertex id outside 0..nv-1.
__global__ void noalloc_check_kernel(int ne, int nsub, int nv, const int* __restrict__ eptr,
                                     const int* __restrict__ eidx, int* err) {
  const int n = ne + 1 > nsub ? ne + 1 : nsub;
  int bad = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (i <= ne) {
      const int b = eptr[i];
      if ((i == 0 && b != 0) || (i == ne && b != nsub) || (i < ne && eptr[i + 1] - b < 3)) bad |= 1;
    }
    if (i < nsub) {
      const int v = eidx[i];
      if (v < 0 || v >= nv) bad |= 2;
    }
  }
  if (bad) atomicOr(err, bad);
}

// The lists the pass reads, and the identity work lists and block layout for
// ne elements of one degree.  Everything the pass reads is rewritten.  With a
// bad elem_ptr (err bit 0) loop e takes vertices 3e .. 3e + 2 and the last
// loop the rest; a bad vertex id becomes 0.  status (caller's, may be null)
// gets 0 or DG_ERR_MESH.
__global__ void noalloc_setup_kernel(int ne, int p, int nsq, int nsub, int nv, const int* __restrict__ eptr,
                                     const int* __restrict__ eidx, const int* __restrict__ err, int* status,
                                     int* eptr_s, int* eidx_s, int* elem_perm, int* diag_blk, int* row_ptr,
                                     int64_t* blk_off, int* e_nqf, int* hf_ptr, int* pe, int* sub_elem) {
  const int bad = *err;
  const int n = ne + 1 > nsub ? ne + 1 : nsub;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (i == 0 && status) *status = bad ? DG_ERR_MESH : DG_OK;
    if (i <= ne) {
      eptr_s[i] = (bad & 1) ? (i == ne ? nsub : 3 * i) : eptr[i];
      row_ptr[i] = i;
      blk_off[i] = (int64_t)i * nsq;
      hf_ptr[i] = 0;
      if (i < ne) {
        elem_perm[i] = i;
        diag_blk[i] = i;
        e_nqf[i] = 0;
        pe[i] = p;
      }
    }
    if (i < nsub) {
      const int v = eidx[i];
      eidx_s[i] = v >= 0 && v < nv ? v : 0;
      int e;
      if (bad & 1) {
        e = i / 3 < ne - 1 ? i / 3 : ne - 1;
      } else {
        // the loop holding position i: eptr is valid, so a binary search
        int lo = 0, hi = ne - 1;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (eptr[mid] <= i)
            lo = mid;
          else
            hi = mid - 1;
        }
        e = lo;
      }
      sub_elem[i] = e;
    }
  }
}

}  // namespace

int fail_na_impl(int code, const char* msg);

namespace {
int fail_na(int code, const char* msg) { return fail_na_impl(code, msg); }
}  // namespace

}  // namespace dg

namespace dg {
namespace {
// Restores the calling thread's current device on every return path.
struct DeviceGuard {
  int prev = -1;
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};
}  // namespace
}  // namespace dg

extern "C" int dg_volume_noalloc(void* stream, int device, int prec, int p, int nv, const double* x,
                                 const double* y, int ne, int nsub, const int* elem_ptr, const int* elem_idx,
                                 const double* a, double bx, double by, double c, void* blocks, int* status) {
  using namespace dg;
  if (device < 0 || device >= kMaxDevices) return fail_na(DG_ERR_ARG, "dg_volume_noalloc: device out of range");
  if (prec != DG_PREC_FP64 && prec != DG_PREC_FP32) return fail_na(DG_ERR_ARG, "dg_volume_noalloc: unknown precision");
  if (p < 1 || p > kPMax2) return fail_na(DG_ERR_ARG, "dg_volume_noalloc: p outside 1..6");
  if (ne <= 0 || nv <= 0 || nsub < 3 * ne) return fail_na(DG_ERR_ARG, "dg_volume_noalloc: bad sizes");
  if (ne > kNoallocMaxElems || nsub > kNoallocMaxSub)
    return fail_na(DG_ERR_ARG, "dg_volume_noalloc: more than 16384 elements or 131072 loop vertices");
  if (!x || !y || !elem_ptr || !elem_idx || !a || !blocks) return fail_na(DG_ERR_ARG, "dg_volume_noalloc: null pointer");

  // per-call records inside the array, after the rule tables: the layout
  // depends on the sizes only, so it is checked before any GPU call
  const int n = nbasis(2, p);
  Carve cv;
  cv.off = kNoallocRuleBytes;
  const size_t o_err = cv.take<int>(1);
  const size_t o_eptr = cv.take<int>(ne + 1), o_eidx = cv.take<int>(nsub);
  const size_t o_perm = cv.take<int>(ne), o_diag = cv.take<int>(ne), o_row = cv.take<int>(ne + 1);
  const size_t o_blk = cv.take<int64_t>(ne + 1), o_nqf = cv.take<int>(ne), o_hf = cv.take<int>(ne + 1);
  const size_t o_p = cv.take<int>(ne), o_sub = cv.take<int>(nsub);
  const size_t o_lo = cv.take<double>(2 * ne), o_L = cv.take<double>(2 * ne), o_cen = cv.take<double>(2 * ne);
  const size_t o_vol = cv.take<double>(ne), o_h = cv.take<double>(ne), o_pen = cv.take<double>(ne);
  const size_t o_eg64 = cv.take<double>((size_t)elem_vals(2) * ne), o_eg32 = cv.take<float>((size_t)elem_vals(2) * ne);
  const size_t o_sg64 = cv.take<double>((size_t)sub_vals(2) * nsub), o_sg32 = cv.take<float>((size_t)sub_vals(2) * nsub);
  if (cv.off > kNoallocScratchBytes) return fail_na(DG_ERR_ARG, "dg_volume_noalloc: mesh exceeds the scratch array");

  DeviceGuard guard;
  if (cudaGetDevice(&guard.prev) != cudaSuccess) {
    guard.prev = -1;
    return fail_na(DG_ERR_CUDA, "dg_volume_noalloc: cudaGetDevice failed");
  }
  if (cudaSetDevice(device) != cudaSuccess) return fail_na(DG_ERR_CUDA, "dg_volume_noalloc: cudaSetDevice failed");
  NoallocDev* nd = nullptr;
  int rc = noalloc_setup(device, &nd);
  if (rc != DG_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned char* b = nd->base;
  int* err = reinterpret_cast<int*>(b + o_err);
  int* eptr_s = reinterpret_cast<int*>(b + o_eptr);
  int* eidx_s = reinterpret_cast<int*>(b + o_eidx);

  DevMesh m{};  // value-initialised: every pointer null, every count zero
  m.dim = 2;
  m.nv = nv;
  m.ne = ne;
  m.nsub = nsub;
  m.nf = 0;
  m.ni = 0;
  m.nhf = 0;
  m.X[0] = x;
  m.X[1] = y;
  m.eptr = eptr_s;
  m.eidx = eidx_s;
  m.uvptr = eptr_s;  // 2D: the loop is the vertex list
  m.uvidx = eidx_s;
  m.sub_elem = reinterpret_cast<const int*>(b + o_sub);
  m.p = reinterpret_cast<const int*>(b + o_p);
  m.a = a;
  m.lo = reinterpret_cast<double*>(b + o_lo);
  m.L = reinterpret_cast<double*>(b + o_L);
  m.cen = reinterpret_cast<double*>(b + o_cen);
  m.vol = reinterpret_cast<double*>(b + o_vol);
  m.h = reinterpret_cast<double*>(b + o_h);
  m.pen = reinterpret_cast<double*>(b + o_pen);
  m.eg64 = reinterpret_cast<double*>(b + o_eg64);
  m.eg32 = reinterpret_cast<float*>(b + o_eg32);
  m.sg64 = reinterpret_cast<double*>(b + o_sg64);
  m.sg32 = reinterpret_cast<float*>(b + o_sg32);
  m.hf_ptr = reinterpret_cast<const int*>(b + o_hf);
  m.e_nqf = reinterpret_cast<const int*>(b + o_nqf);
  m.row_ptr = reinterpret_cast<const int*>(b + o_row);
  m.blk_off = reinterpret_cast<const int64_t*>(b + o_blk);
  m.diag_blk = reinterpret_cast<const int*>(b + o_diag);
  m.elem_perm = reinterpret_cast<const int*>(b + o_perm);
  m.nmax = n;
  m.pmask = 1 << p;
  m.nvals = (int64_t)ne * n * n;  // the caller's block array (a checked build tests writes against it)
  for (int q = 0; q <= 8; ++q) m.elem_pstart[q] = q <= p ? 0 : ne;
  m.pb.b[0] = bx;
  m.pb.b[1] = by;
  m.pb.b[2] = 0.0;
  m.pb.c = c;
  m.pb.source = DG_SRC_ZERO;
  m.pb.c_sigma = 10.0;
  m.pb.neumann = 0;
  m.pb.round_copies();
  m.rt = nd->rt;

  // the check's verdict starts at zero on every call (the array keeps the last call's contents)
  if (cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess)
    return fail_na(DG_ERR_CUDA, "dg_volume_noalloc: clearing the status word failed");
  const int nitems = ne + 1 > nsub ? ne + 1 : nsub;
  const int nblocks = (nitems + 255) / 256;
  noalloc_check_kernel<<<nblocks, 256, 0, st>>>(ne, nsub, nv, elem_ptr, elem_idx, err);
  noalloc_setup_kernel<<<nblocks, 256, 0, st>>>(
      ne, p, n * n, nsub, nv, elem_ptr, elem_idx, err, status, eptr_s, eidx_s, reinterpret_cast<int*>(b + o_perm),
      reinterpret_cast<int*>(b + o_diag), reinterpret_cast<int*>(b + o_row), reinterpret_cast<int64_t*>(b + o_blk),
      reinterpret_cast<int*>(b + o_nqf), reinterpret_cast<int*>(b + o_hf), reinterpret_cast<int*>(b + o_p),
      reinterpret_cast<int*>(b + o_sub));
  launch_geometry(m, st, nullptr, prec == DG_PREC_FP64 ? 1 : 2);
  LaunchOpts lo;
  lo.vol_moments = false;  // the per-point contraction: needs no linearisation tables
  for (int q = 0; q < 9; ++q) lo.pst[q] = st;
  if (prec == DG_PREC_FP64)
    launch_row2d_f64(m, kModeVol, static_cast<double*>(blocks), nullptr, nd->sm_count, lo, nullptr);
  else
    launch_row2d_f32(m, kModeVol, static_cast<float*>(blocks), nullptr, nd->sm_count, lo, nullptr);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail_na(DG_ERR_CUDA, cudaGetErrorString(e));
  return DG_OK;
}
