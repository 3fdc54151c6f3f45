// dg_pattern.cu -- the block-sparse pattern of a mesh built on the device.
//
// The paper builds the sparsity pattern ("indices", the largest term of its
// assembly totals, Tables 1, 2, 5 and 6) with Thrust on the GPU (Sec. 3.4,
// Approach 2 with a precomputed pattern; Sec. 4.2).  Here every step of the
// host pass plan_mesh (dg_host.cu) has a kernel counterpart, and the results
// are the same arrays bit for bit:
//   1. half faces: one per 2D loop edge or 3D tetrahedron triangle, keyed by
//      their sorted vertex ids packed into one integer (base nv);
//   2. a stable LSD radix sort of the keys (8 bits per pass, as many passes
//      as the largest key needs), so equal keys stay in element order;
//   3. matching: a key seen twice is an interior face (owner e0 the lower
//      element, its half face's vertex order), once a boundary face, three
//      times an error; two halves of one 3D element are no face;
//   4. faces ordered by (boundary, e0, e1), stable (radix sort);
//   5. interfaces = runs of equal (e0, e1) among interior faces;
//   6. block rows: per element the interfaces where it is e1 (ascending e0,
//      from a stable sort by e1), itself, those where it is e0 (ascending
//      e1, a contiguous range); block offsets, load-vector offsets and the
//      half-face lists by exclusive scans; per-element face-point offsets;
//   7. the work lists: elements by (degree, cost descending), interfaces by
//      (largest degree, points descending), both stable radix sorts.
// Every reduction that decides an output is an integer operation, so the
// result does not depend on the order in which threads run.
#include <algorithm>
#include <array>
#include <cstdint>
#include <cstring>
#include <functional>
#include <string>
#include <vector>

#include "../../include/dg.h"
#include "dg_internal.h"

namespace dg {
namespace {

constexpr int kT = 256;          // threads per block of the simple kernels
constexpr int kSortItems = 8;    // items per thread in a radix-sort tile
constexpr int kSortTile = kT * kSortItems;
constexpr int kScanItems = 4;    // items per thread in a scan block
constexpr int kScanTile = 1024 * kScanItems;

inline int nblk(int64_t n, int t = kT) { return (int)((n + t - 1) / t); }

// error bits of the device build
enum : int {
  kErrRepeat = 1,     // a loop repeats a vertex on consecutive positions
  kErrManifold = 2,   // a face shared by more than two element pieces
  kErrTwice = 4,      // a 2D element traverses an edge twice
  kErrOrient = 8,     // two 2D loops traverse their common edge in the same direction
  kErrArea = 16,      // a 2D loop with non-positive area or fan triangle
  kErrVolume = 32,    // a tetrahedron of zero volume
};

// ---------------------------------------------------------------------------
// exclusive scan (int32 / int64), out[n] = total
// ---------------------------------------------------------------------------

template <typename T>
__global__ void scan_block_kernel(const T* __restrict__ in, T* __restrict__ out, int64_t n, T* __restrict__ bsum) {
  __shared__ T s[1024];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  T v[kScanItems], run = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = base + i < n ? in[base + i] : T(0);
    run += v[i];
  }
  s[threadIdx.x] = run;
  __syncthreads();
  // Hillis-Steele inclusive scan of the thread totals
  for (int off = 1; off < 1024; off <<= 1) {
    const T x = threadIdx.x >= off ? s[threadIdx.x - off] : T(0);
    __syncthreads();
    s[threadIdx.x] += x;
    __syncthreads();
  }
  T pre = s[threadIdx.x] - run;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < n) out[base + i] = pre;
    pre += v[i];
  }
  if (threadIdx.x == 1023) bsum[blockIdx.x] = s[1023];
}

template <typename T>
__global__ void scan_add_kernel(T* __restrict__ out, int64_t n, const T* __restrict__ boff) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] += boff[i / kScanTile];
}

template <typename T>
__global__ void set_total_kernel(T* out, int64_t n, const T* last_in) {
  out[n] = out[n - 1] + *last_in;
}

// out[0..n] = exclusive scan of in[0..n-1], out[n] the total; in and out may
// not alias.  scratch: device buffers, grown as needed.
template <typename T>
void scan_exclusive(const T* in, T* out, int64_t n, cudaStream_t st, std::vector<void*>& scratch) {
  if (n <= 0) {
    cudaMemsetAsync(out, 0, sizeof(T), st);
    return;
  }
  const int64_t nb = (n + kScanTile - 1) / kScanTile;
  T* bsum = nullptr;
  cudaMalloc(&bsum, sizeof(T) * (nb + 1));
  scratch.push_back(bsum);
  scan_block_kernel<T><<<(int)nb, 1024, 0, st>>>(in, out, n, bsum);
  if (nb > 1) {
    T* boff = nullptr;
    cudaMalloc(&boff, sizeof(T) * (nb + 1));
    scratch.push_back(boff);
    scan_exclusive<T>(bsum, boff, nb, st, scratch);
    scan_add_kernel<T><<<nblk(n), kT, 0, st>>>(out, n, boff);
  }
  set_total_kernel<T><<<1, 1, 0, st>>>(out, n, in + (n - 1));
}

// ---------------------------------------------------------------------------
// stable LSD radix sort of (uint64 key, uint32 value) pairs
// ---------------------------------------------------------------------------

// digit counts of one tile: hist[d * ntiles + tile]
__global__ void radix_hist_kernel(const uint64_t* __restrict__ key, int n, int shift, int ntiles, int* __restrict__ hist) {
  __shared__ int cnt[256];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  const int base = blockIdx.x * kSortTile;
  for (int i = threadIdx.x; i < kSortTile; i += kT) {
    const int j = base + i;
    if (j < n) atomicAdd(&cnt[(key[j] >> shift) & 255], 1);
  }
  __syncthreads();
  hist[threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

// Scatter one tile in input order: items are taken in rounds of kT (thread t
// holds item round * kT + t); within a round the rank of an item among the
// earlier items of its digit comes from the warp's match mask and the
// per-warp digit counts; a running count per digit carries across rounds.
__global__ void radix_scatter_kernel(const uint64_t* __restrict__ key, const uint32_t* __restrict__ val, int n,
                                     int shift, int ntiles, const int* __restrict__ off, uint64_t* __restrict__ okey,
                                     uint32_t* __restrict__ oval) {
  constexpr int W = kT / 32;
  __shared__ int run[256];
  __shared__ int wcnt[W][256];
  __shared__ int goff[256];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  run[threadIdx.x] = 0;
  goff[threadIdx.x] = off[threadIdx.x * ntiles + blockIdx.x];
  const int base = blockIdx.x * kSortTile;
  for (int r = 0; r < kSortItems; ++r) {
    for (int w = 0; w < W; ++w) wcnt[w][threadIdx.x] = 0;
    __syncthreads();
    const int j = base + r * kT + threadIdx.x;
    const bool ok = j < n;
    uint64_t k = 0;
    uint32_t v = 0;
    int d = 256;  // no item
    if (ok) {
      k = key[j];
      v = val[j];
      d = (int)((k >> shift) & 255);
    }
    const unsigned same = __match_any_sync(0xffffffffu, d);
    const int rank = __popc(same & ((1u << lane) - 1u));
    if (ok && rank == 0) wcnt[warp][d] = __popc(same);
    __syncthreads();
    if (ok) {
      int pos = goff[d] + run[d] + rank;
      for (int w = 0; w < warp; ++w) pos += wcnt[w][d];
      okey[pos] = k;
      oval[pos] = v;
    }
    __syncthreads();
    int add = 0;
    for (int w = 0; w < W; ++w) add += wcnt[w][threadIdx.x];
    run[threadIdx.x] += add;
    __syncthreads();
  }
}

__global__ void iota_kernel(uint32_t* v, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = (uint32_t)i;
}

// Sort n pairs by the low `bits` bits of key, stably; the result is in
// (key, val) on return (ping-pong buffers tk, tv of n entries).
void radix_sort(uint64_t*& key, uint32_t*& val, uint64_t*& tk, uint32_t*& tv, int n, int bits, cudaStream_t st,
                std::vector<void*>& scratch) {
  if (n <= 1) return;
  const int ntiles = (n + kSortTile - 1) / kSortTile;
  int *hist = nullptr, *off = nullptr;
  cudaMalloc(&hist, sizeof(int) * 256 * (size_t)ntiles);
  cudaMalloc(&off, sizeof(int) * (256 * (size_t)ntiles + 1));
  scratch.push_back(hist);
  scratch.push_back(off);
  for (int shift = 0; shift < bits; shift += 8) {
    radix_hist_kernel<<<ntiles, kT, 0, st>>>(key, n, shift, ntiles, hist);
    scan_exclusive<int>(hist, off, 256 * (int64_t)ntiles, st, scratch);
    radix_scatter_kernel<<<ntiles, kT, 0, st>>>(key, val, n, shift, ntiles, off, tk, tv);
    std::swap(key, tk);
    std::swap(val, tv);
  }
}

inline int bits_for(uint64_t maxkey) {
  int b = 0;
  while (b < 64 && (maxkey >> b) != 0) ++b;
  return b;
}

// ---------------------------------------------------------------------------
// the steps
// ---------------------------------------------------------------------------

__global__ void sub_elem_kernel(const int* __restrict__ eptr, int ne, int* __restrict__ sub_elem) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  for (int k = eptr[e]; k < eptr[e + 1]; ++k) sub_elem[k] = e;
}

// geometric validity (FP64, as the host check): 2D loops with positive area
// and positive fan triangles about the area centroid; 3D tetrahedra of
// non-zero volume
__global__ void validity2d_kernel(const double* __restrict__ x, const double* __restrict__ y, const int* __restrict__ eptr,
                                  const int* __restrict__ eidx, int ne, int* err) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  const int b = eptr[e], k = eptr[e + 1] - b;
  double A = 0, cx = 0, cy = 0;
  for (int i = 0; i < k; ++i) {
    const int v0 = eidx[b + i], v1 = eidx[b + (i + 1 == k ? 0 : i + 1)];
    const double cr = x[v0] * y[v1] - x[v1] * y[v0];
    A += 0.5 * cr;
    cx += (x[v0] + x[v1]) * cr;
    cy += (y[v0] + y[v1]) * cr;
  }
  if (!(A > 0.0)) {
    atomicOr(err, kErrArea);
    return;
  }
  cx /= 6 * A;
  cy /= 6 * A;
  for (int i = 0; i < k; ++i) {
    const int v0 = eidx[b + i], v1 = eidx[b + (i + 1 == k ? 0 : i + 1)];
    const double tri = (x[v0] - cx) * (y[v1] - cy) - (y[v0] - cy) * (x[v1] - cx);
    if (!(tri > 0.0)) atomicOr(err, kErrArea);
  }
}

// 2D half faces: one per loop position k (edge v_k -> v_{k+1})
__global__ void half2d_kernel(const int* __restrict__ eptr, const int* __restrict__ eidx, const int* __restrict__ sub_elem,
                              int nh, int nv, uint64_t* __restrict__ key, uint32_t* __restrict__ val, int* __restrict__ hv,
                              int* err) {
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= nh) return;
  const int e = sub_elem[h], b = eptr[e], len = eptr[e + 1] - b, i = h - b;
  const int v0 = eidx[h], v1 = eidx[b + (i + 1 == len ? 0 : i + 1)];
  if (v0 == v1) atomicOr(err, kErrRepeat);
  const uint64_t lo = (uint64_t)min(v0, v1), hi = (uint64_t)max(v0, v1);
  key[h] = lo * (uint64_t)nv + hi;
  val[h] = (uint32_t)h;
  hv[3 * h] = v0;
  hv[3 * h + 1] = v1;
  hv[3 * h + 2] = -1;
}

// 3D half faces: the 4 triangles of each tetrahedron, in the tetrahedron's
// vertex order, flagged where (v1-v0) x (v2-v0) points into the tetrahedron
__global__ void half3d_kernel(const double* __restrict__ x, const double* __restrict__ y, const double* __restrict__ z,
                              const int* __restrict__ tet, int nt, int nv, uint64_t* __restrict__ key,
                              uint32_t* __restrict__ val, int* __restrict__ hv, int8_t* __restrict__ hflip, int* err) {
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= 4 * nt) return;
  const int t = h >> 2, o = h & 3;
  const int* tv = tet + 4 * t;
  int v[3], c = 0;
  for (int i = 0; i < 4; ++i)
    if (i != o) v[c++] = tv[i];
  const double* X[3] = {x, y, z};
  double u[3], w[3], s[3];
  for (int q = 0; q < 3; ++q) {
    u[q] = X[q][v[1]] - X[q][v[0]];
    w[q] = X[q][v[2]] - X[q][v[0]];
    s[q] = X[q][tv[o]] - X[q][v[0]];
  }
  const double cr[3] = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]};
  hflip[h] = cr[0] * s[0] + cr[1] * s[1] + cr[2] * s[2] > 0.0 ? 1 : 0;
  if (o == 0) {
    const double det = cr[0] * s[0] + cr[1] * s[1] + cr[2] * s[2];
    if (!(fabs(det) > 0.0)) atomicOr(err, kErrVolume);
  }
  int kk[3] = {v[0], v[1], v[2]};
  if (kk[0] > kk[1]) { const int tt = kk[0]; kk[0] = kk[1]; kk[1] = tt; }
  if (kk[1] > kk[2]) { const int tt = kk[1]; kk[1] = kk[2]; kk[2] = tt; }
  if (kk[0] > kk[1]) { const int tt = kk[0]; kk[0] = kk[1]; kk[1] = tt; }
  key[h] = ((uint64_t)kk[0] * (uint64_t)nv + (uint64_t)kk[1]) * (uint64_t)nv + (uint64_t)kk[2];
  val[h] = (uint32_t)h;
  hv[3 * h] = v[0];
  hv[3 * h + 1] = v[1];
  hv[3 * h + 2] = v[2];
}

// a sorted half face that opens a run of equal keys and emits a face
__global__ void match_kernel(const uint64_t* __restrict__ skey, const uint32_t* __restrict__ sval, int nh,
                             const int* __restrict__ helem, int dim, int* __restrict__ emit, int* err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nh) return;
  int out = 0;
  if (i == 0 || skey[i] != skey[i - 1]) {
    int cnt = 1;
    while (i + cnt < nh && skey[i + cnt] == skey[i] && cnt < 3) ++cnt;
    if (cnt > 2) {
      atomicOr(err, kErrManifold);
    } else if (cnt == 2 && helem[sval[i]] == helem[sval[i + 1]]) {
      if (dim == 2) atomicOr(err, kErrTwice);  // 3D: interior to one element, no face
    } else {
      out = 1;
    }
  }
  emit[i] = out;
}

// face records in key order (fk: the composite order key, fid its index)
__global__ void emit_kernel(const uint64_t* __restrict__ skey, const uint32_t* __restrict__ sval, int nh,
                            const int* __restrict__ emit, const int* __restrict__ fpos, const int* __restrict__ helem,
                            const int* __restrict__ hv, const int8_t* __restrict__ hflip, int dim, int ne,
                            int* __restrict__ fe0, int* __restrict__ fe1, int* __restrict__ fv, int8_t* __restrict__ fflip,
                            uint64_t* __restrict__ fk, uint32_t* __restrict__ fid, int* __restrict__ nint, int* err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nh || !emit[i]) return;
  const int f = fpos[i];
  const uint32_t h0 = sval[i];
  const bool two = i + 1 < nh && skey[i + 1] == skey[i];
  const int e0 = helem[h0], e1 = two ? helem[sval[i + 1]] : -1;
  fe0[f] = e0;
  fe1[f] = e1;
  for (int q = 0; q < dim; ++q) fv[dim * f + q] = hv[3 * h0 + q];
  fflip[f] = hflip ? hflip[h0] : 0;
  if (two && dim == 2) {
    const uint32_t h1 = sval[i + 1];
    if (!(hv[3 * h0] == hv[3 * h1 + 1] && hv[3 * h0 + 1] == hv[3 * h1])) atomicOr(err, kErrOrient);
  }
  if (two) atomicAdd(nint, 1);
  const uint64_t base = (uint64_t)ne + 1;
  fk[f] = ((uint64_t)(e1 < 0) * base + (uint64_t)e0) * base + (uint64_t)(e1 + 1);
  fid[f] = (uint32_t)f;
}

// faces in their final order, points per direction
__global__ void face_order_kernel(const uint32_t* __restrict__ ford, int nf, int dim, const int* __restrict__ fe0,
                                  const int* __restrict__ fe1, const int* __restrict__ fv, const int8_t* __restrict__ fflip,
                                  const int* __restrict__ p, int* __restrict__ f_e0, int* __restrict__ f_e1,
                                  int* __restrict__ f_v, int8_t* __restrict__ f_flip, int* __restrict__ f_nq) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nf) return;
  const int g = (int)ford[f];
  const int e0 = fe0[g], e1 = fe1[g];
  f_e0[f] = e0;
  f_e1[f] = e1;
  for (int q = 0; q < dim; ++q) f_v[dim * f + q] = fv[dim * g + q];
  f_flip[f] = fflip[g];
  f_nq[f] = (e1 >= 0 ? max(p[e0], p[e1]) : p[e0]) + 1;
}

__global__ void iface_head_kernel(const int* __restrict__ f_e0, const int* __restrict__ f_e1, int nint, int* __restrict__ head) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nint) return;
  head[f] = f == 0 || f_e0[f] != f_e0[f - 1] || f_e1[f] != f_e1[f - 1];
}

__global__ void iface_kernel(const int* __restrict__ f_e0, const int* __restrict__ f_e1, int nint,
                             const int* __restrict__ head, const int* __restrict__ ipos, int ni, int* __restrict__ if_e0,
                             int* __restrict__ if_e1, int* __restrict__ if_fptr, int* __restrict__ c0, int* __restrict__ c1,
                             int* __restrict__ first0, uint64_t* __restrict__ k1, uint32_t* __restrict__ v1) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f == 0) if_fptr[ni] = nint;
  if (f >= nint || !head[f]) return;
  const int i = ipos[f];
  const int a = f_e0[f], b = f_e1[f];
  if_e0[i] = a;
  if_e1[i] = b;
  if_fptr[i] = f;
  atomicAdd(&c0[a], 1);
  atomicAdd(&c1[b], 1);
  if (i == 0 || f_e0[f] != f_e0[f - 1]) first0[a] = i;
  k1[i] = (uint64_t)b;
  v1[i] = (uint32_t)i;
}

__global__ void row_count_kernel(const int* __restrict__ c0, const int* __restrict__ c1, int ne, int* __restrict__ rc) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < ne) rc[e] = c0[e] + c1[e] + 1;
}

// block rows: lower neighbours (interfaces where e is e1, ascending e0),
// the element, upper neighbours (where e is e0, ascending e1)
__global__ void rows_kernel(int ne, const int* __restrict__ row_ptr, const int* __restrict__ c0,
                            const int* __restrict__ c1, const int* __restrict__ first0, const int* __restrict__ first1,
                            const uint32_t* __restrict__ list1, const int* __restrict__ if_e0,
                            const int* __restrict__ if_e1, const int* __restrict__ nb, int* __restrict__ col,
                            int* __restrict__ blk_if, int* __restrict__ diag_blk, int* __restrict__ slot01,
                            int* __restrict__ slot10, int64_t* __restrict__ bsz, int* __restrict__ brow) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  int pos = row_ptr[e];
  const int64_t ne_ = nb[e];
  for (int j = 0; j < c1[e]; ++j, ++pos) {
    const int it = (int)list1[first1[e] + j];
    col[pos] = if_e0[it];
    blk_if[pos] = it;
    slot10[it] = pos;
    bsz[pos] = ne_ * nb[if_e0[it]];
    brow[pos] = e;
  }
  col[pos] = e;
  blk_if[pos] = -1;
  diag_blk[e] = pos;
  bsz[pos] = ne_ * ne_;
  brow[pos] = e;
  ++pos;
  for (int j = 0; j < c0[e]; ++j, ++pos) {
    const int it = first0[e] + j;
    col[pos] = if_e1[it];
    blk_if[pos] = it;
    slot01[it] = pos;
    bsz[pos] = ne_ * nb[if_e1[it]];
    brow[pos] = e;
  }
}

__global__ void nbasis_kernel(const int* __restrict__ p, int ne, int dim, int* __restrict__ nb, int64_t* __restrict__ nb64) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  nb[e] = nbasis(dim, p[e]);
  nb64[e] = nb[e];
}

// half-face entries: side 0 of every face, side 1 of interior faces, keyed
// (element, face)
__global__ void half_entries_kernel(const int* __restrict__ f_e0, const int* __restrict__ f_e1, int nf, int nint,
                                    uint64_t* __restrict__ key, uint32_t* __restrict__ val, int* __restrict__ cnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nf + nint) return;
  const int f = i < nf ? i : i - nf, s = i < nf ? 0 : 1;
  const int e = s == 0 ? f_e0[f] : f_e1[f];
  key[i] = (uint64_t)e * (uint64_t)nf + (uint64_t)f;
  val[i] = (uint32_t)(2 * f + s);
  atomicAdd(&cnt[e], 1);
}

__global__ void half_lists_kernel(const uint32_t* __restrict__ sval, int nhf, int nf, int* __restrict__ hf_face,
                                  int8_t* __restrict__ hf_side, int* __restrict__ f_hf) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nhf) return;
  const int f = (int)(sval[k] >> 1), s = (int)(sval[k] & 1);
  hf_face[k] = f;
  hf_side[k] = (int8_t)s;
  f_hf[(size_t)s * nf + f] = k;
}

__global__ void face_points_kernel(int ne, int dim, const int* __restrict__ hf_ptr, const int* __restrict__ hf_face,
                                   const int* __restrict__ f_nq, int* __restrict__ hf_qoff, int* __restrict__ e_nqf) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  int acc = 0;
  for (int k = hf_ptr[e]; k < hf_ptr[e + 1]; ++k) {
    hf_qoff[k] = acc;
    const int nq = f_nq[hf_face[k]];
    acc += dim == 2 ? nq : nq * nq;
  }
  e_nqf[e] = acc;
}

__global__ void blk_rec_kernel(int nnzb, int nf, const int* __restrict__ brow, const int* __restrict__ col,
                               const int* __restrict__ blk_if, const int* __restrict__ if_e0,
                               const int* __restrict__ if_fptr, const int* __restrict__ f_hf, const int* __restrict__ p,
                               int4* __restrict__ rec) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nnzb) return;
  const int it = blk_if[b];
  if (it < 0) {
    rec[b] = make_int4(-1, 0, 0, 0);
    return;
  }
  const int e = brow[b], f0 = if_fptr[it];
  const int hf0 = f_hf[(size_t)(if_e0[it] == e ? 0 : 1) * nf + f0];
  rec[b] = make_int4(col[b], hf0, if_fptr[it + 1] - f0, p[col[b]]);
}

// work list keys: degree ascending, then cost descending (the sort is stable
// in element order)
__global__ void elem_key_kernel(int ne, int dim, const int* __restrict__ eptr, const int* __restrict__ p,
                                const int* __restrict__ e_nqf, uint64_t* __restrict__ key, uint32_t* __restrict__ val,
                                int* __restrict__ pcnt, int* __restrict__ nvq_out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  int qt = 1;
  for (int q = 0; q < dim; ++q) qt *= p[e] + 2;
  const int64_t nvq = (int64_t)(eptr[e + 1] - eptr[e]) * qt;
  const uint64_t cost = (uint64_t)(nvq + e_nqf[e]);
  key[e] = ((uint64_t)p[e] << 40) | ((1ull << 40) - 1 - cost);
  val[e] = (uint32_t)e;
  atomicAdd(&pcnt[p[e]], 1);
  nvq_out[e] = (int)nvq;
}

__global__ void iface_key_kernel(int ni, int dim, const int* __restrict__ if_e0, const int* __restrict__ if_e1,
                                 const int* __restrict__ if_fptr, const int* __restrict__ p, uint64_t* __restrict__ key,
                                 uint32_t* __restrict__ val, int* __restrict__ pcnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ni) return;
  const int pm = max(p[if_e0[i]], p[if_e1[i]]);
  const uint64_t np = (uint64_t)(if_fptr[i + 1] - if_fptr[i]) * (dim == 2 ? (pm + 1) : (pm + 1) * (pm + 1));
  key[i] = ((uint64_t)pm << 40) | ((1ull << 40) - 1 - np);
  val[i] = (uint32_t)i;
  atomicAdd(&pcnt[pm], 1);
}

__global__ void copy_u32_kernel(const uint32_t* __restrict__ in, int n, int* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (int)in[i];
}

// 3D: each element's distinct vertex ids, ascending (one warp per element;
// count pass, then fill pass)
__global__ void uverts_kernel(const int* __restrict__ eptr, const int* __restrict__ tet, int ne, int* __restrict__ cnt,
                              const int* __restrict__ uvptr, int* __restrict__ uvidx) {
  const int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (e >= ne) return;
  const int a = 4 * eptr[e], b = 4 * eptr[e + 1];
  // a vertex id is kept at its first occurrence in the element's list; its
  // rank among the kept ids (by value) is its position
  int kept = 0;
  for (int i = a + lane; i < b; i += 32) {
    const int v = tet[i];
    bool first = true;
    for (int j = a; j < i && first; ++j) first = tet[j] != v;
    if (!first) continue;
    if (!uvptr) {
      ++kept;
      continue;
    }
    int rank = 0;
    for (int j = a; j < b; ++j) {
      const int w = tet[j];
      if (w >= v) continue;
      bool fj = true;
      for (int k = a; k < j && fj; ++k) fj = tet[k] != w;
      rank += fj;
    }
    uvidx[uvptr[e] + rank] = v;
  }
  if (!uvptr) {
    for (int o = 16; o > 0; o >>= 1) kept += __shfl_xor_sync(0xffffffffu, kept, o);
    if (lane == 0) cnt[e] = kept;
  }
}

// Algorithmic work per launch group, the host's accounting (plan_mesh) in
// kernels: every term is an integer or a half integer, so the double
// atomics are exact and the sums do not depend on the order.  acc layout:
// flops [kKinds][9], words [kKinds][9], executed [2][9], interface terms by
// row and neighbour degree [2][9][9] (kAccN values).
constexpr int kAccW = kKinds * 9, kAccX = 2 * kKinds * 9, kAccO = kAccX + 18, kAccN = kAccO + 162;

__global__ void account_elem_kernel(int ne, int dim, bool adv, bool advb, const int* __restrict__ p,
                                    const int* __restrict__ nvq, const int* __restrict__ hf_ptr,
                                    const int* __restrict__ hf_face, const int* __restrict__ f_nq,
                                    const int* __restrict__ f_e1, const int* __restrict__ nsub_e,
                                    const double* __restrict__ tabs /* pt, map, fpt, bnd, mapf [9] */,
                                    double* __restrict__ acc) {
  // per-CTA sums in shared memory, then one global add per bin: the values
  // are integers or halves, exact in double, so the order of the adds does
  // not change the result
  __shared__ double sacc[kAccN];
  for (int t = threadIdx.x; t < kAccN; t += blockDim.x) sacc[t] = 0.0;
  __syncthreads();
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < ne) {
    const int SV = sub_vals(dim), FV = side_vals(dim);
    const int pe = p[e];
    const double n = nbasis(dim, pe);
    const double basis = n * dim * dim + 5.0 * dim * pe;
    const double nv = nvq[e];
    const double vol_direct = nv * (dim * n * (n + 1) / 2 + (adv ? n * n + n * (dim + 1) : 0.0) + basis + n);
    double fma = vol_direct;
    const double vol_words = n * n + n + (double)nsub_e[e] * SV + 2 * dim + 2;
    double w = vol_words, nfq = 0.0, nbq = 0.0;
    for (int k = hf_ptr[e]; k < hf_ptr[e + 1]; ++k) {
      const int f = hf_face[k];
      const double qf = dim == 2 ? f_nq[f] : (double)f_nq[f] * f_nq[f];
      const bool bnd = f_e1[f] < 0;
      fma += qf * (3 * n * n + (advb ? (bnd ? n * n : n * n / 2) : 0.0) + basis + (bnd ? 2 * n : 0.0));
      w += FV + 3;
      nfq += qf;
      if (bnd) nbq += qf;
    }
    atomicAdd(&sacc[0 * 9 + pe], 2.0 * fma);
    atomicAdd(&sacc[kAccW + 0 * 9 + pe], w);
    // the moment path's launches: volume to kind 2, the rest to kind 1; with
    // the own faces, the element's terms to kind 3
    atomicAdd(&sacc[1 * 9 + pe], 2.0 * (fma - vol_direct));
    atomicAdd(&sacc[kAccW + 1 * 9 + pe], w - vol_words);
    atomicAdd(&sacc[2 * 9 + pe], 2.0 * vol_direct);
    atomicAdd(&sacc[kAccW + 2 * 9 + pe], vol_words);
    atomicAdd(&sacc[3 * 9 + pe], 2.0 * fma);
    atomicAdd(&sacc[kAccW + 3 * 9 + pe], w);
    const double vx = nv * tabs[pe] + tabs[9 + pe];
    atomicAdd(&sacc[kAccX + pe], 2.0 * vx);
    atomicAdd(&sacc[kAccX + 9 + pe], 2.0 * (vx + nfq * tabs[18 + pe] + nbq * tabs[27 + pe] + tabs[36 + pe]));
  }
  __syncthreads();
  for (int t = threadIdx.x; t < kAccN; t += blockDim.x)
    if (sacc[t] != 0.0) atomicAdd(&acc[t], sacc[t]);
}

__global__ void account_iface_kernel(int ni, int dim, bool advb, const int* __restrict__ if_e0,
                                     const int* __restrict__ if_e1, const int* __restrict__ if_fptr,
                                     const int* __restrict__ f_nq, const int* __restrict__ p, double* __restrict__ acc) {
  __shared__ double sacc[kAccN];  // per-CTA sums, as in account_elem_kernel
  for (int t = threadIdx.x; t < kAccN; t += blockDim.x) sacc[t] = 0.0;
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < ni) {
    const int FV = side_vals(dim);
    for (int side = 0; side < 2; ++side) {
      const int e = side == 0 ? if_e0[i] : if_e1[i], k = side == 0 ? if_e1[i] : if_e0[i];
      const double ne_ = nbasis(dim, p[e]), nk = nbasis(dim, p[k]);
      double fma = 0.0, w = ne_ * nk;
      for (int f = if_fptr[i]; f < if_fptr[i + 1]; ++f) {
        const double qf = dim == 2 ? f_nq[f] : (double)f_nq[f] * f_nq[f];
        fma += qf * (3 * ne_ * nk + (advb ? ne_ * nk / 2 : 0.0));
        w += 2 * FV + 3;
      }
      atomicAdd(&sacc[0 * 9 + p[e]], 2.0 * fma);
      atomicAdd(&sacc[kAccW + 0 * 9 + p[e]], w);
      atomicAdd(&sacc[1 * 9 + p[e]], 2.0 * fma);
      atomicAdd(&sacc[kAccW + 1 * 9 + p[e]], w);
      atomicAdd(&sacc[kAccO + p[e] * 9 + p[k]], 2.0 * fma);
      atomicAdd(&sacc[kAccO + 81 + p[e] * 9 + p[k]], w);
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < kAccN; t += blockDim.x)
    if (sacc[t] != 0.0) atomicAdd(&acc[t], sacc[t]);
}

__global__ void nsub_kernel(const int* __restrict__ eptr, int ne, int* __restrict__ out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < ne) out[e] = eptr[e + 1] - eptr[e];
}

// element of each 3D half face: that of its tetrahedron
__global__ void expand4_kernel(const int* __restrict__ sub_elem, int nh, int* __restrict__ helem) {
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h < nh) helem[h] = sub_elem[h >> 2];
}

}  // namespace

// Build the pattern of desc on the device.  Inputs are the uploaded
// element lists, degrees and coordinates; alloc provides the device arrays
// that the mesh keeps; everything else is freed before the return.  The
// counts, the degree-group offsets, the host copies of the block layout and
// the accounting come back to the host.  Returns DG_OK, DG_ERR_MESH (with
// *msg) for an invalid mesh, DG_ERR_CUDA / DG_ERR_OOM on a failed call.
int build_pattern_device(const dg_mesh_desc* d, const int* eptr, const int* eidx, const int* p, const double* const* X,
                         const std::function<void*(size_t)>& alloc, cudaStream_t st, DevPattern* P, std::string* msg) {
  const int dim = d->dim, nv = d->nv, ne = d->ne;
  const int nsub = d->elem_ptr[ne];
  std::vector<void*> scratch;
  bool oom = false;
  auto tmp = [&](size_t bytes) {
    void* q = nullptr;
    if (cudaMalloc(&q, std::max<size_t>(bytes, 16)) != cudaSuccess) {
      oom = true;
      return (void*)nullptr;
    }
    scratch.push_back(q);
    return q;
  };
  auto keep = [&](size_t bytes) {
    void* q = alloc(std::max<size_t>(bytes, 16));
    if (!q) oom = true;
    return q;
  };
  auto fin = [&](int rc) {
    cudaStreamSynchronize(st);
    for (void* q : scratch) cudaFree(q);
    return rc;
  };
  auto bad = [&]() -> int {
    if (oom) return fin(DG_ERR_OOM);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      *msg = std::string("device pattern build: ") + cudaGetErrorString(e);
      return fin(DG_ERR_CUDA);
    }
    return DG_OK;
  };
  int* err = (int*)tmp(sizeof(int) * 2);  // [0] error bits, [1] interior faces
  if (oom) return fin(DG_ERR_OOM);
  cudaMemsetAsync(err, 0, sizeof(int) * 2, st);

  // ---- sub-simplex -> element, validity
  P->sub_elem = (int*)keep(sizeof(int) * (size_t)nsub);
  if (int rc = bad()) return rc;
  sub_elem_kernel<<<nblk(ne), kT, 0, st>>>(eptr, ne, P->sub_elem);
  if (dim == 2) validity2d_kernel<<<nblk(ne), kT, 0, st>>>(X[0], X[1], eptr, eidx, ne, err);

  // ---- half faces, sorted by key (stable: element order within a key)
  const int nh = dim == 2 ? nsub : 4 * nsub;
  uint64_t* hk = (uint64_t*)tmp(sizeof(uint64_t) * (size_t)nh);
  uint32_t* hvv = (uint32_t*)tmp(sizeof(uint32_t) * (size_t)nh);
  uint64_t* tk = (uint64_t*)tmp(sizeof(uint64_t) * (size_t)nh);
  uint32_t* tvv = (uint32_t*)tmp(sizeof(uint32_t) * (size_t)nh);
  int* hvert = (int*)tmp(sizeof(int) * 3 * (size_t)nh);
  int* helem = (int*)tmp(sizeof(int) * (size_t)nh);
  int8_t* hflip = dim == 3 ? (int8_t*)tmp((size_t)nh) : nullptr;
  if (int rc = bad()) return rc;
  uint64_t maxkey;
  if (dim == 2) {
    half2d_kernel<<<nblk(nh), kT, 0, st>>>(eptr, eidx, P->sub_elem, nh, nv, hk, hvv, hvert, err);
    cudaMemcpyAsync(helem, P->sub_elem, sizeof(int) * (size_t)nh, cudaMemcpyDeviceToDevice, st);
    maxkey = (uint64_t)nv * nv;
  } else {
    half3d_kernel<<<nblk(nh), kT, 0, st>>>(X[0], X[1], X[2], eidx, nsub, nv, hk, hvv, hvert, hflip, err);
    expand4_kernel<<<nblk(nh), kT, 0, st>>>(P->sub_elem, nh, helem);
    maxkey = (uint64_t)nv * nv * nv;
  }
  radix_sort(hk, hvv, tk, tvv, nh, bits_for(maxkey), st, scratch);

  // ---- matching: faces in key order
  int* emit = (int*)tmp(sizeof(int) * ((size_t)nh + 1));
  int* fpos = (int*)tmp(sizeof(int) * ((size_t)nh + 1));
  if (int rc = bad()) return rc;
  match_kernel<<<nblk(nh), kT, 0, st>>>(hk, hvv, nh, helem, dim, emit, err);
  scan_exclusive<int>(emit, fpos, nh, st, scratch);
  int hcnt[2] = {0, 0};
  cudaMemcpyAsync(&hcnt[0], fpos + nh, sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(&hcnt[1], err, sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  if (int rc = bad()) return rc;
  const int nf = hcnt[0];
  if (hcnt[1] & (kErrRepeat | kErrManifold | kErrTwice | kErrArea | kErrVolume)) {
    const int e = hcnt[1];
    *msg = (e & kErrRepeat)     ? "a loop repeats a vertex"
           : (e & kErrManifold) ? "a face is shared by more than two element pieces (non-manifold)"
           : (e & kErrTwice)    ? "an element traverses an edge twice"
           : (e & kErrArea)     ? "a loop is not counter-clockwise or has a fan triangle of non-positive area"
                                : "a tetrahedron has zero volume";
    return fin(DG_ERR_MESH);
  }
  int* fe0 = (int*)tmp(sizeof(int) * (size_t)nf);
  int* fe1 = (int*)tmp(sizeof(int) * (size_t)nf);
  int* fvv = (int*)tmp(sizeof(int) * (size_t)dim * nf);
  int8_t* ffl = (int8_t*)tmp((size_t)nf);
  uint64_t* fk = (uint64_t*)tmp(sizeof(uint64_t) * (size_t)nf);
  uint32_t* fid = (uint32_t*)tmp(sizeof(uint32_t) * (size_t)nf);
  uint64_t* fk2 = (uint64_t*)tmp(sizeof(uint64_t) * (size_t)nf);
  uint32_t* fid2 = (uint32_t*)tmp(sizeof(uint32_t) * (size_t)nf);
  if (int rc = bad()) return rc;
  emit_kernel<<<nblk(nh), kT, 0, st>>>(hk, hvv, nh, emit, fpos, helem, hvert, hflip, dim, ne, fe0, fe1, fvv, ffl, fk,
                                       fid, err + 1, err);
  // ---- faces by (boundary, e0, e1), stable
  radix_sort(fk, fid, fk2, fid2, nf, bits_for(2ull * ((uint64_t)ne + 1) * ((uint64_t)ne + 1)), st, scratch);
  P->f_e0 = (int*)keep(sizeof(int) * (size_t)nf);
  P->f_e1 = (int*)keep(sizeof(int) * (size_t)nf);
  P->f_v = (int*)keep(sizeof(int) * (size_t)dim * nf);
  P->f_flip = (int8_t*)keep((size_t)nf);
  P->f_nq = (int*)keep(sizeof(int) * (size_t)nf);
  if (int rc = bad()) return rc;
  face_order_kernel<<<nblk(nf), kT, 0, st>>>(fid, nf, dim, fe0, fe1, fvv, ffl, p, P->f_e0, P->f_e1, P->f_v, P->f_flip,
                                             P->f_nq);
  cudaMemcpyAsync(&hcnt[0], err + 1, sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(&hcnt[1], err, sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  if (int rc = bad()) return rc;
  const int nint = hcnt[0];
  if (hcnt[1] & kErrOrient) {
    *msg = "two neighbouring loops traverse their common edge in the same direction";
    return fin(DG_ERR_MESH);
  }

  // ---- interfaces
  int* head = (int*)tmp(sizeof(int) * ((size_t)nint + 1));
  int* ipos = (int*)tmp(sizeof(int) * ((size_t)nint + 1));
  if (int rc = bad()) return rc;
  if (nint > 0) iface_head_kernel<<<nblk(nint), kT, 0, st>>>(P->f_e0, P->f_e1, nint, head);
  scan_exclusive<int>(head, ipos, nint, st, scratch);
  int ni = 0;
  cudaMemcpyAsync(&ni, ipos + nint, sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  P->if_e0 = (int*)keep(sizeof(int) * (size_t)ni);
  P->if_e1 = (int*)keep(sizeof(int) * (size_t)ni);
  P->if_fptr = (int*)keep(sizeof(int) * ((size_t)ni + 1));
  int* c0 = (int*)tmp(sizeof(int) * (size_t)ne);
  int* c1 = (int*)tmp(sizeof(int) * (size_t)ne);
  int* first0 = (int*)tmp(sizeof(int) * (size_t)ne);
  int* first1 = (int*)tmp(sizeof(int) * ((size_t)ne + 1));
  uint64_t* k1 = (uint64_t*)tmp(sizeof(uint64_t) * (size_t)ni);
  uint32_t* v1 = (uint32_t*)tmp(sizeof(uint32_t) * (size_t)ni);
  uint64_t* k1b = (uint64_t*)tmp(sizeof(uint64_t) * (size_t)ni);
  uint32_t* v1b = (uint32_t*)tmp(sizeof(uint32_t) * (size_t)ni);
  if (int rc = bad()) return rc;
  cudaMemsetAsync(c0, 0, sizeof(int) * (size_t)ne, st);
  cudaMemsetAsync(c1, 0, sizeof(int) * (size_t)ne, st);
  iface_kernel<<<nblk(std::max(nint, 1)), kT, 0, st>>>(P->f_e0, P->f_e1, nint, head, ipos, ni, P->if_e0, P->if_e1,
                                                        P->if_fptr, c0, c1, first0, k1, v1);
  // interfaces by e1, stable (ascending e0 within an element)
  radix_sort(k1, v1, k1b, v1b, ni, bits_for((uint64_t)ne), st, scratch);
  scan_exclusive<int>(c1, first1, ne, st, scratch);

  // ---- block rows
  int* rc_ = (int*)tmp(sizeof(int) * (size_t)ne);
  P->row_ptr = (int*)keep(sizeof(int) * ((size_t)ne + 1));
  if (int rc = bad()) return rc;
  row_count_kernel<<<nblk(ne), kT, 0, st>>>(c0, c1, ne, rc_);
  scan_exclusive<int>(rc_, P->row_ptr, ne, st, scratch);
  const int nnzb = ne + 2 * ni;
  P->col = (int*)keep(sizeof(int) * (size_t)nnzb);
  P->blk_if = (int*)keep(sizeof(int) * (size_t)nnzb);
  P->diag_blk = (int*)keep(sizeof(int) * (size_t)ne);
  P->slot01 = (int*)keep(sizeof(int) * (size_t)ni);
  P->slot10 = (int*)keep(sizeof(int) * (size_t)ni);
  P->blk_off = (int64_t*)keep(sizeof(int64_t) * ((size_t)nnzb + 1));
  P->dof_off = (int64_t*)keep(sizeof(int64_t) * ((size_t)ne + 1));
  int64_t* bsz = (int64_t*)tmp(sizeof(int64_t) * (size_t)nnzb);
  int* brow = (int*)tmp(sizeof(int) * (size_t)nnzb);
  int* nb = (int*)tmp(sizeof(int) * (size_t)ne);
  int64_t* nb64 = (int64_t*)tmp(sizeof(int64_t) * (size_t)ne);
  if (int rc = bad()) return rc;
  nbasis_kernel<<<nblk(ne), kT, 0, st>>>(p, ne, dim, nb, nb64);
  rows_kernel<<<nblk(ne), kT, 0, st>>>(ne, P->row_ptr, c0, c1, first0, first1, v1, P->if_e0, P->if_e1, nb, P->col,
                                       P->blk_if, P->diag_blk, P->slot01, P->slot10, bsz, brow);
  scan_exclusive<int64_t>(bsz, P->blk_off, nnzb, st, scratch);
  scan_exclusive<int64_t>(nb64, P->dof_off, ne, st, scratch);

  // ---- half faces of each element, in face order
  const int nhf = nf + nint;
  uint64_t* ek = (uint64_t*)tmp(sizeof(uint64_t) * (size_t)nhf);
  uint32_t* ev = (uint32_t*)tmp(sizeof(uint32_t) * (size_t)nhf);
  uint64_t* ek2 = (uint64_t*)tmp(sizeof(uint64_t) * (size_t)nhf);
  uint32_t* ev2 = (uint32_t*)tmp(sizeof(uint32_t) * (size_t)nhf);
  int* hcnt_e = (int*)tmp(sizeof(int) * (size_t)ne);
  P->hf_ptr = (int*)keep(sizeof(int) * ((size_t)ne + 1));
  P->hf_face = (int*)keep(sizeof(int) * (size_t)nhf);
  P->hf_side = (int8_t*)keep((size_t)nhf);
  P->hf_qoff = (int*)keep(sizeof(int) * (size_t)nhf);
  P->e_nqf = (int*)keep(sizeof(int) * (size_t)ne);
  P->f_hf = (int*)keep(sizeof(int) * 2 * (size_t)nf);
  if (int rc = bad()) return rc;
  cudaMemsetAsync(hcnt_e, 0, sizeof(int) * (size_t)ne, st);
  cudaMemsetAsync(P->f_hf, 0xff, sizeof(int) * 2 * (size_t)nf, st);
  half_entries_kernel<<<nblk(nhf), kT, 0, st>>>(P->f_e0, P->f_e1, nf, nint, ek, ev, hcnt_e);
  radix_sort(ek, ev, ek2, ev2, nhf, bits_for((uint64_t)ne * nf), st, scratch);
  scan_exclusive<int>(hcnt_e, P->hf_ptr, ne, st, scratch);
  half_lists_kernel<<<nblk(nhf), kT, 0, st>>>(ev, nhf, nf, P->hf_face, P->hf_side, P->f_hf);
  face_points_kernel<<<nblk(ne), kT, 0, st>>>(ne, dim, P->hf_ptr, P->hf_face, P->f_nq, P->hf_qoff, P->e_nqf);
  P->blk_rec = (int4*)keep(sizeof(int4) * (size_t)nnzb);
  if (int rc = bad()) return rc;
  blk_rec_kernel<<<nblk(nnzb), kT, 0, st>>>(nnzb, nf, brow, P->col, P->blk_if, P->if_e0, P->if_fptr, P->f_hf, p,
                                            P->blk_rec);

  // ---- unique vertices per element
  if (dim == 2) {
    P->uvptr = eptr;
    P->uvidx = eidx;
  } else {
    int* ucnt = (int*)tmp(sizeof(int) * (size_t)ne);
    int* uptr = (int*)keep(sizeof(int) * ((size_t)ne + 1));
    if (int rc = bad()) return rc;
    uverts_kernel<<<nblk((int64_t)ne * 32), kT, 0, st>>>(eptr, eidx, ne, ucnt, nullptr, nullptr);
    scan_exclusive<int>(ucnt, uptr, ne, st, scratch);
    int nu = 0;
    cudaMemcpyAsync(&nu, uptr + ne, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    int* uidx = (int*)keep(sizeof(int) * (size_t)nu);
    if (int rc = bad()) return rc;
    uverts_kernel<<<nblk((int64_t)ne * 32), kT, 0, st>>>(eptr, eidx, ne, ucnt, uptr, uidx);
    P->uvptr = uptr;
    P->uvidx = uidx;
  }

  // ---- work lists
  uint64_t* wk = (uint64_t*)tmp(sizeof(uint64_t) * (size_t)std::max(ne, ni));
  uint32_t* wv = (uint32_t*)tmp(sizeof(uint32_t) * (size_t)std::max(ne, ni));
  uint64_t* wk2 = (uint64_t*)tmp(sizeof(uint64_t) * (size_t)std::max(ne, ni));
  uint32_t* wv2 = (uint32_t*)tmp(sizeof(uint32_t) * (size_t)std::max(ne, ni));
  int* pcnt = (int*)tmp(sizeof(int) * 18);
  int* nvq = (int*)tmp(sizeof(int) * (size_t)ne);
  P->elem_perm = (int*)keep(sizeof(int) * (size_t)ne);
  P->if_perm = (int*)keep(sizeof(int) * (size_t)std::max(ni, 1));
  if (int rc = bad()) return rc;
  cudaMemsetAsync(pcnt, 0, sizeof(int) * 18, st);
  elem_key_kernel<<<nblk(ne), kT, 0, st>>>(ne, dim, eptr, p, P->e_nqf, wk, wv, pcnt, nvq);
  radix_sort(wk, wv, wk2, wv2, ne, 44, st, scratch);
  copy_u32_kernel<<<nblk(ne), kT, 0, st>>>(wv, ne, P->elem_perm);
  if (ni > 0) {
    iface_key_kernel<<<nblk(ni), kT, 0, st>>>(ni, dim, P->if_e0, P->if_e1, P->if_fptr, p, wk, wv, pcnt + 9);
    radix_sort(wk, wv, wk2, wv2, ni, 44, st, scratch);
    copy_u32_kernel<<<nblk(ni), kT, 0, st>>>(wv, ni, P->if_perm);
  }

  // ---- accounting (the host's formulas)
  double* acc = (double*)tmp(sizeof(double) * kAccN);
  double* tabs = (double*)tmp(sizeof(double) * 45);
  int* nsub_e = (int*)tmp(sizeof(int) * (size_t)ne);
  if (int rc = bad()) return rc;
  {
    MomentOps ops;
    moment_op_tables(dim, ops);
    double h[45];
    for (int i = 0; i < 9; ++i) {
      h[i] = ops.pt[i];
      h[9 + i] = ops.map[i];
      h[18 + i] = ops.fpt[i];
      h[27 + i] = ops.bnd[i];
      h[36 + i] = ops.mapf[i];
      P->mom_pt[i] = 2.0 * ops.pt[i];
    }
    cudaMemcpyAsync(tabs, h, sizeof h, cudaMemcpyHostToDevice, st);
    cudaMemsetAsync(acc, 0, sizeof(double) * kAccN, st);
    const bool advb = d->b[0] != 0.0 || d->b[1] != 0.0 || (dim == 3 && d->b[2] != 0.0);
    const bool adv = advb || d->c != 0.0;
    nsub_kernel<<<nblk(ne), kT, 0, st>>>(eptr, ne, nsub_e);
    account_elem_kernel<<<nblk(ne), kT, 0, st>>>(ne, dim, adv, advb, p, nvq, P->hf_ptr, P->hf_face, P->f_nq,
                                                 P->f_e1, nsub_e, tabs, acc);
    if (ni > 0)
      account_iface_kernel<<<nblk(ni), kT, 0, st>>>(ni, dim, advb, P->if_e0, P->if_e1, P->if_fptr, P->f_nq, p, acc);
    double hacc[kAccN];
    int hp[18];
    cudaMemcpyAsync(hacc, acc, sizeof hacc, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(hp, pcnt, sizeof hp, cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    for (int k = 0; k < kKinds; ++k)
      for (int q = 0; q < 9; ++q) {
        P->flops[k][q] = hacc[k * 9 + q];
        P->words[k][q] = hacc[kAccW + k * 9 + q];
      }
    for (int k = 0; k < 2; ++k)
      for (int q = 0; q < 9; ++q) P->mom_exec[k][q] = hacc[kAccX + k * 9 + q];
    for (int k = 0; k < 2; ++k)
      for (int q = 0; q < 9; ++q)
        for (int r = 0; r < 9; ++r) P->offd[k][q][r] = hacc[kAccO + k * 81 + q * 9 + r];
    P->elem_pstart[0] = P->if_pstart[0] = 0;
    for (int q = 0; q < 8; ++q) {
      P->elem_pstart[q + 1] = P->elem_pstart[q] + hp[q];
      P->if_pstart[q + 1] = P->if_pstart[q] + hp[9 + q];
    }
  }
  // host copies of the layout, the per-element counts the host keeps
  P->h_row_ptr.resize((size_t)ne + 1);
  P->h_col.resize((size_t)nnzb);
  P->h_blk_off.resize((size_t)nnzb + 1);
  P->h_dof_off.resize((size_t)ne + 1);
  P->h_e_nqf.resize((size_t)ne);
  P->h_nvq.resize((size_t)ne);
  P->h_perm.resize((size_t)ne);
  cudaMemcpyAsync(P->h_row_ptr.data(), P->row_ptr, sizeof(int) * ((size_t)ne + 1), cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(P->h_col.data(), P->col, sizeof(int) * (size_t)nnzb, cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(P->h_blk_off.data(), P->blk_off, sizeof(int64_t) * ((size_t)nnzb + 1), cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(P->h_dof_off.data(), P->dof_off, sizeof(int64_t) * ((size_t)ne + 1), cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(P->h_e_nqf.data(), P->e_nqf, sizeof(int) * (size_t)ne, cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(P->h_nvq.data(), nvq, sizeof(int) * (size_t)ne, cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(P->h_perm.data(), P->elem_perm, sizeof(int) * (size_t)ne, cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  if (int rc = bad()) return rc;
  P->nsub = nsub;
  P->nf = nf;
  P->nint = nint;
  P->ni = ni;
  P->nhf = nhf;
  P->nnzb = nnzb;
  P->nvals = P->h_blk_off[nnzb];
  P->ndofs = P->h_dof_off[ne];
  int64_t nqv = 0, nqf = 0;
  for (int e = 0; e < ne; ++e) nqv += P->h_nvq[e];
  {
    // face points, interior faces counted once: sum over faces of nq (2D) or nq^2
    std::vector<int> fnq((size_t)nf);
    cudaMemcpy(fnq.data(), P->f_nq, sizeof(int) * (size_t)nf, cudaMemcpyDeviceToHost);
    for (int f = 0; f < nf; ++f) nqf += dim == 2 ? fnq[f] : (int64_t)fnq[f] * fnq[f];
  }
  P->nqvol = nqv;
  P->nqface = nqf;
  return fin(DG_OK);
}

namespace {
__global__ void iface_rec_kernel(int ni, const int* __restrict__ if_perm, const int* __restrict__ if_e0,
                                 const int* __restrict__ if_e1, const int* __restrict__ if_fptr,
                                 const int* __restrict__ f_hf, const int* __restrict__ s01, const int* __restrict__ s10,
                                 const int* __restrict__ p, int4* __restrict__ rec) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= ni) return;
  const int i = if_perm[k], e0 = if_e0[i], e1 = if_e1[i], f0 = if_fptr[i];
  rec[2 * k] = make_int4(e0, e1, f_hf[f0], if_fptr[i + 1] - f0);
  rec[2 * k + 1] = make_int4(s01[i], s10[i], p[e0] | (p[e1] << 8), 0);
}
}  // namespace

void launch_iface_recs(const DevMesh& dm, int4* rec, cudaStream_t st) {
  if (dm.ni <= 0) return;
  iface_rec_kernel<<<(dm.ni + 255) / 256, 256, 0, st>>>(dm.ni, dm.if_perm, dm.if_e0, dm.if_e1, dm.if_fptr, dm.f_hf,
                                                       dm.if_slot01, dm.if_slot10, dm.p, rec);
}

}  // namespace dg
