// dg_slab.cuh -- index arithmetic of the space-time prism basis (Sec. 2.3),
// shared by the host layout code (dg_host.cu) and the slab kernels
// (dg_slab.cu).  A prism of degree p carries T_k(t) phi_j(x), dofs k-major:
// space 0 (P_p) k = 0..p with j < nbasis(dim, p - k); space 1 (PQ_p)
// k = 0..p with j < nbasis(dim, p).
#pragma once

#include <cmath>

#include "dg_internal.h"

namespace dg {

constexpr int kSlabKMax = 8;  // temporal degrees 0..7 (spatial degrees <= kPMax2 = 6)

// spatial functions carried by temporal degree k
__host__ __device__ inline int slab_nspace(int dim, int p, int space, int k) {
  return nbasis(dim, space == 1 ? p : p - k);
}

// first dof of temporal degree k
__host__ __device__ inline int slab_start(int dim, int p, int space, int k) {
  if (space == 1) return k * nbasis(dim, p);
  int s = 0;
  for (int q = 0; q < k; ++q) s += nbasis(dim, p - q);
  return s;
}

// dofs of a prism of degree p
__host__ __device__ inline int slab_count(int dim, int p, int space) { return slab_start(dim, p, space, p + 1); }

// dof i (0 <= i < slab_count) -> (k, j)
__host__ __device__ inline void slab_decode(int dim, int p, int space, int i, int& k, int& j) {
  if (space == 1) {
    const int n = nbasis(dim, p);
    k = i / n;
    j = i - k * n;
    return;
  }
  k = 0;
  while (k < p && i >= nbasis(dim, p - k)) {
    i -= nbasis(dim, p - k);
    ++k;
  }
  j = i;
}

// Time data of one slab in the kernels' type: D[k][l] = int T_l' T_k dt +
// T_l(t0+) T_k(t0+), the values T_k(t0+) and T_k(t1-), and sqrt(tau) =
// int T_0 dt.
template <typename T>
struct SlabTimes {
  T D[kSlabKMax][kSlabKMax];
  T at0[kSlabKMax];
  T at1[kSlabKMax];
  T sqrt_tau;
};

// Time data of (t0, t1] (host): with T_k = sqrt((2k+1)/tau) P_k(2 (t - t0)/tau - 1),
// int_{-1}^{1} P_l' P_k = 2 for k < l with k + l odd (else 0), P_k(-1) = (-1)^k
// and P_k(1) = 1.
inline SlabTimes<double> slab_time_data(double t0, double t1) {
  SlabTimes<double> tt{};
  const double tau = t1 - t0;
  for (int k = 0; k < kSlabKMax; ++k) {
    for (int l = 0; l < kSlabKMax; ++l) {
      const bool odd = ((k + l) & 1) != 0;
      const double deriv = k < l && odd ? 2.0 : 0.0;
      const double jump = odd ? -1.0 : 1.0;
      tt.D[k][l] = std::sqrt((double)((2 * k + 1) * (2 * l + 1))) / tau * (deriv + jump);
    }
    const double s = std::sqrt((2.0 * k + 1.0) / tau);
    tt.at0[k] = (k & 1) ? -s : s;
    tt.at1[k] = s;
  }
  tt.sqrt_tau = std::sqrt(tau);
  return tt;
}

// Decode tables of every degree's prism dofs: kj[off[p] + i] = (k << 8) | j
// for dof i of a prism of degree p, i < slab_count(p) (the expansion takes
// both indices of an entry from two table reads instead of a division and a
// loop).  2D PQ_6 needs 196 entries; all degrees of either dimension and
// space fit in kSlabDecMax.
constexpr int kSlabDecMax = 512;
struct SlabDecode {
  unsigned short kj[kSlabDecMax];
  int off[kSlabKMax + 1];
};

// fill the decode tables for degrees 1..pmax (entries [off[p], off[p+1]))
__host__ __device__ inline void slab_decode_tables(int dim, int space, int pmax, SlabDecode& t, int tid, int nthreads) {
  int o = 0;
  for (int p = 0; p <= pmax && p < kSlabKMax; ++p) {
    t.off[p] = o;
    o += p == 0 ? 0 : slab_count(dim, p, space);
  }
  for (int p = pmax + 1; p <= kSlabKMax; ++p) t.off[p] = o;
  for (int p = 1; p <= pmax && p < kSlabKMax; ++p) {
    const int n = slab_count(dim, p, space);
    for (int i = tid; i < n; i += nthreads) {
      int k, j;
      slab_decode(dim, p, space, i, k, j);
      t.kj[t.off[p] + i] = (unsigned short)((k << 8) | j);
    }
  }
}

// The block pattern and spatial offsets the slab kernels read (device pointers).
struct SlabPattern {
  int dim, ne, space;
  const int* p;             // [ne]
  const int* row_ptr;       // [ne+1]
  const int* col;           // [nnzb]
  const int* diag_blk;      // [ne]
  const int64_t* blk_off;   // [nnzb+1] spatial blocks
  const int64_t* dof_off;   // [ne+1] spatial dofs
  const int64_t* sblk_off;  // [nnzb+1] slab blocks
  const int64_t* sdof_off;  // [ne+1] slab dofs
  // [ne] rows by degree, ascending (the mesh's work list); the expansion's
  // warps take them from the end, the largest rows first, so that the rows
  // of many sizes share out evenly over the grid-strided warps
  const int* order;
};

// The work of one element row r, shared out over `lanes` threads of which
// this is `lane` (a warp in the kernels).  Plain loads and stores, no
// synchronisation between the lanes.

// slab blocks of row r: [k = l] B[j, m] + [r = s] D_kl M[j, m].  Entry x
// of a block sits at row i = x / nts, column q = x % nts; a lane steps x by
// lanes, so (i, q) advance by (lanes / nts, lanes % nts) with one carry, and
// (k, j), (l, m) come from the decode tables.  D: the time matrix, [k][l]
// with stride kSlabKMax.  Stores are contiguous over the lanes.  A lane
// takes four of its entries per round: their indices first, then their four
// loads, then their four stores, so that four loads are in flight at once.
template <typename T>
__host__ __device__ inline void slab_matrix_row(const SlabPattern& sp, const T* __restrict__ D, const SlabDecode& dec,
                                                const T* __restrict__ B, const T* __restrict__ M,
                                                T* __restrict__ vals, int r, int lane, int lanes) {
  const int pr = sp.p[r];
  const int ntr = slab_count(sp.dim, pr, sp.space);
  const unsigned short* dr = dec.kj + dec.off[pr];
  for (int b = sp.row_ptr[r]; b < sp.row_ptr[r + 1]; ++b) {
    const int s = sp.col[b];
    const int ps = sp.p[s];
    const int nbs = nbasis(sp.dim, ps);
    const int nts = slab_count(sp.dim, ps, sp.space);
    const unsigned short* ds = dec.kj + dec.off[ps];
    const T* Bb = B + sp.blk_off[b];
    const T* Mb = M + sp.blk_off[b];  // the mass matrix sits in the diagonal blocks' places
    T* out = vals + sp.sblk_off[b];
    const bool diag = s == r;
    const int n = ntr * nts;
    const int si = lanes / nts, sq = lanes - si * nts;
    int i = lane / nts, q = lane - (lane / nts) * nts;
    int x = lane;
    for (; x + 3 * lanes < n; x += 4 * lanes) {
      int at[4], kl[4];
      bool same[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int kj = dr[i], lm = ds[q];
        const int k = kj >> 8, l = lm >> 8;
        at[u] = (kj & 255) * nbs + (lm & 255);
        kl[u] = k * kSlabKMax + l;
        same[u] = k == l;
        i += si;
        q += sq;
        if (q >= nts) {
          q -= nts;
          ++i;
        }
      }
      T v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = same[u] ? Bb[at[u]] : T(0);
      if (diag) {
        T w[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) w[u] = Mb[at[u]];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] += D[kl[u]] * w[u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) out[x + u * lanes] = v[u];
    }
    for (; x < n; x += lanes) {
      const int kj = dr[i], lm = ds[q];
      const int k = kj >> 8, j = kj & 255, l = lm >> 8, m = lm & 255;
      const int at = j * nbs + m;
      T v = k == l ? Bb[at] : T(0);
      if (diag) v += D[k * kSlabKMax + l] * Mb[at];
      out[x] = v;
      i += si;
      q += sq;
      if (q >= nts) {
        q -= nts;
        ++i;
      }
    }
  }
}

// load vector of row r: [k = 0] sqrt(tau) l_j + T_k(t0+) (M u_prev)_j
template <typename T>
__host__ __device__ inline void slab_rhs_row(const SlabPattern& sp, const SlabTimes<T>& tt, const T* l, const T* M,
                                             const T* u_prev, T* rhs, int r, int lane, int lanes) {
  const int pr = sp.p[r];
  const int nbr = nbasis(sp.dim, pr);
  const int ntr = slab_count(sp.dim, pr, sp.space);
  const int64_t d0 = sp.dof_off[r];
  const T* Mr = M + sp.blk_off[sp.diag_blk[r]];
  T* out = rhs + sp.sdof_off[r];
  for (int i = lane; i < ntr; i += lanes) {
    int k, j;
    slab_decode(sp.dim, pr, sp.space, i, k, j);
    T v = k == 0 ? tt.sqrt_tau * l[d0 + j] : T(0);
    if (u_prev) {
      T acc = T(0);
      for (int m = 0; m < nbr; ++m) acc += Mr[j * nbr + m] * u_prev[d0 + m];
      v += tt.at0[k] * acc;
    }
    out[i] = v;
  }
}

// trace of row r at t1-: sum_k U(k, j) T_k(t1-) over the k that carry j
template <typename T>
__host__ __device__ inline void slab_trace_row(const SlabPattern& sp, const SlabTimes<T>& tt, const T* U, T* u_end,
                                               int r, int lane, int lanes) {
  const int pr = sp.p[r];
  const int nbr = nbasis(sp.dim, pr);
  const T* Ur = U + sp.sdof_off[r];
  T* out = u_end + sp.dof_off[r];
  for (int j = lane; j < nbr; j += lanes) {
    T acc = T(0);
    for (int k = 0; k <= pr; ++k) {
      if (j >= slab_nspace(sp.dim, pr, sp.space, k)) break;  // P: degree p - k falls below j's
      acc += tt.at1[k] * Ur[slab_start(sp.dim, pr, sp.space, k) + j];
    }
    out[j] = acc;
  }
}

// Launchers (dg_slab.cu); each returns the number of launches (0 for ne = 0).
// fp32 selects float buffers and SlabTimes<float>, else double.
int launch_slab_matrix(const SlabPattern& sp, const SlabTimes<double>& tt, bool fp32, const void* B, const void* M,
                       void* vals, int pmax, int sm_count, cudaStream_t st);
int launch_slab_rhs(const SlabPattern& sp, const SlabTimes<double>& tt, bool fp32, const void* l, const void* M,
                    const void* u_prev, void* rhs, int sm_count, cudaStream_t st);
int launch_slab_trace(const SlabPattern& sp, const SlabTimes<double>& tt, bool fp32, const void* U, void* u_end,
                      int sm_count, cudaStream_t st);

}  // namespace dg
