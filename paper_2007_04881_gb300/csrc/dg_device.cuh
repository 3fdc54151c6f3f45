// dg_device.cuh -- device templates of the assembly kernels.
//
// Formulation used by every kernel.  With xi = 2(x - lo)/L - 1 the
// bounding-box coordinates of an element, the orthonormal Legendre basis
// (Sec. 3.1) is phi_i = s_i Phi_i with
//   Phi_i(xi) = prod_d P_{alpha_d}(xi_d),  s_i = prod_d sqrt((2 alpha_d + 1)/L_d),
// and d phi_i / d x_d = s_i (2/L_d) D_{d,i}, D_{d,i} = P'_{alpha_d} prod_{e != d} P_{alpha_e}.
// Every local block is then a contraction  A = S (U^T V) S  over stacked
// quadrature rows (a "row" = one quadrature point and one term):
//   volume point  (Eq. (2.4), first line; weight W = w_ref |J|):
//     U = [Phi; D_1; ..; D_d],
//     V = W [sum_d b'_d D_d + c Phi;  a'_1 D_1; ..; a'_d D_d],
//     a'_d = 4 a / L_d^2, b'_d = 2 b_d / L_d;
//   own-face point of element k (Eq. (2.4), face terms on its diagonal;
//   n' = 2 n_k / L, n_k outward, DN = sum_d n'_d D_d, kappa = 1/2 on an
//   interior face and 1 on the boundary, inflow where b . n_k < 0):
//     U = [Phi; DN],
//     V = W [ -kappa a DN + sigma Phi - min(b.n_k, 0) Phi;  -kappa a Phi ];
//   interface point (off-diagonal blocks, n0 out of e0):
//     A_01: U = [Phi^0; DN^0], V = W [-a_1 DN^1/2 - sigma Phi^1 + min(b.n0,0) Phi^1; a_0 Phi^1/2]
//     A_10: U = [Phi^1; DN^1], V = W [ a_0 DN^0/2 - sigma Phi^0 - max(b.n0,0) Phi^0; -a_1 Phi^0/2]
// and the load vector (Eq. (2.5)) is s_i sum_rows U_i R with
//     R = W f on volume points (Phi row),
//     R = W [sigma g - min(b.n,0) g;  -a g] on Dirichlet boundary-face points,
//     R = W [g_N; 0], g_N = a grad u . n_k, on Neumann boundary-face points,
// whose V rows are zero (no face term of Eq. (2.4); their records carry
// sigma = -1 and b . n = 0, so kappa = 0 and the penalty is dropped).
// Geometry (bounding boxes, sub-simplex maps, Jacobians, normals, penalty)
// comes from the geometry kernels as records in T: FP64, or for the reduced
// forms FP32 records equal to the rounded FP64 ones; T is the contraction
// type.
#pragma once

#include <cuda_runtime.h>

#include "dg_internal.h"

namespace dg {

__host__ __device__ constexpr int ipow_c(int b, int e) { return e == 0 ? 1 : b * ipow_c(b, e - 1); }

// Register-tile geometry of the element kernel for (D, P): each thread owns a
// TM x TM tile of the (padded) n x n block; G elements share a warp.  TM = n
// (one tile) selects the one-thread-per-element kernel.  Variant 0 of the
// FP32 table is the measured default: on the 65k-cell 2D workload degree 2
// runs a whole element per thread (36 accumulators) and degree 4 uses 8 x 8
// tiles, 4 threads per element; on the 3D workload degree 3 (whose volume
// terms take the moment launch) uses 4 x 4 tiles, 25 threads per element.
// Variants 1 and 2 are the other tile sizes that came close on some
// workload; the recorded pass's autotuner (dg_graph_create) times them.
template <int D, int P, typename T>
__host__ __device__ constexpr int tile_tm(int V) {
  // variant 3: the persistent pass's tiles; degrees whose default is one
  // element per thread get warp tiles of half the block's edge there
  if (V == 3) return tile_tm<D, P, T>(0) == nbasis(D, P) ? (nbasis(D, P) + 1) / 2 : tile_tm<D, P, T>(0);
  if (sizeof(T) == 4 && D == 2) {
    if (P == 1) return 3;
    if (P == 2) return 6;
    if (P == 3) return V == 1 ? 4 : 5;
    if (P == 4) return V == 1 ? 5 : V == 2 ? 4 : 8;
    if (P == 5) return V == 1 ? 6 : V == 2 ? 5 : 7;
    return V == 1 ? 6 : 7;
  }
  if (sizeof(T) == 4 && D == 3) {
    if (P == 1) return 4;
    if (P == 2) return V == 1 ? 4 : 5;
    if (P == 3) return V == 1 ? 5 : V == 2 ? 7 : 4;
    return 7;
  }
  return D == 2 ? (P <= 2 ? 3 : P == 3 ? 5 : P == 4 ? 4 : 7) : (P == 1 ? 4 : P <= 3 ? 5 : 7);
}
// number of distinct tile variants of (D, P, T)
template <int D, int P, typename T>
__host__ __device__ constexpr int tile_variants() {
  return tile_tm<D, P, T>(2) != tile_tm<D, P, T>(0) && tile_tm<D, P, T>(2) != tile_tm<D, P, T>(1) ? 3
         : tile_tm<D, P, T>(1) != tile_tm<D, P, T>(0)                                               ? 2
                                                                                                    : 1;
}

template <int D, int P, typename T = float, int V = 0>
struct TileCfg {
  static constexpr int N = nbasis(D, P);
  static constexpr int TM = tile_tm<D, P, T>(V);
  static constexpr int TR = (N + TM - 1) / TM;
  static constexpr int TPE = TR * TR;
  static constexpr int G = 32 / TPE;
  static constexpr int TMP = (TM + 1) / 2 * 2;  // padded tile stride (paired loads)
  static constexpr int ROW = TR * TMP;
  static constexpr int NT = D + 1;
  static constexpr int QT = ipow_c(P + 2, D);  // volume points per sub-simplex
};

template <int D, typename T>
struct ChunkCfg {
  static constexpr int CW = D == 2 ? 32 : 16;  // quadrature points per warp per chunk
};

// --------------------------------------------------------------------------
// basis
// --------------------------------------------------------------------------

// P_0..P_P and P'_0..P'_P at x (three-term recurrences).
template <int P, typename T>
__device__ __forceinline__ void legendre(T x, T* Lv, T* dL) {
  Lv[0] = T(1);
  dL[0] = T(0);
  if (P >= 1) {
    Lv[1] = x;
    dL[1] = T(1);
  }
#pragma unroll
  for (int k = 1; k < P; ++k) {
    Lv[k + 1] = (T(2 * k + 1) / T(k + 1)) * x * Lv[k] - (T(k) / T(k + 1)) * Lv[k - 1];
    dL[k + 1] = dL[k - 1] + T(2 * k + 1) * Lv[k];
  }
}

// Phi[i], D[d][i] for i < nbasis(D, P), in the order: for k = 0..P,
// 2D: for j = 0..k: alpha = (k-j, j); 3D: for l = 0..k, j = 0..k-l: alpha = (k-j-l, j, l).
template <int D, int P, typename T>
__device__ __forceinline__ void basis_eval(const T* xi, T* Phi, T (*Dd)[nbasis(D, P)]) {
  T Lv[3][P + 1], dL[3][P + 1];
#pragma unroll
  for (int d = 0; d < D; ++d) legendre<P, T>(xi[d], Lv[d], dL[d]);
  int i = 0;
#pragma unroll
  for (int k = 0; k <= P; ++k) {
    if (D == 2) {
#pragma unroll
      for (int j = 0; j <= k; ++j) {
        const int a0 = k - j, a1 = j;
        Phi[i] = Lv[0][a0] * Lv[1][a1];
        Dd[0][i] = dL[0][a0] * Lv[1][a1];
        Dd[1][i] = Lv[0][a0] * dL[1][a1];
        ++i;
      }
    } else {
#pragma unroll
      for (int l = 0; l <= k; ++l) {
#pragma unroll
        for (int j = 0; j <= k - l; ++j) {
          const int a0 = k - j - l, a1 = j, a2 = l;
          const T xy = Lv[0][a0] * Lv[1][a1];
          Phi[i] = xy * Lv[2][a2];
          Dd[0][i] = dL[0][a0] * Lv[1][a1] * Lv[2][a2];
          Dd[1][i] = Lv[0][a0] * dL[1][a1] * Lv[2][a2];
          Dd[2][i] = xy * dL[2][a2];
          ++i;
        }
      }
    }
  }
}

// number of monomials of total degree exactly k in D variables
__host__ __device__ constexpr int ndeg(int D, int k) { return D == 2 ? k + 1 : (k + 1) * (k + 2) / 2; }

// exponent alpha_d of basis function i (runtime index), same order as basis_eval
template <int D>
__device__ __forceinline__ void basis_alpha(int i, int* al) {
  int k = 0, base = 0;
  while (base + ndeg(D, k) <= i) {
    base += ndeg(D, k);
    ++k;
  }
  int r = i - base;  // position within degree k
  if (D == 2) {
    al[0] = k - r;
    al[1] = r;
  } else {
    int l = 0;
    while (r > k - l) {
      r -= (k - l + 1);
      ++l;
    }
    al[0] = k - r - l;
    al[1] = r;
    al[2] = l;
  }
}

// --------------------------------------------------------------------------
// source and Dirichlet data (Eq. (2.1) with manufactured u)
// --------------------------------------------------------------------------

__device__ __forceinline__ void sc_pi(double x, double* s, double* c) { sincospi(x, s, c); }
__device__ __forceinline__ void sc_pi(float x, float* s, float* c) { sincospif(x, s, c); }

template <int D, typename T>
__device__ T exact_u(const Problem& pb, const T* x, T* gu, T* lap) {
  if (pb.source == 1) {
    T s[3], c[3];
#pragma unroll
    for (int d = 0; d < D; ++d) sc_pi(x[d], &s[d], &c[d]);
    T prod = T(1);
#pragma unroll
    for (int d = 0; d < D; ++d) prod *= s[d];
    const T pi = T(3.14159265358979323846);
#pragma unroll
    for (int d = 0; d < D; ++d) {
      T g = pi * c[d];
#pragma unroll
      for (int e = 0; e < D; ++e)
        if (e != d) g *= s[e];
      gu[d] = g;
    }
    *lap = -T(D) * pi * pi * prod;
    return prod;
  }
  if (pb.source == 2) {
    // graded monomials of degree <= 3, same order as the basis exponents
    T pw[3][4];
#pragma unroll
    for (int d = 0; d < D; ++d) {
      pw[d][0] = T(1);
      pw[d][1] = x[d];
      pw[d][2] = x[d] * x[d];
      pw[d][3] = pw[d][2] * x[d];
    }
    T u = T(0), g[3] = {T(0), T(0), T(0)}, l = T(0);
    int m = 0;
#pragma unroll
    for (int k = 0; k <= 3; ++k) {
#pragma unroll
      for (int ll = 0; ll <= (D == 3 ? k : 0); ++ll) {
#pragma unroll
        for (int j = 0; j <= k - ll; ++j) {
          const int e0 = k - j - ll, e1 = j, e2 = ll;
          const int ex[3] = {e0, e1, e2};
          const T cf = pb_val<T>(pb.poly[m], pb.polyf[m]);
          ++m;
          T v = cf;
#pragma unroll
          for (int d = 0; d < D; ++d) v *= pw[d][ex[d]];
          u += v;
#pragma unroll
          for (int d = 0; d < D; ++d) {
            if (ex[d] == 0) continue;
            T gd = cf * T(ex[d]) * pw[d][ex[d] - 1];
#pragma unroll
            for (int e = 0; e < D; ++e)
              if (e != d) gd *= pw[e][ex[e]];
            g[d] += gd;
            if (ex[d] >= 2) {
              T ld = cf * T(ex[d] * (ex[d] - 1)) * pw[d][ex[d] - 2];
#pragma unroll
              for (int e = 0; e < D; ++e)
                if (e != d) ld *= pw[e][ex[e]];
              l += ld;
            }
          }
        }
      }
    }
#pragma unroll
    for (int d = 0; d < D; ++d) gu[d] = g[d];
    *lap = l;
    return u;
  }
#pragma unroll
  for (int d = 0; d < D; ++d) gu[d] = T(0);
  *lap = T(0);
  return T(0);
}

template <int D, typename T>
__device__ __forceinline__ T source_f(const Problem& pb, T a, const T* x) {
  T gu[3], lap;
  const T u = exact_u<D, T>(pb, x, gu, &lap);
  T bg = T(0);
#pragma unroll
  for (int d = 0; d < D; ++d) bg += pb_val<T>(pb.b[d], pb.bf[d]) * gu[d];
  return -a * lap + bg + pb_val<T>(pb.c, pb.cf) * u;
}

template <int D, typename T>
__device__ __forceinline__ T dirichlet_g(const Problem& pb, const T* x) {
  T gu[3], lap;
  return exact_u<D, T>(pb, x, gu, &lap);
}

template <typename T>
__device__ __forceinline__ const T* pick(const double* a, const float* b);
template <>
__device__ __forceinline__ const double* pick<double>(const double* a, const float*) {
  return a;
}
template <>
__device__ __forceinline__ const float* pick<float>(const double*, const float* b) {
  return b;
}

__host__ __device__ constexpr size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Builds with DG_CHECK_BOUNDS: a range [off, off + n) checked against
// [0, cap) before the kernel writes it; outside, bit 1 of the status word is
// set (dg_sync returns DG_ERR_BOUNDS) and the caller skips the write.
// Without the flag: true, and no code.
__device__ __forceinline__ bool dg_in_range(int* status, int64_t off, int64_t n, int64_t cap) {
#ifdef DG_CHECK_BOUNDS
  if (off < 0 || n < 0 || off + n > cap) {
    if (status) atomicOr(status, 2);
    return false;
  }
#else
  (void)status;
  (void)off;
  (void)n;
  (void)cap;
#endif
  return true;
}

// --------------------------------------------------------------------------
// tile loads from shared memory (vectorised where the padded stride allows)
// --------------------------------------------------------------------------

template <typename T, int TM, int TMP>
__device__ __forceinline__ void load_tile(const T* __restrict__ p, T (&o)[TM]) {
  if constexpr (sizeof(T) == 4 && TMP % 4 == 0) {
#pragma unroll
    for (int a = 0; a < TMP / 4; ++a) {
      const float4 v = reinterpret_cast<const float4*>(p)[a];
      if (4 * a + 0 < TM) o[4 * a + 0 < TM ? 4 * a + 0 : 0] = v.x;
      if (4 * a + 1 < TM) o[4 * a + 1 < TM ? 4 * a + 1 : 0] = v.y;
      if (4 * a + 2 < TM) o[4 * a + 2 < TM ? 4 * a + 2 : 0] = v.z;
      if (4 * a + 3 < TM) o[4 * a + 3 < TM ? 4 * a + 3 : 0] = v.w;
    }
  } else if constexpr (sizeof(T) == 4 && TMP % 2 == 0) {
#pragma unroll
    for (int a = 0; a < TMP / 2; ++a) {
      const float2 v = reinterpret_cast<const float2*>(p)[a];
      if (2 * a + 0 < TM) o[2 * a + 0 < TM ? 2 * a + 0 : 0] = v.x;
      if (2 * a + 1 < TM) o[2 * a + 1 < TM ? 2 * a + 1 : 0] = v.y;
    }
  } else if constexpr (sizeof(T) == 8 && TMP % 2 == 0) {
#pragma unroll
    for (int a = 0; a < TMP / 2; ++a) {
      const double2 v = reinterpret_cast<const double2*>(p)[a];
      if (2 * a + 0 < TM) o[2 * a + 0 < TM ? 2 * a + 0 : 0] = v.x;
      if (2 * a + 1 < TM) o[2 * a + 1 < TM ? 2 * a + 1 : 0] = v.y;
    }
  } else {
#pragma unroll
    for (int a = 0; a < TM; ++a) o[a] = p[a];
  }
}

// Basis of a neighbouring element whose degree pk is known only at run time:
// dispatch to the compiled degree and hand each function to sink(i, Phi, D).
template <int D, int PK, typename T, typename Sink>
__device__ __forceinline__ void nbr_basis_p(const T* xi, Sink& sink) {
  constexpr int N = nbasis(D, PK);
  T Phi[N], Dd[D][N];
  basis_eval<D, PK, T>(xi, Phi, Dd);
#pragma unroll
  for (int i = 0; i < N; ++i) {
    T dv[D];
#pragma unroll
    for (int d = 0; d < D; ++d) dv[d] = Dd[d][i];
    sink(i, Phi[i], dv);
  }
}

template <int D, typename T, typename Sink>
__device__ __forceinline__ void nbr_basis(int pk, const T* xi, Sink& sink) {
  switch (pk) {
    case 1: nbr_basis_p<D, 1, T>(xi, sink); break;
    case 2: nbr_basis_p<D, 2, T>(xi, sink); break;
    case 3: nbr_basis_p<D, 3, T>(xi, sink); break;
    case 4: nbr_basis_p<D, 4, T>(xi, sink); break;
    case 5: if constexpr (D == 2) nbr_basis_p<D, 5, T>(xi, sink); break;
    case 6: if constexpr (D == 2) nbr_basis_p<D, 6, T>(xi, sink); break;
    default: break;
  }
}

// --------------------------------------------------------------------------
// common pieces of the row kernels
// --------------------------------------------------------------------------

// C_i = prod_d sqrt(2 alpha_d + 1): with R = 1/sqrt(|bbox|) the basis scale is
// s_i = R C_i, so a block (e, k) is R_e R_k C_i C_j (U^T V)_ij.
template <int D, typename T>
__device__ __forceinline__ void fill_ctab(T* ctab, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    int al[3];
    basis_alpha<D>(i, al);
    double c = 1.0;
#pragma unroll
    for (int d = 0; d < D; ++d) c *= 2.0 * al[d] + 1.0;
    ctab[i] = T(sqrt(c));
  }
}

// per-element parameters in T, read from the contraction-precision record
template <int D, typename T>
struct ElemPar {
  T ap[D], bp[D], lo[D], L[D];
  T c, a, R;
};

template <int D, typename T>
__device__ __forceinline__ void load_elem_par(const DevMesh& m, int e, ElemPar<D, T>& q) {
  const T* EG = pick<T>(m.eg64, m.eg32);
  const T a = T(m.a[e]);
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const T iL = EG[(size_t)(2 * D + d) * m.ne + e];
    q.lo[d] = EG[(size_t)d * m.ne + e];
    q.L[d] = EG[(size_t)(D + d) * m.ne + e];
    q.ap[d] = T(4) * a * iL * iL;      // a'_d = 4 a / L_d^2
    q.bp[d] = T(2) * pb_val<T>(m.pb.b[d], m.pb.bf[d]) * iL;  // b'_d = 2 b_d / L_d
  }
  q.c = pb_val<T>(m.pb.c, m.pb.cf);
  q.a = a;
  q.R = EG[(size_t)(3 * D) * m.ne + e];
}

// Quadrature point of one side of a half-face record (r: the record for the
// own side, the record + FV for the other) at the reference point fr: xi in
// that side's frame and its scaled normal, pointing out of the own element.
template <int D, typename T>
__device__ __forceinline__ void hf_point(const T* r, const T* fr, T* xi, T* np) {
#pragma unroll
  for (int d = 0; d < D; ++d) {
    T v = r[d] + fr[0] * r[D + d];
    if constexpr (D == 3) v += fr[1] * r[2 * D + d];
    xi[d] = v;
    np[d] = r[D * D + d];
  }
}

// Per-point stride (in T) of the staged rows: the staging lane writes 16-byte
// vectors (8-byte for float pairs); an odd stride in vector units keeps the
// 8 (or 16) lanes of one store phase on distinct banks.
template <typename T, int TMP>
__host__ __device__ constexpr int point_stride(int words) {
  if (sizeof(T) == 4 && TMP % 4 == 0) return (words + 3) / 4 % 2 ? (words + 3) / 4 * 4 : (words + 3) / 4 * 4 + 4;
  // float2 or double2 units of 2 elements
  return (words + 1) / 2 % 2 ? (words + 1) / 2 * 2 : (words + 1) / 2 * 2 + 2;
}

// store N values (compile-time indexed) as TR groups of TMP (TM used, the
// rest zero), with 16-byte (or 8-byte) vector stores
template <typename T, int N, int TM, int TMP, int TR>
__device__ __forceinline__ void store_groups(T* __restrict__ dst, const T* v) {
  if constexpr (sizeof(T) == 4 && TMP % 4 == 0) {
#pragma unroll
    for (int r = 0; r < TR; ++r)
#pragma unroll
      for (int q = 0; q < TMP / 4; ++q) {
        T w[4];
#pragma unroll
        for (int l = 0; l < 4; ++l) {
          const int ll = 4 * q + l, i = r * TM + ll;
          w[l] = (ll < TM && i < N) ? v[(ll < TM && i < N) ? i : 0] : T(0);
        }
        reinterpret_cast<float4*>(dst + r * TMP)[q] = make_float4(w[0], w[1], w[2], w[3]);
      }
  } else {
#pragma unroll
    for (int r = 0; r < TR; ++r)
#pragma unroll
      for (int q = 0; q < TMP / 2; ++q) {
        T w[2];
#pragma unroll
        for (int l = 0; l < 2; ++l) {
          const int ll = 2 * q + l, i = r * TM + ll;
          w[l] = (ll < TM && i < N) ? v[(ll < TM && i < N) ? i : 0] : T(0);
        }
        if constexpr (sizeof(T) == 4)
          reinterpret_cast<float2*>(dst + r * TMP)[q] = make_float2(w[0], w[1]);
        else
          reinterpret_cast<double2*>(dst + r * TMP)[q] = make_double2(w[0], w[1]);
      }
  }
}

template <typename T, int TMP>
__device__ __forceinline__ void zero_groups(T* __restrict__ dst, int words) {
  if constexpr (sizeof(T) == 4 && TMP % 4 == 0) {
    for (int q = 0; q < words / 4; ++q) reinterpret_cast<float4*>(dst)[q] = make_float4(0.f, 0.f, 0.f, 0.f);
  } else if constexpr (sizeof(T) == 4) {
    for (int q = 0; q < words / 2; ++q) reinterpret_cast<float2*>(dst)[q] = make_float2(0.f, 0.f);
  } else {
    for (int q = 0; q < words / 2; ++q) reinterpret_cast<double2*>(dst)[q] = make_double2(0.0, 0.0);
  }
}

// --------------------------------------------------------------------------
// lane kernel: a few lanes assemble the whole block row of one element, each
// holding the whole n x n block in registers (low degrees: no staging needed)
// --------------------------------------------------------------------------

template <int D, int P, int PK, typename T>
__device__ __forceinline__ void lane_offdiag(const DevMesh& m, const ElemPar<D, T>& q, int4 br, int64_t off,
                                             const T* __restrict__ HFR, const T* __restrict__ FR, const T* ctab,
                                             T* __restrict__ vals) {
  constexpr int N = nbasis(D, P), NK = nbasis(D, PK);
  constexpr int FV = side_vals(D), RS = hf_rec_vals(D);
  T acc[N][NK];
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j < NK; ++j) acc[i][j] = T(0);
  const T* EG = pick<T>(m.eg64, m.eg32);
  const int k = br.x;
  const T ak = T(m.a[k]);
  const T Rk = EG[(size_t)(3 * D) * m.ne + k];
  constexpr int nq = (P > PK ? P : PK) + 1;
  constexpr int qf = D == 2 ? nq : nq * nq;
  for (int fi = 0; fi < br.z; ++fi) {
    const T* rec = HFR + (size_t)(br.y + fi) * RS;
    const T J = rec[2 * FV], sig = rec[2 * FV + 1], bn = rec[2 * FV + 2];
    const T upw = bn < T(0) ? bn : T(0);
    for (int lq = 0; lq < qf; ++lq) {
      const T* fr = FR + (size_t)(m.rt.face_off[nq] + lq) * (D == 2 ? 2 : 3);
      T xe[D], ne_[D], xk[D], nk_[D];
      hf_point<D, T>(rec, fr, xe, ne_);
      hf_point<D, T>(rec + FV, fr, xk, nk_);
      const T W = fr[D == 2 ? 1 : 2] * J;
      T Pe[N], De[D][N], Pk[NK], Dk[D][NK];
      basis_eval<D, P, T>(xe, Pe, De);
      basis_eval<D, PK, T>(xk, Pk, Dk);
      T dne[N];
#pragma unroll
      for (int i = 0; i < N; ++i) {
        T v = T(0);
#pragma unroll
        for (int d = 0; d < D; ++d) v += ne_[d] * De[d][i];
        dne[i] = v;
      }
#pragma unroll
      for (int j = 0; j < NK; ++j) {
        T dn = T(0);
#pragma unroll
        for (int d = 0; d < D; ++d) dn += nk_[d] * Dk[d][j];
        const T v0 = W * (T(-0.5) * ak * dn + (upw - sig) * Pk[j]);
        const T v1 = W * (T(0.5) * q.a * Pk[j]);
#pragma unroll
        for (int i = 0; i < N; ++i) acc[i][j] = fma(Pe[i], v0, fma(dne[i], v1, acc[i][j]));
      }
    }
  }
  if (!dg_in_range(m.status, off, (int64_t)N * NK, m.nvals)) return;
  T* out = vals + off;
  const T RR = q.R * Rk;
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j < NK; ++j) out[i * NK + j] = RR * ctab[i] * ctab[j] * acc[i][j];
}

// lanes per element of the lane kernel
template <int D, int P, typename T>
__host__ __device__ constexpr int lane_lpe() {
  return 8;
}
// CTAs of kWarps warps that cover `count` elements of the lane kernel: one
// warp per part (1: the diagonal part alone, 2: both) per 32 / lane_lpe
// elements
template <int D, int P, typename T>
__host__ __device__ constexpr int lane_blocks(int count, int parts) {
  return ((count + 32 / lane_lpe<D, P, T>() - 1) / (32 / lane_lpe<D, P, T>()) * parts + kWarps - 1) / kWarps;
}

// Each element is taken by L = lane_lpe lanes of two warps: part 0 the
// diagonal block and the load vector, part 1 the off-diagonal blocks (they
// write disjoint blocks).  In part 0 the element's lanes take every L-th
// volume point and every L-th own-face point, each into a whole n x n
// register block, and a butterfly over the L lanes sums them (a fixed order:
// an element's result does not depend on which mesh or launch holds it); in
// part 1 each lane takes every L-th block of the row, less the blocks of
// interfaces whose larger degree has its bit in the mode (kModeMaskShift:
// the interface kernel writes those).  PARTS = 1: part 0 alone (kModeDiagOnly),
// compiled without part 1, whose neighbour blocks need far more registers.
template <int D, int P, typename T, int PARTS>
__global__ void __launch_bounds__(kWarps * 32)
    row_lane_kernel(const DevMesh m, int mode, T* __restrict__ vals, T* __restrict__ rhs) {
  constexpr int N = nbasis(D, P), QT = ipow_c(P + 2, D), SV = sub_vals(D);
  constexpr int NMAXC = nbasis(D, D == 2 ? kPMax2 : kPMax3);
  constexpr int L = lane_lpe<D, P, T>(), EW = 32 / L;
  static_assert(32 % L == 0, "lanes per element divide the warp");
  __shared__ T rule[QT * (D + 1)];
  __shared__ T ctab[NMAXC];
  const T* vrule = pick<T>(m.rt.vol64, m.rt.vol32) + (size_t)m.rt.vol_off[P] * (D + 1);
  for (int i = threadIdx.x; i < QT * (D + 1); i += blockDim.x) rule[i] = vrule[i];
  fill_ctab<D, T>(ctab, NMAXC);
  __syncthreads();
  const T* SG = pick<T>(m.sg64, m.sg32);
  const T* HFR = pick<T>(m.hfr64, m.hfr32);
  const T* FR = pick<T>(m.rt.face64, m.rt.face32);
  constexpr int FV = side_vals(D), RS = hf_rec_vals(D);
  const bool mat_vol = mode & kModeVol, mat_face = mode & kModeFace, do_rhs = mode & kModeRhs;
  const bool accum = mode & kModeAccum;
  const int base = m.elem_pstart[P], count = m.elem_pstart[P + 1] - base;
  const int lane = threadIdx.x & 31, lig = lane % L;
  // warp-uniform loop: warp gw takes part gw % parts of elements
  // (gw / parts) * EW ..
  static_assert(PARTS == 1 || PARTS == 2, "one or two parts");
  const int nw = (count + EW - 1) / EW * PARTS;
  const int wstride = (gridDim.x * blockDim.x) >> 5;
  for (int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; gw < nw; gw += wstride) {
    const int part = gw % PARTS, slot = (gw / PARTS) * EW + lane / L;
    const bool active = slot < count;
    const int e = active ? m.elem_perm[base + slot] : 0;
    ElemPar<D, T> q;
    if (active) load_elem_par<D, T>(m, e, q);
    if (PARTS == 2 && part == 1) {
      if (mat_face && active) {
        for (int bk = m.row_ptr[e] + lig; bk < m.row_ptr[e + 1]; bk += L) {
          const int4 br = m.blk_rec[bk];  // neighbour, first half face, faces, neighbour degree
          if (br.x < 0 || ((mode >> (kModeMaskShift + (P > br.w ? P : br.w))) & 1)) continue;
          const int64_t off = m.blk_off[bk];
          switch (br.w) {
            case 1: lane_offdiag<D, P, 1, T>(m, q, br, off, HFR, FR, ctab, vals); break;
            case 2: lane_offdiag<D, P, 2, T>(m, q, br, off, HFR, FR, ctab, vals); break;
            case 3: lane_offdiag<D, P, 3, T>(m, q, br, off, HFR, FR, ctab, vals); break;
            case 4: lane_offdiag<D, P, 4, T>(m, q, br, off, HFR, FR, ctab, vals); break;
            case 5: if constexpr (D == 2) lane_offdiag<D, P, 5, T>(m, q, br, off, HFR, FR, ctab, vals); break;
            case 6: if constexpr (D == 2) lane_offdiag<D, P, 6, T>(m, q, br, off, HFR, FR, ctab, vals); break;
            default: break;
          }
        }
      }
      continue;
    }
    // the off-diagonal launch next to the moment launch: the diagonal block
    // and the load vector are the moment launch's (warp-uniform)
    if (mode & kModeOffDiag) continue;
    T acc[N][N], racc[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      racc[i] = T(0);
#pragma unroll
      for (int j = 0; j < N; ++j) acc[i][j] = T(0);
    }
    const bool learned = active && m.lq_ok && m.lq_ok[e];
    const int nvol = !active || !(mat_vol || do_rhs) ? 0 : learned ? 28 : (m.eptr[e + 1] - m.eptr[e]) * QT;
    for (int qv = lig; qv < nvol; qv += L) {
      T xi[D], W;
      if (learned) {
        const T* LQ = pick<T>(m.lq64, m.lq32) + (size_t)e * 84;
        xi[0] = LQ[qv];
        xi[1 % D] = LQ[28 + qv];
        W = LQ[56 + qv];
      } else {
        const int t = qv / QT, r = qv - t * QT;
        const int sub = m.eptr[e] + t;
        T sv[SV];
#pragma unroll
        for (int k = 0; k < SV; ++k) sv[k] = SG[(size_t)k * m.nsub + sub];
        const T* rr = rule + r * (D + 1);
#pragma unroll
        for (int d = 0; d < D; ++d) {
          T v = sv[d] + rr[0] * sv[D + d] + rr[1] * sv[2 * D + d];
          if constexpr (D == 3) v += rr[2] * sv[3 * D + d];
          xi[d] = v;
        }
        W = rr[D] * sv[SV - 1];
      }
      T Phi[N], Dd[D][N];
      basis_eval<D, P, T>(xi, Phi, Dd);
      if (mat_vol) {
#pragma unroll
        for (int j = 0; j < N; ++j) {
          T adv = q.c * Phi[j];
          T vd[D];
#pragma unroll
          for (int d = 0; d < D; ++d) {
            adv += q.bp[d] * Dd[d][j];
            vd[d] = W * q.ap[d] * Dd[d][j];
          }
          adv *= W;
#pragma unroll
          for (int i = 0; i < N; ++i) {
            T s = fma(Phi[i], adv, acc[i][j]);
#pragma unroll
            for (int d = 0; d < D; ++d) s = fma(Dd[d][i], vd[d], s);
            acc[i][j] = s;
          }
        }
      }
      if (do_rhs) {
        T x[D];
#pragma unroll
        for (int d = 0; d < D; ++d) x[d] = q.lo[d] + (xi[d] + T(1)) * T(0.5) * q.L[d];
        const T fw = W * source_f<D, T>(m.pb, q.a, x);
#pragma unroll
        for (int i = 0; i < N; ++i) racc[i] = fma(Phi[i], fw, racc[i]);
      }
    }
    // own-face points, numbered over the element's half faces (hf_qoff: the
    // first point of each, from 0 per element)
    const int h0 = active ? m.hf_ptr[e] : 0;
    const int nhf = active ? m.hf_ptr[e + 1] - h0 : 0;
    const int nfp = active && (mat_face || do_rhs) ? m.e_nqf[e] : 0;
    for (int qv = lig; qv < nfp; qv += L) {
      int hf = h0, hi = h0 + nhf - 1;
      while (hf < hi) {
        const int mid = (hf + hi + 1) >> 1;
        if (m.hf_qoff[mid] <= qv)
          hf = mid;
        else
          hi = mid - 1;
      }
      // the half face's record: own side, then J, sigma, b.n, nq (signed)
      const T* rec = HFR + (size_t)hf * RS;
      const T J = rec[2 * FV], sig = rec[2 * FV + 1], bn = rec[2 * FV + 2], nqs = rec[2 * FV + 3];
      const bool bnd = nqs < T(0);
      const bool neu = sig < T(0);  // Neumann face
      if (!mat_face && !bnd) continue;
      if (neu && !do_rhs) continue;
      const int nq = (int)(bnd ? -nqs : nqs);
      const T kap = neu ? T(0) : bnd ? T(1) : T(0.5);
      const T sgf = neu ? T(0) : sig;
      const T upw = bn < T(0) ? bn : T(0);
      const T* fr = FR + (size_t)(m.rt.face_off[nq] + qv - m.hf_qoff[hf]) * (D == 2 ? 2 : 3);
      T xi[D], np[D];
      hf_point<D, T>(rec, fr, xi, np);
      const T W = fr[D == 2 ? 1 : 2] * J;
      T Phi[N], Dd[D][N], dn[N];
      basis_eval<D, P, T>(xi, Phi, Dd);
#pragma unroll
      for (int i = 0; i < N; ++i) {
        T v = T(0);
#pragma unroll
        for (int d = 0; d < D; ++d) v += np[d] * Dd[d][i];
        dn[i] = v;
      }
      if (mat_face && !neu) {
#pragma unroll
        for (int j = 0; j < N; ++j) {
          const T v0 = W * (-kap * q.a * dn[j] + (sgf - upw) * Phi[j]);
          const T v1 = W * (-kap * q.a * Phi[j]);
#pragma unroll
          for (int i = 0; i < N; ++i) acc[i][j] = fma(Phi[i], v0, fma(dn[i], v1, acc[i][j]));
        }
      }
      if (do_rhs && bnd) {
        T x[D], gu[3], lap;
#pragma unroll
        for (int d = 0; d < D; ++d) x[d] = q.lo[d] + (xi[d] + T(1)) * T(0.5) * q.L[d];
        const T gd = exact_u<D, T>(m.pb, x, gu, &lap);
        T r0 = W * (sgf - upw) * gd, r1 = -W * q.a * gd;
        if (neu) {
          // g_N = a grad u . n_k, n_k = n' L / 2
          T gn = T(0);
#pragma unroll
          for (int d = 0; d < D; ++d) gn += gu[d] * np[d] * q.L[d];
          r0 = W * T(0.5) * q.a * gn;
          r1 = T(0);
        }
#pragma unroll
        for (int i = 0; i < N; ++i) racc[i] = fma(Phi[i], r0, fma(dn[i], r1, racc[i]));
      }
    }
    // butterfly over the element's L lanes (every lane of the warp takes part)
#pragma unroll
    for (int off = L / 2; off > 0; off >>= 1) {
#pragma unroll
      for (int i = 0; i < N; ++i) {
        racc[i] += __shfl_xor_sync(0xffffffffu, racc[i], off);
#pragma unroll
        for (int j = 0; j < N; ++j) acc[i][j] += __shfl_xor_sync(0xffffffffu, acc[i][j], off);
      }
    }
    if (!active) continue;
    if ((mat_vol || mat_face) && dg_in_range(m.status, m.blk_off[m.diag_blk[e]], (int64_t)N * N, m.nvals)) {
      T* out = vals + m.blk_off[m.diag_blk[e]];
      const T RR = q.R * q.R;
#pragma unroll
      for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = 0; j < N; ++j)
          if ((i * N + j) % L == lig) {
            const T v = RR * ctab[i] * ctab[j] * acc[i][j];
            out[i * N + j] = accum ? out[i * N + j] + v : v;
          }
    }
    if (do_rhs && dg_in_range(m.status, m.dof_off[e], N, m.ndofs)) {
#pragma unroll
      for (int i = 0; i < N; ++i)
        if (i % L == lig) rhs[m.dof_off[e] + i] = q.R * ctab[i] * racc[i];
    }
  }
}

// --------------------------------------------------------------------------
// tile kernel: G elements of degree P per warp, each element's block held as
// TM x TM register tiles by TPE threads; quadrature rows are staged in shared
// memory by one lane per point and contracted by the tile threads
// --------------------------------------------------------------------------

template <int D, int P, typename T, int V = 0>
struct RowSmem {
  using Cfg = TileCfg<D, P, T, V>;
  static constexpr int G = Cfg::G, TM = Cfg::TM, TR = Cfg::TR, TMP = Cfg::TMP, ROW = Cfg::ROW, NT = Cfg::NT;
  static constexpr int C = ChunkCfg<D, T>::CW / G > 0 ? ChunkCfg<D, T>::CW / G : 1;
  static constexpr int PSU = point_stride<T, TMP>(NT * ROW);  // staged point: NT rows of ROW
  static constexpr int PT = 4 * D + 5;                         // T parameters per element
  static constexpr int PI = 17;                                // int parameters per element
  static constexpr int NMAXC = nbasis(D, D == 2 ? kPMax2 : kPMax3);
  __host__ __device__ static constexpr int vs(int nmax) { return (nmax + TR * TM - 1) / (TR * TM) * (TR * TM); }
  __host__ __device__ static constexpr int psn(int VS) { return (2 * VS) % 2 ? 2 * VS : 2 * VS + 1; }  // odd
  static constexpr size_t head_bytes = align_up(sizeof(T) * (Cfg::QT * (D + 1) + NMAXC), 16);
  static constexpr size_t u_bytes = align_up(sizeof(T) * G * C * PSU, 16);
  __host__ __device__ static constexpr size_t v_bytes(int VS) {
    return align_up(sizeof(T) * (PSU > psn(VS) ? G * C * PSU : G * C * psn(VS)), 16);
  }
  static constexpr size_t r_bytes = align_up(sizeof(T) * G * C * NT, 16);
  static constexpr size_t p_bytes = align_up(sizeof(T) * G * PT, 16) + align_up(sizeof(int) * G * PI, 16);
  __host__ __device__ static constexpr size_t warp_bytes(int VS) { return u_bytes + v_bytes(VS) + r_bytes + p_bytes; }
  __host__ __device__ static constexpr size_t total(int warps, int nmax) { return head_bytes + warps * warp_bytes(vs(nmax)); }
};

// Integer parameter slots per element (PI array).
enum : int {
  kPiElem = 0,  // element id (-1: empty slot)
  kPiNvol,      // volume points
  kPiNface,     // own-face points
  kPiSub0,      // first sub-simplex
  kPiHf0,       // first half face
  kPiNhf,       // half faces
  kPiRow0,      // first block of the BSR row
  kPiNslot,     // off-diagonal blocks in the row
  kPiDpos,      // position of the diagonal block in the row
  kPiSBlk,      // current slot: block index
  kPiSSide,     // current slot: face points per direction, max(p, p_k) + 1
  kPiSNk,       // current slot: neighbour basis size
  kPiSPk,       // current slot: neighbour degree
  kPiSF0,       // current slot: first half face of the interface in the row
  kPiSQF,       // current slot: points per face
  kPiSNpts,     // current slot: points of the interface
  kPiLrn,       // 1: the element has a learned volume rule
};
// T parameter slots: a'[D], b'[D], lo[D], L[D], then:
enum : int { kPtC = 0, kPtA = 1, kPtR = 2, kPtAk = 3, kPtRk = 4 };

// Bounded wait of the persistent pass: an item that adds to blocks another
// item writes first waits for that item's flag, at most limit_ns of wall
// time (%globaltimer); a wait that runs out sets bit 0 of *status and the
// waiting item skips the writes that depended on it.
struct WaitCtl {
  const int* vdone;  // [ne]: 1 once an element's moment item has written its diagonal block and load vector
  int* status;
  long long limit_ns;
};

__device__ __forceinline__ long long global_ns() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// true once *flag != 0; false when limit_ns of wall time pass first
__device__ __forceinline__ bool wait_flag(const int* flag, long long limit_ns) {
  if (ld_acquire(flag)) return true;
  const long long t0 = global_ns();
  for (;;) {
    __nanosleep(128);
    if (ld_acquire(flag)) return true;
    if (global_ns() - t0 > limit_ns) return false;
  }
}

// One tile of the row kernel: G elements of degree P on this warp.  wb: the
// warp's shared-memory region (RowSmem layout); rule: the degree's volume
// rule and ctab the basis scales, both in shared memory; wc: null, or the
// persistent pass's wait on the elements' moment items before the diagonal
// block and the load vector are added to.
template <int D, int P, typename T, int TV>
__device__ __forceinline__ void row_tile(const DevMesh& m, int mode, T* __restrict__ vals, T* __restrict__ rhs,
                                         int tile, const T* __restrict__ rule, const T* __restrict__ ctab,
                                         unsigned char* wb, const WaitCtl* wc) {
  using Cfg = TileCfg<D, P, T, TV>;
  using SM = RowSmem<D, P, T, TV>;
  constexpr int N = Cfg::N, TM = Cfg::TM, TR = Cfg::TR, TPE = Cfg::TPE, G = Cfg::G;
  constexpr int TMP = Cfg::TMP, ROW = Cfg::ROW, NT = Cfg::NT, QT = Cfg::QT, C = SM::C;
  constexpr int SV = sub_vals(D), PT = SM::PT, PI = SM::PI, PSU = SM::PSU;
  constexpr int X = 4 * D;  // first scalar slot in PT

  const int VS = SM::vs(m.nmax), PSN = SM::psn(VS);
  const int lane = threadIdx.x & 31;
  T* U = reinterpret_cast<T*>(wb);
  wb += SM::u_bytes;
  T* V = reinterpret_cast<T*>(wb);
  wb += SM::v_bytes(VS);
  T* R = reinterpret_cast<T*>(wb);
  wb += SM::r_bytes;
  T* PTv = reinterpret_cast<T*>(wb);
  int* PIv = reinterpret_cast<int*>(wb + align_up(sizeof(T) * G * PT, 16));

  const T* SG = pick<T>(m.sg64, m.sg32);
  const T* HFR = pick<T>(m.hfr64, m.hfr32);
  const T* FR = pick<T>(m.rt.face64, m.rt.face32);
  const T* EG = pick<T>(m.eg64, m.eg32);
  constexpr int FV = side_vals(D), RS = hf_rec_vals(D);

  const bool mat_vol = mode & kModeVol, mat_face = mode & kModeFace, do_rhs = mode & kModeRhs;
  const bool accum = mode & kModeAccum;
  // volume terms already written by the moment kernel: faces only, load vector added
  const bool skip_vol = mode & kModeSkipVol;
  // diagonal block and load vector complete (the moment launch took the own
  // faces too): the off-diagonal blocks only
  const bool off_only = mode & kModeOffDiag;
  // with b = 0 and c = 0 the Phi row of a volume point carries no matrix term
  const bool no_adv = m.pb.b[0] == 0.0 && m.pb.b[1] == 0.0 && m.pb.b[2] == 0.0 && m.pb.c == 0.0;
  const int base = m.elem_pstart[P], count = m.elem_pstart[P + 1] - base;

  const int g_me = lane / TPE;
  const int tr = (lane % TPE) / TR, tc = lane % TR;
  {
    const int gcount = min(G, count - tile * G);
    __syncwarp();
    // ---- per-element setup (one lane per element)
    if (lane < G) {
      int* pi = PIv + lane * PI;
      T* pt = PTv + lane * PT;
      if (lane < gcount) {
        const int e = m.elem_perm[base + tile * G + lane];
        const int lrn = m.lq_ok && m.lq_ok[e] ? 1 : 0;
        pi[kPiElem] = e;
        pi[kPiLrn] = lrn;
        pi[kPiNvol] = lrn ? 28 : (m.eptr[e + 1] - m.eptr[e]) * QT;
        pi[kPiNface] = m.e_nqf[e];
        pi[kPiSub0] = m.eptr[e];
        pi[kPiHf0] = m.hf_ptr[e];
        pi[kPiNhf] = m.hf_ptr[e + 1] - m.hf_ptr[e];
        pi[kPiRow0] = m.row_ptr[e];
        pi[kPiNslot] = m.row_ptr[e + 1] - m.row_ptr[e] - 1;
        pi[kPiDpos] = m.diag_blk[e] - m.row_ptr[e];
        ElemPar<D, T> q;
        load_elem_par<D, T>(m, e, q);
#pragma unroll
        for (int d = 0; d < D; ++d) {
          pt[d] = q.ap[d];
          pt[D + d] = q.bp[d];
          pt[2 * D + d] = q.lo[d];
          pt[3 * D + d] = q.L[d];
        }
        pt[X + kPtC] = q.c;
        pt[X + kPtA] = q.a;
        pt[X + kPtR] = q.R;
      } else {
        pi[kPiElem] = -1;
        pi[kPiNvol] = 0;
        pi[kPiNface] = 0;
        pi[kPiNslot] = 0;
      }
    }
    __syncwarp();
    int nv_l = 0, nf_l = 0, ns_l = 0;
    if (lane < gcount) {
      nv_l = (PIv[lane * PI + kPiNvol] + C - 1) / C;
      nf_l = (PIv[lane * PI + kPiNface] + C - 1) / C;
      ns_l = PIv[lane * PI + kPiNslot];
    }
    const int nvch = __reduce_max_sync(0xffffffffu, nv_l);
    const int nfch = __reduce_max_sync(0xffffffffu, nf_l);
    const int nslot = __reduce_max_sync(0xffffffffu, ns_l);

    T acc[TM][TM];
    T racc[TM];
#pragma unroll
    for (int a = 0; a < TM; ++a) {
      racc[a] = T(0);
#pragma unroll
      for (int b = 0; b < TM; ++b) acc[a][b] = T(0);
    }
    const bool active = g_me < gcount;

    // ---- volume points
    if ((mat_vol || do_rhs) && !skip_vol) {
      for (int ch = 0; ch < nvch; ++ch) {
        for (int idx = lane; idx < G * C; idx += 32) {
          const int g = idx / C, c = idx - g * C, qv = ch * C + c;
          T* Ur = U + (size_t)(g * C + c) * PSU;
          T* Vr = V + (size_t)(g * C + c) * PSU;
          T* Rr = R + (g * C + c) * NT;
          if (g < gcount && qv < PIv[g * PI + kPiNvol]) {
            const T* pt = PTv + g * PT;
            T xi[D], W;
            if (D == 2 && PIv[g * PI + kPiLrn]) {
              // learned rule: 28 points in bounding-box coordinates, physical weights
              const T* LQ = pick<T>(m.lq64, m.lq32) + (size_t)PIv[g * PI + kPiElem] * 84;
              xi[0] = LQ[qv];
              xi[1 % D] = LQ[28 + qv];
              W = LQ[56 + qv];
            } else {
              const int t = qv / QT, r = qv - t * QT;
              const int sub = PIv[g * PI + kPiSub0] + t;
              T sv[SV];
#pragma unroll
              for (int k = 0; k < SV; ++k) sv[k] = SG[(size_t)k * m.nsub + sub];
              const T* rr = rule + r * (D + 1);
#pragma unroll
              for (int d = 0; d < D; ++d) {
                T v = sv[d] + rr[0] * sv[D + d] + rr[1] * sv[2 * D + d];
                if constexpr (D == 3) v += rr[2] * sv[3 * D + d];
                xi[d] = v;
              }
              W = rr[D] * sv[SV - 1];
            }
            T Phi[N], Dd[D][N];
            basis_eval<D, P, T>(xi, Phi, Dd);
            T Vv[N];
#pragma unroll
            for (int i = 0; i < N; ++i) {
              T adv = pt[X + kPtC] * Phi[i];
#pragma unroll
              for (int d = 0; d < D; ++d) adv += pt[D + d] * Dd[d][i];
              Vv[i] = W * adv;
            }
            store_groups<T, N, TM, TMP, TR>(Ur, Phi);
            store_groups<T, N, TM, TMP, TR>(Vr, Vv);
#pragma unroll
            for (int d = 0; d < D; ++d) {
              const T s = W * pt[d];
#pragma unroll
              for (int i = 0; i < N; ++i) Vv[i] = s * Dd[d][i];
              store_groups<T, N, TM, TMP, TR>(Ur + (1 + d) * ROW, Dd[d]);
              store_groups<T, N, TM, TMP, TR>(Vr + (1 + d) * ROW, Vv);
            }
            if (do_rhs) {
              T x[D];
#pragma unroll
              for (int d = 0; d < D; ++d) x[d] = pt[2 * D + d] + (xi[d] + T(1)) * T(0.5) * pt[3 * D + d];
              Rr[0] = W * source_f<D, T>(m.pb, pt[X + kPtA], x);
#pragma unroll
              for (int d = 0; d < D; ++d) Rr[1 + d] = T(0);
            }
          } else {
            // both rows: an unstaged U slot holds whatever the shared memory
            // held before (possibly a NaN pattern), and NaN * 0 is NaN
            zero_groups<T, TMP>(Ur, NT * ROW);
            zero_groups<T, TMP>(Vr, NT * ROW);
#pragma unroll
            for (int t = 0; t < NT; ++t) Rr[t] = T(0);
          }
        }
        __syncwarp();
        if (active) {
#pragma unroll 1
          for (int c = 0; c < C; ++c) {
            const T* Ub = U + (size_t)(g_me * C + c) * PSU + tr * TMP;
            const T* Vb = V + (size_t)(g_me * C + c) * PSU + tc * TMP;
#pragma unroll
            for (int t = 0; t < NT; ++t) {
              T u[TM], v[TM];
              if (t == 0 && no_adv && !do_rhs) continue;
              load_tile<T, TM, TMP>(Ub + t * ROW, u);
              load_tile<T, TM, TMP>(Vb + t * ROW, v);
              if (mat_vol && !(t == 0 && no_adv)) {
#pragma unroll
                for (int a = 0; a < TM; ++a)
#pragma unroll
                  for (int b = 0; b < TM; ++b) acc[a][b] = fma(u[a], v[b], acc[a][b]);
              }
              if (do_rhs && tc == 0) {
                const T rv = R[(g_me * C + c) * NT + t];
#pragma unroll
                for (int a = 0; a < TM; ++a) racc[a] = fma(u[a], rv, racc[a]);
              }
            }
          }
        }
        __syncwarp();
      }
    }

    // ---- own-face points (diagonal-block face terms, boundary load terms)
    if ((mat_face || do_rhs) && !off_only) {
      for (int ch = 0; ch < nfch; ++ch) {
        for (int idx = lane; idx < G * C; idx += 32) {
          const int g = idx / C, c = idx - g * C, qv = ch * C + c;
          T* Ur = U + (size_t)(g * C + c) * PSU;
          T* Vr = V + (size_t)(g * C + c) * PSU;
          T* Rr = R + (g * C + c) * NT;
          if (g < gcount && qv < PIv[g * PI + kPiNface]) {
            const T* pt = PTv + g * PT;
            int lo_ = PIv[g * PI + kPiHf0], hi_ = lo_ + PIv[g * PI + kPiNhf] - 1;
            while (lo_ < hi_) {
              const int mid = (lo_ + hi_ + 1) >> 1;
              if (m.hf_qoff[mid] <= qv)
                lo_ = mid;
              else
                hi_ = mid - 1;
            }
            const int hf = lo_;
            // the half face's record: own side, then J, sigma, b.n, nq (signed)
            const T* rec = HFR + (size_t)hf * RS;
            T sc[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) sc[j] = rec[2 * FV + j];
            const bool bnd = sc[3] < T(0);
            const int nq = (int)(bnd ? -sc[3] : sc[3]);
            const int lq = qv - m.hf_qoff[hf];
            const T* fr = FR + (size_t)(m.rt.face_off[nq] + lq) * (D == 2 ? 2 : 3);
            T xi[D], np[D];
            hf_point<D, T>(rec, fr, xi, np);
            const T W = fr[D == 2 ? 1 : 2] * sc[0];
            const bool neu = sc[1] < T(0);  // Neumann face
            const T sig = neu ? T(0) : sc[1];
            const T bn = sc[2];
            const T kap = neu ? T(0) : bnd ? T(1) : T(0.5);
            const T a = pt[X + kPtA];
            const T upw = bn < T(0) ? bn : T(0);
            T Phi[N], Dd[D][N], dn[N], V0[N], V1[N];
            basis_eval<D, P, T>(xi, Phi, Dd);
#pragma unroll
            for (int i = 0; i < N; ++i) {
              T v = T(0);
#pragma unroll
              for (int d = 0; d < D; ++d) v += np[d] * Dd[d][i];
              dn[i] = v;
              V0[i] = W * (-kap * a * v + (sig - upw) * Phi[i]);
              V1[i] = W * (-kap * a * Phi[i]);
            }
            store_groups<T, N, TM, TMP, TR>(Ur, Phi);
            store_groups<T, N, TM, TMP, TR>(Ur + ROW, dn);
            store_groups<T, N, TM, TMP, TR>(Vr, V0);
            store_groups<T, N, TM, TMP, TR>(Vr + ROW, V1);
            if (do_rhs) {
              if (bnd) {
                T x[D], gu[3], lap;
#pragma unroll
                for (int d = 0; d < D; ++d) x[d] = pt[2 * D + d] + (xi[d] + T(1)) * T(0.5) * pt[3 * D + d];
                const T gd = exact_u<D, T>(m.pb, x, gu, &lap);
                Rr[0] = W * (sig - upw) * gd;
                Rr[1] = -W * a * gd;
                if (neu) {
                  // g_N = a grad u . n_k, n_k = n' L / 2
                  T gn = T(0);
#pragma unroll
                  for (int d = 0; d < D; ++d) gn += gu[d] * np[d] * pt[3 * D + d];
                  Rr[0] = W * T(0.5) * a * gn;
                  Rr[1] = T(0);
                }
              } else {
                Rr[0] = T(0);
                Rr[1] = T(0);
              }
            }
          } else {
            zero_groups<T, TMP>(Ur, 2 * ROW);
            zero_groups<T, TMP>(Vr, 2 * ROW);
            Rr[0] = T(0);
            Rr[1] = T(0);
          }
        }
        __syncwarp();
        if (active) {
#pragma unroll 1
          for (int c = 0; c < C; ++c) {
            const T* Ub = U + (size_t)(g_me * C + c) * PSU + tr * TMP;
            const T* Vb = V + (size_t)(g_me * C + c) * PSU + tc * TMP;
#pragma unroll
            for (int t = 0; t < 2; ++t) {
              T u[TM], v[TM];
              load_tile<T, TM, TMP>(Ub + t * ROW, u);
              load_tile<T, TM, TMP>(Vb + t * ROW, v);
              if (mat_face) {
#pragma unroll
                for (int a = 0; a < TM; ++a)
#pragma unroll
                  for (int b = 0; b < TM; ++b) acc[a][b] = fma(u[a], v[b], acc[a][b]);
              }
              if (do_rhs && tc == 0) {
                const T rv = R[(g_me * C + c) * NT + t];
#pragma unroll
                for (int a = 0; a < TM; ++a) racc[a] = fma(u[a], rv, racc[a]);
              }
            }
          }
        }
        __syncwarp();
      }
    }

    // ---- write the diagonal block and the load vector (in the persistent
    // pass, once the element's moment item has written them)
    bool wr = active && !off_only;
    if (wc && wr && skip_vol && !wait_flag(wc->vdone + PIv[g_me * PI + kPiElem], wc->limit_ns)) {
      atomicOr(wc->status, 1);
      wr = false;
    }
    if (wr) {
      const int e = PIv[g_me * PI + kPiElem];
      const T Re = PTv[g_me * PT + X + kPtR];
      if ((mat_vol || mat_face) && dg_in_range(m.status, m.blk_off[m.diag_blk[e]], (int64_t)N * N, m.nvals)) {
        T* out = vals + m.blk_off[m.diag_blk[e]];
        const T RR = Re * Re;
#pragma unroll
        for (int a = 0; a < TM; ++a) {
          const int i = tr * TM + a;
          if (i < N) {
            const T si = RR * ctab[i];
#pragma unroll
            for (int b = 0; b < TM; ++b) {
              const int j = tc * TM + b;
              if (j < N) {
                const T v = si * ctab[j] * acc[a][b];
                out[i * N + j] = accum ? out[i * N + j] + v : v;
              }
            }
          }
        }
      }
      if (do_rhs && tc == 0 && dg_in_range(m.status, m.dof_off[e], N, m.ndofs)) {
        T* out = rhs + m.dof_off[e];
#pragma unroll
        for (int a = 0; a < TM; ++a) {
          const int i = tr * TM + a;
          if (i < N) out[i] = skip_vol ? out[i] + Re * ctab[i] * racc[a] : Re * ctab[i] * racc[a];
        }
      }
    }

    // ---- off-diagonal blocks of the row: one per neighbour (interface)
    if (mat_face) {
      for (int sl = 0; sl < nslot; ++sl) {
        __syncwarp();
        if (lane < G) {
          int* pi = PIv + lane * PI;
          const int bk = lane < gcount && sl < pi[kPiNslot] ? pi[kPiRow0] + sl + (sl >= pi[kPiDpos] ? 1 : 0) : -1;
          const int4 br = bk >= 0 ? m.blk_rec[bk] : make_int4(0, 0, 0, 0);  // neighbour, first half face, faces, its degree
          // with kModeOffDiag: the interface kernel writes the block when the
          // interface's larger degree is in the mask
          if (bk >= 0 && !(off_only && ((mode >> (kModeMaskShift + (P > br.w ? P : br.w))) & 1))) {
            const int k = br.x, pk = br.w;
            const int nq = (P > pk ? P : pk) + 1;
            const int qf = D == 2 ? nq : nq * nq;
            pi[kPiSBlk] = bk;
            pi[kPiSSide] = nq;
            pi[kPiSPk] = pk;
            pi[kPiSNk] = nbasis(D, pk);
            pi[kPiSF0] = br.y;
            pi[kPiSQF] = qf;
            pi[kPiSNpts] = br.z * qf;
            PTv[lane * PT + X + kPtAk] = T(m.a[k]);
            PTv[lane * PT + X + kPtRk] = EG[(size_t)(3 * D) * m.ne + k];
          } else {
            pi[kPiSNk] = 0;
            pi[kPiSNpts] = 0;
          }
        }
        __syncwarp();
        int np_l = 0, pc_l = 0;
        if (lane < gcount) {
          np_l = (PIv[lane * PI + kPiSNpts] + C - 1) / C;
          pc_l = ((PIv[lane * PI + kPiSNk] + TM - 1) / TM + TR - 1) / TR;
        }
        const int nch = __reduce_max_sync(0xffffffffu, np_l);
        const int npass = __reduce_max_sync(0xffffffffu, pc_l);

        for (int pass = 0; pass < npass; ++pass) {
#pragma unroll
          for (int a = 0; a < TM; ++a)
#pragma unroll
            for (int b = 0; b < TM; ++b) acc[a][b] = T(0);
          const int col0 = (pass * TR + tc) * TM;
          for (int ch = 0; ch < nch; ++ch) {
            if (pass == 0 || nch > 1) {
              __syncwarp();
              for (int idx = lane; idx < G * C; idx += 32) {
                const int g = idx / C, c = idx - g * C, qv = ch * C + c;
                T* Ur = U + (size_t)(g * C + c) * PSU;
                T* Vr = V + (size_t)(g * C + c) * PSN;
                const int* pi = PIv + g * PI;
                if (g < gcount && qv < pi[kPiSNpts]) {
                  const int qf = pi[kPiSQF];
                  const int fi = qv / qf, lq = qv - fi * qf;
                  const int nq = pi[kPiSSide];
                  // the half face's record: both sides, then J, sigma, b.n
                  const T* rec = HFR + (size_t)(pi[kPiSF0] + fi) * RS;
                  const T* fr = FR + (size_t)(m.rt.face_off[nq] + lq) * (D == 2 ? 2 : 3);
                  T xe[D], xk[D], ne_[D], nk_[D], sc[3];
                  hf_point<D, T>(rec, fr, xe, ne_);
                  hf_point<D, T>(rec + FV, fr, xk, nk_);
#pragma unroll
                  for (int j = 0; j < 3; ++j) sc[j] = rec[2 * FV + j];
                  const T W = fr[D == 2 ? 1 : 2] * sc[0];
                  const T sig = sc[1];
                  const T bn = sc[2];
                  const T upw = bn < T(0) ? bn : T(0);
                  const T ae = PTv[g * PT + X + kPtA];
                  const T ak = PTv[g * PT + X + kPtAk];
                  {
                    T Phi[N], Dd[D][N], dn[N];
                    basis_eval<D, P, T>(xe, Phi, Dd);
#pragma unroll
                    for (int i = 0; i < N; ++i) {
                      T v = T(0);
#pragma unroll
                      for (int d = 0; d < D; ++d) v += ne_[d] * Dd[d][i];
                      dn[i] = v;
                    }
                    store_groups<T, N, TM, TMP, TR>(Ur, Phi);
                    store_groups<T, N, TM, TMP, TR>(Ur + ROW, dn);
                  }
                  auto sink = [&](int j, T phik, const T* dk) {
                    T dn = T(0);
#pragma unroll
                    for (int d = 0; d < D; ++d) dn += nk_[d] * dk[d];
                    Vr[j] = W * (T(-0.5) * ak * dn + (upw - sig) * phik);
                    Vr[VS + j] = W * (T(0.5) * ae * phik);
                  };
                  nbr_basis<D, T>(pi[kPiSPk], xk, sink);
                } else {
                  // both rows (an unstaged U slot may hold a NaN pattern)
                  zero_groups<T, TMP>(Ur, 2 * ROW);
                  for (int j = 0; j < VS; ++j) {
                    Vr[j] = T(0);
                    Vr[VS + j] = T(0);
                  }
                }
              }
              __syncwarp();
            }
            if (active) {
#pragma unroll 1
              for (int c = 0; c < C; ++c) {
                const T* Ub = U + (size_t)(g_me * C + c) * PSU + tr * TMP;
                const T* Vb = V + (size_t)(g_me * C + c) * PSN + col0;
#pragma unroll
                for (int t = 0; t < 2; ++t) {
                  T u[TM], v[TM];
                  load_tile<T, TM, TMP>(Ub + t * ROW, u);
#pragma unroll
                  for (int b = 0; b < TM; ++b) v[b] = Vb[t * VS + b];
#pragma unroll
                  for (int a = 0; a < TM; ++a)
#pragma unroll
                    for (int b = 0; b < TM; ++b) acc[a][b] = fma(u[a], v[b], acc[a][b]);
                }
              }
            }
          }
          // this pass's columns of the off-diagonal block
          if (active) {
            const int* pi = PIv + g_me * PI;
            const int nk = pi[kPiSNk];
            if (col0 < nk && dg_in_range(m.status, m.blk_off[pi[kPiSBlk]], (int64_t)N * nk, m.nvals)) {
              T* out = vals + m.blk_off[pi[kPiSBlk]];
              const T RR = PTv[g_me * PT + X + kPtR] * PTv[g_me * PT + X + kPtRk];
#pragma unroll
              for (int a = 0; a < TM; ++a) {
                const int i = tr * TM + a;
                if (i < N) {
                  const T si = RR * ctab[i];
#pragma unroll
                  for (int b = 0; b < TM; ++b) {
                    const int j = col0 + b;
                    if (j < nk) out[i * nk + j] = si * ctab[j] * acc[a][b];
                  }
                }
              }
            }
          }
        }
      }
    }
  }
}

template <int D, int P, typename T, int TV = 0>
__global__ void __launch_bounds__(kWarps * 32)
    row_kernel(const DevMesh m, int mode, T* __restrict__ vals, T* __restrict__ rhs) {
  using Cfg = TileCfg<D, P, T, TV>;
  using SM = RowSmem<D, P, T, TV>;
  constexpr int QT = Cfg::QT, G = Cfg::G;
  const int VS = SM::vs(m.nmax);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5;
  T* rule = reinterpret_cast<T*>(smem_raw);
  T* ctab = rule + QT * (D + 1);
  unsigned char* wb = smem_raw + SM::head_bytes + warp * SM::warp_bytes(VS);
  const T* vrule = pick<T>(m.rt.vol64, m.rt.vol32) + (size_t)m.rt.vol_off[P] * (D + 1);
  for (int i = threadIdx.x; i < QT * (D + 1); i += blockDim.x) rule[i] = vrule[i];
  fill_ctab<D, T>(ctab, SM::NMAXC);
  __syncthreads();
  const int count = m.elem_pstart[P + 1] - m.elem_pstart[P];
  const int ntiles = (count + G - 1) / G;
  for (int tile = blockIdx.x * kWarps + warp; tile < ntiles; tile += gridDim.x * kWarps)
    row_tile<D, P, T, TV>(m, mode, vals, rhs, tile, rule, ctab, wb, nullptr);
}

}  // namespace dg
