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
//     R = W [sigma g - min(b.n,0) g;  -a g] on boundary-face points.
// Geometry (bounding boxes, sub-simplex maps, Jacobians, normals, penalty)
// is computed in FP64 by the geometry kernels; T is the contraction type.
#pragma once

#include <cuda_runtime.h>

#include "dg_internal.h"

namespace dg {

__host__ __device__ constexpr int ipow_c(int b, int e) { return e == 0 ? 1 : b * ipow_c(b, e - 1); }

// Register-tile geometry of the element kernel for (D, P): each thread owns a
// TM x TM tile of the (padded) n x n block; G elements share a warp.
template <int D, int P>
struct TileCfg {
  static constexpr int N = nbasis(D, P);
  static constexpr int TM = D == 2 ? (P <= 2 ? 3 : P == 3 ? 5 : P == 4 ? 4 : 7) : (P == 1 ? 4 : P <= 3 ? 5 : 7);
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
          const T cf = T(pb.poly[m]);
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
  for (int d = 0; d < D; ++d) bg += T(pb.b[d]) * gu[d];
  return -a * lap + bg + T(pb.c) * u;
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
// row kernel: the whole block row of G elements of degree P per warp
// --------------------------------------------------------------------------

// Shared-memory layout (bytes) for a given neighbour stride VS (the widest
// neighbour block, rounded up to the column span TR*TM of one pass).
template <int D, int P, typename T>
struct RowSmem {
  using Cfg = TileCfg<D, P>;
  static constexpr int C = ChunkCfg<D, T>::CW / Cfg::G > 0 ? ChunkCfg<D, T>::CW / Cfg::G : 1;
  static constexpr int NROWS = Cfg::G * C * Cfg::NT;
  static constexpr int PT = 4 * D + 2;  // T parameters per element
  static constexpr int PI = 16;         // int parameters per element
  static constexpr size_t rule_bytes = align_up(sizeof(T) * Cfg::QT * (D + 1), 16);
  __host__ __device__ static constexpr int vs(int nmax) {
    return (nmax + Cfg::TR * Cfg::TM - 1) / (Cfg::TR * Cfg::TM) * (Cfg::TR * Cfg::TM);
  }
  __host__ __device__ static constexpr size_t u_bytes() { return align_up(sizeof(T) * NROWS * Cfg::ROW, 16); }
  __host__ __device__ static constexpr size_t v_bytes(int VS) {
    return align_up(sizeof(T) * (NROWS * Cfg::ROW > Cfg::G * C * 2 * VS ? NROWS * Cfg::ROW : Cfg::G * C * 2 * VS), 16);
  }
  __host__ __device__ static constexpr size_t r_bytes() { return align_up(sizeof(T) * NROWS, 16); }
  __host__ __device__ static constexpr size_t s_bytes(int VS) {
    return align_up(sizeof(T) * Cfg::G * (Cfg::ROW + VS), 16);
  }
  __host__ __device__ static constexpr size_t p_bytes() {
    return align_up(sizeof(T) * Cfg::G * PT, 16) + align_up(sizeof(int) * Cfg::G * PI, 16);
  }
  __host__ __device__ static constexpr size_t warp_bytes(int VS) {
    return u_bytes() + v_bytes(VS) + r_bytes() + s_bytes(VS) + p_bytes();
  }
  __host__ __device__ static constexpr size_t total(int warps, int nmax) {
    return rule_bytes + warps * warp_bytes(vs(nmax));
  }
};

// Integer parameter slots per element (PI array).
enum : int {
  kPiElem = 0,   // element id (-1: empty slot)
  kPiNvol,       // volume points
  kPiNface,      // own-face points
  kPiSub0,       // first sub-simplex
  kPiHf0,        // first half face
  kPiNhf,        // half faces
  kPiRow0,       // first block of the BSR row
  kPiNslot,      // off-diagonal blocks in the row
  kPiDpos,       // position of the diagonal block in the row
  kPiSBlk,       // current slot: block index
  kPiSSide,      // current slot: side of this element in the interface
  kPiSNk,        // current slot: neighbour basis size
  kPiSPk,        // current slot: neighbour degree
  kPiSF0,        // current slot: first face of the interface
  kPiSQF,        // current slot: points per face
  kPiSNpts,      // current slot: points of the interface
};

template <int D, int P, typename T>
__global__ void __launch_bounds__(kWarps * 32)
    row_kernel(const DevMesh m, int mode, T* __restrict__ vals, T* __restrict__ rhs) {
  using Cfg = TileCfg<D, P>;
  using SM = RowSmem<D, P, T>;
  constexpr int N = Cfg::N, TM = Cfg::TM, TR = Cfg::TR, TPE = Cfg::TPE, G = Cfg::G;
  constexpr int TMP = Cfg::TMP, ROW = Cfg::ROW, NT = Cfg::NT, QT = Cfg::QT, C = SM::C;
  constexpr int SV = sub_vals(D), FV = side_vals(D), PT = SM::PT, PI = SM::PI;
  constexpr int NPASS_COLS = TR * TM;  // columns covered by one pass over a neighbour block

  const int VS = SM::vs(m.nmax);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  T* rule = reinterpret_cast<T*>(smem_raw);
  unsigned char* wb = smem_raw + SM::rule_bytes + warp * SM::warp_bytes(VS);
  T* U = reinterpret_cast<T*>(wb);
  wb += SM::u_bytes();
  T* V = reinterpret_cast<T*>(wb);
  wb += SM::v_bytes(VS);
  T* R = reinterpret_cast<T*>(wb);
  wb += SM::r_bytes();
  T* S = reinterpret_cast<T*>(wb);  // [G][ROW] own scaling, then [G][VS] neighbour scaling
  T* SK = S + G * ROW;
  wb += SM::s_bytes(VS);
  T* PTv = reinterpret_cast<T*>(wb);
  int* PIv = reinterpret_cast<int*>(wb + align_up(sizeof(T) * G * PT, 16));

  const T* vrule = pick<T>(m.rt.vol64, m.rt.vol32) + (size_t)m.rt.vol_off[P] * (D + 1);
  for (int i = threadIdx.x; i < QT * (D + 1); i += blockDim.x) rule[i] = vrule[i];
  // zero U / V once: padding slots of the tiles are never written afterwards
  for (int i = lane; i < SM::NROWS * ROW; i += 32) U[i] = T(0);
  for (int i = lane; i < (int)(SM::v_bytes(VS) / sizeof(T)); i += 32) V[i] = T(0);
  __syncthreads();

  const T* SG = pick<T>(m.sg64, m.sg32);
  const T* FS = pick<T>(m.fs64, m.fs32);
  const T* FSC = pick<T>(m.fsc64, m.fsc32);
  const T* FR = pick<T>(m.rt.face64, m.rt.face32);

  const bool mat_vol = mode & kModeVol, mat_face = mode & kModeFace, do_rhs = mode & kModeRhs;
  const bool accum = mode & kModeAccum;
  const int base = m.elem_pstart[P], count = m.elem_pstart[P + 1] - base;
  const int ntiles = (count + G - 1) / G;

  const int g_me = lane / TPE;
  const int tr = (lane % TPE) / TR, tc = lane % TR;
  const bool lane_in_tile = g_me < G;

  for (int tile = blockIdx.x * kWarps + warp; tile < ntiles; tile += gridDim.x * kWarps) {
    const int gcount = min(G, count - tile * G);
    // ---- per-element setup (one lane per element), FP64 -> T
    if (lane < G) {
      int* pi = PIv + lane * PI;
      T* pt = PTv + lane * PT;
      if (lane < gcount) {
        const int e = m.elem_perm[base + tile * G + lane];
        const double a = m.a[e];
        pi[kPiElem] = e;
        pi[kPiNvol] = (m.eptr[e + 1] - m.eptr[e]) * QT;
        pi[kPiNface] = m.e_nqf[e];
        pi[kPiSub0] = m.eptr[e];
        pi[kPiHf0] = m.hf_ptr[e];
        pi[kPiNhf] = m.hf_ptr[e + 1] - m.hf_ptr[e];
        pi[kPiRow0] = m.row_ptr[e];
        pi[kPiNslot] = m.row_ptr[e + 1] - m.row_ptr[e] - 1;
        pi[kPiDpos] = m.diag_blk[e] - m.row_ptr[e];
#pragma unroll
        for (int d = 0; d < D; ++d) {
          const double L = m.L[d * m.ne + e], iL = 1.0 / L;
          pt[d] = T(4.0 * a * iL * iL);         // a'_d
          pt[D + d] = T(2.0 * m.pb.b[d] * iL);  // b'_d
          pt[2 * D + d] = T(m.lo[d * m.ne + e]);
          pt[3 * D + d] = T(L);
        }
        pt[4 * D] = T(m.pb.c);
        pt[4 * D + 1] = T(a);
      } else {
        pi[kPiElem] = -1;
        pi[kPiNvol] = 0;
        pi[kPiNface] = 0;
        pi[kPiNslot] = 0;
      }
    }
    __syncwarp();
    for (int idx = lane; idx < G * N; idx += 32) {
      const int g = idx / N, i = idx - g * N;
      if (g < gcount) {
        int al[3];
        basis_alpha<D>(i, al);
        double sc = 1.0;
        const int e = PIv[g * PI + kPiElem];
#pragma unroll
        for (int d = 0; d < D; ++d) sc *= (2.0 * al[d] + 1.0) / m.L[d * m.ne + e];
        S[g * ROW + i] = T(sqrt(sc));
      }
    }
    int nv_l = 0, nf_l = 0, ns_l = 0;
    if (lane < gcount) {
      nv_l = (PIv[lane * PI + kPiNvol] + C - 1) / C;
      nf_l = (PIv[lane * PI + kPiNface] + C - 1) / C;
      ns_l = PIv[lane * PI + kPiNslot];
    }
    const int nvch = __reduce_max_sync(0xffffffffu, nv_l);
    const int nfch = __reduce_max_sync(0xffffffffu, nf_l);
    const int nslot = __reduce_max_sync(0xffffffffu, ns_l);
    __syncwarp();

    T acc[TM][TM];
    T racc[TM];
#pragma unroll
    for (int a = 0; a < TM; ++a) {
      racc[a] = T(0);
#pragma unroll
      for (int b = 0; b < TM; ++b) acc[a][b] = T(0);
    }
    const bool active = lane_in_tile && g_me < gcount;

    // ---- volume points
    if (mat_vol || do_rhs) {
      for (int ch = 0; ch < nvch; ++ch) {
        for (int idx = lane; idx < G * C; idx += 32) {
          const int g = idx / C, c = idx - g * C, q = ch * C + c;
          const int row0 = (g * C + c) * NT;
          T* Ur = U + row0 * ROW;
          T* Vr = V + row0 * ROW;
          if (g < gcount && q < PIv[g * PI + kPiNvol]) {
            const T* pt = PTv + g * PT;
            const int t = q / QT, r = q - t * QT;
            const int sub = PIv[g * PI + kPiSub0] + t;
            T sv[SV];
#pragma unroll
            for (int k = 0; k < SV; ++k) sv[k] = SG[(size_t)k * m.nsub + sub];
            const T* rr = rule + r * (D + 1);
            T xi[D];
#pragma unroll
            for (int d = 0; d < D; ++d) {
              T v = sv[d] + rr[0] * sv[D + d] + rr[1] * sv[2 * D + d];
              if constexpr (D == 3) v += rr[2] * sv[3 * D + d];
              xi[d] = v;
            }
            const T W = rr[D] * sv[SV - 1];
            T Phi[N], Dd[D][N];
            basis_eval<D, P, T>(xi, Phi, Dd);
#pragma unroll
            for (int i = 0; i < N; ++i) {
              const int pos = (i / TM) * TMP + (i % TM);
              Ur[pos] = Phi[i];
              T adv = pt[4 * D] * Phi[i];
#pragma unroll
              for (int d = 0; d < D; ++d) {
                Ur[(1 + d) * ROW + pos] = Dd[d][i];
                adv += pt[D + d] * Dd[d][i];
                Vr[(1 + d) * ROW + pos] = W * pt[d] * Dd[d][i];
              }
              Vr[pos] = W * adv;
            }
            if (do_rhs) {
              T x[D];
#pragma unroll
              for (int d = 0; d < D; ++d) x[d] = pt[2 * D + d] + (xi[d] + T(1)) * T(0.5) * pt[3 * D + d];
              R[row0] = W * source_f<D, T>(m.pb, pt[4 * D + 1], x);
#pragma unroll
              for (int d = 0; d < D; ++d) R[row0 + 1 + d] = T(0);
            }
          } else {
#pragma unroll
            for (int t = 0; t < NT; ++t) {
#pragma unroll
              for (int i = 0; i < N; ++i) Vr[t * ROW + (i / TM) * TMP + (i % TM)] = T(0);
              R[row0 + t] = T(0);
            }
          }
        }
        __syncwarp();
        if (active) {
#pragma unroll 1
          for (int c = 0; c < C; ++c) {
            const int row0 = (g_me * C + c) * NT;
#pragma unroll
            for (int t = 0; t < NT; ++t) {
              T u[TM], v[TM];
              load_tile<T, TM, TMP>(U + (row0 + t) * ROW + tr * TMP, u);
              load_tile<T, TM, TMP>(V + (row0 + t) * ROW + tc * TMP, v);
              if (mat_vol) {
#pragma unroll
                for (int a = 0; a < TM; ++a)
#pragma unroll
                  for (int b = 0; b < TM; ++b) acc[a][b] = fma(u[a], v[b], acc[a][b]);
              }
              if (do_rhs && tc == 0) {
                const T rv = R[row0 + t];
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
    if (mat_face || do_rhs) {
      for (int ch = 0; ch < nfch; ++ch) {
        for (int idx = lane; idx < G * C; idx += 32) {
          const int g = idx / C, c = idx - g * C, q = ch * C + c;
          const int row0 = (g * C + c) * NT;
          T* Ur = U + row0 * ROW;
          T* Vr = V + row0 * ROW;
          if (g < gcount && q < PIv[g * PI + kPiNface]) {
            const T* pt = PTv + g * PT;
            int lo_ = PIv[g * PI + kPiHf0], hi_ = lo_ + PIv[g * PI + kPiNhf] - 1;
            while (lo_ < hi_) {
              const int mid = (lo_ + hi_ + 1) >> 1;
              if (m.hf_qoff[mid] <= q)
                lo_ = mid;
              else
                hi_ = mid - 1;
            }
            const int hf = lo_;
            const int f = m.hf_face[hf];
            const int s = m.hf_side[hf];
            const int nq = m.f_nq[f];
            const int lq = q - m.hf_qoff[hf];
            const T* fr = FR + (size_t)(m.rt.face_off[nq] + lq) * (D == 2 ? 2 : 3);
            const T* fsd = FS + (size_t)s * FV * m.nf + f;
            T xi[D], np[D];
#pragma unroll
            for (int d = 0; d < D; ++d) {
              T v = fsd[(size_t)d * m.nf] + fr[0] * fsd[(size_t)(D + d) * m.nf];
              if constexpr (D == 3) v += fr[1] * fsd[(size_t)(2 * D + d) * m.nf];
              xi[d] = v;
              np[d] = fsd[(size_t)((D == 2 ? 2 : 3) * D + d) * m.nf];
            }
            const T sgn = s == 0 ? T(1) : T(-1);
            const T W = fr[D == 2 ? 1 : 2] * FSC[f];
            const T sig = FSC[(size_t)m.nf + f];
            const T bn = sgn * FSC[(size_t)2 * m.nf + f];
            const bool bnd = m.f_e1[f] < 0;
            const T kap = bnd ? T(1) : T(0.5);
            const T a = pt[4 * D + 1];
            const T upw = bn < T(0) ? bn : T(0);
            T Phi[N], Dd[D][N];
            basis_eval<D, P, T>(xi, Phi, Dd);
#pragma unroll
            for (int i = 0; i < N; ++i) {
              const int pos = (i / TM) * TMP + (i % TM);
              T dn = T(0);
#pragma unroll
              for (int d = 0; d < D; ++d) dn += sgn * np[d] * Dd[d][i];
              Ur[pos] = Phi[i];
              Ur[ROW + pos] = dn;
              Vr[pos] = W * (-kap * a * dn + (sig - upw) * Phi[i]);
              Vr[ROW + pos] = W * (-kap * a * Phi[i]);
            }
            if (do_rhs) {
              if (bnd) {
                T x[D];
#pragma unroll
                for (int d = 0; d < D; ++d) x[d] = pt[2 * D + d] + (xi[d] + T(1)) * T(0.5) * pt[3 * D + d];
                const T gd = dirichlet_g<D, T>(m.pb, x);
                R[row0] = W * (sig - upw) * gd;
                R[row0 + 1] = -W * a * gd;
              } else {
                R[row0] = T(0);
                R[row0 + 1] = T(0);
              }
            }
          } else {
#pragma unroll
            for (int t = 0; t < 2; ++t) {
#pragma unroll
              for (int i = 0; i < N; ++i) Vr[t * ROW + (i / TM) * TMP + (i % TM)] = T(0);
              R[row0 + t] = T(0);
            }
          }
        }
        __syncwarp();
        if (active) {
#pragma unroll 1
          for (int c = 0; c < C; ++c) {
            const int row0 = (g_me * C + c) * NT;
#pragma unroll
            for (int t = 0; t < 2; ++t) {
              T u[TM], v[TM];
              load_tile<T, TM, TMP>(U + (row0 + t) * ROW + tr * TMP, u);
              load_tile<T, TM, TMP>(V + (row0 + t) * ROW + tc * TMP, v);
              if (mat_face) {
#pragma unroll
                for (int a = 0; a < TM; ++a)
#pragma unroll
                  for (int b = 0; b < TM; ++b) acc[a][b] = fma(u[a], v[b], acc[a][b]);
              }
              if (do_rhs && tc == 0) {
                const T rv = R[row0 + t];
#pragma unroll
                for (int a = 0; a < TM; ++a) racc[a] = fma(u[a], rv, racc[a]);
              }
            }
          }
        }
        __syncwarp();
      }
    }

    // ---- write the diagonal block and the load vector
    if (active) {
      const int e = PIv[g_me * PI + kPiElem];
      const T* Sg = S + g_me * ROW;
      if (mat_vol || mat_face) {
        T* out = vals + m.blk_off[m.diag_blk[e]];
#pragma unroll
        for (int a = 0; a < TM; ++a) {
          const int i = tr * TM + a;
          if (i < N) {
            const T si = Sg[i];
#pragma unroll
            for (int b = 0; b < TM; ++b) {
              const int j = tc * TM + b;
              if (j < N) {
                const T v = si * Sg[j] * acc[a][b];
                out[i * N + j] = accum ? out[i * N + j] + v : v;
              }
            }
          }
        }
      }
      if (do_rhs && tc == 0) {
        T* out = rhs + m.dof_off[e];
#pragma unroll
        for (int a = 0; a < TM; ++a) {
          const int i = tr * TM + a;
          if (i < N) out[i] = Sg[i] * racc[a];
        }
      }
    }

    // ---- off-diagonal blocks of the row: one per neighbour (interface)
    if (mat_face) {
      for (int sl = 0; sl < nslot; ++sl) {
        __syncwarp();
        if (lane < G) {
          int* pi = PIv + lane * PI;
          if (lane < gcount && sl < pi[kPiNslot]) {
            const int e = pi[kPiElem];
            const int bk = pi[kPiRow0] + sl + (sl >= pi[kPiDpos] ? 1 : 0);
            const int it = m.blk_if[bk];
            const int k = m.col[bk];
            const int pk = m.p[k];
            const int f0 = m.if_fptr[it];
            const int nq = m.f_nq[f0];
            const int qf = D == 2 ? nq : nq * nq;
            pi[kPiSBlk] = bk;
            pi[kPiSSide] = m.if_e0[it] == e ? 0 : 1;
            pi[kPiSPk] = pk;
            pi[kPiSNk] = nbasis(D, pk);
            pi[kPiSF0] = f0;
            pi[kPiSQF] = qf;
            pi[kPiSNpts] = (m.if_fptr[it + 1] - f0) * qf;
            PTv[lane * PT + 4 * D] = T(m.a[k]);  // neighbour diffusion (slot c is free here)
          } else {
            pi[kPiSNk] = 0;
            pi[kPiSNpts] = 0;
          }
        }
        __syncwarp();
        // neighbour scaling s_j
        for (int idx = lane; idx < G * VS; idx += 32) {
          const int g = idx / VS, j = idx - g * VS;
          if (g < gcount && j < PIv[g * PI + kPiSNk]) {
            const int k = m.col[PIv[g * PI + kPiSBlk]];
            int al[3];
            basis_alpha<D>(j, al);
            double sc = 1.0;
#pragma unroll
            for (int d = 0; d < D; ++d) sc *= (2.0 * al[d] + 1.0) / m.L[d * m.ne + k];
            SK[g * VS + j] = T(sqrt(sc));
          }
        }
        int np_l = 0, pc_l = 0;
        if (lane < gcount) {
          np_l = (PIv[lane * PI + kPiSNpts] + C - 1) / C;
          pc_l = ((PIv[lane * PI + kPiSNk] + TM - 1) / TM + TR - 1) / TR;
        }
        const int nch = __reduce_max_sync(0xffffffffu, np_l);
        const int npass = __reduce_max_sync(0xffffffffu, pc_l);
        __syncwarp();

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
                const int g = idx / C, c = idx - g * C, q = ch * C + c;
                const int rowu = (g * C + c) * 2;
                T* Ur = U + rowu * ROW;
                T* Vr = V + (size_t)rowu * VS;
                const int* pi = PIv + g * PI;
                if (g < gcount && q < pi[kPiSNpts]) {
                  const int qf = pi[kPiSQF];
                  const int f = pi[kPiSF0] + q / qf, lq = q - (q / qf) * qf;
                  const int se = pi[kPiSSide], sk = 1 - se;
                  const int nq = m.f_nq[f];
                  const T* fr = FR + (size_t)(m.rt.face_off[nq] + lq) * (D == 2 ? 2 : 3);
                  const T* fe = FS + (size_t)se * FV * m.nf + f;
                  const T* fk = FS + (size_t)sk * FV * m.nf + f;
                  const T sgn = se == 0 ? T(1) : T(-1);
                  T xe[D], xk[D], ne_[D], nk_[D];
#pragma unroll
                  for (int d = 0; d < D; ++d) {
                    T v0 = fe[(size_t)d * m.nf] + fr[0] * fe[(size_t)(D + d) * m.nf];
                    T v1 = fk[(size_t)d * m.nf] + fr[0] * fk[(size_t)(D + d) * m.nf];
                    if constexpr (D == 3) {
                      v0 += fr[1] * fe[(size_t)(2 * D + d) * m.nf];
                      v1 += fr[1] * fk[(size_t)(2 * D + d) * m.nf];
                    }
                    xe[d] = v0;
                    xk[d] = v1;
                    ne_[d] = sgn * fe[(size_t)((D == 2 ? 2 : 3) * D + d) * m.nf];
                    nk_[d] = sgn * fk[(size_t)((D == 2 ? 2 : 3) * D + d) * m.nf];
                  }
                  const T W = fr[D == 2 ? 1 : 2] * FSC[f];
                  const T sig = FSC[(size_t)m.nf + f];
                  const T bn = sgn * FSC[(size_t)2 * m.nf + f];
                  const T upw = bn < T(0) ? bn : T(0);
                  const T ae = PTv[g * PT + 4 * D + 1];
                  const T ak = PTv[g * PT + 4 * D];
                  {
                    T Phi[N], Dd[D][N];
                    basis_eval<D, P, T>(xe, Phi, Dd);
#pragma unroll
                    for (int i = 0; i < N; ++i) {
                      const int pos = (i / TM) * TMP + (i % TM);
                      T dn = T(0);
#pragma unroll
                      for (int d = 0; d < D; ++d) dn += ne_[d] * Dd[d][i];
                      Ur[pos] = Phi[i];
                      Ur[ROW + pos] = dn;
                    }
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
                  for (int j = 0; j < VS; ++j) {
                    Vr[j] = T(0);
                    Vr[VS + j] = T(0);
                  }
                }
              }
              __syncwarp();
            }
            if (active) {
              const int cnt = C;
#pragma unroll 1
              for (int c = 0; c < cnt; ++c) {
                const int rowu = (g_me * C + c) * 2;
#pragma unroll
                for (int t = 0; t < 2; ++t) {
                  T u[TM], v[TM];
                  load_tile<T, TM, TMP>(U + (rowu + t) * ROW + tr * TMP, u);
                  const T* vr = V + (size_t)(rowu + t) * VS + col0;
#pragma unroll
                  for (int b = 0; b < TM; ++b) v[b] = vr[b];
#pragma unroll
                  for (int a = 0; a < TM; ++a)
#pragma unroll
                    for (int b = 0; b < TM; ++b) acc[a][b] = fma(u[a], v[b], acc[a][b]);
                }
              }
            }
          }
          // write this pass's columns of the off-diagonal block
          if (active) {
            const int* pi = PIv + g_me * PI;
            const int nk = pi[kPiSNk];
            if (nk > 0 && col0 < nk) {
              T* out = vals + m.blk_off[pi[kPiSBlk]];
              const T* Sg = S + g_me * ROW;
              const T* Sk = SK + g_me * VS;
#pragma unroll
              for (int a = 0; a < TM; ++a) {
                const int i = tr * TM + a;
                if (i < N) {
#pragma unroll
                  for (int b = 0; b < TM; ++b) {
                    const int j = col0 + b;
                    if (j < nk) out[i * nk + j] = Sg[i] * Sk[j] * acc[a][b];
                  }
                }
              }
            }
          }
        }
      }
    }
    __syncwarp();
  }
}

}  // namespace dg
