// dg_varcoef_kernel.cuh -- the kernel of the variable-coefficient terms
// (the formulation is in dg_varcoef.cuh), instantiated per contraction type
// in dg_varcoef_f64.cu and dg_varcoef_f32.cu.
#pragma once

#include <cstdio>

#include "dg_device.cuh"
#include "dg_varcoef.cuh"

namespace dg {

constexpr int kVcWarps = 4;  // warps per CTA, one element row each
constexpr int kVcTR = 5;     // lanes per tile row and column: 25 lanes hold tiles

// b(x) and c(x) from the field table, in T
template <int D, typename T>
__device__ __forceinline__ T vc_fields_at(const VcFields& f, const T* x, T* b) {
#pragma unroll
  for (int d = 0; d < D; ++d) {
    T v = pb_val<T>(f.b0[d], f.b0f[d]);
#pragma unroll
    for (int e = 0; e < D; ++e) v += pb_val<T>(f.bx[d][e], f.bxf[d][e]) * x[e];
    b[d] = v;
  }
  // graded monomials of total degree <= 3, in the order of DG_SRC_POLY
  T pw[3][4];
#pragma unroll
  for (int d = 0; d < D; ++d) {
    pw[d][0] = T(1);
    pw[d][1] = x[d];
    pw[d][2] = x[d] * x[d];
    pw[d][3] = pw[d][2] * x[d];
  }
  T c = T(0);
  int m = 0;
#pragma unroll
  for (int k = 0; k <= 3; ++k) {
#pragma unroll
    for (int l = 0; l <= (D == 3 ? k : 0); ++l) {
#pragma unroll
      for (int j = 0; j <= k - l; ++j) {
        const int ex[3] = {k - j - l, j, l};
        T v = pb_val<T>(f.c[m], f.cf[m]);
        ++m;
#pragma unroll
        for (int d = 0; d < D; ++d) v *= pw[d][ex[d]];
        c += v;
      }
    }
  }
  return c;
}

// basis values (no derivatives) of degree PK at xi, into out[0 .. nbasis)
template <int D, int PK, typename T>
__device__ __forceinline__ void vc_values_p(const T* xi, T* out) {
  constexpr int NK = nbasis(D, PK);
  T Ph[NK], Dk[D][NK];
  basis_eval<D, PK, T>(xi, Ph, Dk);
#pragma unroll
  for (int i = 0; i < NK; ++i) out[i] = Ph[i];
}

// the same for a runtime degree pk (the neighbour of an off-diagonal block)
template <int D, typename T>
__device__ __forceinline__ void vc_basis_values(int pk, const T* xi, T* out) {
  switch (pk) {
    case 1: vc_values_p<D, 1, T>(xi, out); break;
    case 2: vc_values_p<D, 2, T>(xi, out); break;
    case 3: vc_values_p<D, 3, T>(xi, out); break;
    case 4: vc_values_p<D, 4, T>(xi, out); break;
    case 5: if constexpr (D == 2) vc_values_p<D, 5, T>(xi, out); break;
    case 6: if constexpr (D == 2) vc_values_p<D, 6, T>(xi, out); break;
    default: break;
  }
}

// One chunk of staged points into this lane's tile: rows i0 .. i0 + TM of
// the nr rows, columns j0 .. j0 + tw (tw <= TC) of the nc columns; the
// point stride of U and V is NS.  rl: this lane also sums its rows of the
// load term R.
template <typename T, int TM, int TC, int NS>
__device__ __forceinline__ void vc_contract(const T* __restrict__ U, const T* __restrict__ V, const T* __restrict__ R,
                                            int cnt, int i0, int nr, int j0, int tw, int nc, bool rl,
                                            T (&acc)[TM][TC], T (&racc)[TM]) {
  for (int c = 0; c < cnt; ++c) {
    T u[TM], v[TC];
#pragma unroll
    for (int a = 0; a < TM; ++a) u[a] = i0 + a < nr ? U[c * NS + i0 + a] : T(0);
#pragma unroll
    for (int b = 0; b < TC; ++b) v[b] = b < tw && j0 + b < nc ? V[c * NS + j0 + b] : T(0);
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
      for (int b = 0; b < TC; ++b) acc[a][b] = fma(u[a], v[b], acc[a][b]);
    if (rl) {
      const T r = R[c];
#pragma unroll
      for (int a = 0; a < TM; ++a) racc[a] = fma(u[a], r, racc[a]);
    }
  }
}

// shared memory of one CTA: the volume rule, the basis scales, and per warp
// the staged rows U and V (32 points, stride NS) and the load terms R
template <int D, int P, typename T>
struct VcSmem {
  static constexpr int QT = ipow_c(P + 2, D);
  static constexpr int NM = nbasis(D, D == 2 ? kPMax2 : kPMax3);
  static constexpr int NS = NM | 1;  // odd point stride
  static constexpr int head = (QT * (D + 1) + NM + 1) / 2 * 2;  // T words, even (16-byte aligned for double)
  static constexpr int per_warp = 2 * 32 * NS + 32;
  static constexpr size_t bytes = sizeof(T) * (size_t)(head + kVcWarps * per_warp);
};


// One warp per element row of degree P (grid-strided over the degree group):
// the diagonal block (volume points, then the inflow points of each own
// face) and the load vector, then each off-diagonal block (the inflow points
// of the interface's faces).  Every value is ADDED to what the row kernels
// wrote; each entry by one lane.
template <int D, int P, typename T>
__global__ void __launch_bounds__(kVcWarps * 32)
    varcoef_kernel(const DevMesh m, const VcFields f, T* __restrict__ vals, T* __restrict__ rhs) {
  using SM = VcSmem<D, P, T>;
  constexpr int N = nbasis(D, P), QT = SM::QT, NM = SM::NM, NS = SM::NS, SV = sub_vals(D);
  constexpr int TM = (N + kVcTR - 1) / kVcTR;   // tile edge of the diagonal block
  constexpr int TK = (NM + kVcTR - 1) / kVcTR;  // widest column tile of an off-diagonal block
  constexpr int FV = side_vals(D), RS = hf_rec_vals(D);
  extern __shared__ __align__(16) unsigned char vc_smem[];
  T* rule = reinterpret_cast<T*>(vc_smem);
  T* ctab = rule + QT * (D + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  T* U = reinterpret_cast<T*>(vc_smem) + SM::head + (size_t)warp * SM::per_warp;
  T* V = U + 32 * NS;
  T* R = V + 32 * NS;
  {
    const T* vrule = pick<T>(m.rt.vol64, m.rt.vol32) + (size_t)m.rt.vol_off[P] * (D + 1);
    for (int i = threadIdx.x; i < QT * (D + 1); i += blockDim.x) rule[i] = vrule[i];
    fill_ctab<D, T>(ctab, NM);
  }
  __syncthreads();
  const T* SG = pick<T>(m.sg64, m.sg32);
  const T* HFR = pick<T>(m.hfr64, m.hfr32);
  const T* FR = pick<T>(m.rt.face64, m.rt.face32);
  const T* EG = pick<T>(m.eg64, m.eg32);
  const bool do_rhs = rhs != nullptr, src = m.pb.source != DG_SRC_ZERO;
  const int base = m.elem_pstart[P], count = m.elem_pstart[P + 1] - base;
  const int tr = lane / kVcTR, tc = lane - (lane / kVcTR) * kVcTR;
  const bool tl = lane < kVcTR * kVcTR;  // lanes 25..31 only stage
  T* Ur = U + lane * NS;
  T* Vr = V + lane * NS;

  for (int w = blockIdx.x * kVcWarps + warp; w < count; w += gridDim.x * kVcWarps) {
    const int e = m.elem_perm[base + w];
    ElemPar<D, T> q;
    load_elem_par<D, T>(m, e, q);
    T acc[TM][TM], racc[TM];
#pragma unroll
    for (int a = 0; a < TM; ++a) {
      racc[a] = T(0);
#pragma unroll
      for (int b = 0; b < TM; ++b) acc[a][b] = T(0);
    }
    // ---- volume points: U = Phi, V = W (b' . D + c Phi), R = W (b . grad u + c u)
    const int sub0 = m.eptr[e], nvol = (m.eptr[e + 1] - sub0) * QT;
    for (int c0 = 0; c0 < nvol; c0 += 32) {
      const int qv = c0 + lane;
      if (qv < nvol) {
        const int t = qv / QT, r = qv - t * QT;
        T sv[SV];
#pragma unroll
        for (int k = 0; k < SV; ++k) sv[k] = SG[(size_t)k * m.nsub + sub0 + t];
        const T* rr = rule + r * (D + 1);
        T xi[D], x[D], b[D];
#pragma unroll
        for (int d = 0; d < D; ++d) {
          T v = sv[d] + rr[0] * sv[D + d] + rr[1] * sv[2 * D + d];
          if constexpr (D == 3) v += rr[2] * sv[3 * D + d];
          xi[d] = v;
          x[d] = q.lo[d] + (xi[d] + T(1)) * T(0.5) * q.L[d];
        }
        const T W = rr[D] * sv[SV - 1];
        const T c = vc_fields_at<D, T>(f, x, b);
        T bs[D];
#pragma unroll
        for (int d = 0; d < D; ++d) bs[d] = W * b[d] * T(2) / q.L[d];  // W b_d 2 / L_d: physical derivative
        T Phi[N], Dd[D][N];
        basis_eval<D, P, T>(xi, Phi, Dd);
#pragma unroll
        for (int j = 0; j < N; ++j) {
          T v = W * c * Phi[j];
#pragma unroll
          for (int d = 0; d < D; ++d) v += bs[d] * Dd[d][j];
          Ur[j] = Phi[j];
          Vr[j] = v;
        }
        T rv = T(0);
        if (do_rhs && src) {
          T gu[3], lap;
          const T u = exact_u<D, T>(m.pb, x, gu, &lap);
          T bg = T(0);
#pragma unroll
          for (int d = 0; d < D; ++d) bg += b[d] * gu[d];
          rv = W * (bg + c * u);
        }
        R[lane] = rv;
      }
      __syncwarp();
      if (tl)
        vc_contract<T, TM, TM, NS>(U, V, R, min(32, nvol - c0), tr * TM, N, tc * TM, TM, N, do_rhs && tc == 0, acc,
                                   racc);
      __syncwarp();
    }
    // ---- own faces: U = Phi, V = -W min(b . n, 0) Phi; on Dirichlet
    // boundary faces R = -W min(b . n, 0) g.  Neumann faces: nothing.
    for (int h = m.hf_ptr[e]; h < m.hf_ptr[e + 1]; ++h) {
      const T* rec = HFR + (size_t)h * RS;
      const T J = rec[2 * FV], sig = rec[2 * FV + 1], nqs = rec[2 * FV + 3];
      if (sig < T(0)) continue;
      const bool bnd = nqs < T(0);
      const int nq = (int)(bnd ? -nqs : nqs);
      const int qf = D == 2 ? nq : nq * nq;
      for (int c0 = 0; c0 < qf; c0 += 32) {
        const int lq = c0 + lane;
        if (lq < qf) {
          const T* fr = FR + (size_t)(m.rt.face_off[nq] + lq) * (D == 2 ? 2 : 3);
          T xi[D], np[D], x[D], b[D];
          hf_point<D, T>(rec, fr, xi, np);
          const T W = fr[D == 2 ? 1 : 2] * J;
#pragma unroll
          for (int d = 0; d < D; ++d) x[d] = q.lo[d] + (xi[d] + T(1)) * T(0.5) * q.L[d];
          vc_fields_at<D, T>(f, x, b);
          T bn = T(0);
#pragma unroll
          for (int d = 0; d < D; ++d) bn += b[d] * np[d] * q.L[d];
          bn *= T(0.5);  // b . n_r, n_r = n' L / 2
          const T wu = bn < T(0) ? -W * bn : T(0);
          T Phi[N], Dd[D][N];
          basis_eval<D, P, T>(xi, Phi, Dd);
#pragma unroll
          for (int j = 0; j < N; ++j) {
            Ur[j] = Phi[j];
            Vr[j] = wu * Phi[j];
          }
          T rv = T(0);
          if (do_rhs && src && bnd && bn < T(0)) {
            T gu[3], lap;
            rv = wu * exact_u<D, T>(m.pb, x, gu, &lap);
          }
          R[lane] = rv;
        }
        __syncwarp();
        if (tl)
          vc_contract<T, TM, TM, NS>(U, V, R, min(32, qf - c0), tr * TM, N, tc * TM, TM, N, do_rhs && tc == 0, acc,
                                     racc);
        __syncwarp();
      }
    }
    if (tl && dg_in_range(m.status, m.blk_off[m.diag_blk[e]], (int64_t)N * N, m.nvals) &&
        (!do_rhs || dg_in_range(m.status, m.dof_off[e], N, m.ndofs))) {
      T* out = vals + m.blk_off[m.diag_blk[e]];
      const T RR = q.R * q.R;
#pragma unroll
      for (int a = 0; a < TM; ++a) {
        const int i = tr * TM + a;
        if (i >= N) continue;
#pragma unroll
        for (int b = 0; b < TM; ++b) {
          const int j = tc * TM + b;
          if (j < N) out[i * N + j] += RR * ctab[i] * ctab[j] * acc[a][b];
        }
        if (do_rhs && tc == 0) rhs[m.dof_off[e] + i] += q.R * ctab[i] * racc[a];
      }
    }
    // ---- off-diagonal blocks: U = Phi^r, V = W min(b . n_r, 0) Phi^k
    for (int bk = m.row_ptr[e]; bk < m.row_ptr[e + 1]; ++bk) {
      const int4 br = m.blk_rec[bk];  // k, first half face, faces, p_k
      if (br.x < 0) continue;         // the diagonal block
      const int nk = nbasis(D, br.w);
      const int tw = (nk + kVcTR - 1) / kVcTR;
      T ak[TM][TK], dummy[TM];
#pragma unroll
      for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int b = 0; b < TK; ++b) ak[a][b] = T(0);
      for (int fi = 0; fi < br.z; ++fi) {
        const T* rec = HFR + (size_t)(br.y + fi) * RS;
        const T J = rec[2 * FV], nqs = rec[2 * FV + 3];
        const int nq = (int)(nqs < T(0) ? -nqs : nqs);
        const int qf = D == 2 ? nq : nq * nq;
        for (int c0 = 0; c0 < qf; c0 += 32) {
          const int lq = c0 + lane;
          if (lq < qf) {
            const T* fr = FR + (size_t)(m.rt.face_off[nq] + lq) * (D == 2 ? 2 : 3);
            T xr[D], npr[D], xk[D], npk[D], x[D], b[D];
            hf_point<D, T>(rec, fr, xr, npr);
            hf_point<D, T>(rec + FV, fr, xk, npk);
            const T W = fr[D == 2 ? 1 : 2] * J;
#pragma unroll
            for (int d = 0; d < D; ++d) x[d] = q.lo[d] + (xr[d] + T(1)) * T(0.5) * q.L[d];
            vc_fields_at<D, T>(f, x, b);
            T bn = T(0);
#pragma unroll
            for (int d = 0; d < D; ++d) bn += b[d] * npr[d] * q.L[d];
            bn *= T(0.5);
            const T wu = bn < T(0) ? W * bn : T(0);
            T Phi[N], Dd[D][N];
            basis_eval<D, P, T>(xr, Phi, Dd);
#pragma unroll
            for (int j = 0; j < N; ++j) Ur[j] = Phi[j];
            vc_basis_values<D, T>(br.w, xk, Vr);
            for (int j = 0; j < nk; ++j) Vr[j] *= wu;
          }
          __syncwarp();
          if (tl)
            vc_contract<T, TM, TK, NS>(U, V, R, min(32, qf - c0), tr * TM, N, tc * tw, tw, nk, false, ak, dummy);
          __syncwarp();
        }
      }
      if (tl && dg_in_range(m.status, m.blk_off[bk], (int64_t)N * nk, m.nvals)) {
        T* out = vals + m.blk_off[bk];
        const T Rk = EG[(size_t)(3 * D) * m.ne + br.x];
        const T RR = q.R * Rk;
#pragma unroll
        for (int a = 0; a < TM; ++a) {
          const int i = tr * TM + a;
          if (i >= N) continue;
#pragma unroll
          for (int b = 0; b < TK; ++b) {
            const int j = tc * tw + b;
            if (b < tw && j < nk) out[i * nk + j] += RR * ctab[i] * ctab[j] * ak[a][b];
          }
        }
      }
    }
  }
}

// the launch of one degree group (grid: co-resident CTAs, grid-strided)
template <int D, int P, typename T>
int launch_varcoef_p(const DevMesh& m, const VcFields& f, T* vals, T* rhs, int sm_count, cudaStream_t st) {
  const int count = m.elem_pstart[P + 1] - m.elem_pstart[P];
  if (count <= 0) return 0;
  using SM = VcSmem<D, P, T>;
  static_assert(SM::bytes <= 227 * 1024, "variable-coefficient kernel shared memory exceeds 227 KB");
  auto k = varcoef_kernel<D, P, T>;
  if (SM::bytes > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::bytes);
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, kVcWarps * 32, SM::bytes);
  if (occ < 1) occ = 1;
  const int want = (count + kVcWarps - 1) / kVcWarps;
  const int grid = want < occ * sm_count ? want : occ * sm_count;
  k<<<grid, kVcWarps * 32, SM::bytes, st>>>(m, f, vals, rhs);
  return 1;
}

template <typename T>
int launch_varcoef_t(const DevMesh& m, const VcFields& f, T* vals, T* rhs, int sm_count, cudaStream_t st) {
  int n = 0;
  if (m.dim == 2) {
    n += launch_varcoef_p<2, 1, T>(m, f, vals, rhs, sm_count, st);
    n += launch_varcoef_p<2, 2, T>(m, f, vals, rhs, sm_count, st);
    n += launch_varcoef_p<2, 3, T>(m, f, vals, rhs, sm_count, st);
    n += launch_varcoef_p<2, 4, T>(m, f, vals, rhs, sm_count, st);
    n += launch_varcoef_p<2, 5, T>(m, f, vals, rhs, sm_count, st);
    n += launch_varcoef_p<2, 6, T>(m, f, vals, rhs, sm_count, st);
  } else {
    n += launch_varcoef_p<3, 1, T>(m, f, vals, rhs, sm_count, st);
    n += launch_varcoef_p<3, 2, T>(m, f, vals, rhs, sm_count, st);
    n += launch_varcoef_p<3, 3, T>(m, f, vals, rhs, sm_count, st);
    n += launch_varcoef_p<3, 4, T>(m, f, vals, rhs, sm_count, st);
  }
  return n;
}

int launch_varcoef_f64(const DevMesh& m, const VcFields& f, double* vals, double* rhs, int sm_count, cudaStream_t st);
int launch_varcoef_f32(const DevMesh& m, const VcFields& f, float* vals, float* rhs, int sm_count, cudaStream_t st);

}  // namespace dg
