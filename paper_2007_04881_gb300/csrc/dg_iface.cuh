// dg_iface.cuh -- off-diagonal blocks by interface.
//
// The two coupling blocks of an interface between elements A = e0 and B = e1
// (Eq. (2.4), face terms; Sec. 3.1, the four blocks of a face) are, with the
// points, weights and normals of A's half-face records (n out of A, DN =
// n' . grad_xi in each side's frame, upw = min(b.n, 0)):
//   A_AB = sum_q W [Phi_A (-a_B DN_B / 2 + (upw - sigma) Phi_B) + DN_A (a_A Phi_B / 2)],
//   A_BA = sum_q W [Phi_B (a_A DN_A / 2 - (sigma + max(b.n, 0)) Phi_A) + DN_B (-a_B Phi_A / 2)],
// i.e. A_AB = U_A^T V_B and A_BA = U_B^T V_A with U_s = [Phi_s; DN_s] and V_s
// the weighted rows of side s as the column side.  Each row of U and V
// depends on one side's basis only, so a staging lane evaluates one basis at
// one point: half of a chunk's lanes take side A, the other half side B, and
// each basis is evaluated once per point for both blocks (the row kernel
// evaluates both bases per point for each of the two blocks).  Each block is
// written by its interface's warp alone: deterministic, no atomics.
//
// Interfaces come grouped by their larger degree P (if_perm, if_pstart); the
// side of degree P evaluates the compiled basis, the other side dispatches
// on its degree.  imask holds the degrees whose block rows leave their
// off-diagonal blocks to this kernel (the moment launch completing their
// diagonal blocks); a group is launched when P is in imask, and of each
// interface the blocks of the rows whose degree is in imask are written (the
// block rows of the other degrees write their own).
#pragma once

#include "dg_device.cuh"

namespace dg {

// tile edge of the interface kernel for interfaces of larger degree P
template <int D, int P, typename T>
__host__ __device__ constexpr int iface_tm() {
  if (D == 2) return P == 1 ? 3 : P == 2 ? 3 : P == 3 ? 5 : P == 4 ? 8 : 7;
  return P == 1 ? 4 : P == 2 ? 5 : 4;
}

// Each thread owns a TM x TM tile position of the padded n x n grid.  With
// 2 TPB <= 32 the blocks AB and BA take separate threads (TPI = 2 TPB);
// otherwise one thread takes its tile of both (TPI = TPB).  G interfaces per
// warp; C points per interface per staged chunk (2D: the face's P + 1
// points, every 2D interface being one face; 3D: 16 / G, at least 1).
template <int D, int P, typename T>
struct IfaceCfg {
  static constexpr int N = nbasis(D, P);
  static constexpr int TM = iface_tm<D, P, T>();
  static constexpr int TR = (N + TM - 1) / TM;
  static constexpr int TPB = TR * TR;
  static constexpr bool SPLIT = 2 * TPB <= 32;
  static constexpr int TPI = SPLIT ? 2 * TPB : TPB;
  static constexpr int G = 32 / TPI;
  static constexpr int TMP = (TM + 1) / 2 * 2;
  static constexpr int ROW = TR * TMP;
  static constexpr int C = D == 2 ? P + 1 : (16 / G > 0 ? 16 / G : 1);
  static constexpr int PS = point_stride<T, TMP>(2 * ROW);  // staged point: two rows of ROW
  static constexpr int NI = 8;                              // int parameters per interface
  static constexpr int NF = 4;                              // T parameters per interface
  static constexpr int NMAXC = nbasis(D, D == 2 ? kPMax2 : kPMax3);
  static constexpr size_t head_bytes = align_up(sizeof(T) * NMAXC, 16);
  static constexpr size_t uv_bytes = align_up(sizeof(T) * (size_t)G * 2 * C * PS, 16);
  static constexpr size_t warp_bytes = 2 * uv_bytes + align_up(sizeof(T) * G * NF, 16) + align_up(sizeof(int) * G * NI, 16);
  static constexpr size_t total(int warps) { return head_bytes + warps * warp_bytes; }
};

// interface parameter slots
enum : int { kIfA = 0, kIfB, kIfBkAB, kIfBkBA, kIfHf0, kIfNpts, kIfPA, kIfPB };  // bk < 0: block not written here
enum : int { kIfAA = 0, kIfAB, kIfRA, kIfRB };

template <int D, int P, typename T>
__device__ __forceinline__ void iface_tile(const DevMesh& m, int imask, int i0, int nif, T* __restrict__ vals,
                                           int tile, const T* __restrict__ ctab, unsigned char* wb) {
  using Cfg = IfaceCfg<D, P, T>;
  constexpr int N = Cfg::N, TM = Cfg::TM, TR = Cfg::TR, TPB = Cfg::TPB, TPI = Cfg::TPI, G = Cfg::G;
  constexpr int TMP = Cfg::TMP, ROW = Cfg::ROW, C = Cfg::C, PS = Cfg::PS, NI = Cfg::NI, NF = Cfg::NF;
  constexpr bool SPLIT = Cfg::SPLIT;
  constexpr int FV = side_vals(D), RS = hf_rec_vals(D);
  constexpr int nq = P + 1, qf = D == 2 ? nq : nq * nq;  // face rule of the interface

  T* U = reinterpret_cast<T*>(wb);  // [G][2 sides][C][PS]
  T* V = reinterpret_cast<T*>(wb + Cfg::uv_bytes);
  T* FP = reinterpret_cast<T*>(wb + 2 * Cfg::uv_bytes);
  int* IP = reinterpret_cast<int*>(wb + 2 * Cfg::uv_bytes + align_up(sizeof(T) * G * NF, 16));
  const T* HFR = pick<T>(m.hfr64, m.hfr32);
  const T* FR = pick<T>(m.rt.face64, m.rt.face32) + (size_t)m.rt.face_off[nq] * (D == 2 ? 2 : 3);
  const T* EG = pick<T>(m.eg64, m.eg32);
  const int lane = threadIdx.x & 31;
  const int gcount = min(G, nif - tile * G);

  // ---- per-interface setup (one lane per interface).  A = e0 whose half-face
  // records are read, owned or not (a partition's ghost elements have their
  // records too), so that a block comes out bitwise the same in every mesh
  // that holds the interface
  __syncwarp();
  if (lane < G) {
    int* ip = IP + lane * NI;
    T* fp = FP + lane * NF;
    int npts = 0;
    if (lane < gcount) {
      // the interface's record (if_rec, in if_perm order): its elements, the
      // first half face on e0's side, its faces, both slots, both degrees
      const int k = i0 + tile * G + lane;
      const int4 r0 = m.if_rec[2 * k], r1 = m.if_rec[2 * k + 1];
      const int e0 = r0.x, e1 = r0.y;
      const int p0 = r1.z & 255, p1 = r1.z >> 8;
      // a block of the interface is written here when its row is owned and
      // its row's degree is in imask (slot -1: not owned)
      const int s01 = (imask >> p0) & 1 ? r1.x : -1, s10 = (imask >> p1) & 1 ? r1.y : -1;
      if (s01 >= 0 || s10 >= 0) {
        // the interface's faces are consecutive in e0's half-face list
        ip[kIfA] = e0;
        ip[kIfB] = e1;
        ip[kIfBkAB] = s01;
        ip[kIfBkBA] = s10;
        ip[kIfHf0] = r0.z;
        ip[kIfPA] = p0;
        ip[kIfPB] = p1;
        npts = r0.w * qf;
        fp[kIfAA] = T(m.a[e0]);
        fp[kIfAB] = T(m.a[e1]);
        fp[kIfRA] = EG[(size_t)(3 * D) * m.ne + e0];
        fp[kIfRB] = EG[(size_t)(3 * D) * m.ne + e1];
      }
    }
    ip[kIfNpts] = npts;
  }
  __syncwarp();
  int np_l = 0;
  if (lane < gcount) np_l = (IP[lane * NI + kIfNpts] + C - 1) / C;
  const int nch = __reduce_max_sync(0xffffffffu, np_l);

  // contraction roles: interface g_me, block bl (0: AB, 1: BA; both when
  // !SPLIT), tile (tr, tc)
  const int g_me = lane / TPI, r_me = lane % TPI;
  const int bl = SPLIT ? r_me / TPB : 0, tt = SPLIT ? r_me % TPB : r_me;
  const int tr = tt / TR, tc = tt % TR;
  const bool active = g_me < gcount && r_me < (SPLIT ? 2 * TPB : TPB);
  constexpr int NB = SPLIT ? 1 : 2;  // blocks per thread
  T acc[NB][TM][TM];
#pragma unroll
  for (int k = 0; k < NB; ++k)
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
      for (int b = 0; b < TM; ++b) acc[k][a][b] = T(0);

  for (int ch = 0; ch < nch; ++ch) {
    // ---- staging: one lane per (interface, side, point)
    for (int idx = lane; idx < G * 2 * C; idx += 32) {
      const int g = idx / (2 * C), rem = idx - g * (2 * C), s = rem / C, c = rem - s * C;
      const int qv = ch * C + c;
      T* Ur = U + (size_t)((g * 2 + s) * C + c) * PS;
      T* Vr = V + (size_t)((g * 2 + s) * C + c) * PS;
      const int* ip = IP + g * NI;
      if (g < gcount && qv < ip[kIfNpts]) {
        const T* fp = FP + g * NF;
        const int fi = qv / qf, lq = qv - fi * qf;
        const T* rec = HFR + (size_t)(ip[kIfHf0] + fi) * RS;
        const T* fr = FR + (size_t)lq * (D == 2 ? 2 : 3);
        T xi[D], np[D];
        hf_point<D, T>(rec + s * FV, fr, xi, np);
        const T W = fr[D == 2 ? 1 : 2] * rec[2 * FV];
        const T sig = rec[2 * FV + 1], bn = rec[2 * FV + 2];
        const T aA = fp[kIfAA], aB = fp[kIfAB];
        // V rows of side s as the column side: s = B (block AB):
        //   W [-a_B DN / 2 + (min(bn, 0) - sigma) Phi; a_A Phi / 2]
        // s = A (block BA): W [a_A DN / 2 - (sigma + max(bn, 0)) Phi; -a_B Phi / 2]
        const T c0 = s ? T(-0.5) * aB * W : T(0.5) * aA * W;
        const T c1 = s ? ((bn < T(0) ? bn : T(0)) - sig) * W : -(sig + (bn > T(0) ? bn : T(0))) * W;
        const T c2 = s ? T(0.5) * aA * W : T(-0.5) * aB * W;
        const int ps = s ? ip[kIfPB] : ip[kIfPA];
        if (ps == P) {
          T Phi[N], Dd[D][N], dn[N], v0[N], v1[N];
          basis_eval<D, P, T>(xi, Phi, Dd);
#pragma unroll
          for (int i = 0; i < N; ++i) {
            T v = T(0);
#pragma unroll
            for (int d = 0; d < D; ++d) v += np[d] * Dd[d][i];
            dn[i] = v;
            v0[i] = fma(c0, v, c1 * Phi[i]);
            v1[i] = c2 * Phi[i];
          }
          store_groups<T, N, TM, TMP, TR>(Ur, Phi);
          store_groups<T, N, TM, TMP, TR>(Ur + ROW, dn);
          store_groups<T, N, TM, TMP, TR>(Vr, v0);
          store_groups<T, N, TM, TMP, TR>(Vr + ROW, v1);
        } else {
          // lower degree: values at their tile positions; the padding past
          // n_s is never read into a written entry
          auto sink = [&](int j, T phi, const T* dk) {
            T v = T(0);
#pragma unroll
            for (int d = 0; d < D; ++d) v += np[d] * dk[d];
            const int o = (j / TM) * TMP + j % TM;
            Ur[o] = phi;
            Ur[ROW + o] = v;
            Vr[o] = fma(c0, v, c1 * phi);
            Vr[ROW + o] = c2 * phi;
          };
          nbr_basis<D, T>(ps, xi, sink);
        }
      } else {
        // both rows of U and V: a NaN pattern left in an unstaged slot times
        // a zero would be NaN
        zero_groups<T, TMP>(Ur, 2 * ROW);
        zero_groups<T, TMP>(Vr, 2 * ROW);
      }
    }
    __syncwarp();
    // ---- contraction over the chunk's points
    if (active) {
#pragma unroll 1
      for (int c = 0; c < C; ++c) {
#pragma unroll
        for (int k = 0; k < NB; ++k) {
          const int b = SPLIT ? bl : k;  // 0: AB = U_A^T V_B, 1: BA = U_B^T V_A
          const T* Ub = U + (size_t)((g_me * 2 + b) * C + c) * PS + tr * TMP;
          const T* Vb = V + (size_t)((g_me * 2 + (1 - b)) * C + c) * PS + tc * TMP;
#pragma unroll
          for (int t = 0; t < 2; ++t) {
            T u[TM], v[TM];
            load_tile<T, TM, TMP>(Ub + t * ROW, u);
            load_tile<T, TM, TMP>(Vb + t * ROW, v);
#pragma unroll
            for (int a = 0; a < TM; ++a)
#pragma unroll
              for (int bb = 0; bb < TM; ++bb) acc[k][a][bb] = fma(u[a], v[bb], acc[k][a][bb]);
          }
        }
      }
    }
    __syncwarp();
  }

  // ---- write: block AB (n_A x n_B) at slot AB, block BA (n_B x n_A) at slot BA
  if (active) {
    const int* ip = IP + g_me * NI;
    const T* fp = FP + g_me * NF;
    if (ip[kIfNpts] > 0) {
      const T RR = fp[kIfRA] * fp[kIfRB];
#pragma unroll
      for (int k = 0; k < NB; ++k) {
        const int b = SPLIT ? bl : k;
        const int bk = b == 0 ? ip[kIfBkAB] : ip[kIfBkBA];
        const int nr = nbasis(D, b == 0 ? ip[kIfPA] : ip[kIfPB]), nc = nbasis(D, b == 0 ? ip[kIfPB] : ip[kIfPA]);
        if (bk >= 0 && dg_in_range(m.status, m.blk_off[bk], (int64_t)nr * nc, m.nvals)) {
          T* out = vals + m.blk_off[bk];
#pragma unroll
          for (int a = 0; a < TM; ++a) {
            const int i = tr * TM + a;
            if (i < nr) {
              const T si = RR * ctab[i];
#pragma unroll
              for (int bb = 0; bb < TM; ++bb) {
                const int j = tc * TM + bb;
                if (j < nc) out[i * nc + j] = si * ctab[j] * acc[k][a][bb];
              }
            }
          }
        }
      }
    }
  }
}

// interfaces if_perm[i0 .. i1) of larger degree P
template <int D, int P, typename T>
__global__ void __launch_bounds__(kWarps * 32)
    iface_kernel(const DevMesh m, int imask, int i0, int i1, T* __restrict__ vals) {
  using Cfg = IfaceCfg<D, P, T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* ctab = reinterpret_cast<T*>(smem_raw);
  fill_ctab<D, T>(ctab, Cfg::NMAXC);
  __syncthreads();
  const int warp = threadIdx.x >> 5;
  unsigned char* wb = smem_raw + Cfg::head_bytes + warp * Cfg::warp_bytes;
  const int nif = i1 - i0, ntiles = (nif + Cfg::G - 1) / Cfg::G;
  for (int tile = blockIdx.x * kWarps + warp; tile < ntiles; tile += gridDim.x * kWarps)
    iface_tile<D, P, T>(m, imask, i0, nif, vals, tile, ctab, wb);
}

}  // namespace dg
