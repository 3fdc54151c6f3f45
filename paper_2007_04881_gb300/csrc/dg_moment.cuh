// dg_moment.cuh -- volume blocks through Legendre-product moments.
//
// The volume part of Eq. (2.4) for an element with constant a, b, c is a
// sum over the element's quadrature points (the sub-simplex rules of Sec. 3,
// or a learned rule) of products of two basis functions or their
// derivatives.  With the bounding-box basis phi_i = s_i P_a(xi) P_b(eta)
// (P_c(zeta)), every such product is a product, per coordinate, of two
// Legendre polynomials or their derivatives, and each of those is a short
// exact combination of Legendre polynomials (linearisation):
//   P_a P_a' = sum_c G(a, a', c) P_c,  P'_a P_a' = sum_c G1(a, a', c) P_c,
//   P'_a P'_a' = sum_c G2(a, a', c) P_c.
// So the quadrature sum factors through the weighted moments
//   mu_{c d (e)} = sum_q W_q P_c(xi_q) P_d(eta_q) (P_e(zeta_q)),  c + d (+ e) <= 2p,
// (the same rule, the same points, the same weights, added in another
// order), and each block entry is a fixed combination of moments:
//   2D: A_ij = sum_{c,d} mu_cd [Y0(d) Xa(c) + X0(c) Yb(d)],
//   3D: A_ij = sum_{c,d,e} mu_cde [Z0(e) (Y0(d) Xa(c) + X0(c) Yb(d)) + X0(c) Y0(d) Zs(e)],
// X0 = G(ai, aj), Xa = c G(ai, aj) + b'_1 G1(aj, ai) + a'_1 G2(ai, aj),
// Yb = b'_2 G1(bj, bi) + a'_2 G2(bi, bj), Zs = b'_3 G1(cj, ci) + a'_3 G2(ci, cj),
// with the trial function j carrying the advection derivative.  Per point
// this costs the moments (45 for 2D p = 4) instead of the 3 n^2 block
// updates; per element, the combination above, in 2D in two stages:
//   T(c, (bi,bj)) = sum_d mu_cd Y0(d),  U(c, (bi,bj)) = sum_d mu_cd Yb(d),
//   A_ij = sum_c [Xa(c) T(c, (bi,bj)) + X0(c) U(c, (bi,bj))].
// The load vector's volume term (non-polynomial f) is accumulated per point
// as before.
//
// Own-face terms (kModeMomFace).  On the element's faces the diagonal block
// gains sum_q W [(sigma - min(b.n, 0)) Phi_i Phi_j - kappa a (Phi_i DN_j +
// DN_i Phi_j)] with DN = n' . grad_xi: the derivative part is the normal
// derivative of the product Phi_i Phi_j, so with the same linearisation
//   A_ij += sum_{c,d(,e)} X0(c) Y0(d) (Z0(e)) F_cd(e),
//   F_cd = sum_q W [(sigma - upw) P_c P_d - kappa a (n'_1 P'_c P_d + n'_2 P_c P'_d)]
// (3D: one more derivative term), one moment set for all the faces of the
// element, summed over the face rule of each face (exact for the products,
// degree 2p along a face).  The boundary faces' load terms (Eq. (2.5): the
// Dirichlet data or the Neumann flux times Phi_i and DN_i) are added per
// point.  The row kernel then writes only the off-diagonal blocks.
//
// Layout: LPE lanes per element.  Each lane accumulates the moments and the
// load vector of every LPE-th point in registers; a butterfly reduction over
// the lanes gives the sums (a fixed order, no atomics).  The lanes then write
// the element's diagonal block (overwritten, or added with kModeAccum) and
// the volume part of its load vector; the row kernel adds the face terms.
#pragma once

#include "dg_device.cuh"

namespace dg {

// moments c + d (+ e) <= 2p, in total-degree order
template <int D>
__host__ __device__ constexpr int nmom(int q) {
  return D == 2 ? (q + 1) * (q + 2) / 2 : (q + 1) * (q + 2) * (q + 3) / 6;
}
// index of moment (c, d) / (c, d, e): s = total degree, t = d + e
__device__ __forceinline__ int mom2(int c, int d) {
  const int s = c + d;
  return s * (s + 1) / 2 + d;
}
__device__ __forceinline__ int mom3(int c, int d, int e) {
  const int s = c + d + e, t = d + e;
  return s * (s + 1) * (s + 2) / 6 + t * (t + 1) / 2 + e;
}

template <int D, int P, typename T>
struct MomCfg {
  static constexpr int N = nbasis(D, P);
  static constexpr int Q = 2 * P;
  static constexpr int NM = nmom<D>(Q);
  static constexpr int LPE = D == 2 ? (P <= 2 ? 8 : 16) : 32;  // lanes per element
  static constexpr int G = 32 / LPE;                             // elements per warp
  static constexpr int QT = ipow_c(P + 2, D);
  static constexpr int PL = kPMaxLin + 1;   // table stride: degrees 0..kPMaxLin
  static constexpr int CL = 2 * kPMaxLin + 1;
  static constexpr int NLIN = 3 * PL * PL * CL;  // G, G1, G2
  static constexpr int NPAIR = (P + 1) * (P + 1);
  // per element: moments, face moments, and three [NPAIR][Q+1] tables: Xa,
  // then in 2D the stage-one sums T and U, in 3D Yb and Zs
  static constexpr int PER_ELEM = 2 * NM + 3 * NPAIR * (Q + 1);
  static constexpr int NMAXC = nbasis(D, D == 2 ? kPMax2 : kPMax3);
  // the (P + 1)^3 entries of each [NPAIR][Q+1] coefficient table and of the
  // 2D stage-one sums that the block reads (MomLists)
  static constexpr int NX = (P + 1) * (P + 1) * (P + 1);
  // linearisation tables, rule, basis scales, the exponents of the degree's
  // basis functions (int, [N][3]), then the two entry lists (unsigned short)
  static constexpr size_t head_elems = NLIN + QT * (D + 1) + NMAXC + (3 * N * sizeof(int) + sizeof(T) - 1) / sizeof(T) +
                                       (2 * NX * sizeof(unsigned short) + sizeof(T) - 1) / sizeof(T);
  static constexpr size_t total = align_up(sizeof(T) * (head_elems + (size_t)kWarps * G * PER_ELEM), 16);
};

// The entries of the per-element tables that the block's entries read.  A
// coefficient table [pair (a, a')][c] (Xa; in 3D also Yb, Zs) is read at
// c <= a + a' only (c <= ai + aj): xl lists those (P + 1)^3 indices.  The 2D
// stage-one sums [c][pair (b, b')] are read at c <= ai + aj <= 2p - b - b'
// only: sl lists those (P + 1)^3 indices.  The lanes of an element take the
// lists instead of the whole tables (225 entries each at 2D p = 4, 125 of
// them read); the entries computed are the same, so are the blocks.
template <int D, int P>
__device__ inline void mom_lists(unsigned short* xl, unsigned short* sl, int tid, int nthreads) {
  constexpr int NP = (P + 1) * (P + 1), Q = 2 * P;
  for (int pr = tid; pr < NP; pr += nthreads) {
    const int a = pr / (P + 1), ap = pr - a * (P + 1);
    int bx = 0, bs = 0;  // entries of the pairs before pr in each list
    for (int q = 0; q < pr; ++q) {
      const int qa = q / (P + 1), qb = q - qa * (P + 1);
      bx += qa + qb + 1;
      bs += Q - qa - qb + 1;
    }
    for (int c = 0; c <= a + ap; ++c) xl[bx + c] = (unsigned short)(pr * (Q + 1) + c);
    for (int c = 0; c <= Q - a - ap; ++c) sl[bs + c] = (unsigned short)(c * NP + pr);
  }
}

// whether the moment path serves (D, P, T): moments held in registers
template <int D, int P, typename T>
__host__ __device__ constexpr bool moment_volume_ok() {
  return P >= 1 && P <= kPMaxLin && nmom<D>(2 * P) <= (sizeof(T) == 4 ? 96 : 56);
}

// One tile of the moment kernel: G elements of degree P on this warp, LPE
// lanes each.  lin, rule, ctab, alf: the linearisation tables, the degree's
// volume rule, the basis scales and exponents in shared memory; pw: the
// warp's per-element scratch (G * PER_ELEM values); wc: null, or the
// persistent pass's flags, set once an element's diagonal block and load
// vector are written.
template <int D, int P, typename T>
__device__ __forceinline__ void mom_tile(const DevMesh& m, int mode, T* __restrict__ vals, T* __restrict__ rhs,
                                         int tile, const T* __restrict__ lin, const T* __restrict__ rule,
                                         const T* __restrict__ ctab, const int* __restrict__ alf, T* pw,
                                         const WaitCtl* wc, const unsigned short* xl = nullptr,
                                         const unsigned short* sl = nullptr) {
  using Cfg = MomCfg<D, P, T>;
  constexpr int N = Cfg::N, Q = Cfg::Q, NM = Cfg::NM, LPE = Cfg::LPE, G = Cfg::G, QT = Cfg::QT;
  constexpr int PL = Cfg::PL, CL = Cfg::CL, NPAIR = Cfg::NPAIR;
  constexpr int SV = sub_vals(D);
  auto L0 = [&](int a, int b, int c) { return lin[(a * PL + b) * CL + c]; };
  auto L1 = [&](int a, int b, int c) { return lin[PL * PL * CL + (a * PL + b) * CL + c]; };
  auto L2 = [&](int a, int b, int c) { return lin[2 * PL * PL * CL + (a * PL + b) * CL + c]; };

  const T* SG = pick<T>(m.sg64, m.sg32);
  const bool mat_vol = mode & kModeVol, do_rhs = mode & kModeRhs, accum = mode & kModeAccum;
  // own-face terms here (the row kernel then writes the off-diagonal blocks only)
  const bool mface = mode & kModeMomFace;
  const bool mat_face = mface && (mode & kModeFace);
  const bool mat_any = mat_vol || mat_face;
  const int lane = threadIdx.x & 31;
  const int grp = lane / LPE, lig = lane % LPE;
  T* my = pw + (size_t)grp * Cfg::PER_ELEM;  // this element's scratch
  T* smu = my;
  T* sF = my + NM;                 // face moments
  T* sXa = sF + NM;                // [NPAIR][Q+1] per exponent pair (a, a') of dimension 0
  T* sYb = sXa + NPAIR * (Q + 1);  // 3D: dimension 1 [NPAIR][Q+1]; 2D: T [Q+1][NPAIR]
  T* sZs = sYb + NPAIR * (Q + 1);  // 3D: dimension 2 [NPAIR][Q+1]; 2D: U [Q+1][NPAIR]
  const int base = m.elem_pstart[P], count = m.elem_pstart[P + 1] - base;
  {
    const int slot = tile * G + grp;
    const bool active = slot < count;
    const int e = active ? m.elem_perm[base + slot] : 0;
    ElemPar<D, T> q;
    if (active) load_elem_par<D, T>(m, e, q);
    const bool lrn = D == 2 && active && m.lq_ok && m.lq_ok[e];  // learned rules are 2D
    const int npts = !active ? 0 : lrn ? 28 : (m.eptr[e + 1] - m.eptr[e]) * QT;

    // ---- moments and the load vector's volume term, LPE lanes per element
    T mu[NM], racc[N];
#pragma unroll
    for (int k = 0; k < NM; ++k) mu[k] = T(0);
#pragma unroll
    for (int i = 0; i < N; ++i) racc[i] = T(0);
    // exact moments (kModeExactMom): the points carry only the load vector
    const bool exact = active && (mode & kModeExactMom) && !lrn;
    const int npl = exact && !do_rhs ? 0 : npts;
    for (int qv = lig; qv < npl; qv += LPE) {
      T xi[D], W;
      if (D == 2 && lrn) {
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
      T Lv[3][Q + 1];
#pragma unroll
      for (int d = 0; d < D; ++d) {
        Lv[d][0] = T(1);
        Lv[d][1] = xi[d];
#pragma unroll
        for (int k = 1; k < Q; ++k)
          Lv[d][k + 1] = (T(2 * k + 1) / T(k + 1)) * xi[d] * Lv[d][k] - (T(k) / T(k + 1)) * Lv[d][k - 1];
      }
      if (mat_vol && !exact) {
        if constexpr (D == 2) {
#pragma unroll
          for (int c = 0; c <= Q; ++c) {
            const T wc = W * Lv[0][c];
#pragma unroll
            for (int d = 0; c + d <= Q; ++d) {
              const int s = c + d;
              mu[s * (s + 1) / 2 + d] = fma(wc, Lv[1][d], mu[s * (s + 1) / 2 + d]);
            }
          }
        } else {
#pragma unroll
          for (int c = 0; c <= Q; ++c) {
            const T wc = W * Lv[0][c];
#pragma unroll
            for (int d = 0; c + d <= Q; ++d) {
              const T wcd = wc * Lv[1][d];
#pragma unroll
              for (int ee = 0; c + d + ee <= Q; ++ee) {
                const int s = c + d + ee, t = d + ee;
                const int k = s * (s + 1) * (s + 2) / 6 + t * (t + 1) / 2 + ee;
                mu[k] = fma(wcd, Lv[2][ee], mu[k]);
              }
            }
          }
        }
      }
      if (do_rhs) {
        T x[D];
#pragma unroll
        for (int d = 0; d < D; ++d) x[d] = q.lo[d] + (xi[d] + T(1)) * T(0.5) * q.L[d];
        const T wf = W * source_f<D, T>(m.pb, q.a, x);
        // wf P_a P_b (P_c): the products over the trailing coordinates are
        // shared by the basis functions that have them
        T wy[P + 1], wyz[P + 1][P + 1];
#pragma unroll
        for (int j = 0; j <= P; ++j) wy[j] = wf * Lv[1][j];
        if constexpr (D == 3) {
#pragma unroll
          for (int l = 0; l <= P; ++l) {
            const T wz = wf * Lv[2][l];
#pragma unroll
            for (int j = 0; j + l <= P; ++j) wyz[l][j] = wz * Lv[1][j];
          }
        }
        int i = 0;
#pragma unroll
        for (int k = 0; k <= P; ++k) {
          if constexpr (D == 2) {
#pragma unroll
            for (int j = 0; j <= k; ++j) {
              racc[i] = fma(wy[j], Lv[0][k - j], racc[i]);
              ++i;
            }
          } else {
#pragma unroll
            for (int l = 0; l <= k; ++l)
#pragma unroll
              for (int j = 0; j <= k - l; ++j) {
                racc[i] = fma(wyz[l][j], Lv[0][k - j - l], racc[i]);
                ++i;
              }
          }
        }
      }
    }
    // exact moments by Green's theorem in the element's box coordinates:
    // mu_cd = (L_1 L_2 / 4) * closed integral over the loop (counter-clockwise)
    // of Q_c(xi) P_d(eta) d eta, with Q_c an antiderivative of P_c (Q_0 = P_1,
    // Q_c = (P_{c+1} - P_{c-1}) / (2c + 1)).  Along an edge the integrand has
    // degree c + 1 + d <= 2p + 1 in the edge parameter, so the (p + 1)-point
    // Gauss rule of the faces integrates it exactly.  The edge of sub-triangle
    // t runs from its second vertex to its third (the loop's v_t to v_{t+1}).
    if constexpr (D == 2) {
      if (exact && mat_vol) {
        const int sub0 = m.eptr[e], ned = m.eptr[e + 1] - sub0;
        const T* fr = pick<T>(m.rt.face64, m.rt.face32) + (size_t)m.rt.face_off[P + 1] * 2;
        const T jac = T(0.25) * q.L[0] * q.L[1];
        for (int ed = lig; ed < ned; ed += LPE) {
          T sv[SV];
#pragma unroll
          for (int k = 0; k < SV; ++k) sv[k] = SG[(size_t)k * m.nsub + sub0 + ed];
          const T deta = sv[5] - sv[3];
#pragma unroll 1
          for (int g = 0; g <= P; ++g) {
            const T t = fr[2 * g], w = fr[2 * g + 1] * deta * jac;
            const T x = sv[0] + (T(1) - t) * sv[2] + t * sv[4];
            const T y = sv[1] + (T(1) - t) * sv[3] + t * sv[5];
            T px[Q + 2], py[Q + 1];
            px[0] = py[0] = T(1);
            px[1] = x;
            py[1] = y;
#pragma unroll
            for (int k = 1; k <= Q; ++k) {
              px[k + 1] = (T(2 * k + 1) / T(k + 1)) * x * px[k] - (T(k) / T(k + 1)) * px[k - 1];
              if (k < Q) py[k + 1] = (T(2 * k + 1) / T(k + 1)) * y * py[k] - (T(k) / T(k + 1)) * py[k - 1];
            }
#pragma unroll
            for (int c = 0; c <= Q; ++c) {
              const T qc = c == 0 ? px[1] : (px[c + 1] - px[c - 1]) * (T(1) / T(2 * c + 1));
              const T wc = w * qc;
#pragma unroll
              for (int d = 0; c + d <= Q; ++d) {
                const int s = c + d;
                mu[s * (s + 1) / 2 + d] = fma(wc, py[d], mu[s * (s + 1) / 2 + d]);
              }
            }
          }
        }
      }
    }
    // exact moments in 3D by the divergence theorem with the field
    // (L_1 / 2) Q_c(xi) P_d(eta) P_e(zeta) e_1, whose divergence is
    // P_c P_d P_e: mu_cde = sum over the element's boundary triangles (its
    // half faces) of the integral of (L_1 / 2) n_1 Q_c P_d P_e dS, n the
    // physical unit normal out of the element (n_1 = n'_1 L_1 / 2 from the
    // record's scaled normal).  On a triangle the integrand has degree
    // c + 1 + d + e <= 2p + 1, so the collapsed rule with p + 2 points per
    // direction (exact to 2p + 2) integrates it exactly.
    if constexpr (D == 3) {
      if (exact && mat_vol) {
        constexpr int NQ = P + 2, QF = NQ * NQ;
        constexpr int FV = side_vals(3), RS = hf_rec_vals(3);
        const T* HFR = pick<T>(m.hfr64, m.hfr32);
        const T* fr0 = pick<T>(m.rt.face64, m.rt.face32) + (size_t)m.rt.face_off[NQ] * 3;
        const int h0 = m.hf_ptr[e], npt = (m.hf_ptr[e + 1] - h0) * QF;
        const T lx = T(0.25) * q.L[0] * q.L[0];
        for (int idx = lig; idx < npt; idx += LPE) {
          const int h = h0 + idx / QF, g = idx - (idx / QF) * QF;
          const T* rec = HFR + (size_t)h * RS;
          const T* fr = fr0 + 3 * g;
          T xi[3], np[3];
          hf_point<3, T>(rec, fr, xi, np);
          const T w = fr[2] * rec[2 * FV] * np[0] * lx;
          T px[Q + 2], py[Q + 1], pz[Q + 1];
          px[0] = py[0] = pz[0] = T(1);
          px[1] = xi[0];
          py[1] = xi[1];
          pz[1] = xi[2];
#pragma unroll
          for (int k = 1; k <= Q; ++k) {
            const T a1 = T(2 * k + 1) / T(k + 1), a0 = T(k) / T(k + 1);
            px[k + 1] = a1 * xi[0] * px[k] - a0 * px[k - 1];
            if (k < Q) {
              py[k + 1] = a1 * xi[1] * py[k] - a0 * py[k - 1];
              pz[k + 1] = a1 * xi[2] * pz[k] - a0 * pz[k - 1];
            }
          }
#pragma unroll
          for (int c = 0; c <= Q; ++c) {
            const T qc = c == 0 ? px[1] : (px[c + 1] - px[c - 1]) * (T(1) / T(2 * c + 1));
            const T wc = w * qc;
#pragma unroll
            for (int d = 0; c + d <= Q; ++d) {
              const T wcd = wc * py[d];
#pragma unroll
              for (int ee = 0; c + d + ee <= Q; ++ee) {
                const int s = c + d + ee, t = d + ee;
                const int k = s * (s + 1) * (s + 2) / 6 + t * (t + 1) / 2 + ee;
                mu[k] = fma(wcd, pz[ee], mu[k]);
              }
            }
          }
        }
      }
    }
    // butterfly sums over the element's lanes (fixed order); the volume
    // moments go to shared memory (zeros without kModeVol)
    if (mat_vol) {
#pragma unroll
      for (int off = LPE / 2; off > 0; off >>= 1) {
#pragma unroll
        for (int k = 0; k < NM; ++k) mu[k] += __shfl_xor_sync(0xffffffffu, mu[k], off);
      }
    }
    if (mat_any) {
      __syncwarp();
      if (active) {
#pragma unroll
        for (int k = 0; k < NM; ++k)
          if (k % LPE == lig) smu[k] = mu[k];
      }
    }

    // ---- own-face terms (kModeMomFace): face moments in the registers of mu,
    // boundary load terms into racc; one lane per face point
    if (mface && (mat_face || do_rhs)) {
      constexpr int FV = side_vals(D), RS = hf_rec_vals(D);
      const T* HFR = pick<T>(m.hfr64, m.hfr32);
      const T* FRb = pick<T>(m.rt.face64, m.rt.face32);
#pragma unroll
      for (int k = 0; k < NM; ++k) mu[k] = T(0);
      const int h0 = active ? m.hf_ptr[e] : 0;
      const int nhf = active ? m.hf_ptr[e + 1] - h0 : 0;
      const int nfp = active ? m.e_nqf[e] : 0;
      for (int qv = lig; qv < nfp; qv += LPE) {
        // the point's half face: the last one whose first point is <= qv
        int lo_ = h0, hi_ = h0 + nhf - 1;
        while (lo_ < hi_) {
          const int mid = (lo_ + hi_ + 1) >> 1;
          if (m.hf_qoff[mid] <= qv)
            lo_ = mid;
          else
            hi_ = mid - 1;
        }
        // own side, then J, sigma (-1: Neumann), b.n, nq (negative: boundary)
        const T* rec = HFR + (size_t)lo_ * RS;
        const T J = rec[2 * FV], s1 = rec[2 * FV + 1], bn = rec[2 * FV + 2], s3 = rec[2 * FV + 3];
        const bool bnd = s3 < T(0);
        if (!mat_face && !bnd) continue;  // an interior face has no load term
        const int nq = (int)(bnd ? -s3 : s3);
        const T* fr = FRb + (size_t)(m.rt.face_off[nq] + qv - m.hf_qoff[lo_]) * (D == 2 ? 2 : 3);
        T xi[D], np[D];
        hf_point<D, T>(rec, fr, xi, np);
        const T W = fr[D == 2 ? 1 : 2] * J;
        const bool neu = s1 < T(0);
        const T sig = neu ? T(0) : s1;
        const T kap = neu ? T(0) : bnd ? T(1) : T(0.5);
        const T upw = bn < T(0) ? bn : T(0);
        // P_0..P_q and P'_0..P'_q per coordinate (P'_{k+1} = P'_{k-1} + (2k+1) P_k)
        T Lv[3][Q + 1], dL[3][Q + 1];
#pragma unroll
        for (int d = 0; d < D; ++d) {
          Lv[d][0] = T(1);
          dL[d][0] = T(0);
          Lv[d][1] = xi[d];
          dL[d][1] = T(1);
#pragma unroll
          for (int k = 1; k < Q; ++k) {
            Lv[d][k + 1] = (T(2 * k + 1) / T(k + 1)) * xi[d] * Lv[d][k] - (T(k) / T(k + 1)) * Lv[d][k - 1];
            dL[d][k + 1] = fma(T(2 * k + 1), Lv[d][k], dL[d][k - 1]);
          }
        }
        if (mat_face) {
          const T w0 = W * (sig - upw);
          T wn[3];
#pragma unroll
          for (int d = 0; d < D; ++d) wn[d] = -W * kap * q.a * np[d];
          if constexpr (D == 2) {
            // F_cd += P_d (w0 P_c + wn_1 P'_c) + (wn_2 P_c) P'_d
#pragma unroll
            for (int c = 0; c <= Q; ++c) {
              const T A = fma(w0, Lv[0][c], wn[0] * dL[0][c]);
              const T B = wn[1] * Lv[0][c];
#pragma unroll
              for (int d = 0; c + d <= Q; ++d) {
                const int s = c + d, k = s * (s + 1) / 2 + d;
                mu[k] = fma(A, Lv[1][d], fma(B, dL[1][d], mu[k]));
              }
            }
          } else {
            // F_cde += P_e [P_d (w0 P_c + wn_1 P'_c) + wn_2 P_c P'_d] + (wn_3 P_c P_d) P'_e
#pragma unroll
            for (int c = 0; c <= Q; ++c) {
              const T A0 = fma(w0, Lv[0][c], wn[0] * dL[0][c]);
              const T B0 = Lv[0][c];
#pragma unroll
              for (int d = 0; c + d <= Q; ++d) {
                const T A = fma(A0, Lv[1][d], wn[1] * B0 * dL[1][d]);
                const T B = wn[2] * B0 * Lv[1][d];
#pragma unroll
                for (int ee = 0; c + d + ee <= Q; ++ee) {
                  const int s = c + d + ee, t = d + ee;
                  const int k = s * (s + 1) * (s + 2) / 6 + t * (t + 1) / 2 + ee;
                  mu[k] = fma(A, Lv[2][ee], fma(B, dL[2][ee], mu[k]));
                }
              }
            }
          }
        }
        if (do_rhs && bnd) {
          // Dirichlet: R0 = W (sigma - upw) g, R1 = -W a g; Neumann: R0 = W g_N,
          // g_N = a grad u . n (n = n' L / 2), R1 = 0; r_i += R0 Phi_i + R1 DN_i
          T x[D], gu[3], lap;
#pragma unroll
          for (int d = 0; d < D; ++d) x[d] = q.lo[d] + (xi[d] + T(1)) * T(0.5) * q.L[d];
          const T gd = exact_u<D, T>(m.pb, x, gu, &lap);
          T R0 = W * (sig - upw) * gd, R1 = -W * q.a * gd;
          if (neu) {
            T gn = T(0);
#pragma unroll
            for (int d = 0; d < D; ++d) gn += gu[d] * np[d] * q.L[d];
            R0 = W * T(0.5) * q.a * gn;
            R1 = T(0);
          }
          T ax[P + 1];
#pragma unroll
          for (int a = 0; a <= P; ++a) ax[a] = fma(R0, Lv[0][a], R1 * np[0] * dL[0][a]);
          int i = 0;
#pragma unroll
          for (int k = 0; k <= P; ++k) {
            if constexpr (D == 2) {
#pragma unroll
              for (int j = 0; j <= k; ++j) {
                const int a = k - j;
                racc[i] = fma(ax[a], Lv[1][j], fma(R1 * np[1] * Lv[0][a], dL[1][j], racc[i]));
                ++i;
              }
            } else {
#pragma unroll
              for (int l = 0; l <= k; ++l)
#pragma unroll
                for (int j = 0; j <= k - l; ++j) {
                  const int a = k - j - l;
                  const T yz1 = R1 * fma(np[1], dL[1][j] * Lv[2][l], np[2] * Lv[1][j] * dL[2][l]);
                  racc[i] = fma(ax[a], Lv[1][j] * Lv[2][l], fma(Lv[0][a], yz1, racc[i]));
                  ++i;
                }
            }
          }
        }
      }
      if (mat_face) {
#pragma unroll
        for (int off = LPE / 2; off > 0; off >>= 1) {
#pragma unroll
          for (int k = 0; k < NM; ++k) mu[k] += __shfl_xor_sync(0xffffffffu, mu[k], off);
        }
        if (active) {
#pragma unroll
          for (int k = 0; k < NM; ++k)
            if (k % LPE == lig) sF[k] = mu[k];
        }
      }
    }
    if (do_rhs) {
#pragma unroll
      for (int off = LPE / 2; off > 0; off >>= 1) {
#pragma unroll
        for (int i = 0; i < N; ++i) racc[i] += __shfl_xor_sync(0xffffffffu, racc[i], off);
      }
    }

    // ---- load vector (volume term): overwritten
    if (active && do_rhs && dg_in_range(m.status, m.dof_off[e], N, m.ndofs)) {
      T* out = rhs + m.dof_off[e];
#pragma unroll
      for (int i = 0; i < N; ++i)
        if (i % LPE == lig) out[i] = q.R * ctab[i] * racc[i];
    }

    // ---- diagonal block from the moments
    if (mat_any) {
      __syncwarp();
      if (active) {
        // per exponent pair (a, a'): the element's coefficient combinations
        auto xa_entry = [&](int k) {
          const int pr = k / (Q + 1), c = k - pr * (Q + 1);
          const int a = pr / (P + 1), ap = pr - a * (P + 1);
          sXa[k] = q.c * L0(a, ap, c) + q.bp[0] * L1(ap, a, c) + q.ap[0] * L2(a, ap, c);
          if constexpr (D == 3) {
            sYb[k] = q.bp[1 % D] * L1(ap, a, c) + q.ap[1 % D] * L2(a, ap, c);
            sZs[k] = q.bp[2 % D] * L1(ap, a, c) + q.ap[2 % D] * L2(a, ap, c);
          }
        };
        if (xl) {
          for (int t = lig; t < Cfg::NX; t += LPE) xa_entry(xl[t]);
        } else {
          for (int k = lig; k < NPAIR * (Q + 1); k += LPE) xa_entry(k);
        }
      }
      if constexpr (D == 2) {
        __syncwarp();
        // stage one: T(c, pair) and U(c, pair) over d <= b + b', c + d <= 2p
        if (active) {
          const int nst = sl ? Cfg::NX : NPAIR * (Q + 1);
          for (int t = lig; t < nst; t += LPE) {
            const int k = sl ? sl[t] : t;
            const int c = k / NPAIR, pr = k - c * NPAIR;
            const int b = pr / (P + 1), bp = pr - b * (P + 1);
            const int dm = min(b + bp, Q - c);
            const T* g0 = lin + (b * PL + bp) * CL;                  // G(b, b', d)
            const T* g1 = lin + PL * PL * CL + (bp * PL + b) * CL;   // G1(b', b, d)
            const T* g2 = lin + 2 * PL * PL * CL + (b * PL + bp) * CL;  // G2(b, b', d)
            int mi = c * (c + 1) / 2;  // moment (c, 0); (c, d + 1) is c + d + 2 further
            T t0 = T(0), u0 = T(0);
            if (mat_face) {
              // the face moments enter with X0(c) Y0(d), beside the volume's X0(c) Yb(d)
              for (int d = 0; d <= dm; ++d) {
                const T mu_cd = smu[mi], f_cd = sF[mi];
                mi += c + d + 2;
                t0 = fma(mu_cd, g0[d], t0);
                u0 = fma(mu_cd, q.bp[1] * g1[d] + q.ap[1] * g2[d], fma(f_cd, g0[d], u0));
              }
            } else {
              for (int d = 0; d <= dm; ++d) {
                const T mu_cd = smu[mi];
                mi += c + d + 2;
                t0 = fma(mu_cd, g0[d], t0);
                u0 = fma(mu_cd, q.bp[1] * g1[d] + q.ap[1] * g2[d], u0);
              }
            }
            sYb[k] = t0;
            sZs[k] = u0;
          }
        }
      }
      __syncwarp();
      if (active && dg_in_range(m.status, m.blk_off[m.diag_blk[e]], (int64_t)N * N, m.nvals)) {
        T* out = vals + m.blk_off[m.diag_blk[e]];
        const T RR = q.R * q.R;
        for (int ent = lig; ent < N * N; ent += LPE) {
          const int i = ent / N, j = ent - (ent / N) * N;
          const int ai[3] = {alf[3 * i], alf[3 * i + 1], alf[3 * i + 2]};
          const int aj[3] = {alf[3 * j], alf[3 * j + 1], alf[3 * j + 2]};
          T acc = T(0);
          const int px = ai[0] * (P + 1) + aj[0], py = ai[1] * (P + 1) + aj[1];
          const int cmax = ai[0] + aj[0], dmax = ai[1] + aj[1];
          if constexpr (D == 2) {
            (void)dmax;
            const T* xa = sXa + px * (Q + 1);
            const T* x0 = lin + (ai[0] * PL + aj[0]) * CL;
            const T* tt = sYb + py;
            const T* uu = sZs + py;
            for (int c = 0; c <= cmax; ++c)
              acc = fma(xa[c], tt[c * NPAIR], fma(x0[c], uu[c * NPAIR], acc));
          } else {
            const int pz = ai[2] * (P + 1) + aj[2], emax = ai[2] + aj[2];
            for (int c = 0; c <= cmax; ++c) {
              const T x0 = L0(ai[0], aj[0], c), xa = sXa[px * (Q + 1) + c];
              for (int d = 0; d <= dmax; ++d) {
                const T y0 = L0(ai[1], aj[1], d);
                const T k1 = y0 * xa + x0 * sYb[py * (Q + 1) + d], k2 = x0 * y0;
                T s = T(0);
                if (mat_face) {
                  for (int ee = 0; ee <= emax; ++ee) {
                    const int k = mom3(c, d, ee);
                    const T z0 = L0(ai[2], aj[2], ee);
                    s = fma(smu[k], z0 * k1 + sZs[pz * (Q + 1) + ee] * k2, fma(sF[k], z0 * k2, s));
                  }
                } else {
                  for (int ee = 0; ee <= emax; ++ee)
                    s = fma(smu[mom3(c, d, ee)], L0(ai[2], aj[2], ee) * k1 + sZs[pz * (Q + 1) + ee] * k2, s);
                }
                acc += s;
              }
            }
          }
          const T v = RR * ctab[i] * ctab[j] * acc;
          out[i * N + j] = accum ? out[i * N + j] + v : v;
        }
      }
    }
    if (wc) {
      // every lane's writes of the two elements before the flags
      __threadfence();
      __syncwarp();
      if (active && lig == 0) st_release(const_cast<int*>(wc->vdone) + e, 1);
    }
  }
}

template <int D, int P, typename T>
__global__ void __launch_bounds__(kWarps * 32)
    vol_moment_kernel(const DevMesh m, int mode, T* __restrict__ vals, T* __restrict__ rhs) {
  using Cfg = MomCfg<D, P, T>;
  constexpr int N = Cfg::N, G = Cfg::G, QT = Cfg::QT, NLIN = Cfg::NLIN;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* lin = reinterpret_cast<T*>(smem_raw);  // [3][PL][PL][CL]
  T* rule = lin + NLIN;
  T* ctab = rule + QT * (D + 1);
  int* alf = reinterpret_cast<int*>(ctab + Cfg::NMAXC);       // exponents [N][3]
  unsigned short* xl = reinterpret_cast<unsigned short*>(alf + 3 * N);  // entry lists [NX], [NX]
  unsigned short* sl = xl + Cfg::NX;
  T* pe = reinterpret_cast<T*>(smem_raw) + Cfg::head_elems;  // per element scratch
  const T* glin = pick<T>(m.rt.lin64, m.rt.lin32);
  for (int i = threadIdx.x; i < NLIN; i += blockDim.x) lin[i] = glin[i];
  const T* vrule = pick<T>(m.rt.vol64, m.rt.vol32) + (size_t)m.rt.vol_off[P] * (D + 1);
  for (int i = threadIdx.x; i < QT * (D + 1); i += blockDim.x) rule[i] = vrule[i];
  fill_ctab<D, T>(ctab, Cfg::NMAXC);
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    int al[3] = {0, 0, 0};
    basis_alpha<D>(i, al);
    alf[3 * i] = al[0];
    alf[3 * i + 1] = al[1];
    alf[3 * i + 2] = al[2];
  }
  mom_lists<D, P>(xl, sl, threadIdx.x, blockDim.x);
  __syncthreads();
  const int warp = threadIdx.x >> 5;
  T* pw = pe + (size_t)warp * G * Cfg::PER_ELEM;
  const int count = m.elem_pstart[P + 1] - m.elem_pstart[P];
  const int ngroups = (count + G - 1) / G;
  for (int tile = blockIdx.x * kWarps + warp; tile < ngroups; tile += gridDim.x * kWarps)
    mom_tile<D, P, T>(m, mode, vals, rhs, tile, lin, rule, ctab, alf, pw, nullptr, xl, D == 2 ? sl : nullptr);
}

}  // namespace dg
