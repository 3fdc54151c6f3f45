// dg_learned.cu -- learned reduced quadrature for 2D elements.
//
// For an element mapped to its bounding box [-1,1]^2 a rule of 28 points and
// 28 weights is sought that reproduces the 28 moments of P_6 (exact for the
// p = 3 volume integrands with constant coefficients).  The paper motivates
// this by the cost of tailored polytope rules (Sec. 1) and of the
// sub-simplex rules it uses (Sec. 3).  Pipeline:
//   1. lq_prepare_kernel: exact moments of the Legendre products P_a P_b
//      and of the monomials, by the divergence theorem (FP64), and the
//      network input: the normalised vertex loop from a canonical vertex,
//      zero-padded to 12 vertices, in bfloat16;
//   2. the network (24 -> 128 -> 128 -> 84, tanh; bfloat16 operands, FP32
//      accumulation, mma.sync) proposes the points and weights;
//   3. lq_gn_kernel: minimum-norm Gauss-Newton on the moment equations in
//      FP64, one warp per element, a 28 x 28 Cholesky per step;
//   4. acceptance: monomial residual / area < 1e-10 and every point in the
//      bounding box; otherwise the element keeps its sub-triangle rule.
// The same Gauss-Newton, started from a fixed 4 x 7 tensor rule and run to
// convergence, produces the network's training targets.
#include <cuda_bf16.h>

#include <cstdint>

#include "dg_internal.h"

namespace dg {

namespace {

constexpr int LQ_DEG = 6;
constexpr int LQ_NM = 28;  // moments = points
constexpr int LQ_NV = 12;  // max vertices of an eligible element
constexpr int LQ_NIN = 24;
constexpr int LQ_STRIDE = 29;  // padded row of the per-warp tables

// P_0..P_DEG(+1) and derivatives at t
template <int N>
__device__ __forceinline__ void leg(double t, double* P, double* dP) {
  P[0] = 1.0;
  dP[0] = 0.0;
  P[1] = t;
  dP[1] = 1.0;
#pragma unroll
  for (int k = 1; k < N; ++k) {
    P[k + 1] = ((2 * k + 1) * t * P[k] - k * P[k - 1]) / (k + 1);
    dP[k + 1] = dP[k - 1] + (2 * k + 1) * P[k];
  }
}

// Legendre products in the order k = 0..6, j = 0..k: (k - j, j)
__device__ __forceinline__ void lq_lp(double x, double y, double* L, double* Lx, double* Ly) {
  double Px[LQ_DEG + 1], dPx[LQ_DEG + 1], Py[LQ_DEG + 1], dPy[LQ_DEG + 1];
  leg<LQ_DEG>(x, Px, dPx);
  leg<LQ_DEG>(y, Py, dPy);
  int i = 0;
#pragma unroll
  for (int k = 0; k <= LQ_DEG; ++k)
#pragma unroll
    for (int j = 0; j <= k; ++j) {
      const int a = k - j, b = j;
      L[i] = Px[a] * Py[b];
      Lx[i] = dPx[a] * Py[b];
      Ly[i] = Px[a] * dPy[b];
      ++i;
    }
}

__global__ void lq_prepare_kernel(DevMesh m, double* __restrict__ mom, double* __restrict__ mmom,
                                  __nv_bfloat16* __restrict__ feat, int* __restrict__ elig) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m.ne) return;
  const int b = m.eptr[e], nvx = m.eptr[e + 1] - b;
  const double lo0 = m.eg64[e], lo1 = m.eg64[(size_t)m.ne + e];
  const double il0 = m.eg64[(size_t)4 * m.ne + e], il1 = m.eg64[(size_t)5 * m.ne + e];
  // 4-point Gauss on [0,1] from the face tables (exact for the degree-7 edge integrands)
  const double* g4 = m.rt.face64 + (size_t)m.rt.face_off[4] * 2;
  double lm[LQ_NM], mm[LQ_NM];
  for (int k = 0; k < LQ_NM; ++k) lm[k] = mm[k] = 0.0;
  int start = 0;
  double best = -1e300, besty = -1e300;
  for (int i = 0; i < nvx; ++i) {
    const int v0 = m.eidx[b + i], v1 = m.eidx[b + (i + 1 == nvx ? 0 : i + 1)];
    const double x0 = 2.0 * (m.X[0][v0] - lo0) * il0 - 1.0, y0 = 2.0 * (m.X[1][v0] - lo1) * il1 - 1.0;
    const double x1 = 2.0 * (m.X[0][v1] - lo0) * il0 - 1.0, y1 = 2.0 * (m.X[1][v1] - lo1) * il1 - 1.0;
    if (x0 > best || (x0 == best && y0 > besty)) {
      best = x0;
      besty = y0;
      start = i;
    }
    const double dy = y1 - y0;  // n_xi ds of a CCW loop
    for (int q = 0; q < 4; ++q) {
      const double t = g4[2 * q], w = g4[2 * q + 1] * dy;
      const double xs = x0 + t * (x1 - x0), ys = y0 + t * dy;
      double Px[LQ_DEG + 2], dPx[LQ_DEG + 2], Py[LQ_DEG + 1], dPy[LQ_DEG + 1];
      leg<LQ_DEG + 1>(xs, Px, dPx);
      leg<LQ_DEG>(ys, Py, dPy);
      double xp[LQ_DEG + 2], yp[LQ_DEG + 1];
      xp[0] = 1.0;
      yp[0] = 1.0;
      for (int k = 1; k <= LQ_DEG + 1; ++k) xp[k] = xp[k - 1] * xs;
      for (int k = 1; k <= LQ_DEG; ++k) yp[k] = yp[k - 1] * ys;
      int i2 = 0;
      for (int k = 0; k <= LQ_DEG; ++k)
        for (int j = 0; j <= k; ++j) {
          const int a = k - j, bb = j;
          // antiderivative Q_a of P_a: Q_0 = xi, Q_a = (P_{a+1} - P_{a-1}) / (2a + 1)
          const double Qa = a == 0 ? xs : (Px[a + 1] - Px[a - 1]) / (2 * a + 1);
          lm[i2] += w * Qa * Py[bb];
          mm[i2] += w * xp[a + 1] / (a + 1) * yp[bb];
          ++i2;
        }
    }
  }
  for (int k = 0; k < LQ_NM; ++k) {
    mom[(size_t)e * LQ_NM + k] = lm[k];
    mmom[(size_t)e * LQ_NM + k] = mm[k];
  }
  elig[e] = nvx <= LQ_NV ? 1 : 0;
  for (int i = 0; i < LQ_NV; ++i) {
    float fx = 0.f, fy = 0.f;
    if (i < nvx) {
      const int v = m.eidx[b + (start + i) % nvx];
      fx = (float)(2.0 * (m.X[0][v] - lo0) * il0 - 1.0);
      fy = (float)(2.0 * (m.X[1][v] - lo1) * il1 - 1.0);
    }
    feat[(size_t)e * LQ_NIN + 2 * i] = __float2bfloat16_rn(fx);
    feat[(size_t)e * LQ_NIN + 2 * i + 1] = __float2bfloat16_rn(fy);
  }
}

// One warp per element.  z = (x[28], y[28], w[28]) in bounding-box
// coordinates; r_k = sum_i w_i L_k(p_i) - M_k; J = [w L_x, w L_y, L];
// dz = -J^T (J J^T)^-1 r.
constexpr int kGnWarps = 4;
struct GnSmem {
  double L[LQ_NM * LQ_STRIDE], Lx[LQ_NM * LQ_STRIDE], Ly[LQ_NM * LQ_STRIDE], A[LQ_NM * LQ_STRIDE];
  double z[3 * LQ_NM], r[LQ_NM], u[LQ_NM];
  int fail;
};

__global__ void __launch_bounds__(kGnWarps * 32)
    lq_gn_kernel(DevMesh m, const double* __restrict__ mom, const double* __restrict__ mmom,
                 const int* __restrict__ elig, const float* __restrict__ init, int iters, double* __restrict__ rule,
                 float* __restrict__ resid, int* __restrict__ ok) {
  extern __shared__ __align__(16) unsigned char raw[];
  GnSmem& S = reinterpret_cast<GnSmem*>(raw)[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  const int nwarps = gridDim.x * kGnWarps;
  for (int e = blockIdx.x * kGnWarps + (threadIdx.x >> 5); e < m.ne; e += nwarps) {
    const double* M = mom + (size_t)e * LQ_NM;
    const double area = mmom[(size_t)e * LQ_NM];
    // starting rule
    if (lane < LQ_NM) {
      double x, y, w;
      if (init) {
        const float* o = init + (size_t)e * 3 * LQ_NM;
        x = fmin(1.0, fmax(-1.0, (double)o[lane]));
        y = fmin(1.0, fmax(-1.0, (double)o[LQ_NM + lane]));
        w = area / LQ_NM * (1.0 + (double)o[2 * LQ_NM + lane]);
      } else {
        // 4 x 7 tensor Gauss points in [-0.9, 0.9]^2, weights scaled to the area
        const double* g4 = m.rt.face64 + (size_t)m.rt.face_off[4] * 2;
        const double* g7 = m.rt.face64 + (size_t)m.rt.face_off[7] * 2;
        const int ia = lane / 7, ib = lane % 7;
        x = 0.9 * (2.0 * g4[2 * ia] - 1.0);
        y = 0.9 * (2.0 * g7[2 * ib] - 1.0);
        w = g4[2 * ia + 1] * g7[2 * ib + 1] * area;
      }
      S.z[lane] = x;
      S.z[LQ_NM + lane] = y;
      S.z[2 * LQ_NM + lane] = w;
    }
    if (lane == 0) S.fail = 0;
    __syncwarp();
    for (int it = 0; it < iters; ++it) {
      if (lane < LQ_NM) {
        double L[LQ_NM], Lx[LQ_NM], Ly[LQ_NM];
        lq_lp(S.z[lane], S.z[LQ_NM + lane], L, Lx, Ly);
        for (int k = 0; k < LQ_NM; ++k) {
          S.L[lane * LQ_STRIDE + k] = L[k];
          S.Lx[lane * LQ_STRIDE + k] = Lx[k];
          S.Ly[lane * LQ_STRIDE + k] = Ly[k];
        }
      }
      __syncwarp();
      if (lane < LQ_NM) {
        double s = -M[lane];
        for (int q = 0; q < LQ_NM; ++q) s += S.z[2 * LQ_NM + q] * S.L[q * LQ_STRIDE + lane];
        S.r[lane] = s;
      }
      // J J^T (lower triangle): sum_q L_k L_l + w_q^2 (Lx_k Lx_l + Ly_k Ly_l)
      for (int idx = lane; idx < LQ_NM * (LQ_NM + 1) / 2; idx += 32) {
        int k = 0, rem = idx;
        while (rem > k) {
          rem -= k + 1;
          ++k;
        }
        const int l = rem;
        double s = 0.0;
        for (int q = 0; q < LQ_NM; ++q) {
          const double w = S.z[2 * LQ_NM + q];
          const double* Lq = S.L + q * LQ_STRIDE;
          const double* Xq = S.Lx + q * LQ_STRIDE;
          const double* Yq = S.Ly + q * LQ_STRIDE;
          s += Lq[k] * Lq[l] + w * w * (Xq[k] * Xq[l] + Yq[k] * Yq[l]);
        }
        S.A[k * LQ_STRIDE + l] = s;
      }
      __syncwarp();
      // Cholesky A = C C^T in place (lower), tiny diagonal shift for robustness
      if (lane == 0) {
        double tr = 0.0;
        for (int k = 0; k < LQ_NM; ++k) tr += S.A[k * LQ_STRIDE + k];
        const double shift = 1e-15 * tr / LQ_NM;
        for (int k = 0; k < LQ_NM; ++k) S.A[k * LQ_STRIDE + k] += shift;
      }
      for (int j = 0; j < LQ_NM; ++j) {
        __syncwarp();
        if (lane == 0) {
          const double d = S.A[j * LQ_STRIDE + j];
          if (!(d > 0.0)) S.fail = 1;
          S.A[j * LQ_STRIDE + j] = d > 0.0 ? sqrt(d) : 1.0;
        }
        __syncwarp();
        const int i = j + 1 + lane;
        if (i < LQ_NM) S.A[i * LQ_STRIDE + j] /= S.A[j * LQ_STRIDE + j];
        __syncwarp();
        if (i < LQ_NM) {
          const double aij = S.A[i * LQ_STRIDE + j];
          for (int k = j + 1; k <= i; ++k) S.A[i * LQ_STRIDE + k] -= aij * S.A[k * LQ_STRIDE + j];
        }
      }
      __syncwarp();
      if (lane == 0) {
        // C y = r, C^T u = y
        for (int i = 0; i < LQ_NM; ++i) {
          double s = S.r[i];
          for (int k = 0; k < i; ++k) s -= S.A[i * LQ_STRIDE + k] * S.u[k];
          S.u[i] = s / S.A[i * LQ_STRIDE + i];
        }
        for (int i = LQ_NM - 1; i >= 0; --i) {
          double s = S.u[i];
          for (int k = i + 1; k < LQ_NM; ++k) s -= S.A[k * LQ_STRIDE + i] * S.u[k];
          S.u[i] = s / S.A[i * LQ_STRIDE + i];
        }
      }
      __syncwarp();
      if (lane < LQ_NM) {
        double dx = 0.0, dy = 0.0, dw = 0.0;
        for (int k = 0; k < LQ_NM; ++k) {
          const double uk = S.u[k];
          dx += S.Lx[lane * LQ_STRIDE + k] * uk;
          dy += S.Ly[lane * LQ_STRIDE + k] * uk;
          dw += S.L[lane * LQ_STRIDE + k] * uk;
        }
        const double w = S.z[2 * LQ_NM + lane];
        S.z[lane] -= w * dx;
        S.z[LQ_NM + lane] -= w * dy;
        S.z[2 * LQ_NM + lane] -= dw;
      }
      __syncwarp();
    }
    // acceptance: monomial moments of the rule against the exact ones
    double err = 0.0;
    bool inside = true;
    if (lane < LQ_NM) {
      const int ks = lane;
      int k = 0, rem = ks;
      while (rem > k) {
        rem -= k + 1;
        ++k;
      }
      const int a = k - rem, bb = rem;
      double s = -mmom[(size_t)e * LQ_NM + ks];
      for (int q = 0; q < LQ_NM; ++q) {
        double xa = 1.0, yb = 1.0;
        for (int t = 0; t < a; ++t) xa *= S.z[q];
        for (int t = 0; t < bb; ++t) yb *= S.z[LQ_NM + q];
        s += S.z[2 * LQ_NM + q] * xa * yb;
      }
      err = fabs(s);
      inside = fabs(S.z[lane]) <= 1.0 && fabs(S.z[LQ_NM + lane]) <= 1.0;
    }
    // every lane executes both shuffles (no short-circuit around them)
    for (int o = 16; o > 0; o >>= 1) {
      const double e2 = __shfl_xor_sync(0xffffffffu, err, o);
      const int in2 = __shfl_xor_sync(0xffffffffu, inside ? 1 : 0, o);
      err = fmax(err, e2);
      inside = inside && in2 != 0;
    }
    const double rel = err / fabs(area);
    const bool good = !S.fail && elig[e] && inside && rel < 1e-10 && isfinite(rel);
    for (int q = lane; q < 3 * LQ_NM; q += 32) rule[(size_t)e * 3 * LQ_NM + q] = S.z[q];
    if (lane == 0) {
      resid[e] = (float)rel;
      ok[e] = good ? 1 : 0;
    }
    __syncwarp();
  }
}

// install accepted rules in the mesh's assembly tables: physical weight
// W = w_hat L_x L_y / 4 (the bounding-box map's Jacobian)
__global__ void lq_install_kernel(DevMesh m, const double* __restrict__ rule, const int* __restrict__ ok,
                                  double* __restrict__ lq64, float* __restrict__ lq32, int* __restrict__ lq_ok) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m.ne) return;
  const int use = ok[e];
  lq_ok[e] = use;
  const double jac = 0.25 * m.eg64[(size_t)2 * m.ne + e] * m.eg64[(size_t)3 * m.ne + e];
  for (int q = 0; q < 3 * LQ_NM; ++q) {
    double v = rule[(size_t)e * 3 * LQ_NM + q];
    if (q >= 2 * LQ_NM) v *= jac;
    lq64[(size_t)e * 3 * LQ_NM + q] = v;
    lq32[(size_t)e * 3 * LQ_NM + q] = (float)v;
  }
}

// training targets: (x, y, 28 w / area - 1) of a rule
__global__ void lq_targets_kernel(int ne, const double* __restrict__ rule, const double* __restrict__ mmom,
                                  float* __restrict__ tgt) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  const double area = mmom[(size_t)e * LQ_NM];
  for (int q = 0; q < 3 * LQ_NM; ++q) {
    double v = rule[(size_t)e * 3 * LQ_NM + q];
    if (q >= 2 * LQ_NM) v = v * LQ_NM / area - 1.0;
    tgt[(size_t)e * 3 * LQ_NM + q] = (float)v;
  }
}

inline int nb(int n, int t) { return (n + t - 1) / t; }

}  // namespace

void lq_prepare(const DevMesh& m, double* mom, double* mmom, void* feat, int* elig, cudaStream_t st) {
  lq_prepare_kernel<<<nb(m.ne, 128), 128, 0, st>>>(m, mom, mmom, static_cast<__nv_bfloat16*>(feat), elig);
}

void lq_gn(const DevMesh& m, const double* mom, const double* mmom, const int* elig, const float* init, int iters,
           double* rule, float* resid, int* ok, int sm_count, cudaStream_t st) {
  const size_t smem = sizeof(GnSmem) * kGnWarps;
  cudaFuncSetAttribute(lq_gn_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int occ = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, lq_gn_kernel, kGnWarps * 32, smem);
  int grid = nb(m.ne, kGnWarps);
  if (grid > occ * sm_count) grid = occ * sm_count;
  if (grid < 1) grid = 1;
  lq_gn_kernel<<<grid, kGnWarps * 32, smem, st>>>(m, mom, mmom, elig, init, iters, rule, resid, ok);
}

void lq_install(const DevMesh& m, const double* rule, const int* ok, double* lq64, float* lq32, int* lq_ok,
                cudaStream_t st) {
  lq_install_kernel<<<nb(m.ne, 128), 128, 0, st>>>(m, rule, ok, lq64, lq32, lq_ok);
}

void lq_targets(int ne, const double* rule, const double* mmom, float* tgt, cudaStream_t st) {
  lq_targets_kernel<<<nb(ne, 128), 128, 0, st>>>(ne, rule, mmom, tgt);
}

}  // namespace dg
