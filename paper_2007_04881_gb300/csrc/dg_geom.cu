// dg_geom.cu -- geometry kernels (FP64): element bounding boxes, centroids,
// measures and diameters; sub-simplex maps in bounding-box coordinates;
// face normals, measures, per-side maps and penalties.
//
// Subdivision (Sec. 3 intro): 2D elements are split into the triangles
// (centroid, v_i, v_{i+1}) of their CCW loop; 3D elements are the union of
// their tetrahedra.  h_k = diam(k) (Sec. 2.2).  Penalty: the simplified form
// of Appendix A, sigma_F = C_sigma max_k a_k p_k^2 / h_k over F's elements.
#include "dg_internal.h"

namespace dg {

namespace {

// bounding-box coordinate xi = 2 (x - lo) / L - 1, with iL = 1/L precomputed
__device__ __forceinline__ double xi_of(double x, double lo, double iL) { return 2.0 * (x - lo) * iL - 1.0; }

template <int D>
__global__ void elem_geom_kernel(DevMesh m) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m.ne) return;
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  double vol = 0.0, cen[3] = {0.0, 0.0, 0.0};
  // 2D loops of up to KV vertices are loaded once (all loads issued before
  // use); longer loops read the vertex arrays directly
  constexpr int KV = 16;
  double vx[D == 2 ? KV : 1], vy[D == 2 ? KV : 1];
  int kv = 0;
  if (D == 2) {
    const int b = m.eptr[e], k = m.eptr[e + 1] - b;
    if (k <= KV) {
      int vi[KV];
#pragma unroll
      for (int i = 0; i < KV; ++i) vi[i] = i < k ? m.eidx[b + i] : 0;
#pragma unroll
      for (int i = 0; i < KV; ++i)
        if (i < k) {
          vx[i] = m.X[0][vi[i]];
          vy[i] = m.X[1][vi[i]];
        }
      kv = k;
    }
    for (int i = 0; i < k; ++i) {
      const int i1 = i + 1 == k ? 0 : i + 1;
      double x0, y0, x1, y1;
      if (kv) {
        x0 = vx[i];
        y0 = vy[i];
        x1 = vx[i1];
        y1 = vy[i1];
      } else {
        const int v0 = m.eidx[b + i], v1 = m.eidx[b + i1];
        x0 = m.X[0][v0];
        y0 = m.X[1][v0];
        x1 = m.X[0][v1];
        y1 = m.X[1][v1];
      }
      const double cr = x0 * y1 - x1 * y0;
      vol += 0.5 * cr;
      cen[0] += (x0 + x1) * cr;
      cen[1] += (y0 + y1) * cr;
    }
    const double i6v = 1.0 / (6.0 * vol);
    cen[0] *= i6v;
    cen[1] *= i6v;
  } else {
    for (int t = m.eptr[e]; t < m.eptr[e + 1]; ++t) {
      double P[4][3];
      for (int i = 0; i < 4; ++i) {
        const int v = m.eidx[4 * t + i];
        for (int d = 0; d < 3; ++d) P[i][d] = m.X[d][v];
      }
      double u[3], v[3], w[3];
      for (int d = 0; d < 3; ++d) {
        u[d] = P[1][d] - P[0][d];
        v[d] = P[2][d] - P[0][d];
        w[d] = P[3][d] - P[0][d];
      }
      const double det = u[0] * (v[1] * w[2] - v[2] * w[1]) - u[1] * (v[0] * w[2] - v[2] * w[0]) +
                         u[2] * (v[0] * w[1] - v[1] * w[0]);
      const double tv = fabs(det) / 6.0;
      vol += tv;
      for (int d = 0; d < 3; ++d) cen[d] += tv * 0.25 * (P[0][d] + P[1][d] + P[2][d] + P[3][d]);
    }
    for (int d = 0; d < 3; ++d) cen[d] /= vol;
  }
  // bounding box and diameter over the element's distinct vertices.  The
  // largest squared distance is found in FP32, then every pair within a
  // relative 1e-5 of it is re-measured in FP64: the FP64 maximum is among
  // them, so h is the exact FP64 diameter at a fraction of the FP64 work.
  const int ub = m.uvptr[e], ue = m.uvptr[e + 1];
  float h2f = 0.f;
  double h2 = 0.0;
  if (D == 2 && kv) {
    // the 2D loop's vertices are the element's distinct vertices
    float fx[KV], fy[KV];
    for (int i = 0; i < kv; ++i) {
      lo[0] = fmin(lo[0], vx[i]);
      hi[0] = fmax(hi[0], vx[i]);
      lo[1] = fmin(lo[1], vy[i]);
      hi[1] = fmax(hi[1], vy[i]);
      fx[i] = (float)vx[i];
      fy[i] = (float)vy[i];
    }
    for (int i = 0; i < kv; ++i)
      for (int j = i + 1; j < kv; ++j) {
        const float dx = fx[j] - fx[i], dy = fy[j] - fy[i];
        h2f = fmaxf(h2f, fmaf(dx, dx, dy * dy));
      }
    const float cut = h2f * (1.0f - 1e-5f);
    for (int i = 0; i < kv; ++i)
      for (int j = i + 1; j < kv; ++j) {
        const float dx = fx[j] - fx[i], dy = fy[j] - fy[i];
        if (fmaf(dx, dx, dy * dy) < cut) continue;
        const double ddx = vx[j] - vx[i], ddy = vy[j] - vy[i];
        h2 = fmax(h2, ddx * ddx + ddy * ddy);
      }
  } else {
  for (int i = ub; i < ue; ++i) {
    const int vi = m.uvidx[i];
    float pf[3];
    for (int d = 0; d < D; ++d) {
      const double x = m.X[d][vi];
      lo[d] = fmin(lo[d], x);
      hi[d] = fmax(hi[d], x);
      pf[d] = (float)x;
    }
    for (int j = i + 1; j < ue; ++j) {
      const int vj = m.uvidx[j];
      float sf = 0.f;
      for (int d = 0; d < D; ++d) {
        const float df = (float)m.X[d][vj] - pf[d];
        sf = fmaf(df, df, sf);
      }
      h2f = fmaxf(h2f, sf);
    }
  }
  const float cut = h2f * (1.0f - 1e-5f);
  for (int i = ub; i < ue; ++i) {
    const int vi = m.uvidx[i];
    for (int j = i + 1; j < ue; ++j) {
      const int vj = m.uvidx[j];
      float sf = 0.f;
      for (int d = 0; d < D; ++d) {
        const float df = (float)m.X[d][vj] - (float)m.X[d][vi];
        sf = fmaf(df, df, sf);
      }
      if (sf < cut) continue;
      double s2 = 0.0;
      for (int d = 0; d < D; ++d) {
        const double df = m.X[d][vj] - m.X[d][vi];
        s2 += df * df;
      }
      h2 = fmax(h2, s2);
    }
  }
  }
  for (int d = 0; d < D; ++d) {
    m.lo[d * m.ne + e] = lo[d];
    m.L[d * m.ne + e] = hi[d] - lo[d];
    m.cen[d * m.ne + e] = cen[d];
  }
  m.vol[e] = vol;
  const double h = sqrt(h2);
  m.h[e] = h;
  const int pe = m.p[e];
  m.pen[e] = m.a[e] * pe * pe / h;  // a_k p_k^2 / h_k of the penalty
  // contraction-precision record: lo, L, 1/L, R = 1/sqrt(|bbox|) (the basis
  // scale is s_i = R prod_d sqrt(2 alpha_d + 1))
  constexpr int EV = elem_vals(D);
  double rec[EV];
  double box = 1.0;
  for (int d = 0; d < D; ++d) {
    const double L = hi[d] - lo[d];
    rec[d] = lo[d];
    rec[D + d] = L;
    rec[2 * D + d] = 1.0 / L;
    box *= L;
  }
  rec[3 * D] = 1.0 / sqrt(box);
  for (int k = 0; k < EV; ++k) {
    m.eg64[(size_t)k * m.ne + e] = rec[k];
    m.eg32[(size_t)k * m.ne + e] = (float)rec[k];
  }
}

// 3D element records, one warp per element: an agglomerated polyhedron has
// tens of tetrahedra and distinct vertices, so the lanes share the tetrahedra
// (volume, centroid), the vertices (bounding box) and the vertex pairs
// (diameter: FP32 prefilter, FP64 recheck within 1e-5 of the maximum), and
// combine them with butterfly reductions in a fixed order.
__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_min(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

constexpr int kGeomWarps = 4;    // warps per block of the 3D element kernel
constexpr int kGeomVerts = 128;  // distinct vertices staged in shared memory per element

__global__ void __launch_bounds__(kGeomWarps * 32) elem_geom3d_warp_kernel(DevMesh m) {
  // FP32 copies of the element's distinct vertices for the diameter prefilter
  __shared__ float sv[kGeomWarps][3][kGeomVerts];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; e < m.ne; e += nw) {
    double vol = 0.0, cen[3] = {0.0, 0.0, 0.0};
    for (int t = m.eptr[e] + lane; t < m.eptr[e + 1]; t += 32) {
      double P[4][3];
      for (int i = 0; i < 4; ++i) {
        const int v = m.eidx[4 * t + i];
        for (int d = 0; d < 3; ++d) P[i][d] = m.X[d][v];
      }
      double u[3], v[3], w[3];
      for (int d = 0; d < 3; ++d) {
        u[d] = P[1][d] - P[0][d];
        v[d] = P[2][d] - P[0][d];
        w[d] = P[3][d] - P[0][d];
      }
      const double det = u[0] * (v[1] * w[2] - v[2] * w[1]) - u[1] * (v[0] * w[2] - v[2] * w[0]) +
                         u[2] * (v[0] * w[1] - v[1] * w[0]);
      const double tv = fabs(det) / 6.0;
      vol += tv;
      for (int d = 0; d < 3; ++d) cen[d] += tv * 0.25 * (P[0][d] + P[1][d] + P[2][d] + P[3][d]);
    }
    vol = warp_sum(vol);
    for (int d = 0; d < 3; ++d) cen[d] = warp_sum(cen[d]) / vol;
    const int ub = m.uvptr[e], ue = m.uvptr[e + 1], nu = ue - ub;
    const bool staged = nu <= kGeomVerts;
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int i = lane; i < nu; i += 32) {
      const int vi = m.uvidx[ub + i];
      for (int d = 0; d < 3; ++d) {
        const double x = m.X[d][vi];
        lo[d] = fmin(lo[d], x);
        hi[d] = fmax(hi[d], x);
        if (staged) sv[wib][d][i] = (float)x;
      }
    }
    for (int d = 0; d < 3; ++d) {
      lo[d] = warp_min(lo[d]);
      hi[d] = warp_max(hi[d]);
    }
    __syncwarp();
    // FP32 coordinate d of distinct vertex i (staged copy, or the vertex array)
    auto xf = [&](int d, int i) -> float { return staged ? sv[wib][d][i] : (float)m.X[d][m.uvidx[ub + i]]; };
    float h2f = 0.f;
    for (int i = 0; i < nu; ++i) {
      const float xi = xf(0, i), yi = xf(1, i), zi = xf(2, i);
      for (int j = i + 1 + lane; j < nu; j += 32) {
        const float dx = xf(0, j) - xi, dy = xf(1, j) - yi, dz = xf(2, j) - zi;
        h2f = fmaxf(h2f, fmaf(dz, dz, fmaf(dy, dy, dx * dx)));
      }
    }
    h2f = (float)warp_max((double)h2f);
    const float cut = h2f * (1.0f - 1e-5f);
    double h2 = 0.0;
    for (int i = 0; i < nu; ++i) {
      const float xi = xf(0, i), yi = xf(1, i), zi = xf(2, i);
      for (int j = i + 1 + lane; j < nu; j += 32) {
        const float dx = xf(0, j) - xi, dy = xf(1, j) - yi, dz = xf(2, j) - zi;
        if (fmaf(dz, dz, fmaf(dy, dy, dx * dx)) < cut) continue;
        const int vi = m.uvidx[ub + i], vj = m.uvidx[ub + j];
        double s2 = 0.0;
        for (int d = 0; d < 3; ++d) {
          const double df = m.X[d][vj] - m.X[d][vi];
          s2 += df * df;
        }
        h2 = fmax(h2, s2);
      }
    }
    h2 = warp_max(h2);
    __syncwarp();  // the staged copy is reused by the next element
    if (lane == 0) {
      for (int d = 0; d < 3; ++d) {
        m.lo[d * m.ne + e] = lo[d];
        m.L[d * m.ne + e] = hi[d] - lo[d];
        m.cen[d * m.ne + e] = cen[d];
      }
      m.vol[e] = vol;
      const double h = sqrt(h2);
      m.h[e] = h;
      const int pe = m.p[e];
      m.pen[e] = m.a[e] * pe * pe / h;
      constexpr int EV = elem_vals(3);
      double rec[EV];
      double box = 1.0;
      for (int d = 0; d < 3; ++d) {
        const double L = hi[d] - lo[d];
        rec[d] = lo[d];
        rec[3 + d] = L;
        rec[6 + d] = 1.0 / L;
        box *= L;
      }
      rec[9] = 1.0 / sqrt(box);
      for (int k = 0; k < EV; ++k) {
        m.eg64[(size_t)k * m.ne + e] = rec[k];
        m.eg32[(size_t)k * m.ne + e] = (float)rec[k];
      }
    }
  }
}

template <int D>
__device__ __forceinline__ void sub_geom(const DevMesh& m, int wmask, int k) {
  const int e = m.sub_elem[k];
  double lo[3], L[3];
  for (int d = 0; d < D; ++d) {
    lo[d] = m.eg64[(size_t)d * m.ne + e];
    L[d] = m.eg64[(size_t)(2 * D + d) * m.ne + e];  // 1/L
  }
  constexpr int SV = sub_vals(D);
  double out[SV];
  if (D == 2) {
    const int b = m.eptr[e], n = m.eptr[e + 1] - b;
    const int i = k - b;
    const int v1 = m.eidx[k], v2 = m.eidx[b + (i + 1 == n ? 0 : i + 1)];
    const double c[2] = {m.cen[e], m.cen[m.ne + e]};
    const double p1[2] = {m.X[0][v1], m.X[1][v1]}, p2[2] = {m.X[0][v2], m.X[1][v2]};
    for (int d = 0; d < 2; ++d) {
      const double xc = xi_of(c[d], lo[d], L[d]);
      out[d] = xc;
      out[2 + d] = xi_of(p1[d], lo[d], L[d]) - xc;
      out[4 + d] = xi_of(p2[d], lo[d], L[d]) - xc;
    }
    out[6] = fabs((p1[0] - c[0]) * (p2[1] - c[1]) - (p1[1] - c[1]) * (p2[0] - c[0]));
  } else {
    double P[4][3];
    for (int i = 0; i < 4; ++i) {
      const int v = m.eidx[4 * k + i];
      for (int d = 0; d < 3; ++d) P[i][d] = m.X[d][v];
    }
    for (int d = 0; d < 3; ++d) {
      const double x0 = xi_of(P[0][d], lo[d], L[d]);
      out[d] = x0;
      for (int i = 1; i < 4; ++i) out[3 * i + d] = xi_of(P[i][d], lo[d], L[d]) - x0;
    }
    double u[3], v[3], w[3];
    for (int d = 0; d < 3; ++d) {
      u[d] = P[1][d] - P[0][d];
      v[d] = P[2][d] - P[0][d];
      w[d] = P[3][d] - P[0][d];
    }
    out[12] = fabs(u[0] * (v[1] * w[2] - v[2] * w[1]) - u[1] * (v[0] * w[2] - v[2] * w[0]) +
                   u[2] * (v[0] * w[1] - v[1] * w[0]));
  }
  if (wmask & 1)
    for (int j = 0; j < SV; ++j) m.sg64[(size_t)j * m.nsub + k] = out[j];
  if (wmask & 2)
    for (int j = 0; j < SV; ++j) m.sg32[(size_t)j * m.nsub + k] = (float)out[j];
}

// The two half-face records of face f (hf_rec_vals layout): from side s,
// its own values first, then the other side's, normals and b . n times sgn_s.
// Each record is assembled in registers and stored with 16-byte stores.
template <int D, typename V, typename T>
__device__ __forceinline__ void write_hf_records(const DevMesh& m, int f, const V (&sv)[2][side_vals(D)], V J, V sigma,
                                                 V bn, T* hfr) {
  constexpr int FV = side_vals(D), RS = hf_rec_vals(D);
  const bool bnd = m.f_e1[f] < 0;
  const V nq = (V)m.f_nq[f];
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const int h = m.f_hf[(size_t)s * m.nf + f];
    if (h < 0) continue;
    const V sg = s == 0 ? V(1) : V(-1);
    T r[RS];
#pragma unroll
    for (int o = 0; o < 2; ++o)
#pragma unroll
      for (int j = 0; j < FV; ++j) {
        const V x = sv[o == 0 ? s : 1 - s][j];
        r[o * FV + j] = (T)(j >= D * D ? sg * x : x);
      }
    r[2 * FV] = (T)J;
    r[2 * FV + 1] = (T)sigma;
    r[2 * FV + 2] = (T)(sg * bn);
    r[2 * FV + 3] = (T)(bnd ? -nq : nq);
#pragma unroll
    for (int j = 2 * FV + 4; j < RS; ++j) r[j] = T(0);
    T* dst = hfr + (size_t)h * RS;
    if constexpr (sizeof(T) == 4) {
#pragma unroll
      for (int j = 0; j < RS; j += 4)
        *reinterpret_cast<float4*>(dst + j) = make_float4(r[j], r[j + 1], r[j + 2], r[j + 3]);
    } else {
#pragma unroll
      for (int j = 0; j < RS; j += 2) *reinterpret_cast<double2*>(dst + j) = make_double2(r[j], r[j + 1]);
    }
  }
}

// Boundary face f on the Neumann part of the boundary (Eq. (2.2)): all its
// vertices on one marked side of the vertex box, compared exactly.  Its
// records carry sigma = -1 and b . n = 0: the row kernels add no matrix
// term there (Eq. (2.4)) and take g_N v into the load vector (Eq. (2.5)).
template <int D>
__device__ __forceinline__ bool neumann_face(const DevMesh& m, int f) {
  if (m.pb.neumann == 0 || m.f_e1[f] >= 0) return false;
  for (int d = 0; d < D; ++d)
    for (int s = 0; s < 2; ++s) {
      if (!((m.pb.neumann >> (2 * d + s)) & 1)) continue;
      const double side = s ? m.pb.dhi[d] : m.pb.dlo[d];
      bool on = true;
      for (int i = 0; i < D; ++i) on = on && m.X[d][m.f_v[D * f + i]] == side;
      if (on) return true;
    }
  return false;
}

template <int D>
__device__ __forceinline__ void face_geom(const DevMesh& m, int wmask, int f) {
  const int es[2] = {m.f_e0[f], m.f_e1[f]};
  double P[3][3];
  for (int i = 0; i < D; ++i) {
    const int v = m.f_v[D * f + i];
    for (int d = 0; d < D; ++d) P[i][d] = m.X[d][v];
  }
  double n[3], J;
  if (D == 2) {
    const double tx = P[1][0] - P[0][0], ty = P[1][1] - P[0][1];
    const double len = sqrt(tx * tx + ty * ty);
    n[0] = ty / len;  // the CCW loop of e0 has its interior on the left
    n[1] = -tx / len;
    J = len;
  } else {
    double u[3], v[3];
    for (int d = 0; d < 3; ++d) {
      u[d] = P[1][d] - P[0][d];
      v[d] = P[2][d] - P[0][d];
    }
    const double c[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]};
    const double len = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
    const double sg = m.f_flip[f] ? -1.0 : 1.0;  // point out of e0
    for (int d = 0; d < 3; ++d) n[d] = sg * c[d] / len;
    J = len;                                         // = 2 |F| (collapsed triangle rule)
  }
  constexpr int FV = side_vals(D);
  double sigma = 0.0;
  double sv[2][FV];
  for (int s = 0; s < 2; ++s) {
    const int e = es[s];
    double* out = sv[s];
    for (int j = 0; j < FV; ++j) out[j] = 0.0;
    if (e >= 0) {
      for (int d = 0; d < D; ++d) {
        const double lo = m.eg64[(size_t)d * m.ne + e], iL = m.eg64[(size_t)(2 * D + d) * m.ne + e];
        const double x0 = xi_of(P[0][d], lo, iL);
        out[d] = x0;
        for (int i = 1; i < D; ++i) out[i * D + d] = xi_of(P[i][d], lo, iL) - x0;
        out[D * D + d] = 2.0 * n[d] * iL;
      }
      sigma = fmax(sigma, m.pen[e]);
    }
    if (wmask & 1)
      for (int j = 0; j < FV; ++j) m.fs64[((size_t)s * FV + j) * m.nf + f] = out[j];
  }
  sigma *= m.pb.c_sigma;
  double bn = 0.0;
  for (int d = 0; d < D; ++d) bn += m.pb.b[d] * n[d];
  if (neumann_face<D>(m, f)) {
    sigma = -1.0;
    bn = 0.0;
  }
  const double sc[3] = {J, sigma, bn};
  if (wmask & 1)
    for (int j = 0; j < 3; ++j) m.fsc64[(size_t)j * m.nf + f] = sc[j];
  if (wmask & 1) write_hf_records<D>(m, f, sv, J, sigma, bn, m.hfr64);
  if (wmask & 2) write_hf_records<D>(m, f, sv, J, sigma, bn, m.hfr32);
}

// sub-simplex records (threads 0 .. nsub-1) and face records (the rest):
// both read only the element records, so one launch covers them
template <int D>
__global__ void subface_geom_kernel(DevMesh m, int wmask) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < m.nsub)
    sub_geom<D>(m, wmask, t);
  else if (t - m.nsub < m.nf)
    face_geom<D>(m, wmask, t - m.nsub);
}

// ---------------------------------------------------------------------------
// Reduced-precision geometry (the FP32 and tensor-core forms).
//
// Those forms need the records to FP32 accuracy relative to each element's
// own size.  What costs digits in FP32 is only the difference of two absolute
// coordinates (x - lo, an edge vector) when the element is small against its
// distance from the origin.  So every coordinate is split once into an
// unevaluated float pair x = hi + lo (48 significant bits); a difference of
// two pairs, (a.hi - b.hi) + (a.lo - b.lo), then has FP32 relative accuracy,
// and everything else is FP32 arithmetic.  No FP64 arithmetic remains past
// the split, which matters on a part whose FP64 rate is 1/64 of its FP32 rate.
//
// The records are built to agree with the rounded FP64 records, not only to
// be accurate: the box is spanned by the pairs of its extreme vertices, a
// vertex maps to 2 (x - lo) / L - 1 in two-float arithmetic with one final
// rounding (the extreme vertices land on -1 and +1 exactly), and sub-simplex
// and face edges are differences of the rounded vertex coordinates, as in the
// FP64 records.  The map's accuracy matters: a degree-p basis function has a
// relative slope of about p (p + 1) / 2 at the box's edge.
// That keeps boundary points exactly on the boundary, where the Dirichlet
// data of Eq. (2.5) is taken against a penalty of order a p^2 / h.
// ---------------------------------------------------------------------------

__device__ __forceinline__ float pdiff(float2 a, float2 b) { return (a.x - b.x) + (a.y - b.y); }

// a - b for pairs as an unevaluated sum (hi, lo), |lo| <= ulp(hi) / 2
// (Knuth's TwoSum on the high parts, then Dekker's FastTwoSum)
__device__ __forceinline__ float2 pdiff2(float2 a, float2 b) {
  const float s = a.x - b.x;
  const float bb = s - a.x;
  const float t = ((a.x - (s - bb)) + (-b.x - bb)) + (a.y - b.y);
  const float h = s + t;
  return make_float2(h, t - (h - s));
}

// bounding-box coordinate 2 (x - lo) / L - 1 of the pair x in a box with
// lower corner lo and extent L (pairs), iL = 1 / L.hi.  The quotient is
// carried in two floats (a product, then one correction from the exact FMA
// remainder) and 2q - 1 is formed error-free, so the single final rounding
// leaves it as accurate as the rounded FP64 value; x = lo gives -1 and
// x - lo = L gives +1 exactly.
__device__ __forceinline__ float xi_pair(float2 x, float2 lo, float2 L, float iL) {
  const float2 a = pdiff2(x, lo);
  const float q1 = a.x * iL;
  const float q2 = (fmaf(-q1, L.x, a.x) + (a.y - q1 * L.y)) * iL;
  const float t = 2.f * q1, u = t - 1.f;
  const float bv = u - t;
  const float eu = (t - (u - bv)) + (-1.f - bv);
  return u + (eu + 2.f * q2);
}

__device__ __forceinline__ float2 xpair(const DevMesh& m, int d, int v) { return m.xs2[(size_t)d * m.nv + v]; }

// (value, index) minimum / maximum over the warp; ties go to the smaller
// index, so every lane ends with the same pair
__device__ __forceinline__ void warp_argmin(float& v, int& i) {
  for (int o = 16; o > 0; o >>= 1) {
    const float ov = __shfl_xor_sync(0xffffffffu, v, o);
    const int oi = __shfl_xor_sync(0xffffffffu, i, o);
    if (ov < v || (ov == v && oi < i)) {
      v = ov;
      i = oi;
    }
  }
}
__device__ __forceinline__ void warp_argmax(float& v, int& i) {
  for (int o = 16; o > 0; o >>= 1) {
    const float ov = __shfl_xor_sync(0xffffffffu, v, o);
    const int oi = __shfl_xor_sync(0xffffffffu, i, o);
    if (ov > v || (ov == v && oi < i)) {
      v = ov;
      i = oi;
    }
  }
}
__device__ __forceinline__ float warp_maxf(float v) {
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__global__ void vertex_split_kernel(DevMesh m) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m.dim * m.nv) return;
  const int d = i / m.nv;
  const double x = m.X[d][i - d * m.nv];
  const float hi = __double2float_rn(x);
  m.xs2[i] = make_float2(hi, __double2float_rn(x - (double)hi));
}

// element record and reduced-precision scratch: lo = the pairs of the box's
// lower corner, L its extent (pairs), h2 the squared diameter
template <int D>
__device__ __forceinline__ void write_elem_f32(const DevMesh& m, int e, const float2* lo, const float2* L, float h2) {
  constexpr int EV = elem_vals(D);
  float rec[EV], gx[EV];
  float box = 1.f;
  for (int d = 0; d < D; ++d) {
    rec[d] = lo[d].x;  // the pair's high part is the rounded coordinate
    rec[D + d] = L[d].x;
    rec[2 * D + d] = 1.f / L[d].x;
    box *= L[d].x;
    gx[d] = lo[d].x;
    gx[D + d] = lo[d].y;
    gx[2 * D + d] = L[d].y;
  }
  rec[3 * D] = 1.f / sqrtf(box);
  const int pe = m.p[e];
  gx[3 * D] = (float)m.a[e] * (float)(pe * pe) / sqrtf(h2);
  for (int k = 0; k < EV; ++k) {
    m.eg32[(size_t)k * m.ne + e] = rec[k];
    m.gx32[(size_t)k * m.ne + e] = gx[k];
  }
}

// 2D element e with k loop vertices starting at b; u(i) = vertex i relative
// to vertex 0.  NU > 0: loops run to the compile-time bound NU (k <= NU), so
// u indexes registers; NU == 0: runtime loops.  Writes the element record and
// the k sub-triangle records (centroid, v_i, v_{i+1}) of Sec. 3.
template <int NU, class U>
__device__ __forceinline__ void elem2d_f32_body(const DevMesh& m, int e, int b, int k, U u) {
  const int n = NU ? NU : k;
  float lo[2] = {0.f, 0.f}, hi[2] = {0.f, 0.f};
  int il[2] = {0, 0}, ih[2] = {0, 0};
  float a2 = 0.f, cx = 0.f, cy = 0.f, h2 = 0.f;
  // vertex 0 is the origin, so the shoelace terms that touch it vanish
#pragma unroll
  for (int i = 1; i < n; ++i) {
    if (NU && i >= k) break;
    const float2 p = u(i);
    if (p.x < lo[0]) lo[0] = p.x, il[0] = i;
    if (p.x > hi[0]) hi[0] = p.x, ih[0] = i;
    if (p.y < lo[1]) lo[1] = p.y, il[1] = i;
    if (p.y > hi[1]) hi[1] = p.y, ih[1] = i;
    h2 = fmaxf(h2, fmaf(p.x, p.x, p.y * p.y));
    if (i + 1 < n && i + 1 < k) {
      const float2 q = u(i + 1 < n ? i + 1 : i);
      const float cr = p.x * q.y - q.x * p.y;
      a2 += cr;
      cx += (p.x + q.x) * cr;
      cy += (p.y + q.y) * cr;
    }
#pragma unroll
    for (int j = i + 1; j < n; ++j) {
      if (NU && j >= k) break;
      const float2 q = u(j);
      const float dx = q.x - p.x, dy = q.y - p.y;
      h2 = fmaxf(h2, fmaf(dx, dx, dy * dy));
    }
  }
  const float i3 = 1.f / (3.f * a2);
  cx *= i3;
  cy *= i3;
  float2 lp[2], L[2];
  float iL[2];
  for (int d = 0; d < 2; ++d) {
    lp[d] = xpair(m, d, m.eidx[b + il[d]]);
    L[d] = pdiff2(xpair(m, d, m.eidx[b + ih[d]]), lp[d]);
    iL[d] = 1.f / L[d].x;
  }
  write_elem_f32<2>(m, e, lp, L, h2);
  // the fan apex: any interior point gives the same polygon, so its own
  // rounding does not matter; the vertices are mapped as accurately as FP64
  const float xc = 2.f * ((cx - lo[0]) * iL[0]) - 1.f, yc = 2.f * ((cy - lo[1]) * iL[1]) - 1.f;
  const int v0 = m.eidx[b];
  const float2 q0x = xpair(m, 0, v0), q0y = xpair(m, 1, v0);
  const float z0x = xi_pair(q0x, lp[0], L[0], iL[0]), z0y = xi_pair(q0y, lp[1], L[1], iL[1]);
  float2 px = q0x, py = q0y;
  float zx = z0x, zy = z0y;
  const size_t ns = m.nsub;
#pragma unroll
  for (int i = 0; i < n; ++i) {
    if (NU && i >= k) break;
    const bool wrap = i + 1 >= k;
    float2 qx = q0x, qy = q0y;
    float wx = z0x, wy = z0y;
    if (!wrap) {
      const int v = m.eidx[b + i + 1];
      qx = xpair(m, 0, v);
      qy = xpair(m, 1, v);
      wx = xi_pair(qx, lp[0], L[0], iL[0]);
      wy = xi_pair(qy, lp[1], L[1], iL[1]);
    }
    // twice the area of (c, v_i, v_{i+1}) = |(v_i - c) x (v_{i+1} - v_i)|
    const float2 p = u(i);
    const float ax = p.x - cx, ay = p.y - cy, ex = pdiff(qx, px), ey = pdiff(qy, py);
    float* o = m.sg32 + b + i;
    o[0] = xc;
    o[ns] = yc;
    o[2 * ns] = zx - xc;
    o[3 * ns] = zy - yc;
    o[4 * ns] = wx - xc;
    o[5 * ns] = wy - yc;
    o[6 * ns] = fabsf(ax * ey - ay * ex);
    px = qx;
    py = qy;
    zx = wx;
    zy = wy;
  }
}

__global__ void elem_geom2d_f32_kernel(DevMesh m) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m.ne) return;
  const int b = m.eptr[e], k = m.eptr[e + 1] - b;
  const int v0 = m.eidx[b];
  const float2 r0 = xpair(m, 0, v0), r1 = xpair(m, 1, v0);
  constexpr int KV = 16;
  if (k <= KV) {
    float ux[KV], uy[KV];
    ux[0] = uy[0] = 0.f;
#pragma unroll
    for (int i = 1; i < KV; ++i)
      if (i < k) {
        const int v = m.eidx[b + i];
        ux[i] = pdiff(xpair(m, 0, v), r0);
        uy[i] = pdiff(xpair(m, 1, v), r1);
      }
    elem2d_f32_body<KV>(m, e, b, k, [&](int i) { return make_float2(ux[i], uy[i]); });
  } else {
    elem2d_f32_body<0>(m, e, b, k, [&](int i) {
      const int v = m.eidx[b + i];
      return make_float2(pdiff(xpair(m, 0, v), r0), pdiff(xpair(m, 1, v), r1));
    });
  }
}

// 3D, one warp per element: the distinct vertices relative to the first one
// (box, diameter), then the element's tetrahedra (sub-simplex records)
__global__ void __launch_bounds__(kGeomWarps * 32) elem_geom3d_f32_kernel(DevMesh m) {
  __shared__ float sv[kGeomWarps][3][kGeomVerts];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; e < m.ne; e += nw) {
    const int ub = m.uvptr[e], nu = m.uvptr[e + 1] - ub;
    const bool staged = nu <= kGeomVerts;
    const int vr = m.uvidx[ub];
    float2 r[3];
    for (int d = 0; d < 3; ++d) r[d] = xpair(m, d, vr);
    // distinct vertex 0 is the origin: (0, 0) is a valid start on every lane
    float lo[3] = {0.f, 0.f, 0.f}, hi[3] = {0.f, 0.f, 0.f};
    int il[3] = {0, 0, 0}, ih[3] = {0, 0, 0};
    for (int i = lane; i < nu; i += 32) {
      const int v = m.uvidx[ub + i];
      for (int d = 0; d < 3; ++d) {
        const float x = pdiff(xpair(m, d, v), r[d]);
        if (x < lo[d]) lo[d] = x, il[d] = i;
        if (x > hi[d]) hi[d] = x, ih[d] = i;
        if (staged) sv[wib][d][i] = x;
      }
    }
    for (int d = 0; d < 3; ++d) {
      warp_argmin(lo[d], il[d]);
      warp_argmax(hi[d], ih[d]);
    }
    __syncwarp();
    auto xf = [&](int d, int i) -> float { return staged ? sv[wib][d][i] : pdiff(xpair(m, d, m.uvidx[ub + i]), r[d]); };
    float h2 = 0.f;
    for (int i = 0; i < nu; ++i) {
      const float xi = xf(0, i), yi = xf(1, i), zi = xf(2, i);
      for (int j = i + 1 + lane; j < nu; j += 32) {
        const float dx = xf(0, j) - xi, dy = xf(1, j) - yi, dz = xf(2, j) - zi;
        h2 = fmaxf(h2, fmaf(dz, dz, fmaf(dy, dy, dx * dx)));
      }
    }
    h2 = warp_maxf(h2);
    __syncwarp();  // the staged copy is reused by the next element
    float2 lp[3], L[3];
    float iL[3];
    for (int d = 0; d < 3; ++d) {
      lp[d] = xpair(m, d, m.uvidx[ub + il[d]]);
      L[d] = pdiff2(xpair(m, d, m.uvidx[ub + ih[d]]), lp[d]);
      iL[d] = 1.f / L[d].x;
    }
    const size_t ns = m.nsub;
    for (int t = m.eptr[e] + lane; t < m.eptr[e + 1]; t += 32) {
      float2 P[4][3];
      for (int i = 0; i < 4; ++i) {
        const int v = m.eidx[4 * t + i];
        for (int d = 0; d < 3; ++d) P[i][d] = xpair(m, d, v);
      }
      float* o = m.sg32 + t;
      float u[3][3];
      for (int d = 0; d < 3; ++d) {
        const float z0 = xi_pair(P[0][d], lp[d], L[d], iL[d]);
        o[d * ns] = z0;
        for (int i = 1; i < 4; ++i) {
          o[(3 * i + d) * ns] = xi_pair(P[i][d], lp[d], L[d], iL[d]) - z0;
          u[i - 1][d] = pdiff(P[i][d], P[0][d]);
        }
      }
      o[12 * ns] = fabsf(u[0][0] * (u[1][1] * u[2][2] - u[1][2] * u[2][1]) -
                         u[0][1] * (u[1][0] * u[2][2] - u[1][2] * u[2][0]) +
                         u[0][2] * (u[1][0] * u[2][1] - u[1][1] * u[2][0]));
    }
    if (lane == 0) write_elem_f32<3>(m, e, lp, L, h2);
  }
}

// face records from the split coordinates and the elements' box corners;
// the same quantities as face_geom
template <int D>
__global__ void face_geom_f32_kernel(DevMesh m) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= m.nf) return;
  float2 P[D][D];
  for (int i = 0; i < D; ++i) {
    const int v = m.f_v[D * f + i];
    for (int d = 0; d < D; ++d) P[i][d] = xpair(m, d, v);
  }
  float t[D - 1][D];
  for (int i = 1; i < D; ++i)
    for (int d = 0; d < D; ++d) t[i - 1][d] = pdiff(P[i][d], P[0][d]);
  float n[3], J;
  if constexpr (D == 2) {
    const float len = sqrtf(fmaf(t[0][0], t[0][0], t[0][1] * t[0][1]));
    n[0] = t[0][1] / len;  // the CCW loop of e0 has its interior on the left
    n[1] = -t[0][0] / len;
    J = len;
  } else {
    const float* u = t[0];
    const float* v = t[1];
    const float c[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]};
    const float len = sqrtf(fmaf(c[0], c[0], fmaf(c[1], c[1], c[2] * c[2])));
    const float sg = m.f_flip[f] ? -1.f : 1.f;  // point out of e0
    for (int d = 0; d < 3; ++d) n[d] = sg * c[d] / len;
    J = len;  // = 2 |F| (collapsed triangle rule)
  }
  constexpr int FV = side_vals(D);
  const int es[2] = {m.f_e0[f], m.f_e1[f]};
  float sigma = 0.f;
  float sv[2][FV];
  for (int s = 0; s < 2; ++s) {
    const int e = es[s];
    float* out = sv[s];
    for (int j = 0; j < FV; ++j) out[j] = 0.f;
    if (e >= 0) {
      for (int d = 0; d < D; ++d) {
        const float2 lp = make_float2(m.gx32[(size_t)d * m.ne + e], m.gx32[(size_t)(D + d) * m.ne + e]);
        const float2 L = make_float2(m.eg32[(size_t)(D + d) * m.ne + e], m.gx32[(size_t)(2 * D + d) * m.ne + e]);
        const float iL = m.eg32[(size_t)(2 * D + d) * m.ne + e];
        const float z0 = xi_pair(P[0][d], lp, L, iL);
        out[d] = z0;
        for (int i = 1; i < D; ++i) out[i * D + d] = xi_pair(P[i][d], lp, L, iL) - z0;
        out[D * D + d] = 2.f * (n[d] * iL);
      }
      sigma = fmaxf(sigma, m.gx32[(size_t)(3 * D) * m.ne + e]);
    }
  }
  float bn = 0.f;
  for (int d = 0; d < D; ++d) bn = fmaf(m.pb.bf[d], n[d], bn);
  sigma *= m.pb.c_sigmaf;
  if (neumann_face<D>(m, f)) {
    sigma = -1.f;
    bn = 0.f;
  }
  write_hf_records<D>(m, f, sv, J, sigma, bn, m.hfr32);
}

inline int nblk(int n, int t) { return (n + t - 1) / t; }

}  // namespace

int launch_geometry(const DevMesh& m, cudaStream_t st, Tracer* tr, int wmask) {
  const int T = 128;
  // no algorithmic flop count of its own (kind past the counted ones)
  if (tr && tr->on) tr->begin(m.dim == 2 ? "geometry2d" : "geometry3d", kNoCounts, 0, 8, st);
  const int nsf = m.nsub + m.nf;
  if (wmask == 2 && m.xs2 && m.gx32) {
    if (m.nv > 0) vertex_split_kernel<<<nblk(m.dim * m.nv, T), T, 0, st>>>(m);
    if (m.dim == 2) {
      if (m.ne > 0) elem_geom2d_f32_kernel<<<nblk(m.ne, T), T, 0, st>>>(m);
      if (m.nf > 0) face_geom_f32_kernel<2><<<nblk(m.nf, T), T, 0, st>>>(m);
    } else {
      if (m.ne > 0) elem_geom3d_f32_kernel<<<nblk(m.ne * 32, kGeomWarps * 32), kGeomWarps * 32, 0, st>>>(m);
      if (m.nf > 0) face_geom_f32_kernel<3><<<nblk(m.nf, T), T, 0, st>>>(m);
    }
    if (tr && tr->on) tr->end(st);
    return 3;
  }
  if (m.dim == 2) {
    if (m.ne > 0) elem_geom_kernel<2><<<nblk(m.ne, T), T, 0, st>>>(m);
    if (nsf > 0) subface_geom_kernel<2><<<nblk(nsf, T), T, 0, st>>>(m, wmask);
  } else {
    if (m.ne > 0) elem_geom3d_warp_kernel<<<nblk(m.ne * 32, kGeomWarps * 32), kGeomWarps * 32, 0, st>>>(m);
    if (nsf > 0) subface_geom_kernel<3><<<nblk(nsf, T), T, 0, st>>>(m, wmask);
  }
  if (tr && tr->on) tr->end(st);
  return 2;
}

}  // namespace dg
