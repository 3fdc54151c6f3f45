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
  for (int s = 0; s < 2; ++s) {
    const int e = es[s];
    double out[FV];
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
    if (wmask & 2)
      for (int j = 0; j < FV; ++j) m.fs32[((size_t)s * FV + j) * m.nf + f] = (float)out[j];
  }
  sigma *= m.pb.c_sigma;
  double bn = 0.0;
  for (int d = 0; d < D; ++d) bn += m.pb.b[d] * n[d];
  const double sc[3] = {J, sigma, bn};
  if (wmask & 1)
    for (int j = 0; j < 3; ++j) m.fsc64[(size_t)j * m.nf + f] = sc[j];
  if (wmask & 2)
    for (int j = 0; j < 3; ++j) m.fsc32[(size_t)j * m.nf + f] = (float)sc[j];
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

inline int nblk(int n, int t) { return (n + t - 1) / t; }

}  // namespace

int launch_geometry(const DevMesh& m, cudaStream_t st, Tracer* tr, int wmask) {
  const int T = 128;
  // no algorithmic flop count of its own (kind past the counted ones)
  if (tr && tr->on) tr->begin(m.dim == 2 ? "geometry2d" : "geometry3d", kKinds, 0, 8, st);
  const int nsf = m.nsub + m.nf;
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
