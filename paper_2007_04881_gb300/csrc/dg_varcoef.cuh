// dg_varcoef.cuh -- the variable advection and reaction fields of the
// paper's multi-GPU test problem (Sec. 4.2), b_d(x) = 1 + x_d and
// c(x) = 3 + prod_d x_d, evaluated at every quadrature point.
//
// The terms of Eq. (2.4) and Eq. (2.5) that carry b and c, on a mesh whose
// other terms (diffusion, SIPG consistency, symmetry and penalty, the source
// -a Lap u and the Nitsche data) the row kernels have written with b = 0 and
// c = 0:
//   volume  sum_q W [ (b(x_q) . grad phi_j) phi_i + c(x_q) phi_j phi_i ],
//   faces   at every face point where row r's element is inflow,
//           b(x) . n_r < 0 with n_r out of r (b . n = 0 is outflow):
//             A_rr += -(b . n_r) phi^r_j phi^r_i,  A_r,nb += (b . n_r) phi^nb_j phi^r_i,
//   load    sum_q W (b . grad u + c u)(x_q) phi_i on the volume points and
//           -(b . n_r) g phi_i at the inflow points of Dirichlet boundary
//           faces (g = u); Neumann faces carry no b term (Eq. (2.4), (2.5)),
// with the volume and face rules and the geometry records of the row kernels.
//
// The row bodies are host/device functions: a warp runs one element row in
// the kernels (dg_varcoef.cu), and the CPU tests run the same bodies on host
// arrays.  Every lane evaluates the basis functions of its own block entries
// at every point: no sharing, no synchronisation.
#pragma once

#include <cmath>

#include "dg_internal.h"

namespace dg {

constexpr double kVcPi = 3.14159265358979323846;

// b(x) and c(x) at a point
template <int D>
__host__ __device__ inline double vc_fields(const double* x, double* b) {
  double prod = 1.0;
  for (int d = 0; d < D; ++d) {
    b[d] = 1.0 + x[d];
    prod *= x[d];
  }
  return 3.0 + prod;
}

// sin(pi x) and cos(pi x); exactly 0 where the argument is an integer
// (sine) or a half-integer (cosine), as the CUDA functions give them
__host__ __device__ inline void vc_sincospi(double x, double* s, double* c) {
#ifdef __CUDA_ARCH__
  sincospi(x, s, c);
#else
  const double r = x - 2.0 * std::nearbyint(0.5 * x);  // same sine and cosine, r in [-1, 1]
  const double ar = std::fabs(r);
  *s = (ar == 0.0 || ar == 1.0) ? 0.0 : std::sin(kVcPi * r);
  *c = ar == 0.5 ? 0.0 : std::cos(kVcPi * r);
#endif
}

// the manufactured solution u = prod_d sin(pi x_d) of DG_SRC_SINPROD and its
// gradient; zero for DG_SRC_ZERO
template <int D>
__host__ __device__ inline double vc_exact(int source, const double* x, double* gu) {
  if (source != 1) {
    for (int d = 0; d < D; ++d) gu[d] = 0.0;
    return 0.0;
  }
  double s[D], c[D];
  for (int d = 0; d < D; ++d) vc_sincospi(x[d], &s[d], &c[d]);
  double u = 1.0;
  for (int d = 0; d < D; ++d) u *= s[d];
  for (int d = 0; d < D; ++d) {
    double g = kVcPi * c[d];
    for (int e = 0; e < D; ++e)
      if (e != d) g *= s[e];
    gu[d] = g;
  }
  return u;
}

// exponents of basis function i: by total degree k, then 2D j = 0..k with
// alpha = (k - j, j); 3D l = 0..k, j = 0..k - l with alpha = (k - j - l, j, l)
template <int D>
__host__ __device__ inline void vc_alpha(int i, int* al) {
  int k = 0;
  for (;;) {
    const int nk = D == 2 ? k + 1 : (k + 1) * (k + 2) / 2;  // functions of degree exactly k
    if (i < nk) break;
    i -= nk;
    ++k;
  }
  if (D == 2) {
    al[0] = k - i;
    al[1] = i;
    return;
  }
  int l = 0;
  while (i >= k - l + 1) {
    i -= k - l + 1;
    ++l;
  }
  al[0] = k - i - l;
  al[1] = i;
  al[2] = l;
}

// P_n(x) and P_n'(x) by the three-term recurrences
__host__ __device__ inline void vc_legendre(int n, double x, double* P, double* dP) {
  double p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0;
  if (n == 0) {
    *P = 1.0;
    *dP = 0.0;
    return;
  }
  for (int k = 1; k < n; ++k) {
    const double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
    const double d2 = d0 + (2.0 * k + 1.0) * p1;
    p0 = p1;
    p1 = p2;
    d0 = d1;
    d1 = d2;
  }
  *P = p1;
  *dP = d1;
}

// one element's box: lo, L and R = 1 / sqrt(prod_d L_d)
template <int D>
struct VcElem {
  double lo[D], L[D], R;
  int p;
};

// the arrays the bodies read (device pointers in the kernels, host arrays
// in the CPU tests); layouts as the row kernels' (dg_internal.h)
struct VcView {
  int ne, nf, nsub, source;
  const int* p;        // [ne]
  const int* eptr;     // [ne+1]: the element's sub-simplices
  const double* eg;    // [3D+1][ne]: lo, L, 1/L, R
  const double* sg;    // [sub_vals(D)][nsub]: xi0, edge vectors, |J|
  const double* fs;    // [2][side_vals(D)][nf]: per side xi(v0), xi(v_i) - xi(v0), n' = 2 n0 / L
  const double* fsc;   // [3][nf]: J, sigma, b.n (J, and sigma < 0 marking a Neumann face)
  const int* f_e0;     // [nf]
  const int* f_e1;     // [nf], -1 on the boundary
  const int* f_nq;     // [nf] face points per direction
  const int* hf_ptr;   // [ne+1]
  const int* hf_face;  // [nhf]
  const int8_t* hf_side;
  const int* if_fptr;  // [ni+1]
  const int* row_ptr;  // [ne+1]
  const int* col;      // [nnzb]
  const int* blk_if;   // [nnzb], -1 on the diagonal
  const int64_t* blk_off;
  const int64_t* dof_off;
  const double* vol_rule;  // [point][D+1]
  const double* face_rule;  // [point][D]
  int vol_off[8], face_off[10];
  int vol_n[8], face_n[10];
};

template <int D>
__host__ __device__ inline void vc_load_elem(const VcView& v, int e, VcElem<D>& E) {
  for (int d = 0; d < D; ++d) {
    E.lo[d] = v.eg[(size_t)d * v.ne + e];
    E.L[d] = v.eg[(size_t)(D + d) * v.ne + e];
  }
  E.R = v.eg[(size_t)(3 * D) * v.ne + e];
  E.p = v.p[e];
}

// phi_i and its physical gradient at box coordinates xi
template <int D>
__host__ __device__ inline double vc_phi(const VcElem<D>& E, int i, const double* xi, double* grad) {
  int al[D];
  vc_alpha<D>(i, al);
  double P[D], dP[D], s = E.R;
  for (int d = 0; d < D; ++d) {
    vc_legendre(al[d], xi[d], &P[d], &dP[d]);
    s *= sqrt(2.0 * al[d] + 1.0);
  }
  double val = s;
  for (int d = 0; d < D; ++d) val *= P[d];
  for (int d = 0; d < D; ++d) {
    double g = s * 2.0 / E.L[d] * dP[d];
    for (int e = 0; e < D; ++e)
      if (e != d) g *= P[e];
    grad[d] = g;
  }
  return val;
}

// the point of face f on side s (box coordinates of that side's element),
// the unit normal n0 out of the face's first element, and the weight
template <int D>
__host__ __device__ inline void vc_face_point(const VcView& v, int f, int s, const VcElem<D>& E, const double* fr,
                                              double* xi, double* n0) {
  constexpr int FV = side_vals(D);
  const double* F = v.fs + (size_t)s * FV * v.nf + f;
  for (int d = 0; d < D; ++d) {
    double t = F[(size_t)d * v.nf];
    for (int k = 1; k < D; ++k) t += fr[k - 1] * F[(size_t)(k * D + d) * v.nf];
    xi[d] = t;
    n0[d] = F[(size_t)(D * D + d) * v.nf] * 0.5 * E.L[d];
  }
}

template <int D>
__host__ __device__ inline void vc_to_x(const VcElem<D>& E, const double* xi, double* x) {
  for (int d = 0; d < D; ++d) x[d] = E.lo[d] + 0.5 * (xi[d] + 1.0) * E.L[d];
}

// volume part of diagonal entry (i, j) of element r
template <int D>
__host__ __device__ inline double vc_volume_entry(const VcView& v, const VcElem<D>& E, int r, int i, int j) {
  constexpr int SV = sub_vals(D);
  const double* rule = v.vol_rule + (size_t)v.vol_off[E.p] * (D + 1);
  const int nq = v.vol_n[E.p];
  double acc = 0.0;
  for (int k = v.eptr[r]; k < v.eptr[r + 1]; ++k) {
    double rec[SV];
    for (int t = 0; t < SV; ++t) rec[t] = v.sg[(size_t)t * v.nsub + k];
    for (int q = 0; q < nq; ++q) {
      const double* pt = rule + (size_t)q * (D + 1);
      double xi[D], x[D], b[D], gi[D], gj[D];
      for (int d = 0; d < D; ++d) {
        double t = rec[d];
        for (int a = 0; a < D; ++a) t += pt[a] * rec[(a + 1) * D + d];
        xi[d] = t;
      }
      vc_to_x<D>(E, xi, x);
      const double c = vc_fields<D>(x, b);
      const double W = pt[D] * rec[SV - 1];
      const double pi = vc_phi<D>(E, i, xi, gi);
      const double pj = vc_phi<D>(E, j, xi, gj);
      double bg = 0.0;
      for (int d = 0; d < D; ++d) bg += b[d] * gj[d];
      acc += W * (bg * pi + c * pj * pi);
    }
  }
  return acc;
}

// upwind part of entry (i, j) of block (r, s) from face f, r on side sr:
// the diagonal block (s == r) and the block of the face's other element
template <int D>
__host__ __device__ inline double vc_face_entry(const VcView& v, const VcElem<D>& Er, const VcElem<D>& Es, int f,
                                                int sr, bool diag, int i, int j) {
  const int n = v.f_nq[f];
  const double* rule = v.face_rule + (size_t)v.face_off[n] * D;
  const int nq = v.face_n[n];
  const double J = v.fsc[f];
  if (v.fsc[(size_t)v.nf + f] < 0.0) return 0.0;  // Neumann face: no inflow term (Eq. (2.4))
  const double sg = sr == 0 ? 1.0 : -1.0;  // n_r = sg n0
  double acc = 0.0;
  for (int q = 0; q < nq; ++q) {
    const double* pt = rule + (size_t)q * D;
    double xr[D], n0[D], x[D], b[D], gi[D], gj[D];
    vc_face_point<D>(v, f, sr, Er, pt, xr, n0);
    vc_to_x<D>(Er, xr, x);
    vc_fields<D>(x, b);
    double bn = 0.0;
    for (int d = 0; d < D; ++d) bn += b[d] * n0[d];
    bn *= sg;
    if (!(bn < 0.0)) continue;
    const double W = pt[D - 1] * J;
    const double pi = vc_phi<D>(Er, i, xr, gi);
    if (diag) {
      acc -= W * bn * vc_phi<D>(Er, j, xr, gj) * pi;
    } else {
      double xs[D], ns[D];
      vc_face_point<D>(v, f, 1 - sr, Es, pt, xs, ns);
      acc += W * bn * vc_phi<D>(Es, j, xs, gj) * pi;
    }
  }
  return acc;
}

// row r of the matrix: ADDS the b and c terms to every block of the row
template <int D>
__host__ __device__ inline void vc_matrix_row(const VcView& v, double* vals, int r, int lane, int lanes) {
  VcElem<D> Er;
  vc_load_elem<D>(v, r, Er);
  const int nr = nbasis(D, Er.p);
  for (int b = v.row_ptr[r]; b < v.row_ptr[r + 1]; ++b) {
    const int s = v.col[b];
    VcElem<D> Es;
    vc_load_elem<D>(v, s, Es);
    const int nc = nbasis(D, Es.p);
    double* out = vals + v.blk_off[b];
    for (int x = lane; x < nr * nc; x += lanes) {
      const int i = x / nc, j = x - (x / nc) * nc;
      double acc = 0.0;
      if (s == r) {
        acc = vc_volume_entry<D>(v, Er, r, i, j);
        for (int h = v.hf_ptr[r]; h < v.hf_ptr[r + 1]; ++h)
          acc += vc_face_entry<D>(v, Er, Er, v.hf_face[h], v.hf_side[h], true, i, j);
      } else {
        const int itf = v.blk_if[b];
        for (int f = v.if_fptr[itf]; f < v.if_fptr[itf + 1]; ++f)
          acc += vc_face_entry<D>(v, Er, Es, f, v.f_e0[f] == r ? 0 : 1, false, i, j);
      }
      out[x] += acc;
    }
  }
}

// row r of the load vector: ADDS the b and c terms of the source and the
// inflow data
template <int D>
__host__ __device__ inline void vc_rhs_row(const VcView& v, double* rhs, int r, int lane, int lanes) {
  constexpr int SV = sub_vals(D);
  VcElem<D> E;
  vc_load_elem<D>(v, r, E);
  const int nr = nbasis(D, E.p);
  const double* rule = v.vol_rule + (size_t)v.vol_off[E.p] * (D + 1);
  const int nq = v.vol_n[E.p];
  for (int i = lane; i < nr; i += lanes) {
    double acc = 0.0;
    if (v.source == 1) {
      for (int k = v.eptr[r]; k < v.eptr[r + 1]; ++k) {
        double rec[SV];
        for (int t = 0; t < SV; ++t) rec[t] = v.sg[(size_t)t * v.nsub + k];
        for (int q = 0; q < nq; ++q) {
          const double* pt = rule + (size_t)q * (D + 1);
          double xi[D], x[D], b[D], gu[D], gi[D];
          for (int d = 0; d < D; ++d) {
            double t = rec[d];
            for (int a = 0; a < D; ++a) t += pt[a] * rec[(a + 1) * D + d];
            xi[d] = t;
          }
          vc_to_x<D>(E, xi, x);
          const double c = vc_fields<D>(x, b);
          const double u = vc_exact<D>(v.source, x, gu);
          double bg = 0.0;
          for (int d = 0; d < D; ++d) bg += b[d] * gu[d];
          acc += pt[D] * rec[SV - 1] * (bg + c * u) * vc_phi<D>(E, i, xi, gi);
        }
      }
      for (int h = v.hf_ptr[r]; h < v.hf_ptr[r + 1]; ++h) {
        const int f = v.hf_face[h];
        if (v.f_e1[f] >= 0) continue;  // boundary faces only (the element is their side 0)
        if (v.fsc[(size_t)v.nf + f] < 0.0) continue;  // Dirichlet faces only (Eq. (2.5))
        const int n = v.f_nq[f];
        const double* fr = v.face_rule + (size_t)v.face_off[n] * D;
        for (int q = 0; q < v.face_n[n]; ++q) {
          const double* pt = fr + (size_t)q * D;
          double xi[D], n0[D], x[D], b[D], gu[D], gi[D];
          vc_face_point<D>(v, f, 0, E, pt, xi, n0);
          vc_to_x<D>(E, xi, x);
          vc_fields<D>(x, b);
          double bn = 0.0;
          for (int d = 0; d < D; ++d) bn += b[d] * n0[d];
          if (!(bn < 0.0)) continue;
          const double g = vc_exact<D>(v.source, x, gu);
          acc -= pt[D - 1] * v.fsc[f] * bn * g * vc_phi<D>(E, i, xi, gi);
        }
      }
    }
    rhs[v.dof_off[r] + i] += acc;
  }
}

// Launchers (dg_varcoef.cu); each returns the number of launches.
int launch_varcoef(const VcView& v, int dim, double* vals, double* rhs, int sm_count, cudaStream_t st);

}  // namespace dg
