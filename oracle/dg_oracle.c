/*
 * dg_oracle.c -- plain FP64 CPU oracle for interior-penalty dG assembly on
 * polygonal / polyhedral meshes (Dong, Georgoulis, Kappas, "GPU-accelerated
 * discontinuous Galerkin methods on polytopic meshes", arXiv 2007.04881).
 *
 * TEST INFRASTRUCTURE.  This file is the reference that the CUDA library is
 * checked against.  Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg may load it.  It shares no code, header, table or constant
 * generator with the CUDA path.
 *
 * Everything here is written as the definition, with plain loops, in the
 * order the paper states it:
 *   - problem and SIPG forms: Sec. 2.2, bilinear form B, Eq. (2.4), and load
 *     functional l, Eq. (2.5); averages / jumps / upwind jump as defined in
 *     Sec. 2.2;
 *   - basis: tensorised orthonormal Legendre polynomials of total degree p on
 *     each element's bounding box (Sec. 3.1);
 *   - quadrature: subdivision of each element into simplices (2D: fan of
 *     triangles from the area centroid; 3D: the element's tetrahedra), a
 *     standard rule on each sub-simplex (Sec. 3, first paragraphs; Sec. 3.1);
 *     the standard rules are collapsed (Duffy) tensor Gauss-Legendre rules;
 *   - penalty: sigma_F = C_sigma * max over the face's elements of
 *     a_k p_k^2 / h_k (the "10 p^2/h" reading of Appendix A with the max over
 *     the two sides kept).
 *
 * Parity pins (independent of this file's arithmetic) live in tests/.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* 1D Gauss-Legendre rule on [0,1]                                           */
/* ------------------------------------------------------------------------ */

/* Value of P_n and its derivative at t (three-term recurrence). */
static void legendre_pn(int n, double t, double *pn, double *dpn) {
  double p0 = 1.0, p1 = t;
  if (n == 0) {
    *pn = 1.0;
    *dpn = 0.0;
    return;
  }
  for (int k = 1; k < n; ++k) {
    double p2 = ((2.0 * k + 1.0) * t * p1 - k * p0) / (k + 1.0);
    p0 = p1;
    p1 = p2;
  }
  *pn = p1;
  /* (1 - t^2) P_n' = n (P_{n-1} - t P_n) */
  *dpn = n * (p0 - t * p1) / (1.0 - t * t);
}

/* n-point Gauss-Legendre nodes/weights mapped to [0,1]: Newton iteration on
 * P_n from the classical cosine initial guesses; weights 2/((1-t^2)P_n'^2). */
void orc_gauss01(int n, double *x, double *w) {
  for (int i = 0; i < n; ++i) {
    double t = cos(ORC_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double pn, dpn;
      legendre_pn(n, t, &pn, &dpn);
      double dt = pn / dpn;
      t -= dt;
      if (fabs(dt) < 1e-17) break;
    }
    double pn, dpn;
    legendre_pn(n, t, &pn, &dpn);
    double wt = 2.0 / ((1.0 - t * t) * dpn * dpn);
    /* map [-1,1] -> [0,1], ascending order */
    x[n - 1 - i] = 0.5 * (t + 1.0);
    w[n - 1 - i] = 0.5 * wt;
  }
}

/* Collapsed rule on the reference triangle {r,s >= 0, r+s <= 1}:
 * r = a(1-b), s = b, weight w_a w_b (1-b); n points per direction. */
int orc_tri_rule(int n, double *r, double *s, double *w) {
  double g[32], gw[32];
  orc_gauss01(n, g, gw);
  int q = 0;
  for (int ia = 0; ia < n; ++ia)
    for (int ib = 0; ib < n; ++ib) {
      double a = g[ia], b = g[ib];
      r[q] = a * (1.0 - b);
      s[q] = b;
      w[q] = gw[ia] * gw[ib] * (1.0 - b);
      ++q;
    }
  return q;
}

/* Collapsed rule on the reference tetrahedron: r = a(1-b)(1-c), s = b(1-c),
 * t = c, weight w_a w_b w_c (1-b)(1-c)^2. */
int orc_tet_rule(int n, double *r, double *s, double *t, double *w) {
  double g[32], gw[32];
  orc_gauss01(n, g, gw);
  int q = 0;
  for (int ia = 0; ia < n; ++ia)
    for (int ib = 0; ib < n; ++ib)
      for (int ic = 0; ic < n; ++ic) {
        double a = g[ia], b = g[ib], c = g[ic];
        r[q] = a * (1.0 - b) * (1.0 - c);
        s[q] = b * (1.0 - c);
        t[q] = c;
        w[q] = gw[ia] * gw[ib] * gw[ic] * (1.0 - b) * (1.0 - c) * (1.0 - c);
        ++q;
      }
  return q;
}

/* ------------------------------------------------------------------------ */
/* Basis: orthonormal tensor Legendre of total degree p on the bounding box  */
/* ------------------------------------------------------------------------ */

int orc_nbasis(int dim, int p) {
  return dim == 2 ? (p + 1) * (p + 2) / 2 : (p + 1) * (p + 2) * (p + 3) / 6;
}

/* Exponent multi-indices in the fixed order: for k = 0..p;
 * 2D: for j = 0..k: (k-j, j);  3D: for l = 0..k: for j = 0..k-l: (k-j-l, j, l). */
static int basis_alpha(int dim, int p, int alpha[][3]) {
  int m = 0;
  for (int k = 0; k <= p; ++k) {
    if (dim == 2) {
      for (int j = 0; j <= k; ++j) {
        alpha[m][0] = k - j;
        alpha[m][1] = j;
        alpha[m][2] = 0;
        ++m;
      }
    } else {
      for (int l = 0; l <= k; ++l)
        for (int j = 0; j <= k - l; ++j) {
          alpha[m][0] = k - j - l;
          alpha[m][1] = j;
          alpha[m][2] = l;
          ++m;
        }
    }
  }
  return m;
}

void orc_basis_alpha(int dim, int p, int *out) {
  int al[128][3];
  int m = basis_alpha(dim, p, al);
  for (int i = 0; i < m; ++i)
    for (int d = 0; d < 3; ++d) out[3 * i + d] = al[i][d];
}

/* Legendre P_0..P_p and derivatives P'_0..P'_p at t. */
static void legendre_all(int p, double t, double *P, double *dP) {
  P[0] = 1.0;
  dP[0] = 0.0;
  if (p >= 1) {
    P[1] = t;
    dP[1] = 1.0;
  }
  for (int k = 1; k < p; ++k) {
    P[k + 1] = ((2.0 * k + 1.0) * t * P[k] - k * P[k - 1]) / (k + 1.0);
    dP[k + 1] = dP[k - 1] + (2.0 * k + 1.0) * P[k];
  }
}

/* phi_alpha(x) = prod_d sqrt((2 alpha_d + 1)/L_d) P_{alpha_d}(xi_d),
 * xi_d = (2 x_d - lo_d - hi_d)/L_d, L_d = hi_d - lo_d.
 * grad[i*dim + d] = d phi_i / d x_d. */
void orc_basis(int dim, int p, const double *lo, const double *hi, const double *x, double *phi,
               double *grad) {
  int al[128][3];
  int n = basis_alpha(dim, p, al);
  double P[3][32], dP[3][32], L[3];
  for (int d = 0; d < dim; ++d) {
    L[d] = hi[d] - lo[d];
    double xi = (2.0 * x[d] - lo[d] - hi[d]) / L[d];
    legendre_all(p, xi, P[d], dP[d]);
  }
  for (int i = 0; i < n; ++i) {
    double v = 1.0;
    double g[3] = {1.0, 1.0, 1.0};
    for (int d = 0; d < dim; ++d) {
      int a = al[i][d];
      double c = sqrt((2.0 * a + 1.0) / L[d]);
      v *= c * P[d][a];
      for (int e = 0; e < dim; ++e) {
        if (e == d)
          g[e] *= c * dP[d][a] * 2.0 / L[d];
        else
          g[e] *= c * P[d][a];
      }
    }
    phi[i] = v;
    if (grad)
      for (int d = 0; d < dim; ++d) grad[i * dim + d] = g[d];
  }
}

/* ------------------------------------------------------------------------ */
/* Problem data                                                              */
/* ------------------------------------------------------------------------ */

typedef struct {
  int dim;
  double b[3];     /* constant advection field */
  double c;        /* constant reaction */
  int source;      /* 0: f = 0, g_D = 0; 1: u = prod sin(pi x_d); 2: u = polynomial */
  double poly[20]; /* coefficients of u for source 2 (graded monomials, degree <= 3) */
  double c_sigma;  /* penalty constant */
  int coef;        /* 0: b and c the constants above; 1: the fields of the paper's 3D
                      advection-diffusion-reaction test (Sec. 4.2), see coef_at */
  int neumann;     /* Neumann part of the boundary (Eq. (2.2)): bit 2d + s marks the side
                      x_d = min (s = 0) or x_d = max (s = 1) of the vertices' bounding box;
                      a boundary face all of whose vertices lie on a marked side is a
                      Neumann face, every other boundary face a Dirichlet face */
  double fb0[3];   /* coef 2: b_d(x) = fb0[d] + sum_e fbx[3 d + e] x_e */
  double fbx[9];
  double fc[20];   /* coef 2: c(x) = sum_k fc[k] m_k(x), m_k the graded monomials of degree <= 3
                      in the order of poly (2D: the first 10) */
} orc_problem;

static int poly_exps(int dim, int e[][3]);
static double ipow(double x, int k);

/* Advection and reaction at x.  coef 1 is the paper's multi-GPU test problem
 * (Sec. 4.2: b = (1+x, 1+y, 1+z), c = 3 + xyz), written for any dimension as
 * b_d = 1 + x_d and c = 3 + prod_d x_d.  coef 2: an affine b and a cubic c
 * given by their coefficients (fb0, fbx, fc). */
static void coef_at(const orc_problem *pb, const double *x, double *b, double *c) {
  if (pb->coef == 2) {
    for (int d = 0; d < pb->dim; ++d) {
      double v = pb->fb0[d];
      for (int e = 0; e < pb->dim; ++e) v += pb->fbx[3 * d + e] * x[e];
      b[d] = v;
    }
    int ex[20][3];
    int m = poly_exps(pb->dim, ex);
    double s = 0.0;
    for (int k = 0; k < m; ++k) {
      double v = pb->fc[k];
      for (int d = 0; d < pb->dim; ++d) v *= ipow(x[d], ex[k][d]);
      s += v;
    }
    *c = s;
    return;
  }
  if (pb->coef == 1) {
    double prod = 1.0;
    for (int d = 0; d < pb->dim; ++d) {
      b[d] = 1.0 + x[d];
      prod *= x[d];
    }
    *c = 3.0 + prod;
  } else {
    for (int d = 0; d < pb->dim; ++d) b[d] = pb->b[d];
    *c = pb->c;
  }
}

/* Graded monomial exponents up to total degree 3 (2D: 10, 3D: 20). */
static int poly_exps(int dim, int e[][3]) {
  int m = 0;
  for (int k = 0; k <= 3; ++k) {
    if (dim == 2) {
      for (int j = 0; j <= k; ++j) {
        e[m][0] = k - j;
        e[m][1] = j;
        e[m][2] = 0;
        ++m;
      }
    } else {
      for (int l = 0; l <= k; ++l)
        for (int j = 0; j <= k - l; ++j) {
          e[m][0] = k - j - l;
          e[m][1] = j;
          e[m][2] = l;
          ++m;
        }
    }
  }
  return m;
}

static double ipow(double x, int k) {
  double r = 1.0;
  for (int i = 0; i < k; ++i) r *= x;
  return r;
}

/* sin(pi x) and cos(pi x) with the argument reduced exactly (x - 2 round(x/2)
 * and 1 - r are exact in floating point), so that sin(pi x) is exactly 0 at
 * integer x: u = g_D vanishes on the sides of the unit square / cube, and an
 * O(eps) residue there would be amplified by sigma in the Nitsche term of
 * the load functional. */
static double sin_pi(double x) {
  double r = x - 2.0 * nearbyint(0.5 * x); /* r in [-1, 1] */
  double sg = 1.0;
  if (r < 0.0) {
    r = -r;
    sg = -1.0;
  }
  if (r > 0.5) r = 1.0 - r; /* sin(pi r) = sin(pi (1 - r)) */
  return sg * sin(ORC_PI * r);
}

static double cos_pi(double x) {
  double r = fabs(x - 2.0 * nearbyint(0.5 * x)); /* cos is even, r in [0, 1] */
  return sin_pi(0.5 - r);                          /* cos(pi r) = sin(pi (1/2 - r)) */
}

/* Exact solution u, its gradient and Laplacian for the manufactured sources. */
static void exact_u(const orc_problem *pb, const double *x, double *u, double *gu, double *lap) {
  int dim = pb->dim;
  if (pb->source == 1) {
    double s[3], c[3];
    for (int d = 0; d < dim; ++d) {
      s[d] = sin_pi(x[d]);
      c[d] = cos_pi(x[d]);
    }
    double prod = 1.0;
    for (int d = 0; d < dim; ++d) prod *= s[d];
    *u = prod;
    for (int d = 0; d < dim; ++d) {
      double g = ORC_PI * c[d];
      for (int e = 0; e < dim; ++e)
        if (e != d) g *= s[e];
      gu[d] = g;
    }
    *lap = -dim * ORC_PI * ORC_PI * prod;
  } else if (pb->source == 2) {
    int ex[20][3];
    int m = poly_exps(dim, ex);
    double uu = 0.0, g[3] = {0, 0, 0}, l = 0.0;
    for (int k = 0; k < m; ++k) {
      double cf = pb->poly[k];
      if (cf == 0.0) continue;
      double v = cf;
      for (int d = 0; d < dim; ++d) v *= ipow(x[d], ex[k][d]);
      uu += v;
      for (int d = 0; d < dim; ++d) {
        if (ex[k][d] == 0) continue;
        double gd = cf * ex[k][d] * ipow(x[d], ex[k][d] - 1);
        for (int e = 0; e < dim; ++e)
          if (e != d) gd *= ipow(x[e], ex[k][e]);
        g[d] += gd;
        if (ex[k][d] >= 2) {
          double ld = cf * ex[k][d] * (ex[k][d] - 1) * ipow(x[d], ex[k][d] - 2);
          for (int e = 0; e < dim; ++e)
            if (e != d) ld *= ipow(x[e], ex[k][e]);
          l += ld;
        }
      }
    }
    *u = uu;
    for (int d = 0; d < dim; ++d) gu[d] = g[d];
    *lap = l;
  } else {
    *u = 0.0;
    for (int d = 0; d < dim; ++d) gu[d] = 0.0;
    *lap = 0.0;
  }
}

/* f = -a Lap u + b . grad u + c u  (Eq. (2.1) with A = a I, a constant on
 * the element); g_D = u. */
static double source_f(const orc_problem *pb, double a, const double *x) {
  double u, gu[3], lap, b[3], c;
  exact_u(pb, x, &u, gu, &lap);
  coef_at(pb, x, b, &c);
  double bg = 0.0;
  for (int d = 0; d < pb->dim; ++d) bg += b[d] * gu[d];
  return -a * lap + bg + c * u;
}

static double dirichlet_g(const orc_problem *pb, const double *x) {
  double u, gu[3], lap;
  exact_u(pb, x, &u, gu, &lap);
  return u;
}

/* g_N = n . (A grad u) = a grad u . n (Eq. (2.2), A = a I) at x for the
 * unit normal n. */
static double neumann_g(const orc_problem *pb, double a, const double *x, const double *n) {
  double u, gu[3], lap, g = 0.0;
  exact_u(pb, x, &u, gu, &lap);
  for (int d = 0; d < pb->dim; ++d) g += gu[d] * n[d];
  return a * g;
}

double orc_exact_u(const orc_problem *pb, const double *x) { return dirichlet_g(pb, x); }
double orc_source_f(const orc_problem *pb, double a, const double *x) { return source_f(pb, a, x); }

/* ------------------------------------------------------------------------ */
/* Mesh: elements, geometry, faces, interfaces                              */
/* ------------------------------------------------------------------------ */

typedef struct {
  int e[2];      /* e[0] < e[1] for interior; e[1] = -1 on the boundary */
  int v[3];      /* 2D: edge (v0, v1) traversed CCW by e[0]; 3D: triangle */
  double n[3];   /* unit normal pointing out of e[0] */
  double area;   /* |F| */
} orc_face;

typedef struct orc_mesh {
  int dim, nv, ne;
  double *X[3];
  int *eptr, *ev; /* 2D: vertex loops; 3D: tets (4 per entry) */
  /* geometry */
  double *vol, *cen, *lo, *hi, *h;
  /* faces sorted by (e0, e1, then appearance) */
  int nf;
  orc_face *f;
  /* element -> face incidence (CSR) */
  int *efptr, *ef;
  /* interfaces: groups of interior faces with the same element pair */
  int ni;
  int *ifptr; /* faces of interface k: f[ifptr[k] .. ifptr[k+1]) */
  int nbf;    /* number of boundary faces (they follow the interior ones) */
  double dlo[3], dhi[3]; /* bounding box of all vertices (the Neumann sides) */
} orc_mesh;

static double dist(const double *a, const double *b, int dim) {
  double s = 0.0;
  for (int d = 0; d < dim; ++d) s += (a[d] - b[d]) * (a[d] - b[d]);
  return sqrt(s);
}

static void vtx(const orc_mesh *m, int v, double *x) {
  for (int d = 0; d < m->dim; ++d) x[d] = m->X[d][v];
}

/* Area, area centroid, bounding box and diameter of each element. */
static void element_geometry(orc_mesh *m) {
  int dim = m->dim;
  for (int e = 0; e < m->ne; ++e) {
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    double vol = 0.0, cen[3] = {0, 0, 0}, h = 0.0;
    if (dim == 2) {
      int a = m->eptr[e], b = m->eptr[e + 1], k = b - a;
      for (int i = 0; i < k; ++i) {
        double p[3], q[3];
        vtx(m, m->ev[a + i], p);
        vtx(m, m->ev[a + (i + 1) % k], q);
        double cr = p[0] * q[1] - q[0] * p[1]; /* shoelace */
        vol += 0.5 * cr;
        cen[0] += (p[0] + q[0]) * cr / 6.0;
        cen[1] += (p[1] + q[1]) * cr / 6.0;
        for (int d = 0; d < 2; ++d) {
          if (p[d] < lo[d]) lo[d] = p[d];
          if (p[d] > hi[d]) hi[d] = p[d];
        }
        for (int j = 0; j < k; ++j) {
          double r[3];
          vtx(m, m->ev[a + j], r);
          double dd = dist(p, r, 2);
          if (dd > h) h = dd;
        }
      }
      cen[0] /= vol;
      cen[1] /= vol;
    } else {
      int a = m->eptr[e], b = m->eptr[e + 1];
      for (int t = a; t < b; ++t) {
        double P[4][3];
        for (int i = 0; i < 4; ++i) vtx(m, m->ev[4 * t + i], P[i]);
        double u[3], v[3], w[3];
        for (int d = 0; d < 3; ++d) {
          u[d] = P[1][d] - P[0][d];
          v[d] = P[2][d] - P[0][d];
          w[d] = P[3][d] - P[0][d];
        }
        double det = u[0] * (v[1] * w[2] - v[2] * w[1]) - u[1] * (v[0] * w[2] - v[2] * w[0]) +
                     u[2] * (v[0] * w[1] - v[1] * w[0]);
        double tv = fabs(det) / 6.0;
        vol += tv;
        for (int d = 0; d < 3; ++d)
          cen[d] += tv * 0.25 * (P[0][d] + P[1][d] + P[2][d] + P[3][d]);
        for (int i = 0; i < 4; ++i)
          for (int d = 0; d < 3; ++d) {
            if (P[i][d] < lo[d]) lo[d] = P[i][d];
            if (P[i][d] > hi[d]) hi[d] = P[i][d];
          }
      }
      for (int d = 0; d < 3; ++d) cen[d] /= vol;
      /* diameter: max distance over all vertex pairs of the element */
      for (int t = a; t < b; ++t)
        for (int i = 0; i < 4; ++i)
          for (int s = t; s < b; ++s)
            for (int j = 0; j < 4; ++j) {
              double p[3], q[3];
              vtx(m, m->ev[4 * t + i], p);
              vtx(m, m->ev[4 * s + j], q);
              double dd = dist(p, q, 3);
              if (dd > h) h = dd;
            }
    }
    m->vol[e] = vol;
    m->h[e] = h;
    for (int d = 0; d < dim; ++d) {
      m->cen[e * dim + d] = cen[d];
      m->lo[e * dim + d] = lo[d];
      m->hi[e * dim + d] = hi[d];
    }
  }
}

/* half-face record used for matching */
typedef struct {
  int64_t key[3];
  int elem;
  int v[3];
  double n[3];
  double area;
} halfface;

static int cmp_half(const void *pa, const void *pb) {
  const halfface *a = (const halfface *)pa, *b = (const halfface *)pb;
  for (int i = 0; i < 3; ++i) {
    if (a->key[i] < b->key[i]) return -1;
    if (a->key[i] > b->key[i]) return 1;
  }
  if (a->elem != b->elem) return a->elem < b->elem ? -1 : 1;
  return 0;
}

static int cmp_face(const void *pa, const void *pb) {
  const orc_face *a = (const orc_face *)pa, *b = (const orc_face *)pb;
  /* interior faces first (ordered by element pair), boundary faces last */
  int ab = a->e[1] < 0, bb = b->e[1] < 0;
  if (ab != bb) return ab - bb;
  if (a->e[0] != b->e[0]) return a->e[0] < b->e[0] ? -1 : 1;
  if (a->e[1] != b->e[1]) return a->e[1] < b->e[1] ? -1 : 1;
  for (int i = 0; i < 3; ++i)
    if (a->v[i] != b->v[i]) return a->v[i] < b->v[i] ? -1 : 1;
  return 0;
}

static void sort3(int64_t *k) {
  for (int i = 0; i < 3; ++i)
    for (int j = i + 1; j < 3; ++j)
      if (k[j] < k[i]) {
        int64_t t = k[i];
        k[i] = k[j];
        k[j] = t;
      }
}

/* Faces by matching element boundary pieces: 2D edges of the vertex loops,
 * 3D triangles of the tetrahedra.  A piece seen twice from the same element
 * is internal to it (3D) and dropped; seen from two elements it is an
 * interior face; seen once it is a boundary face. */
static int build_faces(orc_mesh *m) {
  int dim = m->dim;
  int nh = 0;
  if (dim == 2)
    nh = m->eptr[m->ne];
  else
    nh = 4 * m->eptr[m->ne];
  halfface *H = (halfface *)calloc((size_t)nh, sizeof(halfface));
  int q = 0;
  for (int e = 0; e < m->ne; ++e) {
    if (dim == 2) {
      int a = m->eptr[e], k = m->eptr[e + 1] - a;
      for (int i = 0; i < k; ++i) {
        int v0 = m->ev[a + i], v1 = m->ev[a + (i + 1) % k];
        double p[3], r[3];
        vtx(m, v0, p);
        vtx(m, v1, r);
        double tx = r[0] - p[0], ty = r[1] - p[1], len = sqrt(tx * tx + ty * ty);
        halfface *hf = &H[q++];
        hf->key[0] = v0 < v1 ? v0 : v1;
        hf->key[1] = v0 < v1 ? v1 : v0;
        hf->key[2] = -1;
        hf->elem = e;
        hf->v[0] = v0;
        hf->v[1] = v1;
        hf->v[2] = -1;
        /* CCW loop: the outward normal is the tangent turned clockwise */
        hf->n[0] = ty / len;
        hf->n[1] = -tx / len;
        hf->n[2] = 0.0;
        hf->area = len;
      }
    } else {
      for (int t = m->eptr[e]; t < m->eptr[e + 1]; ++t) {
        const int *tv = &m->ev[4 * t];
        for (int o = 0; o < 4; ++o) {
          int fv[3], c = 0;
          for (int i = 0; i < 4; ++i)
            if (i != o) fv[c++] = tv[i];
          double A[3], B[3], C[3], D[3];
          vtx(m, fv[0], A);
          vtx(m, fv[1], B);
          vtx(m, fv[2], C);
          vtx(m, tv[o], D);
          double u[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
          double v[3] = {C[0] - A[0], C[1] - A[1], C[2] - A[2]};
          double nn[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]};
          double len = sqrt(nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2]);
          double side = nn[0] * (D[0] - A[0]) + nn[1] * (D[1] - A[1]) + nn[2] * (D[2] - A[2]);
          double sg = side > 0 ? -1.0 : 1.0; /* point away from the opposite vertex */
          halfface *hf = &H[q++];
          for (int i = 0; i < 3; ++i) hf->key[i] = fv[i];
          sort3(hf->key);
          hf->elem = e;
          for (int i = 0; i < 3; ++i) {
            hf->v[i] = fv[i];
            hf->n[i] = sg * nn[i] / len;
          }
          hf->area = 0.5 * len;
        }
      }
    }
  }
  qsort(H, (size_t)nh, sizeof(halfface), cmp_half);
  orc_face *F = (orc_face *)calloc((size_t)nh, sizeof(orc_face));
  int nf = 0;
  for (int i = 0; i < nh;) {
    int j = i + 1;
    while (j < nh && H[j].key[0] == H[i].key[0] && H[j].key[1] == H[i].key[1] &&
           H[j].key[2] == H[i].key[2])
      ++j;
    int cnt = j - i;
    if (cnt > 2) {
      free(H);
      free(F);
      return -1; /* non-manifold */
    }
    if (cnt == 2 && H[i].elem == H[i + 1].elem) {
      /* internal to one element (3D agglomerate): not a face */
    } else {
      orc_face *f = &F[nf++];
      const halfface *h0 = &H[i]; /* lower element id first (sorted by elem) */
      f->e[0] = h0->elem;
      f->e[1] = cnt == 2 ? H[i + 1].elem : -1;
      for (int d = 0; d < 3; ++d) {
        f->v[d] = h0->v[d];
        f->n[d] = h0->n[d];
      }
      f->area = h0->area;
    }
    i = j;
  }
  free(H);
  qsort(F, (size_t)nf, sizeof(orc_face), cmp_face);
  m->f = F;
  m->nf = nf;
  /* interfaces */
  m->ifptr = (int *)malloc(sizeof(int) * (size_t)(nf + 1));
  int ni = 0, k = 0;
  while (k < nf && F[k].e[1] >= 0) {
    m->ifptr[ni++] = k;
    int j = k + 1;
    while (j < nf && F[j].e[1] >= 0 && F[j].e[0] == F[k].e[0] && F[j].e[1] == F[k].e[1]) ++j;
    k = j;
  }
  m->ifptr[ni] = k;
  m->ni = ni;
  m->nbf = nf - k;
  /* element -> face incidence */
  m->efptr = (int *)calloc((size_t)m->ne + 1, sizeof(int));
  for (int i = 0; i < nf; ++i) {
    m->efptr[F[i].e[0] + 1]++;
    if (F[i].e[1] >= 0) m->efptr[F[i].e[1] + 1]++;
  }
  for (int e = 0; e < m->ne; ++e) m->efptr[e + 1] += m->efptr[e];
  m->ef = (int *)malloc(sizeof(int) * (size_t)(m->efptr[m->ne] + 1));
  int *fill = (int *)calloc((size_t)m->ne, sizeof(int));
  for (int i = 0; i < nf; ++i)
    for (int s = 0; s < 2; ++s) {
      int e = F[i].e[s];
      if (e < 0) continue;
      m->ef[m->efptr[e] + fill[e]++] = i;
    }
  free(fill);
  return 0;
}

orc_mesh *orc_mesh_new(int dim, int nv, const double *x, const double *y, const double *z, int ne,
                       const int *eptr, const int *ev) {
  orc_mesh *m = (orc_mesh *)calloc(1, sizeof(orc_mesh));
  m->dim = dim;
  m->nv = nv;
  m->ne = ne;
  const double *src[3] = {x, y, z};
  for (int d = 0; d < dim; ++d) {
    m->X[d] = (double *)malloc(sizeof(double) * (size_t)nv);
    memcpy(m->X[d], src[d], sizeof(double) * (size_t)nv);
  }
  m->eptr = (int *)malloc(sizeof(int) * (size_t)(ne + 1));
  memcpy(m->eptr, eptr, sizeof(int) * (size_t)(ne + 1));
  size_t nev = (size_t)eptr[ne] * (dim == 2 ? 1 : 4);
  m->ev = (int *)malloc(sizeof(int) * (nev + 1));
  memcpy(m->ev, ev, sizeof(int) * nev);
  m->vol = (double *)malloc(sizeof(double) * (size_t)ne);
  m->h = (double *)malloc(sizeof(double) * (size_t)ne);
  m->cen = (double *)malloc(sizeof(double) * (size_t)ne * dim);
  m->lo = (double *)malloc(sizeof(double) * (size_t)ne * dim);
  m->hi = (double *)malloc(sizeof(double) * (size_t)ne * dim);
  for (int d = 0; d < dim; ++d) {
    m->dlo[d] = m->dhi[d] = nv > 0 ? m->X[d][0] : 0.0;
    for (int v = 1; v < nv; ++v) {
      if (m->X[d][v] < m->dlo[d]) m->dlo[d] = m->X[d][v];
      if (m->X[d][v] > m->dhi[d]) m->dhi[d] = m->X[d][v];
    }
  }
  element_geometry(m);
  if (build_faces(m) != 0) {
    return NULL;
  }
  return m;
}

void orc_mesh_free(orc_mesh *m) {
  if (!m) return;
  for (int d = 0; d < m->dim; ++d) free(m->X[d]);
  free(m->eptr);
  free(m->ev);
  free(m->vol);
  free(m->h);
  free(m->cen);
  free(m->lo);
  free(m->hi);
  free(m->f);
  free(m->efptr);
  free(m->ef);
  free(m->ifptr);
  free(m);
}

int orc_num_interfaces(const orc_mesh *m) { return m->ni; }
int orc_num_faces(const orc_mesh *m) { return m->nf; }
int orc_num_boundary_faces(const orc_mesh *m) { return m->nbf; }

void orc_interfaces(const orc_mesh *m, int *e0, int *e1, int *nfaces) {
  for (int k = 0; k < m->ni; ++k) {
    const orc_face *f = &m->f[m->ifptr[k]];
    e0[k] = f->e[0];
    e1[k] = f->e[1];
    nfaces[k] = m->ifptr[k + 1] - m->ifptr[k];
  }
}

void orc_geometry(const orc_mesh *m, double *vol, double *cen, double *lo, double *hi, double *h) {
  int dim = m->dim;
  memcpy(vol, m->vol, sizeof(double) * (size_t)m->ne);
  memcpy(h, m->h, sizeof(double) * (size_t)m->ne);
  memcpy(cen, m->cen, sizeof(double) * (size_t)m->ne * dim);
  memcpy(lo, m->lo, sizeof(double) * (size_t)m->ne * dim);
  memcpy(hi, m->hi, sizeof(double) * (size_t)m->ne * dim);
}

/* ------------------------------------------------------------------------ */
/* Quadrature points of an element and of a face                            */
/* ------------------------------------------------------------------------ */

/* Volume rule of element e with n Gauss points per collapsed direction:
 * 2D fan triangles (centroid, v_k, v_{k+1}), 3D the element's tetrahedra.
 * Returns the number of points written (x: [q*dim], w: physical weights). */
/* Number of points orc_volume_points writes for element e: n^dim per
 * sub-simplex (2D: one triangle per loop edge; 3D: the element's tets). */
int orc_volume_point_count(const orc_mesh *m, int e, int n) {
  int per = m->dim == 2 ? n * n : n * n * n;
  return (m->eptr[e + 1] - m->eptr[e]) * per;
}

int orc_volume_points(const orc_mesh *m, int e, int n, double *xq, double *wq) {
  int dim = m->dim, q = 0;
  if (dim == 2) {
    double r[1024], s[1024], w[1024];
    int nq = orc_tri_rule(n, r, s, w);
    int a = m->eptr[e], k = m->eptr[e + 1] - a;
    const double *c = &m->cen[2 * e];
    for (int t = 0; t < k; ++t) {
      double p1[3], p2[3];
      vtx(m, m->ev[a + t], p1);
      vtx(m, m->ev[a + (t + 1) % k], p2);
      double e1[2] = {p1[0] - c[0], p1[1] - c[1]}, e2[2] = {p2[0] - c[0], p2[1] - c[1]};
      double J = fabs(e1[0] * e2[1] - e1[1] * e2[0]);
      for (int i = 0; i < nq; ++i) {
        xq[2 * q] = c[0] + r[i] * e1[0] + s[i] * e2[0];
        xq[2 * q + 1] = c[1] + r[i] * e1[1] + s[i] * e2[1];
        wq[q] = w[i] * J;
        ++q;
      }
    }
  } else {
    static __thread double r[4096], s[4096], t3[4096], w[4096];
    int nq = orc_tet_rule(n, r, s, t3, w);
    for (int t = m->eptr[e]; t < m->eptr[e + 1]; ++t) {
      double P[4][3];
      for (int i = 0; i < 4; ++i) vtx(m, m->ev[4 * t + i], P[i]);
      double u[3], v[3], z[3];
      for (int d = 0; d < 3; ++d) {
        u[d] = P[1][d] - P[0][d];
        v[d] = P[2][d] - P[0][d];
        z[d] = P[3][d] - P[0][d];
      }
      double J = fabs(u[0] * (v[1] * z[2] - v[2] * z[1]) - u[1] * (v[0] * z[2] - v[2] * z[0]) +
                      u[2] * (v[0] * z[1] - v[1] * z[0]));
      for (int i = 0; i < nq; ++i) {
        for (int d = 0; d < 3; ++d) xq[3 * q + d] = P[0][d] + r[i] * u[d] + s[i] * v[d] + t3[i] * z[d];
        wq[q] = w[i] * J;
        ++q;
      }
    }
  }
  return q;
}

/* Face rule with n Gauss points: 2D edge (n points), 3D triangle (n^2
 * collapsed points).  Weights carry |F| (2D) or 2|F| * reference weight (3D). */
static int face_points(const orc_mesh *m, const orc_face *f, int n, double *xq, double *wq) {
  int dim = m->dim, q = 0;
  if (dim == 2) {
    double g[32], gw[32];
    orc_gauss01(n, g, gw);
    double p[3], r[3];
    vtx(m, f->v[0], p);
    vtx(m, f->v[1], r);
    for (int i = 0; i < n; ++i) {
      xq[2 * q] = p[0] + g[i] * (r[0] - p[0]);
      xq[2 * q + 1] = p[1] + g[i] * (r[1] - p[1]);
      wq[q] = gw[i] * f->area;
      ++q;
    }
  } else {
    double r[1024], s[1024], w[1024];
    int nq = orc_tri_rule(n, r, s, w);
    double A[3], B[3], C[3];
    vtx(m, f->v[0], A);
    vtx(m, f->v[1], B);
    vtx(m, f->v[2], C);
    for (int i = 0; i < nq; ++i) {
      for (int d = 0; d < 3; ++d) xq[3 * q + d] = A[d] + r[i] * (B[d] - A[d]) + s[i] * (C[d] - A[d]);
      wq[q] = w[i] * 2.0 * f->area;
      ++q;
    }
  }
  return q;
}

/* ------------------------------------------------------------------------ */
/* Penalty                                                                   */
/* ------------------------------------------------------------------------ */

/* sigma_F = C_sigma * max_{k in faces' elements} a_k p_k^2 / h_k. */
static double penalty(const orc_mesh *m, const orc_face *f, const int *p, const double *a,
                      double c_sigma) {
  double s = 0.0;
  for (int side = 0; side < 2; ++side) {
    int e = f->e[side];
    if (e < 0) continue;
    double v = a[e] * p[e] * p[e] / m->h[e];
    if (v > s) s = v;
  }
  return c_sigma * s;
}

double orc_face_penalty(const orc_mesh *m, int face, const int *p, const double *a, double c_sigma) {
  return penalty(m, &m->f[face], p, a, c_sigma);
}

/* ------------------------------------------------------------------------ */
/* Local forms                                                               */
/* ------------------------------------------------------------------------ */

#define ORC_NMAX 128

static void elem_basis(const orc_mesh *m, int e, int p, const double *x, double *phi, double *grad) {
  orc_basis(m->dim, p, &m->lo[e * m->dim], &m->hi[e * m->dim], x, phi, grad);
}

/* Volume part of B (Eq. (2.4), first line) on element e, A = a_e I:
 *   A_ee[i][j] += sum_q w_q ( a grad phi_j . grad phi_i
 *                             + (b . grad phi_j) phi_i + c phi_j phi_i ),
 * row i = test function, column j = trial function.  Adds into out (n x n). */
static void volume_block(const orc_mesh *m, int e, int p, double a, const orc_problem *pb,
                         double *out) {
  int dim = m->dim, n = orc_nbasis(dim, p);
  int nq_cap = orc_volume_point_count(m, e, p + 2);
  double *xq = (double *)malloc(sizeof(double) * (size_t)nq_cap * 3);
  double *wq = (double *)malloc(sizeof(double) * (size_t)nq_cap);
  int nq = orc_volume_points(m, e, p + 2, xq, wq);
  double phi[ORC_NMAX], grad[ORC_NMAX * 3];
  for (int q = 0; q < nq; ++q) {
    double b[3], c;
    coef_at(pb, &xq[q * dim], b, &c);
    elem_basis(m, e, p, &xq[q * dim], phi, grad);
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        double gg = 0.0, bg = 0.0;
        for (int d = 0; d < dim; ++d) {
          gg += grad[j * dim + d] * grad[i * dim + d];
          bg += b[d] * grad[j * dim + d];
        }
        out[i * n + j] += wq[q] * (a * gg + bg * phi[i] + c * phi[j] * phi[i]);
      }
  }
  free(xq);
  free(wq);
}

/* Is boundary face f on the Neumann part of the boundary?  Its vertices
 * (2 in 2D, 3 in 3D) all lie on one marked side of the domain's box, compared
 * exactly. */
static int neumann_face(const orc_mesh *m, const orc_face *f, const orc_problem *pb) {
  if (f->e[1] >= 0 || pb->neumann == 0) return 0;
  int nvf = m->dim == 2 ? 2 : 3;
  for (int d = 0; d < m->dim; ++d)
    for (int s = 0; s < 2; ++s) {
      if (!(pb->neumann >> (2 * d + s) & 1)) continue;
      double side = s ? m->dhi[d] : m->dlo[d];
      int on = 1;
      for (int i = 0; i < nvf; ++i)
        if (m->X[d][f->v[i]] != side) on = 0;
      if (on) return 1;
    }
  return 0;
}

/* Contribution of one face to the blocks (r, c) with r, c in {0,1} (0 = the
 * face's first element, whose outward normal is nF).  From Eq. (2.4):
 *   - {a grad w} . [v] - {a grad v} . [w] + sigma [w] . [v]
 * with {.} the average (the trace itself on a boundary face), [v] = v_0 nF -
 * v_1 nF (v_0 nF on a boundary face), and the upwind terms
 *   - (b . n_k)(w^+ - w^-) v^+ on the inflow part of each element k
 *   - (b . n) w v on the inflow part of the Dirichlet boundary.
 * blk[r][c] points to an n_r x n_c row-major block (test r, trial c) or NULL. */
static void face_blocks(const orc_mesh *m, const orc_face *f, const int *p, const double *a,
                        const orc_problem *pb, double *blk[2][2]) {
  int dim = m->dim;
  int bnd = f->e[1] < 0;
  int ns = bnd ? 1 : 2;
  /* Eq. (2.4): the face integrals run over Gamma_int and the Dirichlet part
   * only, the boundary inflow term over the inflow part of the Dirichlet
   * boundary only; a Neumann face adds nothing to B */
  if (neumann_face(m, f, pb)) return;
  int pp[2] = {p[f->e[0]], bnd ? 0 : p[f->e[1]]};
  int pmax = pp[0] > pp[1] ? pp[0] : pp[1];
  int nb[2] = {orc_nbasis(dim, pp[0]), bnd ? 0 : orc_nbasis(dim, pp[1])};
  double aa[2] = {a[f->e[0]], bnd ? 0.0 : a[f->e[1]]};
  double sig = penalty(m, f, p, a, pb->c_sigma);
  double avg = bnd ? 1.0 : 0.5; /* weight of each side in the average */
  double sgn[2] = {1.0, -1.0};  /* jump [v] = (v_0 - v_1) nF */
  double xq[4096 * 3], wq[4096];
  int nq = face_points(m, f, pmax + 1, xq, wq);
  double phi[2][ORC_NMAX], grad[2][ORC_NMAX * 3], dn[2][ORC_NMAX];
  for (int q = 0; q < nq; ++q) {
    /* b . nF at the point: the inflow parts are decided point by point */
    double b[3], c, bn = 0.0;
    coef_at(pb, &xq[q * dim], b, &c);
    for (int d = 0; d < dim; ++d) bn += b[d] * f->n[d];
    for (int s = 0; s < ns; ++s) {
      elem_basis(m, f->e[s], pp[s], &xq[q * dim], phi[s], grad[s]);
      for (int i = 0; i < nb[s]; ++i) {
        double v = 0.0;
        for (int d = 0; d < dim; ++d) v += grad[s][i * dim + d] * f->n[d];
        dn[s][i] = v; /* grad phi . nF */
      }
    }
    for (int r = 0; r < ns; ++r)
      for (int c = 0; c < ns; ++c) {
        double *B = blk[r][c];
        if (!B) continue;
        for (int i = 0; i < nb[r]; ++i)
          for (int j = 0; j < nb[c]; ++j) {
            /* test v = phi^r_i, trial w = phi^c_j */
            double t = 0.0;
            t -= avg * aa[c] * dn[c][j] * sgn[r] * phi[r][i]; /* {a grad w}.[v] */
            t -= avg * aa[r] * dn[r][i] * sgn[c] * phi[c][j]; /* {a grad v}.[w] */
            t += sig * sgn[r] * sgn[c] * phi[c][j] * phi[r][i];
            /* upwind: inflow part of element 0 is where b . nF < 0, of
             * element 1 where b . nF > 0 (b . n = 0 is outflow). */
            if (bn < 0.0 && r == 0) {
              /* -(b.n0)(w^0 - w^1) v^0 ;  on the boundary -(b.n) w^0 v^0 */
              if (c == 0) t -= bn * phi[0][j] * phi[0][i];
              if (c == 1) t += bn * phi[1][j] * phi[0][i];
            }
            if (bn > 0.0 && r == 1) {
              /* -(b.n1)(w^1 - w^0) v^1 with n1 = -nF */
              if (c == 1) t += bn * phi[1][j] * phi[1][i];
              if (c == 0) t -= bn * phi[0][j] * phi[1][i];
            }
            B[i * nb[c] + j] += wq[q] * t;
          }
      }
  }
}

/* Boundary-face part of l (Eq. (2.5)) for the element of boundary face f:
 * on a Dirichlet face
 *   - (b . n) g_D v on the inflow part,  - g_D (a grad v . n - sigma v),
 * on a Neumann face  g_N v. */
static void face_rhs(const orc_mesh *m, const orc_face *f, const int *p, const double *a,
                     const orc_problem *pb, double *out) {
  int dim = m->dim, e = f->e[0], pe = p[e], n = orc_nbasis(dim, pe);
  double xq[4096 * 3], wq[4096];
  int nq = face_points(m, f, pe + 1, xq, wq);
  double phi[ORC_NMAX], grad[ORC_NMAX * 3];
  if (neumann_face(m, f, pb)) {
    for (int q = 0; q < nq; ++q) {
      double g = neumann_g(pb, a[e], &xq[q * dim], f->n);
      elem_basis(m, e, pe, &xq[q * dim], phi, grad);
      for (int i = 0; i < n; ++i) out[i] += wq[q] * g * phi[i];
    }
    return;
  }
  double sig = penalty(m, f, p, a, pb->c_sigma);
  for (int q = 0; q < nq; ++q) {
    double b[3], c, bn = 0.0;
    coef_at(pb, &xq[q * dim], b, &c);
    for (int d = 0; d < dim; ++d) bn += b[d] * f->n[d];
    double g = dirichlet_g(pb, &xq[q * dim]);
    elem_basis(m, e, pe, &xq[q * dim], phi, grad);
    for (int i = 0; i < n; ++i) {
      double dn = 0.0;
      for (int d = 0; d < dim; ++d) dn += grad[i * dim + d] * f->n[d];
      double t = -g * (a[e] * dn - sig * phi[i]);
      if (bn < 0.0) t -= bn * g * phi[i];
      out[i] += wq[q] * t;
    }
  }
}

/* Volume part of l: sum_q w_q f(x_q) phi_i(x_q). */
static void volume_rhs(const orc_mesh *m, int e, int p, double a, const orc_problem *pb,
                       double *out) {
  int dim = m->dim, n = orc_nbasis(dim, p);
  int nq_cap = orc_volume_point_count(m, e, p + 2);
  double *xq = (double *)malloc(sizeof(double) * (size_t)nq_cap * 3);
  double *wq = (double *)malloc(sizeof(double) * (size_t)nq_cap);
  int nq = orc_volume_points(m, e, p + 2, xq, wq);
  double phi[ORC_NMAX];
  for (int q = 0; q < nq; ++q) {
    double fv = source_f(pb, a, &xq[q * dim]);
    elem_basis(m, e, p, &xq[q * dim], phi, NULL);
    for (int i = 0; i < n; ++i) out[i] += wq[q] * fv * phi[i];
  }
  free(xq);
  free(wq);
}

/* ------------------------------------------------------------------------ */
/* Assembly drivers                                                          */
/* ------------------------------------------------------------------------ */

/* Diagonal block of element e: volume part plus, for each face of e, the
 * (e, e) block of that face, in the element's face order. */
void orc_diag_block(const orc_mesh *m, int e, const int *p, const double *a, const orc_problem *pb,
                    double *out) {
  int n = orc_nbasis(m->dim, p[e]);
  memset(out, 0, sizeof(double) * (size_t)n * n);
  volume_block(m, e, p[e], a[e], pb, out);
  for (int k = m->efptr[e]; k < m->efptr[e + 1]; ++k) {
    const orc_face *f = &m->f[m->ef[k]];
    double *blk[2][2] = {{NULL, NULL}, {NULL, NULL}};
    int side = f->e[0] == e ? 0 : 1;
    blk[side][side] = out;
    face_blocks(m, f, p, a, pb, blk);
  }
}

/* Off-diagonal blocks of interface k (elements e0 < e1): A_01 is
 * n0 x n1 (test in e0, trial in e1) and A_10 is n1 x n0. */
void orc_offdiag_blocks(const orc_mesh *m, int k, const int *p, const double *a,
                        const orc_problem *pb, double *a01, double *a10) {
  const orc_face *f0 = &m->f[m->ifptr[k]];
  int n0 = orc_nbasis(m->dim, p[f0->e[0]]), n1 = orc_nbasis(m->dim, p[f0->e[1]]);
  memset(a01, 0, sizeof(double) * (size_t)n0 * n1);
  memset(a10, 0, sizeof(double) * (size_t)n0 * n1);
  for (int i = m->ifptr[k]; i < m->ifptr[k + 1]; ++i) {
    double *blk[2][2] = {{NULL, a01}, {a10, NULL}};
    face_blocks(m, &m->f[i], p, a, pb, blk);
  }
}

/* Load vector entries of element e. */
void orc_rhs_element(const orc_mesh *m, int e, const int *p, const double *a, const orc_problem *pb,
                     double *out) {
  int n = orc_nbasis(m->dim, p[e]);
  memset(out, 0, sizeof(double) * (size_t)n);
  volume_rhs(m, e, p[e], a[e], pb, out);
  for (int k = m->efptr[e]; k < m->efptr[e + 1]; ++k) {
    const orc_face *f = &m->f[m->ef[k]];
    if (f->e[1] < 0) face_rhs(m, f, p, a, pb, out);
  }
}

/* Whole-mesh assembly for listed elements and interfaces.  Output offsets
 * (in doubles) are given by the caller.  nthreads <= 0: library default. */
void orc_assemble(const orc_mesh *m, const int *p, const double *a, const orc_problem *pb, int n_el,
                  const int *elems, double *diag, const int64_t *diag_off, double *rhs,
                  const int64_t *rhs_off, int n_if, const int *ifaces, double *a01, double *a10,
                  const int64_t *off_off, int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 16)
  for (int k = 0; k < n_el; ++k) {
    if (diag) orc_diag_block(m, elems[k], p, a, pb, diag + diag_off[k]);
    if (rhs) orc_rhs_element(m, elems[k], p, a, pb, rhs + rhs_off[k]);
  }
#pragma omp parallel for schedule(dynamic, 64)
  for (int k = 0; k < n_if; ++k)
    orc_offdiag_blocks(m, ifaces[k], p, a, pb, a01 + off_off[k], a10 + off_off[k]);
}

int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Moments (pins for the subdivision + rules)                                */
/* ------------------------------------------------------------------------ */

/* int_e x^i y^j (z^k) with the element's volume rule (n points/direction). */
double orc_moment_rule(const orc_mesh *m, int e, int n, int i, int j, int k) {
  int nq_cap = orc_volume_point_count(m, e, n);
  double *xq = (double *)malloc(sizeof(double) * (size_t)nq_cap * 3);
  double *wq = (double *)malloc(sizeof(double) * (size_t)nq_cap);
  int nq = orc_volume_points(m, e, n, xq, wq), dim = m->dim;
  double s = 0.0;
  for (int q = 0; q < nq; ++q) {
    double v = ipow(xq[q * dim], i) * ipow(xq[q * dim + 1], j);
    if (dim == 3) v *= ipow(xq[q * dim + 2], k);
    s += wq[q] * v;
  }
  free(xq);
  free(wq);
  return s;
}

/* 2D: int_e x^i y^j = 1/(i+1) * sum over boundary edges of
 * int_edge x^(i+1) y^j n_x ds (divergence theorem), each edge integral by
 * Gauss with enough points for its polynomial degree i+j+1. */
double orc_moment_divergence2d(int nvert, const double *xs, const double *ys, int i, int j) {
  int deg = i + j + 1, n = deg / 2 + 1;
  double g[32], gw[32];
  orc_gauss01(n, g, gw);
  double s = 0.0;
  for (int k = 0; k < nvert; ++k) {
    double x0 = xs[k], y0 = ys[k], x1 = xs[(k + 1) % nvert], y1 = ys[(k + 1) % nvert];
    double tx = x1 - x0, ty = y1 - y0, len = sqrt(tx * tx + ty * ty);
    if (len == 0.0) continue;
    double nx = ty / len;
    for (int q = 0; q < n; ++q) {
      double x = x0 + g[q] * tx, y = y0 + g[q] * ty;
      s += gw[q] * len * ipow(x, i + 1) * ipow(y, j) * nx;
    }
  }
  return s / (i + 1);
}

/* 3D: int_e x^i y^j z^k = 1/(i+1) * sum over the element's boundary
 * triangles F of int_F x^(i+1) y^j z^k n_x dS (divergence theorem with the
 * field (x^(i+1) y^j z^k / (i+1), 0, 0)), n the unit normal out of e; each
 * triangle integral by the collapsed rule with enough points for degree
 * i+j+k+1 (exact to 2n-2). */
double orc_moment_divergence3d(const orc_mesh *m, int e, int i, int j, int k) {
  int deg = i + j + k + 1, n = deg / 2 + 2;
  double r[1024], sq[1024], w[1024];
  int nq = orc_tri_rule(n, r, sq, w);
  double s = 0.0;
  for (int t = m->efptr[e]; t < m->efptr[e + 1]; ++t) {
    const orc_face *f = &m->f[m->ef[t]];
    double nx = f->e[0] == e ? f->n[0] : -f->n[0];
    double A[3], B[3], C[3];
    vtx(m, f->v[0], A);
    vtx(m, f->v[1], B);
    vtx(m, f->v[2], C);
    for (int q = 0; q < nq; ++q) {
      double x[3];
      for (int d = 0; d < 3; ++d) x[d] = A[d] + r[q] * (B[d] - A[d]) + sq[q] * (C[d] - A[d]);
      s += w[q] * 2.0 * f->area * ipow(x[0], i + 1) * ipow(x[1], j) * ipow(x[2], k) * nx;
    }
  }
  return s / (i + 1);
}

/* ------------------------------------------------------------------------ */
/* Per-piece access for the pins                                             */
/* ------------------------------------------------------------------------ */

/* Volume part only of element e's diagonal block. */
void orc_volume_block(const orc_mesh *m, int e, const int *p, const double *a,
                      const orc_problem *pb, double *out) {
  int n = orc_nbasis(m->dim, p[e]);
  memset(out, 0, sizeof(double) * (size_t)n * n);
  volume_block(m, e, p[e], a[e], pb, out);
}

/* Elements of face k (e1 = -1 on the boundary) and its measure. */
void orc_face_info(const orc_mesh *m, int k, int *e0, int *e1, double *area, double *normal) {
  const orc_face *f = &m->f[k];
  *e0 = f->e[0];
  *e1 = f->e[1];
  *area = f->area;
  for (int d = 0; d < 3; ++d) normal[d] = f->n[d];
}

/* The n-point rule on face k (the rule the face terms use): points xq
 * [q][dim] and weights wq[q] including the face measure; returns q. */
int orc_face_points(const orc_mesh *m, int k, int n, double *xq, double *wq) {
  return face_points(m, &m->f[k], n, xq, wq);
}

/* All blocks of face k alone: b00 (n0 x n0), b01, b10, b11 (NULL allowed). */
void orc_face_blocks(const orc_mesh *m, int k, const int *p, const double *a,
                     const orc_problem *pb, double *b00, double *b01, double *b10, double *b11) {
  const orc_face *f = &m->f[k];
  int n0 = orc_nbasis(m->dim, p[f->e[0]]);
  int n1 = f->e[1] >= 0 ? orc_nbasis(m->dim, p[f->e[1]]) : 0;
  if (b00) memset(b00, 0, sizeof(double) * (size_t)n0 * n0);
  if (b01) memset(b01, 0, sizeof(double) * (size_t)n0 * n1);
  if (b10) memset(b10, 0, sizeof(double) * (size_t)n0 * n1);
  if (b11) memset(b11, 0, sizeof(double) * (size_t)n1 * n1);
  double *blk[2][2] = {{b00, f->e[1] >= 0 ? b01 : NULL}, {f->e[1] >= 0 ? b10 : NULL, f->e[1] >= 0 ? b11 : NULL}};
  face_blocks(m, f, p, a, pb, blk);
}
