"""Space-time slab assembly for the parabolic special case (Sec. 2.3): plain
FP64 numpy on top of the oracle's geometry, rules and basis.  Test
infrastructure: only the test suite may import it.

The slab I_n x D = (t0, t1] x D over a 2D polygonal or 3D polyhedral mesh
(the paper's computations use 2D) is cut into prisms
kappa_n = I_n x kappa.  On each prism the basis is psi_(k, alpha)(t, x) =
T_k(t) phi_alpha(x), with T_k = sqrt((2k + 1) / tau) P_k(2 (t - t0) / tau - 1)
orthonormal on I_n (tau = t1 - t0) and phi_alpha the element's orthonormal
bounding-box Legendre basis of the oracle.  Two spaces (Sec. 2.3): P_p,
space-time total degree k + |alpha| <= p, and PQ_p, k <= p with |alpha| <= p.

The slab problem is the per-slab system at the end of Sec. 2.3, every
boundary face Dirichlet:

    int_In [(d_t U, W)_D + B_S(U, W)] dt + (U^+_{n-1}, W^+_{n-1})_D
        = int_In [(f, W)_D - int_dD g (a grad W . n - sigma W) ds] dt
          + (U^-_{n-1}, W^+_{n-1})_D,

B_S the spatial dG form of the same section: the volume terms a grad U .
grad W + (w . grad U) W + c U W, the upwind terms of the wind w on the inflow
parts, and the SIPG consistency, symmetry and penalty terms on the interior
and Dirichlet faces.  Readings: a is constant per element (A = a I), w and c
are constants; the penalty of a lateral face I_n x F is the spatial one of F
(10 p^2 / h with the prism's degree p and the spatial diameter h), since the
face terms are spatial jumps; time integrals use p + 2 Gauss points, the
spatial ones the oracle's rules (sub-simplex rule with p + 2 points per
direction, max(p0, p1) + 1 points per face direction), exact for every
integrand here.
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial import legendre as npl

from . import Mesh, basis, gauss01, nbasis


def st_index(p: int, space: str, dim: int = 2):
    """(k, j) pairs of a prism of degree p: temporal degree k and index j of the
    spatial basis function (ordered by total degree, so j < nbasis(dim, d)
    exactly when |alpha_j| <= d)."""
    if space not in ("P", "PQ"):
        raise ValueError(space)
    out = []
    for k in range(p + 1):
        d = p - k if space == "P" else p
        out.extend((k, j) for j in range(nbasis(dim, d)))
    return out


def time_basis(p: int, t: float, t0: float, tau: float):
    """T_k(t) and T_k'(t) for k = 0..p."""
    s = 2.0 * (t - t0) / tau - 1.0
    val = np.zeros(p + 1)
    der = np.zeros(p + 1)
    for k in range(p + 1):
        ck = [0.0] * k + [1.0]
        scale = np.sqrt((2 * k + 1) / tau)
        val[k] = scale * npl.legval(s, ck)
        der[k] = scale * npl.legval(s, npl.legder(ck)) * 2.0 / tau
    return val, der


class Slab:
    """The slab (t0, t1] x D over the oracle mesh om (2D or 3D), degrees p[e]
    (>= 1), diffusion a[e], wind w (dim-vector), reaction c, space "P" or
    "PQ"."""

    def __init__(self, om: Mesh, p, a, w, c: float, space: str, t0: float, t1: float,
                 c_sigma: float = 10.0):
        if om.dim not in (2, 3):
            raise ValueError("the slab oracle takes a 2D or 3D spatial mesh")
        self.om, self.space, self.t0, self.t1 = om, space, float(t0), float(t1)
        self.dim = om.dim
        self.tau = self.t1 - self.t0
        self.p = np.asarray(p, dtype=np.int32)
        self.a = np.asarray(a, dtype=np.float64)
        self.w = np.asarray(w, dtype=np.float64)
        if self.w.shape != (self.dim,):
            raise ValueError("the wind has one component per space dimension")
        self.c = float(c)
        self.c_sigma = float(c_sigma)
        self.idx = [st_index(int(pe), space, self.dim) for pe in self.p]
        self.off = np.concatenate([[0], np.cumsum([len(ix) for ix in self.idx])]).astype(np.int64)

    def _psi(self, e: int, t: float, x):
        """Values, time derivatives and spatial gradients of element e's prism
        basis at (t, x)."""
        pe = int(self.p[e])
        phi, grad = basis(self.dim, pe, self.om.lo[e], self.om.hi[e], x)
        T, dT = time_basis(pe, t, self.t0, self.tau)
        K = np.array([k for k, _ in self.idx[e]])
        J = np.array([j for _, j in self.idx[e]])
        return T[K] * phi[J], dT[K] * phi[J], T[K][:, None] * grad[J]

    def value(self, U, e: int, t: float, x) -> float:
        v, _, _ = self._psi(e, t, x)
        return float(v @ U[self.off[e]:self.off[e + 1]])

    def assemble(self, f, g, u_prev):
        """Dense slab matrix A (test rows, trial columns) and load vector F.
        f(t, x), g(t, x): source and Dirichlet data; u_prev(e, x): U^-_{n-1} on
        the spatial element e (the previous slab's solution at t0, or u_0)."""
        om, n = self.om, int(self.off[-1])
        A = np.zeros((n, n))
        F = np.zeros(n)

        def blk(r, s):
            return A[self.off[r]:self.off[r + 1], self.off[s]:self.off[s + 1]]

        for e in range(om.ne):
            pe = int(self.p[e])
            tg, tw = gauss01(pe + 2)
            xq, wq = om.volume_points(e, pe + 2)
            Ae, Fe = blk(e, e), F[self.off[e]:self.off[e + 1]]
            for x, wx in zip(xq, wq):
                for tt, wt in zip(tg, tw):
                    t = self.t0 + self.tau * tt
                    W = wx * wt * self.tau
                    psi, dpsi, gpsi = self._psi(e, t, x)
                    # (d_t U, W) + a grad U . grad W + (w . grad U) W + c U W
                    Ae += W * (np.outer(psi, dpsi) + self.a[e] * gpsi @ gpsi.T
                               + np.outer(psi, gpsi @ self.w) + self.c * np.outer(psi, psi))
                    Fe += W * f(t, x) * psi
                # the time jump at t0: (U^+, W^+) and (U^-, W^+)
                psi0, _, _ = self._psi(e, self.t0, x)
                Ae += wx * np.outer(psi0, psi0)
                Fe += wx * u_prev(e, x) * psi0

        for k in range(om.nf):
            e0, e1, _, nrm = om.face_info(k)
            bnd = e1 < 0
            sides = [e0] if bnd else [e0, e1]
            pmax = max(int(self.p[s]) for s in sides)
            xq, wq = om.face_points(k, pmax + 1)
            tg, tw = gauss01(pmax + 2)
            sig = om.face_penalty(k, self.p, self.a, self.c_sigma)
            avg = 1.0 if bnd else 0.5
            sgn = [1.0, -1.0]  # [v] = (v_0 - v_1) n_F, n_F out of e0
            bn = float(self.w @ nrm)
            for x, wx in zip(xq, wq):
                for tt, wt in zip(tg, tw):
                    t = self.t0 + self.tau * tt
                    W = wx * wt * self.tau
                    ps, dn = [], []
                    for s in sides:
                        v, _, gr = self._psi(s, t, x)
                        ps.append(v)
                        dn.append(gr @ nrm)
                    for r in range(len(sides)):
                        for q in range(len(sides)):
                            ar, aq = self.a[sides[r]], self.a[sides[q]]
                            term = (-avg * aq * sgn[r] * np.outer(ps[r], dn[q])
                                    - avg * ar * sgn[q] * np.outer(dn[r], ps[q])
                                    + sig * sgn[r] * sgn[q] * np.outer(ps[r], ps[q]))
                            # upwind: inflow of e0 where w . n_F < 0, of e1 where > 0
                            if bn < 0.0 and r == 0:
                                term += (-bn if q == 0 else bn) * np.outer(ps[0], ps[q])
                            if bn > 0.0 and r == 1:
                                term += (bn if q == 1 else -bn) * np.outer(ps[1], ps[q])
                            blk(sides[r], sides[q])[...] += W * term
                    if bnd:
                        gv = g(t, x)
                        rhs = -gv * (self.a[e0] * dn[0] - sig * ps[0])
                        if bn < 0.0:
                            rhs -= bn * gv * ps[0]
                        F[self.off[e0]:self.off[e0 + 1]] += W * rhs
        return A, F
