"""Oracle (test infrastructure) for the learned reduced quadrature: plain
numpy FP64 restatements, used only by the tests.

Pieces, on an element mapped to its bounding box [-1, 1]^2 (xi = 2(x-lo)/L - 1):
  * moments of the 28 Legendre products P_a(xi) P_b(eta), a + b <= 6, by the
    divergence theorem (exact: Gauss on each edge with enough points);
  * monomial moments xi^a eta^b the same way (the acceptance test);
  * minimum-norm Gauss-Newton on the 28 moment equations in the 84 unknowns
    (28 points and 28 weights): dz = -J^T (J J^T)^-1 r;
  * the canonical starting rule (4 x 7 tensor Gauss points in [-0.9, 0.9]^2,
    weights scaled to the element's area);
  * the network: 24 -> 128 -> 128 -> 84, tanh hidden layers, linear output,
    forward and backward (for the gradient check of the CUDA kernels).
A rule is accepted when max_k |monomial residual_k| / |element| < 1e-10 and
every point lies in the bounding box.
"""
from __future__ import annotations

import numpy as np

DEG = 6
NMOM = (DEG + 1) * (DEG + 2) // 2  # 28
NPT = 28
NIN = 24
H = 128
NOUT = 3 * NPT


def exps(deg=DEG):
    """(a, b) in the basis order: k = 0..deg, j = 0..k: (k - j, j)."""
    return [(k - j, j) for k in range(deg + 1) for j in range(k + 1)]


def legendre(n, t):
    """P_0..P_n and P'_0..P'_n at t (arrays)."""
    t = np.asarray(t, dtype=np.float64)
    P = np.zeros((n + 1,) + t.shape)
    dP = np.zeros_like(P)
    P[0] = 1.0
    if n >= 1:
        P[1] = t
        dP[1] = 1.0
    for k in range(1, n):
        P[k + 1] = ((2 * k + 1) * t * P[k] - k * P[k - 1]) / (k + 1)
        dP[k + 1] = dP[k - 1] + (2 * k + 1) * P[k]
    return P, dP


def lp_basis(xi, eta):
    """Legendre products L_k = P_a(xi) P_b(eta) and their derivatives, [28, npts]."""
    Px, dPx = legendre(DEG, xi)
    Py, dPy = legendre(DEG, eta)
    E = exps()
    L = np.stack([Px[a] * Py[b] for a, b in E])
    Lx = np.stack([dPx[a] * Py[b] for a, b in E])
    Ly = np.stack([Px[a] * dPy[b] for a, b in E])
    return L, Lx, Ly


def normalize(xs, ys):
    lo = np.array([xs.min(), ys.min()])
    hi = np.array([xs.max(), ys.max()])
    L = hi - lo
    return 2 * (xs - lo[0]) / L[0] - 1, 2 * (ys - lo[1]) / L[1] - 1


def _edge_gauss(n):
    t, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (t + 1), 0.5 * w


def lp_moments(xi, eta):
    """int_polygon P_a(xi) P_b(eta): divergence theorem with the antiderivative
    Q_a (Q_a' = P_a) in xi, integrated along each edge times n_xi."""
    t, w = _edge_gauss(DEG // 2 + 2)
    E = exps()
    out = np.zeros(NMOM)
    n = xi.size
    for i in range(n):
        x0, y0, x1, y1 = xi[i], eta[i], xi[(i + 1) % n], eta[(i + 1) % n]
        dx, dy = x1 - x0, y1 - y0
        # outward normal times length for a CCW loop: (dy, -dx)
        xs, ys = x0 + t * dx, y0 + t * dy
        Px, _ = legendre(DEG + 1, xs)
        Py, _ = legendre(DEG, ys)
        for k, (a, b) in enumerate(E):
            Qa = xs if a == 0 else (Px[a + 1] - Px[a - 1]) / (2 * a + 1)
            out[k] += np.sum(w * Qa * Py[b]) * dy
    return out


def mono_moments(xi, eta):
    """int_polygon xi^a eta^b by the divergence theorem."""
    t, w = _edge_gauss(DEG // 2 + 2)
    out = np.zeros(NMOM)
    n = xi.size
    for i in range(n):
        x0, y0, x1, y1 = xi[i], eta[i], xi[(i + 1) % n], eta[(i + 1) % n]
        xs, ys = x0 + t * (x1 - x0), y0 + t * (y1 - y0)
        for k, (a, b) in enumerate(exps()):
            out[k] += np.sum(w * xs ** (a + 1) * ys ** b) / (a + 1) * (y1 - y0)
    return out


def canonical_rule(area):
    """4 x 7 tensor Gauss points in [-0.9, 0.9]^2, weights scaled to area."""
    tx, wx = np.polynomial.legendre.leggauss(4)
    ty, wy = np.polynomial.legendre.leggauss(7)
    X, Y = np.meshgrid(0.9 * tx, 0.9 * ty, indexing="ij")
    W = np.outer(wx, wy) / 4.0 * area
    return np.concatenate([X.ravel(), Y.ravel(), W.ravel()])


def residual(z, M):
    x, y, w = z[:NPT], z[NPT:2 * NPT], z[2 * NPT:]
    L, _, _ = lp_basis(x, y)
    return L @ w - M


def gn_step(z, M):
    """One minimum-norm Gauss-Newton step on r(z) = sum_i w_i L(p_i) - M."""
    x, y, w = z[:NPT], z[NPT:2 * NPT], z[2 * NPT:]
    L, Lx, Ly = lp_basis(x, y)
    r = L @ w - M
    J = np.concatenate([Lx * w, Ly * w, L], axis=1)  # [28, 84]: d/dx, d/dy, d/dw
    u = np.linalg.solve(J @ J.T, r)
    return z - J.T @ u


def accept(z, xi, eta, tol=1e-10):
    x, y, w = z[:NPT], z[NPT:2 * NPT], z[2 * NPT:]
    Mm = mono_moments(xi, eta)
    got = np.array([np.sum(w * x ** a * y ** b) for a, b in exps()])
    area = Mm[0]
    inside = bool(np.all(np.abs(x) <= 1.0) and np.all(np.abs(y) <= 1.0))
    return bool(np.max(np.abs(got - Mm)) / area < tol and inside), float(np.max(np.abs(got - Mm)) / area)


# ---------------------------------------------------------------------------
# the network (FP64 reference of the forward and backward passes)
# ---------------------------------------------------------------------------


def mlp_forward(params, X):
    """params = (W1 [24,128], b1, W2 [128,128], b2, W3 [128,84], b3); X [n, 24]."""
    W1, b1, W2, b2, W3, b3 = params
    z1 = X @ W1 + b1
    h1 = np.tanh(z1)
    z2 = h1 @ W2 + b2
    h2 = np.tanh(z2)
    out = h2 @ W3 + b3
    return out, (X, h1, h2)


def mlp_loss_grad(params, X, T):
    """Mean squared error 1/(2n) sum |out - T|^2 and its gradient."""
    W1, b1, W2, b2, W3, b3 = params
    out, (X_, h1, h2) = mlp_forward(params, X)
    n = X.shape[0]
    d = (out - T) / n
    loss = 0.5 * np.sum((out - T) ** 2) / n
    gW3 = h2.T @ d
    gb3 = d.sum(0)
    dh2 = d @ W3.T * (1 - h2 ** 2)
    gW2 = h1.T @ dh2
    gb2 = dh2.sum(0)
    dh1 = dh2 @ W2.T * (1 - h1 ** 2)
    gW1 = X_.T @ dh1
    gb1 = dh1.sum(0)
    return loss, (gW1, gb1, gW2, gb2, gW3, gb3)


def bf16_round(a):
    """Round to the nearest bfloat16 (ties to even), returned as float32."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)
