"""Pins of the learned-quadrature oracle (CPU): moments, Gauss-Newton,
acceptance and the network's backward pass, against independent facts."""
import numpy as np
import pytest

import oracle as O
import oracle.learned as L
from paper_2007_04881_gb300 import meshgen as mg


@pytest.fixture(scope="module")
def cells():
    m = mg.voronoi_square(120, 31)
    out = []
    for e in range(m.ne):
        v = m.elem_v[m.elem_vptr[e]:m.elem_vptr[e + 1]]
        out.append((m.x[v], m.y[v]))
    return out


def test_legendre_products_orthogonal_on_square():
    t, w = np.polynomial.legendre.leggauss(8)
    X, Y = np.meshgrid(t, t, indexing="ij")
    W = np.outer(w, w).ravel()
    Lv, _, _ = L.lp_basis(X.ravel(), Y.ravel())
    G = (Lv * W) @ Lv.T
    a = np.array([e[0] for e in L.exps()])
    b = np.array([e[1] for e in L.exps()])
    np.testing.assert_allclose(G, np.diag(4.0 / ((2 * a + 1) * (2 * b + 1))), atol=1e-13)


def test_moments_of_square_and_subrectangle():
    sq = np.array([-1.0, 1, 1, -1]), np.array([-1.0, -1, 1, 1])
    M = L.lp_moments(*sq)
    assert abs(M[0] - 4) < 1e-14 and np.abs(M[1:]).max() < 1e-14
    # sub-rectangle [x0,x1]x[y0,y1]: product of 1D Gauss integrals (library rule)
    x0, x1, y0, y1 = -0.7, 0.4, -0.2, 0.9
    rect = np.array([x0, x1, x1, x0]), np.array([y0, y0, y1, y1])
    t, w = np.polynomial.legendre.leggauss(8)
    xs, ys = 0.5 * (x1 - x0) * (t + 1) + x0, 0.5 * (y1 - y0) * (t + 1) + y0
    Px, _ = L.legendre(6, xs)
    Py, _ = L.legendre(6, ys)
    ex = np.array([np.sum(0.5 * (x1 - x0) * w * Px[a]) * np.sum(0.5 * (y1 - y0) * w * Py[b]) for a, b in L.exps()])
    np.testing.assert_allclose(L.lp_moments(*rect), ex, atol=1e-14)


def test_moments_match_fan_rule_and_c_divergence(cells):
    for xs, ys in cells[::10]:
        xi, eta = L.normalize(xs, ys)
        # monomials: the C oracle's divergence-theorem routine
        mc = np.array([O.moment_divergence2d(xi, eta, a, b) for a, b in L.exps()])
        np.testing.assert_allclose(L.mono_moments(xi, eta), mc, atol=1e-14)
        # Legendre products: the fan sub-triangle rule in normalised coordinates
        mesh = mg.Mesh2D(np.ascontiguousarray(xi), np.ascontiguousarray(eta), np.array([0, xi.size], np.int32),
                         np.arange(xi.size, dtype=np.int32))
        om = O.Mesh(mesh)
        xq, wq = om.volume_points(0, 6)
        Lq, _, _ = L.lp_basis(xq[:, 0], xq[:, 1])
        np.testing.assert_allclose(L.lp_moments(xi, eta), Lq @ wq, atol=1e-13)


def test_gauss_newton_converges_quadratically(cells):
    for xs, ys in cells[::7]:
        xi, eta = L.normalize(xs, ys)
        M = L.lp_moments(xi, eta)
        z = L.canonical_rule(M[0])
        res = []
        for _ in range(9):
            res.append(np.abs(L.residual(z, M)).max() / M[0])
            z = L.gn_step(z, M)
        res.append(np.abs(L.residual(z, M)).max() / M[0])
        assert res[-1] < 1e-13
        ok, rel = L.accept(z, xi, eta)
        assert ok, rel
        # quadratic phase: once below 1e-3 the next residual is below C r^2
        for r0, r1 in zip(res[:-1], res[1:]):
            if 1e-11 < r0 < 1e-3:
                assert r1 < 50 * r0 * r0 + 1e-14


def test_accept_rejects_outside_point_and_wrong_weights(cells):
    xs, ys = cells[0]
    xi, eta = L.normalize(xs, ys)
    M = L.lp_moments(xi, eta)
    z = L.canonical_rule(M[0])
    for _ in range(9):
        z = L.gn_step(z, M)
    assert L.accept(z, xi, eta)[0]
    bad = z.copy()
    bad[2 * L.NPT] *= 1.0 + 1e-6
    assert not L.accept(bad, xi, eta)[0]
    bad = z.copy()
    bad[0] = 1.5
    assert not L.accept(bad, xi, eta)[0]


def test_mlp_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    shapes = [(24, 128), (128,), (128, 128), (128,), (128, 84), (84,)]
    params = [rng.normal(0, 0.2, s) for s in shapes]
    X = rng.normal(0, 0.5, (7, 24))
    T = rng.normal(0, 0.5, (7, 84))
    loss, grads = L.mlp_loss_grad(params, X, T)
    h = 1e-6
    for pi, (P, G) in enumerate(zip(params, grads)):
        flat = P.reshape(-1)
        for idx in rng.choice(flat.size, 5, replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp, _ = L.mlp_loss_grad(params, X, T)
            flat[idx] = old - h
            lm, _ = L.mlp_loss_grad(params, X, T)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - G.reshape(-1)[idx]) < 1e-7 * max(1.0, abs(fd)), (pi, idx, fd, G.reshape(-1)[idx])
