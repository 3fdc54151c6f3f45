"""Pins for the FP64 oracle against facts fixed by mathematics, not by the oracle.

Each test checks one piece of the oracle (quadrature, geometry, basis, local
forms, SIPG signs, penalty) against a closed form, a library routine, an
invariant or an exact solution, chosen so that a dropped term, a wrong sign
or a swapped index breaks at least one of them.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2007_04881_gb300 import meshgen as mg

# ---------------------------------------------------------------------------
# quadrature rules
# ---------------------------------------------------------------------------


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 12])
def test_gauss01_matches_numpy_and_is_exact(n):
    x, w = O.gauss01(n)
    t, wt = np.polynomial.legendre.leggauss(n)  # library routine on [-1, 1]
    np.testing.assert_allclose(x, 0.5 * (t + 1), rtol=0, atol=1e-15)
    np.testing.assert_allclose(w, 0.5 * wt, rtol=0, atol=1e-15)
    for k in range(2 * n):
        assert abs(np.sum(w * x ** k) - 1.0 / (k + 1)) < 1e-15


@pytest.mark.parametrize("n", [1, 2, 3, 4, 6, 7])
def test_triangle_rule_closed_form(n):
    """int_T r^i s^j = i! j! / (i+j+2)! on the reference triangle, exact for
    total degree <= 2n-2 (collapsed Gauss)."""
    r, s, w = O.tri_rule(n)
    for i in range(2 * n - 1):
        for j in range(2 * n - 1 - i):
            exact = math.factorial(i) * math.factorial(j) / math.factorial(i + j + 2)
            assert abs(np.sum(w * r ** i * s ** j) - exact) < 1e-15 * max(1.0, 1 / exact) * exact + 1e-17
    # the claimed degree is tight: some monomial of degree 2n-1 is not exact
    errs = []
    i_tot = 2 * n - 1
    for i in range(i_tot + 1):
        j = i_tot - i
        exact = math.factorial(i) * math.factorial(j) / math.factorial(i + j + 2)
        errs.append(abs(np.sum(w * r ** i * s ** j) - exact) / exact)
    assert max(errs) > 1e-10


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6])
def test_tet_rule_closed_form(n):
    """int_T r^i s^j t^k = i! j! k! / (i+j+k+3)!, exact for degree <= 2n-3."""
    r, s, t, w = O.tet_rule(n)
    for i in range(2 * n - 2):
        for j in range(2 * n - 2 - i):
            for k in range(2 * n - 2 - i - j):
                exact = math.factorial(i) * math.factorial(j) * math.factorial(k) / math.factorial(i + j + k + 3)
                got = np.sum(w * r ** i * s ** j * t ** k)
                assert abs(got - exact) <= 1e-14 * exact


# ---------------------------------------------------------------------------
# geometry and subdivision
# ---------------------------------------------------------------------------


@pytest.fixture(scope="module")
def vor64():
    return mg.voronoi_square(64, 11)


def _loop(mesh, e):
    v = mesh.elem_v[mesh.elem_vptr[e]:mesh.elem_vptr[e + 1]]
    return mesh.x[v], mesh.y[v]


def test_area_sum_and_geometry(vor64):
    om = O.Mesh(vor64)
    assert abs(om.vol.sum() - 1.0) < 1e-14
    for e in range(om.ne):
        xs, ys = _loop(vor64, e)
        np.testing.assert_allclose(om.lo[e], [xs.min(), ys.min()], atol=0)
        np.testing.assert_allclose(om.hi[e], [xs.max(), ys.max()], atol=0)
        P = np.c_[xs, ys]
        h = np.max(np.linalg.norm(P[:, None, :] - P[None, :, :], axis=-1))
        assert abs(om.h[e] - h) < 1e-15
        # centroid by the divergence theorem moments
        A = O.moment_divergence2d(xs, ys, 0, 0)
        cx = O.moment_divergence2d(xs, ys, 1, 0) / A
        cy = O.moment_divergence2d(xs, ys, 0, 1) / A
        assert abs(A - om.vol[e]) < 1e-16
        assert abs(cx - om.cen[e, 0]) < 1e-14 and abs(cy - om.cen[e, 1]) < 1e-14


def test_divergence_moments_closed_form_rectangle():
    xs = np.array([0.2, 0.9, 0.9, 0.2])
    ys = np.array([-0.1, -0.1, 0.4, 0.4])
    for i in range(6):
        for j in range(6):
            exact = (0.9 ** (i + 1) - 0.2 ** (i + 1)) / (i + 1) * (0.4 ** (j + 1) - (-0.1) ** (j + 1)) / (j + 1)
            assert abs(O.moment_divergence2d(xs, ys, i, j) - exact) < 1e-15


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_fan_rule_moments_match_divergence_theorem(vor64, p):
    """Volume rule (fan from the centroid, (p+2)^2 collapsed points per
    triangle) integrates every monomial of degree <= 2p+2 exactly."""
    om = O.Mesh(vor64)
    for e in range(0, om.ne, 7):
        xs, ys = _loop(vor64, e)
        for i in range(2 * p + 3):
            for j in range(2 * p + 3 - i):
                ex = O.moment_divergence2d(xs, ys, i, j)
                got = om.moment_rule(e, p + 2, i, j)
                assert abs(got - ex) <= 1e-13 * abs(om.vol[e]), (e, i, j, got, ex)


@pytest.mark.parametrize("p", [2, 4, 6])
def test_green_legendre_moments_with_p_plus_1_edge_points(vor64, p):
    """The identity behind the exact-moment volume path.  In an element's box
    coordinates, the integral of P_c(xi) P_d(eta) over the polygon equals the
    closed integral of Q_c(xi) P_d(eta) d eta, with Q_0 = P_1 and
    Q_c = (P_{c+1} - P_{c-1}) / (2c + 1).  Along an edge that integrand has
    degree c + 1 + d <= 2p + 1, so p + 1 Gauss points per edge are exact.
    The reference is the oracle's fan rule with (p + 2)^2 points per
    sub-triangle, exact for the same degrees."""
    from numpy.polynomial import legendre as npl

    def leg(k, x):
        return npl.legval(x, [0.0] * k + [1.0])

    tr, ts, tw = O.tri_rule(p + 2)
    g, gw = O.gauss01(p + 1)
    q = 2 * p
    for e in range(0, vor64.ne, 9):
        xs, ys = _loop(vor64, e)
        xi = 2 * (xs - xs.min()) / (xs.max() - xs.min()) - 1
        eta = 2 * (ys - ys.min()) / (ys.max() - ys.min()) - 1
        k = xi.size
        x1, y1 = np.roll(xi, -1), np.roll(eta, -1)
        cr = xi * y1 - x1 * eta
        cx, cy = ((xi + x1) * cr).sum() / (3 * cr.sum()), ((eta + y1) * cr).sum() / (3 * cr.sum())
        # fan points: (c, v_i, v_{i+1}) for every i
        ax, ay, bx, by = xi - cx, eta - cy, x1 - cx, y1 - cy
        det = np.abs(ax * by - ay * bx)
        FX = cx + np.outer(ax, tr) + np.outer(bx, ts)
        FY = cy + np.outer(ay, tr) + np.outer(by, ts)
        FW = np.outer(det, tw)
        # edge points of the closed integral, counter-clockwise
        EX = xi[:, None] + np.outer(x1 - xi, g)
        EY = eta[:, None] + np.outer(y1 - eta, g)
        EW = np.outer(y1 - eta, gw)
        for c in range(q + 1):
            qc = EX if c == 0 else (leg(c + 1, EX) - leg(c - 1, EX)) / (2 * c + 1)
            pc = leg(c, FX)
            for d in range(q + 1 - c):
                fan = np.sum(FW * pc * leg(d, FY))
                green = np.sum(EW * qc * leg(d, EY))
                assert abs(green - fan) < 1e-12, (e, k, c, d, green, fan)


def test_faces_and_interfaces_counts(vor64):
    om = O.Mesh(vor64)
    nedges = vor64.elem_vptr[-1]
    # every loop edge is one side of a face: 2 * interior + boundary = edges
    assert 2 * om.nf - om.nbf == nedges
    # Voronoi cells are convex: one face per interface
    assert np.all(om.if_nfaces == 1)
    # Euler's formula for the planar subdivision: V - E + F = 1
    assert vor64.nv - om.nf + om.ne == 1
    # boundary length = 4
    L = 0.0
    for k in range(om.nf):
        e0, e1, area, nrm = om.face_info(k)
        if e1 < 0:
            L += area
            assert abs(abs(nrm[0]) + abs(nrm[1]) - 1.0) < 1e-12  # axis-aligned sides
    assert abs(L - 4.0) < 1e-13


# ---------------------------------------------------------------------------
# basis
# ---------------------------------------------------------------------------


def _legendre_dd(m, n):
    """int_{-1}^{1} P_m' P_n' = min(m,n)(min(m,n)+1) if m+n even, else 0."""
    k = min(m, n)
    return float(k * (k + 1)) if (m + n) % 2 == 0 else 0.0


@pytest.mark.parametrize("p", [1, 2, 3, 5])
def test_mass_identity_and_stiffness_closed_form_on_rectangle(p):
    """An axis-aligned rectangle is its own bounding box: the orthonormal
    basis has mass matrix I, and the stiffness has a closed form from
    int P_m' P_n' and Legendre orthogonality."""
    x0, x1, y0, y1 = 0.3, 1.1, -0.2, 0.25
    mesh = mg.rectangle_grid(1, 1, x0, x1, y0, y1)
    om = O.Mesh(mesh)
    pa = np.array([p])
    # mass: a = 0, b = 0, c = 1 -> volume block = mass matrix
    pb = O.make_problem(2, c=1.0)
    M = om.volume_block(0, pa, np.array([0.0]), pb)
    n = O.nbasis(2, p)
    np.testing.assert_allclose(M, np.eye(n), atol=2e-15)
    # stiffness: a = 1, c = 0
    pb = O.make_problem(2)
    K = om.volume_block(0, pa, np.array([1.0]), pb)
    al = O.basis_alpha(2, p)
    Lx, Ly = x1 - x0, y1 - y0
    Kex = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            (a1, a2), (b1, b2) = al[i], al[j]
            kx = math.sqrt((2 * a1 + 1) * (2 * b1 + 1)) / Lx * (2 / Lx) * _legendre_dd(a1, b1) * (a2 == b2)
            ky = math.sqrt((2 * a2 + 1) * (2 * b2 + 1)) / Ly * (2 / Ly) * _legendre_dd(a2, b2) * (a1 == b1)
            Kex[i, j] = kx + ky
    np.testing.assert_allclose(K, Kex, atol=1e-12 * np.abs(Kex).max())


def test_advection_block_closed_form_on_rectangle():
    """int (b . grad phi_j) phi_i on a rectangle: with int_{-1}^{1} P_n' P_m =
    2 if m < n and m+n odd, else 0 (test row i, trial column j)."""
    x0, x1, y0, y1 = 0.0, 0.5, 0.0, 2.0
    p = 3
    om = O.Mesh(mg.rectangle_grid(1, 1, x0, x1, y0, y1))
    bx, by = 0.7, -1.3
    B = om.volume_block(0, np.array([p]), np.array([0.0]), O.make_problem(2, b=(bx, by)))
    al = O.basis_alpha(2, p)
    n = al.shape[0]
    Lx, Ly = x1 - x0, y1 - y0

    def dp(nn, m):  # int P_nn' P_m
        return 2.0 if (m < nn and (m + nn) % 2 == 1) else 0.0

    Bex = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            (i1, i2), (j1, j2) = al[i], al[j]
            cx = math.sqrt((2 * i1 + 1) * (2 * j1 + 1)) / Lx
            cy = math.sqrt((2 * i2 + 1) * (2 * j2 + 1)) / Ly
            # x-derivative of the trial function: (2/Lx) P'_{j1}, dx = Lx/2 dxi
            tx = cx * dp(j1, i1) * (i2 == j2) * (2.0 / (2 * i2 + 1)) * (Ly / 2) * cy
            ty = cy * dp(j2, i2) * (i1 == j1) * (2.0 / (2 * i1 + 1)) * (Lx / 2) * cx
            Bex[i, j] = bx * tx + by * ty
    np.testing.assert_allclose(B, Bex, atol=1e-13 * np.abs(Bex).max())


def test_mass00_equals_area_over_bbox(vor64):
    om = O.Mesh(vor64)
    pb = O.make_problem(2, c=1.0)
    p = np.full(om.ne, 2)
    for e in range(0, om.ne, 5):
        M = om.volume_block(e, p, np.zeros(om.ne), pb)
        box = np.prod(om.hi[e] - om.lo[e])
        assert abs(M[0, 0] - om.vol[e] / box) < 1e-14


def test_diffusion_block_psd_constant_kernel(vor64):
    om = O.Mesh(vor64)
    pb = O.make_problem(2)
    p = np.full(om.ne, 3)
    a = mg.draw_log_uniform(om.ne, 3, -2, 2)
    for e in range(0, om.ne, 9):
        K = om.volume_block(e, p, a, pb)
        s = np.abs(K).max()
        assert np.abs(K - K.T).max() < 1e-13 * s
        assert np.abs(K[0]).max() < 1e-13 * s and np.abs(K[:, 0]).max() < 1e-13 * s
        assert np.linalg.eigvalsh(0.5 * (K + K.T)).min() > -1e-12 * s


# ---------------------------------------------------------------------------
# SIPG faces, penalty
# ---------------------------------------------------------------------------


def test_penalty_formula(vor64):
    om = O.Mesh(vor64)
    p = mg.draw_degrees(om.ne, 4, 1, 4).astype(np.int32)
    a = mg.draw_log_uniform(om.ne, 4, -2, 2)
    for k in range(0, om.nf, 5):
        e0, e1, _, _ = om.face_info(k)
        cand = []
        for e in (e0, e1):
            if e < 0:
                continue
            xs, ys = _loop(vor64, e)
            P = np.c_[xs, ys]
            h = np.max(np.linalg.norm(P[:, None] - P[None], axis=-1))
            cand.append(a[e] * p[e] ** 2 / h)
        assert abs(om.face_penalty(k, p, a, 10.0) - 10.0 * max(cand)) <= 1e-14 * 10 * max(cand)


def test_face_blocks_two_squares_closed_form():
    """Two unit squares sharing x = 1 (a = 1, b = 0, c = 0, p = 1).  On the
    shared edge xi = +1 in the left square and -1 in the right one, so the
    face blocks follow from P_k(+-1) = (+-1)^k, P_k'(+-1) = (+-1)^(k+1) k(k+1)/2
    and orthonormality in y."""
    mesh = mg.rectangle_grid(2, 1, 0.0, 2.0, 0.0, 1.0)
    om = O.Mesh(mesh)
    assert om.ni == 1
    k_int = [k for k in range(om.nf) if om.face_info(k)[1] >= 0][0]
    p = np.array([1, 1])
    a = np.array([1.0, 1.0])
    pb = O.make_problem(2, c_sigma=10.0)
    fb = om.face_blocks(k_int, p, a, pb)
    h = math.sqrt(2.0)
    sig = 10.0 * 1 / h
    al = O.basis_alpha(2, 1)

    def trace(side, i):  # phi_i and d phi_i/dx at the edge, as coefficient of the y-part
        a1, a2 = al[i]
        xi = 1.0 if side == 0 else -1.0
        c = math.sqrt(2 * a1 + 1)
        val = c * xi ** a1
        der = c * (xi ** (a1 + 1)) * a1 * (a1 + 1) / 2 * 2.0  # d/dx = 2/Lx d/dxi, Lx = 1
        return val, der, a2

    n = al.shape[0]
    exp = {k: np.zeros((n, n)) for k in ("b00", "b01", "b10", "b11")}
    sgn = (1.0, -1.0)
    for r in range(2):
        for c in range(2):
            blk = exp[f"b{r}{c}"]
            for i in range(n):
                for j in range(n):
                    vi, di, yi = trace(r, i)
                    vj, dj, yj = trace(c, j)
                    if yi != yj:
                        continue  # orthonormal y-parts
                    t = -0.5 * dj * sgn[r] * vi - 0.5 * di * sgn[c] * vj + sig * sgn[r] * sgn[c] * vi * vj
                    blk[i, j] = t
    for k in exp:
        np.testing.assert_allclose(fb[k], exp[k], atol=1e-13)


def _assemble_dense(om, p, a, pb):
    blk = om.assemble(p, a, pb)
    return O.global_matrix(om, p, blk)


def test_sipg_diffusion_symmetric_positive_definite(vor64):
    om = O.Mesh(vor64)
    p = mg.draw_degrees(om.ne, 5, 1, 3).astype(np.int32)
    a = mg.draw_log_uniform(om.ne, 5, -1, 1)
    A, _, _ = _assemble_dense(om, p, a, O.make_problem(2))
    s = np.abs(A).max()
    assert np.abs(A - A.T).max() < 1e-12 * s
    assert np.linalg.eigvalsh(0.5 * (A + A.T)).min() > 0


def test_interior_face_annihilates_constant(vor64):
    """[1] = 0 and grad 1 = 0: an interior face's 2x2 block system applied to
    the constant function gives zero (constant = sqrt(|bbox|) * phi_0)."""
    om = O.Mesh(vor64)
    p = mg.draw_degrees(om.ne, 6, 1, 4).astype(np.int32)
    a = mg.draw_log_uniform(om.ne, 6, -2, 2)
    pb = O.make_problem(2, b=(0.9, -0.4), c=0.0)
    for k in range(0, om.nf, 3):
        e0, e1, _, _ = om.face_info(k)
        if e1 < 0:
            continue
        fb = om.face_blocks(k, p, a, pb)
        c0 = np.zeros(O.nbasis(2, p[e0]))
        c1 = np.zeros(O.nbasis(2, p[e1]))
        c0[0] = math.sqrt(np.prod(om.hi[e0] - om.lo[e0]))
        c1[0] = math.sqrt(np.prod(om.hi[e1] - om.lo[e1]))
        r0 = fb["b00"] @ c0 + fb["b01"] @ c1
        r1 = fb["b10"] @ c0 + fb["b11"] @ c1
        s = max(np.abs(fb["b00"]).max(), np.abs(fb["b11"]).max())
        assert np.abs(r0).max() < 1e-12 * s and np.abs(r1).max() < 1e-12 * s


# ---------------------------------------------------------------------------
# whole form: polynomial reproduction (consistency) and convergence
# ---------------------------------------------------------------------------


def _solve_and_error(om, p, a, pb, npts=4):
    A, F, off = _assemble_dense(om, p, a, pb)
    U = np.linalg.solve(A, F)
    err = 0.0
    for e in range(om.ne):
        xq, _ = om.volume_points(e, npts)
        for x in xq[:: max(1, xq.shape[0] // 12)]:
            phi, _ = O.basis(om.dim, int(p[e]), om.lo[e], om.hi[e], x)
            err = max(err, abs(phi @ U[off[e]:off[e + 1]] - O.exact_u(pb, x)))
    return err


@pytest.mark.parametrize(
    "b,c,poly,plo,phi_",
    [
        ((0.0, 0.0), 0.0, [1, 1, -2, 0, 1, 0], 2, 2),
        ((1.0, 0.5), 1.0, [1, 1, -2, 0, 1, 0], 2, 3),
        ((-0.8, 0.6), 0.3, [0.5, -1, 2, 1, 0.5, -0.7], 2, 4),
        ((0.3, -1.1), 2.0, [0, 1, 0, 0, 0, 0, 0.5, -1, 0.25, 1], 3, 4),
        ((1.0, 0.0), 1.0, [2, -1, 0.5], 1, 3),
    ],
)
def test_polynomial_reproduction_2d(b, c, poly, plo, phi_):
    """dG consistency: u in P_p globally, constant a, b, c and f = -a Lap u +
    b . grad u + c u, g_D = u  =>  the discrete solution is u (quadrature is
    exact for these integrands)."""
    mesh = mg.voronoi_square(40, 21)
    om = O.Mesh(mesh)
    p = mg.draw_degrees(om.ne, 21, plo, phi_).astype(np.int32)
    a = np.full(om.ne, 0.37)
    pb = O.make_problem(2, b=b, c=c, source=2, poly=poly, c_sigma=10.0)
    assert _solve_and_error(om, p, a, pb) < 1e-9


def test_variable_coefficient_fields_through_the_source():
    """coef 1 is the paper's multi-GPU test problem (Sec. 4.2): b = (1+x, 1+y(, 1+z)),
    c = 3 + xy(z).  Checked through f = -a Lap u + b . grad u + c u for
    u = prod sin(pi x_d), with the derivatives of u written out here."""
    rng = np.random.default_rng(8)
    for dim in (2, 3):
        pb = O.make_problem(dim, source=1, coef=1)
        for _ in range(20):
            x = rng.uniform(0.0, 1.0, dim)
            a = float(rng.uniform(0.01, 2.0))
            s, c = np.sin(np.pi * x), np.cos(np.pi * x)
            u = np.prod(s)
            grad = np.array([np.pi * c[d] * np.prod(np.delete(s, d)) for d in range(dim)])
            lap = -dim * np.pi ** 2 * u
            b, cc = 1.0 + x, 3.0 + np.prod(x)
            f = -a * lap + b @ grad + cc * u
            assert abs(O.source_f(pb, a, x) - f) < 1e-12 * (1 + abs(f)), (dim, x, f)


@pytest.mark.parametrize(
    "poly,plo,phi_",
    [
        ([1, 1, -2, 0, 1, 0], 2, 2),
        ([0.5, -1, 2, 1, 0.5, -0.7], 2, 4),
        ([2, -1, 0.5], 1, 3),
        ([0, 1, 0, 0, 0, 0, 0.5, -1, 0.25, 1], 3, 4),
    ],
)
def test_polynomial_reproduction_2d_variable_coefficients(poly, plo, phi_):
    """dG consistency with the coefficient fields of coef 1: for u in P_p and
    f from the same fields, the discrete solution is u.  The rule stays exact:
    c u v has degree 2 + 2p <= 2p + 2, and the upwind jumps of a continuous u
    and the boundary inflow terms cancel point by point, where b . n changes
    sign along a face too."""
    mesh = mg.voronoi_square(40, 23)
    om = O.Mesh(mesh)
    p = mg.draw_degrees(om.ne, 23, plo, phi_).astype(np.int32)
    a = np.full(om.ne, 0.37)  # a jump in a would break the flux continuity u needs
    pb = O.make_problem(2, source=2, poly=poly, c_sigma=10.0, coef=1)
    assert _solve_and_error(om, p, a, pb) < 1e-9


def test_convergence_rate_variable_coefficients():
    """h^(p+1) L2 convergence for u = sin(pi x) sin(pi y) with the fields of
    coef 1 and a = 1."""
    import scipy.sparse as sps
    import scipy.sparse.linalg as spla

    for pdeg in (1, 2):
        errs = []
        for nsites in (64, 256, 1024):
            mesh = mg.voronoi_square(nsites, 300 + nsites)
            om = O.Mesh(mesh)
            p = np.full(om.ne, pdeg, dtype=np.int32)
            a = np.ones(om.ne)
            pb = O.make_problem(2, source=1, c_sigma=10.0, coef=1)
            blk = om.assemble(p, a, pb)
            A, F, off = O.global_matrix(om, p, blk)
            U = spla.spsolve(sps.csr_matrix(A), F)
            e2 = 0.0
            for e in range(om.ne):
                xq, wq = om.volume_points(e, pdeg + 3)
                for x, w in zip(xq, wq):
                    phi, _ = O.basis(2, pdeg, om.lo[e], om.hi[e], x)
                    e2 += w * (phi @ U[off[e]:off[e + 1]] - O.exact_u(pb, x)) ** 2
            errs.append(math.sqrt(e2))
        rate_n = math.log(errs[0] / errs[2]) / math.log(2.0 ** 2) * 2  # h ~ N^-1/2
        assert rate_n > pdeg + 1 - 0.25, (pdeg, errs)


def test_convergence_rate_sin_solution():
    """h^(p+1) L2 convergence for u = sin(pi x) sin(pi y) (config-0 family)."""
    import scipy.sparse as sps
    import scipy.sparse.linalg as spla

    for pdeg in (1, 2):
        errs, hs = [], []
        for nsites in (64, 256, 1024):
            mesh = mg.voronoi_square(nsites, 100 + nsites)
            om = O.Mesh(mesh)
            p = np.full(om.ne, pdeg, dtype=np.int32)
            a = np.ones(om.ne)
            pb = O.make_problem(2, source=1, c_sigma=10.0)
            blk = om.assemble(p, a, pb)
            A, F, off = O.global_matrix(om, p, blk)
            U = spla.spsolve(sps.csr_matrix(A), F)
            e2 = 0.0
            for e in range(om.ne):
                xq, wq = om.volume_points(e, pdeg + 3)
                for x, w in zip(xq, wq):
                    phi, _ = O.basis(2, pdeg, om.lo[e], om.hi[e], x)
                    e2 += w * (phi @ U[off[e]:off[e + 1]] - O.exact_u(pb, x)) ** 2
            errs.append(math.sqrt(e2))
            hs.append(om.h.max())
        rates = [math.log(errs[i] / errs[i + 1]) / math.log(hs[i] / hs[i + 1]) for i in range(2)]
        rate_n = math.log(errs[0] / errs[2]) / math.log(2.0 ** 2) * 2  # h ~ N^-1/2
        assert rate_n > pdeg + 1 - 0.25, (pdeg, errs, rates)


# ---------------------------------------------------------------------------
# 3D
# ---------------------------------------------------------------------------


def test_3d_box_mass_identity_and_volume():
    mesh = mg.box_tets(2, 1, 1, lo=(0.0, 0.0, 0.0), hi=(1.0, 0.5, 0.5))
    om = O.Mesh(mesh)
    assert om.ne == 2 and om.ni == 1
    assert abs(om.vol.sum() - 0.25) < 1e-15
    # each cube element = 6 Kuhn tets; 2 triangles on the shared square face
    assert om.if_nfaces[0] == 2
    assert om.nbf == 2 * (2 * 5)
    for p in (1, 2, 3):
        M = om.volume_block(0, np.array([p, p]), np.zeros(2), O.make_problem(3, c=1.0))
        np.testing.assert_allclose(M, np.eye(O.nbasis(3, p)), atol=3e-15)


def test_3d_agglomerated_volume_and_moments():
    mesh = mg.kuhn_cube_agglomerated(4, 10, seed=9)
    om = O.Mesh(mesh)
    assert abs(om.vol.sum() - 1.0) < 1e-14
    # sum over elements of the rule moments = moments of the unit cube
    for (i, j, k) in [(1, 0, 0), (2, 1, 0), (0, 3, 2), (2, 2, 2), (5, 0, 0)]:
        tot = sum(om.moment_rule(e, 5, i, j, k) for e in range(om.ne))  # exact to degree 7
        assert abs(tot - 1.0 / ((i + 1) * (j + 1) * (k + 1))) < 1e-14
    # surface: interior triangles counted once, boundary area = 6
    area_b = sum(om.face_info(f)[2] for f in range(om.nf) if om.face_info(f)[1] < 0)
    assert abs(area_b - 6.0) < 1e-13


@pytest.mark.parametrize("b,c", [((0.0, 0.0, 0.0), 0.0), ((1.0, -0.5, 0.25), 1.0)])
def test_polynomial_reproduction_3d(b, c):
    mesh = mg.kuhn_cube_agglomerated(3, 6, seed=2)
    om = O.Mesh(mesh)
    p = np.full(om.ne, 2, dtype=np.int32)
    a = np.full(om.ne, 0.5)
    poly = [1, 0.5, -1, 2, 0.3, 0, 0.7, -0.4, 0.2, 0.1]
    pb = O.make_problem(3, b=b, c=c, source=2, poly=poly, c_sigma=10.0)
    assert _solve_and_error(om, p, a, pb, npts=3) < 1e-9


# ---------------------------------------------------------------------------
# Neumann boundary (Eq. (2.2), Eq. (2.4), Eq. (2.5))
# ---------------------------------------------------------------------------


def _const_coeffs(om, p):
    """Coefficients of the constant function 1: sqrt(|bbox|) on phi_0."""
    out = []
    for e in range(om.ne):
        v = np.zeros(O.nbasis(om.dim, int(p[e])))
        v[0] = math.sqrt(np.prod(om.hi[e] - om.lo[e]))
        out.append(v)
    return np.concatenate(out)


def _elements_on_side(mesh, d, hi):
    """Elements with a boundary face on the side x_d = min / max, found from
    the mesh's own loops (2D) or tetrahedra (3D) by exact comparison."""
    X = [np.asarray(mesh.x), np.asarray(mesh.y)] + ([np.asarray(mesh.z)] if mesh.dim == 3 else [])
    side = X[d].max() if hi else X[d].min()
    on = set()
    if mesh.dim == 2:
        for e in range(len(mesh.elem_vptr) - 1):
            loop = mesh.elem_v[mesh.elem_vptr[e]:mesh.elem_vptr[e + 1]]
            for i in range(len(loop)):
                if X[d][loop[i]] == side and X[d][loop[(i + 1) % len(loop)]] == side:
                    on.add(e)
    else:
        for e in range(len(mesh.elem_tptr) - 1):
            for t in range(mesh.elem_tptr[e], mesh.elem_tptr[e + 1]):
                if sum(X[d][v] == side for v in mesh.tet_v[4 * t:4 * t + 4]) >= 3:
                    on.add(e)
    return on


@pytest.mark.parametrize("dim", [2, 3])
def test_neumann_faces_add_nothing_to_the_operator(dim):
    """Pure diffusion (b = 0, c = 0): grad 1 = 0 and [1] = 0 on interior faces,
    so with the whole boundary Neumann the constant lies in the kernel of B
    (Eq. (2.4) has no Neumann face terms).  With one side Dirichlet, B 1 is
    nonzero exactly on the elements with a face on that side (the penalty
    sees 1 there) and zero on all others."""
    if dim == 2:
        mesh = mg.voronoi_square(64, 5)
        om = O.Mesh(mesh)
        p = mg.draw_degrees(om.ne, 5, 1, 3).astype(np.int32)
    else:
        mesh = mg.kuhn_cube_agglomerated(3, 6, seed=2)
        om = O.Mesh(mesh)
        p = mg.draw_degrees(om.ne, 7, 1, 2).astype(np.int32)
    a = mg.draw_log_uniform(om.ne, 6, -1, 1)
    c1 = _const_coeffs(om, p)
    allsides = (1 << (2 * dim)) - 1
    A, _, off = _assemble_dense(om, p, a, O.make_problem(dim, neumann=allsides))
    s = np.abs(A).max()
    assert np.abs(A @ c1).max() < 1e-12 * s
    for d in range(dim):
        for hi in (0, 1):
            bit = 1 << (2 * d + hi)
            A, _, off = _assemble_dense(om, p, a, O.make_problem(dim, neumann=allsides & ~bit))
            r = A @ c1
            on = _elements_on_side(mesh, d, hi)
            assert on
            for e in range(om.ne):
                re = np.abs(r[off[e]:off[e + 1]]).max()
                if e in on:
                    assert re > 1e-8 * s, (d, hi, e)
                else:
                    assert re < 1e-12 * s, (d, hi, e)


@pytest.mark.parametrize("dim", [2, 3])
def test_neumann_data_balances_the_source(dim):
    """Pure diffusion with uniform a and the whole boundary Neumann: testing
    l with v = 1 gives int f + int g_N = int (-a Lap u) + int a grad u . n = 0
    (divergence theorem); the source part alone is not zero (int Lap u =
    0.7 in 2D and 2.2 in 3D for the polynomials below)."""
    if dim == 2:
        om = O.Mesh(mg.voronoi_square(64, 5))
        poly = [1, 1, 0.5, 1, -0.7, 0.4, 0.3, 0, 0, -1]  # Lap u = 2.8 + 1.8x - 6y
        p = mg.draw_degrees(om.ne, 5, 1, 3).astype(np.int32)
        lap_int = 0.7
    else:
        om = O.Mesh(mg.kuhn_cube_agglomerated(3, 6, seed=2))
        poly = [1, 0.5, -1, 2, 0.3, 0, 0.7, -0.4, 0.2, 0.1]  # Lap u = 2 (0.3 + 0.7 + 0.1)
        p = np.full(om.ne, 2, dtype=np.int32)
        lap_int = 2.2
    a = np.full(om.ne, 0.37)
    c1 = _const_coeffs(om, p)
    allsides = (1 << (2 * dim)) - 1
    pb = O.make_problem(dim, source=2, poly=poly, neumann=allsides)
    _, F, _ = _assemble_dense(om, p, a, pb)
    assert abs(F @ c1) < 1e-12
    # the volume part alone: int f = -a int Lap u
    pb0 = O.make_problem(dim, source=2, poly=poly, neumann=0)
    vol = 0.0
    for e in range(om.ne):
        xq, wq = om.volume_points(e, 4)
        vol += sum(w * O.source_f(pb0, 0.37, x) for x, w in zip(xq, wq))
    assert abs(vol + 0.37 * lap_int) < 1e-12


@pytest.mark.parametrize(
    "dim,b,c,neumann",
    [
        (2, (1.0, 0.5), 1.0, 0b1010),  # outflow sides x = 1, y = 1 Neumann
        (2, (0.0, 0.0), 0.0, 0b1110),  # only x = 0 Dirichlet
        (2, (0.6, -0.8), 0.5, 0b0110),  # x = 1 and y = 0 (outflow) Neumann
        (3, (1.0, -0.5, 0.25), 1.0, 0b100110),  # x = 1, y = 0, z = 1 Neumann
        (3, (0.0, 0.0, 0.0), 0.0, 0b111011),  # only y = 1 Dirichlet
    ],
)
def test_polynomial_reproduction_mixed_boundary(dim, b, c, neumann):
    """dG consistency with Dirichlet and Neumann sides (b . n >= 0 on the
    Neumann ones, as Eq. (2.2) assumes): u in P_p, g_D = u on the Dirichlet
    faces and g_N = a grad u . n on the Neumann faces => the discrete solution
    is u."""
    if dim == 2:
        om = O.Mesh(mg.voronoi_square(40, 21))
        p = mg.draw_degrees(om.ne, 21, 3, 4).astype(np.int32)
        poly = [1, 1, 0.5, 1, -0.7, 0.4, 0.3, 0, 0, -1]
    else:
        om = O.Mesh(mg.kuhn_cube_agglomerated(3, 6, seed=2))
        p = np.full(om.ne, 2, dtype=np.int32)
        poly = [1, 0.5, -1, 2, 0.3, 0, 0.7, -0.4, 0.2, 0.1]
    a = np.full(om.ne, 0.37)
    pb = O.make_problem(dim, b=b, c=c, source=2, poly=poly, c_sigma=10.0, neumann=neumann)
    assert _solve_and_error(om, p, a, pb, npts=3) < 1e-9


# ---------------------------------------------------------------------------
# coefficient fields given by a table (affine b, polynomial c)
# ---------------------------------------------------------------------------


def _sec42_table(dim):
    """The Sec. 4.2 fields written as a table: b = (1, 1, 1) + I x, c = 3 +
    the monomial prod_d x_d (graded index 4 in 2D, 15 in 3D)."""
    c = [0.0] * 20
    c[0] = 3.0
    c[4 if dim == 2 else 15] = 1.0
    return ((1.0, 1.0, 1.0), np.eye(3), c)


@pytest.mark.parametrize("dim", [2, 3])
def test_field_table_reproduces_the_sec42_fields(dim):
    if dim == 2:
        om = O.Mesh(mg.voronoi_square(30, 4))
        p = mg.draw_degrees(om.ne, 4, 1, 3).astype(np.int32)
    else:
        om = O.Mesh(mg.kuhn_cube_agglomerated(3, 6, seed=2))
        p = np.full(om.ne, 2, dtype=np.int32)
    a = mg.draw_log_uniform(om.ne, 4, -1, 1)
    b1 = om.assemble(p, a, O.make_problem(dim, source=1, coef=1))
    b2 = om.assemble(p, a, O.make_problem(dim, source=1, fields=_sec42_table(dim)))
    for key in ("diag", "a01", "a10", "rhs"):
        for x, y in zip(b1[key], b2[key]):
            assert np.array_equal(x, y), key


@pytest.mark.parametrize("dim,neumann", [(2, 0), (2, 0b10), (3, 0), (3, 0b10)])
def test_polynomial_reproduction_field_table(dim, neumann):
    """dG consistency with an affine b (all nine gradient entries free) and a
    polynomial c: u in P_p, f = -a Lap u + b . grad u + c u, g_D = u, g_N = a
    grad u . n on x = max (an outflow side of this b) => u_h = u.  The rules
    stay exact: b . grad w v and the upwind face terms have degree 2p and
    2p + 1; c w v has degree 2p + 2 with a quadratic c in 2D (triangle rule
    exact to 2p + 2) and 2p + 1 with a linear c in 3D (tetrahedron rule exact
    to 2p + 1)."""
    if dim == 2:
        om = O.Mesh(mg.voronoi_square(40, 21))
        p = mg.draw_degrees(om.ne, 21, 3, 4).astype(np.int32)
        poly = [1, 1, 0.5, 1, -0.7, 0.4, 0.3, 0, 0, -1]
        fields = ((0.7, -0.4, 0.0), [[0.3, -0.2, 0], [0.5, 0.1, 0], [0, 0, 0]], [1.0, 0.5, -0.3, 0.2, 0.1, 0.0])
        npts = 3
    else:
        om = O.Mesh(mg.kuhn_cube_agglomerated(3, 6, seed=2))
        p = np.full(om.ne, 2, dtype=np.int32)
        poly = [1, 0.5, -1, 2, 0.3, 0, 0.7, -0.4, 0.2, 0.1]
        fields = ((0.8, -0.3, 0.5), [[0.2, 0.1, -0.1], [0.0, 0.3, 0.2], [-0.2, 0.1, 0.1]], [1.5, 0.2, -0.1, 0.3])
        npts = 3
    a = np.full(om.ne, 0.37)
    pb = O.make_problem(dim, source=2, poly=poly, c_sigma=10.0, neumann=neumann, fields=fields)
    assert _solve_and_error(om, p, a, pb, npts=npts) < 1e-9


def test_field_table_through_the_source():
    """The table's b and c checked through f = -a Lap u + b . grad u + c u for
    u = prod sin(pi x_d), with b = b0 + B x (B not symmetric) and c written
    out here monomial by monomial (2D: 1, x, y, x^2, xy, y^2, ...; 3D:
    1, x, y, z, x^2, xy, y^2, xz, yz, z^2, ...)."""
    rng = np.random.default_rng(11)
    for dim in (2, 3):
        b0 = rng.uniform(-1, 1, 3)
        B = rng.uniform(-1, 1, (3, 3))
        cc = rng.uniform(-1, 1, 20)
        pb = O.make_problem(dim, source=1, fields=(b0, B, cc))
        for _ in range(10):
            x = rng.uniform(0.0, 1.0, dim)
            a = float(rng.uniform(0.1, 2.0))
            s, co = np.sin(np.pi * x), np.cos(np.pi * x)
            u = np.prod(s)
            grad = np.array([np.pi * co[d] * np.prod(np.delete(s, d)) for d in range(dim)])
            b = b0[:dim] + B[:dim, :dim] @ x
            if dim == 2:
                X, Y = x
                mons = [1, X, Y, X * X, X * Y, Y * Y, X ** 3, X * X * Y, X * Y * Y, Y ** 3]
            else:
                X, Y, Z = x
                mons = [1, X, Y, Z, X * X, X * Y, Y * Y, X * Z, Y * Z, Z * Z,
                        X ** 3, X * X * Y, X * Y * Y, Y ** 3, X * X * Z, X * Y * Z, Y * Y * Z, X * Z * Z, Y * Z * Z,
                        Z ** 3]
            c = float(np.dot(cc[:len(mons)], mons))
            f = a * dim * np.pi ** 2 * u + b @ grad + c * u
            assert abs(O.source_f(pb, a, x) - f) < 1e-12 * (1 + abs(f)), (dim, x)


# ---------------------------------------------------------------------------
# 3D moments by the divergence theorem (the exact-moment volume path)
# ---------------------------------------------------------------------------


@pytest.mark.parametrize("p", [1, 2, 3])
def test_tet_rule_moments_match_divergence_theorem_3d(p):
    """The sub-tetrahedron rule ((p+2)^3 collapsed points per tet) integrates
    every monomial of degree <= 2p+1 over an agglomerated polyhedron exactly:
    equal to the divergence theorem over the element's boundary triangles."""
    om = O.Mesh(mg.kuhn_cube_agglomerated(4, 10, seed=5))
    for e in range(0, om.ne, 3):
        for i in range(2 * p + 2):
            for j in range(2 * p + 2 - i):
                for k in range(2 * p + 2 - i - j):
                    ex = om.moment_divergence3d(e, i, j, k)
                    got = om.moment_rule(e, p + 2, i, j, k)
                    assert abs(got - ex) <= 1e-13 * abs(om.vol[e]), (e, i, j, k, got, ex)


def _boundary_triangles(mesh, e):
    """The element's boundary triangles (tet faces seen once inside the
    element), each oriented with its normal pointing out of the element."""
    T = mesh.tet_v.reshape(-1, 4)[mesh.elem_tptr[e]:mesh.elem_tptr[e + 1]]
    X = np.c_[mesh.x, mesh.y, mesh.z]
    seen = {}
    for t in T:
        for o in range(4):
            f = [t[i] for i in range(4) if i != o]
            seen.setdefault(tuple(sorted(f)), []).append((f, t[o]))
    out = []
    for lst in seen.values():
        if len(lst) != 1:
            continue
        f, opp = lst[0]
        A, B, C = X[f[0]], X[f[1]], X[f[2]]
        n = np.cross(B - A, C - A)
        if np.dot(n, X[opp] - A) > 0:
            B, C = C, B
        out.append((A, B, C))
    return out


@pytest.mark.parametrize("p", [2, 3])
def test_divergence_legendre_moments_3d_with_p_plus_2_triangle_points(p):
    """The identity behind the 3D exact-moment volume path.  With the
    element's box coordinates xi = 2 (x - lo) / L - 1, the integral of
    P_c(xi) P_d(eta) P_e(zeta) over the polyhedron equals the sum over its
    boundary triangles of the integral of (L_x / 2) Q_c(xi) P_d(eta) P_e(zeta)
    n_x dS, with Q_c the antiderivative of P_c (Q_0 = P_1, Q_c = (P_{c+1} -
    P_{c-1}) / (2c + 1)).  On a triangle that integrand has degree
    c + d + e + 1 <= 2p + 1, so the collapsed rule with p + 2 points per
    direction (exact to 2p + 2) is exact.  The reference is the sub-tet rule
    written out here with numpy."""
    from numpy.polynomial import legendre as npl

    def leg(k, x):
        return npl.legval(x, [0.0] * k + [1.0])

    def qleg(c, x):
        return x if c == 0 else (leg(c + 1, x) - leg(c - 1, x)) / (2 * c + 1)

    mesh = mg.kuhn_cube_agglomerated(4, 10, seed=5)
    tr, ts, tt, tw = O.tet_rule(p + 2)
    fr, fs, fw = O.tri_rule(p + 2)
    q = 2 * p
    X = np.c_[mesh.x, mesh.y, mesh.z]
    for e in range(0, mesh.ne, 2):
        T = mesh.tet_v.reshape(-1, 4)[mesh.elem_tptr[e]:mesh.elem_tptr[e + 1]]
        V = X[np.unique(T)]
        lo, L = V.min(axis=0), V.max(axis=0) - V.min(axis=0)
        # volume points of the sub-tet rule, in box coordinates
        VP, VW = [], []
        for t in T:
            P0, P1, P2, P3 = X[t]
            J = abs(np.dot(P1 - P0, np.cross(P2 - P0, P3 - P0)))
            VP.append(P0 + np.outer(tr, P1 - P0) + np.outer(ts, P2 - P0) + np.outer(tt, P3 - P0))
            VW.append(tw * J)
        VP = 2 * (np.concatenate(VP) - lo) / L - 1
        VW = np.concatenate(VW)
        # boundary points with the weight (L_x / 2) n_x dS
        BP, BW = [], []
        for A, B, C in _boundary_triangles(mesh, e):
            n = np.cross(B - A, C - A)
            area2 = np.linalg.norm(n)
            BP.append(A + np.outer(fr, B - A) + np.outer(fs, C - A))
            BW.append(fw * area2 * (n[0] / area2) * L[0] / 2)
        BP = 2 * (np.concatenate(BP) - lo) / L - 1
        BW = np.concatenate(BW)
        scale = np.sum(VW)
        for c in range(q + 1):
            for d in range(q + 1 - c):
                for f in range(q + 1 - c - d):
                    vol = np.sum(VW * leg(c, VP[:, 0]) * leg(d, VP[:, 1]) * leg(f, VP[:, 2]))
                    div = np.sum(BW * qleg(c, BP[:, 0]) * leg(d, BP[:, 1]) * leg(f, BP[:, 2]))
                    assert abs(div - vol) < 1e-12 * scale, (e, c, d, f, div, vol)
