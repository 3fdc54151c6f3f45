"""Pins of the space-time slab oracle (oracle/spacetime.py, Sec. 2.3).

- The two spaces have their dimensions: |P_p| = C(p + 3, 3) in (t, x, y),
  |PQ_p| = (p + 1) C(p + 2, 2).
- Without diffusion, wind or source the slab scheme is discontinuous Galerkin
  in time of degree q = p for y' = -c y, whose one-step factor is the (q, q+1)
  Pade approximant of exp(-c tau) (a textbook property of the method): pinned
  against the approximant written from its closed form, with the time jump
  (U^+, W^+) = (U^-, W^+) carrying the initial value.
- dG consistency in space-time: for u in the slab space, constant a, w, c, and
  f = u_t - a Lap u + w . grad u + c u, g = u, u_0 = u(0), the discrete solution
  is u on the first slab and, fed the first slab's trace, on the second.  PQ is
  checked with a u that has t x terms, which P of the same degree lacks.  The
  same over polyhedra (3D), one slab.
- PQ factorisation: every PQ slab block is [k = l] B + [r = s] D_kl M, B and M
  from the 2D and 3D oracles, D in closed form; this pins the interior jump
  terms, which an exact solution does not see.
- P is PQ restricted: the P slab system is the PQ one on the P index set.
- Planted mistakes in a copy of the slab oracle each fail one of these pins.
"""
import math

import numpy as np
import pytest

import oracle as O
from oracle import spacetime as S
from paper_2007_04881_gb300 import meshgen as mg


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_space_dimensions(p):
    assert len(S.st_index(p, "P")) == math.comb(p + 3, 3)
    assert len(S.st_index(p, "PQ")) == (p + 1) * math.comb(p + 2, 2)


def pade(q: int, z: float) -> float:
    """The (q, q+1) Pade approximant of exp(z): numerator and denominator
    coefficients (L + M - j)! L! / ((L + M)! j! (L - j)!) and the same with M,
    alternating in the denominator, for L = q, M = q + 1."""
    L, M = q, q + 1
    num = sum(math.factorial(L + M - j) * math.factorial(L) / (math.factorial(L + M) * math.factorial(j)
                                                              * math.factorial(L - j)) * z ** j for j in range(L + 1))
    den = sum(math.factorial(L + M - j) * math.factorial(M) / (math.factorial(L + M) * math.factorial(j)
                                                              * math.factorial(M - j)) * (-z) ** j for j in range(M + 1))
    return num / den


def test_pade_closed_form():
    assert abs(pade(0, -0.5) - 1 / 1.5) < 1e-15  # implicit Euler
    assert abs(pade(1, -0.5) - (1 - 0.5 / 3) / (1 + 2 * 0.5 / 3 + 0.25 / 6)) < 1e-15
    for q in range(4):  # order 2q + 1 at 0
        z = 1e-2
        assert abs(pade(q, z) - math.exp(z)) < 10 * z ** (2 * q + 2)


@pytest.mark.parametrize("space", ["P", "PQ"])
@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("ctau", [0.5, 3.0])
def test_time_dg_step_is_the_pade_approximant(space, p, ctau):
    check_pade(S, space, p, ctau)


def check_pade(S, space, p, ctau):
    om = O.Mesh(mg.rectangle_grid(1, 1, 0.2, 0.9, -0.1, 0.5))
    t0, t1 = 0.3, 0.8
    c = ctau / (t1 - t0)
    slab = S.Slab(om, [p], [0.0], (0.0, 0.0), c, space, t0, t1)
    A, F = slab.assemble(lambda t, x: 0.0, lambda t, x: 0.0, lambda e, x: 1.0)
    U = np.linalg.solve(A, F)
    want = pade(p, -ctau)
    for x in ([0.3, 0.0], [0.85, 0.45], [0.55, 0.2]):
        assert abs(slab.value(U, 0, t1, np.array(x)) - want) < 1e-12, (x, want)


def _manufactured(coef, a, w, c):
    """u(t, x, y) = sum coef[(i, j, k)] t^i x^j y^k and the source that goes
    with it."""
    def u(t, x):
        return sum(cf * t ** i * x[0] ** j * x[1] ** k for (i, j, k), cf in coef.items())

    def f(t, x):
        ut = lap = ux = uy = 0.0
        for (i, j, k), cf in coef.items():
            ut += cf * i * t ** max(i - 1, 0) * x[0] ** j * x[1] ** k if i else 0.0
            ux += cf * j * t ** i * x[0] ** max(j - 1, 0) * x[1] ** k if j else 0.0
            uy += cf * k * t ** i * x[0] ** j * x[1] ** max(k - 1, 0) if k else 0.0
            lap += cf * j * (j - 1) * t ** i * x[0] ** max(j - 2, 0) * x[1] ** k if j > 1 else 0.0
            lap += cf * k * (k - 1) * t ** i * x[0] ** j * x[1] ** max(k - 2, 0) if k > 1 else 0.0
        return ut - a * lap + w[0] * ux + w[1] * uy + c * u(t, x)

    return u, f


@pytest.mark.parametrize(
    "space,pset,coef",
    [
        ("P", (2, 2), {(0, 0, 0): 1.0, (1, 0, 0): 0.5, (0, 1, 0): -0.3, (0, 0, 1): 0.7, (1, 1, 0): 0.4,
                       (0, 0, 2): -0.2, (2, 0, 0): 0.1}),
        ("P", (2, 3), {(0, 0, 0): -0.4, (1, 0, 0): 1.2, (0, 1, 1): 0.8, (0, 2, 0): 0.5, (1, 0, 1): -0.6}),
        ("PQ", (1, 1), {(0, 0, 0): 1.0, (0, 1, 0): -0.3, (0, 0, 1): 0.7, (1, 0, 0): 0.5, (1, 1, 0): -0.15,
                        (1, 0, 1): 0.35}),
        ("PQ", (2, 2), {(0, 0, 0): 0.3, (2, 0, 2): 0.9, (1, 1, 1): -0.5, (2, 1, 0): 0.4, (0, 2, 0): 0.2}),
    ],
)
def test_space_time_polynomial_reproduction_over_two_slabs(space, pset, coef):
    check_reproduction(S, space, pset, coef)


def check_reproduction(S, space, pset, coef, n=10):
    mesh = mg.voronoi_square(n, 5)
    om = O.Mesh(mesh)
    p = mg.draw_degrees(om.ne, 5, pset[0], pset[1]).astype(np.int32)
    a, w, c = 0.3, (0.8, -0.4), 0.6
    u, f = _manufactured(coef, a, w, c)
    prev = lambda e, x: u(0.0, x)  # noqa: E731
    for t0, t1 in ((0.0, 0.25), (0.25, 0.45)):
        slab = S.Slab(om, p, np.full(om.ne, a), w, c, space, t0, t1)
        A, F = slab.assemble(f, u, prev)
        U = np.linalg.solve(A, F)
        err = 0.0
        for e in range(om.ne):
            xq, _ = om.volume_points(e, 3)
            for x in xq[::5]:
                for t in (t0, 0.5 * (t0 + t1), t1):
                    err = max(err, abs(slab.value(U, e, t, x) - u(t, x)))
        assert err < 1e-9, (space, t0, err)
        prev = (lambda sl, UU: (lambda e, x: sl.value(UU, e, sl.t1, x)))(slab, U)


def test_slab_factorises_into_time_and_space():
    check_factorisation(S)


def check_factorisation(S, n=12):
    """PQ: every slab block is
        A[(k, j), (l, m)] = delta_kl B_S[j, m] + D[k, l] M_S[j, m],
    B_S the 2D oracle's spatial block (its own pins hold it: volume, SIPG and
    upwind face terms, mixed degrees), M_S the element's spatial mass matrix
    (the bounding-box basis is orthonormal on the box, not on the element) and
    D the time part in closed form for the orthonormal T_k,
    int T_l' T_k dt + T_l(t0) T_k(t0) = sqrt((2k+1)(2l+1)) / tau *
    (2 [k < l, k + l odd] + (-1)^(k + l)).  This pins the spatial terms that a
    continuous exact solution cannot see (the interior jumps)."""
    om = O.Mesh(mg.voronoi_square(n, 8))
    p = mg.draw_degrees(om.ne, 8, 1, 3).astype(np.int32)
    a = mg.draw_log_uniform(om.ne, 8, -1.0, 0.5)
    w, c, t0, t1 = (0.9, -0.6), 0.7, 0.1, 0.35
    tau = t1 - t0
    slab = S.Slab(om, p, a, w, c, "PQ", t0, t1)
    zero = lambda *args: 0.0  # noqa: E731
    A, _ = slab.assemble(zero, zero, zero)
    ob = om.assemble(p, a, O.make_problem(2, b=w, c=c, source=0, c_sigma=10.0), rhs=False)

    def D(k, l):
        jump = 2.0 if (k < l and (k + l) % 2 == 1) else 0.0
        return math.sqrt((2 * k + 1) * (2 * l + 1)) / tau * (jump + (-1.0) ** (k + l))

    mass = O.make_problem(2, b=(0.0, 0.0), c=1.0, source=0, c_sigma=0.0)

    def check(r, s, B2, with_time):
        got = A[slab.off[r]:slab.off[r + 1], slab.off[s]:slab.off[s + 1]]
        M = om.volume_block(r, p, np.zeros(om.ne), mass) if with_time else None
        want = np.zeros_like(got)
        for i, (k, j) in enumerate(slab.idx[r]):
            for q, (l, m) in enumerate(slab.idx[s]):
                want[i, q] = (B2[j, m] if k == l else 0.0) + (D(k, l) * M[j, m] if with_time else 0.0)
        assert np.abs(got - want).max() <= 1e-11 * np.abs(want).max(), (r, s)

    for pos, e in enumerate(ob["elems"]):
        check(int(e), int(e), ob["diag"][pos], True)
    for pos, i in enumerate(ob["ifaces"]):
        e0, e1 = int(om.if_e0[i]), int(om.if_e1[i])
        check(e0, e1, ob["a01"][pos], False)
        check(e1, e0, ob["a10"][pos], False)


def test_p_slab_is_the_pq_slab_restricted():
    """P_p is a subspace of PQ_p with the same form, rules and penalty, and the
    spatial basis is ordered by total degree: the P slab matrix and load vector
    are the PQ ones restricted to the (k, j) with j < nbasis(2, p - k)."""
    om = O.Mesh(mg.voronoi_square(8, 6))
    p = mg.draw_degrees(om.ne, 6, 1, 3).astype(np.int32)
    a = mg.draw_log_uniform(om.ne, 6, -1.0, 0.5)
    args = (om, p, a, (0.4, 0.8), 0.9)
    pq = S.Slab(*args, "PQ", 0.2, 0.5)
    pp = S.Slab(*args, "P", 0.2, 0.5)
    f = lambda t, x: np.cos(t + x[0]) * x[1]  # noqa: E731
    g = lambda t, x: t * x[0] - x[1] ** 2  # noqa: E731
    u0 = lambda e, x: 1.0 + x[0] * x[1]  # noqa: E731
    Aq, Fq = pq.assemble(f, g, u0)
    Ap, Fp = pp.assemble(f, g, u0)
    keep = np.concatenate([pq.off[e] + np.array([pq.idx[e].index(kj) for kj in pp.idx[e]]) for e in range(om.ne)])
    assert np.abs(Aq[np.ix_(keep, keep)] - Ap).max() <= 1e-12 * np.abs(Ap).max()
    assert np.abs(Fq[keep] - Fp).max() <= 1e-12 * np.abs(Fp).max()


def _mesh3d():
    from paper_2007_04881_gb300 import configs

    wl = configs.small3d(2, 4, 5, 1, 2)  # 4 polyhedra of 12 tetrahedra, p in 1..2
    return O.Mesh(wl.mesh), wl.p.astype(np.int32), wl.a


def test_slab_3d_factorises_into_time_and_space():
    """The factorisation pin over polyhedra: every PQ slab block is
    [k = l] B + [r = s] D_kl M with B, M from the 3D oracle."""
    om, p, a = _mesh3d()
    w, c, t0, t1 = (0.6, -0.3, 0.45), 0.5, 0.0, 0.3
    sl = S.Slab(om, p, a, w, c, "PQ", t0, t1)
    zero = lambda *args: 0.0  # noqa: E731
    A, _ = sl.assemble(zero, zero, zero)
    ob = om.assemble(p, a, O.make_problem(3, b=w, c=c, source=0, c_sigma=10.0), rhs=False)
    mass = O.make_problem(3, c=1.0, c_sigma=0.0)
    tau = t1 - t0

    def D(k, l):
        deriv = 2.0 if (k < l and (k + l) % 2 == 1) else 0.0
        return math.sqrt((2 * k + 1) * (2 * l + 1)) / tau * (deriv + (-1.0) ** (k + l))

    def check(r, s, B2, M):
        got = A[sl.off[r]:sl.off[r + 1], sl.off[s]:sl.off[s + 1]]
        want = np.zeros_like(got)
        for i, (k, j) in enumerate(sl.idx[r]):
            for q, (l, m) in enumerate(sl.idx[s]):
                want[i, q] = (B2[j, m] if k == l else 0.0) + (D(k, l) * M[j, m] if M is not None else 0.0)
        assert np.abs(got - want).max() <= 1e-11 * np.abs(want).max(), (r, s)

    for pos, e in enumerate(ob["elems"]):
        e = int(e)
        check(e, e, ob["diag"][pos], om.volume_block(e, p, np.zeros(om.ne), mass))
    for pos, i in enumerate(ob["ifaces"]):
        e0, e1 = int(om.if_e0[i]), int(om.if_e1[i])
        check(e0, e1, ob["a01"][pos], None)
        check(e1, e0, ob["a10"][pos], None)


@pytest.mark.parametrize("space", ["P", "PQ"])
def test_slab_3d_reproduces_space_time_polynomials(space):
    """u = 1 + 0.5 t + x - 0.7 y + 0.4 z (+ 0.3 t x in PQ, outside P_1) with
    f = u_t + w . grad u + c u and g = u: the slab solution is u."""
    om, p, _ = _mesh3d()
    a = np.full(om.ne, 0.8)  # constant: with a jump in a, the flux of u would jump too
    w, c, t0, t1 = np.array([0.6, -0.3, 0.45]), 0.5, 0.1, 0.35
    tx = 0.3 if space == "PQ" else 0.0

    def u(t, x):
        return 1.0 + 0.5 * t + x[0] - 0.7 * x[1] + 0.4 * x[2] + tx * t * x[0]

    def f(t, x):
        grad = np.array([1.0 + tx * t, -0.7, 0.4])
        return 0.5 + tx * x[0] + w @ grad + c * u(t, x)

    sl = S.Slab(om, p, a, w, c, space, t0, t1)
    A, F = sl.assemble(f, u, lambda e, x: u(t0, x))
    U = np.linalg.solve(A, F)
    err = 0.0
    for e in range(om.ne):
        xq, _ = om.volume_points(e, 2)
        for x in xq[::11]:
            for t in (t0, t1):
                err = max(err, abs(sl.value(U, e, t, x) - u(t, x)))
    assert err < 1e-9, err


# Planted mistakes: each one, made in a copy of the slab oracle, fails a pin.
MUTATIONS = {
    "time_jump_dropped": ("Ae += wx * np.outer(psi0, psi0)", "pass"),
    "time_derivative_transposed": ("np.outer(psi, dpsi)", "np.outer(dpsi, psi)"),
    "time_basis_not_orthonormal": ("np.sqrt((2 * k + 1) / tau)", "np.sqrt((2 * k + 1) / 2.0)"),
    "upwind_outflow_side_sign": ("(bn if q == 1 else -bn)", "(bn if q == 1 else bn)"),
    "symmetry_term_dropped": ("- avg * ar * sgn[q] * np.outer(dn[r], ps[q])", "- 0.0 * np.outer(dn[r], ps[q])"),
    "nitsche_rhs_penalty_sign": ("- sig * ps[0])", "+ sig * ps[0])"),
    "previous_slab_at_t1": ("psi0, _, _ = self._psi(e, self.t0, x)", "psi0, _, _ = self._psi(e, self.t1, x)"),
    "time_rule_one_point_short": ("tg, tw = gauss01(pe + 2)", "tg, tw = gauss01(pe)"),
}


def _load_mutant(name):
    import types

    src = open(S.__file__).read()
    old, new = MUTATIONS[name]
    assert src.count(old) == 1, f"mutation anchor missing: {name}"
    src = src.replace(old, new).replace("from . import ", "from oracle import ")
    mod = types.ModuleType(f"spacetime_mut_{name}")
    exec(compile(src, f"spacetime_mut_{name}", "exec"), mod.__dict__)
    return mod


def _pins_pass(M) -> bool:
    try:
        check_pade(M, "PQ", 2, 3.0)
        check_reproduction(M, "PQ", (1, 2), {(0, 0, 0): 0.3, (1, 1, 0): -0.5, (1, 0, 1): 0.4, (0, 1, 0): 0.2},
                           n=6)
        check_factorisation(M, n=6)
        return True
    except (AssertionError, np.linalg.LinAlgError):
        return False


def test_unmutated_slab_copy_passes():
    assert _pins_pass(S)


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_slab_mutation_is_caught(name):
    assert not _pins_pass(_load_mutant(name)), f"planted mistake '{name}' passed every pin"
