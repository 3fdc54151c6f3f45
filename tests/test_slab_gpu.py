"""Space-time slab systems on the GPU (dg_assemble_slab, dg_slab_trace;
Sec. 2.3) against the oracle.

- Small 2D meshes, both spaces, mixed degrees: every slab block, the load
  vector with the previous slab's trace and the trace itself against the
  slab oracle (oracle/spacetime.py), which assembles the space-time form
  with its own space-time quadrature.  FP64: block max-norm relative error
  2e-12, the FP64 spatial bound 1e-12 of each of the two parts B and D M of
  a diagonal block.  With variable a the source is zero (the oracle's source
  takes no element), so the load vector is the time jump alone.
- Full size (65,536 cells, the launch configuration of the spatial pass)
  and 3D: a seeded sample of blocks and load-vector segments against the
  factorisation A = I (x) B + D (x) M built from the 2D / 3D oracle's blocks,
  B its spatial blocks, M its mass matrix and D the closed-form time matrix;
  the CPU tests pin that identity against the slab oracle (1e-11).
- The steady spatial solution is a fixed point of a slab step: with
  B u = l and u_prev = u, the slab solution is sqrt(tau) T_0 (x) u and its
  trace is u again.
- FP32 against FP64 (relative Frobenius 2e-6, the FP32 form's 1e-6 for the
  two parts) and the argument checks.
"""
import math

import numpy as np
import pytest

import oracle as O
from oracle import spacetime as S
from paper_2007_04881_gb300 import configs, dg, meshgen as mg

from .helpers import dg_problem, oracle_problem

pytestmark = pytest.mark.gpu

TOL64 = 2e-12
SPACES = {dg.DG_SPACE_P: "P", dg.DG_SPACE_PQ: "PQ"}


@pytest.fixture(scope="module")
def ctx(cuda):
    import torch

    from paper_2007_04881_gb300 import build as B

    B.build()
    c = dg.Context(0, torch.cuda.current_stream().cuda_stream)
    yield c
    c.close()


def _assemble(ctx, m, prec, space, t0, t1, u_prev=None, rhs=True):
    import torch

    dt = torch.float64 if prec == dg.DG_PREC_FP64 else torch.float32
    nv, nd = m.dg_slab_layout(space)
    vals = torch.full((nv,), float("nan"), dtype=dt, device="cuda")
    r = torch.full((nd,), float("nan"), dtype=dt, device="cuda") if rhs else None
    up = None if u_prev is None else torch.as_tensor(u_prev, dtype=dt, device="cuda")
    m.dg_assemble_slab(prec, space, t0, t1, vals, r, up)
    ctx.dg_sync()
    assert bool(torch.isfinite(vals).all()), "a slab value was not written"
    assert r is None or bool(torch.isfinite(r).all()), "a load-vector entry was not written"
    return vals, r


def _time_matrix(tau):
    def D(k, l):
        deriv = 2.0 if (k < l and (k + l) % 2 == 1) else 0.0
        return math.sqrt((2 * k + 1) * (2 * l + 1)) / tau * (deriv + (-1.0) ** (k + l))
    return D


def _blk(row_ptr, col, r, s):
    return int(row_ptr[r] + np.nonzero(col[row_ptr[r]:row_ptr[r + 1]] == s)[0][0])


def _rel(got, want):
    return float(np.abs(got - want).max() / max(np.abs(want).max(), 1e-300))


# ---------------------------------------------------------------------------
# small 2D: the slab oracle


def _small_case(seed, const_a):
    mesh = mg.voronoi_square(10, seed)
    om = O.Mesh(mesh)
    p = mg.draw_degrees(om.ne, seed, 1, 3).astype(np.int32)
    a = np.full(om.ne, 0.7) if const_a else mg.draw_log_uniform(om.ne, seed, -1.0, 0.5)
    w, c = (0.9, -0.6), 0.7
    src = configs.SRC_SINPROD if const_a else configs.SRC_ZERO
    return mesh, om, p, a, w, c, src


@pytest.mark.parametrize("space", sorted(SPACES))
@pytest.mark.parametrize("const_a", [False, True])
def test_small2d_against_slab_oracle(ctx, space, const_a):
    mesh, om, p, a, w, c, src = _small_case(5, const_a)
    m = dg.Mesh(ctx, mesh, p, a, dg.Problem(b=(w[0], w[1], 0.0), c=c, source=src))
    row_ptr, col, _, dof_off = m.dg_bsr_pattern()
    sblk, sdof = m.dg_slab_pattern(space)
    t0, t1 = 0.15, 0.4
    rng = np.random.default_rng(11)
    u_prev = rng.standard_normal(m.ndofs)
    vals, rhs = _assemble(ctx, m, dg.DG_PREC_FP64, space, t0, t1, u_prev)
    v, r = vals.cpu().numpy(), rhs.cpu().numpy()

    pb = O.make_problem(2, b=w, c=c, source=src, c_sigma=10.0)
    sl = S.Slab(om, p, a, w, c, SPACES[space], t0, t1)
    a0 = float(a[0])

    def prev(e, x):
        phi, _ = O.basis(2, int(p[e]), om.lo[e], om.hi[e], x)
        return float(phi @ u_prev[dof_off[e]:dof_off[e + 1]])

    A, F = sl.assemble(lambda t, x: O.source_f(pb, a0, x), lambda t, x: O.exact_u(pb, x), prev)
    assert np.array_equal(sdof, sl.off)
    err = 0.0
    for rr in range(om.ne):
        for b in range(row_ptr[rr], row_ptr[rr + 1]):
            s = int(col[b])
            got = v[sblk[b]:sblk[b + 1]].reshape(sdof[rr + 1] - sdof[rr], sdof[s + 1] - sdof[s])
            err = max(err, _rel(got, A[sl.off[rr]:sl.off[rr + 1], sl.off[s]:sl.off[s + 1]]))
    assert err < TOL64, err
    e_r = max(_rel(r[sdof[e]:sdof[e + 1]], F[sl.off[e]:sl.off[e + 1]]) for e in range(om.ne))
    assert e_r < TOL64, e_r

    # the trace of the slab solution at t1 against the oracle's value there
    import torch

    U = np.linalg.solve(A, F)
    u_end = torch.full((m.ndofs,), float("nan"), dtype=torch.float64, device="cuda")
    m.dg_slab_trace(dg.DG_PREC_FP64, space, t0, t1, torch.as_tensor(U, device="cuda"), u_end)
    ctx.dg_sync()
    ue = u_end.cpu().numpy()
    e_t = 0.0
    for e in range(om.ne):
        xq, _ = om.volume_points(e, 2)
        for x in xq[::4]:
            phi, _ = O.basis(2, int(p[e]), om.lo[e], om.hi[e], x)
            want = sl.value(U, e, t1, x)
            e_t = max(e_t, abs(phi @ ue[dof_off[e]:dof_off[e + 1]] - want) / (1.0 + abs(want)))
    assert e_t < 1e-11, e_t


# ---------------------------------------------------------------------------
# the factorisation from the spatial oracle, sampled


def _identity_check(ctx, wl, space, prec, nsample, seed, tol_blk, tol_rhs):
    """Sampled slab blocks and load-vector segments against I (x) B + D (x) M
    from the spatial oracle's blocks."""
    m = dg.Mesh(ctx, wl.mesh, wl.p, wl.a, dg_problem(wl))
    dim = m.dim
    row_ptr, col, _, dof_off = m.dg_bsr_pattern()
    sblk, sdof = m.dg_slab_pattern(space)
    t0, t1 = 0.0, 0.3
    rng = np.random.default_rng(seed)
    u_prev = rng.standard_normal(m.ndofs)
    vals, rhs = _assemble(ctx, m, prec, space, t0, t1, u_prev)
    om = O.Mesh(wl.mesh)
    p = wl.p.astype(np.int32)
    elems = np.sort(rng.choice(m.ne, min(nsample, m.ne), replace=False)).astype(np.int32)
    ifs = np.sort(rng.choice(om.ni, min(nsample, om.ni), replace=False)).astype(np.int32)
    ob = om.assemble(p, wl.a, oracle_problem(wl), elems=elems, ifaces=ifs)
    mass = O.make_problem(dim, c=1.0, c_sigma=0.0)
    D = _time_matrix(t1 - t0)
    idx = {e: S.st_index(int(p[e]), SPACES[space]) if dim == 2 else _st_index(dim, int(p[e]), space)
           for e in set(elems.tolist()) | set(om.if_e0[ifs].tolist()) | set(om.if_e1[ifs].tolist())}

    def got_block(r, s):
        b = _blk(row_ptr, col, r, s)
        g = vals[int(sblk[b]):int(sblk[b + 1])].double().cpu().numpy()
        return g.reshape(len(idx[r]), len(idx[s]))

    def want_block(r, s, B2, M2):
        want = np.zeros((len(idx[r]), len(idx[s])))
        for i, (k, j) in enumerate(idx[r]):
            for q, (l, mm) in enumerate(idx[s]):
                want[i, q] = (B2[j, mm] if k == l else 0.0) + (D(k, l) * M2[j, mm] if M2 is not None else 0.0)
        return want

    e_d = e_o = e_r = 0.0
    for pos, e in enumerate(elems):
        e = int(e)
        M2 = om.volume_block(e, p, np.zeros(om.ne), mass)
        e_d = max(e_d, _rel(got_block(e, e), want_block(e, e, ob["diag"][pos], M2)))
        # load vector: [k = 0] sqrt(tau) l_j + T_k(t0+) (M u_prev)_j
        Mu = M2 @ u_prev[dof_off[e]:dof_off[e + 1]]
        tau = t1 - t0
        want = np.array([(math.sqrt(tau) * ob["rhs"][pos][j] if k == 0 else 0.0)
                         + math.sqrt((2 * k + 1) / tau) * (-1.0) ** k * Mu[j] for k, j in idx[e]])
        got = rhs[int(sdof[e]):int(sdof[e + 1])].double().cpu().numpy()
        e_r = max(e_r, _rel(got, want))
    for pos, i in enumerate(ifs):
        e0, e1 = int(om.if_e0[i]), int(om.if_e1[i])
        e_o = max(e_o, _rel(got_block(e0, e1), want_block(e0, e1, ob["a01"][pos], None)))
        e_o = max(e_o, _rel(got_block(e1, e0), want_block(e1, e0, ob["a10"][pos], None)))
    assert e_d < tol_blk and e_o < tol_blk and e_r < tol_rhs, (e_d, e_o, e_r)
    return m, vals, rhs


def _st_index(dim, p, space):
    """(k, j) pairs of a prism over a dim-dimensional element (the layout of
    include/dg.h), for the 3D check; 2D uses the slab oracle's."""
    out = []
    for k in range(p + 1):
        d = p - k if space == dg.DG_SPACE_P else p
        out.extend((k, j) for j in range(O.nbasis(dim, d)))
    return out


@pytest.mark.parametrize("space", sorted(SPACES))
def test_adr2d_65k_sampled(ctx, space):
    """Full-size 2D ADR mesh (p = 1..4, a log-uniform over four decades),
    FP64: 300 sampled elements and interfaces."""
    _identity_check(ctx, configs.adr2d(), space, dg.DG_PREC_FP64, 300, 17, TOL64, TOL64)


@pytest.mark.parametrize("space", sorted(SPACES))
def test_small3d(ctx, space):
    wl = configs.small3d(4, 10, 5, 1, 4)
    _identity_check(ctx, wl, space, dg.DG_PREC_FP64, 60, 19, TOL64, TOL64)


# ---------------------------------------------------------------------------


@pytest.mark.parametrize("space", sorted(SPACES))
def test_steady_state_is_a_fixed_point(ctx, space):
    import torch

    wl = configs.small2d(120, 9, 1, 3)
    m = dg.Mesh(ctx, wl.mesh, wl.p, wl.a, dg_problem(wl))
    v = torch.empty(m.nvals, dtype=torch.float64, device="cuda")
    l = torch.empty(m.ndofs, dtype=torch.float64, device="cuda")
    m.dg_assemble(dg.DG_PREC_FP64, v, l)
    ctx.dg_sync()
    u = np.linalg.solve(_dense(m.dg_bsr_pattern(), v.cpu().numpy(), m.ndofs), l.cpu().numpy())
    t0, t1 = 0.2, 0.45
    vals, rhs = _assemble(ctx, m, dg.DG_PREC_FP64, space, t0, t1, u)
    sblk, sdof = m.dg_slab_pattern(space)
    row_ptr, col, _, dof_off = m.dg_bsr_pattern()
    A = _dense((row_ptr, col, sblk, sdof), vals.cpu().numpy(), int(sdof[-1]))
    U = np.linalg.solve(A, rhs.cpu().numpy())
    want = np.zeros_like(U)
    for e in range(m.ne):
        nb = int(dof_off[e + 1] - dof_off[e])
        want[sdof[e]:sdof[e] + nb] = math.sqrt(t1 - t0) * u[dof_off[e]:dof_off[e + 1]]
    assert np.abs(U - want).max() < 1e-9 * np.abs(want).max()
    u_end = torch.empty(m.ndofs, dtype=torch.float64, device="cuda")
    m.dg_slab_trace(dg.DG_PREC_FP64, space, t0, t1, torch.as_tensor(U, device="cuda"), u_end)
    ctx.dg_sync()
    assert np.abs(u_end.cpu().numpy() - u).max() < 1e-9 * np.abs(u).max()


def _dense(pattern, vals, n):
    row_ptr, col, blk_off, dof_off = pattern
    A = np.zeros((n, n))
    for r in range(len(row_ptr) - 1):
        for b in range(row_ptr[r], row_ptr[r + 1]):
            s = int(col[b])
            A[dof_off[r]:dof_off[r + 1], dof_off[s]:dof_off[s + 1]] = vals[blk_off[b]:blk_off[b + 1]].reshape(
                dof_off[r + 1] - dof_off[r], dof_off[s + 1] - dof_off[s])
    return A


@pytest.mark.parametrize("space", sorted(SPACES))
def test_fp32_against_fp64(ctx, space):
    """The FP32 slab form against the FP64 one with the spatial FP32 form's
    bounds: 5e-5 per block and 1e-6 relative Frobenius for each of the two
    parts (2e-6 for their sum), 1e-4 per element for the load vector."""
    wl = configs.small2d(400, 13, 1, 4)
    m = dg.Mesh(ctx, wl.mesh, wl.p, wl.a, dg_problem(wl))
    u_prev = np.random.default_rng(5).standard_normal(m.ndofs)
    v64, r64 = _assemble(ctx, m, dg.DG_PREC_FP64, space, 0.0, 0.2, u_prev)
    v32, r32 = _assemble(ctx, m, dg.DG_PREC_FP32, space, 0.0, 0.2, u_prev)
    rel = float((v32.double() - v64).norm() / v64.norm())
    assert rel < 2e-6, rel
    sblk, sdof = m.dg_slab_pattern(space)
    a64, a32 = v64.cpu().numpy(), v32.double().cpu().numpy()
    e_b = max(_rel(a32[sblk[b]:sblk[b + 1]], a64[sblk[b]:sblk[b + 1]]) for b in range(len(sblk) - 1))
    assert e_b < 5e-5, e_b
    b64, b32 = r64.cpu().numpy(), r32.double().cpu().numpy()
    e_r = max(_rel(b32[sdof[e]:sdof[e + 1]], b64[sdof[e]:sdof[e + 1]]) for e in range(m.ne))
    assert e_r < 1e-4, e_r


def test_layout_and_argument_checks(ctx):
    import torch

    wl = configs.small2d(60, 3, 1, 4)
    m = dg.Mesh(ctx, wl.mesh, wl.p, wl.a, dg_problem(wl))
    for space in SPACES:
        nv, nd = m.dg_slab_layout(space)
        sblk, sdof = m.dg_slab_pattern(space)
        assert nv == sblk[-1] and nd == sdof[-1]
    nv, nd = m.dg_slab_layout(dg.DG_SPACE_PQ)
    vals = torch.zeros(nv, dtype=torch.float64, device="cuda")
    bad = [
        dict(space=2), dict(t0=0.5, t1=0.5), dict(t0=0.5, t1=0.1), dict(t1=float("inf")),
        dict(prec=dg.DG_PREC_BF16X3), dict(prec=dg.DG_PREC_TF32X3),
    ]
    for kw in bad:
        args = dict(prec=dg.DG_PREC_FP64, space=dg.DG_SPACE_PQ, t0=0.0, t1=0.1)
        args.update(kw)
        with pytest.raises(dg.DGError) as ei:
            m.dg_assemble_slab(args["prec"], args["space"], args["t0"], args["t1"], vals)
        assert ei.value.code == -1, kw
    with pytest.raises(dg.DGError):
        m.dg_slab_layout(5)
    # a partition mesh holds ghost rows that no pass writes
    part = dg.dg_partition(wl.mesh, wl.p, wl.a, dg_problem(wl), 2)
    mp = dg.Mesh(ctx, wl.mesh, wl.p, wl.a, dg_problem(wl), part=part, my_part=0)
    with pytest.raises(dg.DGError) as ei:
        mp.dg_slab_layout(dg.DG_SPACE_P)
    assert ei.value.code == -1


@pytest.mark.parametrize("space", sorted(SPACES))
def test_slab_graph_equals_direct(ctx, space):
    """The slab step recorded as one CUDA graph (dg_slab_graph_create) writes
    the same matrix and load vector as the direct call, bit for bit, on every
    replay; mixed degrees 1..6, FP32."""
    import torch

    w = configs.small2d(400, 95, 1, 6, b=(1.0, 0.5), c=1.0)
    m = dg.Mesh(ctx, w.mesh, w.p, w.a, dg_problem(w))
    t0, t1 = 0.0, 0.05
    g = torch.Generator().manual_seed(5)
    u_prev = torch.randn(m.ndofs, generator=g, dtype=torch.float32).cuda()
    v_ref, r_ref = _assemble(ctx, m, dg.DG_PREC_FP32, space, t0, t1, u_prev)
    nv, nd = m.dg_slab_layout(space)
    vals = torch.zeros(nv, dtype=torch.float32, device="cuda")
    rhs = torch.zeros(nd, dtype=torch.float32, device="cuda")
    gr = m.dg_slab_graph_create(dg.DG_PREC_FP32, space, t0, t1, vals, rhs, u_prev)
    for _ in range(3):
        vals.zero_()
        rhs.zero_()
        gr.dg_graph_launch()
        ctx.dg_sync()
        assert torch.equal(vals, v_ref) and torch.equal(rhs, r_ref)
    gr.close()
