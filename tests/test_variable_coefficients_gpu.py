"""Variable advection and reaction on the GPU (dg_assemble_varcoef; the
fields of Sec. 4.2, b_d(x) = 1 + x_d, c(x) = 3 + prod_d x_d, at every
quadrature point, inflow decided point by point) against the oracle with
the same fields (oracle coef 1).

- Mixed-degree 2D meshes, every degree 1..6, and polyhedra, every degree
  1..4, the sin source and the zero source: every block and every
  load-vector segment, FP64, block max-norm relative 1e-12 (the FP64 parity
  bound of the constant-coefficient path).
- The full-size 65,536-cell mesh: a seeded sample of 300 elements and
  interfaces against oracle blocks computed one by one.
- Fields from a table (dg_mesh_set_fields: an affine b with a full
  gradient, a cubic c) against the oracle's coef 2, FP64 at 1e-12 and the
  FP32 form at the FP32 tolerances of the other parity tests (5e-5 per
  block, 1e-4 per load-vector segment).
- Polynomial reproduction through the GPU system with table fields and
  mixed Dirichlet/Neumann sides.
- The argument checks: a mesh uploaded with b or c, a precision other than
  FP64/FP32 and a partition mesh are refused.
"""
import numpy as np
import pytest

import oracle as O
from paper_2007_04881_gb300 import configs, dg

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


@pytest.fixture(scope="module")
def ctx(cuda):
    import torch

    from paper_2007_04881_gb300 import build as B

    B.build()
    c = dg.Context(0, torch.cuda.current_stream().cuda_stream)
    yield c
    c.close()


def _run(ctx, mesh, p, a, source):
    import torch

    m = dg.Mesh(ctx, mesh, p, a, dg.Problem(b=(0.0, 0.0, 0.0), c=0.0, source=source))
    vals = torch.full((m.nvals,), float("nan"), dtype=torch.float64, device="cuda")
    rhs = torch.full((m.ndofs,), float("nan"), dtype=torch.float64, device="cuda")
    m.dg_assemble_varcoef(vals, rhs)
    ctx.dg_sync()
    v, r = vals.cpu().numpy(), rhs.cpu().numpy()
    assert np.isfinite(v).all() and np.isfinite(r).all()
    return m, dg.to_blocks(m, v, r)


def _compare(om, p, a, source, got, elems=None, ifaces=None):
    ob = om.assemble(np.asarray(p, np.int32), a, O.make_problem(om.dim, source=source, coef=1, c_sigma=10.0),
                     elems=elems, ifaces=ifaces)
    e_d = e_o = e_r = 0.0
    for pos, e in enumerate(ob["elems"]):
        e = int(e)
        ref = ob["diag"][pos]
        e_d = max(e_d, np.abs(got["diag"][e] - ref).max() / np.abs(ref).max())
        rr = ob["rhs"][pos]
        e_r = max(e_r, np.abs(got["rhs"][e] - rr).max() / max(np.abs(rr).max(), 1e-300))
    for pos, i in enumerate(ob["ifaces"]):
        e0, e1 = int(om.if_e0[i]), int(om.if_e1[i])
        for key, ref in (((e0, e1), ob["a01"][pos]), ((e1, e0), ob["a10"][pos])):
            e_o = max(e_o, np.abs(got["off"][key] - ref).max() / np.abs(ref).max())
    return e_d, e_o, e_r


@pytest.mark.parametrize("source", [configs.SRC_SINPROD, configs.SRC_ZERO])
def test_small2d_every_degree(ctx, source):
    wl = configs.small2d(180, 7, 1, 6)
    _, got = _run(ctx, wl.mesh, wl.p, wl.a, source)
    e_d, e_o, e_r = _compare(O.Mesh(wl.mesh), wl.p, wl.a, source, got)
    assert e_d < TOL64 and e_o < TOL64, (e_d, e_o)
    if source == configs.SRC_SINPROD:
        assert e_r < TOL64, e_r
    else:
        assert e_r == 0.0, e_r


@pytest.mark.parametrize("source", [configs.SRC_SINPROD, configs.SRC_ZERO])
def test_small3d_every_degree(ctx, source):
    wl = configs.small3d(4, 10, 5, 1, 4)
    _, got = _run(ctx, wl.mesh, wl.p, wl.a, source)
    e_d, e_o, e_r = _compare(O.Mesh(wl.mesh), wl.p, wl.a, source, got)
    assert e_d < TOL64 and e_o < TOL64, (e_d, e_o)
    if source == configs.SRC_SINPROD:
        assert e_r < TOL64, e_r
    else:
        assert e_r == 0.0, e_r


def test_adr2d_65k_sampled(ctx):
    wl = configs.adr2d()
    _, got = _run(ctx, wl.mesh, wl.p, wl.a, configs.SRC_SINPROD)
    om = O.Mesh(wl.mesh)
    rng = np.random.default_rng(29)
    elems = np.sort(rng.choice(wl.ne, 300, replace=False)).astype(np.int32)
    ifs = np.sort(rng.choice(om.ni, 300, replace=False)).astype(np.int32)
    e_d, e_o, e_r = _compare(om, wl.p, wl.a, configs.SRC_SINPROD, got, elems, ifs)
    assert e_d < TOL64 and e_o < TOL64 and e_r < TOL64, (e_d, e_o, e_r)


def test_argument_checks(ctx):
    import torch

    wl = configs.small2d(60, 3, 1, 3)
    v = torch.zeros(1 << 16, dtype=torch.float64, device="cuda")
    for pb in (dg.Problem(b=(1.0, 0.0, 0.0), source=1), dg.Problem(c=0.5, source=1)):
        m = dg.Mesh(ctx, wl.mesh, wl.p, wl.a, pb)
        with pytest.raises(dg.DGError) as ei:
            m.dg_assemble_varcoef(v)
        assert ei.value.code == -1
    m = dg.Mesh(ctx, wl.mesh, wl.p, wl.a, dg.Problem(source=1))
    with pytest.raises(dg.DGError):
        m.dg_assemble_varcoef(v, prec=dg.DG_PREC_BF16X3)
    with pytest.raises(dg.DGError):
        m.dg_mesh_set_fields(b0=(float("nan"), 0, 0))
    part = dg.dg_partition(wl.mesh, wl.p, wl.a, dg.Problem(source=1), 2)
    mp = dg.Mesh(ctx, wl.mesh, wl.p, wl.a, dg.Problem(source=1), part=part, my_part=0)
    with pytest.raises(dg.DGError):
        mp.dg_assemble_varcoef(v)


TOL32 = 5e-5
TOL32_RHS = 1e-4
# an affine b with every gradient entry set and a cubic c (2D: the first 10
# monomials; 3D: all 20)
FIELDS = {
    2: ((0.7, -0.4, 0.0), [[0.3, -0.2, 0.0], [0.5, 0.1, 0.0], [0.0, 0.0, 0.0]],
        [1.0, 0.5, -0.3, 0.2, 0.1, 0.3, 0.2, -0.1, 0.15, 0.05]),
    3: ((0.8, -0.3, 0.5), [[0.2, 0.1, -0.1], [0.0, 0.3, 0.2], [-0.2, 0.1, 0.1]],
        [1.5, 0.2, -0.1, 0.3, 0.1, 0.05, 0.2, -0.1, 0.1, 0.05, 0.1, 0.0, 0.05, 0.1, -0.05, 0.2, 0.0, 0.1, 0.05, 0.1]),
}


def _run_fields(ctx, wl, prec, fields, source, neumann=0, poly=()):
    import torch

    m = dg.Mesh(ctx, wl.mesh, wl.p, wl.a, dg.Problem(source=source, poly=list(poly), neumann=neumann))
    if fields is not None:
        m.dg_mesh_set_fields(*fields)
    dt = torch.float64 if prec == dg.DG_PREC_FP64 else torch.float32
    vals = torch.full((m.nvals,), float("nan"), dtype=dt, device="cuda")
    rhs = torch.full((m.ndofs,), float("nan"), dtype=dt, device="cuda")
    m.dg_assemble_varcoef(vals, rhs, prec=prec)
    ctx.dg_sync()
    v, r = vals.double().cpu().numpy(), rhs.double().cpu().numpy()
    assert np.isfinite(v).all() and np.isfinite(r).all()
    return m, v, r


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("prec", [dg.DG_PREC_FP64, dg.DG_PREC_FP32])
@pytest.mark.parametrize("table", [False, True])
def test_fields_and_forms_vs_oracle(ctx, dim, prec, table):
    from .helpers import compare

    wl = configs.small2d(180, 7, 1, 6) if dim == 2 else configs.small3d(4, 10, 5, 1, 4)
    fields = FIELDS[dim] if table else None
    m, v, r = _run_fields(ctx, wl, prec, fields, configs.SRC_SINPROD)
    om = O.Mesh(wl.mesh)
    pb = O.make_problem(dim, source=1, c_sigma=10.0, coef=1, fields=fields)
    ob = om.assemble(np.asarray(wl.p, np.int32), wl.a, pb)
    ed, eo, er = compare(dg.to_blocks(m, v, r), om, ob, wl)
    if prec == dg.DG_PREC_FP64:
        assert ed < TOL64 and eo < TOL64 and er < TOL64, (ed, eo, er)
    else:
        assert ed < TOL32 and eo < TOL32 and er < TOL32_RHS, (ed, eo, er)


@pytest.mark.parametrize("neumann", [0, 0b10])
def test_fields_polynomial_reproduction_through_gpu(ctx, neumann):
    """u in P_p with table fields (quadratic c, so the 2D rules stay exact)
    and, optionally, the outflow side x = 1 Neumann: the GPU system's
    solution is u (dG consistency of Eq. (2.4), (2.5) with variable b, c)."""
    poly = [1, 1, 0.5, 1, -0.7, 0.4, 0.3, 0, 0, -1]
    fields = ((0.7, -0.4, 0.0), [[0.3, -0.2, 0], [0.5, 0.1, 0], [0, 0, 0]], [1.0, 0.5, -0.3, 0.2, 0.1, 0.0])
    wl = configs.small2d(40, 21, 3, 4)
    wl.a[:] = 0.37
    m, v, r = _run_fields(ctx, wl, dg.DG_PREC_FP64, fields, configs.SRC_POLY, neumann=neumann, poly=poly)
    row_ptr, col, blk_off, dof_off = m.dg_bsr_pattern()
    N = int(dof_off[-1])
    A = np.zeros((N, N))
    for rr in range(m.ne):
        for k in range(row_ptr[rr], row_ptr[rr + 1]):
            cc = col[k]
            A[dof_off[rr]:dof_off[rr + 1], dof_off[cc]:dof_off[cc + 1]] = v[blk_off[k]:blk_off[k + 1]].reshape(
                dof_off[rr + 1] - dof_off[rr], dof_off[cc + 1] - dof_off[cc])
    U = np.linalg.solve(A, r)
    om = O.Mesh(wl.mesh)
    pb = O.make_problem(2, source=2, poly=poly)
    err = 0.0
    for e in range(om.ne):
        xq, _ = om.volume_points(e, 3)
        for x in xq[::4]:
            phi, _ = O.basis(2, int(wl.p[e]), om.lo[e], om.hi[e], x)
            err = max(err, abs(phi @ U[dof_off[e]:dof_off[e + 1]] - O.exact_u(pb, x)))
    assert err < 1e-9, err
