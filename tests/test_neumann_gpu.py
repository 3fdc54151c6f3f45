"""Neumann boundary (Eq. (2.2)) on the GPU: faces on marked sides of the
vertex box add no matrix term (Eq. (2.4)) and g_N v = (a grad u . n) v to the
load vector (Eq. (2.5)).  Every form and launch shape against the FP64
oracle, at the tolerances of the other parity tests (FP64 1e-12 block
max-norm relative; FP32 5e-5, load vectors 1e-4; the tensor forms as in
their own tests); the device-built pattern, the partition and the batch
bitwise equal to the whole-mesh host-pattern pass; the constant in the kernel
of pure diffusion with a fully Neumann boundary at full size; and polynomial
reproduction through the GPU system with mixed sides."""
import numpy as np
import pytest

import oracle as O
from paper_2007_04881_gb300 import configs, dg

from .helpers import compare, dg_problem, oracle_blocks

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 5e-5
TOL32_RHS = 1e-4
TOL_TC = {dg.DG_PREC_TF32X3: 5e-5, dg.DG_PREC_BF16X3: 2e-4}

# b = (0.8, -0.45): outflow through x = max and y = min (bits 1 and 2)
MASK2 = 0b0110
# b = (0.6, -0.3, 0.45): outflow through x = max, y = min, z = max
MASK3 = 0b100110


@pytest.fixture(scope="module")
def ctx(cuda):
    import torch

    from paper_2007_04881_gb300 import build as B

    B.build()
    c = dg.Context(0, torch.cuda.current_stream().cuda_stream)
    yield c
    c.close()


def _system(ctx, m, prec, how="fused"):
    import torch

    dt = torch.float64 if prec == dg.DG_PREC_FP64 else torch.float32
    v = torch.full((m.nvals,), float("nan"), dtype=dt, device="cuda")
    r = torch.full((m.ndofs,), float("nan"), dtype=dt, device="cuda")
    if how == "split":
        m.dg_assemble_volume(prec, v)
        m.dg_assemble_faces(prec, v)
        m.dg_assemble_rhs(prec, r)
    elif how == "step":
        m.dg_assemble_step(prec, v, r)
    else:
        m.dg_assemble(prec, v, r)
    ctx.dg_sync()
    v, r = v.double().cpu().numpy(), r.double().cpu().numpy()
    assert np.isfinite(v).all() and np.isfinite(r).all()
    return v, r


def _wl2d(**kw):
    return configs.small2d(300, 17, 1, 6, neumann=MASK2, **kw)


def _wl3d(**kw):
    return configs.small3d(4, 10, 5, 1, 4, neumann=MASK3, **kw)


def _n_neumann_faces(om, wl):
    """Boundary faces on the marked sides (counted from the oracle's faces)."""
    X = [np.asarray(wl.mesh.x), np.asarray(wl.mesh.y)] + ([np.asarray(wl.mesh.z)] if wl.dim == 3 else [])
    n = 0
    for f in range(om.nf):
        e0, e1, area, nrm = om.face_info(f)
        if e1 >= 0:
            continue
        for d in range(wl.dim):
            for s in (0, 1):
                if wl.problem["neumann"] >> (2 * d + s) & 1 and abs(nrm[d]) == 1.0 and np.sign(nrm[d]) == (1 if s else -1):
                    n += 1
    return n


@pytest.mark.parametrize("prec,how", [(dg.DG_PREC_FP64, "fused"), (dg.DG_PREC_FP64, "split"),
                                      (dg.DG_PREC_FP32, "fused"), (dg.DG_PREC_FP32, "step")])
def test_neumann_2d_vs_oracle(ctx, prec, how):
    wl = _wl2d()
    om, ob = oracle_blocks(wl)
    assert _n_neumann_faces(om, wl) > 10
    m = dg.Mesh(ctx, wl.mesh, wl.p, wl.a, dg_problem(wl))
    v, r = _system(ctx, m, prec, how)
    ed, eo, er = compare(dg.to_blocks(m, v, r), om, ob, wl)
    if prec == dg.DG_PREC_FP64:
        assert ed < TOL64 and eo < TOL64 and er < TOL64, (ed, eo, er)
    else:
        assert ed < TOL32 and eo < TOL32 and er < TOL32_RHS, (ed, eo, er)


@pytest.mark.parametrize("prec", [dg.DG_PREC_FP64, dg.DG_PREC_FP32])
@pytest.mark.parametrize("src", [configs.SRC_SINPROD, configs.SRC_POLY])
def test_neumann_3d_vs_oracle(ctx, prec, src):
    wl = _wl3d(source=src, poly=[1, 0.5, -1, 2, 0.3, 0, 0.7, -0.4, 0.2, 0.1, 0.05, -0.2])
    om, ob = oracle_blocks(wl)
    m = dg.Mesh(ctx, wl.mesh, wl.p, wl.a, dg_problem(wl))
    v, r = _system(ctx, m, prec)
    ed, eo, er = compare(dg.to_blocks(m, v, r), om, ob, wl)
    if prec == dg.DG_PREC_FP64:
        assert ed < TOL64 and eo < TOL64 and er < TOL64, (ed, eo, er)
    else:
        assert ed < TOL32 and eo < TOL32 and er < TOL32_RHS, (ed, eo, er)


@pytest.mark.parametrize("prec", [dg.DG_PREC_TF32X3, dg.DG_PREC_BF16X3])
def test_neumann_tensor_forms(ctx, prec):
    wl = _wl2d()
    om, ob = oracle_blocks(wl)
    m = dg.Mesh(ctx, wl.mesh, wl.p, wl.a, dg_problem(wl))
    v, r = _system(ctx, m, prec)
    ed, eo, er = compare(dg.to_blocks(m, v, r), om, ob, wl)
    assert ed < TOL_TC[prec] and eo < TOL_TC[prec] and er < TOL32_RHS, (ed, eo, er)


@pytest.mark.parametrize("path", [0, 1, 2])
@pytest.mark.parametrize("persistent", [False, True])
def test_neumann_volume_paths_and_persistent(ctx, path, persistent):
    wl = configs.small2d(500, 19, 1, 5, b=(1.0, 0.5), c=1.0, neumann=0b1010)
    om, ob = oracle_blocks(wl)
    m = dg.Mesh(ctx, wl.mesh, wl.p, wl.a, dg_problem(wl))
    ctx.dg_set_volume_path(path)
    ctx.dg_set_persistent(persistent)
    try:
        v, r = _system(ctx, m, dg.DG_PREC_FP32, "step")
    finally:
        ctx.dg_set_volume_path(1)
        ctx.dg_set_persistent(False)
    ed, eo, er = compare(dg.to_blocks(m, v, r), om, ob, wl)
    assert ed < TOL32 and eo < TOL32 and er < TOL32_RHS, (ed, eo, er)


@pytest.mark.parametrize("which", ["2d", "3d"])
def test_neumann_device_pattern_partition_batch_bitwise(ctx, which):
    """The classification reads only vertex coordinates and the box: the
    device-built pattern, each part of a partition (whose vertex box is
    smaller than the whole mesh's) and a batch of members spanning the same
    box give bitwise the whole mesh's rows."""
    wl = _wl2d() if which == "2d" else _wl3d()
    pb = dg_problem(wl)
    prec = dg.DG_PREC_FP32
    full = dg.Mesh(ctx, wl.mesh, wl.p, wl.a, pb)
    fv, fr = _system(ctx, full, prec, "step")
    ctx.dg_set_pattern_device(True)
    try:
        md = dg.Mesh(ctx, wl.mesh, wl.p, wl.a, pb)
    finally:
        ctx.dg_set_pattern_device(False)
    dv, dr = _system(ctx, md, prec, "step")
    assert np.array_equal(dv, fv) and np.array_equal(dr, fr)
    md.close()
    f_rp, f_col, f_bo, f_do = full.dg_bsr_pattern()
    nparts = 3
    part = dg.dg_partition(wl.mesh, wl.p, wl.a, pb, nparts)
    for k in range(nparts):
        pm = dg.Mesh(ctx, wl.mesh, wl.p, wl.a, pb, part=part, my_part=k)
        pv, pr = _system(ctx, pm, prec, "step")
        rp, col, bo, do = pm.dg_bsr_pattern()
        eg = pm.elem_global
        for e in np.flatnonzero(pm.owned):
            g = int(eg[e])
            fcols = f_col[f_rp[g]:f_rp[g + 1]]
            for bk in range(rp[e], rp[e + 1]):
                fb = f_rp[g] + int(np.searchsorted(fcols, int(eg[col[bk]])))
                assert np.array_equal(pv[bo[bk]:bo[bk + 1]], fv[f_bo[fb]:f_bo[fb + 1]]), (k, g)
            assert np.array_equal(pr[do[e]:do[e + 1]], fr[f_do[g]:f_do[g + 1]]), (k, g)
        pm.close()
    # a batch of the mesh with itself: each member's rows are the mesh's own
    bm = dg.Mesh(ctx, None, problem=pb, members=[(wl.mesh, wl.p, wl.a)] * 2)
    bv, br = _system(ctx, bm, prec, "step")
    n, nd = fv.size, fr.size
    assert bv.size == 2 * n and np.array_equal(bv[:n], fv) and np.array_equal(bv[n:], fv)
    assert np.array_equal(br[:nd], fr) and np.array_equal(br[nd:], fr)
    bm.close()
    full.close()


def test_neumann_batch_members_must_share_the_box(ctx):
    a = configs.small2d(60, 3, 1, 2, neumann=MASK2)
    b = configs.small2d(60, 4, 1, 2, neumann=MASK2)
    b.mesh.x = np.asarray(b.mesh.x) * 0.5  # spans [0, 0.5] x [0, 1]
    with pytest.raises(dg.DGError, match="another box"):
        dg.Mesh(ctx, None, problem=dg_problem(a), members=[(a.mesh, a.p, a.a), (b.mesh, b.p, b.a)])
    with pytest.raises(dg.DGError, match="neumann mask"):
        dg.Mesh(ctx, a.mesh, a.p, a.a, dg.Problem(neumann=1 << 4))


@pytest.mark.parametrize("mask,b,c", [(0b1010, (1.0, 0.5), 1.0), (0b1110, (0.0, 0.0), 0.0)])
def test_neumann_polynomial_reproduction_through_gpu(ctx, mask, b, c):
    """Solve the GPU-assembled FP64 system densely with Dirichlet and Neumann
    sides: u_h reproduces a global cubic (consistency of Eq. (2.4), (2.5))."""
    poly = [1, 1, 0.5, 1, -0.7, 0.4, 0.3, 0, 0, -1]
    wl = configs.small2d(40, 21, 3, 4, b=b, c=c, source=configs.SRC_POLY, poly=poly, neumann=mask)
    wl.a[:] = 0.37
    m = dg.Mesh(ctx, wl.mesh, wl.p, wl.a, dg_problem(wl))
    v, r = _system(ctx, m, dg.DG_PREC_FP64)
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
    pb = O.make_problem(2, b=b, c=c, source=2, poly=poly)
    err = 0.0
    for e in range(om.ne):
        xq, _ = om.volume_points(e, 3)
        for x in xq[::4]:
            phi, _ = O.basis(2, int(wl.p[e]), om.lo[e], om.hi[e], x)
            err = max(err, abs(phi @ U[dof_off[e]:dof_off[e + 1]] - O.exact_u(pb, x)))
    assert err < 1e-9, err


def test_neumann_full_size_sampled_and_constant_kernel(ctx):
    """65,536 cells: sampled blocks of the cells along the Neumann sides
    against the oracle (FP64 and FP32); and with b = 0, c = 0 and the whole
    boundary Neumann, the FP64 matrix maps the constant to zero in every row
    (no face term survives on the boundary)."""
    wl = configs.adr2d()
    wl.problem["neumann"] = 0b1010
    om = O.Mesh(wl.mesh)
    near = np.flatnonzero((om.hi[:, 0] == 1.0) | (om.hi[:, 1] == 1.0))
    rng = np.random.default_rng(5)
    elems = np.sort(rng.choice(near, 48, replace=False)).astype(np.int32)
    ifaces = np.flatnonzero(np.isin(om.if_e0, elems))[:96].astype(np.int32)
    ob = om.assemble(wl.p.astype(np.int32), wl.a, O.make_problem(
        2, b=wl.problem["b"], c=wl.problem["c"], source=wl.problem["source"], neumann=0b1010), elems=elems,
        ifaces=ifaces)
    m = dg.Mesh(ctx, wl.mesh, wl.p, wl.a, dg_problem(wl))
    for prec, tol, tr in ((dg.DG_PREC_FP64, TOL64, TOL64), (dg.DG_PREC_FP32, TOL32, TOL32_RHS)):
        v, r = _system(ctx, m, prec, "step")
        ed, eo, er = compare(dg.to_blocks(m, v, r), om, ob, wl)
        assert ed < tol and eo < tol and er < tr, (prec, ed, eo, er)
    m.close()
    pb = dg.Problem(source=configs.SRC_SINPROD, neumann=0b1111)
    m = dg.Mesh(ctx, wl.mesh, wl.p, wl.a, pb)
    v, _ = _system(ctx, m, dg.DG_PREC_FP64)
    row_ptr, col, blk_off, dof_off = m.dg_bsr_pattern()
    nb = np.diff(dof_off)
    c1 = np.sqrt(np.prod(om.hi - om.lo, axis=1))
    out = np.zeros(int(dof_off[-1]))
    scale = np.zeros(m.ne)
    rows = np.repeat(np.arange(m.ne), np.diff(row_ptr))
    for rr_n in np.unique(nb):
        for cc_n in np.unique(nb):
            sel = np.flatnonzero((nb[rows] == rr_n) & (nb[col] == cc_n))
            if sel.size == 0:
                continue
            # column 0 of each block: entries blk_off + i * n_c
            idx = blk_off[sel][:, None] + np.arange(rr_n)[None, :] * cc_n
            contrib = v[idx] * c1[col[sel]][:, None]
            np.add.at(out, dof_off[rows[sel]][:, None] + np.arange(rr_n)[None, :], contrib)
            blk = v[blk_off[sel][:, None] + np.arange(rr_n * cc_n)[None, :]]
            np.maximum.at(scale, rows[sel], np.abs(blk).max(axis=1))
    res = np.array([np.abs(out[dof_off[e]:dof_off[e + 1]]).max() for e in range(m.ne)])
    assert (res <= 1e-12 * scale).all(), float((res / scale).max())
    m.close()


@pytest.mark.parametrize("which", ["2d", "3d"])
def test_neumann_variable_coefficients(ctx, which):
    """dg_assemble_varcoef (the fields b_d = 1 + x_d, c = 3 + prod x_d of
    Sec. 4.2) with the outflow sides x_d = max Neumann: no inflow term there,
    g_N v in the load; against the oracle's coef 1 with the same sides."""
    import torch

    if which == "2d":
        wl = configs.small2d(150, 7, 1, 6)
        mask = 0b1010
    else:
        wl = configs.small3d(4, 10, 5, 1, 4)
        mask = 0b101010
    m = dg.Mesh(ctx, wl.mesh, wl.p, wl.a, dg.Problem(source=configs.SRC_SINPROD, neumann=mask))
    vals = torch.full((m.nvals,), float("nan"), dtype=torch.float64, device="cuda")
    rhs = torch.full((m.ndofs,), float("nan"), dtype=torch.float64, device="cuda")
    m.dg_assemble_varcoef(vals, rhs)
    ctx.dg_sync()
    got = dg.to_blocks(m, vals.cpu().numpy(), rhs.cpu().numpy())
    om = O.Mesh(wl.mesh)
    ob = om.assemble(wl.p.astype(np.int32), wl.a,
                     O.make_problem(wl.dim, source=1, coef=1, c_sigma=10.0, neumann=mask))
    ed, eo, er = compare(got, om, ob, wl)
    assert ed < TOL64 and eo < TOL64 and er < TOL64, (ed, eo, er)
