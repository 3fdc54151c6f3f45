"""The ways of forming the volume blocks, against the FP64 oracle: the
per-point contraction in the row kernels (path 0), the Legendre-product
moments over the quadrature points (path 1, the default) and the same moments
exact from the element's boundary (path 2: in 2D by Green's theorem along the
edges, in 3D by the divergence theorem on the boundary triangles), in FP64
and FP32, with every degree, with learned rules, and through the separate
volume / faces / load-vector calls.  The moment path adds the same quadrature
terms in another order, and for the polynomial volume integrands of constant
coefficients the sub-simplex rule is exact, so path 2 equals it up to
rounding: the tolerances are those of the other parity tests."""
import numpy as np
import pytest

from paper_2007_04881_gb300 import configs, dg

from .helpers import compare, dg_problem, oracle_blocks, polygon_workload

pytestmark = pytest.mark.gpu

TOL = {dg.DG_PREC_FP64: 1e-12, dg.DG_PREC_FP32: 5e-5}
TOL_RHS = {dg.DG_PREC_FP64: 1e-12, dg.DG_PREC_FP32: 1e-4}


@pytest.fixture(scope="module")
def ctx(cuda):
    import torch

    from paper_2007_04881_gb300 import build as B

    B.build()
    c = dg.Context(0, torch.cuda.current_stream().cuda_stream)
    yield c
    c.dg_set_volume_path(1)
    c.close()


def run(ctx, wl, prec, path, how="fused", m=None):
    import torch

    ctx.dg_set_volume_path(path)
    m = m or dg.Mesh(ctx, wl.mesh, wl.p, wl.a, dg_problem(wl))
    dt = torch.float64 if prec == dg.DG_PREC_FP64 else torch.float32
    v = torch.full((m.nvals,), float("nan"), dtype=dt, device="cuda")
    r = torch.full((m.ndofs,), float("nan"), dtype=dt, device="cuda")
    if how == "split":
        m.dg_assemble_volume(prec, v)
        m.dg_assemble_faces(prec, v)
        m.dg_assemble_rhs(prec, r)
    else:
        m.dg_assemble(prec, v, r)
    ctx.dg_sync()
    ctx.dg_set_volume_path(1)
    return m, v.double().cpu().numpy(), r.double().cpu().numpy()


@pytest.mark.parametrize("path", [0, 1, 2])
@pytest.mark.parametrize("prec", [dg.DG_PREC_FP64, dg.DG_PREC_FP32])
@pytest.mark.parametrize("which", ["2d", "3d"])
def test_paths_against_oracle(ctx, path, prec, which):
    wl = configs.small2d(180, 7, 1, 6) if which == "2d" else configs.small3d(4, 10, 5, 1, 4)
    m, v, r = run(ctx, wl, prec, path)
    assert np.isfinite(v).all() and np.isfinite(r).all()
    om, ob = oracle_blocks(wl)
    ed, eo, er = compare(dg.to_blocks(m, v, r), om, ob, wl)
    assert ed < TOL[prec] and eo < TOL[prec] and er < TOL_RHS[prec], (ed, eo, er)


@pytest.mark.parametrize("path", [1, 2])
@pytest.mark.parametrize("prec", [dg.DG_PREC_FP64, dg.DG_PREC_FP32])
def test_moment_path_split_calls(ctx, prec, path):
    """volume (moments) then faces (row kernel adds to the diagonal), and the
    load vector alone, equal the fused pass within the parity tolerance"""
    wl = configs.small2d(220, 17, 2, 5, b=(1.0, 0.5), c=1.0)
    m, v1, r1 = run(ctx, wl, prec, path)
    _, v2, r2 = run(ctx, wl, prec, path, how="split", m=m)
    assert np.abs(v1 - v2).max() <= TOL[prec] * np.abs(v1).max()
    assert np.abs(r1 - r2).max() <= TOL[prec] * np.abs(r1).max()
    _, v3, r3 = run(ctx, wl, prec, path, m=m)
    assert np.array_equal(v1, v3) and np.array_equal(r1, r3)  # deterministic


def test_exact_moments_match_quadrature_moments(ctx):
    """FP64: the exact moments and the quadrature moments give the same
    matrix up to rounding, with every 2D degree, advection and reaction; the
    load vector is the same sum"""
    wl = configs.small2d(600, 23, 1, 6, b=(1.0, -0.7), c=2.0)
    m, v1, r1 = run(ctx, wl, dg.DG_PREC_FP64, 1)
    _, v2, r2 = run(ctx, wl, dg.DG_PREC_FP64, 2, m=m)
    assert np.abs(v2 - v1).max() <= 1e-12 * np.abs(v1).max()
    assert np.abs(r2 - r1).max() <= 1e-12 * np.abs(r1).max()


def test_moment_path_with_learned_rules(ctx):
    wl = configs.small2d(300, 45, 3, 3, b=(1.0, 0.5), c=1.0)
    m = dg.Mesh(ctx, wl.mesh, wl.p, wl.a, dg_problem(wl))
    m.dg_quad_prepare()
    st = m.dg_quad_fit(None, iters=8, install=True)
    assert st["accepted"] > 0.8 * m.ne
    _, v0, r0 = run(ctx, wl, dg.DG_PREC_FP64, 0, m=m)
    for path in (1, 2):
        _, v1, r1 = run(ctx, wl, dg.DG_PREC_FP64, path, m=m)
        assert np.abs(v1 - v0).max() <= 1e-12 * np.abs(v0).max(), path
        assert np.abs(r1 - r0).max() <= 1e-12 * np.abs(r0).max(), path


@pytest.mark.parametrize("path", [-1, 3])
def test_bad_path_rejected(ctx, path):
    with pytest.raises(dg.DGError):
        ctx.dg_set_volume_path(path)


@pytest.mark.parametrize("p", [3, 6])
@pytest.mark.parametrize("prec", [dg.DG_PREC_FP64, dg.DG_PREC_FP32])
def test_exact_moments_long_loop(ctx, p, prec):
    """a single 20-gon: more edges than the lanes of an element, so a lane
    takes two; against the oracle's sub-triangle rule"""
    wl = polygon_workload(20, p)
    om, ob = oracle_blocks(wl)
    for path in (1, 2):
        m, v, r = run(ctx, wl, prec, path)
        ed, eo, er = compare(dg.to_blocks(m, v, r), om, ob, wl)
        assert ed < TOL[prec] and er < TOL_RHS[prec], (path, ed, er)


@pytest.mark.parametrize("prec", [dg.DG_PREC_FP64, dg.DG_PREC_FP32])
def test_exact_moments_3d_match_quadrature_moments(ctx, prec):
    """3D, degrees 2 and 3 (the moment path's 3D degrees), advection and
    reaction, polyhedra of about 40 tetrahedra: the divergence-theorem moments
    and the sub-tet quadrature moments give the same system up to rounding,
    and both match the oracle"""
    wl = configs.small3d(6, 24, 31, 2, 3, b=(0.7, -0.4, 0.3), c=1.5)
    m, v1, r1 = run(ctx, wl, prec, 1)
    _, v2, r2 = run(ctx, wl, prec, 2, m=m)
    assert np.abs(v2 - v1).max() <= TOL[prec] * np.abs(v1).max()
    assert np.abs(r2 - r1).max() <= TOL_RHS[prec] * np.abs(r1).max()  # the load vector keeps the rule's points
    om, ob = oracle_blocks(wl)
    ed, eo, er = compare(dg.to_blocks(m, v2, r2), om, ob, wl)
    assert ed < TOL[prec] and eo < TOL[prec] and er < TOL_RHS[prec], (ed, eo, er)


def test_exact_moments_3d_persistent(ctx):
    """The persistent pass on volume path 2 in 3D (FP32) against the oracle."""
    import torch

    wl = configs.small3d(6, 24, 32, 1, 3, b=(0.7, -0.4, 0.3), c=1.5)
    m = dg.Mesh(ctx, wl.mesh, wl.p, wl.a, dg_problem(wl))
    ctx.dg_set_volume_path(2)
    ctx.dg_set_persistent(True)
    try:
        v = torch.full((m.nvals,), float("nan"), dtype=torch.float32, device="cuda")
        r = torch.full((m.ndofs,), float("nan"), dtype=torch.float32, device="cuda")
        m.dg_assemble_step(dg.DG_PREC_FP32, v, r)
        ctx.dg_sync()
    finally:
        ctx.dg_set_persistent(False)
        ctx.dg_set_volume_path(1)
    v, r = v.double().cpu().numpy(), r.double().cpu().numpy()
    om, ob = oracle_blocks(wl)
    ed, eo, er = compare(dg.to_blocks(m, v, r), om, ob, wl)
    tol, tr = TOL[dg.DG_PREC_FP32], TOL_RHS[dg.DG_PREC_FP32]
    assert ed < tol and eo < tol and er < tr, (ed, eo, er)
