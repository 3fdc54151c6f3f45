"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle.

Tolerances (block max-norm relative, i.e. max |G - O| / max |O| per block):
  FP64 form: 1e-12.  Both sides sum a few hundred FP64 products per entry in
  different orders; the rounding difference is ~K * 2^-53 ~ 1e-13 at most.
  FP32 form (geometry records equal to the rounded FP64 ones, FP32 basis and
  contraction): 5e-5 per block.
  Basis values carry ~p^2 * 2^-24 relative error and the accumulations run
  over up to ~10^3 rows with partial cancellation; the whole-matrix relative
  Frobenius error is checked against 1e-6.  FP32 load vectors: 1e-4 per
  element.  With the sin source, an element's vector can be small against
  the values of f*phi it sums (cells where u changes sign or vanishes on the
  boundary), and the FP32 rounding of those terms shows relative to the
  vector's own maximum: 5.9e-5 at worst over all 65,536 cells of the 65k-cell
  mesh.
"""
import numpy as np
import pytest

import oracle as O
from paper_2007_04881_gb300 import configs, dg

from .helpers import compare, dg_problem, oracle_blocks

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 5e-5
TOL32_RHS = 1e-4


@pytest.fixture(scope="module")
def ctx(cuda):
    import torch

    from paper_2007_04881_gb300 import build as B

    B.build()
    c = dg.Context(0, torch.cuda.current_stream().cuda_stream)
    yield c
    c.close()


def run_gpu(ctx, wl, prec, split=False, rhs=True, step=False):
    """One assembly.  step=True goes through dg_assemble_step, which also
    recomputes the geometry in the pass's precision: for the reduced forms
    that is the reduced-precision geometry the timed pass uses, where
    dg_assemble takes the records of the upload's FP64 geometry."""
    import torch

    m = dg.Mesh(ctx, wl.mesh, wl.p, wl.a, dg_problem(wl))
    dt = torch.float64 if prec == dg.DG_PREC_FP64 else torch.float32
    vals = torch.full((m.nvals,), float("nan"), dtype=dt, device="cuda")
    r = torch.full((m.ndofs,), float("nan"), dtype=dt, device="cuda") if rhs else None
    if split:
        m.dg_assemble_volume(prec, vals)
        m.dg_assemble_faces(prec, vals)
        if rhs:
            m.dg_assemble_rhs(prec, r)
    elif step:
        m.dg_assemble_step(prec, vals, r)
    else:
        m.dg_assemble(prec, vals, r)
    ctx.dg_sync()
    v = vals.double().cpu().numpy()
    rr = r.double().cpu().numpy() if rhs else None
    return m, v, rr


def blocks(m, v, r):
    return dg.to_blocks(m, v, r)


# ---------------------------------------------------------------------------


@pytest.mark.parametrize("split", [False, True])
def test_small2d_mixed_degree_fp64(ctx, split):
    wl = configs.small2d(180, 7, 1, 6)  # every 2D degree, ragged tiles
    m, v, r = run_gpu(ctx, wl, dg.DG_PREC_FP64, split=split)
    assert np.isfinite(v).all() and np.isfinite(r).all()
    om, ob = oracle_blocks(wl)
    ed, eo, er = compare(blocks(m, v, r), om, ob, wl)
    assert ed < TOL64 and eo < TOL64 and er < TOL64, (ed, eo, er)


@pytest.mark.parametrize("step", [False, True])
def test_small2d_mixed_degree_fp32(ctx, step):
    wl = configs.small2d(180, 7, 1, 6)
    m, v, r = run_gpu(ctx, wl, dg.DG_PREC_FP32, step=step)
    om, ob = oracle_blocks(wl)
    ed, eo, er = compare(blocks(m, v, r), om, ob, wl)
    assert ed < TOL32 and eo < TOL32 and er < TOL32_RHS, (ed, eo, er)


@pytest.mark.parametrize("src", [configs.SRC_SINPROD, configs.SRC_POLY])
def test_small3d_fp64(ctx, src):
    poly = [1, 0.5, -1, 2, 0.3, 0, 0.7, -0.4, 0.2, 0.1, 0.05, -0.2]
    wl = configs.small3d(4, 10, 5, 1, 4, source=src, poly=poly)
    m, v, r = run_gpu(ctx, wl, dg.DG_PREC_FP64)
    om, ob = oracle_blocks(wl)
    ed, eo, er = compare(blocks(m, v, r), om, ob, wl)
    assert ed < TOL64 and eo < TOL64 and er < TOL64, (ed, eo, er)


@pytest.mark.parametrize("step", [False, True])
def test_small3d_fp32(ctx, step):
    wl = configs.small3d(4, 10, 5, 1, 4)
    m, v, r = run_gpu(ctx, wl, dg.DG_PREC_FP32, step=step)
    om, ob = oracle_blocks(wl)
    ed, eo, er = compare(blocks(m, v, r), om, ob, wl)
    assert ed < TOL32 and eo < TOL32 and er < TOL32_RHS, (ed, eo, er)


def test_poisson2d_1k_full_fp64_and_fp32(ctx):
    wl = configs.poisson2d()
    om, ob = oracle_blocks(wl)
    m, v, r = run_gpu(ctx, wl, dg.DG_PREC_FP64)
    ed, eo, er = compare(blocks(m, v, r), om, ob, wl)
    assert ed < TOL64 and eo < TOL64 and er < TOL64, (ed, eo, er)
    m32, v32, r32 = run_gpu(ctx, wl, dg.DG_PREC_FP32)
    rel_fro = np.linalg.norm(v32 - v) / np.linalg.norm(v)
    assert rel_fro < 1e-6, rel_fro


def test_adr2d_65k_sampled(ctx):
    """Full-size 2D ADR workload, in the launch configuration the benchmark
    times; the oracle computes a seeded sample of blocks one by one."""
    wl = configs.adr2d()
    m, v, r = run_gpu(ctx, wl, dg.DG_PREC_FP64)
    assert np.isfinite(v).all()
    rng = np.random.default_rng(123)
    om = O.Mesh(wl.mesh)
    elems = np.sort(rng.choice(wl.ne, 400, replace=False))
    ifs = np.sort(rng.choice(om.ni, 400, replace=False))
    _, ob = oracle_blocks(wl, elems=elems, ifaces=ifs, om=om)
    ed, eo, er = compare(blocks(m, v, r), om, ob, wl)
    assert ed < TOL64 and eo < TOL64 and er < TOL64, (ed, eo, er)
    for step in (False, True):
        m32, v32, r32 = run_gpu(ctx, wl, dg.DG_PREC_FP32, step=step)
        ed, eo, er = compare(blocks(m32, v32, r32), om, ob, wl)
        assert ed < TOL32 and eo < TOL32 and er < TOL32_RHS, (step, ed, eo, er)
        rel_fro = np.linalg.norm(v32 - v) / np.linalg.norm(v)
        assert rel_fro < 1e-6, (step, rel_fro)


def test_bitwise_reproducible(ctx):
    wl = configs.small2d(300, 9, 1, 5)
    _, v1, r1 = run_gpu(ctx, wl, dg.DG_PREC_FP64)
    _, v2, r2 = run_gpu(ctx, wl, dg.DG_PREC_FP64)
    assert np.array_equal(v1, v2) and np.array_equal(r1, r2)
    _, v1, _ = run_gpu(ctx, wl, dg.DG_PREC_FP32)
    _, v2, _ = run_gpu(ctx, wl, dg.DG_PREC_FP32)
    assert np.array_equal(v1, v2)


def test_split_equals_fused(ctx):
    wl = configs.small3d(3, 6, 2, 1, 3)
    _, v1, r1 = run_gpu(ctx, wl, dg.DG_PREC_FP64)
    _, v2, r2 = run_gpu(ctx, wl, dg.DG_PREC_FP64, split=True)
    assert np.abs(v1 - v2).max() <= 1e-13 * np.abs(v1).max()
    assert np.abs(r1 - r2).max() <= 1e-13 * np.abs(r1).max()


def test_order_error(ctx):
    import torch

    wl = configs.small2d(30, 1, 1, 2)
    m = dg.Mesh(ctx, wl.mesh, wl.p, wl.a, dg_problem(wl))
    vals = torch.zeros(m.nvals, dtype=torch.float64, device="cuda")
    with pytest.raises(dg.DGError) as ei:
        m.dg_assemble_faces(dg.DG_PREC_FP64, vals)
    assert ei.value.code == -5


@pytest.mark.parametrize("nx,ny,p", [(1, 1, 6), (2, 1, 1), (3, 2, 4)])
def test_edge_meshes(ctx, nx, ny, p):
    """Single element (no interfaces), two elements, highest degree."""
    from paper_2007_04881_gb300 import meshgen as mg

    mesh = mg.rectangle_grid(nx, ny)
    wl = configs.Workload("rect", mesh, np.full(mesh.ne, p, np.int8), np.linspace(0.5, 2.0, mesh.ne),
                          dict(b=(0.3, -0.7, 0.0), c=0.2, source=1, poly=[], c_sigma=10.0))
    m, v, r = run_gpu(ctx, wl, dg.DG_PREC_FP64)
    om, ob = oracle_blocks(wl)
    ed, eo, er = compare(blocks(m, v, r), om, ob, wl)
    assert ed < TOL64 and eo < TOL64 and er < TOL64


def test_polynomial_reproduction_through_gpu(ctx):
    """Solve the GPU-assembled system densely: u_h reproduces a global
    quadratic (dG consistency), which pins every sign of the GPU path."""
    import torch

    wl = configs.small2d(40, 21, 2, 4, b=(1.0, 0.5), c=1.0, source=configs.SRC_POLY, poly=[1, 1, -2, 0.3, 1, -0.5])
    wl.a[:] = 0.37
    m, v, r = run_gpu(ctx, wl, dg.DG_PREC_FP64)
    row_ptr, col, blk_off, dof_off = m.dg_bsr_pattern()
    N = int(dof_off[-1])
    A = np.zeros((N, N))
    for rr in range(m.ne):
        for k in range(row_ptr[rr], row_ptr[rr + 1]):
            c = col[k]
            A[dof_off[rr]:dof_off[rr + 1], dof_off[c]:dof_off[c + 1]] = v[blk_off[k]:blk_off[k + 1]].reshape(
                dof_off[rr + 1] - dof_off[rr], dof_off[c + 1] - dof_off[c])
    U = np.linalg.solve(A, r)
    om = O.Mesh(wl.mesh)
    pb = O.make_problem(2, b=(1.0, 0.5), c=1.0, source=2, poly=[1, 1, -2, 0.3, 1, -0.5])
    err = 0.0
    for e in range(om.ne):
        xq, _ = om.volume_points(e, 3)
        for x in xq[::4]:
            phi, _ = O.basis(2, int(wl.p[e]), om.lo[e], om.hi[e], x)
            err = max(err, abs(phi @ U[dof_off[e]:dof_off[e + 1]] - O.exact_u(pb, x)))
    assert err < 1e-9, err


def test_host_entry_point_matches_device(ctx):
    import torch

    wl = configs.small2d(120, 4, 1, 4)
    m, v, r = run_gpu(ctx, wl, dg.DG_PREC_FP64)
    vh = np.zeros(m.nvals)
    rh = np.zeros(m.ndofs)
    m.dg_assemble_host(dg.DG_PREC_FP64, vh, rh, x=np.ascontiguousarray(wl.mesh.x), y=np.ascontiguousarray(wl.mesh.y),
                       a=np.ascontiguousarray(wl.a))
    assert np.array_equal(vh, v) and np.array_equal(rh, r)


def test_diff3d_32k_sampled(ctx):
    """Full-size 3D diffusion workload (32,768 agglomerated polyhedra, p=3):
    FP64 and FP32 forms against oracle blocks of a seeded sample."""
    wl = configs.diff3d()
    m, v, r = run_gpu(ctx, wl, dg.DG_PREC_FP64)
    assert np.isfinite(v).all() and np.isfinite(r).all()
    rng = np.random.default_rng(321)
    om = O.Mesh(wl.mesh)
    elems = np.sort(rng.choice(wl.ne, 48, replace=False))
    ifs = np.sort(rng.choice(om.ni, 200, replace=False))
    _, ob = oracle_blocks(wl, elems=elems, ifaces=ifs, om=om)
    ed, eo, er = compare(blocks(m, v, r), om, ob, wl)
    assert ed < TOL64 and eo < TOL64 and er < TOL64, (ed, eo, er)
    for step in (False, True):
        m32, v32, r32 = run_gpu(ctx, wl, dg.DG_PREC_FP32, step=step)
        ed, eo, er = compare(blocks(m32, v32, r32), om, ob, wl)
        assert ed < TOL32 and eo < TOL32 and er < TOL32_RHS, (step, ed, eo, er)
        rel_fro = np.linalg.norm(v32 - v) / np.linalg.norm(v)
        assert rel_fro < 1e-6, (step, rel_fro)
