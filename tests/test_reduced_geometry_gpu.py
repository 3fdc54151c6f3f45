"""Reduced-precision geometry of the FP32 and tensor-core forms.

A reduced pass (dg_assemble_step, the recorded graph, the host-buffer entry
point) recomputes its geometry records in FP32 from coordinates split into
float pairs, with no FP64 arithmetic past the split.  The records are built
to reproduce the rounded FP64 records that dg_assemble uses after an upload,
and these tests hold them to that:

- accuracy parity: on mixed-degree 2D and 3D meshes and a batch of meshes
  the reduced pass is as close to the FP64 form as the FP32 pass on the FP64
  geometry's records (relative Frobenius of the matrix and the load vector,
  within 1.25x + 2e-8; a single element within 1.25x + 2 FP32 epsilons);
- element by element: no element's load vector or diagonal block is more
  than 2x + 1e-6 (block max-norm relative) further from the FP64 form than
  the FP32 pass on FP64 records.  With a strong penalty (a = 100, p = 6) a
  boundary point that leaves the boundary by one ulp multiplies the
  Dirichlet data's rounding by sigma ~ 10^6, and so does a box map that is a
  few ulps off through the basis' slope p (p + 1) / 2 at the box's edge;
- translation: the matrix does not depend on where the mesh sits, so the
  reduced pass on the mesh moved by (1000, -500) agrees with the FP64 form
  of the unmoved mesh to the FP32 form's own accuracy (FP32 coordinates alone
  would lose five of their seven digits there);
- coordinate updates: after dg_mesh_update (an affine map of the mesh) the
  next reduced pass agrees with the FP64 pass on the new coordinates.
"""
import dataclasses

import numpy as np
import pytest

from paper_2007_04881_gb300 import configs, dg

from .helpers import dg_problem, polygon_workload

pytestmark = pytest.mark.gpu

FP32, FP64 = dg.DG_PREC_FP32, dg.DG_PREC_FP64


@pytest.fixture(scope="module")
def ctx(cuda):
    import torch

    from paper_2007_04881_gb300 import build as B

    B.build()
    c = dg.Context(0, torch.cuda.current_stream().cuda_stream)
    yield c
    c.close()


def assemble(ctx, m, prec, step):
    import torch

    dt = torch.float64 if prec == FP64 else torch.float32
    vals = torch.full((m.nvals,), float("nan"), dtype=dt, device="cuda")
    r = torch.full((m.ndofs,), float("nan"), dtype=dt, device="cuda")
    (m.dg_assemble_step if step else m.dg_assemble)(prec, vals, r)
    ctx.dg_sync()
    v, rr = vals.double().cpu().numpy(), r.double().cpu().numpy()
    assert np.isfinite(v).all() and np.isfinite(rr).all()
    return v, rr


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def seg_rel_max(got, ref, off):
    """Per segment [off[i], off[i+1]): max |got - ref| / max |ref|."""
    off = np.asarray(off, dtype=np.int64)
    keep = off[1:] > off[:-1]
    err = np.maximum.reduceat(np.abs(got - ref), off[:-1][keep])
    scale = np.maximum.reduceat(np.abs(ref), off[:-1][keep])
    return err / np.maximum(scale, 1e-300)


def diag_offsets(m):
    row_ptr, col, blk_off, _ = m.dg_bsr_pattern()
    starts, ends = [], []
    for e in range(m.ne):
        b = row_ptr[e] + int(np.nonzero(col[row_ptr[e]:row_ptr[e + 1]] == e)[0][0])
        starts.append(blk_off[b])
        ends.append(blk_off[b + 1])
    return np.array(starts), np.array(ends)


def check_against_fp64_records(ctx, m, floor=2e-8):
    """floor: the additive slack of the accuracy-parity check.  On a mesh of
    many elements the relative Frobenius errors average the rounding of many
    blocks, and 2e-8 holds; a single element's error is one sample of FP32
    rounding (about eps = 6e-8 relative), so two such samples, on two sets of
    records, differ by a few eps whatever the records."""
    v64, r64 = assemble(ctx, m, FP64, False)
    v_old, r_old = assemble(ctx, m, FP32, False)  # FP32 pass on the FP64 geometry's records
    v_new, r_new = assemble(ctx, m, FP32, True)  # reduced-precision geometry
    for got, ref, old in ((v_new, v64, v_old), (r_new, r64, r_old)):
        assert rel(got, ref) <= 1.25 * rel(old, ref) + floor, (rel(got, ref), rel(old, ref))
    dof = m.dg_bsr_pattern()[3]
    e_new, e_old = seg_rel_max(r_new, r64, dof), seg_rel_max(r_old, r64, dof)
    bad = np.nonzero(e_new > 2 * e_old + 1e-6)[0]
    assert bad.size == 0, (bad[:8], e_new[bad[:8]], e_old[bad[:8]])
    s, t = diag_offsets(m)
    d_new = np.array([np.abs(v_new[a:b] - v64[a:b]).max() / np.abs(v64[a:b]).max() for a, b in zip(s, t)])
    d_old = np.array([np.abs(v_old[a:b] - v64[a:b]).max() / np.abs(v64[a:b]).max() for a, b in zip(s, t)])
    bad = np.nonzero(d_new > 2 * d_old + 1e-6)[0]
    assert bad.size == 0, (bad[:8], d_new[bad[:8]], d_old[bad[:8]])
    return v64, v_new


def test_small2d_every_degree(ctx):
    wl = configs.small2d(180, 7, 1, 6)
    m = dg.Mesh(ctx, wl.mesh, wl.p, wl.a, dg_problem(wl))
    check_against_fp64_records(ctx, m)


def test_strong_penalty_boundary(ctx):
    wl = configs.small2d(2000, 11, 6, 6)
    wl = dataclasses.replace(wl, a=np.full(wl.ne, 100.0))
    m = dg.Mesh(ctx, wl.mesh, wl.p, wl.a, dg_problem(wl))
    check_against_fp64_records(ctx, m)


@pytest.mark.parametrize("p", [2, 4])
def test_long_loop(ctx, p):
    """a single 20-gon: the loop exceeds the 16 vertices the element kernel
    keeps in registers, so its runtime-length branch runs"""
    wl = polygon_workload(20, p)
    m = dg.Mesh(ctx, wl.mesh, wl.p, wl.a, dg_problem(wl))
    check_against_fp64_records(ctx, m, floor=2 * float(np.finfo(np.float32).eps))


def test_small3d(ctx):
    wl = configs.small3d(4, 10, 5, 1, 4)
    m = dg.Mesh(ctx, wl.mesh, wl.p, wl.a, dg_problem(wl))
    check_against_fp64_records(ctx, m)


def test_batch(ctx):
    members = configs.batch2d(n_meshes=6, lo=64, hi=600, pmax=5, workers=-1)
    m = dg.Mesh(ctx, None, members=[(w.mesh, w.p, w.a) for w in members], problem=dg_problem(members[0]))
    check_against_fp64_records(ctx, m)


@pytest.mark.parametrize("dim", [2, 3])
def test_translation(ctx, dim):
    if dim == 2:
        wl = configs.small2d(400, 5, 1, 5, source=configs.SRC_ZERO)
        shift = dict(x=1000.0, y=-500.0)
    else:
        wl = configs.small3d(4, 10, 5, 1, 4, source=configs.SRC_ZERO)
        shift = dict(x=1000.0, y=-500.0, z=250.0)
    moved = dataclasses.replace(wl.mesh, **{k: getattr(wl.mesh, k) + s for k, s in shift.items()})
    m0 = dg.Mesh(ctx, wl.mesh, wl.p, wl.a, dg_problem(wl))
    m1 = dg.Mesh(ctx, moved, wl.p, wl.a, dg_problem(wl))
    v64, _ = assemble(ctx, m0, FP64, False)
    v32, _ = assemble(ctx, m0, FP32, True)
    v32_moved, _ = assemble(ctx, m1, FP32, True)
    assert rel(v32_moved, v64) <= 1.5 * rel(v32, v64) + 1e-8, (rel(v32_moved, v64), rel(v32, v64))


def test_coordinate_update(ctx):
    wl = configs.small2d(300, 9, 1, 5)
    m = dg.Mesh(ctx, wl.mesh, wl.p, wl.a, dg_problem(wl))
    assemble(ctx, m, FP32, True)
    # an orientation-preserving affine map (determinant 0.98) moves every
    # vertex and keeps every cell valid
    x0, y0 = wl.mesh.x, wl.mesh.y
    x = np.ascontiguousarray(1.1 * x0 + 0.2 * y0)
    y = np.ascontiguousarray(0.05 * x0 + 0.9 * y0 + 0.3)
    m.dg_mesh_update(x=x, y=y)  # host arrays; the update reruns the FP64 geometry
    v64, r64 = assemble(ctx, m, FP64, True)
    v32, r32 = assemble(ctx, m, FP32, True)
    assert rel(v32, v64) < 1e-6 and rel(r32, r64) < 1e-6, (rel(v32, v64), rel(r32, r64))
    moved = dataclasses.replace(wl.mesh, x=x, y=y)
    m2 = dg.Mesh(ctx, moved, wl.p, wl.a, dg_problem(wl))
    v64b, _ = assemble(ctx, m2, FP64, False)
    assert rel(v64, v64b) < 1e-12
