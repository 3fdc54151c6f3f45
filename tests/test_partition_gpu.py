"""Partitions on one GPU (Sec. 4.2): each part, uploaded with its halo and
assembled alone, reproduces its block rows and load-vector entries of the
whole mesh bit for bit, and the parts together cover the whole matrix."""
import numpy as np
import pytest

from paper_2007_04881_gb300 import configs, dg

from .helpers import dg_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(cuda):
    import torch

    from paper_2007_04881_gb300 import build as B

    B.build()
    c = dg.Context(0, torch.cuda.current_stream().cuda_stream)
    yield c
    c.close()


def _assemble(ctx, mesh, prec):
    import torch

    dt = torch.float64 if prec == dg.DG_PREC_FP64 else torch.float32
    v = torch.full((mesh.nvals,), float("nan"), dtype=dt, device="cuda")
    r = torch.full((max(mesh.ndofs, 1),), float("nan"), dtype=dt, device="cuda")
    mesh.dg_assemble_step(prec, v, r)
    ctx.dg_sync()
    return v.cpu().numpy(), r.cpu().numpy()


@pytest.mark.parametrize("prec", [dg.DG_PREC_FP64, dg.DG_PREC_FP32])
@pytest.mark.parametrize("which,nparts", [("2d", 4), ("3d", 3)])
def test_parts_reproduce_whole_mesh_bitwise(ctx, prec, which, nparts):
    if which == "2d":
        wl = configs.small2d(600, 81, 1, 5, b=(1.0, 0.5), c=1.0)
    else:
        wl = configs.small3d(6, 70, 82, 1, 3)
    pb = dg_problem(wl)
    full = dg.Mesh(ctx, wl.mesh, wl.p, wl.a, pb)
    fv, fr = _assemble(ctx, full, prec)
    f_rp, f_col, f_bo, f_do = full.dg_bsr_pattern()
    part = dg.dg_partition(wl.mesh, wl.p, wl.a, pb, nparts)
    covered_vals = np.zeros(full.nvals, bool)
    covered_dofs = np.zeros(full.ndofs, bool)
    for k in range(nparts):
        pm = dg.Mesh(ctx, wl.mesh, wl.p, wl.a, pb, part=part, my_part=k)
        assert pm.nowned == int(np.sum(part == k))
        pv, pr = _assemble(ctx, pm, prec)
        rp, col, bo, do = pm.dg_bsr_pattern()
        eg = pm.elem_global
        for e in np.flatnonzero(pm.owned):
            g = int(eg[e])
            fcols = f_col[f_rp[g]:f_rp[g + 1]]
            for bk in range(rp[e], rp[e + 1]):
                gc = int(eg[col[bk]])
                fb = f_rp[g] + int(np.searchsorted(fcols, gc))
                assert f_col[fb] == gc
                a = pv[bo[bk]:bo[bk + 1]]
                b = fv[f_bo[fb]:f_bo[fb + 1]]
                assert a.shape == b.shape and np.array_equal(a, b), (k, g, gc)
                covered_vals[f_bo[fb]:f_bo[fb + 1]] = True
            assert np.array_equal(pr[do[e]:do[e + 1]], fr[f_do[g]:f_do[g + 1]])
            covered_dofs[f_do[g]:f_do[g + 1]] = True
        assert pm.vert_global.size > 0 and np.all(np.diff(pm.vert_global) > 0)
        pm.close()
    assert covered_vals.all() and covered_dofs.all()
    full.close()
