"""The block pattern built on the device (dg_set_pattern_device): every
array of the pattern (faces, interfaces, block rows and offsets, half-face
lists, face points, work lists) bitwise equal to the host build, on 2D and
3D meshes with mixed degrees, batches and single elements; the assembled
system bitwise equal; the mesh errors of the host build reported alike."""
import numpy as np
import pytest

from paper_2007_04881_gb300 import configs, dg

from .helpers import dg_problem, polygon_workload

pytestmark = pytest.mark.gpu

ARRAYS = ["row_ptr", "col", "blk_off", "dof_off", "blk_if", "diag_blk", "blk_rec", "f_e0", "f_e1", "f_v", "f_flip",
          "f_nq", "f_hf", "hf_ptr", "hf_face", "hf_side", "hf_qoff", "e_nqf", "if_e0", "if_e1", "if_fptr",
          "if_slot01", "if_slot10", "elem_perm", "if_perm", "sub_elem", "uvptr", "uvidx", "elem_pstart", "if_pstart"]


@pytest.fixture(scope="module")
def ctx(cuda):
    import torch

    from paper_2007_04881_gb300 import build as B

    B.build()
    c = dg.Context(0, torch.cuda.current_stream().cuda_stream)
    yield c
    c.close()


def _upload(ctx, w, device):
    ctx.dg_set_pattern_device(device)
    try:
        return dg.Mesh(ctx, w.mesh, w.p, w.a, dg_problem(w))
    finally:
        ctx.dg_set_pattern_device(False)


def _same_system(ctx, mh, md, prec):
    import torch

    dt = torch.float64 if prec == dg.DG_PREC_FP64 else torch.float32
    out = []
    for m in (mh, md):
        v = torch.full((m.nvals,), float("nan"), dtype=dt, device="cuda")
        r = torch.full((m.ndofs,), float("nan"), dtype=dt, device="cuda")
        m.dg_assemble(prec, v, r)
        ctx.dg_sync()
        out.append((v.cpu().numpy(), r.cpu().numpy()))
    return np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


WORKLOADS = [
    lambda: configs.small2d(900, 81, 1, 6, b=(1.0, 0.5), c=1.0),
    lambda: configs.small2d(64, 82, 2, 2),
    lambda: polygon_workload(20, 3),
    lambda: configs.small3d(8, 40, 83, 1, 4),
    lambda: configs.small3d(6, 1, 84, 2, 2),
]


@pytest.mark.parametrize("k", range(len(WORKLOADS)))
def test_device_pattern_equals_host(ctx, k):
    w = WORKLOADS[k]()
    mh = _upload(ctx, w, False)
    md = _upload(ctx, w, True)
    assert md.dg_mesh_timings()["on_device"] and not mh.dg_mesh_timings()["on_device"]
    ih, idv = mh.info, md.info
    for f in ("ne", "nnzb", "nvals", "ndofs", "nfaces", "ninterfaces", "nbfaces", "nsub", "nqvol", "nqface"):
        assert getattr(ih, f) == getattr(idv, f), f
    for name in ARRAYS:
        a, b = mh.dg_mesh_array(name), md.dg_mesh_array(name)
        assert a.shape == b.shape and np.array_equal(a, b), name
    assert _same_system(ctx, mh, md, dg.DG_PREC_FP64)
    assert _same_system(ctx, mh, md, dg.DG_PREC_FP32)


def test_device_pattern_full_size(ctx):
    """The 65,536-cell workload: the pattern bitwise, and the device build
    faster than the host plan."""
    w = configs.adr2d()
    mh = _upload(ctx, w, False)
    md = _upload(ctx, w, True)
    for name in ("row_ptr", "col", "blk_off", "f_e0", "f_e1", "hf_face", "hf_qoff", "elem_perm", "blk_rec"):
        assert np.array_equal(mh.dg_mesh_array(name), md.dg_mesh_array(name)), name
    th, td = mh.dg_mesh_timings(), md.dg_mesh_timings()
    assert td["pattern_ms"] < th["pattern_ms"], (td, th)


def test_device_pattern_mesh_errors(ctx):
    """A loop traversed clockwise and two loops sharing an edge in the same
    direction: DG_ERR_MESH from the device build as from the host build."""
    w = configs.small2d(30, 85, 1, 2)
    mesh = w.mesh
    # reverse the first loop: clockwise
    v = mesh.elem_v.copy()
    a, b = mesh.elem_vptr[0], mesh.elem_vptr[1]
    v[a:b] = v[a:b][::-1]
    bad = type(mesh)(x=mesh.x, y=mesh.y, elem_vptr=mesh.elem_vptr, elem_v=v)
    wb = configs.Workload(name="bad", mesh=bad, p=w.p, a=w.a, problem=w.problem)
    for device in (False, True):
        with pytest.raises(dg.DGError) as ei:
            _upload(ctx, wb, device)
        assert ei.value.code == dg.DG_ERR_MESH
