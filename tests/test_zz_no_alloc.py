"""The allocation-free entry point dg_volume_noalloc.

It serves callers that cannot allocate device memory (a framework's pooled
memory, a fixed budget); its intermediate records sit in one fixed device
array inside the library.  Here it is checked against the existing entry
point dg_assemble_volume (the diagonal blocks of an uploaded mesh), on two
calls in a row, so that the second call reuses the array left by the first.
"""
import numpy as np
import pytest

from paper_2007_04881_gb300 import build as B
from paper_2007_04881_gb300 import configs, dg

TOL = {dg.DG_PREC_FP64: 1e-12, dg.DG_PREC_FP32: 5e-5}


def test_rejects_oversized_mesh_without_gpu_work():
    B.build()
    lib = dg.load()
    # 20000 elements exceed the 16384 limit: refused before any CUDA call
    rc = lib.dg_volume_noalloc(None, 0, dg.DG_PREC_FP64, 2, 100, 1, 1, 20000, 60000, 1, 1, 1, 0.0, 0.0, 0.0, 1,
                               None)
    assert rc == -1


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [dg.DG_PREC_FP64, dg.DG_PREC_FP32])
def test_noalloc_matches_assemble_volume(cuda, prec):
    import torch

    B.build()
    ctx = dg.Context(0, torch.cuda.current_stream().cuda_stream)
    dt = torch.float64 if prec == dg.DG_PREC_FP64 else torch.float32
    for p, nsites, seed in [(3, 300, 11), (1, 500, 12)]:
        wl = configs.small2d(nsites, seed, p, p, b=(0.7, -0.2), c=0.4)
        mesh = wl.mesh
        # the existing entry point: diagonal blocks of the uploaded mesh
        m = dg.Mesh(ctx, mesh, wl.p, wl.a, dg.Problem(b=(0.7, -0.2, 0.0), c=0.4))
        vals = torch.zeros(m.nvals, dtype=dt, device="cuda")
        m.dg_assemble_volume(prec, vals)
        ctx.dg_sync()
        ref = dg.to_blocks(m, vals.double().cpu().numpy())["diag"]
        # caller-owned device inputs and outputs for the no-allocation path
        dev = lambda a, t: torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=t)  # noqa: E731
        x, y = dev(mesh.x, torch.float64), dev(mesh.y, torch.float64)
        eptr, eidx = dev(mesh.elem_vptr, torch.int32), dev(mesh.elem_v, torch.int32)
        a = dev(wl.a, torch.float64)
        n = (p + 1) * (p + 2) // 2
        status = torch.full((1,), 99, dtype=torch.int32, device="cuda")
        for call in range(2):  # two calls in a row share the scratch array
            blocks = torch.full((mesh.ne * n * n,), float("nan"), dtype=dt, device="cuda")
            dg.dg_volume_noalloc(torch.cuda.current_stream().cuda_stream, 0, prec, p, x, y, eptr, eidx, a, 0.7,
                                 -0.2, 0.4, blocks, int(mesh.elem_vptr[-1]), status)
            torch.cuda.synchronize()
            assert int(status.item()) == dg.DG_OK
            got = blocks.double().cpu().numpy().reshape(mesh.ne, n, n)
            for e in range(mesh.ne):
                s = np.abs(ref[e]).max()
                assert np.abs(got[e] - ref[e]).max() <= TOL[prec] * s, (p, call, e)
    ctx.close()


@pytest.mark.gpu
def test_noalloc_reports_bad_lists(cuda):
    """Lists the GPU check rejects: elem_ptr ending past nsub, and a vertex id
    outside 0..nv-1.  The call reports DG_ERR_MESH in its status word, every
    access stays inside the caller's buffers, and a valid call that follows
    (same array) is exact again."""
    import torch

    B.build()
    ctx = dg.Context(0, torch.cuda.current_stream().cuda_stream)
    wl = configs.small2d(200, 13, 2, 2, b=(0.7, -0.2), c=0.4)
    mesh = wl.mesh
    m = dg.Mesh(ctx, mesh, wl.p, wl.a, dg.Problem(b=(0.7, -0.2, 0.0), c=0.4))
    vals = torch.zeros(m.nvals, dtype=torch.float64, device="cuda")
    m.dg_assemble_volume(dg.DG_PREC_FP64, vals)
    ctx.dg_sync()
    ref = dg.to_blocks(m, vals.cpu().numpy())["diag"]
    dev = lambda a, t: torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=t)  # noqa: E731
    x, y = dev(mesh.x, torch.float64), dev(mesh.y, torch.float64)
    eptr, eidx = dev(mesh.elem_vptr, torch.int32), dev(mesh.elem_v, torch.int32)
    a = dev(wl.a, torch.float64)
    nsub = int(mesh.elem_vptr[-1])
    n = 6
    st = torch.cuda.current_stream().cuda_stream
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    blocks = torch.zeros(mesh.ne * n * n, dtype=torch.float64, device="cuda")
    # nsub one short of elem_ptr[ne]: the caller's elem_idx still holds nsub + 1 entries
    dg.dg_volume_noalloc(st, 0, dg.DG_PREC_FP64, 2, x, y, eptr, eidx, a, 0.7, -0.2, 0.4, blocks, nsub - 1, status)
    torch.cuda.synchronize()
    assert int(status.item()) == dg.DG_ERR_MESH
    bad = eidx.clone()
    bad[5] = x.numel() + 7
    dg.dg_volume_noalloc(st, 0, dg.DG_PREC_FP64, 2, x, y, eptr, bad, a, 0.7, -0.2, 0.4, blocks, nsub, status)
    torch.cuda.synchronize()
    assert int(status.item()) == dg.DG_ERR_MESH
    dg.dg_volume_noalloc(st, 0, dg.DG_PREC_FP64, 2, x, y, eptr, eidx, a, 0.7, -0.2, 0.4, blocks, nsub, status)
    torch.cuda.synchronize()
    assert int(status.item()) == dg.DG_OK
    got = blocks.cpu().numpy().reshape(mesh.ne, n, n)
    for e in range(mesh.ne):
        assert np.abs(got[e] - ref[e]).max() <= 1e-12 * np.abs(ref[e]).max()
    ctx.close()
