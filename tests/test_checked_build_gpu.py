"""The checked build (DG_CHECK_BOUNDS=1: every kernel tests its output ranges
before writing and reports a failure through dg_sync as DG_ERR_BOUNDS instead
of faulting).  Built and run in a subprocess, since one process loads one
library: on valid meshes no check fires (dg_sync returns DG_OK) and the
systems equal the default build's (FP64 to 1e-13 and FP32 to 1e-6 of each
array's largest entry: the checks wrap the writes, the arithmetic is the
same).  No test plants an out-of-range index: an access the checks do not
cover could then fault the GPU."""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2007_04881_gb300 import configs, dg

from .helpers import dg_problem

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
from paper_2007_04881_gb300 import build as B
from paper_2007_04881_gb300 import configs, dg
B.build()
from tests.helpers import dg_problem
out = {}
ctx = dg.Context(0, torch.cuda.current_stream().cuda_stream)
cases = {"2d": configs.small2d(300, 17, 1, 6, neumann=0b0110), "3d": configs.small3d(4, 10, 5, 1, 4)}
for name, wl in cases.items():
    m = dg.Mesh(ctx, wl.mesh, wl.p, wl.a, dg_problem(wl))
    for prec, dt in ((dg.DG_PREC_FP64, torch.float64), (dg.DG_PREC_FP32, torch.float32),
                     (dg.DG_PREC_TF32X3, torch.float32)):
        v = torch.zeros(m.nvals, dtype=dt, device="cuda")
        r = torch.zeros(m.ndofs, dtype=dt, device="cuda")
        m.dg_assemble_step(prec, v, r)
        ctx.dg_sync()
        out[f"{name}_{prec}_v"] = v.double().cpu().numpy()
        out[f"{name}_{prec}_r"] = r.double().cpu().numpy()
    m.close()
wl = configs.small3d(4, 10, 5, 1, 4)
m = dg.Mesh(ctx, wl.mesh, wl.p, wl.a, dg.Problem(source=1))
v = torch.zeros(m.nvals, dtype=torch.float32, device="cuda")
r = torch.zeros(m.ndofs, dtype=torch.float32, device="cuda")
m.dg_assemble_varcoef(v, r, prec=dg.DG_PREC_FP32)
ctx.dg_sync()
out["vc_v"], out["vc_r"] = v.double().cpu().numpy(), r.double().cpu().numpy()
np.savez(sys.argv[2], **out)
'''


def _default(ctx_arrays):
    import torch

    out = {}
    ctx = dg.Context(0, torch.cuda.current_stream().cuda_stream)
    cases = {"2d": configs.small2d(300, 17, 1, 6, neumann=0b0110), "3d": configs.small3d(4, 10, 5, 1, 4)}
    for name, wl in cases.items():
        m = dg.Mesh(ctx, wl.mesh, wl.p, wl.a, dg_problem(wl))
        for prec, dt in ((dg.DG_PREC_FP64, torch.float64), (dg.DG_PREC_FP32, torch.float32),
                         (dg.DG_PREC_TF32X3, torch.float32)):
            v = torch.zeros(m.nvals, dtype=dt, device="cuda")
            r = torch.zeros(m.ndofs, dtype=dt, device="cuda")
            m.dg_assemble_step(prec, v, r)
            ctx.dg_sync()
            out[f"{name}_{prec}_v"] = v.double().cpu().numpy()
            out[f"{name}_{prec}_r"] = r.double().cpu().numpy()
        m.close()
    wl = configs.small3d(4, 10, 5, 1, 4)
    m = dg.Mesh(ctx, wl.mesh, wl.p, wl.a, dg.Problem(source=1))
    v = torch.zeros(m.nvals, dtype=torch.float32, device="cuda")
    r = torch.zeros(m.ndofs, dtype=torch.float32, device="cuda")
    m.dg_assemble_varcoef(v, r, prec=dg.DG_PREC_FP32)
    ctx.dg_sync()
    out["vc_v"], out["vc_r"] = v.double().cpu().numpy(), r.double().cpu().numpy()
    ctx.close()
    return out


def test_checked_build_matches_default(cuda, tmp_path):
    from paper_2007_04881_gb300 import build as B

    B.build()
    res = tmp_path / "checked.npz"
    env = dict(os.environ, DG_CHECK_BOUNDS="1")
    r = subprocess.run([sys.executable, "-c", SCRIPT, ROOT, str(res)], env=env, cwd=ROOT, capture_output=True,
                       text=True, timeout=1200)
    assert r.returncode == 0, r.stderr[-3000:]
    got = np.load(res)
    ref = _default(None)
    assert set(got.files) == set(ref)
    for k, a in ref.items():
        b = got[k]
        tol = 1e-13 if f"_{dg.DG_PREC_FP64}_" in k else 1e-6
        assert a.shape == b.shape and np.abs(a - b).max() <= tol * max(np.abs(a).max(), 1e-300), k


def test_nvtx_ranges_leave_results_unchanged(cuda):
    import torch

    ctx = dg.Context(0, torch.cuda.current_stream().cuda_stream)
    wl = configs.small2d(200, 9, 1, 4)
    m = dg.Mesh(ctx, wl.mesh, wl.p, wl.a, dg_problem(wl))
    out = []
    for on in (False, True):
        ctx.dg_set_nvtx(on)
        v = torch.zeros(m.nvals, dtype=torch.float32, device="cuda")
        r = torch.zeros(m.ndofs, dtype=torch.float32, device="cuda")
        m.dg_assemble_step(dg.DG_PREC_FP32, v, r)
        ctx.dg_sync()
        out.append((v.cpu().numpy(), r.cpu().numpy()))
    ctx.dg_set_nvtx(False)
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    m.close()
    ctx.close()
