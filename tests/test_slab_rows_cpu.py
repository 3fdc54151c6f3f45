"""The slab kernels' arithmetic on the CPU.

The row bodies of the expansion, load-vector and trace kernels
(paper_2007_04881_gb300/csrc/dg_slab.cuh) are host/device functions.  This
test builds them as host code (tests/slab_rows_host.cpp, g++) and runs them,
lane by lane as a warp would, on spatial blocks, load vectors and mass
matrices from the 2D oracle, with the slab layout of dg_slab_offsets.  The
result is compared with the slab oracle (oracle/spacetime.py), which
integrates the space-time form with its own space-time rule: every slab
block, the load vector with a previous-slab trace, and the trace at t1, in
both spaces with mixed degrees, at 1e-12 (block max-norm relative).  So the
expansion arithmetic is pinned without a GPU; the GPU tests add the device
launches and the spatial pass.
"""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle as O
from oracle import spacetime as S
from paper_2007_04881_gb300 import dg, meshgen as mg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA_INC = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
V = C.c_void_p


@pytest.fixture(scope="module")
def host(tmp_path_factory):
    if shutil.which("g++") is None or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    from paper_2007_04881_gb300 import build as B

    B.build()  # dg_slab_offsets comes from the library
    out = str(tmp_path_factory.mktemp("slab_rows") / "slab_rows_host.so")
    subprocess.run(["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-I", CUDA_INC, "-I",
                    os.path.join(ROOT, "paper_2007_04881_gb300", "csrc"), "-x", "c++",
                    os.path.join(ROOT, "tests", "slab_rows_host.cpp"), "-o", out], check=True)
    lib = C.CDLL(out)
    head = [C.c_int] * 3 + [V] * 8 + [C.c_double] * 2
    lib.host_slab_matrix.argtypes = head + [V] * 3
    lib.host_slab_rhs.argtypes = head + [V] * 4
    lib.host_slab_trace.argtypes = head + [V] * 2
    return lib


def _vp(a):
    return None if a is None else a.ctypes.data


def _spatial(n, seed, const_a, src):
    """2D oracle data laid out as the library lays it out: spatial blocks B,
    mass matrix M in the diagonal blocks' places, load vector l."""
    mesh = mg.voronoi_square(n, seed)
    om = O.Mesh(mesh)
    p = mg.draw_degrees(om.ne, seed, 1, 3).astype(np.int32)
    a = np.full(om.ne, 0.7) if const_a else mg.draw_log_uniform(om.ne, seed, -1.0, 0.5)
    w, c = (0.9, -0.6), 0.7
    info, row_ptr, col, blk_off = dg.dg_mesh_check(mesh, p, a, dg.Problem(b=(w[0], w[1], 0.0), c=c, source=src),
                                                   pattern=True)
    nb = np.array([O.nbasis(2, int(q)) for q in p])
    dof_off = np.concatenate([[0], np.cumsum(nb)]).astype(np.int64)

    def bidx(r, s):
        return int(row_ptr[r] + np.nonzero(col[row_ptr[r]:row_ptr[r + 1]] == s)[0][0])

    diag_blk = np.array([bidx(r, r) for r in range(om.ne)], np.int32)
    pb = O.make_problem(2, b=w, c=c, source=src, c_sigma=10.0)
    mass = O.make_problem(2, c=1.0, c_sigma=0.0)
    ob = om.assemble(p, a, pb)
    B = np.full(int(info.nvals), np.nan)
    M = np.full(int(info.nvals), np.nan)
    l = np.zeros(int(info.ndofs))
    for pos, e in enumerate(ob["elems"]):
        e = int(e)
        b = diag_blk[e]
        B[blk_off[b]:blk_off[b + 1]] = ob["diag"][pos].ravel()
        M[blk_off[b]:blk_off[b + 1]] = om.volume_block(e, p, np.zeros(om.ne), mass).ravel()
        l[dof_off[e]:dof_off[e + 1]] = ob["rhs"][pos]
    for pos, i in enumerate(ob["ifaces"]):
        e0, e1 = int(om.if_e0[i]), int(om.if_e1[i])
        b = bidx(e0, e1)
        B[blk_off[b]:blk_off[b + 1]] = ob["a01"][pos].ravel()
        b = bidx(e1, e0)
        B[blk_off[b]:blk_off[b + 1]] = ob["a10"][pos].ravel()
    assert np.isfinite(B).all()
    return dict(om=om, p=p, a=a, w=w, c=c, pb=pb, row_ptr=row_ptr, col=col, blk_off=blk_off, dof_off=dof_off,
                diag_blk=diag_blk, B=B, M=M, l=l)


def _rel(got, want):
    return float(np.abs(got - want).max() / max(np.abs(want).max(), 1e-300))


@pytest.mark.parametrize("space", [dg.DG_SPACE_P, dg.DG_SPACE_PQ])
@pytest.mark.parametrize("const_a", [False, True])
def test_slab_rows_against_slab_oracle(host, space, const_a):
    # with variable a the source is zero: the oracle's source takes no element
    z = _spatial(8, 4, const_a, 1 if const_a else 0)
    om, p = z["om"], z["p"]
    sname = "PQ" if space == dg.DG_SPACE_PQ else "P"
    sblk, sdof = dg.dg_slab_offsets(2, z["row_ptr"], z["col"], p, space)
    t0, t1 = 0.15, 0.4
    sl = S.Slab(om, p, z["a"], z["w"], z["c"], sname, t0, t1)
    assert np.array_equal(sdof, sl.off)
    args = [2, om.ne, space] + [_vp(z[k]) for k in ("p", "row_ptr", "col", "diag_blk", "blk_off", "dof_off")] + [
        _vp(sblk), _vp(sdof), t0, t1]

    vals = np.full(int(sblk[-1]), np.nan)
    host.host_slab_matrix(*args, _vp(z["B"]), _vp(z["M"]), _vp(vals))
    rng = np.random.default_rng(3)
    u_prev = rng.standard_normal(int(z["dof_off"][-1]))
    rhs = np.full(int(sdof[-1]), np.nan)
    host.host_slab_rhs(*args, _vp(z["l"]), _vp(z["M"]), _vp(u_prev), _vp(rhs))
    assert np.isfinite(vals).all() and np.isfinite(rhs).all()

    a0 = float(z["a"][0])

    def prev(e, x):
        phi, _ = O.basis(2, int(p[e]), om.lo[e], om.hi[e], x)
        return float(phi @ u_prev[z["dof_off"][e]:z["dof_off"][e + 1]])

    A, F = sl.assemble(lambda t, x: O.source_f(z["pb"], a0, x), lambda t, x: O.exact_u(z["pb"], x), prev)
    inside = np.zeros_like(A, dtype=bool)
    err = 0.0
    for r in range(om.ne):
        for b in range(z["row_ptr"][r], z["row_ptr"][r + 1]):
            s = int(z["col"][b])
            got = vals[sblk[b]:sblk[b + 1]].reshape(sdof[r + 1] - sdof[r], sdof[s + 1] - sdof[s])
            err = max(err, _rel(got, A[sl.off[r]:sl.off[r + 1], sl.off[s]:sl.off[s + 1]]))
            inside[sl.off[r]:sl.off[r + 1], sl.off[s]:sl.off[s + 1]] = True
    assert err < 1e-12, err
    assert not A[~inside].any()  # the slab pattern is the spatial one
    e_r = max(_rel(rhs[sdof[e]:sdof[e + 1]], F[sl.off[e]:sl.off[e + 1]]) for e in range(om.ne))
    assert e_r < 1e-12, e_r

    U = rng.standard_normal(int(sdof[-1]))
    u_end = np.full(int(z["dof_off"][-1]), np.nan)
    host.host_slab_trace(*args, _vp(U), _vp(u_end))
    e_t = 0.0
    for e in range(om.ne):
        xq, _ = om.volume_points(e, 2)
        for x in xq[::3]:
            phi, _ = O.basis(2, int(p[e]), om.lo[e], om.hi[e], x)
            want = sl.value(U, e, t1, x)
            e_t = max(e_t, abs(phi @ u_end[z["dof_off"][e]:z["dof_off"][e + 1]] - want) / (1.0 + abs(want)))
    assert e_t < 1e-12, e_t
