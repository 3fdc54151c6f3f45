"""The variable-coefficient kernels' arithmetic on the CPU (2D).

The row bodies that add the b(x) = 1 + x, c(x) = 3 + xy terms (Sec. 4.2;
paper_2007_04881_gb300/csrc/dg_varcoef.cuh) are host/device functions.  This
test builds them as host code (tests/varcoef_rows_host.cpp, g++) and runs
them, lane by lane as a warp would, on geometry records laid out as the row
kernels' (element boxes, fan sub-triangles in box coordinates, face sides
with their scaled normals) and on the reference rules.  What they add must
equal the oracle's system with the variable fields minus the oracle's system
with b = 0, c = 0 (oracle coef 1 minus coef 0): every block and every
load-vector entry, mixed degrees, the sin source and the zero source, at
1e-12 of each block's largest entry.
"""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle as O
from paper_2007_04881_gb300 import dg, meshgen as mg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA_INC = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
V = C.c_void_p


@pytest.fixture(scope="module")
def host(tmp_path_factory):
    if shutil.which("g++") is None or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    from paper_2007_04881_gb300 import build as B

    B.build()  # dg_mesh_check (the block pattern) comes from the library
    out = str(tmp_path_factory.mktemp("varcoef_rows") / "varcoef_rows_host.so")
    subprocess.run(["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-I", CUDA_INC, "-I",
                    os.path.join(ROOT, "paper_2007_04881_gb300", "csrc"), "-x", "c++",
                    os.path.join(ROOT, "tests", "varcoef_rows_host.cpp"), "-o", out], check=True)
    lib = C.CDLL(out)
    lib.host_varcoef_2d.argtypes = [V] * 24
    return lib


def _gauss01(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def _rules():
    """Volume rules of degree 0..7 ((p + 2)^2 collapsed points (r, s, w)) and
    face rules of 0..9 points ((t, w)), packed, with their offsets."""
    vol, vol_off, vol_n = [], [], []
    for p in range(8):
        g, gw = _gauss01(p + 2)
        vol_off.append(len(vol) // 3)
        for ia in range(p + 2):
            for ib in range(p + 2):
                a, b = g[ia], g[ib]
                vol += [a * (1.0 - b), b, gw[ia] * gw[ib] * (1.0 - b)]
        vol_n.append((p + 2) ** 2)
    face, face_off, face_n = [], [], []
    for n in range(10):
        face_off.append(len(face) // 2)
        if n > 0:
            g, gw = _gauss01(n)
            for t, w in zip(g, gw):
                face += [t, w]
        face_n.append(n)
    offs = np.array(vol_off + vol_n + face_off + face_n, np.int32)
    return np.array(vol), np.array(face), offs


def _records(mesh, p, row_ptr, col):
    """Geometry records and face topology of a 2D mesh in the row kernels'
    layouts (fan apex = area centroid, faces along the first element's CCW
    loop with the normal out of it)."""
    ne = mesh.ne
    X = np.stack([mesh.x, mesh.y])
    ptr, idx = mesh.elem_vptr, mesh.elem_v
    lo = np.zeros((2, ne))
    L = np.zeros((2, ne))
    cen = np.zeros((2, ne))
    for e in range(ne):
        v = idx[ptr[e]:ptr[e + 1]]
        P = X[:, v]
        lo[:, e] = P.min(axis=1)
        L[:, e] = P.max(axis=1) - P.min(axis=1)
        Q = np.roll(P, -1, axis=1)
        cr = P[0] * Q[1] - Q[0] * P[1]
        area = 0.5 * cr.sum()
        cen[:, e] = ((P + Q) * cr).sum(axis=1) / (6.0 * area)
    eg = np.concatenate([lo, L, 1.0 / L, (1.0 / np.sqrt(L[0] * L[1]))[None, :]])

    def xi(x, e):
        return 2.0 * (x - lo[:, e]) / L[:, e] - 1.0

    nsub = int(ptr[-1])
    sg = np.zeros((7, nsub))
    for e in range(ne):
        v = idx[ptr[e]:ptr[e + 1]]
        c = cen[:, e]
        for i in range(len(v)):
            p1, p2 = X[:, v[i]], X[:, v[(i + 1) % len(v)]]
            k = ptr[e] + i
            sg[0:2, k] = xi(c, e)
            sg[2:4, k] = xi(p1, e) - xi(c, e)
            sg[4:6, k] = xi(p2, e) - xi(c, e)
            sg[6, k] = abs((p1[0] - c[0]) * (p2[1] - c[1]) - (p1[1] - c[1]) * (p2[0] - c[0]))
    # faces: every loop edge, owned by the lower element that sees it
    seen = {}
    for e in range(ne):
        v = idx[ptr[e]:ptr[e + 1]]
        for i in range(len(v)):
            a, b = int(v[i]), int(v[(i + 1) % len(v)])
            seen.setdefault(frozenset((a, b)), []).append((e, a, b))
    faces = []
    for key, sides in seen.items():
        sides.sort()
        e0, a, b = sides[0]
        e1 = sides[1][0] if len(sides) > 1 else -1
        faces.append((e0, e1, a, b))
    faces.sort(key=lambda f: (min(f[0], f[1]) if f[1] >= 0 else f[0], max(f[0], f[1]), f[2]))
    pairs = sorted({(f[0], f[1]) for f in faces if f[1] >= 0})
    iface = {pr: i for i, pr in enumerate(pairs)}
    faces.sort(key=lambda f: (iface.get((f[0], f[1]), len(pairs)), f[2], f[3]))
    nf = len(faces)
    f_e0 = np.array([f[0] for f in faces], np.int32)
    f_e1 = np.array([f[1] for f in faces], np.int32)
    f_nq = np.array([max(p[f[0]], p[f[1]] if f[1] >= 0 else 0) + 1 for f in faces], np.int32)
    if_fptr = np.zeros(len(pairs) + 1, np.int32)
    for f in faces:
        if f[1] >= 0:
            if_fptr[iface[(f[0], f[1])] + 1] += 1
    if_fptr = np.cumsum(if_fptr).astype(np.int32)
    fs = np.zeros((2, 6, nf))
    fsc = np.zeros((3, nf))
    for k, (e0, e1, a, b) in enumerate(faces):
        P0, P1 = X[:, a], X[:, b]
        t = P1 - P0
        ln = np.hypot(t[0], t[1])
        n0 = np.array([t[1], -t[0]]) / ln  # the CCW loop of e0 has its interior on the left
        fsc[0, k] = ln
        for s, e in enumerate((e0, e1)):
            if e < 0:
                continue
            fs[s, 0:2, k] = xi(P0, e)
            fs[s, 2:4, k] = xi(P1, e) - xi(P0, e)
            fs[s, 4:6, k] = 2.0 * n0 / L[:, e]
    hf = [[] for _ in range(ne)]
    for k, (e0, e1, _, _) in enumerate(faces):
        hf[e0].append((k, 0))
        if e1 >= 0:
            hf[e1].append((k, 1))
    hf_ptr = np.concatenate([[0], np.cumsum([len(h) for h in hf])]).astype(np.int32)
    hf_face = np.array([k for h in hf for k, _ in h], np.int32)
    hf_side = np.array([s for h in hf for _, s in h], np.int8)
    blk_if = np.full(col.size, -1, np.int32)
    for r in range(ne):
        for b in range(row_ptr[r], row_ptr[r + 1]):
            s = int(col[b])
            if s != r:
                blk_if[b] = iface[(min(r, s), max(r, s))]
    return dict(eg=np.ascontiguousarray(eg), sg=sg, fs=fs, fsc=fsc, f_e0=f_e0, f_e1=f_e1, f_nq=f_nq,
                hf_ptr=hf_ptr, hf_face=hf_face, hf_side=hf_side, if_fptr=if_fptr, blk_if=blk_if, nf=nf, nsub=nsub)


def _vp(a):
    return a.ctypes.data


@pytest.mark.parametrize("source", [0, 1])
@pytest.mark.parametrize("n,seed", [(12, 3), (30, 8)])
def test_varcoef_rows_against_oracle(host, source, n, seed):
    mesh = mg.voronoi_square(n, seed)
    om = O.Mesh(mesh)
    p = mg.draw_degrees(om.ne, seed, 1, 4).astype(np.int32)
    a = mg.draw_log_uniform(om.ne, seed, -1.0, 1.0)
    info, row_ptr, col, blk_off = dg.dg_mesh_check(mesh, p, a, dg.Problem(source=source), pattern=True)
    nb = np.array([O.nbasis(2, int(q)) for q in p])
    dof_off = np.concatenate([[0], np.cumsum(nb)]).astype(np.int64)
    R = _records(mesh, p, row_ptr, col)
    vol, face, offs = _rules()
    vals = np.zeros(int(info.nvals))
    rhs = np.zeros(int(info.ndofs))
    ints = np.array([om.ne, R["nf"], R["nsub"], source], np.int32)
    eptr = np.ascontiguousarray(mesh.elem_vptr, np.int32)
    host.host_varcoef_2d(_vp(ints), _vp(p), _vp(eptr), _vp(R["eg"]), _vp(R["sg"]), _vp(R["fs"]), _vp(R["fsc"]),
                         _vp(R["f_e0"]), _vp(R["f_e1"]), _vp(R["f_nq"]), _vp(R["hf_ptr"]), _vp(R["hf_face"]),
                         _vp(R["hf_side"]), _vp(R["if_fptr"]), _vp(row_ptr), _vp(col), _vp(R["blk_if"]),
                         _vp(blk_off), _vp(dof_off), _vp(vol), _vp(face), _vp(offs), _vp(vals), _vp(rhs))
    assert np.isfinite(vals).all() and np.isfinite(rhs).all()

    o1 = om.assemble(p, a, O.make_problem(2, source=source, coef=1, c_sigma=10.0))
    o0 = om.assemble(p, a, O.make_problem(2, b=(0.0, 0.0), c=0.0, source=source, c_sigma=10.0))

    def block(r, s):
        b = int(row_ptr[r] + np.nonzero(col[row_ptr[r]:row_ptr[r + 1]] == s)[0][0])
        return vals[blk_off[b]:blk_off[b + 1]].reshape(nb[r], nb[s])

    err = 0.0
    for pos, e in enumerate(o1["elems"]):
        e = int(e)
        want = o1["diag"][pos] - o0["diag"][pos]
        err = max(err, np.abs(block(e, e) - want).max() / np.abs(o1["diag"][pos]).max())
    for pos, i in enumerate(o1["ifaces"]):
        e0, e1 = int(om.if_e0[i]), int(om.if_e1[i])
        for got, w1, w0 in ((block(e0, e1), o1["a01"][pos], o0["a01"][pos]),
                            (block(e1, e0), o1["a10"][pos], o0["a10"][pos])):
            err = max(err, np.abs(got - (w1 - w0)).max() / np.abs(w1).max())
    assert err < 1e-12, err
    e_r = 0.0
    for pos, e in enumerate(o1["elems"]):
        e = int(e)
        want = o1["rhs"][pos] - o0["rhs"][pos]
        scale = max(np.abs(o1["rhs"][pos]).max(), 1e-300)
        e_r = max(e_r, np.abs(rhs[dof_off[e]:dof_off[e + 1]] - want).max() / scale)
    assert e_r < 1e-12, e_r
