"""The variable-coefficient kernels' arithmetic on the CPU (2D and 3D).

The row bodies that add the b_d(x) = 1 + x_d, c(x) = 3 + prod x_d terms (Sec. 4.2;
paper_2007_04881_gb300/csrc/dg_varcoef.cuh) are host/device functions.  This
test builds them as host code (tests/varcoef_rows_host.cpp, g++) and runs
them, lane by lane as a warp would, on geometry records laid out as the row
kernels' (element boxes, fan sub-triangles or the element's tetrahedra in box
coordinates, face sides with their scaled normals, 3D faces in the vertex
order of the lower element's tetrahedron) and on the reference rules.  What they add must
equal the oracle's system with the variable fields minus the oracle's system
with b = 0, c = 0 (oracle coef 1 minus coef 0): every block and every
load-vector entry, mixed degrees, polygons and polyhedra, the sin source and
the zero source, at 1e-12 of each block's largest entry.
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
    lib.host_varcoef_3d.argtypes = [V] * 24
    return lib


def _gauss01(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def _rules(dim):
    """Volume rules of degree 0..7 ((p + 2)^dim collapsed points) and face
    rules of 0..9 points per direction (Gauss on an edge, collapsed on a
    triangle), packed as [point][coordinates, weight], with their offsets."""
    vol, vol_off, vol_n = [], [], []
    for p in range(8):
        g, gw = _gauss01(p + 2)
        vol_off.append(len(vol) // (dim + 1))
        n0 = len(vol)
        for ia in range(p + 2):
            for ib in range(p + 2):
                if dim == 2:
                    a, b = g[ia], g[ib]
                    vol += [a * (1.0 - b), b, gw[ia] * gw[ib] * (1.0 - b)]
                    continue
                for ic in range(p + 2):
                    a, b, c = g[ia], g[ib], g[ic]
                    vol += [a * (1.0 - b) * (1.0 - c), b * (1.0 - c), c,
                            gw[ia] * gw[ib] * gw[ic] * (1.0 - b) * (1.0 - c) ** 2]
        vol_n.append((len(vol) - n0) // (dim + 1))
    face, face_off, face_n = [], [], []
    for n in range(10):
        face_off.append(len(face) // dim)
        n0 = len(face)
        if n > 0:
            g, gw = _gauss01(n)
            for ia in range(n):
                if dim == 2:
                    face += [g[ia], gw[ia]]
                    continue
                for ib in range(n):
                    a, b = g[ia], g[ib]
                    face += [a * (1.0 - b), b, gw[ia] * gw[ib] * (1.0 - b)]
        face_n.append((len(face) - n0) // dim)
    offs = np.array(vol_off + vol_n + face_off + face_n, np.int32)
    return np.array(vol), np.array(face), offs


def _topology(ne, faces, row_ptr, col):
    """Interfaces (element pairs, faces grouped consecutively), half faces and
    the interface of every off-diagonal block; faces are (e0, e1, ...)."""
    pairs = sorted({(f[0], f[1]) for f in faces if f[1] >= 0})
    iface = {pr: i for i, pr in enumerate(pairs)}
    order = sorted(range(len(faces)), key=lambda k: (iface.get((faces[k][0], faces[k][1]), len(pairs)), k))
    faces = [faces[k] for k in order]
    if_fptr = np.zeros(len(pairs) + 1, np.int32)
    for f in faces:
        if f[1] >= 0:
            if_fptr[iface[(f[0], f[1])] + 1] += 1
    if_fptr = np.cumsum(if_fptr).astype(np.int32)
    hf = [[] for _ in range(ne)]
    for k, f in enumerate(faces):
        hf[f[0]].append((k, 0))
        if f[1] >= 0:
            hf[f[1]].append((k, 1))
    hf_ptr = np.concatenate([[0], np.cumsum([len(h) for h in hf])]).astype(np.int32)
    hf_face = np.array([k for h in hf for k, _ in h], np.int32)
    hf_side = np.array([s for h in hf for _, s in h], np.int8)
    blk_if = np.full(col.size, -1, np.int32)
    for r in range(ne):
        for b in range(row_ptr[r], row_ptr[r + 1]):
            s = int(col[b])
            if s != r:
                blk_if[b] = iface[(min(r, s), max(r, s))]
    return faces, dict(if_fptr=if_fptr, hf_ptr=hf_ptr, hf_face=hf_face, hf_side=hf_side, blk_if=blk_if)


def _records3d(mesh, p, row_ptr, col):
    """Geometry records and face topology of a 3D mesh in the row kernels'
    layouts: the element's tetrahedra; faces in the vertex order of the lower
    element's tetrahedron, the normal out of that element."""
    ne = mesh.ne
    X = np.stack([mesh.x, mesh.y, mesh.z])
    tptr, tv = mesh.elem_tptr, np.asarray(mesh.tet_v).reshape(-1, 4)
    lo = np.zeros((3, ne))
    L = np.zeros((3, ne))
    for e in range(ne):
        P = X[:, np.unique(tv[tptr[e]:tptr[e + 1]])]
        lo[:, e] = P.min(axis=1)
        L[:, e] = P.max(axis=1) - P.min(axis=1)
    eg = np.concatenate([lo, L, 1.0 / L, (1.0 / np.sqrt(L.prod(axis=0)))[None, :]])

    def xi(x, e):
        return 2.0 * (x - lo[:, e]) / L[:, e] - 1.0

    nsub = int(tptr[-1])
    sg = np.zeros((13, nsub))
    half = {}
    for e in range(ne):
        for t in range(tptr[e], tptr[e + 1]):
            P = X[:, tv[t]]
            sg[0:3, t] = xi(P[:, 0], e)
            for i in range(1, 4):
                sg[3 * i:3 * i + 3, t] = xi(P[:, i], e) - xi(P[:, 0], e)
            sg[12, t] = abs(np.linalg.det(np.stack([P[:, 1] - P[:, 0], P[:, 2] - P[:, 0], P[:, 3] - P[:, 0]])))
            for o in range(4):
                v = [int(tv[t][i]) for i in range(4) if i != o]
                cr = np.cross(X[:, v[1]] - X[:, v[0]], X[:, v[2]] - X[:, v[0]])
                flip = float(cr @ (X[:, tv[t][o]] - X[:, v[0]])) > 0.0
                half.setdefault(tuple(sorted(v)), []).append((e, v, flip))
    faces = []
    for key in sorted(half):
        hs = sorted(half[key], key=lambda h: h[0])
        if len(hs) == 2 and hs[0][0] == hs[1][0]:
            continue  # between two tetrahedra of one element
        e0, v, flip = hs[0]
        faces.append((e0, hs[1][0] if len(hs) == 2 else -1, v, flip))
    faces, topo = _topology(ne, faces, row_ptr, col)
    nf = len(faces)
    fs = np.zeros((2, 12, nf))
    fsc = np.zeros((3, nf))
    for k, (e0, e1, v, flip) in enumerate(faces):
        P0, P1, P2 = X[:, v[0]], X[:, v[1]], X[:, v[2]]
        cr = np.cross(P1 - P0, P2 - P0)
        ln = np.linalg.norm(cr)
        n0 = (-1.0 if flip else 1.0) * cr / ln
        fsc[0, k] = ln  # 2 |F|, for the collapsed rule's weights summing to 1/2
        for s, e in enumerate((e0, e1)):
            if e < 0:
                continue
            fs[s, 0:3, k] = xi(P0, e)
            fs[s, 3:6, k] = xi(P1, e) - xi(P0, e)
            fs[s, 6:9, k] = xi(P2, e) - xi(P0, e)
            fs[s, 9:12, k] = 2.0 * n0 / L[:, e]
    f_e0 = np.array([f[0] for f in faces], np.int32)
    f_e1 = np.array([f[1] for f in faces], np.int32)
    f_nq = np.array([max(p[f[0]], p[f[1]] if f[1] >= 0 else 0) + 1 for f in faces], np.int32)
    return dict(eg=np.ascontiguousarray(eg), sg=sg, fs=fs, fsc=fsc, f_e0=f_e0, f_e1=f_e1, f_nq=f_nq, nf=nf,
                nsub=nsub, eptr=np.ascontiguousarray(tptr, np.int32), **topo)


def _records2d(mesh, p, row_ptr, col):
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


CASES = {"2d_small": (2, 12, 3, 0), "2d": (2, 30, 8, 0), "3d_small": (3, 2, 5, 4), "3d": (3, 3, 7, 9)}


@pytest.mark.parametrize("source", [0, 1])
@pytest.mark.parametrize("case", sorted(CASES))
def test_varcoef_rows_against_oracle(host, source, case):
    dim, n, seed, clusters = CASES[case]
    if dim == 2:
        mesh = mg.voronoi_square(n, seed)
        p = mg.draw_degrees(mesh.ne, seed, 1, 4).astype(np.int32)
        a = mg.draw_log_uniform(mesh.ne, seed, -1.0, 1.0)
    else:
        from paper_2007_04881_gb300 import configs

        wl = configs.small3d(n, clusters, seed, 1, 3)  # n^3 cubes of 6 tetrahedra in clusters polyhedra, p 1..3
        mesh, p, a = wl.mesh, wl.p.astype(np.int32), wl.a
    om = O.Mesh(mesh)
    info, row_ptr, col, blk_off = dg.dg_mesh_check(mesh, p, a, dg.Problem(source=source), pattern=True)
    nb = np.array([O.nbasis(dim, int(q)) for q in p])
    dof_off = np.concatenate([[0], np.cumsum(nb)]).astype(np.int64)
    if dim == 2:
        R = _records2d(mesh, p, row_ptr, col)
        R["eptr"] = np.ascontiguousarray(mesh.elem_vptr, np.int32)
    else:
        R = _records3d(mesh, p, row_ptr, col)
    vol, face, offs = _rules(dim)
    vals = np.zeros(int(info.nvals))
    rhs = np.zeros(int(info.ndofs))
    ints = np.array([om.ne, R["nf"], R["nsub"], source], np.int32)
    fn = host.host_varcoef_2d if dim == 2 else host.host_varcoef_3d
    fn(_vp(ints), _vp(p), _vp(R["eptr"]), _vp(R["eg"]), _vp(R["sg"]), _vp(R["fs"]), _vp(R["fsc"]),
       _vp(R["f_e0"]), _vp(R["f_e1"]), _vp(R["f_nq"]), _vp(R["hf_ptr"]), _vp(R["hf_face"]), _vp(R["hf_side"]),
       _vp(R["if_fptr"]), _vp(row_ptr), _vp(col), _vp(R["blk_if"]), _vp(blk_off), _vp(dof_off), _vp(vol),
       _vp(face), _vp(offs), _vp(vals), _vp(rhs))
    assert np.isfinite(vals).all() and np.isfinite(rhs).all()

    o1 = om.assemble(p, a, O.make_problem(dim, source=source, coef=1, c_sigma=10.0))
    o0 = om.assemble(p, a, O.make_problem(dim, source=source, c_sigma=10.0))

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
