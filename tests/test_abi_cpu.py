"""CPU-only checks of the C ABI: the library loads, exports every symbol that
include/dg.h declares, fails loudly without a GPU, and its host-side mesh
logic (validation, faces, interfaces, block-sparse pattern) is right."""
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_2007_04881_gb300 import build as B
from paper_2007_04881_gb300 import configs, dg, meshgen as mg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return dg.load()


def test_exports_every_declared_symbol(lib):
    hdr = open(os.path.join(ROOT, "include", "dg.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    declared = set(re.findall(r"\b(dg_[a-z_0-9]+)\s*\(", hdr))
    assert declared, "no declarations parsed"
    missing = [s for s in sorted(declared) if not hasattr(lib, s)]
    assert not missing, missing
    assert declared == set(dg.EXPORTS)


def test_create_fails_loudly_without_gpu(lib):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(dg.DGError) as ei:
        dg.Context(0)
    assert ei.value.code in (-1, -3)


def test_pipelined_host_calls_reject_null_arguments(lib):
    """dg_assemble_host_submit / _wait check their arguments before any CUDA
    call: a null context, mesh, output or ticket pointer is DG_ERR_ARG, with
    the message naming the call."""
    import ctypes as C

    t = C.c_longlong(-7)
    assert lib.dg_assemble_host_submit(None, None, dg.DG_PREC_FP32, None, None, None, None, None, None,
                                       C.byref(t)) == dg.DG_ERR_ARG
    assert "dg_assemble_host_submit" in lib.dg_last_error().decode()
    assert t.value == -7  # no ticket issued
    assert lib.dg_assemble_host_submit(None, None, dg.DG_PREC_FP32, None, None, None, None, None, None,
                                       None) == dg.DG_ERR_ARG
    assert lib.dg_assemble_host_wait(None, None, C.c_longlong(0)) == dg.DG_ERR_ARG
    assert "dg_assemble_host_wait" in lib.dg_last_error().decode()


def _check(wl):
    return dg.dg_mesh_check(wl.mesh, wl.p, wl.a, dg.Problem(**wl.problem), pattern=True)


@pytest.mark.parametrize("dim", [2, 3])
def test_pattern_matches_oracle_topology(lib, dim):
    wl = configs.small2d(150, 3, 1, 6) if dim == 2 else configs.small3d(4, 12, 5, 1, 4)
    info, row_ptr, col, blk_off = _check(wl)
    om = O.Mesh(wl.mesh)
    assert info.ne == om.ne
    assert info.ninterfaces == om.ni
    assert info.nfaces == om.nf
    assert info.nbfaces == om.nbf
    assert info.nnzb == om.ne + 2 * om.ni
    nb = np.array([O.nbasis(dim, int(q)) for q in wl.p])
    # rows: self + neighbours from the oracle's interfaces, ascending
    nbr = [set([e]) for e in range(om.ne)]
    for e0, e1 in zip(om.if_e0, om.if_e1):
        nbr[e0].add(int(e1))
        nbr[e1].add(int(e0))
    for r in range(om.ne):
        assert list(col[row_ptr[r]:row_ptr[r + 1]]) == sorted(nbr[r])
    sizes = np.array([nb[r] * nb[c] for r in range(om.ne) for c in col[row_ptr[r]:row_ptr[r + 1]]])
    assert np.array_equal(np.diff(blk_off), sizes)
    assert info.nvals == sizes.sum()
    assert info.ndofs == nb.sum()
    # quadrature point counts
    qt = (wl.p.astype(np.int64) + 2) ** dim
    nsub = np.diff(wl.mesh.elem_vptr if dim == 2 else wl.mesh.elem_tptr)
    assert info.nqvol == int((nsub * qt).sum())


def _desc_case(kind):
    m = mg.voronoi_square(20, 4)
    p = np.full(m.ne, 2, np.int8)
    a = np.ones(m.ne)
    pb = dict(b=(0.0, 0.0, 0.0), c=0.0, source=0, poly=[], c_sigma=10.0)
    if kind == "cw_loop":
        v = m.elem_v.copy()
        s, e = m.elem_vptr[3], m.elem_vptr[4]
        v[s:e] = v[s:e][::-1]
        m = mg.Mesh2D(m.x, m.y, m.elem_vptr, v)
    elif kind == "index_range":
        v = m.elem_v.copy()
        v[5] = m.nv + 3
        m = mg.Mesh2D(m.x, m.y, m.elem_vptr, v)
    elif kind == "p_range":
        p[2] = 9
    elif kind == "p_zero":
        p[2] = 0
    elif kind == "a_nonpositive":
        a[1] = 0.0
    elif kind == "c_negative":
        pb["c"] = -1.0
    elif kind == "sigma":
        pb["c_sigma"] = 0.0
    elif kind == "duplicate_element":
        # the same polygon twice: every edge is seen by three loops or twice in one direction
        ptr = np.concatenate([m.elem_vptr, [m.elem_vptr[-1] + (m.elem_vptr[1] - m.elem_vptr[0])]]).astype(np.int32)
        v = np.concatenate([m.elem_v, m.elem_v[m.elem_vptr[0]:m.elem_vptr[1]]]).astype(np.int32)
        m = mg.Mesh2D(m.x, m.y, ptr, v)
        p = np.full(m.ne, 2, np.int8)
        a = np.ones(m.ne)
    return m, p, a, pb


@pytest.mark.parametrize(
    "kind,code",
    [("cw_loop", -2), ("index_range", -2), ("p_range", -2), ("p_zero", -2), ("a_nonpositive", -2),
     ("c_negative", -2), ("sigma", -2), ("duplicate_element", -2)],
)
def test_invalid_meshes_rejected(lib, kind, code):
    m, p, a, pb = _desc_case(kind)
    with pytest.raises(dg.DGError) as ei:
        dg.dg_mesh_check(m, p, a, dg.Problem(**pb))
    assert ei.value.code == code


def test_nonmanifold_3d_rejected(lib):
    # three tetrahedra sharing one triangle
    x = np.array([0.0, 1.0, 0.0, 0.3, 0.3, -0.2])
    y = np.array([0.0, 0.0, 1.0, 0.3, 0.2, 0.5])
    z = np.array([0.0, 0.0, 0.0, 1.0, -1.0, 0.7])
    tets = np.array([0, 1, 2, 3, 0, 1, 2, 4, 0, 1, 2, 5], np.int32)
    m = mg.Mesh3D(x, y, z, np.array([0, 1, 2, 3], np.int32), tets)
    with pytest.raises(dg.DGError) as ei:
        dg.dg_mesh_check(m, np.ones(3, np.int8), np.ones(3), dg.Problem())
    assert ei.value.code == -2


def test_single_element_and_rectangles(lib):
    m = mg.rectangle_grid(1, 1)
    info = dg.dg_mesh_check(m, np.array([3], np.int8), np.ones(1), dg.Problem())
    assert info.nnzb == 1 and info.ninterfaces == 0 and info.nbfaces == 4
    m = mg.rectangle_grid(3, 2)
    info = dg.dg_mesh_check(m, np.full(6, 1, np.int8), np.ones(6), dg.Problem())
    assert info.ninterfaces == 7 and info.nbfaces == 10 and info.nnzb == 6 + 14


def test_empty_and_degenerate_inputs_rejected(lib):
    # no elements
    m = mg.Mesh2D(np.zeros(3), np.zeros(3), np.zeros(1, np.int32), np.zeros(0, np.int32))
    with pytest.raises(dg.DGError) as ei:
        dg.dg_mesh_check(m, np.zeros(0, np.int8), np.zeros(0), dg.Problem())
    assert ei.value.code == -1
    # a flat tetrahedron (zero volume)
    x = np.array([0.0, 1.0, 0.0, 0.5])
    y = np.array([0.0, 0.0, 1.0, 0.5])
    z = np.zeros(4)
    m = mg.Mesh3D(x, y, z, np.array([0, 1], np.int32), np.array([0, 1, 2, 3], np.int32))
    with pytest.raises(dg.DGError) as ei:
        dg.dg_mesh_check(m, np.ones(1, np.int8), np.ones(1), dg.Problem())
    assert ei.value.code == -2
    # a polygon with two vertices
    m = mg.Mesh2D(np.array([0.0, 1.0]), np.array([0.0, 0.0]), np.array([0, 2], np.int32), np.array([0, 1], np.int32))
    with pytest.raises(dg.DGError) as ei:
        dg.dg_mesh_check(m, np.ones(1, np.int8), np.ones(1), dg.Problem())
    assert ei.value.code == -2


def test_precision_flags_match_header(lib):
    # the precision flags of include/dg.h: FP64, FP32, split-BF16, 3xTF32
    assert (dg.DG_PREC_FP64, dg.DG_PREC_FP32, dg.DG_PREC_BF16X3, dg.DG_PREC_TF32X3) == (0, 1, 2, 3)
    hdr = open(os.path.join(os.path.dirname(__file__), "..", "include", "dg.h")).read()
    for name, val in (("DG_PREC_BF16X3", 2), ("DG_PREC_TF32X3", 3)):
        assert f"#define {name} {val}" in hdr


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("space", [dg.DG_SPACE_P, dg.DG_SPACE_PQ])
def test_slab_offsets(lib, dim, space):
    """Space-time slab layout (host only): a prism of degree p has
    C(p + dim + 1, dim + 1) dofs in P and (p + 1) C(p + dim, dim) in PQ; 2D
    dof offsets equal the slab oracle's, and block (r, s) holds nt_r nt_s."""
    import math

    wl = configs.small2d(150, 3, 1, 6) if dim == 2 else configs.small3d(4, 12, 5, 1, 4)
    info, row_ptr, col, _ = _check(wl)
    p = wl.p.astype(np.int32)
    blk_off, dof_off = dg.dg_slab_offsets(dim, row_ptr, col, p, space)
    nt = np.array([math.comb(int(q) + dim + 1, dim + 1) if space == dg.DG_SPACE_P
                   else (int(q) + 1) * math.comb(int(q) + dim, dim) for q in p])
    assert np.array_equal(np.diff(dof_off), nt)
    sizes = [nt[r] * nt[c] for r in range(info.ne) for c in col[row_ptr[r]:row_ptr[r + 1]]]
    assert np.array_equal(np.diff(blk_off), sizes) and blk_off[0] == 0
    if dim == 2:
        from oracle import spacetime as S

        sl = S.Slab(O.Mesh(wl.mesh), p, wl.a, (0.0, 0.0), 0.0, "P" if space == dg.DG_SPACE_P else "PQ", 0.0, 1.0)
        assert np.array_equal(dof_off, sl.off)


def test_slab_offsets_rejects_bad_input(lib):
    wl = configs.small2d(40, 3, 1, 3)
    _, row_ptr, col, _ = _check(wl)
    p = wl.p.astype(np.int32)
    for bad in (dict(dim=4), dict(space=2), dict(p=np.where(np.arange(p.size) == 3, 0, p)),
                dict(p=np.where(np.arange(p.size) == 3, 7, p)), dict(col=np.where(np.arange(col.size) == 5, p.size, col))):
        kw = dict(dim=2, row_ptr=row_ptr, col=col, p=p, space=dg.DG_SPACE_P)
        kw.update(bad)
        with pytest.raises(dg.DGError) as ei:
            dg.dg_slab_offsets(**kw)
        assert ei.value.code == -1
