"""Shared helpers of the parity tests: run the oracle and the CUDA library on
the same workload and compare block by block."""
from __future__ import annotations

import numpy as np

import oracle as O
from paper_2007_04881_gb300 import dg


def oracle_problem(wl):
    pb = wl.problem
    return O.make_problem(wl.dim, b=pb["b"], c=pb["c"], source=pb["source"], poly=pb["poly"], c_sigma=pb["c_sigma"],
                          coef=pb.get("coef", 0), neumann=pb.get("neumann", 0))


def dg_problem(wl):
    pb = wl.problem
    return dg.Problem(b=pb["b"], c=pb["c"], source=pb["source"], poly=pb["poly"], c_sigma=pb["c_sigma"],
                      neumann=pb.get("neumann", 0))


def oracle_blocks(wl, elems=None, ifaces=None, om=None, rhs=True):
    om = om or O.Mesh(wl.mesh)
    return om, om.assemble(wl.p.astype(np.int32), wl.a, oracle_problem(wl), elems=elems, ifaces=ifaces, rhs=rhs)


def rel_block_err(got, ref):
    """max |got - ref| / max |ref| over one block (block max-norm relative)."""
    s = np.abs(ref).max()
    if s == 0:
        return float(np.abs(got).max())
    return float(np.abs(got - ref).max() / s)


def compare(gpu, om, ob, wl):
    """Largest block-relative error over the diagonal blocks, off-diagonal
    blocks and per-element load vectors present in the oracle result."""
    ed = eo = er = 0.0
    for k, e in enumerate(ob["elems"]):
        ed = max(ed, rel_block_err(gpu["diag"][int(e)], ob["diag"][k]))
        if "rhs" in ob and "rhs" in gpu:
            er = max(er, rel_block_err(gpu["rhs"][int(e)], ob["rhs"][k]))
    for k, i in enumerate(ob["ifaces"]):
        e0, e1 = int(om.if_e0[i]), int(om.if_e1[i])
        eo = max(eo, rel_block_err(gpu["off"][(e0, e1)], ob["a01"][k]))
        eo = max(eo, rel_block_err(gpu["off"][(e1, e0)], ob["a10"][k]))
    return ed, eo, er


def polygon_workload(nvert: int, p: int, b=(1.0, -0.5), c: float = 1.5):
    """One convex element: the regular nvert-gon of radius 0.4 about
    (0.5, 0.5), counter-clockwise, every edge a boundary face.  A loop longer
    than 16 vertices takes the kernels' runtime-length paths."""
    from paper_2007_04881_gb300 import configs, meshgen

    t = 2.0 * np.pi * np.arange(nvert) / nvert
    mesh = meshgen.Mesh2D(x=0.5 + 0.4 * np.cos(t), y=0.5 + 0.4 * np.sin(t),
                          elem_vptr=np.array([0, nvert], dtype=np.int32),
                          elem_v=np.arange(nvert, dtype=np.int32))
    return configs.Workload(name=f"polygon_{nvert}", mesh=mesh, p=np.array([p], dtype=np.int8),
                            a=np.array([0.7]), problem=dict(b=(b[0], b[1], 0.0), c=c,
                                                            source=configs.SRC_SINPROD, poly=[],
                                                            c_sigma=10.0))
