"""The oracle pins have teeth: each plausible mistake planted in a copy of the
oracle source (a flipped sign, a dropped term, a transposed operand, a wrong
index or factor) makes at least one pin fail.  Runs on the CPU only."""
import importlib.util
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2007_04881_gb300 import meshgen as mg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "dg_oracle.c")

MUTATIONS = {
    "upwind_offdiag_sign": (
        "if (c == 1) t += bn * phi[1][j] * phi[0][i];",
        "if (c == 1) t -= bn * phi[1][j] * phi[0][i];",
    ),
    "dropped_symmetry_term": (
        "t -= avg * aa[r] * dn[r][i] * sgn[c] * phi[c][j]; /* {a grad v}.[w] */",
        "/* dropped */",
    ),
    "transposed_advection": (
        "bg += b[d] * grad[j * dim + d];",
        "bg += b[d] * grad[i * dim + d];",
    ),
    "legendre_derivative_index": (
        "dP[k + 1] = dP[k - 1] + (2.0 * k + 1.0) * P[k];",
        "dP[k + 1] = dP[k - 1] + (2.0 * k - 1.0) * P[k];",
    ),
    "nitsche_rhs_sign": (
        "double t = -g * (a[e] * dn - sig * phi[i]);",
        "double t = -g * (a[e] * dn + sig * phi[i]);",
    ),
    "collapsed_weight_factor": (
        "w[q] = gw[ia] * gw[ib] * (1.0 - b);",
        "w[q] = gw[ia] * gw[ib];",
    ),
    "penalty_min_instead_of_max": (
        "if (v > s) s = v;",
        "if (s == 0.0 || v < s) s = v;",
    ),
    "variable_field_sign": (
        "b[d] = 1.0 + x[d];",
        "b[d] = 1.0 - x[d];",
    ),
    "variable_coefficients_at_centroid": (
        "coef_at(pb, &xq[q * dim], b, &c);",
        "coef_at(pb, &m->cen[e * dim], b, &c);",
    ),
    "average_weight_on_boundary": (
        "double avg = bnd ? 1.0 : 0.5;",
        "double avg = 0.5;",
    ),
    "neumann_face_keeps_face_terms": (
        "if (neumann_face(m, f, pb)) return;",
        "/* dropped */",
    ),
    "neumann_data_sign": (
        "return a * g;",
        "return -a * g;",
    ),
    "neumann_side_bit": (
        "if (!(pb->neumann >> (2 * d + s) & 1)) continue;",
        "if (!(pb->neumann >> (d + 2 * s) & 1)) continue;",
    ),
    "field_table_transposed_gradient": (
        "for (int e = 0; e < pb->dim; ++e) v += pb->fbx[3 * d + e] * x[e];",
        "for (int e = 0; e < pb->dim; ++e) v += pb->fbx[3 * e + d] * x[e];",
    ),
    "neumann_data_without_a": (
        "double g = neumann_g(pb, a[e], &xq[q * dim], f->n);",
        "double g = neumann_g(pb, 1.0, &xq[q * dim], f->n);",
    ),
}


def _load_variant(tmp_path, name, old, new):
    src = open(SRC).read()
    assert old in src, f"mutation anchor missing: {name}"
    d = tmp_path / name
    (d / "_build").mkdir(parents=True)
    (d / "dg_oracle.c").write_text(src.replace(old, new, 1))
    shutil.copy(os.path.join(ROOT, "oracle", "__init__.py"), d / "__init__.py")
    spec = importlib.util.spec_from_file_location(f"oracle_mut_{name}", d / "__init__.py")
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _pins_pass(O) -> bool:
    """A compact subset of the pins; True when all of them hold."""
    try:
        # polygon moments vs divergence theorem
        mesh = mg.voronoi_square(30, 3)
        om = O.Mesh(mesh)
        for e in range(0, om.ne, 5):
            v = mesh.elem_v[mesh.elem_vptr[e]:mesh.elem_vptr[e + 1]]
            for i, j in [(0, 0), (2, 1), (3, 3)]:
                if abs(om.moment_rule(e, 4, i, j) - O.moment_divergence2d(mesh.x[v], mesh.y[v], i, j)) > 1e-13:
                    return False
        # rectangle mass / stiffness closed forms
        rm = O.Mesh(mg.rectangle_grid(1, 1, 0.0, 0.5, 0.0, 2.0))
        M = rm.volume_block(0, np.array([3]), np.array([0.0]), O.make_problem(2, c=1.0))
        if np.abs(M - np.eye(10)).max() > 1e-13:
            return False
        K = rm.volume_block(0, np.array([2]), np.array([1.0]), O.make_problem(2))
        # phi = sqrt(3/(Lx Ly)) P_1(xi): d/dx = sqrt(3/(Lx Ly)) 2/Lx; int = 3/(Lx Ly) 4/Lx^2 Lx Ly
        if abs(K[1, 1] - 3.0 * 4.0 / 0.25) > 1e-12 * 48:
            return False
        # penalty on a two-square mesh: 10 * max(a p^2 / h)
        two = O.Mesh(mg.rectangle_grid(2, 1, 0.0, 2.0, 0.0, 1.0))
        kint = [k for k in range(two.nf) if two.face_info(k)[1] >= 0][0]
        if abs(two.face_penalty(kint, np.array([1, 2]), np.array([1.0, 1.0]), 10.0) - 40 / math.sqrt(2)) > 1e-12:
            return False
        # polynomial reproduction with advection and reaction, mixed degrees
        om = O.Mesh(mg.voronoi_square(24, 7))
        p = mg.draw_degrees(om.ne, 7, 2, 3).astype(np.int32)
        a = np.full(om.ne, 0.6)
        pb = O.make_problem(2, b=(0.9, -0.5), c=0.7, source=2, poly=[1, 0.5, -1, 0.3, 0.2, -0.4])
        blk = om.assemble(p, a, pb)
        A, F, off = O.global_matrix(om, p, blk)
        U = np.linalg.solve(A, F)
        for e in range(om.ne):
            xq, _ = om.volume_points(e, 3)
            for x in xq[::7]:
                phi, _ = O.basis(2, int(p[e]), om.lo[e], om.hi[e], x)
                if abs(phi @ U[off[e]:off[e + 1]] - O.exact_u(pb, x)) > 1e-9:
                    return False
        # the coefficient fields of coef 1 through the source term ...
        pbc = O.make_problem(2, source=1, coef=1)
        x = np.array([0.3, 0.7])
        sx, cx = np.sin(np.pi * x), np.cos(np.pi * x)
        grad = np.pi * np.array([cx[0] * sx[1], sx[0] * cx[1]])
        f = 0.5 * 2 * np.pi ** 2 * sx.prod() + (1 + x) @ grad + (3 + x.prod()) * sx.prod()
        if abs(O.source_f(pbc, 0.5, x) - f) > 1e-12 * abs(f):
            return False
        # ... and polynomial reproduction with them
        om = O.Mesh(mg.voronoi_square(24, 9))
        p = np.full(om.ne, 2, dtype=np.int32)
        a = np.full(om.ne, 0.5)
        pb = O.make_problem(2, source=2, poly=[1, 0.5, -1, 0.3, 0.2, -0.4], coef=1)
        blk = om.assemble(p, a, pb)
        A, F, off = O.global_matrix(om, p, blk)
        U = np.linalg.solve(A, F)
        for e in range(om.ne):
            xq, _ = om.volume_points(e, 3)
            for x in xq[::7]:
                phi, _ = O.basis(2, 2, om.lo[e], om.hi[e], x)
                if abs(phi @ U[off[e]:off[e + 1]] - O.exact_u(pb, x)) > 1e-9:
                    return False
        # Neumann sides: the constant in the kernel of pure diffusion with the
        # whole boundary Neumann; with x = max Dirichlet, B 1 nonzero exactly
        # on the elements with a face there
        mesh = mg.voronoi_square(24, 11)
        om = O.Mesh(mesh)
        p = mg.draw_degrees(om.ne, 11, 1, 3).astype(np.int32)
        a = mg.draw_log_uniform(om.ne, 11, -1, 1)
        c1 = np.concatenate([np.eye(O.nbasis(2, int(p[e])))[0] * math.sqrt(np.prod(om.hi[e] - om.lo[e]))
                             for e in range(om.ne)])
        for mask in (0b1111, 0b1101):
            A, _, off = O.global_matrix(om, p, om.assemble(p, a, O.make_problem(2, neumann=mask)))
            r = A @ c1
            s = np.abs(A).max()
            xmax = np.asarray(mesh.x).max()
            for e in range(om.ne):
                loop = mesh.elem_v[mesh.elem_vptr[e]:mesh.elem_vptr[e + 1]]
                on = mask == 0b1101 and any(mesh.x[loop[i]] == xmax and mesh.x[loop[(i + 1) % len(loop)]] == xmax
                                            for i in range(len(loop)))
                re = np.abs(r[off[e]:off[e + 1]]).max()
                if (re > 1e-8 * s) != on:
                    return False
        # ... and reproduction with outflow sides Neumann, a != 1
        om = O.Mesh(mg.voronoi_square(24, 7))
        p = mg.draw_degrees(om.ne, 7, 2, 3).astype(np.int32)
        a = np.full(om.ne, 0.6)
        pb = O.make_problem(2, b=(0.9, 0.5), c=0.7, source=2, poly=[1, 0.5, -1, 0.3, 0.2, -0.4], neumann=0b1010)
        A, F, off = O.global_matrix(om, p, om.assemble(p, a, pb))
        U = np.linalg.solve(A, F)
        for e in range(om.ne):
            xq, _ = om.volume_points(e, 3)
            for x in xq[::7]:
                phi, _ = O.basis(2, int(p[e]), om.lo[e], om.hi[e], x)
                if abs(phi @ U[off[e]:off[e + 1]] - O.exact_u(pb, x)) > 1e-9:
                    return False
        # a table of fields (affine b with a non-symmetric gradient, quadratic c)
        # through the source term
        b0, B, cc = np.array([0.3, -0.2, 0.0]), np.array([[0.4, -0.7, 0], [0.2, 0.1, 0], [0, 0, 0]]), np.zeros(20)
        cc[:6] = [1.0, 0.2, -0.5, 0.3, 0.7, -0.1]
        pbt = O.make_problem(2, source=1, fields=(b0, B, cc))
        x = np.array([0.3, 0.7])
        sx, cx = np.sin(np.pi * x), np.cos(np.pi * x)
        grad = np.pi * np.array([cx[0] * sx[1], sx[0] * cx[1]])
        bb = b0[:2] + B[:2, :2] @ x
        c = cc[0] + cc[1] * x[0] + cc[2] * x[1] + cc[3] * x[0] ** 2 + cc[4] * x[0] * x[1] + cc[5] * x[1] ** 2
        f = 0.5 * 2 * np.pi ** 2 * sx.prod() + bb @ grad + c * sx.prod()
        if abs(O.source_f(pbt, 0.5, x) - f) > 1e-12 * abs(f):
            return False
        return True
    except Exception:
        return False


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_unmutated_copy_passes(tmp_path):
    O = _load_variant(tmp_path, "none", "#define ORC_PI", "#define ORC_PI")
    assert _pins_pass(O)


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutation_is_caught(tmp_path, name):
    old, new = MUTATIONS[name]
    O = _load_variant(tmp_path, name, old, new)
    assert not _pins_pass(O), f"planted mistake '{name}' passed every pin"
