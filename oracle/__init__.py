"""FP64 CPU oracle for SIPG dG assembly on polytopic meshes (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library: the arithmetic lives in ``dg_oracle.c`` (plain loops, FP64), and this
module only loads it with ``ctypes`` and marshals arrays.

Layout of results (independent of the library's block-sparse layout):
  * ``diag[e]``: n_e x n_e diagonal block of element e (volume + its faces),
  * interfaces ``(e0, e1)`` with e0 < e1, sorted; ``a01[k]`` (n_e0 x n_e1, test
    functions of e0, trial functions of e1) and ``a10[k]`` (n_e1 x n_e0),
  * ``rhs[e]``: the n_e load-vector entries of element e.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dg_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile dg_oracle.c into oracle/_build/liboracle.so (gcc -O3, OpenMP).

    -std=c11 (ISO C) keeps floating-point contraction off, so the results are
    the same on every host; no -march flag, for the same reason."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if not force and os.path.exists(_OUT) and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC):
        return _OUT
    tmp = _OUT + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O3", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _OUT)
    return _OUT


class _Problem(C.Structure):
    _fields_ = [
        ("dim", C.c_int),
        ("b", C.c_double * 3),
        ("c", C.c_double),
        ("source", C.c_int),
        ("poly", C.c_double * 20),
        ("c_sigma", C.c_double),
        ("coef", C.c_int),
        ("neumann", C.c_int),
        ("fb0", C.c_double * 3),
        ("fbx", C.c_double * 9),
        ("fc", C.c_double * 20),
    ]


_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)
_L = C.POINTER(C.c_int64)


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        lib.orc_gauss01.argtypes = [C.c_int, _D, _D]
        lib.orc_tri_rule.argtypes = [C.c_int, _D, _D, _D]
        lib.orc_tri_rule.restype = C.c_int
        lib.orc_tet_rule.argtypes = [C.c_int, _D, _D, _D, _D]
        lib.orc_tet_rule.restype = C.c_int
        lib.orc_nbasis.argtypes = [C.c_int, C.c_int]
        lib.orc_nbasis.restype = C.c_int
        lib.orc_basis_alpha.argtypes = [C.c_int, C.c_int, _I]
        lib.orc_basis.argtypes = [C.c_int, C.c_int, _D, _D, _D, _D, _D]
        lib.orc_mesh_new.argtypes = [C.c_int, C.c_int, _D, _D, _D, C.c_int, _I, _I]
        lib.orc_mesh_new.restype = C.c_void_p
        lib.orc_mesh_free.argtypes = [C.c_void_p]
        for f in ("orc_num_interfaces", "orc_num_faces", "orc_num_boundary_faces"):
            getattr(lib, f).argtypes = [C.c_void_p]
            getattr(lib, f).restype = C.c_int
        lib.orc_interfaces.argtypes = [C.c_void_p, _I, _I, _I]
        lib.orc_geometry.argtypes = [C.c_void_p, _D, _D, _D, _D, _D]
        lib.orc_volume_points.argtypes = [C.c_void_p, C.c_int, C.c_int, _D, _D]
        lib.orc_volume_points.restype = C.c_int
        lib.orc_volume_point_count.argtypes = [C.c_void_p, C.c_int, C.c_int]
        lib.orc_volume_point_count.restype = C.c_int
        lib.orc_face_penalty.argtypes = [C.c_void_p, C.c_int, _I, _D, C.c_double]
        lib.orc_face_penalty.restype = C.c_double
        lib.orc_diag_block.argtypes = [C.c_void_p, C.c_int, _I, _D, C.POINTER(_Problem), _D]
        lib.orc_offdiag_blocks.argtypes = [C.c_void_p, C.c_int, _I, _D, C.POINTER(_Problem), _D, _D]
        lib.orc_rhs_element.argtypes = [C.c_void_p, C.c_int, _I, _D, C.POINTER(_Problem), _D]
        lib.orc_assemble.argtypes = [
            C.c_void_p, _I, _D, C.POINTER(_Problem), C.c_int, _I, _D, _L, _D, _L,
            C.c_int, _I, _D, _D, _L, C.c_int,
        ]
        lib.orc_max_threads.restype = C.c_int
        lib.orc_moment_rule.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int]
        lib.orc_moment_rule.restype = C.c_double
        lib.orc_moment_divergence2d.argtypes = [C.c_int, _D, _D, C.c_int, C.c_int]
        lib.orc_moment_divergence2d.restype = C.c_double
        lib.orc_moment_divergence3d.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int]
        lib.orc_moment_divergence3d.restype = C.c_double
        lib.orc_volume_block.argtypes = [C.c_void_p, C.c_int, _I, _D, C.POINTER(_Problem), _D]
        lib.orc_face_info.argtypes = [C.c_void_p, C.c_int, _I, _I, _D, _D]
        lib.orc_face_points.argtypes = [C.c_void_p, C.c_int, C.c_int, _D, _D]
        lib.orc_face_points.restype = C.c_int
        lib.orc_face_blocks.argtypes = [C.c_void_p, C.c_int, _I, _D, C.POINTER(_Problem), _D, _D, _D, _D]
        lib.orc_exact_u.argtypes = [C.POINTER(_Problem), _D]
        lib.orc_exact_u.restype = C.c_double
        lib.orc_source_f.argtypes = [C.POINTER(_Problem), C.c_double, _D]
        lib.orc_source_f.restype = C.c_double
        _lib = lib
        return lib


def _dp(a):
    return a.ctypes.data_as(_D)


def _ip(a):
    return a.ctypes.data_as(_I)


def _lp(a):
    return a.ctypes.data_as(_L)


def nbasis(dim: int, p: int) -> int:
    return _load().orc_nbasis(dim, p)


def basis_alpha(dim: int, p: int) -> np.ndarray:
    n = nbasis(dim, p)
    out = np.zeros(3 * n, dtype=np.int32)
    _load().orc_basis_alpha(dim, p, _ip(out))
    return out.reshape(n, 3)[:, :dim]


def gauss01(n: int):
    x = np.zeros(n)
    w = np.zeros(n)
    _load().orc_gauss01(n, _dp(x), _dp(w))
    return x, w


def tri_rule(n: int):
    r, s, w = (np.zeros(n * n) for _ in range(3))
    _load().orc_tri_rule(n, _dp(r), _dp(s), _dp(w))
    return r, s, w


def tet_rule(n: int):
    r, s, t, w = (np.zeros(n ** 3) for _ in range(4))
    _load().orc_tet_rule(n, _dp(r), _dp(s), _dp(t), _dp(w))
    return r, s, t, w


def basis(dim: int, p: int, lo, hi, x):
    """Physical-frame basis values [n] and gradients [n, dim] at point x."""
    n = nbasis(dim, p)
    lo = np.ascontiguousarray(lo, dtype=np.float64)
    hi = np.ascontiguousarray(hi, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    phi = np.zeros(n)
    grad = np.zeros(n * dim)
    _load().orc_basis(dim, p, _dp(lo), _dp(hi), _dp(x), _dp(phi), _dp(grad))
    return phi, grad.reshape(n, dim)


def make_problem(dim, b=(0.0, 0.0, 0.0), c=0.0, source=0, poly=None, c_sigma=10.0, coef=0, neumann=0,
                 fields=None) -> _Problem:
    """coef 0: constant b and c; coef 1: the fields b_d = 1 + x_d, c = 3 + prod x_d of
    the paper's 3D advection-diffusion-reaction test (Sec. 4.2).  fields =
    (b0[3], bx[3][3], c[20]) sets coef 2: b_d = b0[d] + sum_e bx[d][e] x_e and c
    the polynomial with coefficients c on the graded monomials of poly.
    neumann: bit 2d + s marks the side x_d = min (s = 0) / max (s = 1) of the
    vertices' bounding box as Neumann boundary (Eq. (2.2)); the rest is
    Dirichlet."""
    pb = _Problem()
    pb.dim = dim
    for i in range(3):
        pb.b[i] = float(b[i]) if i < len(b) else 0.0
    pb.c = float(c)
    pb.source = int(source)
    poly = [] if poly is None else list(poly)
    for i in range(20):
        pb.poly[i] = float(poly[i]) if i < len(poly) else 0.0
    pb.c_sigma = float(c_sigma)
    pb.coef = int(coef)
    pb.neumann = int(neumann)
    if fields is not None:
        b0, bx, cc = fields
        pb.coef = 2
        bx = np.asarray(bx, dtype=np.float64).reshape(3, 3)
        for i in range(3):
            pb.fb0[i] = float(b0[i]) if i < len(b0) else 0.0
            for j in range(3):
                pb.fbx[3 * i + j] = float(bx[i, j])
        for i in range(20):
            pb.fc[i] = float(cc[i]) if i < len(cc) else 0.0
    return pb


def exact_u(pb: _Problem, x) -> float:
    x = np.ascontiguousarray(x, dtype=np.float64)
    return _load().orc_exact_u(C.byref(pb), _dp(x))


def source_f(pb: _Problem, a: float, x) -> float:
    """f = -a Lap u + b . grad u + c u at x, with b and c the problem's fields there."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    return _load().orc_source_f(C.byref(pb), float(a), _dp(x))


class Mesh:
    """Oracle-side mesh: geometry, faces and interfaces built in C."""

    def __init__(self, mesh):
        lib = _load()
        self.dim = mesh.dim
        self._keep = []
        x = np.ascontiguousarray(mesh.x, dtype=np.float64)
        y = np.ascontiguousarray(mesh.y, dtype=np.float64)
        if self.dim == 2:
            z = np.zeros(1)
            eptr = np.ascontiguousarray(mesh.elem_vptr, dtype=np.int32)
            ev = np.ascontiguousarray(mesh.elem_v, dtype=np.int32)
        else:
            z = np.ascontiguousarray(mesh.z, dtype=np.float64)
            eptr = np.ascontiguousarray(mesh.elem_tptr, dtype=np.int32)
            ev = np.ascontiguousarray(mesh.tet_v, dtype=np.int32)
        self.ne = int(eptr.shape[0] - 1)
        self.nv = int(x.shape[0])
        h = lib.orc_mesh_new(self.dim, self.nv, _dp(x), _dp(y), _dp(z), self.ne, _ip(eptr), _ip(ev))
        if not h:
            raise ValueError("oracle: non-manifold mesh")
        self._h = C.c_void_p(h)
        self.ni = lib.orc_num_interfaces(self._h)
        self.nf = lib.orc_num_faces(self._h)
        self.nbf = lib.orc_num_boundary_faces(self._h)
        e0 = np.zeros(self.ni, dtype=np.int32)
        e1 = np.zeros(self.ni, dtype=np.int32)
        nfc = np.zeros(self.ni, dtype=np.int32)
        lib.orc_interfaces(self._h, _ip(e0), _ip(e1), _ip(nfc))
        self.if_e0, self.if_e1, self.if_nfaces = e0, e1, nfc
        d = self.dim
        self.vol = np.zeros(self.ne)
        self.cen = np.zeros(self.ne * d)
        self.lo = np.zeros(self.ne * d)
        self.hi = np.zeros(self.ne * d)
        self.h = np.zeros(self.ne)
        lib.orc_geometry(self._h, _dp(self.vol), _dp(self.cen), _dp(self.lo), _dp(self.hi), _dp(self.h))
        self.cen = self.cen.reshape(self.ne, d)
        self.lo = self.lo.reshape(self.ne, d)
        self.hi = self.hi.reshape(self.ne, d)

    def __del__(self):
        try:
            if getattr(self, "_h", None):
                _load().orc_mesh_free(self._h)
                self._h = None
        except Exception:
            pass

    def volume_points(self, e: int, n: int):
        cap = _load().orc_volume_point_count(self._h, int(e), int(n))
        xq = np.zeros(cap * self.dim)
        wq = np.zeros(cap)
        q = _load().orc_volume_points(self._h, int(e), int(n), _dp(xq), _dp(wq))
        return xq[: q * self.dim].reshape(q, self.dim), wq[:q]

    def moment_rule(self, e: int, n: int, i: int, j: int, k: int = 0) -> float:
        return _load().orc_moment_rule(self._h, int(e), int(n), int(i), int(j), int(k))

    def moment_divergence3d(self, e: int, i: int, j: int, k: int) -> float:
        """int_e x^i y^j z^k by the divergence theorem over the element's boundary triangles."""
        return _load().orc_moment_divergence3d(self._h, int(e), int(i), int(j), int(k))

    def assemble(self, p, a, pb: _Problem, elems=None, ifaces=None, rhs=True, diag=True, nthreads=0):
        """Oracle blocks for the listed elements (default all) and interfaces."""
        lib = _load()
        p = np.ascontiguousarray(p, dtype=np.int32)
        a = np.ascontiguousarray(a, dtype=np.float64)
        elems = np.arange(self.ne, dtype=np.int32) if elems is None else np.ascontiguousarray(elems, dtype=np.int32)
        ifaces = np.arange(self.ni, dtype=np.int32) if ifaces is None else np.ascontiguousarray(ifaces, dtype=np.int32)
        nb = np.array([nbasis(self.dim, int(q)) for q in range(0, 16)])
        ne_l = nb[p[elems]]
        doff = np.zeros(elems.size + 1, dtype=np.int64)
        doff[1:] = np.cumsum(ne_l.astype(np.int64) ** 2)
        roff = np.zeros(elems.size + 1, dtype=np.int64)
        roff[1:] = np.cumsum(ne_l)
        n0 = nb[p[self.if_e0[ifaces]]].astype(np.int64)
        n1 = nb[p[self.if_e1[ifaces]]].astype(np.int64)
        ooff = np.zeros(ifaces.size + 1, dtype=np.int64)
        ooff[1:] = np.cumsum(n0 * n1)
        dbuf = np.zeros(max(int(doff[-1]), 1))
        rbuf = np.zeros(max(int(roff[-1]), 1))
        b01 = np.zeros(max(int(ooff[-1]), 1))
        b10 = np.zeros(max(int(ooff[-1]), 1))
        lib.orc_assemble(
            self._h, _ip(p), _dp(a), C.byref(pb), int(elems.size), _ip(elems),
            _dp(dbuf) if diag else None, _lp(doff), _dp(rbuf) if rhs else None, _lp(roff),
            int(ifaces.size), _ip(ifaces), _dp(b01), _dp(b10), _lp(ooff), int(nthreads),
        )
        out = {"elems": elems, "ifaces": ifaces}
        if diag:
            out["diag"] = [dbuf[doff[k]:doff[k + 1]].reshape(ne_l[k], ne_l[k]) for k in range(elems.size)]
        if rhs:
            out["rhs"] = [rbuf[roff[k]:roff[k + 1]].copy() for k in range(elems.size)]
        out["a01"] = [b01[ooff[k]:ooff[k + 1]].reshape(n0[k], n1[k]) for k in range(ifaces.size)]
        out["a10"] = [b10[ooff[k]:ooff[k + 1]].reshape(n1[k], n0[k]) for k in range(ifaces.size)]
        return out

    def volume_block(self, e: int, p, a, pb: _Problem):
        p = np.ascontiguousarray(p, dtype=np.int32)
        a = np.ascontiguousarray(a, dtype=np.float64)
        n = nbasis(self.dim, int(p[e]))
        out = np.zeros(n * n)
        _load().orc_volume_block(self._h, int(e), _ip(p), _dp(a), C.byref(pb), _dp(out))
        return out.reshape(n, n)

    def face_info(self, k: int):
        e0 = C.c_int()
        e1 = C.c_int()
        area = np.zeros(1)
        nrm = np.zeros(3)
        _load().orc_face_info(self._h, int(k), C.byref(e0), C.byref(e1), _dp(area), _dp(nrm))
        return e0.value, e1.value, float(area[0]), nrm[: self.dim].copy()

    def face_points(self, k: int, n: int):
        """The n-point rule of face k: points [q][dim] and weights (with the face
        measure)."""
        xq = np.zeros(n * n * 3)
        wq = np.zeros(n * n)
        q = _load().orc_face_points(self._h, int(k), int(n), _dp(xq), _dp(wq))
        return xq[: q * self.dim].reshape(q, self.dim), wq[:q]

    def face_blocks(self, k: int, p, a, pb: _Problem):
        p = np.ascontiguousarray(p, dtype=np.int32)
        a = np.ascontiguousarray(a, dtype=np.float64)
        e0, e1, _, _ = self.face_info(k)
        n0 = nbasis(self.dim, int(p[e0]))
        n1 = nbasis(self.dim, int(p[e1])) if e1 >= 0 else 0
        b00, b01, b10, b11 = np.zeros(n0 * n0), np.zeros(max(n0 * n1, 1)), np.zeros(max(n0 * n1, 1)), np.zeros(max(n1 * n1, 1))
        _load().orc_face_blocks(self._h, int(k), _ip(p), _dp(a), C.byref(pb), _dp(b00), _dp(b01), _dp(b10), _dp(b11))
        out = {"b00": b00.reshape(n0, n0)}
        if e1 >= 0:
            out.update(b01=b01[: n0 * n1].reshape(n0, n1), b10=b10[: n0 * n1].reshape(n1, n0), b11=b11[: n1 * n1].reshape(n1, n1))
        return out

    def face_penalty(self, face: int, p, a, c_sigma: float) -> float:
        p = np.ascontiguousarray(p, dtype=np.int32)
        a = np.ascontiguousarray(a, dtype=np.float64)
        return _load().orc_face_penalty(self._h, int(face), _ip(p), _dp(a), float(c_sigma))


def moment_divergence2d(xs, ys, i: int, j: int) -> float:
    xs = np.ascontiguousarray(xs, dtype=np.float64)
    ys = np.ascontiguousarray(ys, dtype=np.float64)
    return _load().orc_moment_divergence2d(int(xs.size), _dp(xs), _dp(ys), int(i), int(j))


def max_threads() -> int:
    return _load().orc_max_threads()


def global_matrix(om: Mesh, p, blocks):
    """Dense global matrix from oracle blocks (small meshes; for solves)."""
    nb = np.array([nbasis(om.dim, int(q)) for q in p])
    off = np.zeros(om.ne + 1, dtype=np.int64)
    off[1:] = np.cumsum(nb)
    N = int(off[-1])
    A = np.zeros((N, N))
    for k, e in enumerate(blocks["elems"]):
        A[off[e]:off[e + 1], off[e]:off[e + 1]] = blocks["diag"][k]
    for k, i in enumerate(blocks["ifaces"]):
        e0, e1 = om.if_e0[i], om.if_e1[i]
        A[off[e0]:off[e0 + 1], off[e1]:off[e1 + 1]] = blocks["a01"][k]
        A[off[e1]:off[e1 + 1], off[e0]:off[e0 + 1]] = blocks["a10"][k]
    F = None
    if "rhs" in blocks:
        F = np.zeros(N)
        for k, e in enumerate(blocks["elems"]):
            F[off[e]:off[e + 1]] = blocks["rhs"][k]
    return A, F, off
