"""Thin Python binding of libdg's C ABI (include/dg.h).

Argument marshalling only: every step of the assembly runs in the CUDA
library.  Device buffers are torch tensors (PyTorch provides device memory and
streams).  If the compiled library is missing the import of this module fails
loudly; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# DG_CHECK_BOUNDS=1: the checked build (paper_2007_04881_gb300/build.py)
LIB_PATH = os.path.join(_HERE, "_build_checked" if os.environ.get("DG_CHECK_BOUNDS", "0") not in ("", "0")
                        else "_build", "libdg.so")

DG_OK = 0
DG_ERR = {
    -1: "DG_ERR_ARG",
    -2: "DG_ERR_MESH",
    -3: "DG_ERR_CUDA",
    -4: "DG_ERR_OOM",
    -5: "DG_ERR_ORDER",
    -6: "DG_ERR_TIMEOUT",
    -7: "DG_ERR_BOUNDS",
}
DG_ERR_ARG, DG_ERR_MESH, DG_ERR_CUDA, DG_ERR_OOM, DG_ERR_ORDER, DG_ERR_TIMEOUT = -1, -2, -3, -4, -5, -6
DG_ERR_BOUNDS = -7
DG_PREC_FP64 = 0
DG_PREC_FP32 = 1
DG_PREC_BF16X3 = 2
DG_PREC_TF32X3 = 3
DG_GEOM_FP64 = 16  # OR-ed into prec: the pass's geometry in FP64 (the FP32 records its rounding)
DG_SRC_ZERO, DG_SRC_SINPROD, DG_SRC_POLY = 0, 1, 2
DG_PMAX_2D, DG_PMAX_3D = 6, 4
DG_SPACE_P, DG_SPACE_PQ = 0, 1


class DGError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{DG_ERR.get(code, code)}: {msg}")
        self.code = code


class dg_mesh_desc(C.Structure):
    _fields_ = [
        ("dim", C.c_int),
        ("nv", C.c_int),
        ("x", C.POINTER(C.c_double)),
        ("y", C.POINTER(C.c_double)),
        ("z", C.POINTER(C.c_double)),
        ("ne", C.c_int),
        ("elem_ptr", C.POINTER(C.c_int)),
        ("elem_idx", C.POINTER(C.c_int)),
        ("p", C.POINTER(C.c_int8)),
        ("a", C.POINTER(C.c_double)),
        ("b", C.c_double * 3),
        ("c", C.c_double),
        ("source", C.c_int),
        ("poly", C.c_double * 20),
        ("c_sigma", C.c_double),
        ("neumann", C.c_int),
    ]


class dg_kernel_stat(C.Structure):
    _fields_ = [("name", C.c_char * 48), ("ms", C.c_float), ("flops", C.c_double), ("bytes", C.c_double)]


class dg_quad_stats(C.Structure):
    _fields_ = [("elements", C.c_int), ("eligible", C.c_int), ("accepted", C.c_int),
                ("max_accepted_residual", C.c_float)]


class dg_fields(C.Structure):
    _fields_ = [("b0", C.c_double * 3), ("bx", (C.c_double * 3) * 3), ("c", C.c_double * 20)]


class dg_bsr_info(C.Structure):
    _fields_ = [
        ("ne", C.c_int),
        ("nnzb", C.c_int),
        ("nvals", C.c_int64),
        ("ndofs", C.c_int64),
        ("nfaces", C.c_int),
        ("ninterfaces", C.c_int),
        ("nbfaces", C.c_int),
        ("nsub", C.c_int),
        ("nqvol", C.c_int64),
        ("nqface", C.c_int64),
    ]


_lib = None


def load() -> C.CDLL:
    """Load libdg.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libdg.so not built ({LIB_PATH}); run paper_2007_04881_gb300.build.build()")
    lib = C.CDLL(LIB_PATH)
    V = C.c_void_p
    lib.dg_create.argtypes = [C.POINTER(V), C.c_int, V]
    lib.dg_destroy.argtypes = [V]
    lib.dg_destroy.restype = None
    lib.dg_last_error.restype = C.c_char_p
    lib.dg_mesh_upload.argtypes = [V, C.POINTER(dg_mesh_desc), C.POINTER(V)]
    lib.dg_mesh_free.argtypes = [V]
    lib.dg_mesh_check.argtypes = [C.POINTER(dg_mesh_desc), C.POINTER(dg_bsr_info), V, V, V]
    lib.dg_mesh_update.argtypes = [V, V, V, V, V, V]
    lib.dg_geometry.argtypes = [V, V]
    lib.dg_bsr_layout.argtypes = [V, C.POINTER(dg_bsr_info)]
    lib.dg_bsr_pattern.argtypes = [V, V, V, V, V]
    for n in ("dg_assemble_volume", "dg_assemble_faces", "dg_assemble_rhs"):
        getattr(lib, n).argtypes = [V, V, C.c_int, V]
    lib.dg_assemble.argtypes = [V, V, C.c_int, V, V]
    lib.dg_assemble_host.argtypes = [V, V, C.c_int, V, V, V, V, V, V]
    lib.dg_assemble_host_submit.argtypes = [V, V, C.c_int, V, V, V, V, V, V, C.POINTER(C.c_longlong)]
    lib.dg_assemble_host_wait.argtypes = [V, V, C.c_longlong]
    lib.dg_assemble_step.argtypes = [V, V, C.c_int, V, V]
    lib.dg_set_timing.argtypes = [V, C.c_int]
    lib.dg_kernel_stats.argtypes = [V, C.POINTER(dg_kernel_stat), C.c_int]
    lib.dg_batch_upload.argtypes = [V, C.POINTER(C.POINTER(dg_mesh_desc)), C.c_int, C.POINTER(V)]
    lib.dg_batch_offsets.argtypes = [V, V, V, V, V]
    lib.dg_graph_create.argtypes = [V, V, C.c_int, V, V, C.c_int, C.POINTER(V)]
    lib.dg_graph_launch.argtypes = [V, V]
    lib.dg_graph_info.argtypes = [V, V, V, V, V, V]
    lib.dg_graph_free.argtypes = [V]
    lib.dg_graph_tiles.argtypes = [V, V, V, V]
    lib.dg_set_wait_limit.argtypes = [V, C.c_double]
    lib.dg_set_persistent.argtypes = [V, C.c_int]
    lib.dg_set_pattern_device.argtypes = [V, C.c_int]
    lib.dg_slab_graph_create.argtypes = [V, V, C.c_int, C.c_int, C.c_double, C.c_double, V, V, V, C.POINTER(V)]
    lib.dg_mesh_timings.argtypes = [V, V, V, V]
    lib.dg_mesh_array.argtypes = [V, C.c_char_p, V, C.c_int64, C.POINTER(C.c_int64)]
    lib.dg_wait_probe.argtypes = [V, V, C.c_double]
    lib.dg_set_tile_variants.argtypes = [V, V]
    lib.dg_set_group_split.argtypes = [V, V]
    lib.dg_set_nvtx.argtypes = [V, C.c_int]
    lib.dg_graph_splits.argtypes = [V, V]
    lib.dg_volume_noalloc.argtypes = [V, C.c_int, C.c_int, C.c_int, C.c_int, V, V, C.c_int, C.c_int, V, V, V,
                                      C.c_double, C.c_double, C.c_double, V, V]
    lib.dg_quad_prepare.argtypes = [V, V]
    lib.dg_quad_fit.argtypes = [V, V, V, C.c_int, C.c_int, C.POINTER(dg_quad_stats)]
    lib.dg_quad_targets.argtypes = [V, V, V]
    lib.dg_quad_buffers.argtypes = [V, C.POINTER(V), C.POINTER(V), C.POINTER(V), C.POINTER(V), C.POINTER(V)]
    lib.dg_quad_clear.argtypes = [V, V]
    lib.dg_mlp_create.argtypes = [V, C.c_int, C.POINTER(V)]
    lib.dg_mlp_free.argtypes = [V]
    lib.dg_mlp_num_params.restype = C.c_int64
    lib.dg_mlp_get_params.argtypes = [V, V, C.POINTER(C.c_int64)]
    lib.dg_mlp_set_params.argtypes = [V, V, C.c_int64]
    lib.dg_mlp_get_state.argtypes = [V, V, V]
    lib.dg_mlp_set_state.argtypes = [V, V, V]
    lib.dg_mlp_forward.argtypes = [V, V, V, C.c_int, V]
    lib.dg_mlp_grad.argtypes = [V, V, V, V, C.c_int, V, V]
    lib.dg_mlp_train_step.argtypes = [V, V, V, V, C.c_int, C.c_float, V]
    lib.dg_mlp_save.argtypes = [V, V, C.c_char_p, C.c_uint64, C.c_int64]
    lib.dg_mlp_load.argtypes = [V, V, C.c_char_p, C.POINTER(C.c_uint64), C.POINTER(C.c_int64)]
    lib.dg_quad_learn.argtypes = [V, V, V, C.c_int, C.POINTER(dg_quad_stats)]
    lib.dg_assemble_batch.argtypes = [V, V, C.c_int, C.c_int, V, V, C.c_int]
    lib.dg_set_volume_path.argtypes = [V, C.c_int]
    lib.dg_partition.argtypes = [C.POINTER(dg_mesh_desc), C.c_int, V]
    lib.dg_mesh_upload_part.argtypes = [V, C.POINTER(dg_mesh_desc), V, C.c_int, C.POINTER(V)]
    lib.dg_part_map.argtypes = [V, V, V, V, V, V]
    lib.dg_part_check.argtypes = [C.POINTER(dg_mesh_desc), V, C.c_int, C.POINTER(dg_bsr_info), V, V, V, V, V, V]
    lib.dg_sync.argtypes = [V]
    lib.dg_last_launch_count.argtypes = [V]
    lib.dg_slab_offsets.argtypes = [C.c_int, C.c_int, V, V, V, C.c_int, V, V]
    lib.dg_slab_layout.argtypes = [V, C.c_int, V, V]
    lib.dg_assemble_slab.argtypes = [V, V, C.c_int, C.c_int, C.c_double, C.c_double, V, V, V]
    lib.dg_slab_trace.argtypes = [V, V, C.c_int, C.c_int, C.c_double, C.c_double, V, V]
    lib.dg_assemble_varcoef.argtypes = [V, V, V, V]
    lib.dg_assemble_varcoef_form.argtypes = [V, V, C.c_int, V, V]
    lib.dg_mesh_set_fields.argtypes = [V, V]
    _lib = lib
    return lib


# names of every symbol declared in include/dg.h
EXPORTS = (
    "dg_create", "dg_destroy", "dg_last_error", "dg_mesh_upload", "dg_mesh_free", "dg_mesh_check",
    "dg_mesh_update",
    "dg_geometry", "dg_bsr_layout", "dg_bsr_pattern", "dg_assemble_volume", "dg_assemble_faces",
    "dg_assemble_rhs", "dg_assemble", "dg_assemble_host", "dg_assemble_host_submit", "dg_assemble_host_wait",
    "dg_sync", "dg_last_launch_count",
    "dg_assemble_step", "dg_set_timing", "dg_kernel_stats", "dg_batch_upload", "dg_batch_offsets",
    "dg_graph_create", "dg_graph_launch", "dg_graph_info", "dg_graph_free", "dg_volume_noalloc",
    "dg_quad_prepare", "dg_quad_fit", "dg_quad_targets", "dg_quad_buffers", "dg_quad_clear",
    "dg_mlp_create", "dg_mlp_free", "dg_mlp_num_params", "dg_mlp_get_params", "dg_mlp_set_params",
    "dg_mlp_get_state", "dg_mlp_set_state", "dg_mlp_forward", "dg_mlp_grad", "dg_mlp_train_step",
    "dg_partition", "dg_mesh_upload_part", "dg_part_map", "dg_part_check", "dg_set_volume_path",
    "dg_slab_offsets", "dg_slab_layout", "dg_assemble_slab", "dg_slab_trace", "dg_assemble_varcoef", "dg_assemble_varcoef_form", "dg_mesh_set_fields",
    "dg_mlp_save", "dg_mlp_load", "dg_quad_learn", "dg_assemble_batch", "dg_graph_tiles",
    "dg_set_tile_variants", "dg_set_group_split", "dg_graph_splits", "dg_set_nvtx", "dg_set_wait_limit", "dg_wait_probe",
    "dg_set_persistent", "dg_set_pattern_device", "dg_mesh_timings", "dg_mesh_array",
    "dg_slab_graph_create",
)


def _check(rc: int):
    if rc != DG_OK:
        raise DGError(rc, load().dg_last_error().decode())


def _ptr(a: Optional[np.ndarray], ct):
    return None if a is None else a.ctypes.data_as(C.POINTER(ct))


def _vp(x) -> Optional[int]:
    """Raw pointer of a torch tensor / numpy array / int / None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


@dataclass
class Problem:
    """Constant problem data of Eq. (2.1): advection b, reaction c, source;
    ``neumann``: bit 2d + s marks the side x_d = min (s = 0) / max (s = 1) of
    the vertices' bounding box as Neumann boundary (Eq. (2.2))."""

    b: Sequence[float] = (0.0, 0.0, 0.0)
    c: float = 0.0
    source: int = DG_SRC_ZERO
    poly: Sequence[float] = field(default_factory=list)
    c_sigma: float = 10.0
    neumann: int = 0


class Context:
    """dg_create / dg_destroy.  ``stream`` is a cudaStream_t handle (int) or None."""

    def __init__(self, device: int = 0, stream: Optional[int] = None):
        lib = load()
        h = C.c_void_p()
        _check(lib.dg_create(C.byref(h), int(device), stream))
        self._h = h
        self.device = device

    def close(self):
        if getattr(self, "_h", None):
            load().dg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def dg_sync(self):
        _check(load().dg_sync(self._h))

    def dg_set_volume_path(self, path: int):
        """1: volume blocks through Legendre-product moments (default); 0: per-point contraction."""
        _check(load().dg_set_volume_path(self._h, int(path)))

    def dg_set_tile_variants(self, variants=None):
        """Row-kernel tile variant per degree (9 ints, or None for the defaults)."""
        v = None if variants is None else np.ascontiguousarray(variants, dtype=np.int32)
        _check(load().dg_set_tile_variants(self._h, _vp(v)))

    def dg_set_nvtx(self, on: bool = True):
        """NVTX ranges around this context's calls and their stages."""
        _check(load().dg_set_nvtx(self._h, int(on)))

    def dg_set_group_split(self, split=None):
        """Parts (1..4) per degree group of untuned concurrent passes (9 ints, or None for all 1)."""
        v = None if split is None else np.ascontiguousarray(split, dtype=np.int32)
        _check(load().dg_set_group_split(self._h, _vp(v)))

    def dg_set_pattern_device(self, on: bool):
        _check(load().dg_set_pattern_device(self._h, int(bool(on))))

    def dg_set_persistent(self, on: bool):
        _check(load().dg_set_persistent(self._h, int(bool(on))))

    def dg_set_wait_limit(self, seconds: float):
        _check(load().dg_set_wait_limit(self._h, float(seconds)))

    def dg_wait_probe(self, flag, seconds: float):
        """The bounded device wait on flag (a one-int device tensor)."""
        _check(load().dg_wait_probe(self._h, _vp(flag), float(seconds)))

    def launches(self) -> int:
        return load().dg_last_launch_count(self._h)

    def dg_set_timing(self, enable: bool):
        _check(load().dg_set_timing(self._h, int(bool(enable))))

    def dg_kernel_stats(self):
        """[(name, ms, flops, bytes)] of the most recent call's launches."""
        buf = (dg_kernel_stat * 64)()
        n = load().dg_kernel_stats(self._h, buf, 64)
        if n < 0:
            _check(n)
        return [(buf[i].name.decode(), float(buf[i].ms), float(buf[i].flops), float(buf[i].bytes)) for i in range(n)]


def make_desc(mesh, p, a, problem: Problem):
    """dg_mesh_desc for a generator mesh; returns (desc, arrays kept alive)."""
    d = dg_mesh_desc()
    keep = []
    dim = mesh.dim

    def arr(x, dt):
        v = np.ascontiguousarray(x, dtype=dt)
        keep.append(v)
        return v

    x = arr(mesh.x, np.float64)
    y = arr(mesh.y, np.float64)
    z = arr(mesh.z, np.float64) if dim == 3 else None
    if dim == 2:
        eptr, eidx = arr(mesh.elem_vptr, np.int32), arr(mesh.elem_v, np.int32)
    else:
        eptr, eidx = arr(mesh.elem_tptr, np.int32), arr(mesh.tet_v, np.int32)
    pp = arr(p, np.int8)
    aa = arr(a, np.float64)
    d.dim = dim
    d.nv = int(x.shape[0])
    d.x, d.y, d.z = _ptr(x, C.c_double), _ptr(y, C.c_double), _ptr(z, C.c_double)
    d.ne = int(eptr.shape[0] - 1)
    d.elem_ptr, d.elem_idx = _ptr(eptr, C.c_int), _ptr(eidx, C.c_int)
    d.p, d.a = _ptr(pp, C.c_int8), _ptr(aa, C.c_double)
    for i in range(3):
        d.b[i] = float(problem.b[i]) if i < len(problem.b) else 0.0
    d.c = float(problem.c)
    d.source = int(problem.source)
    for i in range(20):
        d.poly[i] = float(problem.poly[i]) if i < len(problem.poly) else 0.0
    d.c_sigma = float(problem.c_sigma)
    d.neumann = int(getattr(problem, "neumann", 0))
    return d, keep


def dg_mesh_check(mesh, p, a, problem: Problem, pattern: bool = False):
    """Host-only validation + pattern (no GPU).  Returns info or (info, row_ptr, col, blk_off)."""
    lib = load()
    d, keep = make_desc(mesh, p, a, problem)
    info = dg_bsr_info()
    _check(lib.dg_mesh_check(C.byref(d), C.byref(info), None, None, None))
    if not pattern:
        return info
    row_ptr = np.zeros(info.ne + 1, np.int32)
    col = np.zeros(info.nnzb, np.int32)
    blk_off = np.zeros(info.nnzb + 1, np.int64)
    _check(lib.dg_mesh_check(C.byref(d), C.byref(info), _vp(row_ptr), _vp(col), _vp(blk_off)))
    return info, row_ptr, col, blk_off


def dg_slab_offsets(dim: int, row_ptr, col, p, space: int):
    """Host-only slab layout of a block pattern: (blk_off [nnzb+1], dof_off [ne+1])."""
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    p = np.ascontiguousarray(p, dtype=np.int32)
    ne = p.size
    blk_off = np.zeros(col.size + 1, np.int64)
    dof_off = np.zeros(ne + 1, np.int64)
    _check(load().dg_slab_offsets(int(dim), int(ne), _vp(row_ptr), _vp(col), _vp(p), int(space), _vp(blk_off),
                                  _vp(dof_off)))
    return blk_off, dof_off


def dg_partition(mesh, p, a, problem: Problem, nparts: int) -> np.ndarray:
    """Space-filling-curve partition of the elements into nparts runs of equal cost (host only)."""
    d, keep = make_desc(mesh, p, a, problem)
    part = np.zeros(d.ne, np.int32)
    _check(load().dg_partition(C.byref(d), int(nparts), _vp(part)))
    return part


def dg_part_check(mesh, p, a, problem: Problem, part, my_part: int):
    """Host part of a partition upload: local layout and local -> global element map."""
    lib = load()
    d, keep = make_desc(mesh, p, a, problem)
    part = np.ascontiguousarray(part, dtype=np.int32)
    info = dg_bsr_info()
    nowned = C.c_int()
    _check(lib.dg_part_check(C.byref(d), _vp(part), int(my_part), C.byref(info), C.byref(nowned),
                             None, None, None, None, None))
    row_ptr = np.zeros(info.ne + 1, np.int32)
    col = np.zeros(info.nnzb, np.int32)
    blk_off = np.zeros(info.nnzb + 1, np.int64)
    elem_global = np.zeros(info.ne, np.int32)
    owned = np.zeros(info.ne, np.int8)
    _check(lib.dg_part_check(C.byref(d), _vp(part), int(my_part), C.byref(info), C.byref(nowned),
                             _vp(row_ptr), _vp(col), _vp(blk_off), _vp(elem_global), _vp(owned)))
    return dict(info=info, nowned=nowned.value, row_ptr=row_ptr, col=col, blk_off=blk_off,
                elem_global=elem_global, owned=owned)


class Mesh:
    """dg_mesh_upload of a generator mesh (meshgen.Mesh2D / Mesh3D); with
    ``part`` and ``my_part``, dg_mesh_upload_part of one part of it; with a
    list of (mesh, p, a) members, dg_batch_upload of their disjoint union."""

    def __init__(self, ctx: Context, mesh, p=None, a=None, problem: Problem = None, members=None,
                 part=None, my_part=None):
        lib = load()
        self.ctx = ctx
        h = C.c_void_p()
        if part is not None:
            self.dim = mesh.dim
            d, keep = make_desc(mesh, p, a, problem)
            prt = np.ascontiguousarray(part, dtype=np.int32)
            _check(lib.dg_mesh_upload_part(ctx._h, C.byref(d), _vp(prt), int(my_part), C.byref(h)))
            self._h = h
            ne_loc = C.c_int()
            info = dg_bsr_info()
            _check(lib.dg_bsr_layout(h, C.byref(info)))
            self.elem_global = np.zeros(info.ne, np.int32)
            self.owned = np.zeros(info.ne, np.int8)
            nv_loc = C.c_int()
            _check(lib.dg_part_map(h, C.byref(ne_loc), C.byref(nv_loc), _vp(self.elem_global), _vp(self.owned),
                                   None))
            self.nowned = ne_loc.value
            self.vert_global = np.zeros(nv_loc.value, np.int32)
            _check(lib.dg_part_map(h, None, None, None, None, _vp(self.vert_global)))
            self.p = np.asarray(keep[-2])[self.elem_global]
        elif members is None:
            self.dim = mesh.dim
            d, keep = make_desc(mesh, p, a, problem)
            pp = keep[-2]
            _check(lib.dg_mesh_upload(ctx._h, C.byref(d), C.byref(h)))
            self.p = np.asarray(pp)
        else:
            self.dim = members[0][0].dim
            descs, keeps = [], []
            for (mm, pm, am) in members:
                d, keep = make_desc(mm, pm, am, problem)
                descs.append(d)
                keeps.append(keep)
            arr = (C.POINTER(dg_mesh_desc) * len(descs))(*[C.pointer(d) for d in descs])
            _check(lib.dg_batch_upload(ctx._h, arr, len(descs), C.byref(h)))
            self.p = np.concatenate([np.asarray(k[-2]) for k in keeps])
        self._h = h
        info = dg_bsr_info()
        _check(lib.dg_bsr_layout(h, C.byref(info)))
        self.info = info
        self.ne = info.ne
        self.nvals = int(info.nvals)
        self.ndofs = int(info.ndofs)

    def close(self):
        if getattr(self, "_h", None):
            load().dg_mesh_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def dg_bsr_pattern(self):
        ne, nnzb = self.info.ne, self.info.nnzb
        row_ptr = np.zeros(ne + 1, np.int32)
        col = np.zeros(nnzb, np.int32)
        blk_off = np.zeros(nnzb + 1, np.int64)
        dof_off = np.zeros(ne + 1, np.int64)
        _check(load().dg_bsr_pattern(self._h, _vp(row_ptr), _vp(col), _vp(blk_off), _vp(dof_off)))
        return row_ptr, col, blk_off, dof_off

    def dg_assemble_volume(self, prec: int, vals):
        _check(load().dg_assemble_volume(self.ctx._h, self._h, prec, _vp(vals)))

    def dg_assemble_faces(self, prec: int, vals):
        _check(load().dg_assemble_faces(self.ctx._h, self._h, prec, _vp(vals)))

    def dg_assemble_rhs(self, prec: int, rhs):
        _check(load().dg_assemble_rhs(self.ctx._h, self._h, prec, _vp(rhs)))

    def dg_assemble(self, prec: int, vals, rhs=None):
        _check(load().dg_assemble(self.ctx._h, self._h, prec, _vp(vals), _vp(rhs)))

    def dg_batch_offsets(self):
        n = C.c_int()
        _check(load().dg_batch_offsets(self._h, C.byref(n), None, None, None))
        eo = np.zeros(n.value + 1, np.int32)
        vo = np.zeros(n.value + 1, np.int64)
        do = np.zeros(n.value + 1, np.int64)
        _check(load().dg_batch_offsets(self._h, None, _vp(eo), _vp(vo), _vp(do)))
        return eo, vo, do

    def dg_mesh_timings(self):
        pm, um, od = C.c_double(), C.c_double(), C.c_int()
        _check(load().dg_mesh_timings(self._h, C.byref(pm), C.byref(um), C.byref(od)))
        return {"pattern_ms": pm.value, "upload_ms": um.value, "on_device": bool(od.value)}

    def dg_mesh_array(self, name: str) -> np.ndarray:
        """A copy of one of the mesh's internal arrays (dg_mesh_array)."""
        nb = C.c_int64()
        _check(load().dg_mesh_array(self._h, name.encode(), None, 0, C.byref(nb)))
        dt = {"f_flip": np.int8, "hf_side": np.int8, "blk_off": np.int64, "dof_off": np.int64}.get(name, np.int32)
        out = np.zeros(int(nb.value) // np.dtype(dt).itemsize, dt)
        _check(load().dg_mesh_array(self._h, name.encode(), _vp(out), int(nb.value), None))
        return out

    def dg_graph_create(self, prec: int, vals, rhs=None, autotune: bool = True) -> "Graph":
        h = C.c_void_p()
        _check(load().dg_graph_create(self.ctx._h, self._h, prec, _vp(vals), _vp(rhs), int(autotune), C.byref(h)))
        return Graph(self.ctx, h)

    # ---- learned volume rules (2D)
    def dg_quad_prepare(self):
        _check(load().dg_quad_prepare(self.ctx._h, self._h))

    def dg_quad_fit(self, init=None, iters: int = 3, install: bool = False):
        st = dg_quad_stats()
        _check(load().dg_quad_fit(self.ctx._h, self._h, _vp(init), int(iters), int(install), C.byref(st)))
        return {"elements": st.elements, "eligible": st.eligible, "accepted": st.accepted,
                "max_accepted_residual": st.max_accepted_residual}

    def dg_quad_learn(self, net=None, iters: int = 3):
        """Proposals of net (None: the fixed start), Gauss-Newton, install."""
        st = dg_quad_stats()
        _check(load().dg_quad_learn(self.ctx._h, self._h, net._h if net is not None else None, int(iters),
                                    C.byref(st)))
        return {"elements": st.elements, "eligible": st.eligible, "accepted": st.accepted,
                "max_accepted_residual": st.max_accepted_residual}

    def dg_quad_targets(self, out):
        _check(load().dg_quad_targets(self.ctx._h, self._h, _vp(out)))

    def dg_quad_buffers(self):
        """Raw device addresses of the library-owned learned-rule arrays."""
        f, r, e, o, mo = (C.c_void_p() for _ in range(5))
        _check(load().dg_quad_buffers(self._h, C.byref(f), C.byref(r), C.byref(e), C.byref(o), C.byref(mo)))
        return {"feat": f.value, "rules": r.value, "resid": e.value, "ok": o.value, "moments": mo.value}

    def dg_quad_clear(self):
        _check(load().dg_quad_clear(self.ctx._h, self._h))

    def dg_assemble_varcoef(self, vals, rhs=None, prec=None):
        """The system with the mesh's fields b(x), c(x) (dg_mesh_set_fields; the
        Sec. 4.2 fields by default) in prec (FP64 by default, or FP32); the
        mesh is uploaded with b = 0, c = 0."""
        if prec is None:
            _check(load().dg_assemble_varcoef(self.ctx._h, self._h, _vp(vals), _vp(rhs)))
        else:
            _check(load().dg_assemble_varcoef_form(self.ctx._h, self._h, int(prec), _vp(vals), _vp(rhs)))

    def dg_mesh_set_fields(self, b0=None, bx=None, c=None):
        """Fields b_d = b0[d] + sum_e bx[d][e] x_e and c = sum_k c[k] m_k(x) (graded
        monomials of degree <= 3); no arguments: the Sec. 4.2 fields."""
        if b0 is None and bx is None and c is None:
            _check(load().dg_mesh_set_fields(self._h, None))
            return
        f = dg_fields()
        b0 = list(b0) if b0 is not None else [0.0] * 3
        bx = np.zeros((3, 3)) if bx is None else np.asarray(bx, dtype=np.float64).reshape(3, 3)
        c = list(c) if c is not None else []
        for d in range(3):
            f.b0[d] = float(b0[d]) if d < len(b0) else 0.0
            for e in range(3):
                f.bx[d][e] = float(bx[d, e])
        for k in range(20):
            f.c[k] = float(c[k]) if k < len(c) else 0.0
        _check(load().dg_mesh_set_fields(self._h, C.byref(f)))

    def dg_slab_layout(self, space: int):
        """(nvals, ndofs) of the space-time slab system over this mesh."""
        nv, nd = C.c_int64(), C.c_int64()
        _check(load().dg_slab_layout(self._h, int(space), C.byref(nv), C.byref(nd)))
        return nv.value, nd.value

    def dg_slab_pattern(self, space: int):
        """Host (blk_off, dof_off) of the slab system; the block graph is dg_bsr_pattern's."""
        row_ptr, col, _, _ = self.dg_bsr_pattern()
        return dg_slab_offsets(self.dim, row_ptr, col, self.p, space)

    def dg_assemble_slab(self, prec: int, space: int, t0: float, t1: float, vals, rhs=None, u_prev=None):
        _check(load().dg_assemble_slab(self.ctx._h, self._h, prec, int(space), float(t0), float(t1), _vp(u_prev),
                                       _vp(vals), _vp(rhs)))

    def dg_slab_graph_create(self, prec: int, space: int, t0: float, t1: float, vals, rhs=None, u_prev=None):
        """The slab step recorded as one CUDA graph (replay: Graph.dg_graph_launch)."""
        h = C.c_void_p()
        _check(load().dg_slab_graph_create(self.ctx._h, self._h, prec, int(space), float(t0), float(t1),
                                           _vp(u_prev), _vp(vals), _vp(rhs), C.byref(h)))
        return Graph(self.ctx, h)

    def dg_slab_trace(self, prec: int, space: int, t0: float, t1: float, U, u_end):
        _check(load().dg_slab_trace(self.ctx._h, self._h, prec, int(space), float(t0), float(t1), _vp(U),
                                    _vp(u_end)))

    def dg_assemble_step(self, prec: int, vals, rhs=None):
        _check(load().dg_assemble_step(self.ctx._h, self._h, prec, _vp(vals), _vp(rhs)))

    def dg_geometry(self):
        _check(load().dg_geometry(self.ctx._h, self._h))

    def dg_mesh_update(self, x=None, y=None, z=None, a=None):
        _check(load().dg_mesh_update(self.ctx._h, self._h, _vp(x), _vp(y), _vp(z), _vp(a)))

    def dg_assemble_host(self, prec: int, vals_host, rhs_host=None, x=None, y=None, z=None, a=None):
        _check(load().dg_assemble_host(self.ctx._h, self._h, prec, _vp(x), _vp(y), _vp(z), _vp(a),
                                       _vp(vals_host), _vp(rhs_host)))

    def dg_assemble_host_submit(self, prec: int, vals_host, rhs_host=None, x=None, y=None, z=None, a=None) -> int:
        """Queue one host-buffer assembly; returns its ticket (the buffers stay
        in use until dg_assemble_host_wait(ticket) returns)."""
        t = C.c_longlong(-1)
        _check(load().dg_assemble_host_submit(self.ctx._h, self._h, prec, _vp(x), _vp(y), _vp(z), _vp(a),
                                              _vp(vals_host), _vp(rhs_host), C.byref(t)))
        return t.value

    def dg_assemble_host_wait(self, ticket: int):
        _check(load().dg_assemble_host_wait(self.ctx._h, self._h, C.c_longlong(int(ticket))))


def dg_volume_noalloc(stream, device: int, prec: int, p: int, x, y, elem_ptr, elem_idx, a, bx: float, by: float,
                      c: float, blocks, nsub: int, status=None):
    """Allocation-free volume blocks (all array arguments are device buffers;
    status, a one-int device tensor or None, receives the list check's code)."""
    _check(load().dg_volume_noalloc(stream, int(device), int(prec), int(p), int(x.numel()), _vp(x), _vp(y),
                                    int(a.numel()), int(nsub), _vp(elem_ptr), _vp(elem_idx), _vp(a), float(bx),
                                    float(by), float(c), _vp(blocks), _vp(status) if status is not None else None))


def dg_assemble_batch(ctx: Context, meshes, prec: int, vals, rhs=None, use_graph: bool = False):
    """Separately uploaded meshes, each into its own vals[k] / rhs[k] (device
    tensors; rhs may be None or hold None entries), in one call."""
    n = len(meshes)
    mh = (C.c_void_p * n)(*[m._h.value for m in meshes])
    vh = (C.c_void_p * n)(*[_vp(v) for v in vals])
    rh = (C.c_void_p * n)(*[_vp(r) for r in rhs]) if rhs is not None else None
    _check(load().dg_assemble_batch(ctx._h, mh, n, int(prec), vh, rh, int(bool(use_graph))))


def device_view(ptr: int, shape, dtype: str):
    """A torch tensor viewing library-owned device memory (no copy).
    dtype: 'f8', 'f4', 'i4' or 'bf16'."""
    import torch

    typestr = {"f8": "<f8", "f4": "<f4", "i4": "<i4", "bf16": "<i2"}[dtype]

    class _View:
        __cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (int(ptr), False),
                                    "version": 3}

    t = torch.as_tensor(_View(), device="cuda")
    return t.view(torch.bfloat16) if dtype == "bf16" else t


class MLP:
    """The quadrature-proposal network (dg_mlp_*)."""

    def __init__(self, ctx: Context, seed: int = 0):
        self.ctx = ctx
        h = C.c_void_p()
        _check(load().dg_mlp_create(ctx._h, int(seed), C.byref(h)))
        self._h = h
        self.nparams = int(load().dg_mlp_num_params())

    def close(self):
        if getattr(self, "_h", None):
            load().dg_mlp_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self):
        out = np.zeros(self.nparams, np.float32)
        step = C.c_int64()
        _check(load().dg_mlp_get_params(self._h, _vp(out), C.byref(step)))
        return out, step.value

    def set_params(self, params, step: int = 0):
        params = np.ascontiguousarray(params, dtype=np.float32)
        _check(load().dg_mlp_set_params(self._h, _vp(params), int(step)))

    def get_state(self):
        m1 = np.zeros(self.nparams, np.float32)
        m2 = np.zeros(self.nparams, np.float32)
        _check(load().dg_mlp_get_state(self._h, _vp(m1), _vp(m2)))
        return m1, m2

    def set_state(self, m1, m2):
        m1 = np.ascontiguousarray(m1, dtype=np.float32)
        m2 = np.ascontiguousarray(m2, dtype=np.float32)
        _check(load().dg_mlp_set_state(self._h, _vp(m1), _vp(m2)))

    def forward(self, x_bf16, n: int, out):
        _check(load().dg_mlp_forward(self.ctx._h, self._h, _vp(x_bf16), int(n), _vp(out)))

    def grad(self, x_bf16, target, n: int, grad, loss):
        _check(load().dg_mlp_grad(self.ctx._h, self._h, _vp(x_bf16), _vp(target), int(n), _vp(grad), _vp(loss)))

    def train_step(self, x_bf16, target, n: int, lr: float, loss=None):
        _check(load().dg_mlp_train_step(self.ctx._h, self._h, _vp(x_bf16), _vp(target), int(n), float(lr), _vp(loss)))

    def save(self, path: str, seed: int, cursor: int):
        """Checkpoint file: parameters, Adam moments, step, and the training
        loop's data seed and cursor (dg_mlp_save)."""
        _check(load().dg_mlp_save(self.ctx._h, self._h, os.fsencode(path), int(seed), int(cursor)))

    def load(self, path: str):
        """Restore a checkpoint; returns (seed, cursor)."""
        seed, cursor = C.c_uint64(), C.c_int64()
        _check(load().dg_mlp_load(self.ctx._h, self._h, os.fsencode(path), C.byref(seed), C.byref(cursor)))
        return seed.value, cursor.value


class Graph:
    """A recorded assembly pass (dg_graph_create); keep the buffers alive."""

    def __init__(self, ctx: Context, h):
        self.ctx = ctx
        self._h = h

    def dg_graph_launch(self):
        _check(load().dg_graph_launch(self.ctx._h, self._h))

    def dg_graph_info(self):
        occ, conc, ms, nl, vp = C.c_int(), C.c_int(), C.c_float(), C.c_int(), C.c_int()
        _check(load().dg_graph_info(self._h, C.byref(occ), C.byref(conc), C.byref(ms), C.byref(nl), C.byref(vp)))
        tm = np.zeros(9, np.int32)
        tr, pk = C.c_int(), C.c_int()
        _check(load().dg_graph_tiles(self._h, _vp(tm), C.byref(tr), C.byref(pk)))
        sp = np.ones(9, np.int32)
        _check(load().dg_graph_splits(self._h, _vp(sp)))
        return {"occ_cap": occ.value, "concurrent": bool(conc.value), "tuned_ms": ms.value, "launches": nl.value,
                "volume_path": {0: "per-point", 1: "moments", 2: "exact-moments"}.get(vp.value, "per-point"),
                "tile_tm": {f"p{p}": int(tm[p]) for p in range(9) if tm[p] != 0}, "tuner_trials": tr.value,
                "persistent": bool(pk.value),
                "split": {f"p{p}": int(sp[p]) for p in range(9) if tm[p] != 0}}

    def close(self):
        if getattr(self, "_h", None):
            load().dg_graph_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def to_blocks(mesh: Mesh, vals: np.ndarray, rhs: Optional[np.ndarray] = None):
    """Split BSR values (host array) into per-element diagonal blocks and
    per-(row, col) off-diagonal blocks (dicts keyed by element ids)."""
    row_ptr, col, blk_off, dof_off = mesh.dg_bsr_pattern()
    from math import comb

    nb = np.array([comb(int(q) + mesh.dim, mesh.dim) for q in mesh.p])
    diag, off = {}, {}
    for r in range(mesh.ne):
        for k in range(row_ptr[r], row_ptr[r + 1]):
            c = int(col[k])
            blk = vals[blk_off[k]:blk_off[k + 1]].reshape(nb[r], nb[c])
            if c == r:
                diag[r] = blk
            else:
                off[(r, c)] = blk
    out = {"diag": diag, "off": off}
    if rhs is not None:
        out["rhs"] = {e: rhs[dof_off[e]:dof_off[e + 1]] for e in range(mesh.ne)}
    return out
