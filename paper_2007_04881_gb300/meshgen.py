"""Seeded synthetic mesh and coefficient generators.

This module produces the inputs shared by the CUDA path, the CPU oracle, the
tests and the benchmark.  It holds none of the assembly method's arithmetic:
it only draws random sites / coefficients and builds polygon and polyhedron
connectivity.  Both the library and the oracle derive every geometric and
discrete quantity (faces, normals, quadrature, basis) on their own.

Generators
----------
* ``voronoi_square``: clipped Voronoi tessellation of the unit square from
  uniformly drawn sites, relaxed by Lloyd iterations (cells are convex, loops
  are counter-clockwise, vertices are shared between neighbouring cells).
* ``kuhn_cube_agglomerated``: a structured n^3 cube mesh split into 6 Kuhn
  tetrahedra per cube, agglomerated into connected polyhedra by seeded
  k-means on tetrahedron centroids followed by a connectivity repair.

The paper (Sec. 4.1 and Sec. 4.2) measures on agglomerated meshes of a
503,596-triangle background mesh and on METIS-partitioned tetrahedral meshes;
neither mesh is available, so these generators stand in for them with the
same structure (general polygons / polyhedra with many faces).
"""
from __future__ import annotations

import dataclasses
import hashlib
import os
from typing import Optional

import numpy as np

__all__ = [
    "Mesh2D",
    "Mesh3D",
    "voronoi_square",
    "kuhn_cube_agglomerated",
    "draw_degrees",
    "draw_log_uniform",
]


@dataclasses.dataclass
class Mesh2D:
    """Polygonal mesh: shared vertices and one CCW vertex loop per element."""

    x: np.ndarray  # float64 [nv]
    y: np.ndarray  # float64 [nv]
    elem_vptr: np.ndarray  # int32 [ne+1]
    elem_v: np.ndarray  # int32 [elem_vptr[-1]]

    @property
    def dim(self) -> int:
        return 2

    @property
    def ne(self) -> int:
        return int(self.elem_vptr.shape[0] - 1)

    @property
    def nv(self) -> int:
        return int(self.x.shape[0])


@dataclasses.dataclass
class Mesh3D:
    """Polyhedral mesh: shared vertices, each element a list of tetrahedra."""

    x: np.ndarray  # float64 [nv]
    y: np.ndarray
    z: np.ndarray
    elem_tptr: np.ndarray  # int32 [ne+1]
    tet_v: np.ndarray  # int32 [4 * ntet], tets grouped by element

    @property
    def dim(self) -> int:
        return 3

    @property
    def ne(self) -> int:
        return int(self.elem_tptr.shape[0] - 1)

    @property
    def nv(self) -> int:
        return int(self.x.shape[0])

    @property
    def ntet(self) -> int:
        return int(self.tet_v.shape[0] // 4)


def _cache_dir() -> Optional[str]:
    d = os.environ.get("DG_MESH_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "dg_meshgen"))
    if d in ("", "0", "off"):
        return None
    try:
        os.makedirs(d, exist_ok=True)
    except OSError:
        return None
    return d


def _cached(key: str, build):
    d = _cache_dir()
    if d is None:
        return build()
    h = hashlib.sha1(key.encode()).hexdigest()[:16]
    path = os.path.join(d, f"mesh_{h}.npz")
    if os.path.exists(path):
        try:
            with np.load(path) as z:
                return {k: z[k] for k in z.files}
        except Exception:  # corrupt cache entry: rebuild
            pass
    out = build()
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "wb") as f:
        np.savez(f, **out)
    os.replace(tmp, path)
    return out


# ----------------------------------------------------------------------------
# 2D: clipped Voronoi tessellation of the unit square with Lloyd relaxation
# ----------------------------------------------------------------------------


def _voronoi_cells(sites: np.ndarray):
    """Voronoi cells of ``sites`` clipped to [0,1]^2.

    Mirroring every site across the four sides of the square makes the
    bisector between a site and its mirror image the side itself, so the cells
    of the original sites in the augmented diagram are exactly the clipped
    cells.  Returns shared vertex coordinates and CCW loops.
    """
    from scipy.spatial import Voronoi, cKDTree

    n = sites.shape[0]
    sx, sy = sites[:, 0], sites[:, 1]
    # Only sites near a side can own a clipped edge; mirror those (the result
    # is checked below and recomputed with every site mirrored if it fails).
    margin = min(1.0, 8.0 / np.sqrt(max(n, 1)))
    for attempt in range(2):
        if attempt == 1:
            margin = 2.0
        parts = [sites]
        for m, img in (
            (sx < margin, np.c_[-sx, sy]),
            (sx > 1.0 - margin, np.c_[2.0 - sx, sy]),
            (sy < margin, np.c_[sx, -sy]),
            (sy > 1.0 - margin, np.c_[sx, 2.0 - sy]),
        ):
            parts.append(img[m])
        vor = Voronoi(np.concatenate(parts))
        regions = [vor.regions[vor.point_region[i]] for i in range(n)]
        used = np.unique(np.concatenate([np.asarray(r, dtype=np.int64) for r in regions]))
        ok = used.size > 0 and used[0] >= 0
        if ok:
            Vu = vor.vertices[used]
            ok = bool(np.all(Vu > -1e-9) and np.all(Vu < 1.0 + 1e-9))
        if ok:
            break
    if not ok:
        raise RuntimeError("clipped Voronoi construction failed")
    V = vor.vertices[used].copy()
    # snap to the square's sides (the mirror construction puts these vertices on
    # the sides up to rounding)
    for d in range(2):
        col = V[:, d]
        col[np.abs(col) < 1e-12] = 0.0
        col[np.abs(col - 1.0) < 1e-12] = 1.0
    remap = np.full(vor.vertices.shape[0], -1, dtype=np.int64)
    remap[used] = np.arange(used.size)
    # merge vertices that coincide to 1e-12 (degenerate co-circular configurations)
    tree = cKDTree(V)
    pairs = tree.query_pairs(r=1e-12, output_type="ndarray")
    vmap = np.arange(V.shape[0])
    if pairs.shape[0]:
        parent = np.arange(V.shape[0])

        def find(i):
            while parent[i] != i:
                parent[i] = parent[parent[i]]
                i = parent[i]
            return i

        for a, b in pairs:
            ra, rb = find(a), find(b)
            if ra != rb:
                parent[max(ra, rb)] = min(ra, rb)
        roots = np.array([find(i) for i in range(V.shape[0])])
        keep = np.unique(roots)
        compact = np.full(V.shape[0], -1, dtype=np.int64)
        compact[keep] = np.arange(keep.size)
        vmap = compact[roots]
        V = V[keep]

    cnt = np.array([len(r) for r in regions])
    owner = np.repeat(np.arange(n), cnt)
    flat = vmap[remap[np.concatenate([np.asarray(r, dtype=np.int64) for r in regions])]]
    ang = np.arctan2(V[flat, 1] - sites[owner, 1], V[flat, 0] - sites[owner, 0])
    order = np.lexsort((ang, owner))  # CCW around each site
    flat = flat[order]
    # drop consecutive duplicates (within a loop, cyclically) left by merging
    start = np.zeros(n + 1, dtype=np.int64)
    start[1:] = np.cumsum(cnt)
    prev = np.empty_like(flat)
    prev[1:] = flat[:-1]
    prev[start[:-1]] = flat[start[1:] - 1]
    keepm = flat != prev
    flat = flat[keepm]
    cnt = np.bincount(owner[keepm], minlength=n)
    if cnt.min() < 3:
        raise RuntimeError("degenerate Voronoi cell")
    loops = np.split(flat, np.cumsum(cnt)[:-1])
    return V, loops


def _loop_centroids(V: np.ndarray, loops) -> np.ndarray:
    """Area centroids of polygons (generator-side Lloyd update only)."""
    cnt = np.array([l.size for l in loops])
    flat = np.concatenate(loops)
    nxt = np.concatenate([np.roll(l, -1) for l in loops])
    owner = np.repeat(np.arange(len(loops)), cnt)
    x0, y0 = V[flat, 0], V[flat, 1]
    x1, y1 = V[nxt, 0], V[nxt, 1]
    cr = x0 * y1 - x1 * y0
    A = np.bincount(owner, cr) * 0.5
    cx = np.bincount(owner, (x0 + x1) * cr) / (6.0 * A)
    cy = np.bincount(owner, (y0 + y1) * cr) / (6.0 * A)
    return np.c_[cx, cy]


def voronoi_square(n_sites: int, seed: int, lloyd: int = 5) -> Mesh2D:
    """Clipped Voronoi mesh of the unit square.

    Sites are drawn uniformly with ``numpy.random.default_rng(seed)`` (PCG64)
    and moved ``lloyd`` times to the area centroid of their clipped cell.
    """

    def build():
        rng = np.random.default_rng(seed)
        sites = rng.random((n_sites, 2))
        for _ in range(lloyd):
            V, loops = _voronoi_cells(sites)
            sites = _loop_centroids(V, loops)
        V, loops = _voronoi_cells(sites)
        vptr = np.zeros(len(loops) + 1, dtype=np.int32)
        vptr[1:] = np.cumsum([l.size for l in loops])
        return {
            "x": np.ascontiguousarray(V[:, 0]),
            "y": np.ascontiguousarray(V[:, 1]),
            "elem_vptr": vptr,
            "elem_v": np.concatenate(loops).astype(np.int32),
        }

    d = _cached(f"voronoi2d:{n_sites}:{seed}:{lloyd}:v1", build)
    return Mesh2D(x=d["x"], y=d["y"], elem_vptr=d["elem_vptr"], elem_v=d["elem_v"])


def rectangle_grid(nx: int, ny: int, x0=0.0, x1=1.0, y0=0.0, y1=1.0) -> Mesh2D:
    """Structured nx-by-ny grid of axis-aligned rectangles (CCW loops)."""
    xs = np.linspace(x0, x1, nx + 1)
    ys = np.linspace(y0, y1, ny + 1)
    X, Y = np.meshgrid(xs, ys, indexing="xy")
    vid = lambda i, j: j * (nx + 1) + i  # noqa: E731
    loops = []
    for j in range(ny):
        for i in range(nx):
            loops.append([vid(i, j), vid(i + 1, j), vid(i + 1, j + 1), vid(i, j + 1)])
    vptr = np.arange(0, 4 * len(loops) + 1, 4, dtype=np.int32)
    return Mesh2D(
        x=X.ravel().astype(np.float64),
        y=Y.ravel().astype(np.float64),
        elem_vptr=vptr,
        elem_v=np.asarray(loops, dtype=np.int32).ravel(),
    )


# ----------------------------------------------------------------------------
# 3D: Kuhn tetrahedra of a structured cube mesh, agglomerated by k-means
# ----------------------------------------------------------------------------

# The six Kuhn tetrahedra of the unit cube: each follows one monotone lattice
# path from corner (0,0,0) to (1,1,1); corners indexed as bit (x | y<<1 | z<<2).
_KUHN_PATHS = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]


def kuhn_cube_tets(n: int):
    """Vertices and tetrahedra of an n^3 cube mesh of [0,1]^3, 6 Kuhn tets/cube."""
    g = np.linspace(0.0, 1.0, n + 1)
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    x, y, z = X.ravel(), Y.ravel(), Z.ravel()
    i, j, k = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()  # i = z index, j = y, k = x

    def vid(dx, dy, dz):
        return ((i + dz) * (n + 1) + (j + dy)) * (n + 1) + (k + dx)

    tets = []
    for path in _KUHN_PATHS:
        c = [0, 0, 0]
        verts = [vid(0, 0, 0)]
        for axis in path:
            c[axis] += 1
            verts.append(vid(c[0], c[1], c[2]))
        tets.append(np.stack(verts, axis=1))
    # order: cube-major, then the 6 tets of that cube
    T = np.stack(tets, axis=1).reshape(-1, 4).astype(np.int32)
    return x, y, z, T


def _tet_face_adjacency(T: np.ndarray):
    """Pairs of tetrahedra sharing a triangle (array [m,2])."""
    faces = np.concatenate([T[:, [1, 2, 3]], T[:, [0, 2, 3]], T[:, [0, 1, 3]], T[:, [0, 1, 2]]])
    owner = np.tile(np.arange(T.shape[0]), 4)
    faces = np.sort(faces, axis=1).astype(np.int64)
    nv = int(faces.max()) + 1
    key = (faces[:, 0] * nv + faces[:, 1]) * nv + faces[:, 2]
    order = np.argsort(key, kind="stable")
    ks = key[order]
    same = ks[1:] == ks[:-1]
    a = owner[order][:-1][same]
    b = owner[order][1:][same]
    return np.c_[a, b]


def kuhn_cube_agglomerated(n: int, n_clusters: int, seed: int, iters: int = 10) -> Mesh3D:
    """Agglomerate the Kuhn tetrahedra of an n^3 cube mesh into polyhedra.

    Seeded k-means (``iters`` Lloyd steps) on tetrahedron centroids, then a
    connectivity repair: every cluster keeps its largest face-connected
    component; each other fragment joins the neighbouring cluster with which it
    shares the most faces, repeated until all clusters are connected.  Empty
    clusters are dropped, so the element count may fall below ``n_clusters``.
    """

    def build():
        from scipy.spatial import cKDTree
        from scipy.sparse import coo_matrix
        from scipy.sparse.csgraph import connected_components

        x, y, z, T = kuhn_cube_tets(n)
        P = np.c_[x, y, z]
        cen = P[T].mean(axis=1)
        rng = np.random.default_rng(seed)
        C = cen[rng.choice(cen.shape[0], size=n_clusters, replace=False)].copy()
        lab = None
        for _ in range(iters):
            _, lab = cKDTree(C).query(cen, workers=-1)
            cnt = np.bincount(lab, minlength=n_clusters)
            for d in range(3):
                s = np.bincount(lab, cen[:, d], minlength=n_clusters)
                nz = cnt > 0
                C[nz, d] = s[nz] / cnt[nz]
        _, lab = cKDTree(C).query(cen, workers=-1)
        lab = lab.astype(np.int64)
        adj = _tet_face_adjacency(T)
        nt = T.shape[0]
        for _round in range(100):
            same = lab[adj[:, 0]] == lab[adj[:, 1]]
            e = adj[same]
            g = coo_matrix((np.ones(e.shape[0]), (e[:, 0], e[:, 1])), shape=(nt, nt))
            ncomp, comp = connected_components(g, directed=False)
            # largest component per cluster
            comp_size = np.bincount(comp, minlength=ncomp)
            comp_lab = np.zeros(ncomp, dtype=np.int64)
            comp_lab[comp] = lab
            best = np.full(n_clusters, -1, dtype=np.int64)
            order = np.lexsort((-comp_size, comp_lab))  # by cluster, size desc
            first = np.ones(order.size, dtype=bool)
            first[1:] = comp_lab[order][1:] != comp_lab[order][:-1]
            best[comp_lab[order][first]] = order[first]
            frag = best[comp_lab] != np.arange(ncomp)  # component is a fragment
            if not frag.any():
                break
            # for each fragment, neighbouring cluster sharing most faces
            cross = ~same
            ea, eb = adj[cross, 0], adj[cross, 1]
            ca, cb = comp[ea], comp[eb]
            src = np.concatenate([ca, cb])
            dst_lab = np.concatenate([lab[eb], lab[ea]])
            m = frag[src]
            src, dst_lab = src[m], dst_lab[m]
            if src.size == 0:
                break
            key = src * (n_clusters + 1) + dst_lab
            uk, cntk = np.unique(key, return_counts=True)
            fsrc = uk // (n_clusters + 1)
            fdst = uk % (n_clusters + 1)
            o = np.lexsort((-cntk, fsrc))
            firstf = np.ones(o.size, dtype=bool)
            firstf[1:] = fsrc[o][1:] != fsrc[o][:-1]
            newlab = comp_lab.copy()
            newlab[fsrc[o][firstf]] = fdst[o][firstf]
            lab = newlab[comp]
        # compact labels; order tets by element
        used, lab = np.unique(lab, return_inverse=True)
        order = np.argsort(lab, kind="stable")
        cnt = np.bincount(lab, minlength=used.size)
        tptr = np.zeros(used.size + 1, dtype=np.int32)
        tptr[1:] = np.cumsum(cnt)
        return {
            "x": x,
            "y": y,
            "z": z,
            "elem_tptr": tptr,
            "tet_v": T[order].ravel().astype(np.int32),
        }

    d = _cached(f"kuhn3d:{n}:{n_clusters}:{seed}:{iters}:v1", build)
    return Mesh3D(x=d["x"], y=d["y"], z=d["z"], elem_tptr=d["elem_tptr"], tet_v=d["tet_v"])


def kuhn_cube_grown(n: int, size: int, seed: int) -> Mesh3D:
    """Agglomerate the Kuhn tetrahedra of an n^3 cube mesh into small
    polyhedra of about ``size`` tetrahedra each, by greedy region growing:
    the tetrahedra are visited in a seeded random order, and each one not yet
    taken starts a new element that grows breadth-first across shared faces
    until it holds ``size`` tetrahedra or has no free neighbour left.  An
    element that stays a single tetrahedron joins the smallest element it
    shares a face with.  Every element is face-connected by construction and
    holds at most 2 size - 1 tetrahedra (k-means with a few tetrahedra per
    cluster fragments, and its repair can chain fragments into very large
    elements)."""

    def build():
        from collections import deque

        x, y, z, T = kuhn_cube_tets(n)
        nt = T.shape[0]
        adj = _tet_face_adjacency(T)
        a = np.concatenate([adj[:, 0], adj[:, 1]])
        b = np.concatenate([adj[:, 1], adj[:, 0]])
        o = np.argsort(a, kind="stable")
        nbr = b[o].astype(np.int64)
        ptr = np.zeros(nt + 1, dtype=np.int64)
        ptr[1:] = np.cumsum(np.bincount(a, minlength=nt))
        nbr_l, ptr_l = nbr.tolist(), ptr.tolist()
        order = np.random.default_rng(seed).permutation(nt).tolist()
        lab = [-1] * nt
        sizes = []
        for t in order:
            if lab[t] >= 0:
                continue
            c = len(sizes)
            lab[t] = c
            cnt = 1
            q = deque([t])
            while q and cnt < size:
                u = q.popleft()
                for v in nbr_l[ptr_l[u]:ptr_l[u + 1]]:
                    if lab[v] < 0 and cnt < size:
                        lab[v] = c
                        cnt += 1
                        q.append(v)
            sizes.append(cnt)
        # single tetrahedra join their smallest neighbouring element
        for t in range(nt):
            c = lab[t]
            if sizes[c] != 1:
                continue
            best = -1
            for v in nbr_l[ptr_l[t]:ptr_l[t + 1]]:
                if lab[v] != c and sizes[lab[v]] < size * 2 - 1 and (best < 0 or sizes[lab[v]] < sizes[best]):
                    best = lab[v]
            if best >= 0:
                sizes[best] += 1
                sizes[c] = 0
                lab[t] = best
        lab = np.asarray(lab, dtype=np.int64)
        used, lab = np.unique(lab, return_inverse=True)
        order_t = np.argsort(lab, kind="stable")
        cnt = np.bincount(lab, minlength=used.size)
        tptr = np.zeros(used.size + 1, dtype=np.int32)
        tptr[1:] = np.cumsum(cnt)
        return {"x": x, "y": y, "z": z, "elem_tptr": tptr, "tet_v": T[order_t].ravel().astype(np.int32)}

    d = _cached(f"kuhn3d_grown:{n}:{size}:{seed}:v1", build)
    return Mesh3D(x=d["x"], y=d["y"], z=d["z"], elem_tptr=d["elem_tptr"], tet_v=d["tet_v"])


def box_tets(nx: int, ny: int, nz: int, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)) -> Mesh3D:
    """Structured box mesh: one element per cube, each cube = 6 Kuhn tets."""
    xs = np.linspace(lo[0], hi[0], nx + 1)
    ys = np.linspace(lo[1], hi[1], ny + 1)
    zs = np.linspace(lo[2], hi[2], nz + 1)
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    vid = lambda i, j, k: (k * (ny + 1) + j) * (nx + 1) + i  # noqa: E731
    tets = []
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                for path in _KUHN_PATHS:
                    c = [0, 0, 0]
                    vs = [vid(i, j, k)]
                    for axis in path:
                        c[axis] += 1
                        vs.append(vid(i + c[0], j + c[1], k + c[2]))
                    tets.append(vs)
    ne = nx * ny * nz
    return Mesh3D(
        x=X.ravel().astype(np.float64),
        y=Y.ravel().astype(np.float64),
        z=Z.ravel().astype(np.float64),
        elem_tptr=np.arange(0, 6 * ne + 1, 6, dtype=np.int32),
        tet_v=np.asarray(tets, dtype=np.int32).ravel(),
    )


# ----------------------------------------------------------------------------
# per-element degrees and coefficients
# ----------------------------------------------------------------------------


def draw_degrees(ne: int, seed: int, lo: int, hi: int) -> np.ndarray:
    """Per-element polynomial degree, uniform on {lo..hi} (int8)."""
    rng = np.random.default_rng(seed + 7919)
    return rng.integers(lo, hi + 1, size=ne).astype(np.int8)


def draw_log_uniform(ne: int, seed: int, lo_exp: float, hi_exp: float) -> np.ndarray:
    """Per-element coefficient 10**U(lo_exp, hi_exp) (float64)."""
    rng = np.random.default_rng(seed + 104729)
    return 10.0 ** rng.uniform(lo_exp, hi_exp, size=ne)
