"""Seeded synthetic workloads (inputs only: meshes, degrees, coefficients).

Each workload names its mesh generator, per-element degree and diffusion
coefficient draws, and the constant problem data (advection b, reaction c,
manufactured source, penalty constant).  Nothing here computes any part of
the assembly; the oracle and the CUDA library consume the same inputs.

Workloads (stand-ins for the paper's meshes, which are not available):
  poisson2d_1k     unit square, 1,024 Voronoi cells (5 Lloyd steps), p = 2,
                   a = 1, b = 0, c = 0, u = sin(pi x) sin(pi y)
  adr2d_65k        65,536 Voronoi cells, p ~ U{1..4}, a = 10^U(-2, 2),
                   b = (1, 0.5), c = 1
  diff3d_32k       64^3 cubes x 6 Kuhn tetrahedra agglomerated by k-means
                   into 32,768 polyhedra, p = 3, a = 10^U(-2, 2), b = 0, c = 0
  batch2d_256      256 meshes, cell counts log-uniform in 512..16,384,
                   per-mesh p ~ U{1..5}
  adr3d_varcoef    50^3 cubes x 6 Kuhn tetrahedra grown into polyhedra of
                   about 4 tetrahedra, p = 3, a = 0.01, the fields of Sec. 4.2
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List

import numpy as np

from . import meshgen as mg

SRC_ZERO, SRC_SINPROD, SRC_POLY = 0, 1, 2


@dataclasses.dataclass
class Workload:
    name: str
    mesh: object  # meshgen.Mesh2D | meshgen.Mesh3D
    p: np.ndarray  # int8 [ne]
    a: np.ndarray  # float64 [ne]
    problem: Dict  # b, c, source, poly, c_sigma

    @property
    def dim(self) -> int:
        return self.mesh.dim

    @property
    def ne(self) -> int:
        return self.mesh.ne


def poisson2d(n_sites: int = 1024, seed: int = 0) -> Workload:
    m = mg.voronoi_square(n_sites, seed)
    return Workload(
        name=f"poisson2d_{n_sites}",
        mesh=m,
        p=np.full(m.ne, 2, dtype=np.int8),
        a=np.ones(m.ne),
        problem=dict(b=(0.0, 0.0, 0.0), c=0.0, source=SRC_SINPROD, poly=[], c_sigma=10.0),
    )


def adr2d(n_sites: int = 65536, seed: int = 1, plo: int = 1, phi: int = 4) -> Workload:
    m = mg.voronoi_square(n_sites, seed)
    return Workload(
        name=f"adr2d_{n_sites}",
        mesh=m,
        p=mg.draw_degrees(m.ne, seed, plo, phi),
        a=mg.draw_log_uniform(m.ne, seed, -2.0, 2.0),
        problem=dict(b=(1.0, 0.5, 0.0), c=1.0, source=SRC_SINPROD, poly=[], c_sigma=10.0),
    )


def diff3d(n: int = 64, clusters: int = 32768, seed: int = 2, p: int = 3) -> Workload:
    m = mg.kuhn_cube_agglomerated(n, clusters, seed)
    return Workload(
        name=f"diff3d_{n}cubed_{clusters}",
        mesh=m,
        p=np.full(m.ne, p, dtype=np.int8),
        a=mg.draw_log_uniform(m.ne, seed, -2.0, 2.0),
        problem=dict(b=(0.0, 0.0, 0.0), c=0.0, source=SRC_SINPROD, poly=[], c_sigma=10.0),
    )


def _batch_member(k: int, lo: int, hi: int, pmax: int, base_seed: int):
    s = base_seed + k
    rng = np.random.default_rng(10_000 + s)
    n = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
    pm = int(rng.integers(1, pmax + 1))
    return n, s, pm


def _gen_member(args):
    n, s = args
    mg.voronoi_square(n, s)  # fills the mesh cache
    return True


def batch2d(n_meshes: int = 256, lo: int = 512, hi: int = 16384, pmax: int = 5, base_seed: int = 3,
            workers: int = 0) -> List[Workload]:
    """Independent 2D meshes; mesh k uses seed base_seed + k, cell count
    round(exp(U(ln lo, ln hi))) and degree U{1..pmax} from rng(10000 + seed).

    Missing meshes are generated in a spawned process pool (workers = 0: all
    cores) and cached, so the serial pass below only reads the cache."""
    members = [_batch_member(k, lo, hi, pmax, base_seed) for k in range(n_meshes)]
    if workers >= 0 and mg._cache_dir() is not None:
        import concurrent.futures as cf
        import multiprocessing as mp
        import os

        nw = workers or (os.cpu_count() or 1)
        if nw > 1:
            todo = [(n, s) for n, s, _ in members]
            todo.sort(key=lambda t: -t[0])
            with cf.ProcessPoolExecutor(max_workers=nw, mp_context=mp.get_context("spawn")) as ex:
                list(ex.map(_gen_member, todo, chunksize=1))
    out = []
    for k, (n, s, pm) in enumerate(members):
        m = mg.voronoi_square(n, s)
        out.append(
            Workload(
                name=f"batch2d_{k}",
                mesh=m,
                p=np.full(m.ne, pm, dtype=np.int8),
                a=mg.draw_log_uniform(m.ne, s, -2.0, 2.0),
                problem=dict(b=(1.0, 0.5, 0.0), c=1.0, source=SRC_SINPROD, poly=[], c_sigma=10.0),
            )
        )
    return out


def learned2d(n_sites: int = 262144, seed: int = 4) -> Workload:
    """Learned-quadrature test mesh: p = 3 everywhere (28-point rules are exact
    for its volume integrands), coefficients as adr2d."""
    m = mg.voronoi_square(n_sites, seed)
    return Workload(
        name=f"learned2d_{n_sites}",
        mesh=m,
        p=np.full(m.ne, 3, dtype=np.int8),
        a=mg.draw_log_uniform(m.ne, seed, -2.0, 2.0),
        problem=dict(b=(1.0, 0.5, 0.0), c=1.0, source=SRC_SINPROD, poly=[], c_sigma=10.0),
    )


def learned_training_meshes(n_meshes: int = 16, n_sites: int = 65536, base_seed: int = 1000,
                            workers: int = 0) -> List[Workload]:
    """Training polygons for the rule-proposal network: n_meshes independent
    Voronoi meshes (seeds base_seed + k), p = 3; generated in a spawned pool."""
    if workers >= 0 and mg._cache_dir() is not None:
        import concurrent.futures as cf
        import multiprocessing as mp
        import os

        nw = workers or (os.cpu_count() or 1)
        if nw > 1:
            with cf.ProcessPoolExecutor(max_workers=nw, mp_context=mp.get_context("spawn")) as ex:
                list(ex.map(_gen_member, [(n_sites, base_seed + k) for k in range(n_meshes)]))
    out = []
    for k in range(n_meshes):
        m = mg.voronoi_square(n_sites, base_seed + k)
        out.append(Workload(f"train_{k}", m, np.full(m.ne, 3, dtype=np.int8), np.ones(m.ne),
                            dict(b=(0.0, 0.0, 0.0), c=0.0, source=SRC_ZERO, poly=[], c_sigma=10.0)))
    return out


def adr3d_varcoef(n: int = 50, size: int = 4, seed: int = 7, p: int = 3) -> Workload:
    """The 3D problem of Sec. 4.2 on an agglomerated tetrahedral mesh: A =
    0.01 I, b = (1+x, 1+y, 1+z), c = 3 + xyz (the fields come from the
    variable-coefficient call; the mesh carries b = 0, c = 0), u = sin(pi x)
    sin(pi y) sin(pi z).  50^3 cubes x 6 Kuhn tets = 750,000 tets grown into
    polyhedra of about 4 tets (184,628 elements; the paper's p = 3 case has
    197k elements of 786k tets)."""
    m = mg.kuhn_cube_grown(n, size, seed)
    return Workload(
        name=f"adr3d_varcoef_{n}cubed_{size}tets",
        mesh=m,
        p=np.full(m.ne, p, dtype=np.int8),
        a=np.full(m.ne, 0.01),
        problem=dict(b=(0.0, 0.0, 0.0), c=0.0, source=SRC_SINPROD, poly=[], c_sigma=10.0),
    )


def small2d(n_sites: int, seed: int, plo: int, phi: int, b=(0.8, -0.45), c: float = 0.7,
            source: int = SRC_SINPROD, poly=(), neumann: int = 0) -> Workload:
    """Small mixed-degree 2D case for parity tests."""
    m = mg.voronoi_square(n_sites, seed)
    return Workload(
        name=f"small2d_{n_sites}_{seed}",
        mesh=m,
        p=mg.draw_degrees(m.ne, seed, plo, phi),
        a=mg.draw_log_uniform(m.ne, seed, -2.0, 2.0),
        problem=dict(b=(b[0], b[1], 0.0), c=c, source=source, poly=list(poly), c_sigma=10.0, neumann=neumann),
    )


def small3d(n: int, clusters: int, seed: int, plo: int, phi: int, b=(0.6, -0.3, 0.45), c: float = 0.5,
            source: int = SRC_SINPROD, poly=(), neumann: int = 0) -> Workload:
    """Small agglomerated 3D case for parity tests."""
    m = mg.kuhn_cube_agglomerated(n, clusters, seed)
    return Workload(
        name=f"small3d_{n}_{clusters}_{seed}",
        mesh=m,
        p=mg.draw_degrees(m.ne, seed, plo, phi),
        a=mg.draw_log_uniform(m.ne, seed, -1.0, 1.0),
        problem=dict(b=tuple(b), c=c, source=source, poly=list(poly), c_sigma=10.0, neumann=neumann),
    )
