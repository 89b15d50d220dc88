"""Named synthetic workloads shaped like the paper's test bodies (Sec. 4).

Each workload bundles a mesh, a quadrature rule (points per triangle), a
seeded nodal magnetisation, the oversampled FFT grid, the arithmetic
precision and the relative L2 tolerance it is judged at.

  cube     unit cube, 8x8 squares per face (768 triangles, 386 nodes), 3-point
           rule, m = (1,0,0) + U[-0.1,0.1]^3 renormalised, grid 32^3, FP64,
           tolerance 1e-10.  (Paper: cube runs, Sec. 4 / Table 4.)
  sphere   icosphere level 5, R = 1 (20480 triangles, 10242 nodes), 7-point
           rule, vortex m with N(0, 0.05^2) noise, grid 128^3, FP32,
           tolerance 1e-5.  (Paper: uniformly magnetised sphere, Sec. 4.)
  plate    2000 x 500 x 20 box, 5x5 squares (168000 triangles, 84002 nodes),
           3-point rule, smooth random m, grid 512x128x16 requested, FP32,
           tolerance 1e-5.  (Paper: thin film, Table 3.)
  batched  64 smooth random states on the level-5 sphere, plus 16 meshes of
           uneven size (cubes, spheres, plates; ~1.2k to ~200k triangles) with
           4 states each (batched_items).
  served   eight resident meshes (cube, sphere, plate, torus; ~2k to 1.92M
           triangles) with their grids (served_pool).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import fields, meshes


@dataclass
class Workload:
    name: str
    V: np.ndarray
    T: np.ndarray
    quad: int
    m_nodal: np.ndarray
    grid: tuple
    precision: int
    tolerance: float
    seed: int
    info: dict = field(default_factory=dict)

    @property
    def n_targets(self) -> int:
        return int(self.V.shape[0])

    @property
    def n_sources(self) -> int:
        return int(self.T.shape[0]) * self.quad


def cube(nper: int = 8, grid=(32, 32, 32), precision: int = 64, tolerance: float = 1e-10,
         index: int = 0) -> Workload:
    V, T = meshes.cube(nper)
    seed = fields.workload_seed(index)
    m = fields.perturbed_uniform(V, seed)
    return Workload(f"cube{nper}", V, T, 3, m, tuple(grid), precision, tolerance, seed)


def cube_large(nper: int = 400, grid=(1024, 1024, 1024), precision: int = 32, tolerance: float = 1e-5,
               index: int = 5) -> Workload:
    """Largest serving mesh: unit cube, nper x nper squares per face (1.92M
    triangles at 400), 3-point rule, smooth random field."""
    V, T = meshes.cube(nper)
    seed = fields.workload_seed(index)
    m = fields.smooth_random(V, seed)
    return Workload(f"cube{nper}", V, T, 3, m, tuple(grid), precision, tolerance, seed)


def sphere(level: int = 5, grid=(128, 128, 128), precision: int = 32, tolerance: float = 1e-5,
           quad: int = 7, index: int = 1) -> Workload:
    V, T = meshes.icosphere(level, 1.0)
    seed = fields.workload_seed(index)
    m = fields.vortex(V, seed)
    return Workload(f"sphere_L{level}", V, T, quad, m, tuple(grid), precision, tolerance, seed)


def plate(dims=(2000.0, 500.0, 20.0), cell: float = 5.0, grid=(512, 128, 16), precision: int = 32,
          tolerance: float = 1e-5, index: int = 2) -> Workload:
    n = tuple(int(round(d / cell)) for d in dims)
    V, T = meshes.box(*dims, *n)
    seed = fields.workload_seed(index)
    m = fields.smooth_random(V, seed)
    return Workload(f"plate_{int(dims[0])}x{int(dims[1])}x{int(dims[2])}", V, T, 3, m, tuple(grid),
                    precision, tolerance, seed)


def torus(R=2.0, r=0.5, nu=64, nv=32, grid=(128, 128, 64), precision=32, tolerance=1e-5,
          index: int = 4) -> Workload:
    V, T = meshes.torus(R, r, nu, nv)
    seed = fields.workload_seed(index)
    m = fields.smooth_random(V, seed)
    return Workload(f"torus_{nu}x{nv}", V, T, 3, m, tuple(grid), precision, tolerance, seed)


def batched_items():
    """(name, V, T, q, grid or None for autotuned, [nodal m states]) of the
    batched workload: 64 seeded smooth states on the level-5 sphere at 128^3,
    plus 16 meshes of uneven size (cubes, spheres, plates; ~1.2k to ~200k
    triangles) with 4 states each."""
    items = []
    V, T = meshes.icosphere(5)
    items.append(("sphere_L5", V, T, 7, (128, 128, 128), [fields.smooth_random(V, 7000 + i) for i in range(64)]))
    shapes = [("cube10", meshes.cube(10), 3), ("cube20", meshes.cube(20), 3), ("cube40", meshes.cube(40), 3),
              ("cube70", meshes.cube(70), 3), ("cube100", meshes.cube(100), 3), ("cube128", meshes.cube(128), 3),
              ("sphere_L3", meshes.icosphere(3), 7), ("sphere_L4", meshes.icosphere(4), 7),
              ("sphere_L5b", meshes.icosphere(5, 2.0), 3), ("sphere_L6", meshes.icosphere(6), 3),
              ("sphere_L4b", meshes.icosphere(4, 0.5), 3),
              ("plate_a", meshes.box(400.0, 100.0, 4.0, 40, 10, 2), 3),
              ("plate_b", meshes.box(1000.0, 250.0, 10.0, 100, 25, 2), 3),
              ("plate_c", meshes.box(2000.0, 500.0, 20.0, 200, 50, 2), 3),
              ("plate_d", meshes.box(1000.0, 1000.0, 20.0, 150, 150, 3), 3),
              ("plate_e", meshes.box(2000.0, 500.0, 20.0, 300, 75, 3), 3)]
    for k, (name, (V, T), q) in enumerate(shapes):
        items.append((name, V, T, q, None, [fields.smooth_random(V, 8000 + 10 * k + i) for i in range(4)]))
    return items


def served_pool():
    """(name, (V, T), q, grid) of the eight resident meshes of the served
    workload: cube, sphere, plates and tori, ~2k to 1.92M triangles (the
    largest a unit cube with 400 x 400 squares per face)."""
    return [("cube13", meshes.cube(13), 3, (64, 64, 64)),
            ("sphere_L5", meshes.icosphere(5), 7, (128, 128, 128)),
            ("plate_2000x500x20_c10", meshes.box(2000.0, 500.0, 20.0, 200, 50, 2), 3, (512, 128, 128)),
            ("torus_400x100", meshes.torus(2.0, 0.5, 400, 100), 3, (256, 256, 128)),
            ("sphere_L6", meshes.icosphere(6), 3, (256, 256, 256)),
            ("plate_2000x500x20_c5", meshes.box(2000.0, 500.0, 20.0, 400, 100, 4), 3, (512, 256, 256)),
            ("torus_800x200", meshes.torus(2.0, 0.5, 800, 200), 3, (512, 512, 256)),
            ("cube400", meshes.cube(400), 3, (1024, 1024, 1024))]
