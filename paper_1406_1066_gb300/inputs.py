"""Seeded synthetic inputs for sparse assembly (shared by tests, bench and smoke).

This module only draws index triplets and values; it holds none of the
assembly arithmetic.  Every array is produced on the host with numpy's
``Generator(PCG64(seed))`` and is returned as contiguous int32 (unit-offset
indices) and float64 (values).

Workloads (shapes follow the paper's problem class, §1 and §4.2: FEM
assembly with many collisions, and random triplets):

* ``mesh2d(N)``: structured N x N vertex grid of the unit square, each cell
  split into two triangles (p00,p10,p11) and (p00,p11,p01); vertex id
  1 + x + N*y (x fastest), cells in the same order; element e emits its
  local 3x3 matrix row-major, triplet k = 9e + 3a + b with i = v_a, j = v_b.
* ``mesh3d(N)``: structured N^3 vertex cube, each cell split into the 6
  Kuhn tetrahedra, one per axis permutation in lexicographic order
  (xyz, xzy, yxz, yzx, zxy, zyx): (v000, v000+e1, v000+e1+e2, v111);
  vertex id 1 + x + N*y + N^2*z; triplet k = 16e + 4a + b.
* ``uniform(...)``: iid uniform rows and columns, N(0,1) values.
* ``pooled(...)``: draws from a fixed pool of distinct pairs (high collision).
* ``ransparse(...)``: the paper's benchmark generator (§4.2, listing
  "Benchmark data generator"): every row repeated nnz_row times, uniform
  columns, every pair replicated nrep times, a random permutation, values 1.
* ``batch(...)``: many uneven 2D/3D mesh instances.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


@dataclass
class Triplets:
    ii: np.ndarray            # int32[L], unit-offset rows
    jj: np.ndarray            # int32[L], unit-offset columns
    s: np.ndarray             # float64[L]
    m: int
    n: int
    nzmax: int = 0
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def L(self) -> int:
        return int(self.ii.size)


def mesh2d_elements(N: int) -> np.ndarray:
    """Triangle connectivity (E x 3, unit-offset vertex ids) of the N x N grid."""
    c = np.arange(N - 1)
    x, y = np.meshgrid(c, c, indexing="xy")          # x fastest after ravel
    x, y = x.ravel(), y.ravel()
    p00 = 1 + x + N * y
    p10, p01, p11 = p00 + 1, p00 + N, p00 + N + 1
    t0 = np.stack([p00, p10, p11], axis=1)
    t1 = np.stack([p00, p11, p01], axis=1)
    tri = np.stack([t0, t1], axis=1).reshape(-1, 3)  # element e = 2*cell + t
    return tri.astype(np.int32)


_KUHN = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]


def mesh3d_elements(N: int) -> np.ndarray:
    """Kuhn tetrahedra (E x 4, unit-offset vertex ids) of the N^3 cube."""
    c = np.arange(N - 1)
    z, y, x = np.meshgrid(c, c, c, indexing="ij")   # x fastest after ravel
    base = (1 + x + N * y + N * N * z).ravel()
    step = [1, N, N * N]
    tets = np.empty((base.size, 6, 4), np.int64)
    for t, (a, b, _) in enumerate(_KUHN):
        tets[:, t, 0] = base
        tets[:, t, 1] = base + step[a]
        tets[:, t, 2] = base + step[a] + step[b]
        tets[:, t, 3] = base + 1 + N + N * N
    return tets.reshape(-1, 4).astype(np.int32)


def _element_triplets(elem: np.ndarray):
    """Local dense element matrices, row-major: k = d*d*e + d*a + b."""
    d = elem.shape[1]
    ii = np.repeat(elem, d, axis=1).ravel()
    jj = np.tile(elem, (1, d)).ravel()
    return np.ascontiguousarray(ii, np.int32), np.ascontiguousarray(jj, np.int32)


def mesh2d(N: int, seed: int, name: str = "") -> Triplets:
    ii, jj = _element_triplets(mesh2d_elements(N))
    s = _rng(seed).uniform(-1.0, 1.0, ii.size)
    return Triplets(ii, jj, s, N * N, N * N, 0, name or f"mesh2d_{N}", {"N": N, "dim": 2})


def mesh3d(N: int, seed: int, name: str = "") -> Triplets:
    ii, jj = _element_triplets(mesh3d_elements(N))
    s = _rng(seed).uniform(-1.0, 1.0, ii.size)
    return Triplets(ii, jj, s, N ** 3, N ** 3, 0, name or f"mesh3d_{N}", {"N": N, "dim": 3})


def mesh_values(L: int, seed: int) -> np.ndarray:
    """Fresh U(-1,1) values for re-assembly steps of a fixed pattern."""
    return _rng(seed).uniform(-1.0, 1.0, L)


def uniform(m: int, n: int, L: int, seed: int, name: str = "") -> Triplets:
    g = _rng(seed)
    ii = g.integers(1, m + 1, L, dtype=np.int32)
    jj = g.integers(1, n + 1, L, dtype=np.int32)
    s = g.standard_normal(L)
    return Triplets(ii, jj, s, m, n, 0, name or f"uniform_{m}x{n}_{L}")


def pooled(m: int, n: int, L: int, pool: int, seed: int, name: str = "") -> Triplets:
    """L draws from a pool of ``pool`` distinct pairs (kept in first-drawn order)."""
    g = _rng(seed)
    keys = np.empty(0, np.int64)
    while keys.size < pool:
        need = pool - keys.size
        bi = g.integers(0, m, need + need // 8 + 64, dtype=np.int64)
        bj = g.integers(0, n, bi.size, dtype=np.int64)
        cand = np.concatenate([keys, bj * m + bi])
        _, first = np.unique(cand, return_index=True)
        keys = cand[np.sort(first)]
    keys = keys[:pool]
    pi = (keys % m + 1).astype(np.int32)
    pj = (keys // m + 1).astype(np.int32)
    idx = g.integers(0, pool, L, dtype=np.int64)
    s = g.standard_normal(L)
    return Triplets(np.ascontiguousarray(pi[idx]), np.ascontiguousarray(pj[idx]), s, m, n, 0,
                    name or f"pooled_{m}x{n}_{L}_{pool}", {"pool": pool})


def ransparse(siz: int, nnz_row: int, nrep: int, seed: int) -> Triplets:
    """The paper's benchmark generator (§4.2), values all ones."""
    g = _rng(seed)
    ii = np.tile(np.arange(1, siz + 1, dtype=np.int32), nnz_row)
    jj = g.integers(1, siz + 1, siz * nnz_row, dtype=np.int32)
    ii, jj = np.tile(ii, nrep), np.tile(jj, nrep)
    p = g.permutation(ii.size)
    return Triplets(np.ascontiguousarray(ii[p]), np.ascontiguousarray(jj[p]),
                    np.ones(ii.size), siz, siz, 0, f"ransparse_{siz}_{nnz_row}_{nrep}")


def random_small(L: int, m: int, n: int, seed: int, dup: float = 0.3,
                 values: str = "normal") -> Triplets:
    """Tiny random triplets with forced duplicates (test cases)."""
    g = _rng(seed)
    ii = g.integers(1, m + 1, L, dtype=np.int32)
    jj = g.integers(1, n + 1, L, dtype=np.int32)
    if L > 1 and dup > 0:
        src = g.integers(0, L, L)
        take = g.random(L) < dup
        ii = np.where(take, ii[src], ii).astype(np.int32)
        jj = np.where(take, jj[src], jj).astype(np.int32)
    if values == "normal":
        s = g.standard_normal(L)
    elif values == "int":
        s = g.integers(-8, 9, L).astype(np.float64)
    else:
        s = np.ones(L)
    return Triplets(ii, jj, s, m, n, 0, f"random_{L}_{m}x{n}")


@dataclass
class Batch:
    instances: List[Triplets]

    @property
    def L(self) -> int:
        return sum(t.L for t in self.instances)


def batch(count: int, seed: int, side2d=(16, 128), side3d=(8, 40)) -> Batch:
    """Uneven 2D/3D mesh instances: fair coin for the kind, side uniform (inclusive)."""
    g = _rng(seed)
    kinds = g.integers(0, 2, count)
    sides = [int(g.integers(side2d[0], side2d[1] + 1)) if k == 0 else
             int(g.integers(side3d[0], side3d[1] + 1)) for k in kinds]
    out = []
    for b, (k, N) in enumerate(zip(kinds, sides)):
        vseed = seed * 1000 + b + 1
        out.append(mesh2d(N, vseed) if k == 0 else mesh3d(N, vseed))
    return Batch(out)


# Named workloads (seeds fixed here; sizes as the benchmark configurations).
def workload(name: str, small: Optional[int] = None) -> Triplets:
    if name == "mesh2d_64":
        return mesh2d(64, 1406, name)
    if name == "uniform_1e6":
        return uniform(10**6, 10**6, 2 * 10**7, 1407, name)
    if name == "pooled_2e4":
        return pooled(20000, 20000, 2 * 10**7, 2 * 10**6, 1408, name)
    if name == "mesh3d_100":
        return mesh3d(100, 1409, name)
    if name == "mesh3d_60":
        return mesh3d(60, 1413, name)
    if name.startswith("mesh3d_"):
        return mesh3d(int(name.split("_")[1]), 1400 + int(name.split("_")[1]), name)
    raise KeyError(name)
