"""Structured triangle meshes of the unit square.

Each of the n^2 cells with lower-left corner v and edge h = 1/n is split along
its diagonal into conv{v, v + h e_x, v + h (1,1)} and conv{v, v + h (1,1),
v + h e_y}.  The split is translation invariant, so the mesh is conforming and
also conforming across a periodic wrap.  As for the tetrahedral meshes:
interior vertices may be jittered by U[-a, a]^2 (boundary vertices stay on the
square's edges), opposite edges may be identified by periodic keys, and the
vertex order inside each triangle may be shuffled (seeded).
"""

from dataclasses import dataclass
from typing import Optional

import numpy as np


@dataclass
class TriMesh:
    n: int
    xy: np.ndarray                   # (nv, 2) float64 vertex coordinates
    tris: np.ndarray                 # (nt, 3) int32 vertex ids
    vertex_key: Optional[np.ndarray]  # (nv,) int32 periodic identification, or None

    @property
    def nv(self):
        return self.xy.shape[0]

    @property
    def nt(self):
        return self.tris.shape[0]

    @property
    def h(self):
        return 1.0 / self.n


def square_tri_mesh(n, jitter=0.0, seed=None, periodic=False, shuffle_local=False):
    """Triangle mesh of [0,1]^2 with n cells per direction (2 n^2 triangles)."""
    if n < 1:
        raise ValueError("n must be >= 1")
    h = 1.0 / n
    m = n + 1
    ii, jj = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")
    vid = lambda i, j: i + m * j
    ids = vid(ii, jj).ravel()
    xy = np.zeros((m * m, 2))
    xy[ids, 0] = ii.ravel() * h
    xy[ids, 1] = jj.ravel() * h
    rng = np.random.Generator(np.random.PCG64(seed if seed is not None else 0))
    if jitter > 0.0:
        a = jitter * h
        interior = ((ii > 0) & (ii < n) & (jj > 0) & (jj < n)).ravel()
        disp = rng.uniform(-a, a, size=(m * m, 2))
        xy[ids[interior]] += disp[interior]
    tris = []
    for cj in range(n):
        for ci in range(n):
            v0, v1, v2, v3 = vid(ci, cj), vid(ci + 1, cj), vid(ci + 1, cj + 1), vid(ci, cj + 1)
            tris.append((v0, v1, v2))
            tris.append((v0, v2, v3))
    tris = np.array(tris, dtype=np.int32)
    if shuffle_local:
        for t in range(tris.shape[0]):
            tris[t] = tris[t][rng.permutation(3)]
    key = None
    if periodic:
        key = vid(ii % n, jj % n).ravel()[np.argsort(ids)].astype(np.int32)
    return TriMesh(n=n, xy=xy, tris=tris, vertex_key=key)
