"""Structured tetrahedral meshes of the unit cube (Kuhn subdivision).

Each of the n^3 sub-cubes with lower corner v and edge h = 1/n is split into
the six tetrahedra conv{v, v + h e_a, v + h (e_a + e_b), v + h (1,1,1)} over
the six orderings (a, b, c) of the axes.  The split is translation invariant,
so the mesh is conforming and also conforming across a periodic wrap.

Optional inputs follow the workload descriptions of the time-domain examples:
interior vertices jittered by U[-a, a]^3 (boundary vertices stay on the cube
faces), periodic identification keys for the box [0,1]^3, and a seeded shuffle
of the vertex order inside each tetrahedron (the discretisation re-sorts the
vertices itself; the shuffle exercises that).
"""

from dataclasses import dataclass
from itertools import permutations
from typing import Optional

import numpy as np


@dataclass
class KuhnMesh:
    n: int
    xyz: np.ndarray                 # (nv, 3) float64 vertex coordinates
    tets: np.ndarray                # (nt, 4) int32 vertex ids
    vertex_key: Optional[np.ndarray]  # (nv,) int32 periodic identification, or None
    period: Optional[np.ndarray]    # (3,) float64 box periods, or None

    @property
    def nv(self):
        return self.xyz.shape[0]

    @property
    def nt(self):
        return self.tets.shape[0]

    @property
    def h(self):
        return 1.0 / self.n


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def kuhn_cube_mesh(n, jitter=0.0, seed=None, periodic=False, shuffle_local=False):
    """Kuhn mesh of [0,1]^3 with n cubes per direction (6 n^3 tetrahedra).

    jitter: maximal interior vertex displacement as a fraction of h.
    periodic: add vertex keys identifying opposite faces of the box.
    shuffle_local: permute the 4 vertex ids of every tet (seeded).
    """
    if n < 1:
        raise ValueError("n must be >= 1")
    h = 1.0 / n
    m = n + 1
    ii, jj, kk = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
    # vertex id = i + m*(j + m*k)
    vid = lambda i, j, k: i + m * (j + m * k)
    xyz = np.zeros((m ** 3, 3))
    ids = vid(ii, jj, kk).ravel()
    xyz[ids, 0] = ii.ravel() * h
    xyz[ids, 1] = jj.ravel() * h
    xyz[ids, 2] = kk.ravel() * h

    rng = _rng(seed if seed is not None else 0)
    if jitter > 0.0:
        a = jitter * h
        interior = ((ii > 0) & (ii < n) & (jj > 0) & (jj < n) & (kk > 0) & (kk < n)).ravel()
        disp = rng.uniform(-a, a, size=(m ** 3, 3))
        sel = ids[interior]
        xyz[sel] += disp[interior]

    unit = np.eye(3, dtype=np.int64)
    tets = []
    for ck in range(n):
        for cj in range(n):
            for ci in range(n):
                base = np.array([ci, cj, ck])
                for perm in permutations(range(3)):
                    p0 = base
                    p1 = p0 + unit[perm[0]]
                    p2 = p1 + unit[perm[1]]
                    p3 = base + 1
                    tets.append([vid(*p0), vid(*p1), vid(*p2), vid(*p3)])
    tets = np.asarray(tets, dtype=np.int64)

    if shuffle_local:
        for t in range(tets.shape[0]):
            tets[t] = tets[t, rng.permutation(4)]

    key = None
    period = None
    if periodic:
        ki = (ii % n) + n * ((jj % n) + n * (kk % n))
        key = np.zeros(m ** 3, dtype=np.int64)
        key[ids] = ki.ravel()
        key = key.astype(np.int32)
        period = np.ones(3)
        # only vertices referenced by tets matter; all are referenced here.
    return KuhnMesh(n=n, xyz=xyz, tets=tets.astype(np.int32), vertex_key=key, period=period)


def workload_mesh(n, jitter_frac, seed, periodic=False, shuffle_local=False):
    """Mesh used by the named time-domain workloads (see workloads.configs)."""
    return kuhn_cube_mesh(n, jitter=jitter_frac, seed=seed, periodic=periodic,
                          shuffle_local=shuffle_local)
