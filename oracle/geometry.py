"""Element maps, facet adjacency and physical normals (oracle).

Coefficient convention (an interface definition shared with the CUDA path,
not a computational shortcut): the four vertices of every tetrahedron are
ordered by ascending vertex key (the periodic identification key, or the
vertex id when there is none); the element map is Phi(xh) = X0 + F xh with
F = [X1-X0, X2-X0, X3-X0] (Sec. 3.2.1); fields are F^{-T} sum_a c_a phi_a.

Everything else here is computed directly in physical space: faces are
matched by their key triples, the periodic translation between the two copies
of a face is read off the vertex coordinates, outward normals come from cross
products oriented away from the opposite vertex.
"""

import numpy as np


class Geometry:
    def __init__(self, xyz, tets, vertex_key=None):
        xyz = np.asarray(xyz, dtype=float)
        tets = np.asarray(tets, dtype=np.int64)
        nt = tets.shape[0]
        key = np.arange(xyz.shape[0]) if vertex_key is None else np.asarray(vertex_key, dtype=np.int64)
        order = np.argsort(key[tets], axis=1, kind="stable")
        self.tets = np.take_along_axis(tets, order, axis=1)
        self.keys = key[self.tets]
        if np.any(self.keys[:, 1:] == self.keys[:, :-1]):
            raise ValueError("tetrahedron with repeated vertex keys")
        self.X = xyz[self.tets]                                   # (nt, 4, 3)
        self.X0 = self.X[:, 0, :]
        self.F = np.stack([self.X[:, 1] - self.X0, self.X[:, 2] - self.X0,
                           self.X[:, 3] - self.X0], axis=2)      # columns = edges
        self.detF = np.linalg.det(self.F)
        if np.any(np.abs(self.detF) <= 1e-14):
            raise ValueError("degenerate tetrahedron")
        self.Finv = np.linalg.inv(self.F)
        self.nt = nt

        # face f = opposite local vertex f
        self.face_local = [tuple(v for v in range(4) if v != f) for f in range(4)]
        table = {}
        for t in range(nt):
            for f in range(4):
                kt = tuple(self.keys[t, list(self.face_local[f])])
                table.setdefault(kt, []).append((t, f))
        self.nbr = -np.ones((nt, 4), dtype=np.int64)
        self.nbr_face = -np.ones((nt, 4), dtype=np.int64)
        self.shift = np.zeros((nt, 4, 3))
        self.faces = []          # list of (key triple, [(t,f), ...])
        for kt, lst in table.items():
            if len(lst) > 2:
                raise ValueError("face shared by more than two tetrahedra")
            self.faces.append((kt, sorted(lst)))
            if len(lst) == 2:
                (t0, f0), (t1, f1) = lst
                self.nbr[t0, f0], self.nbr_face[t0, f0] = t1, f1
                self.nbr[t1, f1], self.nbr_face[t1, f1] = t0, f0
                a0 = self.X[t0, self.face_local[f0][0]]
                a1 = self.X[t1, self.face_local[f1][0]]
                self.shift[t0, f0] = a1 - a0
                self.shift[t1, f1] = a0 - a1
        self.faces.sort(key=lambda e: e[1][0])

        # physical outward unit normals and face areas
        self.normal = np.zeros((nt, 4, 3))
        self.area2 = np.zeros((nt, 4))       # |t1 x t2| = 2 * area
        for f in range(4):
            a, b, c = self.face_local[f]
            t1 = self.X[:, b] - self.X[:, a]
            t2 = self.X[:, c] - self.X[:, a]
            n = np.cross(t1, t2)
            ln = np.linalg.norm(n, axis=1)
            n = n / ln[:, None]
            towards = np.einsum("ti,ti->t", n, self.X[:, f] - self.X[:, a])
            n[towards > 0] *= -1.0
            self.normal[:, f] = n
            self.area2[:, f] = ln

    def to_ref(self, t, x):
        """Reference coordinates of physical points x (..., 3) in element(s) t."""
        return np.einsum("...ij,...j->...i", self.Finv[t], x - self.X0[t])

    def to_phys(self, t, xh):
        return self.X0[t] + np.einsum("...ij,...j->...i", self.F[t], xh)
