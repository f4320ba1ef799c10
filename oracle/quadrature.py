"""Gauss rules on the reference tetrahedron and triangle (oracle).

Conical (Stroud) product rules: Gauss-Jacobi nodes in the collapsed
coordinates x = a, y = (1-a) b, z = (1-a)(1-b) c, whose Jacobian (1-a)^2 (1-b)
is absorbed into the Jacobi weights.  q points per direction integrate every
polynomial of total degree <= 2q-1 exactly.  Nodes come from
scipy.special.roots_jacobi.
"""

import numpy as np
from scipy.special import roots_jacobi, roots_legendre


def _gj01(q, alpha):
    """Nodes/weights on [0,1] for the weight (1-t)^alpha."""
    if alpha == 0:
        t, w = roots_legendre(q)
    else:
        t, w = roots_jacobi(q, alpha, 0.0)
    return 0.5 * (1.0 + t), w / 2.0 ** (alpha + 1)


def tet_rule(q):
    """(pts (q^3, 3), wts (q^3,)) on {x,y,z >= 0, x+y+z <= 1}; sum(wts) = 1/6."""
    a, wa = _gj01(q, 2)
    b, wb = _gj01(q, 1)
    c, wc = _gj01(q, 0)
    A, B, C = np.meshgrid(a, b, c, indexing="ij")
    W = wa[:, None, None] * wb[None, :, None] * wc[None, None, :]
    x = A
    y = (1 - A) * B
    z = (1 - A) * (1 - B) * C
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1), W.ravel()


def tri_rule(q):
    """(pts (q^2, 2), wts) on {s,u >= 0, s+u <= 1}; sum(wts) = 1/2."""
    a, wa = _gj01(q, 1)
    b, wb = _gj01(q, 0)
    A, B = np.meshgrid(a, b, indexing="ij")
    W = wa[:, None] * wb[None, :]
    return np.stack([A.ravel(), ((1 - A) * B).ravel()], axis=1), W.ravel()
