"""Dubiner bases on the reference triangle and tetrahedron (oracle).

3D (Sec. 4.2.2):
  phi_ijk(x,y,z) = (1-x-y)^i (1-x)^j P_i(2z/(1-x-y) - 1)
                   P_j^{(2i+1,0)}(2y/(1-x) - 1) P_k^{(2i+2j+2,0)}(2x - 1)
2D (Eq. (4)):
  psi_ij(s,u) = P_i(2u/(1-s) - 1) (1-s)^i P_j^{(2i+1,0)}(2s - 1)

Index order: lexicographic with the first index outermost, total degree <= p.

Evaluation: each factor s^n P_n^{(a,b)}(w/s) is computed without division by
the textbook three-term recurrence of Jacobi polynomials (Abramowitz & Stegun
22.7.1) multiplied through by s^{n+1}.  Gradients are carried along the same
recurrence in forward mode (value and the three partial derivatives of every
intermediate), so no separate derivative identity is used.
"""

import numpy as np


def index3(p):
    """Multi-indices (i,j,k), i+j+k <= p, i outermost, k innermost."""
    return [(i, j, k) for i in range(p + 1) for j in range(p + 1 - i)
            for k in range(p + 1 - i - j)]


def index2(p):
    """Multi-indices (i,j), i+j <= p, i outermost."""
    return [(i, j) for i in range(p + 1) for j in range(p + 1 - i)]


def n3(p):
    return (p + 1) * (p + 2) * (p + 3) // 6 if p >= 0 else 0


def n2(p):
    return (p + 1) * (p + 2) // 2 if p >= 0 else 0


# --- forward-mode "dual" arrays: shape (1 + nd, npts) = value, d/dx_1 .. d/dx_nd ---

def _dmul(a, b):
    out = np.empty_like(a)
    out[0] = a[0] * b[0]
    out[1:] = a[0] * b[1:] + a[1:] * b[0]
    return out


def _scaled_jacobi(nmax, a, b, w, s):
    """[s^n P_n^{(a,b)}(w/s) for n = 0..nmax] as dual arrays (w, s are duals)."""
    one = np.zeros_like(w)
    one[0] = 1.0
    out = [one]
    if nmax == 0:
        return out
    q1 = 0.5 * ((a + b + 2) * w + (a - b) * s)
    out.append(q1)
    s2 = _dmul(s, s)
    for n in range(1, nmax):
        c = 2 * n + a + b
        a1 = 2.0 * (n + 1) * (n + a + b + 1) * c
        a2 = (c + 1.0) * (a * a - b * b)
        a3 = c * (c + 1.0) * (c + 2.0)
        a4 = 2.0 * (n + a) * (n + b) * (c + 2.0)
        lin = a2 * s + a3 * w
        nxt = (_dmul(lin, out[n]) - a4 * _dmul(s2, out[n - 1])) / a1
        out.append(nxt)
    return out


def _linear_dual(coef_grad, const, pts):
    """Dual of the affine function const + coef_grad . x at pts (npts, d)."""
    d = pts.shape[1]
    v = np.empty((1 + d, pts.shape[0]))
    v[0] = const + pts @ np.asarray(coef_grad, dtype=float)
    for r in range(d):
        v[1 + r] = coef_grad[r]
    return v


def phi3(p, pts):
    """Values and reference gradients of phi_ijk, |ijk| <= p, at pts (npts,3).

    Returns (val (N, npts), grad (N, npts, 3)).
    """
    pts = np.asarray(pts, dtype=float)
    s1 = _linear_dual([-1.0, -1.0, 0.0], 1.0, pts)       # 1 - x - y
    w1 = _linear_dual([1.0, 1.0, 2.0], -1.0, pts)        # 2z - (1 - x - y)
    s2 = _linear_dual([-1.0, 0.0, 0.0], 1.0, pts)        # 1 - x
    w2 = _linear_dual([1.0, 2.0, 0.0], -1.0, pts)        # 2y - (1 - x)
    s3 = _linear_dual([0.0, 0.0, 0.0], 1.0, pts)         # 1
    w3 = _linear_dual([2.0, 0.0, 0.0], -1.0, pts)        # 2x - 1
    A = _scaled_jacobi(p, 0, 0, w1, s1)
    idx = index3(p)
    vals = np.empty((len(idx), pts.shape[0]))
    grads = np.empty((len(idx), pts.shape[0], 3))
    cacheB = {}
    cacheC = {}
    for r, (i, j, k) in enumerate(idx):
        if i not in cacheB:
            cacheB[i] = _scaled_jacobi(p - i, 2 * i + 1, 0, w2, s2)
        key = i + j
        if key not in cacheC:
            cacheC[key] = _scaled_jacobi(p - i - j, 2 * i + 2 * j + 2, 0, w3, s3)
        f = _dmul(_dmul(A[i], cacheB[i][j]), cacheC[key][k])
        vals[r] = f[0]
        grads[r] = f[1:].T
    return vals, grads


def psi2(p, pts, grad=False):
    """Values of the face basis psi_ij, |ij| <= p, at pts (npts, 2) = (s, u);
    with grad=True also the gradients (N, npts, 2)."""
    pts = np.asarray(pts, dtype=float)
    s1 = _linear_dual([-1.0, 0.0], 1.0, pts)             # 1 - s
    w1 = _linear_dual([1.0, 2.0], -1.0, pts)             # 2u - (1 - s)
    s3 = _linear_dual([0.0, 0.0], 1.0, pts)
    w3 = _linear_dual([2.0, 0.0], -1.0, pts)             # 2s - 1
    A = _scaled_jacobi(p, 0, 0, w1, s1)
    idx = index2(p)
    vals = np.empty((len(idx), pts.shape[0]))
    grads = np.empty((len(idx), pts.shape[0], 2))
    for r, (i, j) in enumerate(idx):
        B = _scaled_jacobi(p - i, 2 * i + 1, 0, w3, s3)
        f = _dmul(A[i], B[j])
        vals[r] = f[0]
        grads[r] = f[1:].T
    return (vals, grads) if grad else vals


def legendre(n, x):
    """P_0..P_n at x (plain three-term recurrence), shape (n+1, len(x))."""
    x = np.asarray(x, dtype=float)
    out = np.empty((n + 1, x.size))
    out[0] = 1.0
    if n >= 1:
        out[1] = x
    for m in range(1, n):
        out[m + 1] = ((2 * m + 1) * x * out[m] - m * out[m - 1]) / (m + 1)
    return out
