"""L2 projection of point-wise fields and L2 errors (oracle).

Projection onto the covariant space of one element: find c with
(N c, N_b)_T = (u, N_b)_T for all covariant basis functions N_b, integrals by a
Gauss rule with q = p + 4 points per direction, mass solved by Cholesky.
"""

import numpy as np

from .basis import phi3
from .quadrature import tet_rule
from .dg import _covariant_values


def project(dg, fn, degree, q=None, chunk=256):
    """Coefficients (nt*3*N,) of the L2 projection of fn(x) -> (..., 3) onto the
    covariant space of the given degree, canonical layout [t][m][a]."""
    g = dg.geo
    q = q or dg.p + 4
    xq, wq = tet_rule(q)
    phi, _ = phi3(degree, xq)
    A = phi.shape[0]
    out = np.empty((dg.nt, 3 * A))
    for s in range(0, dg.nt, chunk):
        ts = np.arange(s, min(dg.nt, s + chunk))
        N = _covariant_values(g.Finv[ts], phi)                      # (B,A,3,Q,3)
        w = wq[None, :] * np.abs(g.detF[ts])[:, None]
        x = g.to_phys(ts[:, None], xq[None, :, :])                  # (B,Q,3)
        u = fn(x)                                                   # (B,Q,3)
        b = np.einsum("bq,bamqc,bqc->bma", w, N, u).reshape(len(ts), 3 * A)
        M = np.einsum("bq,bamqc,bdlqc->bmald", w, N, N).reshape(len(ts), 3 * A, 3 * A)
        L = np.linalg.cholesky(M)
        y = np.linalg.solve(L, b[..., None])
        out[ts] = np.linalg.solve(np.swapaxes(L, 1, 2), y)[..., 0]
    return out.ravel()


def l2_error(dg, coef, fn, degree, q=None, chunk=256):
    """(||u_h - u||_L2, ||u||_L2) with u_h = sum coef N, by a q = p+4 Gauss rule."""
    g = dg.geo
    q = q or dg.p + 4
    xq, wq = tet_rule(q)
    phi, _ = phi3(degree, xq)
    A = phi.shape[0]
    c = np.asarray(coef).reshape(dg.nt, 3, A)
    err2 = 0.0
    ref2 = 0.0
    for s in range(0, dg.nt, chunk):
        ts = np.arange(s, min(dg.nt, s + chunk))
        N = _covariant_values(g.Finv[ts], phi)
        w = wq[None, :] * np.abs(g.detF[ts])[:, None]
        x = g.to_phys(ts[:, None], xq[None, :, :])
        uh = np.einsum("bamqc,bma->bqc", N, c[ts])
        u = fn(x)
        err2 += np.einsum("bq,bqc->", w, (uh - u) ** 2)
        ref2 += np.einsum("bq,bqc->", w, u ** 2)
    return np.sqrt(err2), np.sqrt(ref2)


def point_values(dg, coef, degree, t, xh):
    """Physical field values of element t at reference points xh (n,3)."""
    phi, _ = phi3(degree, xh)
    A = phi.shape[0]
    c = np.asarray(coef).reshape(dg.nt, 3, A)[t]                    # (3,A)
    # u = F^{-T} sum_a c[:,a] phi_a
    return (dg.geo.Finv[t].T @ (c @ phi)).T
