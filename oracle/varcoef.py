"""Material parameters that vary inside an element: the exact mass and the
approximate inverse mass of Sec. 3.3.2 (oracle, FP64; test infrastructure).

With eps(x) not constant on an element T the mass matrix of Sec. 3.3.1 is no
longer block diagonal in the basis.  For a flat element, with the covariant
basis N_{a,m} = F^{-T} e_m phi'_a (phi' orthonormal on the reference element),

  M_{(a,m),(b,l)} = int_T eps N_{a,m} . N_{b,l} dx = |det F| G_{ml} (E_eps)_{ab},
  G = F^{-1} F^{-T},  (E_eps)_{ab} = int_Th eps(Phi(xh)) phi'_a phi'_b dxh,

so M^{-1} = |det F|^{-1} G^{-1} (x) E_eps^{-1}.  Sec. 3.3.2 replaces E_eps^{-1}
by the operator of two quadrature steps: "reverse numerical integration" turns
the functional values s_b into point values f_i = sum_b phi'_b(x_i) s_b (the
ones whose quadrature reproduces s exactly), these are divided by eps(x_i), and
numerical integration gives u_a = sum_i w_i phi'_a(x_i) f_i / eps(x_i).  That is
the mass matrix of 1/eps, E_{1/eps}: symmetric positive definite, exact when eps
is constant on the element.  The time loop with it conserves the energy in the
norm of the approximate mass (E_{1/eps})^{-1}.

Functions here take an oracle.dg.OracleDG (flat elements) and a coefficient
function c(x, t) -> (Q,) for the points x (Q, 3) of element t (piecewise smooth
parameters may depend on the element).
"""

import numpy as np

from .basis import phi3
from .quadrature import tet_rule


def _points(dg, t, q):
    xq, wq = tet_rule(q)
    g = dg.geo
    x = g.X0[t] + xq @ g.F[t].T
    return xq, wq, x


def weighted_reference_mass(dg, t, coef, degree, q):
    """(E_c)_{ab} = int_Th c(Phi(xh)) phi'_a phi'_b dxh for element t."""
    xq, wq, x = _points(dg, t, q)
    phi, _ = phi3(degree, xq)
    nrm = np.sqrt(np.einsum("q,aq,aq->a", wq, phi, phi))
    phi = phi / nrm[:, None]
    return np.einsum("q,aq,bq->ab", wq * coef(x, t), phi, phi)


def exact_mass_blocks(dg, coef, which="E", q=None):
    """Per element the mass with the varying coefficient, (nt, 3A, 3A), in the
    printed covariant basis (the layout of OracleDG.assemble()["ME"])."""
    q = q or dg.p + 6
    deg = dg.p if which == "E" else dg.pH
    g = dg.geo
    out = []
    for t in range(dg.nt):
        xq, wq, x = _points(dg, t, q)
        phi, _ = phi3(deg, xq)
        N = np.einsum("mc,aq->amqc", g.Finv[t], phi)          # covariant printed basis
        w = wq * abs(g.detF[t]) * coef(x, t)
        A = phi.shape[0]
        out.append(np.einsum("q,amqc,dlqc->mald", w, N, N).reshape(3 * A, 3 * A))
    return np.array(out)


def approx_inverse_blocks(dg, coef, which="E", q=None):
    """Per element the approximate inverse mass of Sec. 3.3.2, (nt, 3A, 3A), for
    the printed covariant basis: the two quadrature steps (reverse integration,
    division by the coefficient at the points, integration) applied to each
    unit functional, composed with |det F|^{-1} G^{-1} and the basis norms."""
    q = q or dg.p + 6
    deg = dg.p if which == "E" else dg.pH
    g = dg.geo
    xq, wq = tet_rule(q)
    phi, _ = phi3(deg, xq)
    nrm = np.sqrt(np.einsum("q,aq,aq->a", wq, phi, phi))
    phio = phi / nrm[:, None]                                  # orthonormal on the reference element
    A = phi.shape[0]
    out = []
    for t in range(dg.nt):
        x = g.X0[t] + xq @ g.F[t].T
        c = coef(x, t)
        # reverse numerical integration of each unit functional s = e_b, then / c, then integration
        S = np.eye(A)
        f_pts = phio.T @ S                                     # (Q, A): point values per functional
        U = phio @ (wq[:, None] * f_pts / c[:, None])          # (A, A) = E_{1/c}
        G = g.Finv[t] @ g.Finv[t].T
        Ginv = np.linalg.inv(G)
        # printed basis: coefficient c_a = c'_a / ||phi_a||, functional r_a = ||phi_a|| r'_a
        Uprint = U / np.outer(nrm, nrm)
        out.append(np.kron(Ginv, Uprint) / abs(g.detF[t]))
    return np.array(out)


def run(dg, ME, MEinv, E0, H0, dt, nsteps):
    """Leapfrog of Sec. 3 (central flux) with the given E-mass blocks ME and the
    inverse blocks MEinv used in the update; returns E^N, H^N and the energies
    W^n = 1/2 E^n ME E^n + 1/2 H^{n-1/2} MH H^{n+1/2}."""
    A = dg.assemble()
    bm = dg._blockmul
    E = np.array(E0, dtype=float)
    H = np.array(H0, dtype=float)
    kick = lambda E: dt * bm(A["MHinv"], A["CH"] @ E)
    dH = kick(E)
    lo, hi = H - 0.5 * dH, H + 0.5 * dH
    W = [0.5 * E @ bm(ME, E) + 0.5 * lo @ bm(A["MH"], hi)]
    H = hi
    for _ in range(nsteps):
        E = E + dt * bm(MEinv, A["CE"] @ H)
        dH = kick(E)
        W.append(0.5 * E @ bm(ME, E) + 0.5 * H @ bm(A["MH"], H + dH))
        H = H + dH
    H = H - 0.5 * dH
    return E, H, np.array(W)
