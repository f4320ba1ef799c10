"""Energy-conserving DG operator for 2D (TE) Maxwell on triangles (oracle, FP64).

Test infrastructure: the plain, slow definition that a 2D triangle solver is
checked against; nothing of the product imports it.

The fields of the 2D TE problem are E = (E_x, E_y) in the plane and H = H_z;
with curl E = d_x E_y - d_y E_x (a scalar) and curl H = (d_y H, -d_x H):
eps dE/dt = curl H, mu dH/dt = -curl E.  The scheme is the central-flux system
of Sec. 2.1, written for these fields with the same sign reading as the 3D
oracle (oracle/dg.py):

  d/dt (eps E, e)_T = (H, curl e)_T - ({{H}}, n x e)_dT
  d/dt (mu H, h)_T  = -(curl E, h)_T + (1/2 n x [[E]], h)_dT

with n the outward unit normal of T, n x v = n_x v_y - n_y v_x (the tangential
component of v), [[E]] = E_T - E_nbr and {{H}} = (H_T + H_nbr)/2 on dT; on a
PEC edge the ghost state is E_nbr = -E_T (tangentially), H_nbr = H_T.  The 3D
facet terms -(1/2 [[E]] x nu, h) and -({{H}} x nu, e) reduce to these for
fields in the plane and H along z.

Spaces (Sec. 2: V^{k+1} x V^k): E of degree p, covariant (Sec. 3.2.1),
E|_T(x) = F^{-T} sum_a c_{m,a} e_m psi_a(Phi^{-1} x), m = 0, 1; H of degree
p - 1, a scalar, H|_T(x) = sum_b d_b psi_b(Phi^{-1} x); psi the 2D Dubiner
basis of Eq. (4) on the reference triangle, Phi(xh) = X0 + F xh with the
triangle's vertices ordered by ascending key.  Every integral is a Gauss sum in
physical space; a neighbour's basis is evaluated at the same physical point
through the neighbour's own inverse map (shifted across a periodic wrap).

Layouts: E[t, m, a], H[t, b].
"""

import numpy as np
import scipy.linalg as sl
import scipy.sparse as sps
from scipy.special import roots_legendre

from .basis import n2, psi2
from .quadrature import tri_rule


class Geometry2D:
    """Element maps, edge adjacency (with periodic shifts) and outward normals."""

    def __init__(self, xy, tris, vertex_key=None):
        xy = np.asarray(xy, dtype=float)
        tris = np.asarray(tris, dtype=np.int64)
        key = np.arange(xy.shape[0]) if vertex_key is None else np.asarray(vertex_key, dtype=np.int64)
        order = np.argsort(key[tris], axis=1, kind="stable")
        self.tris = np.take_along_axis(tris, order, axis=1)
        self.keys = key[self.tris]
        if np.any(self.keys[:, 1:] == self.keys[:, :-1]):
            raise ValueError("triangle with repeated vertex keys")
        self.X = xy[self.tris]                                        # (nt, 3, 2)
        self.X0 = self.X[:, 0, :]
        self.F = np.stack([self.X[:, 1] - self.X0, self.X[:, 2] - self.X0], axis=2)
        self.detF = np.linalg.det(self.F)
        if np.any(np.abs(self.detF) <= 1e-14):
            raise ValueError("degenerate triangle")
        self.Finv = np.linalg.inv(self.F)
        self.nt = self.tris.shape[0]
        # edge f: the two vertices other than local vertex f
        self.edge_local = [tuple(v for v in range(3) if v != f) for f in range(3)]
        owners = {}
        for t in range(self.nt):
            for f in range(3):
                a, b = self.edge_local[f]
                owners.setdefault((self.keys[t, a], self.keys[t, b]), []).append((t, f))
        self.nbr = -np.ones((self.nt, 3), dtype=np.int64)
        self.nbr_edge = -np.ones((self.nt, 3), dtype=np.int64)
        self.shift = np.zeros((self.nt, 3, 2))
        for k, lst in owners.items():
            if len(lst) > 2:
                raise ValueError("edge shared by more than two triangles")
            if len(lst) == 2:
                (t1, f1), (t2, f2) = lst
                if t1 == t2:
                    raise ValueError("triangle glued to itself")
                for (ta, fa), (tb, fb) in (((t1, f1), (t2, f2)), ((t2, f2), (t1, f1))):
                    self.nbr[ta, fa] = tb
                    self.nbr_edge[ta, fa] = fb
                    # same key -> same vertex of the edge on both sides: the translation
                    # carrying this side's copy of the edge onto the neighbour's
                    va = self.edge_local[fa][0]
                    vb = self.edge_local[fb][0]
                    self.shift[ta, fa] = self.X[tb, vb] - self.X[ta, va]
        # outward unit normals and lengths
        self.normal = np.zeros((self.nt, 3, 2))
        self.length = np.zeros((self.nt, 3))
        for f in range(3):
            a, b = self.edge_local[f]
            d = self.X[:, b] - self.X[:, a]
            L = np.linalg.norm(d, axis=1)
            n = np.stack([d[:, 1], -d[:, 0]], axis=1) / L[:, None]
            away = np.einsum("tc,tc->t", n, self.X[:, f] - self.X[:, a]) > 0
            n[away] *= -1.0
            self.normal[:, f] = n
            self.length[:, f] = L


def _cross_n(n, v):
    """n x v = n_x v_y - n_y v_x for v[..., 2]."""
    return n[0] * v[..., 1] - n[1] * v[..., 0]


class OracleDG2D:
    def __init__(self, xy, tris, p, eps, mu, vertex_key=None):
        if p < 1:
            raise ValueError("p >= 1 required")
        self.geo = Geometry2D(xy, tris, vertex_key)
        self.p = p
        self.pH = p - 1
        self.nt = self.geo.nt
        self.NE = n2(p)
        self.NH = n2(p - 1)
        self.eps = np.broadcast_to(np.asarray(eps, dtype=float), (self.nt,)).copy()
        self.mu = np.broadcast_to(np.asarray(mu, dtype=float), (self.nt,)).copy()
        if np.any(self.eps <= 0) or np.any(self.mu <= 0):
            raise ValueError("eps, mu must be positive")
        q = p + 2
        self.vq, self.vw = tri_rule(q)
        s, w = roots_legendre(q)
        self.lq, self.lw = 0.5 * (s + 1.0), 0.5 * w
        self._assembled = None

    @property
    def sizeE(self):
        return self.nt * 2 * self.NE

    @property
    def sizeH(self):
        return self.nt * self.NH

    # ------------------------------------------------------------ basis values
    def _xhat(self, t, x):
        return (x - self.geo.X0[t]) @ self.geo.Finv[t].T

    def _E_values(self, t, xhat, curl=False):
        """N[a, m, q, c] = (F^{-T} e_m)_c psi_a(xhat_q), and curl N[a, m, q]."""
        Finv = self.geo.Finv[t]
        vals, grads = psi2(self.p, xhat, grad=True)
        N = np.einsum("mc,aq->amqc", Finv, vals)
        if not curl:
            return N
        pg = np.einsum("dc,aqd->aqc", Finv, grads)                      # physical gradients
        # curl(psi v) = grad psi x v for the constant vector v = F^{-T} e_m
        cN = pg[:, None, :, 0] * Finv[None, :, None, 1] - pg[:, None, :, 1] * Finv[None, :, None, 0]
        return N, cN

    def _H_values(self, xhat):
        return psi2(self.pH, xhat)

    # ---------------------------------------------------------------- blocks
    def element_blocks(self, t):
        """Volume terms VH = -(curl E, h)_T (H rows), VE = (H, curl e)_T (E rows),
        masses ME, MH of element t."""
        g = self.geo
        x = g.X0[t] + self.vq @ g.F[t].T
        w = self.vw * abs(g.detF[t])
        xh = self._xhat(t, x)
        N, cN = self._E_values(t, xh, curl=True)
        psiH = self._H_values(xh)
        NE, NH = self.NE, self.NH
        VH = -np.einsum("q,amq,bq->bma", w, cN, psiH).reshape(NH, 2 * NE)
        VE = np.einsum("q,bq,amq->mab", w, psiH, cN).reshape(2 * NE, NH)
        ME = self.eps[t] * np.einsum("q,amqc,dlqc->mald", w, N, N).reshape(2 * NE, 2 * NE)
        MH = self.mu[t] * np.einsum("q,bq,dq->bd", w, psiH, psiH)
        return VH, VE, ME, MH

    def edge_blocks(self, t, f):
        """Edge f of element t: AH_own, AH_nbr (H rows of t, E columns of t / of the
        neighbour) and AE_own, AE_nbr (E rows of t, H columns of t / neighbour)."""
        g = self.geo
        a, b = g.edge_local[f]
        Xa, Xb = g.X[t, a], g.X[t, b]
        x = Xa[None, :] + self.lq[:, None] * (Xb - Xa)[None, :]
        w = self.lw * g.length[t, f]
        n = g.normal[t, f]
        xh = self._xhat(t, x)
        nN = _cross_n(n, self._E_values(t, xh))                          # (A, 2, Q)
        psiH = self._H_values(xh)
        NE, NH = self.NE, self.NH
        nb = g.nbr[t, f]
        own = 0.5 if nb >= 0 else 1.0     # PEC: 1/2 n x (E - E_ghost) = n x E, {{H}} = H
        out = dict(nbr=nb)
        out["AH_own"] = own * np.einsum("q,bq,amq->bma", w, psiH, nN).reshape(NH, 2 * NE)
        out["AE_own"] = -own * np.einsum("q,amq,bq->mab", w, nN, psiH).reshape(2 * NE, NH)
        if nb >= 0:
            xn = self._xhat(nb, x + g.shift[t, f])
            nNn = _cross_n(n, self._E_values(nb, xn))
            psiHn = self._H_values(xn)
            out["AH_nbr"] = -0.5 * np.einsum("q,bq,amq->bma", w, psiH, nNn).reshape(NH, 2 * NE)
            out["AE_nbr"] = -0.5 * np.einsum("q,amq,bq->mab", w, nN, psiHn).reshape(2 * NE, NH)
        return out

    def assemble(self):
        if self._assembled is not None:
            return self._assembled
        NE, NH = self.NE, self.NH
        rh, ch, vh, re, ce, ve = [], [], [], [], [], []
        ME = np.empty((self.nt, 2 * NE, 2 * NE))
        MH = np.empty((self.nt, NH, NH))
        eH = lambda t: np.arange(NH) + NH * t
        eE = lambda t: np.arange(2 * NE) + 2 * NE * t

        def add(rows, cols, vals, R, C, V):
            rows.append(np.repeat(R, len(C)))
            cols.append(np.tile(C, len(R)))
            vals.append(V.ravel())

        for t in range(self.nt):
            VH, VE, ME[t], MH[t] = self.element_blocks(t)
            add(rh, ch, vh, eH(t), eE(t), VH)
            add(re, ce, ve, eE(t), eH(t), VE)
            for f in range(3):
                e = self.edge_blocks(t, f)
                add(rh, ch, vh, eH(t), eE(t), e["AH_own"])
                add(re, ce, ve, eE(t), eH(t), e["AE_own"])
                if e["nbr"] >= 0:
                    add(rh, ch, vh, eH(t), eE(e["nbr"]), e["AH_nbr"])
                    add(re, ce, ve, eE(t), eH(e["nbr"]), e["AE_nbr"])
        cat = np.concatenate
        CH = sps.csr_matrix((cat(vh), (cat(rh), cat(ch))), shape=(self.sizeH, self.sizeE))
        CE = sps.csr_matrix((cat(ve), (cat(re), cat(ce))), shape=(self.sizeE, self.sizeH))
        self._assembled = dict(CH=CH, CE=CE, ME=ME, MH=MH, MEinv=np.linalg.inv(ME), MHinv=np.linalg.inv(MH))
        return self._assembled

    @staticmethod
    def _blockmul(Mb, v):
        nb, m, _ = Mb.shape
        return np.einsum("bij,bj->bi", Mb, v.reshape(nb, m)).ravel()

    # -------------------------------------------------------- time stepping
    def run(self, E0, H0, dt, nsteps):
        """Leapfrog of Sec. 3 with opening and closing half kicks of H; returns
        E^N, H^N and W^n = 1/2 E^n M E^n + 1/2 H^{n-1/2} M H^{n+1/2}, n = 0..N."""
        A = self.assemble()
        E = np.array(E0, dtype=float)
        H = np.array(H0, dtype=float)
        kick = lambda E: dt * self._blockmul(A["MHinv"], A["CH"] @ E)
        dH = kick(E)
        lo, hi = H - 0.5 * dH, H + 0.5 * dH
        W = [0.5 * E @ self._blockmul(A["ME"], E) + 0.5 * lo @ self._blockmul(A["MH"], hi)]
        H = hi
        for _ in range(nsteps):
            E = E + dt * self._blockmul(A["MEinv"], A["CE"] @ H)
            dH = kick(E)
            W.append(0.5 * E @ self._blockmul(A["ME"], E) + 0.5 * H @ self._blockmul(A["MH"], H + dH))
            H = H + dH
        H = H - 0.5 * dH
        return E, H, np.array(W)

    # ----------------------------------------------------------- projection
    def project(self, fE=None, fH=None, q=None):
        """Coefficients of the L2 projections of fE(x) -> (..., 2) onto the covariant
        degree-p space and of fH(x) -> (...) onto the degree p-1 space."""
        q = q or self.p + 4
        xq, wq = tri_rule(q)
        g = self.geo
        E = np.zeros((self.nt, 2 * self.NE)) if fE is not None else None
        H = np.zeros((self.nt, self.NH)) if fH is not None else None
        A = self.assemble()
        for t in range(self.nt):
            x = g.X0[t] + xq @ g.F[t].T
            w = wq * abs(g.detF[t])
            if fE is not None:
                N = self._E_values(t, xq)
                rhs = np.einsum("q,amqc,qc->ma", w, N, fE(x)).ravel()
                E[t] = np.linalg.solve(A["ME"][t] / self.eps[t], rhs)
            if fH is not None:
                psi = self._H_values(xq)
                H[t] = np.linalg.solve(A["MH"][t] / self.mu[t], psi @ (w * fH(x)))
        return (E.ravel() if E is not None else None), (H.ravel() if H is not None else None)

    def l2_error(self, E, fE, q=None):
        """||E_h - fE||_{L2} and ||fE||_{L2} by quadrature."""
        q = q or self.p + 4
        xq, wq = tri_rule(q)
        g = self.geo
        E = E.reshape(self.nt, 2, self.NE)
        err = ref = 0.0
        for t in range(self.nt):
            x = g.X0[t] + xq @ g.F[t].T
            w = wq * abs(g.detF[t])
            N = self._E_values(t, xq)
            Eh = np.einsum("ma,amqc->qc", E[t], N)
            ex = fE(x)
            err += w @ ((Eh - ex) ** 2).sum(1)
            ref += w @ (ex ** 2).sum(1)
        return np.sqrt(err), np.sqrt(ref)

    # ------------------------------------------------------------ spectrum
    def resonances(self):
        """Frequencies omega >= 0 of the semi-discrete operator (dense): omega^2 are
        the eigenvalues of M_E^{-1} C_H^T M_H^{-1} C_H (which equals
        -M_E^{-1} C_E M_H^{-1} C_H by skew-adjointness)."""
        A = self.assemble()
        CH = A["CH"].toarray()
        K = CH.T @ sl.block_diag(*A["MHinv"]) @ CH
        lam = sl.eigh(0.5 * (K + K.T), sl.block_diag(*A["ME"]), eigvals_only=True)
        return np.sqrt(np.clip(lam, 0.0, None))
