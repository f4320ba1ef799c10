"""Curved elements (Sec. 3.3.2): the central-flux operator of Sec. 2.1 on a
conforming tetrahedral mesh deformed by a smooth global map, with the exact
mass and the approximate inverse mass (oracle, FP64; test infrastructure).

The mesh is an affine tetrahedral mesh in coordinates y; the physical domain is
x = Psi(y) for a smooth map Psi with det DPsi > 0, so element T has the map
Phi_T(xh) = Psi(X0 + F xh) with Jacobian J(xh) = DPsi(y) F, and both sides of a
face meet at the same y (plus a periodic shift), which keeps the mesh conforming.
Fields are covariant through the element map (Sec. 3.2.1 with J in place of F):
E|_T = J^{-T} sum_a c_{m,a} e_m phi_a, H likewise with degree p - 1.  Every
integral is a Gauss sum over the reference element (volumes) or reference face
(faces) with the physical measure; curl by the Piola identity
curl(J^{-T} v) = det(J)^{-1} J curlh(v); on a face the physical normal is
DPsi^{-T} n_y / |DPsi^{-T} n_y| and the surface element |det DPsi| |DPsi^{-T} n_y|
times the flat one (Nanson's formula), n_y the face's outward normal in y.
The facet terms and the PEC ghost state are those of oracle/dg.py.

Masses are no longer block diagonal in the basis: the exact ones are dense per
element and inverted directly; the approximate inverse of Sec. 3.3.2 inverts the
pointwise metric instead:  M~^{-1} = sum_i w_i (phi'_i phi'_i^T) (x) J_i^T J_i /
(c_i |det J_i|), exact when J and the coefficient c are constant on the element.
"""

import numpy as np
import scipy.sparse as sps

from .basis import phi3
from .geometry import Geometry
from .quadrature import tet_rule, tri_rule


class CurvedDG:
    def __init__(self, xyz, tets, p, eps, mu, psi, dpsi, vertex_key=None, q=None):
        """psi(y) -> x and dpsi(y) -> DPsi for points y (..., 3)."""
        if p < 1:
            raise ValueError("p >= 1 required")
        self.geo = Geometry(xyz, tets, vertex_key)
        self.psi, self.dpsi = psi, dpsi
        self.p, self.pH = p, p - 1
        self.nt = self.geo.nt
        self.eps = np.broadcast_to(np.asarray(eps, dtype=float), (self.nt,)).copy()
        self.mu = np.broadcast_to(np.asarray(mu, dtype=float), (self.nt,)).copy()
        q = q or p + 3
        self.vq, self.vw = tet_rule(q)
        self.fq, self.fw = tri_rule(q)
        self.phiE, self.gE = phi3(p, self.vq)
        self.phiH, self.gH = phi3(p - 1, self.vq)
        self.NE, self.NH = self.phiE.shape[0], self.phiH.shape[0]
        self._assembled = None

    @property
    def sizeE(self):
        return self.nt * 3 * self.NE

    @property
    def sizeH(self):
        return self.nt * 3 * self.NH

    # ------------------------------------------------------------ element maps
    def _jac(self, t, xh):
        g = self.geo
        y = g.X0[t] + xh @ g.F[t].T
        J = self.dpsi(y) @ g.F[t]                               # (Q, 3, 3)
        return y, J

    @staticmethod
    def _cov(J, vals):
        """N[a, m, q, c] = (J_q^{-T} e_m)_c vals[a, q]."""
        Jinv = np.linalg.inv(J)
        return np.einsum("qmc,aq->amqc", Jinv, vals)

    @staticmethod
    def _curl(J, grads):
        """curl N_{a,m} = det(J)^{-1} J (gradh phi_a x e_m), (A, 3, Q, 3)."""
        detJ = np.linalg.det(J)
        A, Q, _ = grads.shape
        out = np.empty((A, 3, Q, 3))
        for m in range(3):
            em = np.zeros(3)
            em[m] = 1.0
            ref = np.cross(grads, em)                           # (A, Q, 3)
            out[:, m] = np.einsum("qcd,aqd->aqc", J, ref) / detJ[None, :, None]
        return out

    # ---------------------------------------------------------------- blocks
    def element_blocks(self, t):
        _, J = self._jac(t, self.vq)
        w = self.vw * np.abs(np.linalg.det(J))
        NE = self._cov(J, self.phiE)
        NH = self._cov(J, self.phiH)
        cE = self._curl(J, self.gE)
        A, B = self.NE, self.NH
        VH = -np.einsum("q,amqc,blqc->lbma", w, cE, NH).reshape(3 * B, 3 * A)
        VE = np.einsum("q,blqc,amqc->malb", w, NH, cE).reshape(3 * A, 3 * B)
        ME = self.eps[t] * np.einsum("q,amqc,dlqc->mald", w, NE, NE).reshape(3 * A, 3 * A)
        MH = self.mu[t] * np.einsum("q,amqc,dlqc->mald", w, NH, NH).reshape(3 * B, 3 * B)
        return VH, VE, ME, MH

    def face_blocks(self, t, f):
        g = self.geo
        a, b, c = g.face_local[f]
        Xa, Xb, Xc = g.X[t, a], g.X[t, b], g.X[t, c]
        y = Xa[None, :] + self.fq[:, 0:1] * (Xb - Xa)[None, :] + self.fq[:, 1:2] * (Xc - Xa)[None, :]
        D = self.dpsi(y)
        ny = g.normal[t, f]
        m = np.einsum("qdc,d->qc", np.linalg.inv(D), ny)        # DPsi^{-T} n_y
        lm = np.linalg.norm(m, axis=1)
        nu = m / lm[:, None]
        ws = self.fw * g.area2[t, f] * np.abs(np.linalg.det(D)) * lm
        xh = (y - g.X0[t]) @ g.Finv[t].T
        J = D @ g.F[t]
        vE, _ = phi3(self.p, xh)
        vH, _ = phi3(self.pH, xh)
        NEo, NHo = self._cov(J, vE), self._cov(J, vH)
        nb = g.nbr[t, f]
        cown = 0.5 if nb >= 0 else 1.0
        cr = lambda N: np.cross(N, nu[None, None, :, :])
        A, B = self.NE, self.NH
        out = dict(nbr=nb)
        out["AH_own"] = -cown * np.einsum("q,amqc,blqc->lbma", ws, cr(NEo), NHo).reshape(3 * B, 3 * A)
        out["AE_own"] = -cown * np.einsum("q,blqc,amqc->malb", ws, cr(NHo), NEo).reshape(3 * A, 3 * B)
        if nb >= 0:
            yn = y + g.shift[t, f]
            xn = (yn - g.X0[nb]) @ g.Finv[nb].T
            Jn = self.dpsi(yn) @ g.F[nb]
            vEn, _ = phi3(self.p, xn)
            vHn, _ = phi3(self.pH, xn)
            NEn, NHn = self._cov(Jn, vEn), self._cov(Jn, vHn)
            out["AH_nbr"] = 0.5 * np.einsum("q,amqc,blqc->lbma", ws, cr(NEn), NHo).reshape(3 * B, 3 * A)
            out["AE_nbr"] = -0.5 * np.einsum("q,blqc,amqc->malb", ws, cr(NHn), NEo).reshape(3 * A, 3 * B)
        return out

    def assemble(self):
        if self._assembled is not None:
            return self._assembled
        A, B = self.NE, self.NH
        rh, ch, vh, re, ce, ve = [], [], [], [], [], []
        ME = np.empty((self.nt, 3 * A, 3 * A))
        MH = np.empty((self.nt, 3 * B, 3 * B))
        iE = lambda t: np.arange(3 * A) + 3 * A * t
        iH = lambda t: np.arange(3 * B) + 3 * B * t

        def add(rows, cols, vals, R, C, V):
            rows.append(np.repeat(R, len(C)))
            cols.append(np.tile(C, len(R)))
            vals.append(V.ravel())

        for t in range(self.nt):
            VH, VE, ME[t], MH[t] = self.element_blocks(t)
            add(rh, ch, vh, iH(t), iE(t), VH)
            add(re, ce, ve, iE(t), iH(t), VE)
            for f in range(4):
                e = self.face_blocks(t, f)
                add(rh, ch, vh, iH(t), iE(t), e["AH_own"])
                add(re, ce, ve, iE(t), iH(t), e["AE_own"])
                if e["nbr"] >= 0:
                    add(rh, ch, vh, iH(t), iE(e["nbr"]), e["AH_nbr"])
                    add(re, ce, ve, iE(t), iH(e["nbr"]), e["AE_nbr"])
        cat = np.concatenate
        CH = sps.csr_matrix((cat(vh), (cat(rh), cat(ch))), shape=(self.sizeH, self.sizeE))
        CE = sps.csr_matrix((cat(ve), (cat(re), cat(ce))), shape=(self.sizeE, self.sizeH))
        self._assembled = dict(CH=CH, CE=CE, ME=ME, MH=MH, MEinv=np.linalg.inv(ME), MHinv=np.linalg.inv(MH))
        return self._assembled

    def approx_inverse(self, which="E"):
        """The approximate inverse mass of Sec. 3.3.2 per element, printed basis."""
        phi = self.phiE if which == "E" else self.phiH
        coef = self.eps if which == "E" else self.mu
        nrm = np.sqrt(np.einsum("q,aq,aq->a", self.vw, phi, phi))
        po = phi / nrm[:, None]
        A = phi.shape[0]
        out = np.empty((self.nt, 3 * A, 3 * A))
        for t in range(self.nt):
            _, J = self._jac(t, self.vq)
            K = np.einsum("qdm,qdl->qml", J, J) / (coef[t] * np.abs(np.linalg.det(J)))[:, None, None]
            U = np.einsum("q,aq,bq,qml->malb", self.vw, po, po, K).reshape(3 * A, 3 * A)
            out[t] = U / np.outer(np.tile(nrm, 3), np.tile(nrm, 3))
        return out

    @staticmethod
    def _blockmul(Mb, v):
        nb, m, _ = Mb.shape
        return np.einsum("bij,bj->bi", Mb, v.reshape(nb, m)).ravel()

    def run(self, E0, H0, dt, nsteps, MEinv=None):
        """Leapfrog of Sec. 3; MEinv: the inverse E-mass blocks used in the update
        (default the exact ones); energies in the norm of their inverse."""
        A = self.assemble()
        MEinv = A["MEinv"] if MEinv is None else MEinv
        ME = A["ME"] if MEinv is A["MEinv"] else np.linalg.inv(MEinv)
        bm = self._blockmul
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

    # ----------------------------------------------------------- projection
    def project(self, fn, which="E"):
        """L2 projection of fn(x) -> (..., 3) onto the covariant space."""
        phi = self.phiE if which == "E" else self.phiH
        A = phi.shape[0]
        out = np.empty((self.nt, 3 * A))
        for t in range(self.nt):
            y, J = self._jac(t, self.vq)
            w = self.vw * np.abs(np.linalg.det(J))
            N = self._cov(J, phi)
            G = np.einsum("q,amqc,dlqc->mald", w, N, N).reshape(3 * A, 3 * A)
            rhs = np.einsum("q,amqc,qc->ma", w, N, fn(self.psi(y))).ravel()
            out[t] = np.linalg.solve(G, rhs)
        return out.ravel()

    def l2_error(self, E, fn):
        E = E.reshape(self.nt, 3, self.NE)
        err = ref = 0.0
        for t in range(self.nt):
            y, J = self._jac(t, self.vq)
            w = self.vw * np.abs(np.linalg.det(J))
            N = self._cov(J, self.phiE)
            Eh = np.einsum("ma,amqc->qc", E[t], N)
            ex = fn(self.psi(y))
            err += w @ ((Eh - ex) ** 2).sum(1)
            ref += w @ (ex ** 2).sum(1)
        return np.sqrt(err), np.sqrt(ref)
