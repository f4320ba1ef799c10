"""Energy-conserving DG operator for time-domain Maxwell (oracle, FP64).

Sec. 2.1, final time-domain system (stabilized central flux), with the sign
reading stated in the package header:

  d/dt sum_T (eps E, e)_T = sum_T [ (H, curl e)_T - ({{H}} x nu_T, e)_dT ]
                            + sum_F (H^F x nu_F, [[e]])_F
  d/dt sum_T (mu H, h)_T  = sum_T [ -(curl E, h)_T - (1/2 [[E]] x nu_T, h)_dT ]
  d/dt sum_F (h_F/alpha) (H^F, h^F)_F = sum_F ([[E]] x nu_F, h^F)_F

[[E]] = E_T - E_nbr on dT (relative to nu_T), {{H}} = (H_T + H_nbr)/2; on a
PEC face the ghost state is E_nbr = -E_T, H_nbr = H_T.  The central flux is
the same system without H^F.  Spaces: E, e of degree p, H, h of degree p-1
(Sec. 2, V^{k+1} x V^k) or, for the equal-order variant, of degree p; H^F
tangential of degree p on each face.

Every integral is a Gauss sum in physical space over covariant basis functions
N_{a,m}(x) = F^{-T} e_m phi_a(Phi^{-1}(x)) (Sec. 3.2.1), curl by the chain rule:
curl N_{a,m} = (F^{-T} grad phi_a) x (F^{-T} e_m).  The face unknowns are the
covariant tangential components K_i = H^F . t_i in the face frame
x = X_a + s t_1 + u t_2 (face vertices by ascending key), expanded in the face
Dubiner basis psi(s,u): H^F = sum psi_g (K_1g t^1 + K_2g t^2) with t^i the
dual basis of (t_1, t_2) in the face plane.

Vector layouts (the library's canonical layout):
  E[t, m, a]  (a over degree-p indices), H[t, n, b] (degree p-1),
  K[F, i, g]  (faces numbered by first occurrence in (element, local face)).
"""

import numpy as np
import scipy.sparse as sps

from .basis import phi3, psi2, n3, n2
from .quadrature import tet_rule, tri_rule
from .geometry import Geometry


def _covariant_values(Finv, vals):
    """N[b, a, m, q, c] = Finv[b, m, c] * vals[b?, a, q]."""
    if vals.ndim == 2:
        return np.einsum("bmc,aq->bamqc", Finv, vals)
    return np.einsum("bmc,baq->bamqc", Finv, vals)


def _phys_grad(Finv, grads):
    """grad phi in physical coordinates: G[b,a,q,c] = sum_d Finv[b,d,c] g[.., a, q, d]."""
    if grads.ndim == 3:
        return np.einsum("bdc,aqd->baqc", Finv, grads)
    return np.einsum("bdc,baqd->baqc", Finv, grads)


def _curl_values(Finv, pgrad):
    """curl N[b,a,m,q,:] = pgrad[b,a,q,:] x Finv[b,m,:]."""
    B, A, Q, _ = pgrad.shape
    out = np.empty((B, A, 3, Q, 3))
    for m in range(3):
        out[:, :, m] = np.cross(pgrad, Finv[:, None, None, m, :])
    return out


class OracleDG:
    def __init__(self, xyz, tets, p, eps, mu, vertex_key=None, flux="central",
                 alpha0=1.0, chunk=64, h_degree=None):
        """h_degree: degree of H; p - 1 (default, the spaces V^{k+1} x V^k of
        Sec. 2) or p (the equal-order variant: E and H of the same degree)."""
        if p < 1:
            raise ValueError("p >= 1 required")
        self.pH = p - 1 if h_degree is None else int(h_degree)
        if self.pH not in (p - 1, p):
            raise ValueError("h_degree must be p - 1 or p")
        self.geo = Geometry(xyz, tets, vertex_key)
        self.p = p
        self.nt = self.geo.nt
        self.NE = n3(p)
        self.NH = n3(self.pH)
        self.N2 = n2(p)
        self.eps = np.broadcast_to(np.asarray(eps, dtype=float), (self.nt,)).copy()
        self.mu = np.broadcast_to(np.asarray(mu, dtype=float), (self.nt,)).copy()
        if np.any(self.eps <= 0) or np.any(self.mu <= 0):
            raise ValueError("eps, mu must be positive")
        self.flux = flux
        self.alpha = alpha0 * p * p
        self.chunk = chunk
        q = p + 2
        self.vq, self.vw = tet_rule(q)
        self.fq, self.fw = tri_rule(q)
        self.phiE, self.gE = phi3(p, self.vq)
        self.phiH, self.gH = phi3(self.pH, self.vq)
        self.nfaces = len(self.geo.faces)
        self._assembled = None

    # ------------------------------------------------------------------ sizes
    @property
    def sizeE(self):
        return self.nt * 3 * self.NE

    @property
    def sizeH(self):
        return self.nt * 3 * self.NH

    @property
    def sizeK(self):
        return self.nfaces * 2 * self.N2 if self.flux == "stabilized" else 0

    # --------------------------------------------------------- local blocks
    def volume_blocks(self, ts):
        """VH[b] : E_t -> r_H on t (= -(curl E, h)_T) and VE[b] : H_t -> r_E on t
        (= (H, curl e)_T), both by volume quadrature."""
        g = self.geo
        Finv = g.Finv[ts]
        w = self.vw[None, :] * np.abs(g.detF[ts])[:, None]                # (B,Q)
        NEv = _covariant_values(Finv, self.phiE)                            # (B,A,3,Q,3)
        NHv = _covariant_values(Finv, self.phiH)
        curlE = _curl_values(Finv, _phys_grad(Finv, self.gE))              # (B,A,3,Q,3)
        B = len(ts)
        VH = -np.einsum("bq,bamqc,bnlqc->blnma", w, curlE, NHv).reshape(B, 3 * self.NH, 3 * self.NE)
        # note: index order (l, n) = (component, basis) for rows, (m, a) for cols
        VE = np.einsum("bq,bnlqc,bamqc->bmaln", w, NHv, curlE).reshape(B, 3 * self.NE, 3 * self.NH)
        return VH, VE

    def mass_blocks(self, ts, which):
        g = self.geo
        Finv = g.Finv[ts]
        coef = self.eps[ts] if which == "E" else self.mu[ts]
        w = self.vw[None, :] * (np.abs(g.detF[ts]) * coef)[:, None]
        Nv = _covariant_values(Finv, self.phiE if which == "E" else self.phiH)
        B, A = Nv.shape[0], Nv.shape[1]
        M = np.einsum("bq,bamqc,bdlqc->bmald", w, Nv, Nv).reshape(B, 3 * A, 3 * A)
        return M

    def _face_points(self, t, f):
        g = self.geo
        a, b, c = g.face_local[f]
        Xa, Xb, Xc = g.X[t, a], g.X[t, b], g.X[t, c]
        x = Xa[:, None, :] + self.fq[None, :, 0:1] * (Xb - Xa)[:, None, :] \
            + self.fq[None, :, 1:2] * (Xc - Xa)[:, None, :]
        ws = self.fw[None, :] * g.area2[t, f][:, None]
        return x, ws

    def _eval_at(self, t, x, degree):
        """Covariant basis values of elements t (B,) at physical points x (B,Q,3)."""
        xh = self.geo.to_ref(t[:, None], x)
        B, Q, _ = x.shape
        vals, _ = phi3(degree, xh.reshape(-1, 3))
        vals = vals.reshape(vals.shape[0], B, Q).transpose(1, 0, 2)        # (B,A,Q)
        return _covariant_values(self.geo.Finv[t], vals)                     # (B,A,3,Q,3)

    def face_blocks(self, ts, f):
        """Facet blocks of elements ts on local face f.

        Returns dict with
          AH_own (B, 3NH, 3NE): E_t   -> r_H on t   from -(1/2 [[E]] x nu, h)
          AH_nbr (B, 3NH, 3NE): E_nbr -> r_H on t
          AE_own (B, 3NE, 3NH): H_t   -> r_E on t   from -({{H}} x nu, e)
          AE_nbr (B, 3NE, 3NH): H_nbr -> r_E on t
          nbr (B,) neighbour ids (-1 on PEC faces; the *_nbr blocks are then 0).
        """
        g = self.geo
        ts = np.asarray(ts)
        B = len(ts)
        x, ws = self._face_points(ts, f)
        nu = g.normal[ts, f]                                               # (B,3)
        nb = g.nbr[ts, f]
        interior = nb >= 0
        NEo = self._eval_at(ts, x, self.p)
        NHo = self._eval_at(ts, x, self.pH)
        NEn = np.zeros_like(NEo)
        NHn = np.zeros_like(NHo)
        if np.any(interior):
            ti = ts[interior]
            xn = x[interior] + g.shift[ti, f][:, None, :]
            NEn[interior] = self._eval_at(nb[interior], xn, self.p)
            NHn[interior] = self._eval_at(nb[interior], xn, self.pH)
        cown = np.where(interior, 0.5, 1.0)     # PEC ghost: [[E]] = 2E, {{H}} = H
        nuB = nu[:, None, None, None, :]
        ExnuO = np.cross(NEo, np.broadcast_to(nuB, NEo.shape))
        ExnuN = np.cross(NEn, np.broadcast_to(nuB, NEn.shape))
        HxnuO = np.cross(NHo, np.broadcast_to(nuB, NHo.shape))
        HxnuN = np.cross(NHn, np.broadcast_to(nuB, NHn.shape))
        AH_own = -np.einsum("b,bq,bamqc,bdlqc->bldma", cown, ws, ExnuO, NHo)
        AH_nbr = 0.5 * np.einsum("bq,bamqc,bdlqc->bldma", ws, ExnuN, NHo)
        AE_own = -np.einsum("b,bq,bdlqc,bamqc->bmald", cown, ws, HxnuO, NEo)
        AE_nbr = -0.5 * np.einsum("bq,bdlqc,bamqc->bmald", ws, HxnuN, NEo)
        r = lambda A, m, n: A.reshape(B, m, n)
        return dict(AH_own=r(AH_own, 3 * self.NH, 3 * self.NE),
                    AH_nbr=r(AH_nbr, 3 * self.NH, 3 * self.NE),
                    AE_own=r(AE_own, 3 * self.NE, 3 * self.NH),
                    AE_nbr=r(AE_nbr, 3 * self.NE, 3 * self.NH),
                    nbr=nb)

    # ------------------------------------------------ stabilisation (faces)
    def face_unknown_blocks(self, F):
        """Blocks of global face F (index into geo.faces) for the H^F system.

        Returns (MF (2N2,2N2), [(t, S_t (2N2, 3NE), CEK_t (3NE, 2N2)), ...]) with
          MF  = (h_F/alpha) (psi t^i, psi t^j)_F,
          S_t : E_t -> r_K   from ([[E]] x nu_F, h^F)_F,
          CEK_t : K -> r_E on t from (H^F x nu_F, [[e]])_F.
        """
        g = self.geo
        kt, sides = g.faces[F]
        t0, f0 = sides[0]
        a, b, c = g.face_local[f0]
        Xa, Xb, Xc = g.X[t0, a], g.X[t0, b], g.X[t0, c]
        t1, t2 = Xb - Xa, Xc - Xa
        cr = np.cross(t1, t2)
        J = np.linalg.norm(cr)
        nF = cr / J
        d1 = np.cross(t2, nF) / J
        d2 = np.cross(nF, t1) / J
        x = Xa[None, :] + self.fq[:, 0:1] * t1[None, :] + self.fq[:, 1:2] * t2[None, :]
        ws = self.fw * J
        psi = psi2(self.p, self.fq)                                        # (G,Q)
        HFb = np.stack([psi[:, :, None] * d1[None, None, :],
                        psi[:, :, None] * d2[None, None, :]], axis=0)      # (2,G,Q,3)
        hF = min(abs(g.detF[t]) / g.area2[t, f] for (t, f) in sides)
        MF = (hF / self.alpha) * np.einsum("q,igqc,jdqc->igjd", ws, HFb, HFb).reshape(
            2 * self.N2, 2 * self.N2)
        HFxnu = np.cross(HFb, np.broadcast_to(nF, HFb.shape))
        out = []
        cfac = 1.0 if len(sides) == 2 else 2.0       # PEC: [[E]] = 2E, [[e]] = 2e
        for (t, f) in sides:
            xs = x if (t, f) == (t0, f0) else x + g.shift[t0, f0][None, :]
            sgn = np.sign(np.dot(nF, g.normal[t, f]))
            NE = self._eval_at(np.array([t]), xs[None], self.p)[0]         # (A,3,Q,3)
            Exnu = np.cross(NE, np.broadcast_to(nF, NE.shape))
            S = cfac * sgn * np.einsum("q,amqc,igqc->igma", ws, Exnu, HFb).reshape(
                2 * self.N2, 3 * self.NE)
            CEK = cfac * sgn * np.einsum("q,igqc,amqc->maig", ws, HFxnu, NE).reshape(
                3 * self.NE, 2 * self.N2)
            out.append((t, S, CEK))
        return MF, out

    # ----------------------------------------------------------- assembly
    def assemble(self):
        """Global sparse operators (small meshes only)."""
        if self._assembled is not None:
            return self._assembled
        nt, NE, NH = self.nt, self.NE, self.NH
        rows_h, cols_h, vals_h = [], [], []
        rows_e, cols_e, vals_e = [], [], []
        ME, MH = [], []
        eH = lambda t: (np.arange(3 * NH)[None, :] + (3 * NH) * np.asarray(t)[:, None])
        eE = lambda t: (np.arange(3 * NE)[None, :] + (3 * NE) * np.asarray(t)[:, None])

        def add(rows, cols, vals, R, C, V):
            rr = np.broadcast_to(R[:, :, None], V.shape)
            cc = np.broadcast_to(C[:, None, :], V.shape)
            rows.append(rr.ravel()); cols.append(cc.ravel()); vals.append(V.ravel())

        for s in range(0, nt, self.chunk):
            ts = np.arange(s, min(nt, s + self.chunk))
            VH, VE = self.volume_blocks(ts)
            add(rows_h, cols_h, vals_h, eH(ts), eE(ts), VH)
            add(rows_e, cols_e, vals_e, eE(ts), eH(ts), VE)
            for f in range(4):
                fb = self.face_blocks(ts, f)
                add(rows_h, cols_h, vals_h, eH(ts), eE(ts), fb["AH_own"])
                add(rows_e, cols_e, vals_e, eE(ts), eH(ts), fb["AE_own"])
                it = fb["nbr"] >= 0
                if np.any(it):
                    add(rows_h, cols_h, vals_h, eH(ts[it]), eE(fb["nbr"][it]), fb["AH_nbr"][it])
                    add(rows_e, cols_e, vals_e, eE(ts[it]), eH(fb["nbr"][it]), fb["AE_nbr"][it])
            ME.append(self.mass_blocks(ts, "E"))
            MH.append(self.mass_blocks(ts, "H"))
        cat = np.concatenate
        CH = sps.csr_matrix((cat(vals_h), (cat(rows_h), cat(cols_h))), shape=(self.sizeH, self.sizeE))
        CE = sps.csr_matrix((cat(vals_e), (cat(rows_e), cat(cols_e))), shape=(self.sizeE, self.sizeH))
        ME = cat(ME)
        MH = cat(MH)
        out = dict(CH=CH, CE=CE, ME=ME, MH=MH,
                   MEinv=np.linalg.inv(ME), MHinv=np.linalg.inv(MH))
        if self.flux == "stabilized":
            N2 = self.N2
            rs, cs, vs = [], [], []
            re, ce, ve = [], [], []
            MF = np.empty((self.nfaces, 2 * N2, 2 * N2))
            for F in range(self.nfaces):
                MFb, sides = self.face_unknown_blocks(F)
                MF[F] = MFb
                kr = np.arange(2 * N2) + 2 * N2 * F
                for (t, S, CEK) in sides:
                    er = np.arange(3 * NE) + 3 * NE * t
                    rs.append(np.repeat(kr, 3 * NE)); cs.append(np.tile(er, 2 * N2)); vs.append(S.ravel())
                    re.append(np.repeat(er, 2 * N2)); ce.append(np.tile(kr, 3 * NE)); ve.append(CEK.ravel())
            out["S"] = sps.csr_matrix((cat(vs), (cat(rs), cat(cs))), shape=(self.sizeK, self.sizeE))
            out["CEK"] = sps.csr_matrix((cat(ve), (cat(re), cat(ce))), shape=(self.sizeE, self.sizeK))
            out["MF"] = MF
            out["MFinv"] = np.linalg.inv(MF)
        self._assembled = out
        return out

    # ------------------------------------------------ operator application
    @staticmethod
    def _blockmul(Mb, v):
        nb, m, _ = Mb.shape
        return np.einsum("bij,bj->bi", Mb, v.reshape(nb, m)).ravel()

    def residual_H(self, E):
        return self.assemble()["CH"] @ E

    def residual_E(self, H, K=None):
        A = self.assemble()
        r = A["CE"] @ H
        if self.flux == "stabilized" and K is not None:
            r = r + A["CEK"] @ K
        return r

    def residual_K(self, E):
        return self.assemble()["S"] @ E

    def energy(self, E, H_lo, H_hi, K_lo=None, K_hi=None):
        A = self.assemble()
        W = 0.5 * E @ self._blockmul(A["ME"], E) + 0.5 * H_lo @ self._blockmul(A["MH"], H_hi)
        if self.flux == "stabilized" and K_lo is not None:
            W += 0.5 * K_lo @ self._blockmul(A["MF"], K_hi)
        return W

    def run(self, E0, H0, dt, nsteps, K0=None, source=None):
        """Leapfrog (symplectic Euler with H staggered by dt/2, Sec. 3), started and
        finished with half kicks so that E and H are reported at the same time.

        Per step: E^{n+1} = E^n + dt M_eps^{-1} r_E(H^{n+1/2}, K^{n+1/2});
                  H^{n+3/2} = H^{n+1/2} + dt M_mu^{-1} r_H(E^{n+1}) (same for K).
        Returns E^N, H^N, K^N and the discrete energies
        W^n = 1/2 E^n M E^n + 1/2 H^{n-1/2} M H^{n+1/2} (+ same for K), n = 0..N.
        source: optional callable n -> vector added to r_E at step n (E-phase
        from t_n to t_{n+1}, evaluated at t_{n+1/2}).
        """
        A = self.assemble()
        stab = self.flux == "stabilized"
        E = np.array(E0, dtype=float)
        H = np.array(H0, dtype=float)
        K = np.zeros(self.sizeK) if (stab and K0 is None) else (np.array(K0, dtype=float) if stab else None)

        def kickH(E):
            dH = dt * self._blockmul(A["MHinv"], A["CH"] @ E)
            dK = dt * self._blockmul(A["MFinv"], A["S"] @ E) if stab else None
            return dH, dK

        W = []
        dH, dK = kickH(E)
        lo, hi = H - 0.5 * dH, H + 0.5 * dH
        Wn = 0.5 * E @ self._blockmul(A["ME"], E) + 0.5 * lo @ self._blockmul(A["MH"], hi)
        if stab:
            klo, khi = K - 0.5 * dK, K + 0.5 * dK
            Wn += 0.5 * klo @ self._blockmul(A["MF"], khi)
            K = khi
        W.append(Wn)
        H = hi
        for n in range(nsteps):
            rE = A["CE"] @ H
            if stab:
                rE = rE + A["CEK"] @ K
            if source is not None:
                rE = rE + source(n)
            E = E + dt * self._blockmul(A["MEinv"], rE)
            dH, dK = kickH(E)
            Wn = 0.5 * E @ self._blockmul(A["ME"], E) + 0.5 * H @ self._blockmul(A["MH"], H + dH)
            if stab:
                Wn += 0.5 * K @ self._blockmul(A["MF"], K + dK)
            W.append(Wn)
            if n < nsteps - 1:
                H = H + dH
                if stab:
                    K = K + dK
            else:
                H = H + 0.5 * dH
                if stab:
                    K = K + 0.5 * dK
        return E, H, K, np.array(W)

    # ------------------------------------------- sampled (matrix-free) path
    def local_residual_H(self, E, ts):
        """r_H on elements ts for a global E (no global assembly)."""
        ts = np.asarray(ts)
        Ev = np.asarray(E).reshape(self.nt, 3 * self.NE)
        VH, _ = self.volume_blocks(ts)
        r = np.einsum("bij,bj->bi", VH, Ev[ts])
        for f in range(4):
            fb = self.face_blocks(ts, f)
            r += np.einsum("bij,bj->bi", fb["AH_own"], Ev[ts])
            nb = np.where(fb["nbr"] >= 0, fb["nbr"], 0)
            r += np.einsum("bij,bj->bi", fb["AH_nbr"], Ev[nb])
        return r

    def local_residual_E(self, H, ts):
        ts = np.asarray(ts)
        Hv = np.asarray(H).reshape(self.nt, 3 * self.NH)
        _, VE = self.volume_blocks(ts)
        r = np.einsum("bij,bj->bi", VE, Hv[ts])
        for f in range(4):
            fb = self.face_blocks(ts, f)
            r += np.einsum("bij,bj->bi", fb["AE_own"], Hv[ts])
            nb = np.where(fb["nbr"] >= 0, fb["nbr"], 0)
            r += np.einsum("bij,bj->bi", fb["AE_nbr"], Hv[nb])
        return r

    def local_kick_H(self, E, ts, dt):
        """dt M_mu^{-1} r_H on elements ts (quadrature mass, Cholesky solve)."""
        r = self.local_residual_H(E, ts)
        M = self.mass_blocks(np.asarray(ts), "H")
        L = np.linalg.cholesky(M)
        y = np.linalg.solve(L, r[..., None])
        return dt * np.linalg.solve(np.swapaxes(L, 1, 2), y)[..., 0]

    def local_kick_E(self, H, ts, dt):
        r = self.local_residual_E(H, ts)
        M = self.mass_blocks(np.asarray(ts), "E")
        L = np.linalg.cholesky(M)
        y = np.linalg.solve(L, r[..., None])
        return dt * np.linalg.solve(np.swapaxes(L, 1, 2), y)[..., 0]


# ------------------------------------------------------------ observations
def locate_points(dg, pts):
    """Element containing each physical point (brute force over barycentric
    coordinates) and the point's reference coordinates in that element."""
    g = dg.geo
    out_t, out_xh = [], []
    for x in np.asarray(pts, dtype=float):
        xh = np.einsum("tij,tj->ti", g.Finv, x[None, :] - g.X0)
        bary = np.concatenate([1 - xh.sum(1, keepdims=True), xh], axis=1)
        t = int(np.argmax(bary.min(1)))
        if bary[t].min() < -1e-12:
            raise ValueError("point outside the mesh")
        out_t.append(t)
        out_xh.append(xh[t])
    return np.array(out_t), np.array(out_xh)


def observation_matrix(dg, pts):
    """Sparse P (3 nobs x sizeE): rows = physical E components at the points."""
    ts, xhs = locate_points(dg, pts)
    vals, _ = phi3(dg.p, xhs)                        # (NE, nobs)
    rows, cols, data = [], [], []
    for o, (t, xh) in enumerate(zip(ts, xhs)):
        Finv = dg.geo.Finv[t]
        # E(x) = F^{-T} sum_a c[:, a] phi_a  ->  E_c = sum_{m,a} Finv[m, c] phi_a c[m, a]
        for c in range(3):
            for mm in range(3):
                for a in range(dg.NE):
                    rows.append(3 * o + c)
                    cols.append((t * 3 + mm) * dg.NE + a)
                    data.append(Finv[mm, c] * vals[a, o])
    return sps.csr_matrix((data, (rows, cols)), shape=(3 * len(ts), dg.sizeE))


def adjoint_grad_eps(dg, E0, H0, dt, nsteps, pts):
    """J and dJ/d eps of adjoint_grad (the permittivity part)."""
    J, geps, _ = adjoint_grad(dg, E0, H0, dt, nsteps, pts)
    return J, geps


def adjoint_grad(dg, E0, H0, dt, nsteps, pts):
    """J = sum_{n=1..N} sum_o |E^n(x_o)|^2 for the leapfrog of OracleDG.run (central
    flux; G^n = H^{n+1/2}) and its gradients by the discrete adjoint.  Forward:
      G^0 = H^0 + dt/2 A E^0,  E^{n+1} = E^n + dt B G^n,  G^{n+1} = G^n + dt A E^{n+1},
    A = M_mu^{-1} C_H (H-kick), B = M_eps^{-1} C_E (E-kick).  Multipliers e^m of the
    E-updates and g^m of the G-updates (Lagrangian J - sum e.R_E - sum g.R_G):
      e^m = 2 P^T P E^m + dt A^T g^m + e^{m+1},   g^{m-1} = g^m + dt B^T e^m,
    e^{N+1} = 0, g^N = 0.  Since d M^{-1}/d c_T = -M^{-1}|_T / c_T (c = eps, mu):
      dJ/d eps_T = -(1/eps_T) sum_{m=1..N} e^m_T . (E^m - E^{m-1})_T,
      dJ/d mu_T  = -(1/mu_T) [sum_{m=1..N} g^m_T . (G^m - G^{m-1})_T + g^0_T . (G^0 - H^0)_T]."""
    A_ = dg.assemble()
    P = observation_matrix(dg, pts)
    PtP = (P.T @ P).tocsr()
    E = np.array(E0, dtype=float)
    H = np.array(H0, dtype=float)
    G = H + 0.5 * dt * dg._blockmul(A_["MHinv"], A_["CH"] @ E)
    Es, Gs = [E.copy()], [G.copy()]
    J = 0.0
    for n in range(nsteps):
        E = E + dt * dg._blockmul(A_["MEinv"], A_["CE"] @ G)
        Es.append(E.copy())
        J += float(E @ (PtP @ E))
        G = G + dt * dg._blockmul(A_["MHinv"], A_["CH"] @ E)
        Gs.append(G.copy())
    # transposes of A = MHinv CH and B = MEinv CE (block inverses are symmetric)
    e_next = np.zeros(dg.sizeE)
    g = np.zeros(dg.sizeH)
    geps = np.zeros(dg.nt)
    gmu = np.zeros(dg.nt)
    for m in range(nsteps, 0, -1):
        e = 2 * (PtP @ Es[m]) + dt * (A_["CH"].T @ dg._blockmul(A_["MHinv"], g)) + e_next
        dE = (Es[m] - Es[m - 1]).reshape(dg.nt, -1)
        geps -= np.einsum("ti,ti->t", e.reshape(dg.nt, -1), dE) / dg.eps
        dG = (Gs[m] - Gs[m - 1]).reshape(dg.nt, -1)
        gmu -= np.einsum("ti,ti->t", g.reshape(dg.nt, -1), dG) / dg.mu
        g = g + dt * (A_["CE"].T @ dg._blockmul(A_["MEinv"], e))
        e_next = e
    dG0 = (Gs[0] - np.asarray(H0, dtype=float)).reshape(dg.nt, -1)
    gmu -= np.einsum("ti,ti->t", g.reshape(dg.nt, -1), dG0) / dg.mu
    return J, geps, gmu


def objective(dg, E0, H0, dt, nsteps, pts):
    """J of adjoint_grad_eps by a plain forward run (for finite differences)."""
    A_ = dg.assemble()
    P = observation_matrix(dg, pts)
    E = np.array(E0, dtype=float)
    G = np.array(H0, dtype=float) + 0.5 * dt * dg._blockmul(A_["MHinv"], A_["CH"] @ E)
    J = 0.0
    for n in range(nsteps):
        E = E + dt * dg._blockmul(A_["MEinv"], A_["CE"] @ G)
        v = P @ E
        J += float(v @ v)
        G = G + dt * dg._blockmul(A_["MHinv"], A_["CH"] @ E)
    return J


def dipole_source_vector(dg, xs, direction, fval):
    """r_E contribution -(J, e) of a point current J = direction delta(x - xs) f:
    entries -f direction . N_{a,m}(xs) on the element containing xs."""
    ts, xhs = locate_points(dg, [xs])
    t, xh = ts[0], xhs[0]
    vals, _ = phi3(dg.p, xh[None, :])
    Finv = dg.geo.Finv[t]
    out = np.zeros(dg.sizeE)
    d = np.asarray(direction, dtype=float)
    for mm in range(3):
        # N_{a,m}(x) = F^{-T} e_m phi_a  ->  d . N = (Finv d)_m phi_a
        coef = Finv[mm] @ d
        out[(t * 3 + mm) * dg.NE:(t * 3 + mm + 1) * dg.NE] = -fval * coef * vals[:, 0]
    return out


def resonances(dg, zero_rel=1e-8):
    """Resonance frequencies of the cavity (the frequency-domain problem of Sec. 2.2,
    i omega eps E = curl H, i omega mu H = -curl E, PEC), discretised by the DG
    operator of Sec. 2.1.  Eliminating H (and H^F) from the semi-discrete system
      M_eps E' = C_E H + C_EK K,  M_mu H' = C_H E,  M_F K' = S E
    gives E'' = -M_eps^{-1} Kc E with Kc = -(C_E M_mu^{-1} C_H + C_EK M_F^{-1} S),
    symmetric positive semi-definite because C_E = -C_H^T and C_EK = -S^T (Sec. 2.1,
    skew-adjointness).  A time-harmonic field gives omega^2 M_eps e = Kc e; the
    generalized symmetric eigenproblem is solved densely (small meshes only).
    Returns (omega of the eigenvalues above zero_rel * the largest, ascending; the
    number of eigenvalues at or below it: the discrete null space)."""
    import scipy.linalg as sl
    A_ = dg.assemble()
    CE, CH = A_["CE"].toarray(), A_["CH"].toarray()
    Kc = -(CE @ sl.block_diag(*A_["MHinv"]) @ CH)
    if dg.flux == "stabilized":
        Kc -= A_["CEK"].toarray() @ sl.block_diag(*A_["MFinv"]) @ A_["S"].toarray()
    Kc = 0.5 * (Kc + Kc.T)     # exactly symmetric in exact arithmetic; remove rounding
    lam = np.sort(sl.eigh(Kc, sl.block_diag(*A_["ME"]), eigvals_only=True))
    zero = lam <= zero_rel * lam.max()
    return np.sqrt(lam[~zero]), int(zero.sum())


def run_composed(dg, E0, H0, dt, nsteps, order, K0=None):
    """Symmetric composition of leapfrog steps (Sec. 3 admits any explicit
    integrator; compositions of the symplectic leapfrog stay symplectic).
    order 2: one leapfrog step of size dt per step.  order 4: three leapfrog
    steps of sizes w1 dt, w0 dt, w1 dt with w1 = 1/(2 - 2^(1/3)), w0 = 1 - 2 w1
    (Yoshida's triple jump).  Each substep is a complete OracleDG.run step with
    its own opening and closing half kicks (no merging).  Returns E, H, K."""
    if order == 2:
        ws = [1.0]
    elif order == 4:
        w1 = 1.0 / (2.0 - 2.0 ** (1.0 / 3.0))
        ws = [w1, 1.0 - 2.0 * w1, w1]
    else:
        raise ValueError(order)
    E, H, K = np.array(E0, dtype=float), np.array(H0, dtype=float), K0
    for _ in range(nsteps):
        for w in ws:
            E, H, K, _ = dg.run(E, H, w * dt, 1, K0=K)
    return E, H, K
