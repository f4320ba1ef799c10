"""Convenience wrapper owning the C-ABI handles of one problem.

Argument marshalling only: every step runs in libdgm.so.
"""

import numpy as np

from . import _capi as capi


class Solver:
    """mesh + p + eps + mu -> device-resident DG Maxwell problem (include/dgm.h)."""

    def __init__(self, xyz, tets, p, eps, mu, vertex_key=None, precision="fp64",
                 flux="central", alpha0=1.0, device=0, variant=0, compensated=False, equal_order=False):
        self.ctx = capi.dgm_create(device)
        self.mesh = capi.dgm_mesh_create(self.ctx, xyz, tets, vertex_key)
        self.nt, self.nfaces, self.nboundary = capi.dgm_mesh_info(self.mesh)
        opt = capi.dgm_default_options()
        opt.precision = {"fp64": capi.DGM_PREC_FP64, "fp32": capi.DGM_PREC_FP32,
                         "tc32": capi.DGM_PREC_TC32, "tc16": capi.DGM_PREC_TC16,
                         "tcbf16": capi.DGM_PREC_TCBF16, "tc16x2": capi.DGM_PREC_TC16X2}[precision]
        opt.variant = variant
        opt.compensated = 1 if compensated else 0
        opt.equal_order = 1 if equal_order else 0
        opt.flux = {"central": capi.DGM_FLUX_CENTRAL, "stabilized": capi.DGM_FLUX_STABILIZED}[flux]
        opt.alpha0 = alpha0
        eps = np.broadcast_to(np.asarray(eps, dtype=np.float64), (self.nt,))
        mu = np.broadcast_to(np.asarray(mu, dtype=np.float64), (self.nt,))
        self.prob = capi.dgm_problem_create(self.ctx, self.mesh, p, eps, mu, opt)
        self.eps = np.array(eps)
        self.mu = np.array(mu)
        self.p = p
        self.nE, self.nH, self.nHF = capi.dgm_problem_sizes(self.prob)

    def set_fields(self, E, H, HF=None):
        capi.dgm_set_fields(self.prob, E, H, HF)

    def get_fields(self):
        E = np.empty(self.nE)
        H = np.empty(self.nH)
        HF = np.empty(self.nHF) if self.nHF else None
        capi.dgm_get_fields(self.prob, E, H, HF)
        return (E, H, HF) if self.nHF else (E, H)

    def kick(self, which, dt, stream=None):
        capi.dgm_kick(self.prob, which, dt, stream)

    def run_composed(self, dt, nsteps, order=4, stream=None):
        """Symplectic composition of leapfrog steps (order 2 or 4); no energies."""
        capi.dgm_run_composed(self.prob, dt, nsteps, order, stream)

    def run(self, dt, nsteps, stream=None, energies=False):
        out = np.empty(nsteps + 1) if energies else None
        capi.dgm_run(self.prob, dt, nsteps, stream, out)
        return out

    def autotune(self, steps=5):
        """Time the launch-configuration candidates on this problem (fields
        unchanged) and keep the fastest; -> (configs, ms_per_step, chosen)."""
        return capi.dgm_autotune(self.prob, steps)

    def project(self, fn, q1d=None):
        """Set E, H to the covariant L2 projections of fn(x) -> (E(x), H(x)) (arrays
        [..., 3] for points x [..., 3]) sampled at this problem's quadrature points."""
        q1d = q1d or self.p + 2
        x = capi.dgm_quad_points(self.prob, q1d, self.nt)
        E, H = fn(x)
        capi.dgm_project(self.prob, q1d, E, H)

    def resonances(self, m=300, nev=8, zero_rel=1e-8):
        """Smallest nonzero cavity resonance frequencies by Lanczos on the GPU
        operator (FP64); -> (omega, relative residuals)."""
        return capi.dgm_resonances(self.prob, m, nev, zero_rel)

    def energy(self):
        return capi.dgm_energy(self.prob)

    def close(self):
        if getattr(self, "prob", None):
            capi.dgm_problem_destroy(self.prob)
            self.prob = None
        if getattr(self, "mesh", None):
            capi.dgm_mesh_destroy(self.mesh)
            self.mesh = None
        if getattr(self, "ctx", None):
            capi.dgm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Solver2D:
    """2D triangle mesh + p + eps + mu -> device-resident TE problem (include/dgm.h:
    E in the plane of degree p, H along z of degree p - 1)."""

    def __init__(self, xy, tris, p, eps, mu, vertex_key=None, precision="fp64", device=0):
        self.ctx = capi.dgm_create(device)
        prec = {"fp64": capi.DGM_PREC_FP64, "fp32": capi.DGM_PREC_FP32}.get(precision, -1)
        self.prob = capi.dgm_problem2d_create(self.ctx, xy, tris, p, eps, mu, vertex_key, prec)
        self.p = p
        self.nE, self.nH = capi.dgm_problem2d_sizes(self.prob)

    def set_fields(self, E, H):
        capi.dgm_set_fields2d(self.prob, E, H)

    def get_fields(self):
        E = np.empty(self.nE)
        H = np.empty(self.nH)
        capi.dgm_get_fields2d(self.prob, E, H)
        return E, H

    def kick(self, which, dt):
        capi.dgm_kick2d(self.prob, which, dt)

    def run(self, dt, nsteps, energies=False):
        return capi.dgm_run2d(self.prob, dt, nsteps, None, energies)

    def close(self):
        if getattr(self, "prob", None):
            capi.dgm_problem2d_destroy(self.prob)
            self.prob = None
        if getattr(self, "ctx", None):
            capi.dgm_destroy(self.ctx)
            self.ctx = None

