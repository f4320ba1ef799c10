"""Pins of the curved-element oracle, oracle/curved.py (Sec. 3.3.2).

* With the identity map it reproduces the flat oracle's operator and masses
  (oracle/dg.py, pinned separately), so every term carries over.
* On a curved mesh the operator stays skew-adjoint (C_E = -C_H^T) and the
  leapfrog conserves the energy, with the exact mass and with the approximate
  inverse mass (in the norm of the approximate mass).
* The approximate inverse equals the exact one where the map is affine, and its
  error elsewhere is second order in the element size.
* The unit cube deformed inside by a smooth map that fixes its boundary is still
  the PEC cube, so the TE110 mode is an exact solution: the curved scheme
  converges to it under h-refinement at the rate of the flat one (R15: p - 1 for
  E with the central flux).
"""

import numpy as np
import pytest

from oracle.curved import CurvedDG
from oracle.dg import OracleDG
from workloads.fields import te110_fields
from workloads.mesh import kuhn_cube_mesh

A0 = 0.06
V = np.ones(3) / np.sqrt(3.0)


def _psi(y):
    s = np.sin(np.pi * y[..., 0]) * np.sin(np.pi * y[..., 1]) * np.sin(np.pi * y[..., 2])
    return y + A0 * s[..., None] * V


def _dpsi(y):
    sx, sy, sz = (np.sin(np.pi * y[..., k]) for k in range(3))
    cx, cy, cz = (np.cos(np.pi * y[..., k]) for k in range(3))
    grad = np.pi * np.stack([cx * sy * sz, sx * cy * sz, sx * sy * cz], -1)
    return np.eye(3) + A0 * np.einsum("i,...j->...ij", V, grad)


B0 = 0.1


def _quad(y):
    """A gentle quadratic map (the mass-error rate is reached already on coarse meshes)."""
    return y + B0 * np.stack([y[..., 1] ** 2, y[..., 2] ** 2, y[..., 0] ** 2], -1)


def _dquad(y):
    D = np.zeros(y.shape[:-1] + (3, 3))
    D[..., 0, 0] = D[..., 1, 1] = D[..., 2, 2] = 1.0
    D[..., 0, 1] = 2 * B0 * y[..., 1]
    D[..., 1, 2] = 2 * B0 * y[..., 2]
    D[..., 2, 0] = 2 * B0 * y[..., 0]
    return D


def _ident(y):
    return y


def _dident(y):
    return np.broadcast_to(np.eye(3), y.shape[:-1] + (3, 3)).copy()


def test_identity_map_reproduces_flat_oracle():
    m = kuhn_cube_mesh(2, jitter=0.1, seed=3, shuffle_local=True)
    eps = np.random.default_rng(4).uniform(1, 4, m.nt)
    flat = OracleDG(m.xyz, m.tets, 2, eps, 1.5).assemble()
    cur = CurvedDG(m.xyz, m.tets, 2, eps, 1.5, _ident, _dident).assemble()
    assert abs(cur["CH"] - flat["CH"]).max() < 1e-13 * abs(flat["CH"]).max()
    assert abs(cur["CE"] - flat["CE"]).max() < 1e-13 * abs(flat["CE"]).max()
    assert np.abs(cur["ME"] - flat["ME"]).max() < 1e-13 * np.abs(flat["ME"]).max()
    assert np.abs(cur["MH"] - flat["MH"]).max() < 1e-13 * np.abs(flat["MH"]).max()


def test_curved_operator_skew_and_energy():
    m = kuhn_cube_mesh(2, jitter=0.1, seed=5)
    eps = np.random.default_rng(6).uniform(1, 4, m.nt)
    dg = CurvedDG(m.xyz, m.tets, 2, eps, 1.0, _psi, _dpsi)
    A = dg.assemble()
    assert abs(A["CE"] + A["CH"].T).max() < 1e-13 * abs(A["CH"]).max()
    rng = np.random.default_rng(7)
    E0, H0 = rng.standard_normal(dg.sizeE), rng.standard_normal(dg.sizeH)
    for Mi in (None, dg.approx_inverse("E")):
        _, _, W = dg.run(E0, H0, 0.01, 20, MEinv=Mi)
        assert np.abs(W - W[0]).max() < 1e-12 * W[0]


def test_approximate_inverse_exact_on_affine_and_second_order():
    m = kuhn_cube_mesh(2)
    flat = CurvedDG(m.xyz, m.tets, 2, 2.0, 1.0, _ident, _dident)
    Fa = flat.assemble()
    assert np.abs(flat.approx_inverse("E") - Fa["MEinv"]).max() < 1e-11 * np.abs(Fa["MEinv"]).max()
    errs = []
    for n in (2, 4):
        mm = kuhn_cube_mesh(n)
        dg = CurvedDG(mm.xyz, mm.tets, 2, 1.0, 1.0, _quad, _dquad)
        M = np.array([dg.element_blocks(t)[2] for t in range(dg.nt)])
        Mi = dg.approx_inverse("E")
        I = np.eye(M.shape[1])
        errs.append(max(np.linalg.norm(Mi[t] @ M[t] - I, 2) for t in range(dg.nt)))
    assert errs[0] / errs[1] > 2 ** 1.7, errs      # observed 2^1.93 (2^1.87 from n = 1 to 2)


@pytest.mark.parametrize("p", [2, 3])
def test_te110_converges_on_the_curved_cube(p):
    fE = lambda x: te110_fields(x, 0.0)[0]
    fH0 = lambda x: te110_fields(x, 0.0)[1]
    T = 0.25
    errs = []
    for n in (2, 4):
        m = kuhn_cube_mesh(n)
        dg = CurvedDG(m.xyz, m.tets, p, 1.0, 1.0, _psi, _dpsi)
        E0, H0 = dg.project(fE, "E"), dg.project(fH0, "H")
        steps = int(np.ceil(T / (0.1 / n / p ** 2)))
        E, _, W = dg.run(E0, H0, T / steps, steps)
        e, r = dg.l2_error(E, lambda x: te110_fields(x, T)[0])
        errs.append(e / r)
        assert np.abs(W - W[0]).max() < 1e-12 * W[0]
    rate = np.log2(errs[0] / errs[1])
    assert rate > p - 1 - 0.3, (p, errs, rate)
