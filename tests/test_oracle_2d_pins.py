"""Pins of the 2D (TE) triangle oracle, oracle/dg2d.py, against what the
mathematics fixes (CPU only).

* The central-flux operator of Sec. 2.1, restated for E in the plane and H
  along z, is skew-adjoint: C_E = -C_H^T, on PEC and periodic meshes.
* It is exact on polynomial fields: a continuous E of degree p whose tangential
  component vanishes on the PEC boundary gives M_H^{-1} C_H E = -curl E, any
  continuous H of degree p - 1 gives M_E^{-1} C_E H = curl H (both right-hand
  sides lie in the discrete spaces).  Constant fields on a periodic mesh have
  zero residual (the periodic edge matching).
* The leapfrog of Sec. 3 conserves the modified energy.
* The PEC unit square's TE modes (omega = pi sqrt(m^2 + n^2), closed form):
  the smallest nonzero discrete frequencies approach them, the static subspace
  has exactly the dimension that counting fixes (dim E - dim H + 1: the range of
  C_H misses only the constant H), and the TE11 mode converges under h-refinement
  at the rate of H's degree, p - 1, as the 3D pair does (a dropped or mis-signed
  term breaks all three).
"""

import numpy as np
import pytest

from oracle.dg2d import OracleDG2D
from workloads.mesh2d import square_tri_mesh


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("periodic", [False, True])
@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_2d_operator_is_skew(p, periodic):
    m = square_tri_mesh(3, jitter=0.15, seed=3, periodic=periodic, shuffle_local=True)
    eps = np.random.default_rng(1).uniform(1, 4, m.nt)
    dg = OracleDG2D(m.xy, m.tris, p, eps, 1.5, vertex_key=m.vertex_key)
    A = dg.assemble()
    assert abs(A["CE"] + A["CH"].T).max() < 1e-14 * abs(A["CH"]).max()


@pytest.mark.parametrize("p", [3, 4])
def test_2d_exact_on_polynomial_fields(p):
    m = square_tri_mesh(3, jitter=0.15, seed=3, shuffle_local=True)
    dg = OracleDG2D(m.xy, m.tris, p, 1.0, 1.0)
    A = dg.assemble()
    x_, y_ = (lambda x: x[..., 0]), (lambda x: x[..., 1])
    # E_x vanishes on y = 0, 1 and E_y on x = 0, 1: tangential E = 0 on the square's edges
    fE = lambda x: np.stack([y_(x) * (1 - y_(x)) * x_(x) ** (p - 2),
                             x_(x) * (1 - x_(x)) * (1 + y_(x) ** (p - 2))], -1)
    curlE = lambda x: ((1 - 2 * x_(x)) * (1 + y_(x) ** (p - 2))
                       - x_(x) ** (p - 2) * (1 - 2 * y_(x)))
    E, _ = dg.project(fE=fE)
    _, cE = dg.project(fH=curlE)
    dH = dg._blockmul(A["MHinv"], A["CH"] @ E)
    assert _rel(dH, -cE) < 1e-12
    fH = lambda x: x_(x) ** (p - 1) - x_(x) * y_(x) + 3 * y_(x)
    curlH = lambda x: np.stack([-x_(x) + 3, -((p - 1) * x_(x) ** (p - 2) - y_(x))], -1)
    _, H = dg.project(fH=fH)
    cH, _ = dg.project(fE=curlH)
    dE = dg._blockmul(A["MEinv"], A["CE"] @ H)
    assert _rel(dE, cH) < 1e-12


def test_2d_constant_fields_on_periodic_mesh():
    m = square_tri_mesh(4, jitter=0.1, seed=5, periodic=True, shuffle_local=True)
    dg = OracleDG2D(m.xy, m.tris, 2, 1.0, 1.0, vertex_key=m.vertex_key)
    A = dg.assemble()
    E, H = dg.project(fE=lambda x: np.broadcast_to([0.3, -1.2], x.shape).copy(),
                      fH=lambda x: np.full(x.shape[:-1], 0.7))
    assert np.abs(A["CH"] @ E).max() < 1e-13 * np.abs(E).max()
    assert np.abs(A["CE"] @ H).max() < 1e-13 * np.abs(H).max()


@pytest.mark.parametrize("periodic", [False, True])
def test_2d_energy_is_conserved(periodic):
    m = square_tri_mesh(3, jitter=0.1, seed=7, periodic=periodic)
    rng = np.random.default_rng(8)
    dg = OracleDG2D(m.xy, m.tris, 3, rng.uniform(1, 4, m.nt), rng.uniform(1, 2, m.nt), vertex_key=m.vertex_key)
    _, _, W = dg.run(rng.standard_normal(dg.sizeE), rng.standard_normal(dg.sizeH), 0.01, 30)
    assert np.abs(W - W[0]).max() < 1e-13 * W[0]


def test_2d_cavity_spectrum():
    m = square_tri_mesh(4, jitter=0.1, seed=2)
    dg = OracleDG2D(m.xy, m.tris, 3, 1.0, 1.0)
    om = dg.resonances()
    zero = om <= 1e-6 * om.max()
    assert zero.sum() == dg.sizeE - dg.sizeH + 1
    exact = np.pi * np.sqrt(np.array([1, 1, 2, 4, 4, 5, 5], dtype=float))
    assert np.all(np.abs(om[~zero][:7] - exact) < 1e-2 * exact)


def test_2d_te11_mode_converges():
    w = np.pi * np.sqrt(2.0)

    def fE(x, t):
        X, Y = np.pi * x[..., 0], np.pi * x[..., 1]
        return np.stack([-np.pi * np.cos(X) * np.sin(Y), np.pi * np.sin(X) * np.cos(Y)], -1) * np.sin(w * t) / w

    def fH(x, t):
        return np.cos(np.pi * x[..., 0]) * np.cos(np.pi * x[..., 1]) * np.cos(w * t)

    T = 0.25
    for p in (2, 3):
        errs = []
        for n in (4, 8):
            m = square_tri_mesh(n)
            dg = OracleDG2D(m.xy, m.tris, p, 1.0, 1.0)
            E0, H0 = dg.project(fE=lambda x: fE(x, 0.0), fH=lambda x: fH(x, 0.0))
            steps = int(np.ceil(T / (0.2 / n / p ** 2)))
            E, _, W = dg.run(E0, H0, T / steps, steps)
            e, r = dg.l2_error(E, lambda x: fE(x, T))
            errs.append(e / r)
            assert np.abs(W - W[0]).max() < 1e-12 * W[0]
        rate = np.log2(errs[0] / errs[1])
        assert p - 1 - 0.2 < rate < p - 1 + 0.6, (p, errs, rate)
