"""The library's 2D reference tables (dgm_reference_table_2d, host, no GPU)
against the oracle's 2D basis and quadrature and against the 2D relations the
paper prints in Sec. 4.2.1.

* D_x, D_y and the edge traces equal the oracle's brute-force integrals of the
  Eq. (4) basis (oracle/basis.psi2, oracle/quadrature.tri_rule) to round-off.
* The derivative tables satisfy the printed relations exactly: a relation
  sum c (D_x) psi_{i+m, j+n} = 0 (tests/golden/relations_2d.txt) becomes, in the
  basis, sum over its D_x terms of c times column (i+m, j+n) of the unnormalised
  D_x, plus sum over its plain terms of c times the unit vector of (i+m, j+n),
  equal to zero.
"""

import os

import numpy as np
import pytest
import sympy as sp

from oracle.basis import index2, legendre, n2, psi2
from oracle.quadrature import tri_rule

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def capi():
    from paper_1104_4208_gb300 import build
    build.build()
    from paper_1104_4208_gb300 import _capi
    return _capi


def _norms(p):
    return np.array([1.0 / (2.0 * (2 * i + 1) * (i + j + 1)) for i, j in index2(p)])


@pytest.mark.parametrize("p", [1, 2, 4, 6])
def test_2d_derivative_tables_match_oracle(capi, p):
    x, w = tri_rule(p + 2)
    vE, gE = psi2(p, x, grad=True)
    vH = psi2(p - 1, x)
    nE, nH = np.sqrt(_norms(p)), np.sqrt(_norms(p - 1))
    assert np.allclose(capi.dgm_reference_table_2d(p, 8), _norms(p), rtol=1e-15, atol=0)
    for d in range(2):
        ref = np.einsum("q,bq,aq->ba", w, vH, gE[:, :, d]) / np.outer(nH, nE)
        got = capi.dgm_reference_table_2d(p, d).reshape(n2(p - 1), n2(p))
        assert np.abs(got - ref).max() < 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("p", [1, 3, 5])
def test_2d_edge_traces_match_oracle(capi, p):
    verts = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    s, ws = np.polynomial.legendre.leggauss(p + 3)
    s, ws = 0.5 * (s + 1.0), 0.5 * ws
    for deg, base in ((p, 2), (p - 1, 5)):
        nrm = np.sqrt(_norms(deg))
        for f in range(3):
            a, b = [v for v in range(3) if v != f]
            pts = verts[a][None, :] + s[:, None] * (verts[b] - verts[a])[None, :]
            psi = psi2(deg, pts) / nrm[:, None]
            L = legendre(deg, 2.0 * s - 1.0) * np.sqrt(2.0 * np.arange(deg + 1) + 1.0)[:, None]
            ref = np.einsum("q,gq,aq->ga", ws, L, psi)
            got = capi.dgm_reference_table_2d(p, base + f).reshape(deg + 1, n2(deg))
            assert np.abs(got - ref).max() < 1e-13 * max(np.abs(ref).max(), 1.0)


def _relations():
    out = {}
    for line in open(os.path.join(GOLDEN, "relations_2d.txt")):
        if line.startswith("#") or not line.strip():
            continue
        name, c, si, sj, d = [x.strip() for x in line.split("|")]
        out.setdefault(name, []).append((c, int(si), int(sj), int(d)))
    return out


@pytest.mark.parametrize("name,dcomp,reach", [("dx", 0, 3), ("dy", 1, 4)])
def test_2d_derivative_tables_satisfy_printed_relations(capi, name, dcomp, reach):
    I, J = sp.symbols("i j")
    terms = [(sp.sympify(c, locals={"i": I, "j": J}), si, sj, d) for c, si, sj, d in _relations()[name]]
    for i in range(4):
        for j in range(5 - i):
            P = i + j + reach
            pos = {ij: r for r, ij in enumerate(index2(P))}          # columns (degree <= P)
            row = {ij: r for r, ij in enumerate(index2(P - 1))}      # rows (degree <= P - 1)
            D = capi.dgm_reference_table_2d(P, dcomp).reshape(n2(P - 1), n2(P))
            Dun = D * np.sqrt(_norms(P))[None, :] / np.sqrt(_norms(P - 1))[:, None]
            total = np.zeros(n2(P - 1))
            scale = 0.0
            for coef, si, sj, d in terms:
                c = float(coef.subs({I: i, J: j}))
                if d:
                    v = c * Dun[:, pos[(i + si, j + sj)]]
                else:
                    v = np.zeros(n2(P - 1))
                    v[row[(i + si, j + sj)]] = c
                total += v
                scale = max(scale, np.abs(v).max())
            assert np.abs(total).max() < 1e-11 * scale, (name, i, j)


def test_2d_table_arguments(capi):
    with pytest.raises(capi.DgmError):
        capi.dgm_reference_table_2d(0, 0)
    with pytest.raises(capi.DgmError):
        capi.dgm_reference_table_2d(3, 9)


def test_2d_mesh_adjacency(capi):
    """The adjacency the 2D solver builds: an n x n square split into 2 n^2
    triangles has 3 n^2 + 2 n edges, 4 n on the boundary; with periodic keys
    3 n^2 edges and none on the boundary; refusals as for the solver."""
    from workloads.mesh2d import square_tri_mesh
    for n in (1, 3, 5):
        m = square_tri_mesh(n, jitter=0.1 if n > 1 else 0.0, seed=2, shuffle_local=True)
        assert capi.dgm_mesh2d_info(m.xy, m.tris) == (3 * n * n + 2 * n, 4 * n)
        if n > 1:
            mp = square_tri_mesh(n, periodic=True, shuffle_local=True, seed=3)
            assert capi.dgm_mesh2d_info(mp.xy, mp.tris, mp.vertex_key) == (3 * n * n, 0)
    m = square_tri_mesh(2)
    bad = m.xy.copy()
    bad[m.tris[0, 1]] = bad[m.tris[0, 0]]
    with pytest.raises(capi.DgmError) as e:
        capi.dgm_mesh2d_info(bad, m.tris)
    assert e.value.code == capi.DGM_ERR_INVALID_ARG
    tris = m.tris.copy()
    tris[0, 2] = m.nv
    with pytest.raises(capi.DgmError):
        capi.dgm_mesh2d_info(m.xy, tris)
    dup = np.concatenate([m.tris, m.tris[:1]])        # one edge shared by three triangles
    with pytest.raises(capi.DgmError):
        capi.dgm_mesh2d_info(m.xy, dup)

