"""Pins of the FP64 oracle to facts the paper and the mathematics fix.

Each test would fail for a plausible slip in the oracle: a wrong Jacobi
parameter or index (basis vs the printed formula, printed 2D relations,
orthogonality/norms), a transposed or mis-signed operand in the curl or the
fluxes (skew-adjointness, exact curl of polynomial fields), a wrong mass scaling
(flat-element closed form), a dropped facet term (consistency, energy).
"""

import math
import os
from fractions import Fraction

import numpy as np
import pytest
import sympy as sp

from oracle.basis import phi3, psi2, index3, index2, legendre
from oracle.quadrature import tet_rule, tri_rule
from oracle.dg import OracleDG
from oracle.project import project, l2_error
from workloads.mesh import kuhn_cube_mesh
from workloads.fields import te110_fields

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- basis
def _sympy_phi3(i, j, k):
    X, Y, Z = sp.symbols("x y z")
    phi = ((1 - X - Y) ** i * (1 - X) ** j * sp.legendre(i, 2 * Z / (1 - X - Y) - 1)
           * sp.jacobi(j, 2 * i + 1, 0, 2 * Y / (1 - X) - 1)
           * sp.jacobi(k, 2 * i + 2 * j + 2, 0, 2 * X - 1))
    return (X, Y, Z), phi


def test_phi3_matches_printed_formula_sympy():
    """Sec. 4.2.2 definition, evaluated exactly by sympy at rational points."""
    p = 3
    rng = np.random.default_rng(11)
    pts = []
    for _ in range(4):
        a, b, c = rng.integers(1, 20, size=3)
        s = a + b + c + rng.integers(1, 10)
        pts.append((Fraction(int(a), int(s)), Fraction(int(b), int(s)), Fraction(int(c), int(s))))
    P = np.array([[float(v) for v in q] for q in pts])
    val, grad = phi3(p, P)
    for r, (i, j, k) in enumerate(index3(p)):
        (X, Y, Z), phi = _sympy_phi3(i, j, k)
        dphi = [sp.diff(phi, v) for v in (X, Y, Z)]
        for q, pt in enumerate(pts):
            sub = {X: sp.Rational(pt[0].numerator, pt[0].denominator),
                   Y: sp.Rational(pt[1].numerator, pt[1].denominator),
                   Z: sp.Rational(pt[2].numerator, pt[2].denominator)}
            assert val[r, q] == pytest.approx(float(phi.subs(sub)), abs=1e-13)
            for d in range(3):
                assert grad[r, q, d] == pytest.approx(float(dphi[d].subs(sub)), abs=1e-12)


# the 16 monomials of the printed support of the 3D d/dx relation (Sec. 4.2.2):
# shifts (i, j, k) of the terms with D_x, then of the terms without
_SUPPORT_DX_D = [(1, 1, 2), (1, 0, 3), (0, 2, 2), (0, 1, 3), (1, 1, 1), (1, 0, 2), (0, 2, 1), (0, 1, 2),
                 (1, 1, 0), (1, 0, 1), (0, 2, 0), (0, 1, 1)]
_SUPPORT_DX_0 = [(1, 1, 1), (1, 0, 2), (0, 2, 1), (0, 1, 2)]


def _support_nullspace(i, j, k, drop=None):
    """Rational nullspace of sum_m c_m D_x phi_{(i,j,k)+s_m} + sum_m c_m phi_{(i,j,k)+s_m} = 0
    as a polynomial identity (coefficient comparison in x, y, z)."""
    cols = []
    for s, deriv in [(s, True) for s in _SUPPORT_DX_D] + [(s, False) for s in _SUPPORT_DX_0]:
        (X, Y, Z), phi = _sympy_phi3(i + s[0], j + s[1], k + s[2])
        poly = sp.Poly(sp.expand(sp.cancel(sp.together(phi))), X, Y, Z)
        cols.append(poly.diff(X) if deriv else poly)
    if drop is not None:
        cols = [c for n, c in enumerate(cols) if n != drop]
    monos = sorted({m for c in cols for m in c.as_dict()})
    return sp.Matrix([[c.as_dict().get(m, 0) for c in cols] for m in monos]).nullspace()


def test_printed_3d_dx_support_carries_one_relation():
    """Sec. 4.2.2 names the 16 monomials of the d/dx relation for the 3D shape
    functions (coefficients not printed).  At generic indices the ansatz on that
    support has exactly one solution (up to scale), with all 16 coefficients
    nonzero, so the support is minimal; without the leading term S_j S_k^3 D_x
    no relation is left.  Exact rational arithmetic."""
    for ijk in [(1, 0, 1), (1, 1, 1), (2, 1, 0)]:
        ns = _support_nullspace(*ijk)
        assert len(ns) == 1, ijk
        assert all(v != 0 for v in ns[0]), ijk
    assert len(_support_nullspace(1, 1, 1, drop=3)) == 0


def test_psi2_matches_eq4_sympy():
    X, Y = sp.symbols("x y")
    pts = [(sp.Rational(1, 7), sp.Rational(2, 5)), (sp.Rational(3, 8), sp.Rational(1, 9))]
    P = np.array([[float(a), float(b)] for a, b in pts])
    val, grad = psi2(3, P, grad=True)
    for r, (i, j) in enumerate(index2(3)):
        psi = sp.legendre(i, 2 * Y / (1 - X) - 1) * (1 - X) ** i * sp.jacobi(j, 2 * i + 1, 0, 2 * X - 1)
        for q, (a, b) in enumerate(pts):
            assert val[r, q] == pytest.approx(float(psi.subs({X: a, Y: b})), abs=1e-13)
            assert grad[r, q, 0] == pytest.approx(float(sp.diff(psi, X).subs({X: a, Y: b})), abs=1e-12)
            assert grad[r, q, 1] == pytest.approx(float(sp.diff(psi, Y).subs({X: a, Y: b})), abs=1e-12)


def test_quadrature_exact_on_monomials():
    """int_T x^a y^b z^c = a! b! c! / (a+b+c+3)!  (exact for total degree <= 2q-1)."""
    q = 4
    x, w = tet_rule(q)
    for a in range(8):
        for b in range(8 - a):
            for c in range(8 - a - b):
                exact = math.factorial(a) * math.factorial(b) * math.factorial(c) / math.factorial(a + b + c + 3)
                got = np.sum(w * x[:, 0] ** a * x[:, 1] ** b * x[:, 2] ** c)
                assert got == pytest.approx(exact, rel=1e-13, abs=1e-16)
    s, ws = tri_rule(q)
    for a in range(8):
        for b in range(8 - a):
            exact = math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
            assert np.sum(ws * s[:, 0] ** a * s[:, 1] ** b) == pytest.approx(exact, rel=1e-13)


@pytest.mark.parametrize("p", [1, 3, 6])
def test_orthogonality_and_closed_form_norms(p):
    """L2-orthogonality (Sec. 3.1, Sec. 4.2.2) with
    ||phi_ijk||^2 = 1/(2(2i+1)(i+j+1)(2i+2j+2k+3)), ||psi_ij||^2 = 1/(2(2i+1)(i+j+1))."""
    x, w = tet_rule(p + 2)
    v, _ = phi3(p, x)
    M = (v * w) @ v.T
    d = np.array([1.0 / (2 * (2 * i + 1) * (i + j + 1) * (2 * i + 2 * j + 2 * k + 3))
                  for i, j, k in index3(p)])
    assert np.abs(M - np.diag(d)).max() < 1e-15 * max(1, p)
    assert d[0] == pytest.approx(1.0 / 6.0)
    s, ws = tri_rule(p + 2)
    pv = psi2(p, s)
    M2 = (pv * ws) @ pv.T
    d2 = np.array([1.0 / (2 * (2 * i + 1) * (i + j + 1)) for i, j in index2(p)])
    assert np.abs(M2 - np.diag(d2)).max() < 1e-15 * max(1, p)


def _read_relations(name):
    rel = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = [t.strip() for t in line.split("|")]
            rel.setdefault(parts[0], []).append(parts[1:])
    return rel


def test_printed_2d_relations_hold():
    """The two printed 2D FindRelation outputs of Sec. 4.2.1 annihilate phi_ij of Eq. (4)."""
    rel = _read_relations("relations_2d.txt")
    pmax = 12
    rng = np.random.default_rng(5)
    pts = rng.uniform(0.05, 0.45, size=(7, 2))
    val, grad = psi2(pmax, pts, grad=True)
    pos = {ij: r for r, ij in enumerate(index2(pmax))}
    I, J = sp.symbols("i j")
    for name, dcomp in (("dx", 0), ("dy", 1)):
        terms = [(sp.sympify(c, locals={"i": I, "j": J}), int(si), int(sj), int(d))
                 for c, si, sj, d in rel[name]]
        for i in range(4):
            for j in range(4):
                total = np.zeros(len(pts))
                scale = 0.0
                for coef, si, sj, d in terms:
                    c = float(coef.subs({I: i, J: j}))
                    r = pos[(i + si, j + sj)]
                    f = grad[r, :, dcomp] if d else val[r]
                    total += c * f
                    scale = max(scale, np.abs(c * f).max())
                assert np.abs(total).max() <= 1e-12 * scale, (name, i, j)


def test_printed_relations_are_not_vacuous():
    """Changing one printed coefficient breaks the dx relation (guards the test above)."""
    rel = _read_relations("relations_2d.txt")
    pts = np.array([[0.2, 0.3], [0.1, 0.15]])
    val, grad = psi2(8, pts, grad=True)
    pos = {ij: r for r, ij in enumerate(index2(8))}
    I, J = sp.symbols("i j")
    terms = [(sp.sympify(c, locals={"i": I, "j": J}), int(si), int(sj), int(d)) for c, si, sj, d in rel["dx"]]
    i, j = 1, 1
    total = 0.0
    for n, (coef, si, sj, d) in enumerate(terms):
        c = float(coef.subs({I: i, J: j})) * (1.01 if n == 0 else 1.0)
        r = pos[(i + si, j + sj)]
        total = total + c * (grad[r, :, 0] if d else val[r])
    assert np.abs(total).max() > 1e-6


def test_legendre_worked_example():
    """Eq. (5) and the ansatz solution of Sec. 4.1, plus the backward sweep of Sec. 3.2.2
    reproducing exact differentiation of a random Legendre series."""
    rel = _read_relations("legendre_relation.txt")["term"]
    x = np.linspace(-0.95, 0.95, 9)
    N = 12
    P = legendre(N + 2, x)
    h = 1e-6
    dP = (legendre(N + 2, x + h) - legendre(N + 2, x - h)) / (2 * h)
    nsym = sp.Symbol("n")
    for n in range(N):
        s = sum(float(sp.sympify(c, locals={"n": nsym}).subs(nsym, n)) * (dP if int(d) else P)[n + int(sh)]
                for c, sh, d in rel)
        assert np.abs(s).max() < 1e-7
    # backward sweep: v' = sum w_i P_i
    rng = np.random.default_rng(3)
    v = rng.standard_normal(N + 1)
    vt = v.copy()
    wv = np.zeros(N)
    for n in range(N, 0, -1):
        wv[n - 1] = (2 * n - 1) * vt[n]
        if n - 2 >= 0:
            vt[n - 2] += vt[n]
    lhs = v @ dP[: N + 1]
    rhs = wv @ P[:N]
    assert np.abs(lhs - rhs).max() < 1e-6 * np.abs(lhs).max()


# -------------------------------------------------------------- operator
def _mesh(kind):
    if kind == "jitter":
        return kuhn_cube_mesh(2, jitter=0.15, seed=5, shuffle_local=True)
    if kind == "periodic":
        return kuhn_cube_mesh(3, periodic=True, shuffle_local=True, seed=2)
    return kuhn_cube_mesh(2)


@pytest.mark.parametrize("kind", ["plain", "jitter", "periodic"])
@pytest.mark.parametrize("flux", ["central", "stabilized"])
def test_skew_adjointness(kind, flux):
    """Eq. (2): the evolution matrix is antisymmetric, r_E = -C^T H (and -S^T K)."""
    m = _mesh(kind)
    eps = np.random.default_rng(1).uniform(1, 4, m.nt)
    dg = OracleDG(m.xyz, m.tets, 2, eps, 1.0, vertex_key=m.vertex_key, flux=flux)
    A = dg.assemble()
    CH, CE = A["CH"].toarray(), A["CE"].toarray()
    assert np.abs(CE + CH.T).max() <= 1e-14 * np.abs(CH).max()
    if flux == "stabilized":
        S, CEK = A["S"].toarray(), A["CEK"].toarray()
        assert np.abs(CEK + S.T).max() <= 1e-14 * np.abs(S).max()


def test_mesh_topology_counts():
    m = kuhn_cube_mesh(3)
    dg = OracleDG(m.xyz, m.tets, 1, 1.0, 1.0)
    assert (dg.geo.nbr < 0).sum() == 12 * 9           # 6 sides x n^2 squares x 2 triangles
    mp = kuhn_cube_mesh(3, periodic=True)
    dgp = OracleDG(mp.xyz, mp.tets, 1, 1.0, 1.0, vertex_key=mp.vertex_key)
    assert (dgp.geo.nbr < 0).sum() == 0
    assert dgp.nfaces == 2 * dgp.nt
    # neighbour relation is an involution
    g = dgp.geo
    t = np.arange(g.nt)
    for f in range(4):
        assert np.all(g.nbr[g.nbr[t, f], g.nbr_face[t, f]] == t)


def _poly_fields():
    def E(x):
        X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
        o = np.zeros(x.shape)
        o[..., 0] = Y * (1 - Y) * Z * (1 - Z)
        o[..., 2] = X * (1 - X) * Y * (1 - Y)
        return o

    def curlE(x):
        X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
        o = np.zeros(x.shape)
        o[..., 0] = X * (1 - X) * (1 - 2 * Y)
        o[..., 1] = Y * (1 - Y) * (1 - 2 * Z) - (1 - 2 * X) * Y * (1 - Y)
        o[..., 2] = -(1 - 2 * Y) * Z * (1 - Z)
        return o

    def H(x):
        X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
        return np.stack([Y ** 2 * Z, X * Z ** 2, X ** 3], -1)

    def curlH(x):
        X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
        return np.stack([-2 * X * Z, Y ** 2 - 3 * X ** 2, Z ** 2 - 2 * Y * Z], -1)
    return E, curlE, H, curlH


def test_exact_curl_of_polynomial_fields():
    """Sec. 3.2.2: the modal curl is exact for polynomials of the space; a continuous
    field with vanishing tangential trace on the PEC boundary has no jumps, so one
    H-kick gives exactly -curl E and one E-kick exactly curl H (consistency).
    A flipped facet sign or a dropped facet term fails this."""
    p = 4
    m = kuhn_cube_mesh(2, jitter=0.15, seed=5, shuffle_local=True)
    dg = OracleDG(m.xyz, m.tets, p, 1.0, 1.0)
    E, curlE, H, curlH = _poly_fields()
    A = dg.assemble()
    Ec = project(dg, E, p)
    dH = dg._blockmul(A["MHinv"], A["CH"] @ Ec)
    c = project(dg, curlE, p - 1)
    assert np.abs(dH + c).max() < 1e-12 * np.abs(c).max()
    Hc = project(dg, H, p - 1)
    dE = dg._blockmul(A["MEinv"], A["CE"] @ Hc)
    ce = project(dg, curlH, p)
    assert np.abs(dE - ce).max() < 1e-11 * np.abs(ce).max()


def test_local_kicks_exact_and_equal_to_assembly():
    """The element-local kick path (used for sampled parity at full size) gives the
    exact curl of the polynomial fields of the test above on every element, and on
    random fields the same kicks as the assembled operator."""
    p = 4
    m = kuhn_cube_mesh(2, jitter=0.15, seed=5, shuffle_local=True)
    dg = OracleDG(m.xyz, m.tets, p, 1.0, 1.0)
    E, curlE, H, curlH = _poly_fields()
    ts = np.arange(dg.nt)
    c = project(dg, curlE, p - 1)
    dH = dg.local_kick_H(project(dg, E, p), ts, 1.0).ravel()
    assert np.abs(dH + c).max() < 1e-12 * np.abs(c).max()
    ce = project(dg, curlH, p)
    dE = dg.local_kick_E(project(dg, H, p - 1), ts, 1.0).ravel()
    assert np.abs(dE - ce).max() < 1e-11 * np.abs(ce).max()
    A = dg.assemble()
    rng = np.random.default_rng(8)
    Er, Hr = rng.standard_normal(dg.sizeE), rng.standard_normal(dg.sizeH)
    ref_H = 0.3 * dg._blockmul(A["MHinv"], A["CH"] @ Er)
    ref_E = 0.3 * dg._blockmul(A["MEinv"], A["CE"] @ Hr)
    assert np.abs(dg.local_kick_H(Er, ts, 0.3).ravel() - ref_H).max() < 1e-12 * np.abs(ref_H).max()
    assert np.abs(dg.local_kick_E(Hr, ts, 0.3).ravel() - ref_E).max() < 1e-12 * np.abs(ref_E).max()


def test_point_observation_and_source_closed_forms():
    """Point evaluation and the point source on a linear field, which the degree-2
    space reproduces exactly: the observation rows give the field at the points,
    point_values gives it at mapped reference points, located reference points map
    back to the physical points, and the dipole source vector contracted with the
    field's coefficients is -f dir . E(x_s) (its entries are -f dir . N_{a,m}(x_s))."""
    from oracle.dg import observation_matrix, locate_points, dipole_source_vector
    from oracle.project import point_values
    m = kuhn_cube_mesh(2, jitter=0.15, seed=5, shuffle_local=True)
    dg = OracleDG(m.xyz, m.tets, 2, 1.0, 1.0)
    A = np.array([[0.3, -1.0, 0.2], [0.5, 0.1, -0.7], [1.1, 0.4, 0.0]])
    b = np.array([0.2, -0.1, 0.4])
    lin = lambda x: x @ A.T + b
    Ec = project(dg, lin, 2)
    rng = np.random.default_rng(21)
    pts = rng.uniform(0.05, 0.95, (6, 3))
    P = observation_matrix(dg, pts)
    assert np.abs((P @ Ec).reshape(-1, 3) - lin(pts)).max() < 1e-12
    ts, xhs = locate_points(dg, pts)
    for t, xh, x in zip(ts, xhs, pts):
        assert np.abs(dg.geo.to_phys(t, xh) - x).max() < 1e-14
        assert xh.min() > -1e-12 and xh.sum() < 1 + 1e-12
        assert np.abs(point_values(dg, Ec, 2, t, xh[None, :])[0] - lin(x)).max() < 1e-12
    xs, d, f = np.array([0.43, 0.52, 0.47]), np.array([0.3, -0.2, 0.9]), 1.7
    src = dipole_source_vector(dg, xs, d, f)
    assert src @ Ec == pytest.approx(-f * d @ lin(xs), rel=1e-12)


def test_flat_mass_closed_form():
    """Sec. 3.3.1: flat elements, constant eps: M = |det F| eps (F^{-1} F^{-T}) (x) diag(||phi||^2)."""
    p = 3
    m = kuhn_cube_mesh(2, jitter=0.15, seed=5, shuffle_local=True)
    eps = np.random.default_rng(2).uniform(1, 4, m.nt)
    dg = OracleDG(m.xyz, m.tets, p, eps, 1.0)
    ts = np.arange(dg.nt)
    M = dg.mass_blocks(ts, "E")
    d = np.array([1.0 / (2 * (2 * i + 1) * (i + j + 1) * (2 * i + 2 * j + 2 * k + 3)) for i, j, k in index3(p)])
    for t in ts:
        G = abs(dg.geo.detF[t]) * eps[t] * dg.geo.Finv[t] @ dg.geo.Finv[t].T
        ref = np.kron(G, np.diag(d))
        assert np.abs(M[t] - ref).max() < 1e-13 * np.abs(ref).max()


def test_geometry_free_reference_integrals():
    """Sec. 3.2.1: (H, curl e)_T and the facet integrals equal the reference-element
    ones up to sign, so the physical blocks of every element are sign(det F) times
    those of the reference tetrahedron."""
    p = 3
    m = kuhn_cube_mesh(2, jitter=0.15, seed=5, shuffle_local=True)
    dg = OracleDG(m.xyz, m.tets, p, 1.0, 1.0)
    ref_xyz = np.array([[0., 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]])
    dgr = OracleDG(ref_xyz, np.array([[0, 1, 2, 3]]), p, 1.0, 1.0)
    VHr, VEr = dgr.volume_blocks(np.array([0]))
    ts = np.arange(dg.nt)
    VH, VE = dg.volume_blocks(ts)
    s = np.sign(dg.geo.detF)
    assert np.abs(VH - s[:, None, None] * VHr).max() < 1e-12 * np.abs(VHr).max()
    for f in range(4):
        fr = dgr.face_blocks(np.array([0]), f)["AH_own"]      # PEC on the lone tet: c = 1
        fb = dg.face_blocks(ts, f)
        own = fb["AH_own"] * np.where(fb["nbr"] >= 0, 2.0, 1.0)[:, None, None]
        assert np.abs(own - s[:, None, None] * fr).max() < 1e-12 * np.abs(fr).max()


@pytest.mark.parametrize("flux", ["central", "stabilized"])
def test_energy_conserved(flux):
    """Sec. 2.1 / Sec. 3: antisymmetric evolution + symplectic Euler conserve the
    modified discrete energy to round-off."""
    m = kuhn_cube_mesh(2, jitter=0.1, seed=7)
    eps = np.random.default_rng(4).uniform(1, 4, m.nt)
    dg = OracleDG(m.xyz, m.tets, 3, eps, 1.0, flux=flux)
    rng = np.random.default_rng(0)
    E0 = rng.standard_normal(dg.sizeE)
    H0 = rng.standard_normal(dg.sizeH)
    _, _, _, W = dg.run(E0, H0, 0.2 * 0.5 / 9, 40)
    assert np.abs(W - W[0]).max() < 1e-13 * W[0]


def test_te110_cavity_convergence():
    """Analytic PEC cavity mode: errors shrink under h-refinement at p=3."""
    errs = []
    for n in (2, 4):
        m = kuhn_cube_mesh(n)
        dg = OracleDG(m.xyz, m.tets, 3, 1.0, 1.0)
        E0 = project(dg, lambda x: te110_fields(x, 0.0)[0], 3)
        H0 = project(dg, lambda x: te110_fields(x, 0.0)[1], 2)
        dt = 0.2 / n / 9
        N = int(round(0.25 / dt))
        E, H, _, _ = dg.run(E0, H0, dt, N)
        e, r = l2_error(dg, E, lambda x: te110_fields(x, N * dt)[0], 3)
        errs.append(e / r)
    assert errs[1] < 0.05
    assert errs[0] / errs[1] > 4.0


@pytest.mark.parametrize("flux,e_lo,e_hi", [("central", 0.8, 1.3), ("stabilized", 2.0, 9.0)])
def test_h_refinement_rates(flux, e_lo, e_hi):
    """TE110 cavity mode, p = 2 (E of degree 2, H of degree 1), n = 4 -> 8, to
    t = 0.25 with dt = 0.1 h / p^2.  H converges at rate p (about 2) with either
    flux.  E converges at rate p - 1 with the central flux, one order below H,
    as the flux is known to cost, and at rate >= p with the stabilized flux of
    Sec. 2.1.  Observed E rates: 1.0 and 2.3; H rates: 2.1 and 2.0."""
    rates_E, errs = [], []
    for n in (4, 8):
        m = kuhn_cube_mesh(n)
        dg = OracleDG(m.xyz, m.tets, 2, 1.0, 1.0, flux=flux)
        E0 = project(dg, lambda x: te110_fields(x, 0.0)[0], 2)
        H0 = project(dg, lambda x: te110_fields(x, 0.0)[1], 1)
        dt = 0.1 / n / 4
        N = int(round(0.25 / dt))
        E, H, _, _ = dg.run(E0, H0, dt, N)
        eE, rE = l2_error(dg, E, lambda x: te110_fields(x, N * dt)[0], 2)
        eH, rH = l2_error(dg, H, lambda x: te110_fields(x, N * dt)[1], 1)
        errs.append((eE / rE, eH / rH))
    rE = math.log2(errs[0][0] / errs[1][0])
    rH = math.log2(errs[0][1] / errs[1][1])
    assert e_lo < rE < e_hi, (rE, errs)
    assert rH > 1.7, (rH, errs)


def test_equal_order_variant():
    """The equal-order variant (E and H both of degree p; the scheme of Sec. 2.1 with
    V^k x V^k): skew-adjoint, exact on polynomial fields, energy conserving; with the
    stabilized flux its null space is still exactly the discrete gradients, with the
    central flux it keeps spurious modes; on the TE110 mode at p = 2, n = 4 -> 8
    (central) E converges at about p + 1 (observed 2.9) and H at about p (2.2)."""
    import scipy.linalg as sl
    p = 4
    m = kuhn_cube_mesh(2, jitter=0.15, seed=5, shuffle_local=True)
    dg = OracleDG(m.xyz, m.tets, p, 1.0, 1.0, h_degree=p)
    A = dg.assemble()
    CH, CE = A["CH"], A["CE"]
    assert abs(CE + CH.T).max() < 1e-14 * abs(CH).max()
    E, curlE, H, curlH = _poly_fields()
    c = project(dg, curlE, p)
    dH = dg._blockmul(A["MHinv"], CH @ project(dg, E, p))
    assert np.abs(dH + c).max() < 1e-12 * np.abs(c).max()
    ce = project(dg, curlH, p)
    dE = dg._blockmul(A["MEinv"], CE @ project(dg, H, p))
    assert np.abs(dE - ce).max() < 1e-11 * np.abs(ce).max()
    rng = np.random.default_rng(4)
    _, _, _, W = dg.run(rng.standard_normal(dg.sizeE), rng.standard_normal(dg.sizeH), 0.01, 20)
    assert np.abs(W - W[0]).max() < 1e-13 * W[0]
    # null spaces on the PEC cube, n = 2, p = 2
    mc = kuhn_cube_mesh(2)
    counts = {}
    for flux in ("central", "stabilized"):
        d2 = OracleDG(mc.xyz, mc.tets, 2, 1.0, 1.0, flux=flux, h_degree=2)
        A2 = d2.assemble()
        K = A2["CH"].toarray().T @ sl.block_diag(*A2["MHinv"]) @ A2["CH"].toarray()
        if flux == "stabilized":
            S = A2["S"].toarray()
            K = K + S.T @ sl.block_diag(*A2["MFinv"]) @ S
        ev = np.sort(sl.eigh(K, sl.block_diag(*A2["ME"]), eigvals_only=True))
        counts[flux] = int((ev <= 1e-8 * ev.max()).sum())
    assert counts["stabilized"] == (3 * 2 - 1) ** 3
    assert counts["central"] > counts["stabilized"] + 100
    # h-refinement rates, central flux, p = 2
    errs = []
    for n in (4, 8):
        mn = kuhn_cube_mesh(n)
        dn = OracleDG(mn.xyz, mn.tets, 2, 1.0, 1.0, h_degree=2)
        E0 = project(dn, lambda x: te110_fields(x, 0.0)[0], 2)
        H0 = project(dn, lambda x: te110_fields(x, 0.0)[1], 2)
        dt = 0.1 / n / 4
        N = int(round(0.25 / dt))
        En, Hn, _, _ = dn.run(E0, H0, dt, N)
        eE, rE = l2_error(dn, En, lambda x: te110_fields(x, N * dt)[0], 2)
        eH, rH = l2_error(dn, Hn, lambda x: te110_fields(x, N * dt)[1], 2)
        errs.append((eE / rE, eH / rH))
    assert math.log2(errs[0][0] / errs[1][0]) > 2.5, errs
    assert math.log2(errs[0][1] / errs[1][1]) > 1.8, errs


def test_spurious_modes_removed_by_stabilization():
    """Sec. 2.1: the central flux leaves many non-physical zero modes; the stabilized
    central flux removes them.  On the PEC unit cube (n=2, p=2) the null space of the
    stabilized curl-curl operator is exactly the discrete gradient space, the
    interior nodes of continuous P^{p+1}: ((p+1) n - 1)^3 = 125; the first nonzero
    eigenvalues approximate the cavity values 2 pi^2 (x3) and 3 pi^2 (x2)."""
    import scipy.linalg as sl
    p, n = 2, 2
    m = kuhn_cube_mesh(n)
    counts = {}
    for flux in ("central", "stabilized"):
        dg = OracleDG(m.xyz, m.tets, p, 1.0, 1.0, flux=flux)
        A = dg.assemble()
        CH = A["CH"].toarray()
        K = CH.T @ sl.block_diag(*A["MHinv"]) @ CH
        if flux == "stabilized":
            S = A["S"].toarray()
            K = K + S.T @ sl.block_diag(*A["MFinv"]) @ S
        ev = np.sort(sl.eigh(K, sl.block_diag(*A["ME"]), eigvals_only=True))
        zero = ev <= 1e-8 * ev.max()
        counts[flux] = int(zero.sum())
        if flux == "stabilized":
            nz = ev[~zero]
            assert np.allclose(nz[:3], 2 * np.pi ** 2, rtol=0.01)
            assert np.allclose(nz[3:5], 3 * np.pi ** 2, rtol=0.01)
    assert counts["stabilized"] == ((p + 1) * n - 1) ** 3
    assert counts["central"] > counts["stabilized"] + 500


def cube_cavity_frequencies(count):
    """Closed form for the PEC unit cube: omega = pi sqrt(l^2 + m^2 + n^2), l, m, n >= 0
    with at most one of them zero; two independent polarisations when all three are
    nonzero, one otherwise.  The `count` smallest, with multiplicity."""
    w = []
    for l in range(8):
        for m in range(8):
            for n in range(8):
                nz = (l > 0) + (m > 0) + (n > 0)
                if nz >= 2:
                    w += [math.pi * math.sqrt(l * l + m * m + n * n)] * (2 if nz == 3 else 1)
    return np.sort(w)[:count]


def test_cavity_resonances_converge_under_p_refinement():
    """Sec. 2.2 (Fig. 1): on a fixed coarse mesh the resonance frequencies converge
    as p grows.  PEC unit cube as one Kuhn cube (6 tets), stabilized central flux:
    the 8 smallest discrete frequencies approach the closed-form cavity values
    (pi sqrt 2 x3, pi sqrt 3 x2, pi sqrt 5 x3 of 6), the error falls at every step
    p = 3..6 (below 1e-3 at p = 6), and the discrete null space is the gradient
    space of continuous P^{p+1} with zero tangential trace, (p (n=1) )^3 = p^3."""
    from oracle.dg import resonances
    m = kuhn_cube_mesh(1)
    exact = cube_cavity_frequencies(8)
    errs = []
    for p in (3, 4, 5, 6):
        om, nnull = resonances(OracleDG(m.xyz, m.tets, p, 1.0, 1.0, flux="stabilized"))
        assert nnull == p ** 3
        errs.append(float(np.max(np.abs(om[:8] - exact) / exact)))
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-3 and errs[0] < 3e-2
    # h-refinement at fixed p agrees: n = 2, p = 3
    m2 = kuhn_cube_mesh(2)
    om, nnull = resonances(OracleDG(m2.xyz, m2.tets, 3, 1.0, 1.0, flux="stabilized"))
    assert nnull == (4 * 2 - 1) ** 3
    assert np.max(np.abs(om[:8] - exact) / exact) < 2e-3


@pytest.mark.parametrize("flux", ["central", "stabilized"])
def test_composed_integrators_have_their_order(flux):
    """Sec. 3 (any explicit integrator): the leapfrog and its symmetric triple-jump
    composition against the exact solution of the semi-discrete system,
    y(T) = expm(L T) y(0) with L the block operator of the kicks (one Kuhn cube,
    p = 2).  Halving dt divides the error by 4 (order 2) and by 16 (order 4); a
    step forward then backward returns the start (symmetric methods)."""
    import scipy.linalg as sl
    from oracle.dg import run_composed
    m = kuhn_cube_mesh(1)
    dg = OracleDG(m.xyz, m.tets, 2, 1.0, 1.0, flux=flux)
    A = dg.assemble()
    nE, nH = dg.sizeE, dg.sizeH
    nK = dg.sizeK if flux == "stabilized" else 0
    MEinv, MHinv = sl.block_diag(*A["MEinv"]), sl.block_diag(*A["MHinv"])
    L = np.zeros((nE + nH + nK, nE + nH + nK))
    L[:nE, nE:nE + nH] = MEinv @ A["CE"].toarray()
    L[nE:nE + nH, :nE] = MHinv @ A["CH"].toarray()
    if nK:
        L[:nE, nE + nH:] = MEinv @ A["CEK"].toarray()
        L[nE + nH:, :nE] = sl.block_diag(*A["MFinv"]) @ A["S"].toarray()
    rng = np.random.default_rng(0)
    E0, H0 = rng.standard_normal(nE), rng.standard_normal(nH)
    K0 = np.zeros(nK) if nK else None
    y0 = np.concatenate([E0, H0, np.zeros(nK)])
    T = 0.05
    yT = sl.expm(L * T) @ y0
    for order, lo, hi in ((2, 3.8, 4.2), (4, 14.0, 18.0)):
        errs = []
        for ns in (10, 20):
            E, H, K = run_composed(dg, E0, H0, T / ns, ns, order, K0=K0)
            y = np.concatenate([E, H, K if nK else np.zeros(0)])
            errs.append(np.linalg.norm(y - yT) / np.linalg.norm(yT))
        assert lo < errs[0] / errs[1] < hi, (order, errs)
    E, H, K = run_composed(dg, E0, H0, T / 10, 1, 4, K0=K0)
    E2, H2, _ = run_composed(dg, E, H, -T / 10, 1, 4, K0=K)
    assert np.abs(E2 - E0).max() < 1e-13 and np.abs(H2 - H0).max() < 1e-13


def test_adjoint_gradient_matches_finite_differences():
    """Discrete adjoint of the leapfrog (objective J = sum_n sum_o |E^n(x_o)|^2,
    derivative with respect to per-element eps) vs central finite differences with
    delta = 1e-6 eps_T, both on the oracle (brute force on a tiny case)."""
    from oracle.dg import adjoint_grad_eps, objective
    m = kuhn_cube_mesh(2, jitter=0.1, seed=3)
    p = 2
    rng = np.random.default_rng(0)
    eps = rng.uniform(1, 4, m.nt)
    dg = OracleDG(m.xyz, m.tets, p, eps, 1.0)
    E0 = rng.standard_normal(dg.sizeE) * 0.1
    H0 = rng.standard_normal(dg.sizeH) * 0.1
    pts = rng.uniform(0.1, 0.9, (4, 3))
    dt, N = 0.01, 20
    J, grad = adjoint_grad_eps(dg, E0, H0, dt, N, pts)
    assert J == pytest.approx(objective(dg, E0, H0, dt, N, pts), rel=1e-13)
    for T in (0, 5, 17, 33):
        d = 1e-6 * eps[T]
        ep, em = eps.copy(), eps.copy()
        ep[T] += d
        em[T] -= d
        fd = (objective(OracleDG(m.xyz, m.tets, p, ep, 1.0), E0, H0, dt, N, pts)
              - objective(OracleDG(m.xyz, m.tets, p, em, 1.0), E0, H0, dt, N, pts)) / (2 * d)
        assert grad[T] == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_adjoint_mu_gradient_matches_finite_differences():
    """dJ/d mu of the discrete adjoint (the multiplier of the H-kicks times the
    H-increments, including the opening half kick) vs central finite differences
    with delta = 1e-6 mu_T; dJ/d eps on the same case as a cross-check.  Both on
    the oracle, tiny case."""
    from oracle.dg import adjoint_grad, objective
    m = kuhn_cube_mesh(2, jitter=0.1, seed=4)
    p = 2
    rng = np.random.default_rng(1)
    eps = rng.uniform(1, 4, m.nt)
    mu = rng.uniform(1, 2, m.nt)
    dg = OracleDG(m.xyz, m.tets, p, eps, mu)
    E0 = rng.standard_normal(dg.sizeE) * 0.1
    H0 = rng.standard_normal(dg.sizeH) * 0.1
    pts = rng.uniform(0.1, 0.9, (4, 3))
    dt, N = 0.01, 20
    J, geps, gmu = adjoint_grad(dg, E0, H0, dt, N, pts)
    assert J == pytest.approx(objective(dg, E0, H0, dt, N, pts), rel=1e-13)
    for T in (0, 7, 21, 40):
        for which, g in (("mu", gmu), ("eps", geps)):
            c = mu if which == "mu" else eps
            d = 1e-6 * c[T]
            cp, cm = c.copy(), c.copy()
            cp[T] += d
            cm[T] -= d
            mk = (lambda v: OracleDG(m.xyz, m.tets, p, eps, v)) if which == "mu" else \
                 (lambda v: OracleDG(m.xyz, m.tets, p, v, mu))
            fd = (objective(mk(cp), E0, H0, dt, N, pts) - objective(mk(cm), E0, H0, dt, N, pts)) / (2 * d)
            # abs: rounding of the differenced objective (~1e-8 here) against gradients up to ~2
            assert g[T] == pytest.approx(fd, rel=1e-6, abs=1e-7), (which, T)
