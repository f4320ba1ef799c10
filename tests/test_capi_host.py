"""Host-side checks of the C-ABI library (no GPU needed).

The library must load and export every entry point that include/dgm.h
declares; the reference tables it generates on the host must agree with the
oracle's own quadrature of the printed basis; input validation must reject
bad meshes and arguments with the documented codes.
"""

import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def capi():
    from paper_1104_4208_gb300 import build
    build.build()
    from paper_1104_4208_gb300 import _capi
    return _capi


def _declared():
    src = open(os.path.join(ROOT, "include", "dgm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dgm_\w+)\s*\(", src)))


def test_exports_every_declared_symbol(capi):
    declared = _declared()
    assert len(declared) >= 18
    for name in declared:
        assert hasattr(capi._lib, name), name
    assert set(declared) <= set(capi.exported_symbols())


def test_version_and_defaults(capi):
    assert capi.dgm_version() >= 100
    o = capi.dgm_default_options()
    assert o.flux == capi.DGM_FLUX_CENTRAL and o.precision == capi.DGM_PREC_FP64 and o.alpha0 == 1.0
    assert o.variant == 0 and o.compensated == 0 and o.equal_order == 0


def test_options_struct_layout_matches_header(capi, tmp_path):
    """The binding's dgm_options has the C struct's size and field offsets."""
    import ctypes
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    fields = [f for f, _ in capi.dgm_options._fields_]
    src = tmp_path / "layout.c"
    body = "".join(f'    printf("{f} %zu\\n", offsetof(dgm_options, {f}));\n' for f in fields)
    src.write_text('#include "dgm.h"\n#include <stddef.h>\n#include <stdio.h>\nint main(void) {\n'
                   '    printf("size %zu\\n", sizeof(dgm_options));\n' + body + '    return 0;\n}\n')
    exe = tmp_path / "layout.out"
    r = subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    out = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                         timeout=60).stdout.splitlines())
    assert int(out["size"]) == ctypes.sizeof(capi.dgm_options)
    for f in fields:
        assert int(out[f]) == getattr(capi.dgm_options, f).offset, f


def _oracle_tables(p):
    from oracle.basis import phi3, psi2, index3
    from oracle.quadrature import tet_rule, tri_rule
    x, w = tet_rule(p + 2)
    vE, gE = phi3(p, x)
    vH, _ = phi3(p - 1, x)
    nE = np.sqrt((vE * w * vE).sum(1))
    nH = np.sqrt((vH * w * vH).sum(1))
    D = [((vH * w) @ gE[:, :, d].T) / nH[:, None] / nE[None, :] for d in range(3)]
    s, ws = tri_rule(p + 2)
    ps = psi2(p, s)
    nps = np.sqrt((ps * ws * ps).sum(1))
    V = np.array([[0., 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]])
    Tr = []
    for f in range(4):
        a, b, c = [v for v in range(4) if v != f]
        xh = V[a] + s[:, :1] * (V[b] - V[a]) + s[:, 1:] * (V[c] - V[a])
        ph, _ = phi3(p, xh)
        Tr.append(((ps * ws) @ ph.T) / nps[:, None] / nE[None, :])
    return D, Tr, nE ** 2


@pytest.mark.parametrize("p", [1, 2, 4, 6, 8])
def test_reference_tables_match_oracle_quadrature(capi, p):
    """Sec. 3.2.2 / 3.2.3 tables (orthonormal basis) vs the oracle's quadrature of the
    printed basis: derivative matrices, face traces and squared norms."""
    D, Tr, n2 = _oracle_tables(p)
    for d in range(3):
        got = capi.dgm_reference_table(p, d).reshape(D[d].shape)
        assert np.abs(got - D[d]).max() < 1e-12 * max(1.0, np.abs(D[d]).max())
    for f in range(4):
        got = capi.dgm_reference_table(p, 3 + f).reshape(Tr[f].shape)
        assert np.abs(got - Tr[f]).max() < 1e-13
    assert np.allclose(capi.dgm_reference_table(p, 7), n2, rtol=1e-13, atol=0)


def test_reference_table_rejects_bad_p(capi):
    with pytest.raises(capi.DgmError) as e:
        capi.dgm_reference_table(0, 0)
    assert e.value.code == -1
    with pytest.raises(capi.DgmError):
        capi.dgm_reference_table(capi.DGM_PMAX + 1, 0)


def test_device_absent_is_an_error_not_a_crash(capi):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(capi.DgmError) as e:
        capi.dgm_create(0)
    assert e.value.code == -3


def test_mesh_counts_and_adjacency(capi):
    from workloads.mesh import kuhn_cube_mesh
    for n in (1, 2, 3):
        m = kuhn_cube_mesh(n, jitter=0.1, seed=n, shuffle_local=True)
        h = capi.dgm_mesh_create(None, m.xyz, m.tets)
        nt, nf, nb = capi.dgm_mesh_info(h)
        assert nt == 6 * n ** 3
        assert nb == 12 * n * n
        assert 4 * nt == 2 * nf - nb
        capi.dgm_mesh_destroy(h)
    mp = kuhn_cube_mesh(3, periodic=True, shuffle_local=True, seed=4)
    h = capi.dgm_mesh_create(None, mp.xyz, mp.tets, mp.vertex_key)
    nt, nf, nb = capi.dgm_mesh_info(h)
    assert nb == 0 and nf == 2 * nt
    capi.dgm_mesh_destroy(h)


def test_mesh_validation_errors(capi):
    xyz = np.array([[0., 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 1], [0.5, 0.5, 0]])
    bad = [
        np.array([[0, 1, 2, 7]]),                 # id out of range
        np.array([[0, 1, 2, 2]]),                 # repeated vertex
        np.array([[0, 1, 2, 5]]),                 # coplanar: degenerate
        np.array([[0, 1, 2, 3], [1, 2, 0, 4], [0, 2, 1, 5 - 1]]),   # face (0,1,2) on three tets
    ]
    for tets in bad:
        with pytest.raises(capi.DgmError) as e:
            capi.dgm_mesh_create(None, xyz, tets)
        assert e.value.code == -1
    key = np.array([0, 1, 2, 3, 3, 5])          # vertices 3 and 4 share a key
    with pytest.raises(capi.DgmError):
        capi.dgm_mesh_create(None, xyz, np.array([[0, 1, 3, 4]]), key)


def test_tridiagonal_eigen_helper(capi):
    """Host helper of dgm_resonances: eigenvalues by Sturm bisection and unit
    eigenvectors by inverse iteration, against a dense symmetric eigensolver on
    matrices of the Lanczos kind (wide spread, clustered pairs, tiny couplings)."""
    import scipy.linalg as sl
    rng = np.random.default_rng(11)
    cases = [(rng.uniform(0, 1e4, 60), rng.uniform(0.1, 50, 59)),
             (np.repeat(rng.uniform(1, 10, 20), 2), np.tile([1e-9, 3.0], 20)[:39]),
             (np.array([2.5]), np.array([])),
             # 40 decoupled copies of one 3x3 block: every eigenvalue 40-fold, so inverse
             # iteration meets 40 near-zero pivots (the solve must not overflow)
             (np.tile([1.0, 2.0, 3.0], 40), np.tile([0.5, 0.5, 0.0], 40)[:119])]
    for d, e in cases:
        k = d.shape[0]
        T = np.diag(d) + (np.diag(e, 1) + np.diag(e, -1) if k > 1 else 0)
        ref, vref = np.linalg.eigh(T)
        vals, vecs = capi.dgm_tridiag_eig(d, e, 0, k, vectors=True)
        scale = np.abs(ref).max()
        assert np.max(np.abs(vals - ref)) <= 1e-13 * scale
        for i in range(k):
            y = vecs[i]
            assert abs(np.linalg.norm(y) - 1) < 1e-12
            assert np.linalg.norm(T @ y - vals[i] * y) <= 1e-10 * scale
        # a window of indices
        mid = capi.dgm_tridiag_eig(d, e, k // 3, k // 3 + 1)
        assert mid[0] == pytest.approx(ref[k // 3], abs=1e-13 * scale)
        sel = sl.eigvalsh_tridiagonal(d, e) if k > 1 else d
        assert np.allclose(np.sort(sel), ref, rtol=0, atol=1e-12 * scale)
    with pytest.raises(capi.DgmError) as ex:
        capi.dgm_tridiag_eig(np.ones(3), np.ones(2), 2, 2)
    assert ex.value.code == capi.DGM_ERR_INVALID_ARG


def _n3(q):
    return (q + 1) * (q + 2) * (q + 3) // 6


_PRINTED_DX = {(1, 1, 2, 1), (1, 0, 3, 1), (0, 2, 2, 1), (0, 1, 3, 1), (1, 1, 1, 1), (1, 0, 2, 1), (0, 2, 1, 1),
               (0, 1, 2, 1), (1, 1, 0, 1), (1, 0, 1, 1), (0, 2, 0, 1), (0, 1, 1, 1),
               (1, 1, 1, 0), (1, 0, 2, 0), (0, 2, 1, 0), (0, 1, 2, 0)}


def test_grad_supports(capi):
    """The d/dx support is the one printed in Sec. 4.2.2; each support's lead is
    its unique highest derivative term in the order (degree, k, j, i)."""
    sh, lead = capi.dgm_grad_support(0)
    assert set(map(tuple, sh)) == _PRINTED_DX and tuple(sh[lead]) == (0, 1, 3, 1)
    for d in (0, 1, 2):
        sh, lead = capi.dgm_grad_support(d)
        key = lambda s: (s[0] + s[1] + s[2], s[2], s[1], s[0])
        ders = [tuple(s) for s in sh if s[3] == 1]
        assert max(ders, key=key) == tuple(sh[lead])
        assert sum(1 for t in ders if key(t) == key(tuple(sh[lead]))) == 1
        # value terms are of degree one less than the lead
        assert all(s[0] + s[1] + s[2] == key(tuple(sh[lead]))[0] - 1 for s in sh if s[3] == 0)


@pytest.mark.parametrize("direction,ijk,p", [(0, (1, 1, 1), 7), (1, (1, 1, 1), 8), (2, (1, 0, 0), 8)])
def test_grad_recurrence_equals_exact_relation(capi, direction, ijk, p):
    """The library's numerically found relation against the exact rational
    nullspace of its support (sympy, direct symbolic differentiation of the
    printed 3D shape functions): one relation, equal coefficients."""
    sp = pytest.importorskip("sympy")
    X, Y, Z = sp.symbols("x y z")
    V = (X, Y, Z)[direction]

    def phi(i, j, k):
        e = ((1 - X - Y) ** i * (1 - X) ** j * sp.legendre(i, 2 * Z / (1 - X - Y) - 1)
             * sp.jacobi(j, 2 * i + 1, 0, 2 * Y / (1 - X) - 1) * sp.jacobi(k, 2 * i + 2 * j + 2, 0, 2 * X - 1))
        return sp.Poly(sp.expand(sp.cancel(sp.together(e))), X, Y, Z)
    sh, lead = capi.dgm_grad_support(direction)
    i, j, k = ijk
    cols = [phi(i + a, j + b, k + c).diff(V) if der else phi(i + a, j + b, k + c) for a, b, c, der in sh]
    monos = sorted({m for c in cols for m in c.as_dict()})
    ns = sp.Matrix([[c.as_dict().get(m, 0) for c in cols] for m in monos]).nullspace()
    assert len(ns) == 1
    exact = np.array([float(v / ns[0][lead]) for v in ns[0]])
    got_ijk, coef = capi.dgm_grad_recurrence(p, direction)
    r = [n for n, t in enumerate(got_ijk) if tuple(t) == ijk]
    assert len(r) == 1
    assert np.abs(coef[r[0]] - exact).max() < 1e-9 * np.abs(exact).max()


@pytest.mark.parametrize("direction", [0, 1, 2])
def test_grad_relations_hold_with_the_oracle_basis(capi, direction):
    """Every relation at p = 8 annihilates the oracle's phi and its derivative
    (textbook Jacobi recurrence, forward-mode derivatives) at points the library
    never sampled; relations exist at every index for x and y, and at i >= 1 for
    z (d/dz of phi_0jk vanishes, so those columns need none)."""
    from oracle.basis import phi3, index3
    p = 8
    sh, lead = capi.dgm_grad_support(direction)
    top = int(sh[lead][0] + sh[lead][1] + sh[lead][2])
    ijk, coef = capi.dgm_grad_recurrence(p, direction)
    assert sorted(map(tuple, ijk)) == sorted(t for t in index3(p - top) if t[0] >= 1 or direction < 2)
    rng = np.random.default_rng(2)
    pts = rng.dirichlet([1, 1, 1, 1], 40)[:, :3]
    val, grad = phi3(p, pts)
    pos = {t: r for r, t in enumerate(index3(p))}
    for (i, j, k), c in zip(ijk, coef):
        terms = [c[n] * (grad[pos[(i + a, j + b, k + cc)], :, direction] if der else val[pos[(i + a, j + b, k + cc)]])
                 for n, (a, b, cc, der) in enumerate(sh)]
        scale = max(np.abs(t).max() for t in terms)
        assert np.abs(sum(terms)).max() < 1e-10 * scale, (i, j, k)


@pytest.mark.parametrize("direction", [0, 1, 2])
@pytest.mark.parametrize("p", [1, 3, 6, 8])
def test_grad_sweep_equals_direct_differentiation(capi, direction, p):
    """The backward sweep (relations where they lead, dense columns elsewhere)
    against the derivative of the series projected by exact quadrature with the
    oracle's basis and the closed-form norms.  The sweep chains relations (at
    i = 0 the minimum-norm one of several), so rounding grows mildly with p:
    observed up to 3.7e-13 (x, p = 8), 3.3e-13 (y), 1.1e-13 (z)."""
    from oracle.basis import phi3, index3
    from oracle.quadrature import tet_rule
    rng = np.random.default_rng(10 * p + direction)
    a = rng.standard_normal(_n3(p))
    b, swept = capi.dgm_grad_sweep(p, direction, a)
    xq, wq = tet_rule(p + 2)
    _, grad = phi3(p, xq)
    valH, _ = phi3(p - 1, xq)
    du = a @ grad[:, :, direction]
    norms = np.array([1.0 / (2 * (2 * i + 1) * (i + j + 1) * (2 * i + 2 * j + 2 * k + 3)) for (i, j, k) in index3(p - 1)])
    ref = (valH * (wq * du)[None, :]).sum(1) / norms
    assert np.abs(b - ref).max() < 1e-12 * np.abs(ref).max()
    assert swept == len(capi.dgm_grad_recurrence(p, direction)[0])


def test_header_is_plain_c_and_links(capi, tmp_path):
    """The boundary is a C ABI: include/dgm.h compiles as pedantic C99, and a C
    program links against the library and calls a host-only entry point."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "t.c"
    src.write_text('#include "dgm.h"\n#include <stdio.h>\n'
                   'int main(void) {\n'
                   '    dgm_options o; double vals[2]; const double d[3] = {2.0, 2.0, 2.0}, e[2] = {1.0, 1.0};\n'
                   '    dgm_default_options(&o);\n'
                   '    if (dgm_tridiag_eig(3, d, e, 0, 2, vals, 0) != DGM_OK) return 1;\n'
                   '    printf("%d %.12f %.12f\\n", o.precision, vals[0], vals[1]);\n'
                   '    return 0;\n}\n')
    lib = os.path.dirname(capi.LIB_PATH)
    exe = tmp_path / "t.out"
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
                        str(src), "-L", lib, "-ldgm", f"-Wl,-rpath,{lib}", "-o", str(exe)],
                       capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stderr
    prec, l0, l1 = out.stdout.split()
    # eigenvalues of tridiag(1, 2, 1) of size 3: 2 - sqrt 2, 2, 2 + sqrt 2
    assert int(prec) == 0 and abs(float(l0) - (2 - 2 ** 0.5)) < 1e-12 and abs(float(l1) - 2.0) < 1e-12
