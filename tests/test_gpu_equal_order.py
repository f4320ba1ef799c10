"""The equal-order pair (E and H both of degree p: the option equal_order) on the
GPU against the oracle's equal-order operator (OracleDG(h_degree=p)).

Sec. 2 builds the scheme on V^{k+1} x V^k; the same weak form and flux (Sec. 2.1)
and time stepping (Sec. 3) on V^k x V^k give the equal-order pair, which the
oracle pins separately (skew-adjoint, exact on polynomials, energy conserving,
null space of the stabilized operator = discrete gradients).  Here: one H-kick and
one E-kick with the central flux for every CUDA-core kernel variant, and with the
stabilized flux (H and H^F updates, the H^F term of the E-kick); a stabilized
leapfrog trajectory with its modified energy; the projection onto the degree-p H
space; the refusal on the tensor-core precisions.
"""

import numpy as np
import pytest

from workloads.mesh import kuhn_cube_mesh

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 2e-5}
TOL_TRAJ = {"fp64": 1e-12, "fp32": 2e-4}


@pytest.fixture(scope="module")
def capi():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1104_4208_gb300 import build
    build.build()
    from paper_1104_4208_gb300 import _capi
    return _capi


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _solver(m, p, eps, mu, precision, flux="central", variant=0):
    from paper_1104_4208_gb300.solver import Solver
    return Solver(m.xyz, m.tets, p, eps, mu, vertex_key=m.vertex_key, precision=precision, flux=flux,
                  variant=variant, equal_order=True)


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("p", [1, 3, 5])
def test_equal_order_central_kicks(capi, p, precision, variant):
    """Central flux, 162 jittered tets (several element groups and a ragged tail),
    eps ~ U[1,4], mu ~ U[1,2]; variants: automatic, dense curl, sparse curl,
    element groups."""
    from oracle.dg import OracleDG
    m = kuhn_cube_mesh(3, jitter=0.15, seed=6, shuffle_local=True)
    rng = np.random.default_rng(300 + p)
    eps = rng.uniform(1, 4, m.nt)
    mu = rng.uniform(1, 2, m.nt)
    dg = OracleDG(m.xyz, m.tets, p, eps, mu, vertex_key=m.vertex_key, h_degree=p)
    A = dg.assemble()
    S = _solver(m, p, eps, mu, precision, variant=variant)
    assert S.nH == S.nE == dg.sizeH
    E0 = rng.standard_normal(S.nE)
    H0 = rng.standard_normal(S.nH)
    dt = 0.05
    S.set_fields(E0, H0)
    S.kick(0, dt)
    _, H = S.get_fields()
    assert _rel(H - H0, dt * dg._blockmul(A["MHinv"], A["CH"] @ E0)) < TOL[precision]
    S.set_fields(E0, H0)
    S.kick(1, dt)
    E, _ = S.get_fields()
    assert _rel(E - E0, dt * dg._blockmul(A["MEinv"], A["CE"] @ H0)) < TOL[precision]
    S.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("p", [2, 4])
def test_equal_order_stabilized_kicks(capi, p, precision):
    """Stabilized flux: the H-kick advances H and H^F from E, the E-kick includes the
    (H^F x nu_F, [[e]]) term."""
    from oracle.dg import OracleDG
    m = kuhn_cube_mesh(2, jitter=0.15, seed=5, shuffle_local=True)
    rng = np.random.default_rng(400 + p)
    eps = rng.uniform(1, 4, m.nt)
    dg = OracleDG(m.xyz, m.tets, p, eps, 1.0, vertex_key=m.vertex_key, flux="stabilized", h_degree=p)
    A = dg.assemble()
    S = _solver(m, p, eps, 1.0, precision, flux="stabilized")
    assert S.nHF == dg.sizeK
    E0 = rng.standard_normal(S.nE)
    H0 = rng.standard_normal(S.nH)
    K0 = rng.standard_normal(S.nHF)
    dt = 0.02
    S.set_fields(E0, H0, K0)
    S.kick(0, dt)
    _, H, K = S.get_fields()
    assert _rel(H - H0, dt * dg._blockmul(A["MHinv"], A["CH"] @ E0)) < TOL[precision]
    assert _rel(K - K0, dt * dg._blockmul(A["MFinv"], A["S"] @ E0)) < TOL[precision]
    S.set_fields(E0, H0, K0)
    S.kick(1, dt)
    E, _, _ = S.get_fields()
    dE = dt * dg._blockmul(A["MEinv"], A["CE"] @ H0 + A["CEK"] @ K0)
    assert _rel(E - E0, dE) < TOL[precision]
    S.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_equal_order_stabilized_trajectory(capi, precision):
    """30 leapfrog steps with the stabilized flux on a jittered PEC cube (n = 3,
    p = 3, eps ~ U[1,4]): fields, H^F and the modified energy vs the oracle, and the
    energy conserved."""
    from oracle.dg import OracleDG
    m = kuhn_cube_mesh(3, jitter=0.1, seed=31, shuffle_local=True)
    rng = np.random.default_rng(32)
    eps = rng.uniform(1, 4, m.nt)
    p = 3
    dg = OracleDG(m.xyz, m.tets, p, eps, 1.0, flux="stabilized", h_degree=p)
    E0 = rng.standard_normal(dg.sizeE)
    H0 = rng.standard_normal(dg.sizeH)
    dt = 0.1 * (1 / 3) / p ** 2
    Eo, Ho, Ko, Wo = dg.run(E0, H0, dt, 30)
    S = _solver(m, p, eps, 1.0, precision, flux="stabilized")
    S.set_fields(E0, H0, np.zeros(S.nHF))
    W = S.run(dt, 30, energies=True)
    E, H, K = S.get_fields()
    assert _rel(E, Eo) < TOL_TRAJ[precision]
    assert _rel(H, Ho) < TOL_TRAJ[precision]
    assert _rel(K, Ko) < TOL_TRAJ[precision]
    assert np.abs(W - Wo).max() / Wo[0] < TOL_TRAJ[precision]
    assert np.abs(W - W[0]).max() / W[0] < (1e-11 if precision == "fp64" else 1e-5)
    S.close()


def test_equal_order_projection(capi):
    """Fields of degree p (cubic at p = 3) lie in the equal-order spaces: the
    library's projection onto the degree-p H space reproduces the oracle's (both
    exact for these fields), which the default degree p - 1 space could not."""
    from oracle.dg import OracleDG
    from oracle.project import project
    m = kuhn_cube_mesh(2, jitter=0.1, seed=7)
    p = 3
    dg = OracleDG(m.xyz, m.tets, p, 1.0, 1.0, h_degree=p)
    fE = lambda x: np.stack([x[..., 1] ** 2 * x[..., 2], x[..., 0] * x[..., 2], x[..., 0] ** 3], -1)
    fH = lambda x: np.stack([x[..., 1] ** 3, x[..., 2] ** 2 * x[..., 0], x[..., 0] * x[..., 1] * x[..., 2]], -1)
    S = _solver(m, p, 1.0, 1.0, "fp64")
    S.project(lambda x: (fE(x), fH(x)))
    E, H = S.get_fields()
    assert _rel(H, project(dg, fH, p)) < 1e-11
    assert _rel(E, project(dg, fE, p)) < 1e-11
    S.close()


def test_equal_order_refused_on_tensor_cores(capi):
    m = kuhn_cube_mesh(1)
    for prec in ("tc32", "tc16", "tcbf16", "tc16x2"):
        with pytest.raises(capi.DgmError) as e:
            _solver(m, 2, 1.0, 1.0, prec)
        assert e.value.code == capi.DGM_ERR_UNSUPPORTED
