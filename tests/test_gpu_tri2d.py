"""The 2D triangle solver (TE fields, dgm_problem2d_*) against the 2D oracle
(oracle/dg2d.py): one H-kick and one E-kick for p = 1..6 on jittered PEC and
periodic meshes with shuffled vertex order and eps ~ U[1,4], mu ~ U[1,2]; a
leapfrog trajectory with its modified energy; the refusals.
"""

import numpy as np
import pytest

from workloads.mesh2d import square_tri_mesh

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


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("periodic", [False, True])
@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
def test_2d_kick_parity(capi, p, periodic, precision):
    from oracle.dg2d import OracleDG2D
    from paper_1104_4208_gb300.solver import Solver2D
    m = square_tri_mesh(5, jitter=0.15, seed=11, periodic=periodic, shuffle_local=True)   # 50 triangles
    rng = np.random.default_rng(500 + p)
    eps = rng.uniform(1, 4, m.nt)
    mu = rng.uniform(1, 2, m.nt)
    dg = OracleDG2D(m.xy, m.tris, p, eps, mu, vertex_key=m.vertex_key)
    A = dg.assemble()
    S = Solver2D(m.xy, m.tris, p, eps, mu, vertex_key=m.vertex_key, precision=precision)
    assert (S.nE, S.nH) == (dg.sizeE, dg.sizeH)
    E0 = rng.standard_normal(S.nE)
    H0 = rng.standard_normal(S.nH)
    dt = 0.01
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
def test_2d_trajectory_and_energy(capi, precision):
    """50 leapfrog steps on a jittered PEC square (n = 4, p = 3, eps ~ U[1,4]):
    fields and the per-step modified energy vs the oracle; energy conserved."""
    from oracle.dg2d import OracleDG2D
    from paper_1104_4208_gb300.solver import Solver2D
    m = square_tri_mesh(4, jitter=0.1, seed=12, shuffle_local=True)
    rng = np.random.default_rng(13)
    eps = rng.uniform(1, 4, m.nt)
    p = 3
    dg = OracleDG2D(m.xy, m.tris, p, eps, 1.0)
    E0 = rng.standard_normal(dg.sizeE)
    H0 = rng.standard_normal(dg.sizeH)
    dt = 0.2 * 0.25 / p ** 2
    Eo, Ho, Wo = dg.run(E0, H0, dt, 50)
    S = Solver2D(m.xy, m.tris, p, eps, 1.0, precision=precision)
    S.set_fields(E0, H0)
    W = S.run(dt, 50, energies=True)
    E, H = S.get_fields()
    assert _rel(E, Eo) < TOL_TRAJ[precision]
    assert _rel(H, Ho) < TOL_TRAJ[precision]
    assert np.abs(W - Wo).max() / Wo[0] < TOL_TRAJ[precision]
    assert np.abs(W - W[0]).max() / W[0] < (1e-12 if precision == "fp64" else 1e-5)
    S.close()


def test_2d_refusals(capi):
    from paper_1104_4208_gb300.solver import Solver2D
    m = square_tri_mesh(2)
    with pytest.raises(capi.DgmError) as e:
        Solver2D(m.xy, m.tris, 2, 1.0, 1.0, precision="tc16")
    assert e.value.code == capi.DGM_ERR_UNSUPPORTED
    bad = m.xy.copy()
    bad[m.tris[0, 1]] = bad[m.tris[0, 0]]          # collapse one triangle
    with pytest.raises(capi.DgmError) as e:
        Solver2D(bad, m.tris, 2, 1.0, 1.0)
    assert e.value.code == capi.DGM_ERR_INVALID_ARG
    with pytest.raises(capi.DgmError):
        Solver2D(m.xy, m.tris, 0, 1.0, 1.0)
    with pytest.raises(capi.DgmError):
        Solver2D(m.xy, m.tris, 2, -1.0, 1.0)
