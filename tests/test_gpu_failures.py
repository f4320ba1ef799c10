"""Failure paths of the library, reached without faulting the GPU.

* An unstable time step (3x the bound dgm_estimate_dt reports, Sec. 3's
  stability condition read as dt <= 2 / sqrt(rho)) makes the energy grow; the
  energy watchdog of dgm_run returns DGM_ERR_UNSTABLE.
* The tensor-core kernels bound every wait.  dgm_inject_wait_timeout makes the
  next phase launch wait on a barrier that nothing arrives at; the wait runs
  out after about a millisecond, before any copy or MMA is in flight, and the
  host reports DGM_ERR_TIMEOUT.  The problem stays usable: the same run
  repeated afterwards gives bitwise the fields of a fresh problem.
"""

import numpy as np
import pytest

from workloads.mesh import kuhn_cube_mesh

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1104_4208_gb300 import build
    build.build()
    from paper_1104_4208_gb300 import _capi
    return _capi


def _solver(m, p, eps, precision):
    from paper_1104_4208_gb300.solver import Solver
    return Solver(m.xyz, m.tets, p, eps, 1.0, precision=precision)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "tc32", "tc16", "tcbf16", "tc16x2"])
def test_unstable_time_step_is_reported(capi, precision):
    m = kuhn_cube_mesh(3, jitter=0.1, seed=31)
    eps = np.random.default_rng(32).uniform(1, 4, m.nt)
    S = _solver(m, 3, eps, precision)
    rng = np.random.default_rng(33)
    E0, H0 = rng.standard_normal(S.nE), rng.standard_normal(S.nH)
    S.set_fields(E0, H0)
    _, dt_max = capi.dgm_estimate_dt(S.prob, 60)
    # a stable run first: no error
    S.set_fields(E0, H0)
    S.run(0.5 * dt_max, 20, energies=True)
    S.set_fields(E0, H0)
    with pytest.raises(capi.DgmError) as e:
        S.run(3.0 * dt_max, 200, energies=True)
    assert e.value.code == capi.DGM_ERR_UNSTABLE
    S.close()


@pytest.mark.parametrize("precision", ["tc32", "tc16", "tcbf16", "tc16x2"])
def test_injected_wait_timeout_is_reported_and_recovered(capi, precision):
    m = kuhn_cube_mesh(4, jitter=0.1, seed=41)          # 384 tets: 3 tiles
    eps = np.random.default_rng(42).uniform(1, 4, m.nt)
    rng = np.random.default_rng(43)
    S = _solver(m, 3, eps, precision)
    E0, H0 = rng.standard_normal(S.nE), rng.standard_normal(S.nH)
    dt = 0.2 / 4 / 9
    S.set_fields(E0, H0)
    capi.dgm_inject_wait_timeout(S.prob, 1)
    with pytest.raises(capi.DgmError) as e:
        S.run(dt, 5, energies=True)
    assert e.value.code == capi.DGM_ERR_TIMEOUT
    # the error word was read and cleared; the same problem runs normally again
    S.set_fields(E0, H0)
    W = S.run(dt, 5, energies=True)
    E1, H1 = S.get_fields()
    R = _solver(m, 3, eps, precision)
    R.set_fields(E0, H0)
    Wr = R.run(dt, 5, energies=True)
    E2, H2 = R.get_fields()
    assert np.array_equal(E1, E2) and np.array_equal(H1, H2) and np.array_equal(W, Wr)
    # the injection counts launches; zero cancels; CUDA-core precisions have no waits
    capi.dgm_inject_wait_timeout(S.prob, 0)
    S.run(dt, 2)
    for prec in ("fp64", "fp32"):
        C = _solver(m, 2, eps, prec)
        with pytest.raises(capi.DgmError) as e:
            capi.dgm_inject_wait_timeout(C.prob, 1)
        assert e.value.code == capi.DGM_ERR_UNSUPPORTED
        C.close()
    S.close()
    R.close()
