"""The allocation-free energy entry point against the allocating one.

dgm_energy_noalloc exists for callers that may not allocate device memory
(for instance applications whose pool allocator owns the whole device); it
keeps its partial sums in a fixed device array instead.  This test calls it
through the C ABI twice in a row, on two different states of the same
problem, and checks each result against dgm_energy on that state, for every
precision (the tensor-core ones reduce the tiled state's partial sums).  The
second call must leave the device's free memory unchanged.  It lives in its
own file, collected last, and passes both alone in a fresh process and after
the other GPU tests.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "fp32", "tc32", "tc16", "tcbf16", "tc16x2"])
def test_energy_noalloc_matches_dgm_energy(precision):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1104_4208_gb300 import build
    build.build()
    from paper_1104_4208_gb300 import _capi as capi
    from paper_1104_4208_gb300.solver import Solver
    from workloads.mesh import kuhn_cube_mesh

    m = kuhn_cube_mesh(3, jitter=0.1, seed=12, shuffle_local=True)
    rng = np.random.default_rng(21)
    eps = rng.uniform(1, 4, m.nt)
    S = Solver(m.xyz, m.tets, 3, eps, 1.0, precision=precision)
    S.set_fields(rng.standard_normal(S.nE), rng.standard_normal(S.nH))
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    capi.dgm_energy_noalloc(S.prob, out[0:1].data_ptr(), stream.cuda_stream)
    torch.cuda.synchronize()
    ref0 = S.energy()

    S.kick(0, 0.01)
    S.kick(1, 0.01)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    capi.dgm_energy_noalloc(S.prob, out[1:2].data_ptr(), stream.cuda_stream)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    ref1 = S.energy()

    got = out.cpu().numpy()
    assert abs(got[0] - ref0) <= 1e-12 * abs(ref0)
    assert abs(got[1] - ref1) <= 1e-12 * abs(ref1)
    assert ref0 != ref1
    assert free1 == free0, (free0, free1)
    S.close()
