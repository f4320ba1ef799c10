"""The five named time-domain workloads (sizes, materials, initial data).

cavity_n4_p3      unit cube PEC, n=4 (384 tets), p=3, eps=mu=1, TE110 mode, 100 steps
pulse_n16_p4      unit cube PEC, n=16 (24,576 tets), jitter 0.15h, p=4, eps~U[1,4], mu=1,
                  Gaussian pulse (width 0.1, centre ~U[0.3,0.7]^3), H=0, 1,000 steps
planewave_n32_p6  periodic [0,1]^3, n=32 (196,608 tets), p=6, eps=mu=1,
                  plane wave k = 2 pi (1,2,3), 2,000 steps
pulse_n32_p4      the pulse_n16_p4 recipe on n=32 (196,608 tets, p=4): its state
                  (130 MB in fp32) no longer fits in the 129 MB L2
batched_64        64 runs, n in {8,12,16}, jitter 0.1h, p in {2..6}, eps~U[1,4], dipole source, 500 steps
                  (make_workload("batched_64:r") builds run r alone)
adjoint_n16_p4    mesh/p of pulse_n16_p4, 8 observation points, 500 steps, checkpoint every 50

The time step is dt = 0.2 h / p^2 with h = 1/n, the polynomial order p is the
degree of E.  Seeds: 1000 + workload number (batched run r: 4000 + r).
"""

from dataclasses import dataclass, field
from typing import Optional

import numpy as np

from .mesh import kuhn_cube_mesh, KuhnMesh


@dataclass
class Workload:
    name: str
    n: int
    p: int
    steps: int
    periodic: bool
    jitter: float
    seed: int
    init: str                        # "te110" | "pulse" | "plane"
    eps_range: Optional[tuple] = None  # None: eps = 1
    centre: Optional[np.ndarray] = None
    mesh: Optional[KuhnMesh] = None
    eps: Optional[np.ndarray] = None
    mu: Optional[np.ndarray] = None

    @property
    def h(self):
        return 1.0 / self.n

    @property
    def dt(self):
        return 0.2 * self.h / self.p ** 2

    @property
    def nt(self):
        return 6 * self.n ** 3


def _materials(w: Workload):
    nt = w.nt
    if w.eps_range is None:
        eps = np.ones(nt)
    else:
        rng = np.random.Generator(np.random.PCG64([w.seed, 1]))
        eps = rng.uniform(w.eps_range[0], w.eps_range[1], size=nt)
    return eps, np.ones(nt)


def make_workload(name, n=None, p=None, steps=None, shuffle_local=False):
    """Build a named workload; n, p, steps may be overridden for smaller cases."""
    table = {
        "cavity_n4_p3": dict(n=4, p=3, steps=100, periodic=False, jitter=0.0, seed=1001,
                             init="te110"),
        "pulse_n16_p4": dict(n=16, p=4, steps=1000, periodic=False, jitter=0.15, seed=1002,
                             init="pulse", eps_range=(1.0, 4.0)),
        "pulse_n32_p4": dict(n=32, p=4, steps=1000, periodic=False, jitter=0.15, seed=1002,
                             init="pulse", eps_range=(1.0, 4.0)),
        "planewave_n32_p6": dict(n=32, p=6, steps=2000, periodic=True, jitter=0.0, seed=1003,
                                 init="plane"),
        "adjoint_n16_p4": dict(n=16, p=4, steps=500, periodic=False, jitter=0.15, seed=1002,
                               init="pulse", eps_range=(1.0, 4.0)),
    }
    if name.startswith("batched_64:"):
        # run r of the batched workload: its own n, p, seed; jitter 0.1h, eps ~ U[1,4]
        n_r, p_r, seed_r = batched_runs(64)[int(name.split(":")[1])]
        kw = dict(n=n_r, p=p_r, steps=500, periodic=False, jitter=0.1, seed=seed_r, init="pulse",
                  eps_range=(1.0, 4.0))
    elif name not in table:
        raise KeyError(name)
    else:
        kw = dict(table[name])
    if n is not None:
        kw["n"] = n
    if p is not None:
        kw["p"] = p
    if steps is not None:
        kw["steps"] = steps
    w = Workload(name=name, **kw)
    w.mesh = kuhn_cube_mesh(w.n, jitter=w.jitter, seed=w.seed, periodic=w.periodic,
                            shuffle_local=shuffle_local)
    w.eps, w.mu = _materials(w)
    if w.init == "pulse":
        rng = np.random.Generator(np.random.PCG64([w.seed, 2]))
        w.centre = rng.uniform(0.3, 0.7, size=3)
    return w


def batched_runs(count=64):
    """Per-run (n, p, seed) of the batched workload: n in {8,12,16}, p in {2..6}."""
    runs = []
    for r in range(count):
        rng = np.random.Generator(np.random.PCG64(4000 + r))
        n = int(rng.choice([8, 12, 16]))
        p = int(rng.integers(2, 7))
        runs.append((n, p, 4000 + r))
    return runs
