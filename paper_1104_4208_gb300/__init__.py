"""GB300 (sm_103a) implementation of the energy-conserving DG time step for the
time-domain Maxwell equations (arXiv:1104.4208).

The computation lives in the C-ABI library libdgm.so (include/dgm.h); this
package holds its sources (csrc/), the in-tree build (build.py) and a thin
ctypes binding (_capi.py) plus a small convenience wrapper (solver.py).
"""

from . import build as _build  # noqa: F401


def load():
    """Import the binding (raises ImportError if libdgm.so is missing)."""
    from . import _capi
    return _capi
