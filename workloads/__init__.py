"""Seeded synthetic inputs for the DG Maxwell hot path.

This package holds only input data: tetrahedral meshes (Kuhn subdivision of a
cube, optional vertex jitter, optional periodic identification), per-element
material draws, analytic fields evaluated at points, and random source /
observation positions.  It contains none of the discretisation's arithmetic
(no basis, no quadrature, no operator), so both the CUDA path and the FP64
oracle can draw their inputs from it without sharing any method code.

All randomness uses NumPy's PCG64 with an explicit seed.
"""

from .mesh import KuhnMesh, kuhn_cube_mesh, workload_mesh
from .fields import (te110_fields, gaussian_pulse_fields, plane_wave_fields,
                     dipole_waveform, random_points)

__all__ = ["KuhnMesh", "kuhn_cube_mesh", "workload_mesh", "te110_fields",
           "gaussian_pulse_fields", "plane_wave_fields", "dipole_waveform",
           "random_points"]
