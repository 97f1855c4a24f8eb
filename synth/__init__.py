"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package only generates inputs: triangle meshes, incidence directions and
polarisations, random right-hand sides.  It holds none of the solver's
arithmetic (no basis functions, no Green's function, no tree, no series), so
that the CPU oracle and the CUDA path can both consume the same inputs while
sharing no code of the method.
"""

from .meshes import (icosphere, closed_cylinder, box_surface, plate, cube_tets, box_tets, ball_tets, shell_tets,  # noqa: F401
                     random_permittivity)
from .incidence import plane_wave_z, monostatic_sweep, random_incidences  # noqa: F401
