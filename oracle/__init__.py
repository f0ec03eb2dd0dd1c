"""FP64 CPU oracle for the SWIFT multi-resolution SPH density/force path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` use it.  It shares no code with the
CUDA path; both take their inputs from ``paper_1309_3783_gb300.inputs``.

Modules
-------
``sph``           -- kernel, density, h iteration, ghost, force, reductions
                     (FP64, brute force or a k-d tree candidate search).
``decomposition`` -- the paper's hierarchical cell decomposition: top grid, cell
                     split rule, self/pair interaction lists with recursive
                     splitting (Section II-B), in plain Python for small inputs.
``sweep``         -- the paper's sorted cell-pair interaction (Section II-C,
                     Fig. 3) next to the naive double loop, in plain Python.
``riemann``       -- exact solution of the 1-D Riemann problem (the Sod shock
                     of Section III).
``sedov``         -- Sedov-Taylor similarity solution of a point explosion (the
                     Sedov blast of Section III).
"""
from . import sph, decomposition, sweep  # noqa: F401
