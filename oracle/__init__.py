"""FP64 CPU oracle for the PonD two-population van der Waals step (arXiv:2002.09217).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this package.
The product path (``paper_2002_09217_gb300``) never imports it and shares no code
with it.

``oracle/pond_oracle.c`` holds the time step (plain C, FP64, no FMA contraction);
this module compiles it with gcc and wraps it with ctypes.  ``oracle/thermo.py``
holds closed-form thermodynamics of the vdW fluid (Maxwell construction,
Rankine-Hugoniot states, sound speed) used for initial conditions and pins.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
(closed forms, invariants, library routines, brute force).
"""
from .core import (Params, NPLANES, PL, build, lib_path, gauge_matrix, moment_matrix,
                   lagrange4, nonlocal_fields, init_state, stream_node, macro, collide,
                   step, step_nodes, moments, num_threads, weights, velocities)

__all__ = ["Params", "NPLANES", "PL", "build", "lib_path", "gauge_matrix", "moment_matrix",
           "lagrange4", "nonlocal_fields", "init_state", "stream_node", "macro", "collide",
           "step", "step_nodes", "moments", "num_threads", "weights", "velocities"]
