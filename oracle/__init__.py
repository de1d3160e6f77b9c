"""FP64 CPU oracle of the per-sub-grid hydro step (arXiv 2107.10987, Sec. III-B).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py``, never by the product package.  It shares
no code with the CUDA library; the two meet only through the seeded input
generators in ``paper_2107_10987_gb300.workloads``.

Contents
  * ``core``      ctypes binding of the C++ oracle (primitives, PPM line, point
                  flux, sub-grid step, RK3 update, operation counts)
  * ``mesh``      ghost fill of uniform sub-grid meshes (periodic / outflow) and
                  an RK3 driver on a whole box
  * ``analytic``  exact Riemann solver, Sedov-Taylor similarity constant
"""
from .core import OracleParams, lib, step, update, primitives, ppm_line, point_flux, count_ops, face_values, build  # noqa: F401
