"""FP64 CPU oracle for the rounded-polytope DEM (arXiv:1607.02427).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package; the product path (the
CUDA library and its binding) never does.  The arithmetic lives in
``dem_oracle.c`` (plain C, FP64); this module only packs arguments.

Parity status of each function (what pins it, see tests/test_oracle_*.py):
  forces()        pinned: WCA closed form, sphere limit, brute-force nearest
                  points, finite differences, Newton III / angular momentum,
                  invariance, face-to-face cube and corner-to-corner square
                  counts, zero energy beyond the cutoff.
  run()           pinned: free flight, principal-axis free rotor, time
                  reversibility, dt^2 scaling of the NVE energy error,
                  conserved NVT quantity and equipartition.
  primitives      pinned: dense brute-force sampling.
  set_parallel()  timed CPU baseline only: the same pairs and terms through a
                  cell list and OpenMP threads; pinned against the plain
                  evaluation (tests/test_oracle_parallel.py).
"""
from .oracle import (build, lib_path, pack_shapes, forces, run, point_segment,  # noqa: F401
                     point_face, segment_segment, wca, set_parallel, max_threads,
                     DEFAULT_PAR_EPS)
