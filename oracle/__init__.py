"""Oracle: test infrastructure, not part of the library.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import, call, link or execute
anything in this package. It shares no code with the CUDA library and never
imports it.

* ``direct``   -- FP64 direct summation over hyperbolas (plain C, OpenMP),
  the discretisation of Eq. (3) the paper uses as its reference (Section 5).
* ``logpolar`` -- FP64 log-polar method in numpy, the paper's steps in order
  (Sections 2-4), the reference for the CUDA path on the same lattices.
* ``closed_forms`` -- exact values the two are pinned against.
"""
