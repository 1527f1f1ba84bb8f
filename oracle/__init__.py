"""CPU oracle for tiled QR (thesis Chapter 3).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` may import anything under ``oracle/``.
The library (``paper_1303_3182_gb300``) never imports it, and it imports nothing from
the library; the two share only the seeded generators of ``synthetic``.

* ``elimlists``  - the elimination-list generators, the validity conditions, the tile
  task graph and its critical path (integer-exact).
* ``householder`` - unblocked FP64 Householder QR, the TT tile kernels and the TS
  kernels TSQRT/TSMQR applied one reflector at a time, the tiled algorithm (TT form,
  and the TS form of a list: TS kernels for the rows that never pivot in a column),
  apply-Q, back substitution, least squares.
* ``zhouseholder`` - the same in double complex (the thesis's second precision): LAPACK's
  complex reflector convention (real beta, H^H [alpha; x] = [beta; 0]), the complex tile
  kernels (TT and TS), the tiled algorithm, Q^H / Q, least squares.
* ``refine``     - FP64 least-squares checks (backward error, residual).
* ``schedule``   - bounded-processor scheduling of the task graph (thesis Chapter 5):
  Backflow priorities, the CP-method list schedule, the ALAP Derived bound.

Parity status: every function is pinned by ``tests/test_oracle_*.py`` (thesis tables,
closed forms, brute force against unblocked QR and LAPACK), except the ASAP critical
path of the 128 x 64 case, where the thesis prints 1748 and this oracle gives 1734
(parity unpinned for that one cell; GrASAP does not depend on it), and three cells of
the 5 x 5 schedule-length table (listed in tests/golden/schedule_5x5.txt).
"""
