"""Plain, slow FP64 CPU oracle for SketchyCGAL (Yurtsever et al., arXiv 1912.02949).

TEST INFRASTRUCTURE ONLY.  This package restates the paper's method step by
step, in FP64 numpy, so that the CUDA library can be checked against it.  It
shares no code with the CUDA path and must never be imported by the product
path: only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
baseline leg (``cpu_baseline`` and ``--impl reference``) may use it.

Modules (each function cites the passage it follows):

* ``philox``      -- Philox4x32-10 counter-based generator + Box-Muller normals
                     (the random draws of Alg. 4.1 line "randn" and of the
                     Nystrom test matrix, Alg. 5.1).
* ``problems``    -- the black-box primitives of Eq. 2.3 for MaxCut (Section 2.4)
                     and coded-diffraction phase retrieval (Section 7.3, App. F.1),
                     plus the problem scaling of Eq. 7.1.
* ``lanczos``     -- ApproxMinEvec, Alg. 4.1 (storage-optimal) and Remark 4.2
                     (stored basis).
* ``nystrom``     -- NystromSketch, Alg. 5.1 / Alg. B.1, trace correction (App. B.4).
* ``sketchycgal`` -- SketchyCGAL, Alg. 6.1, with the dual step of Eq. 6.4, the
                     objective tracking of Section 6.2.2, the stopping rule
                     Eq. E.1 and the trace-bounded LMO of App. D.2; and the
                     general template of Alg. D.1 with inequality constraints
                     A(X) <= b (App. D.3), pinned by ``tests/test_oracle_general.py``.
* ``cgal_dense``  -- CGAL with an explicit matrix iterate, Alg. 3.1 (tiny n only).
* ``rounding``    -- MaxCut rounding (Section 7.2.1), brute-force max cut,
                     phase-retrieval rounding and error (Section 7.3.2-7.3.3).

Parity status of every function is pinned by ``tests/test_oracle_*.py``
against facts the paper and the mathematics fix; nothing here is marked
"parity unpinned".
"""
