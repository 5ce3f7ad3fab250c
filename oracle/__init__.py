"""FP64 CPU oracle for the BOSP linear-response eigensolver.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg may import this package.  It shares no code
with the CUDA path: no kernels, headers, helpers or constants; the only
shared module is the seeded input generator
``paper_2506_08355_gb300.synth`` (inputs only, no solver arithmetic).

Modules
  lrep_ref  the definition (dense SVD route), Alg. 1 (MGS-Biorth), the small
            LREP, CG, residuals and a literal Alg. 2 with batching/moving.
  philox    Philox4x32-10 counter-based generator and the Box-Muller normals
            the solver draws for its random start.

Parity status per function is stated in each docstring; every function
listed here is pinned by ``tests/test_oracle_pins.py``.
"""
