"""CPU oracle for the augmented HOC biharmonic method: TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its binding) never imports, calls or links it, and this package shares no code
with the product path: the only common module is the seeded input generator
``paper_2609_16478_b300.inputs``, which holds none of the method's arithmetic.

What the oracle computes is the plain definition of the discrete method:
  * ``stencils``   -- the compact fourth-order operators L_h and M and the
                      one-sided second normal derivative (Sec. 2.2);
  * ``coupled``    -- the coupled block system of Sec. 2.2 (U, V and the
                      augmented boundary unknowns Q) assembled as a sparse
                      FP64 matrix and solved directly by SuperLU; the Schur
                      complement S_h = A22 - A21 A11^-1 A12 and its right-hand
                      side from the assembled blocks (Sec. 2.3, Lemma 1);
  * ``residual``   -- the same equations applied to given grid functions by
                      array slicing (a residual certificate for grids too
                      large for a direct solve);
  * ``dst``        -- the DST-I by its defining sum.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
(closed forms, polynomial exactness, the paper's printed cavity and plate
values, convergence order, Lemma 1); none is "parity unpinned".
"""
