"""Matrix-free augmented high-order compact (HOC) solver for clamped,
variable-coefficient biharmonic problems on B300 (sm_103a).

The compute path lives in the shared library built from ``csrc/`` and is
reached through :mod:`paper_2609_16478_b300.ahoc` (a thin ctypes binding over
the C ABI declared in ``include/ahoc.h``).  :mod:`paper_2609_16478_b300.inputs`
holds the seeded synthetic problem generators and nothing of the method.

Importing the package does not load the library; ``ahoc.lib()`` does, and it
raises if the library has not been built.
"""

__all__ = ["inputs", "ahoc"]
