"""CPU oracle for FP64 emulation by split-integer arithmetic in LU / Cholesky.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously correct
CPU statement of what the GPU library computes.  Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import it.  The product path (the CUDA library and its
Python binding) never imports, links or executes anything here, and nothing
here imports the product path: the two share no code.  Seeded inputs come from
``paper_2509_23565_gb300.inputs`` which holds no arithmetic of the method.

Modules and the passages of arXiv 2509.23565 they follow:

* ``split``     -- per-row / per-column power-of-two scales and the signed
                   7-bit slices of each FP64 entry (Section 2, Eq. 1-4).
* ``emulgemm``  -- slice-pair level sums (exact integers) with the truncation
                   threshold t, exact recombination and the C update
                   (Section 2, Eq. 2; Section 4, Eq. 7).
* ``exact``     -- exact (rational) reference products used as pins.
* ``lu``        -- blocked right-looking LU with partial pivoting, getrs,
                   blocked Cholesky, potrs (Section 4, Eq. 5-7).
* ``residual``  -- scaled residual of Eq. 8 and the normwise backward error.
* ``bounds``    -- a-priori error bound of the emulated product.

Numbers are float64 and Python/numpy integers.  Library primitives used as a
single step: numpy float64 matmul applied to integer-valued matrices whose
partial sums stay below 2**53 (exact in any summation order), numpy float64
matmul for the plain FP64 trailing update, and scipy triangular solves.
Python's int/int true division and int->float conversion are correctly
rounded; they give the single rounding of the recombination.
"""
from . import split, emulgemm, exact, lu, residual, bounds  # noqa: F401
