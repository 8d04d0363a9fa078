"""FP64 CPU oracle for the anharmonic lattice-dynamics hot path.

TEST INFRASTRUCTURE.  Only the tests, the smoke check of `__graft_entry__`
and the CPU-baseline leg of `bench.py` may import or run anything in this
package; the library (`paper_2009_01967_gb300`) never does, and this package
imports nothing from the library.  It shares only the seeded input generators
(`kald_inputs`) with the GPU path.

Each function follows one equation of arXiv:2009.01967 step by step in plain
NumPy/SciPy FP64 (modules `phonons`, `anharmonic`, `conductivity`), and is
pinned by the `-m "not gpu"` tests against closed forms, invariants and
brute-force sums that do not use it.

Parity unpinned: the absolute prefactor hbar*pi/8 of Eq. gamma_operators is
taken as printed (it agrees with the golden-rule self-energy); no number in
the paper fixes it for these inputs.
"""

from . import units, phonons, anharmonic, conductivity, ifc  # noqa: F401
