"""Plain CPU FP64 oracle for the Fast-QMMD / SP2 hot path.

TEST INFRASTRUCTURE ONLY.  This package is the slow, obviously correct
reference that the CUDA path is checked against.  Only the tests, the smoke
check and the benchmark's CPU-baseline leg may import it; the product path
(the CUDA library and its Python binding) never does, and it shares no code
with it: the only common module is `workloads`, which generates inputs and
holds none of the method's arithmetic.

Modules
  tb          orthogonal SCC tight-binding model: cut-off tail, Slater-Koster
              hopping blocks, gamma, h(R), H[n] and their derivatives (App. D)
  density     density matrices by diagonalisation (T_e = 0 step function and
              Fermi-Dirac, Eq. EL_4c / Eq. DM_perp), the SP2 recursion and its
              thresholded block-sparse form (Sec. III.B), entropy (Eq. Entropy)
  observables Mulliken charges, energy and forces (Eq. EL_Orth_a/c,
              Eq. Etot_Orth, with the reading stated there)
  md          SCF initialisation, velocity Verlet, the modified Verlet scheme
              for n (Eq. Verl_n), XL-BOMD and BOMD drivers

Parity pins: every function is checked in tests/test_oracle_*.py against
closed forms, invariants, finite differences or textbook special cases.
Functions without such a pin say "parity unpinned" in their docstring.
"""
