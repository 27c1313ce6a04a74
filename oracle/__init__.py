"""FP64 CPU oracle for the Daubechies-wavelet local Hamiltonian (periodic BC).

TEST INFRASTRUCTURE ONLY: plain, slow, obviously correct numpy code used to
check the CUDA library.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it; the library never does, and
the two share no code.

Modules:
* ``filters`` -- derivation of h, g (Eq. refinement), the magic filter
  (Eq. magicfilter) and the kinetic filter (Eqs. kiner, fprod) in 80-digit
  decimal arithmetic, rounded once to FP64.
* ``wavelet`` -- the operators of Sec. "Full local hamiltonian" and
  Sec. "Local density calculation" as plain periodic tap loops.

Parity status: every function here is pinned by tests in ``tests/`` against
closed forms, invariants, an independent cascade/Fourier construction of the
scaling function, or dense brute force; none is "parity unpinned".
"""
