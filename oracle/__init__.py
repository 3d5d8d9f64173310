"""CPU oracle for the Cholesky-decomposed relativistic LR-CCSD response path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package: only
``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may use it.  It shares no code with the CUDA library.

Plain, slow and obviously correct: complex128 PyTorch CPU tensors, explicit
antisymmetrised integral tensors <pq||rs>, library einsum/solve as the only
primitives.  Modules:

* ``integrals``  -- <pq|rs> from Cholesky vectors, Fock/one-body split, pivoted
                    Cholesky of the ERI supermatrix (Sec. 3).
* ``ccsd``       -- spin-orbital CCSD energy and residual Omega(T) (Sec. 2.2 amplitude
                    equations), first-order amplitudes, packing of unique amplitudes.
* ``secondq``    -- brute-force second quantisation on determinant bit strings:
                    e^{-T} H e^{T} projected (Sec. 2.2), FCI, sum over states (Eq. sos).
* ``jacobian``   -- sigma = A X: the polynomial-exact stencil of Omega (definition of
                    the Jacobian, Sec. 2.2) and the connected H-bar X term list in the
                    T1-dressed Cholesky form; transpose product via autograd.
* ``response``   -- xi, eta, Lambda, F X, the linear solves and alpha(omega) (Sec. 2.2,
                    response function with P(A,B) symmetrisation).

Every function cites the passage it follows.  Pins live in ``tests/test_oracle_*.py``.
"""
