"""CPU oracle for the phaseless-AFQMC walker step (test infrastructure only).

Plain complex128 numpy restatement of the method, written to be read against
the paper (Sec. V, Eqs. (1) and (3), and the phaseless algorithm it cites:
Zhang & Krakauer 2003, Motta & Zhang 2018).  It is slow on purpose and shares
no code with the CUDA path.  Only the test suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it; the product path never
calls it and has no CPU fallback.

Modules:
  afqmc    -- Green's function, local energy, force bias, propagator, weights,
              QR re-orthonormalisation, the full step and the trajectory driver.
  adjoint  -- gradients of the local energy and log-overlap w.r.t. the trial
              orbitals and the Cholesky tensor.
  fock     -- brute-force Fock-space Hamiltonian, FCI and exact propagation on
              tiny systems (used only to pin the other modules).
  philox   -- Philox4x32-10 counter-based generator and Box-Muller fields.
  backprop -- the back-propagated one-body density matrix of a window of steps.
  msd      -- multi-determinant trial expansions (orthogonal or non-orthogonal).
  thc      -- tensor-hypercontraction Hamiltonians: their structured Cholesky form and
              the direct local energy.

Parity pins: every function here is checked in ``tests/test_oracle_*.py``
against closed forms, brute force or library routines; see the module
docstrings for which pin covers which function.
"""
