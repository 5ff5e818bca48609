"""Plain, slow, FP64 CPU oracle for the DQMC sweep of the half-filled Hubbard model.

TEST INFRASTRUCTURE ONLY. Nothing in the product path imports, calls or links this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use it. It shares no code with the CUDA library (no kernels, headers,
tables, constant generators, pre- or post-processing) and never imports it.

Module map (paper = arXiv 2106.00712, Supplemental Material Sec. I.2):

* ``philox``   -- Philox4x32-10 counter-based generator, written from its published
  definition (Salmon, Moraes, Dror, Shaw, SC'11). The paper fixes no generator.
* ``dqmc``     -- the model (Eq. 3), the Trotter split and discrete Hubbard-Stratonovich
  transform (SM Sec. I.2), the determinant weight and B matrices (SM Sec. I.2, last two
  equations), local Metropolis flips with determinant ratios, wraps, UDV stabilization and
  the equal-time estimators of E, double occupancy and S(pi,pi) (Eq. 4 definition of S(Q)).
* ``nimc``     -- network initialization (Algorithm 1 steps 2-3): the generator of SM Sec. II
  (3D transposed convolutions, sigmoid), the observable loss of Eq. 4 through the
  determinant weight and its gradient, Adam, Bernoulli discretization of generated fields.

Every algorithmic step the paper leaves open (acceptance rule, fast update, wrap, sweep
order, stabilization, measurement cadence) follows one stated reading; each function's
docstring names the passage it follows and the reading it takes.

Pins: see ``tests/test_oracle_*.py`` (U=0 closed form, Fock-space trace of the
Trotterized partition function and observables by full field enumeration, exact
diagonalization as dtau -> 0, determinant ratios against full determinants, wrapped and
fast-updated G against direct inversion, particle-hole invariants, Metropolis sampling
against the enumerated distribution, Philox against cuRAND's host generator).
"""
