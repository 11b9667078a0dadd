"""Plain, slow FP64 CPU oracle for the batched astrochemistry hot path.

TEST INFRASTRUCTURE ONLY. Nothing on the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
(and ``bench.py --impl reference``) may use it. It shares no code with the CUDA
library; the one module both sides use is the seeded input generator
``paper_2511_10558_gb300.synth``, which holds no arithmetic of the method.

Contents:

* ``chem``    - rate coefficients (Sec. 2 Kooij-Arrhenius and cosmic-ray forms,
  App. B.1 photo form), the mass-action right-hand side (Sec. 2 ODE) built from
  the incidence matrix (Sec. 4), its analytic Jacobian, and the element/charge
  invariants.
* ``bdf``     - the variable-order (1-5), quasi-constant-step BDF integrator in
  backward-difference form (Sec. 1 names BDF as the field's integrator; the
  variant is Shampine & Reichelt 1997 with kappa = 0), dense LU with partial
  pivoting for the Newton systems.
* ``adjoint`` - the discrete adjoint of the oracle's own BDF steps.

Parity status: every function here is pinned by tests in ``tests/``
(closed forms, matrix exponentials, conservation, finite differences,
self-convergence, a library BDF). Full synthetic networks have no published
values: for them the pins are the invariants and self-convergence only.
"""
