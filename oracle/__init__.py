"""FP64 CPU oracle for the conservative adaptive-precision (AP) EAM+ACE potential.

TEST INFRASTRUCTURE ONLY. This package is a plain, slow, obviously correct
restatement of what the GPU library computes, written from the paper
(arxiv 2512.07693, "Conservative adaptive-precision interatomic potentials")
so that the CUDA path can be checked against it.  Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import it.  The product path (the C-ABI library and
its Python binding) never imports, calls or links anything here, and this
package imports nothing from the product path.

Everything is float64 numpy.  Each module cites the passage it follows:

  ftrans    -- transition function f_trans, Eq. S1 (also Eq. 2, Eq. S3)
  neighbors -- minimum-image pair search (O(N^2) brute force and a k-d tree)
  eam       -- EAM energy and lambda-weighted forces, Eq. B1, S7-S12
  csp       -- differentiable CSP^list with a pair list fixed at t=0, Eq. B3/S22
  switch    -- locally averaged descriptor and switch, Eq. 6/S2, S3
  ace       -- atomic cluster expansion (standard construction; the paper
               defines ACE only by reference, see the module docstring)
  apip      -- total energy Eq. 4 and force F = -grad E, Eq. 5 / S4-S29
  verlet    -- velocity-Verlet NVE integrator

Sign convention: ``lam`` is the ACE (precise) weight,
lam_i = 1 - f_trans(d_i, d_lo, d_hi); the paper's lambda (Eq. 2) is the
fast-model weight, lambda = 1 - lam.
"""
