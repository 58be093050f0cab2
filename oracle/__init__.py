"""CPU FP64 oracle for the explicit upwind-DG convection step.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import or call
this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It is a
plain, slow, readable restatement of what the paper defines, written in
numpy, and it shares no code, table or helper with the CUDA library.

What it computes (Lehrenfeld & Schoeberl, arXiv:1508.04245):

* ``dg.ConvectionOracle.apply``  -- (M^V)^{-1} C^V(u) w, the upwind DG
  trilinear form of Sec. 2.3 with the diagonal mass matrix of an
  L2-orthonormal element basis, evaluated in physical coordinates with
  exact quadrature and a brute-force (affine inversion) neighbour lookup;
* ``dg.rk_substeps`` -- explicit SSP Runge-Kutta integration of the
  propagation problem of Sec. 3.2.2, dv/ds = -(M^V)^{-1} C^V v;
* ``dg.transfer`` / ``dg.transfer_T`` -- the embedding I of Sec. 2.4
  (the L2 problem that defines it) and its transpose I^T;
* ``hdiv`` -- the H(div)-conforming BDM_k velocity space of Sec. 2.1.1
  (facet normal moments + Nedelec interior moments), the DOFs of analytic
  fields and the divergence-free winds built as curls of potentials;
* ``quad`` / ``hexa`` -- the same for parallelograms and parallelepipeds
  (uncurved quadrilaterals and hexahedra of Sec. 2: [Q^k]^d with tensor
  Legendre bases, the H(div) subspace of the Piola images);
* ``curved`` -- quadratic (curved) triangles (remark on curved elements in
  Sec. 2.4: dense mass blocks, I as the L2 projection).

Every function is pinned by ``tests/test_oracle_*.py`` against closed forms,
invariants the paper states (exact divergence, upwind stability, the
embedding W_h in V_h) or brute force on tiny meshes, never against itself.
"""
