"""Plain, slow FP64 CPU oracle for tensor-product B-spline smoothing.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU
baseline / reference arm of bench.py may import or run anything in this
package.  The product (the CUDA library and its Python binding) never calls it
and shares no code with it.

It follows Siebenborn & Wagner, "A Multigrid Preconditioner for Tensor Product
Spline Smoothing" (arXiv:1901.00654):

* spline.py -- knots, Cox-de Boor basis, cell index and sort key, the explicit
  sparse Phi, the 1-D Gram matrices, the penalty Lambda, the subdivision
  (prolongation) matrices, A_g and b (Sections 2.1, 2.2, 2.4, 3.2).
* mgcg.py -- the direct solve of (Phi'Phi + lambda Lambda) alpha = Phi'y and
  the multigrid-preconditioned CG of Algorithms 6-8 on assembled matrices.
* sampled.py -- operator outputs computed one coefficient at a time, and a
  chunked matrix-free apply, for full-size checks.

Parity unpinned: none of the functions here; every function is checked by the
pins in tests/test_oracle_pins.py (closed forms, invariants, brute force and
library cross-checks).  The paper's Table 2 iteration counts and Table 3
condition numbers depend on parameters the paper does not state and are
therefore not used as pins.
"""
