"""CPU FP64 oracle for the gamblet multiresolution method (test infrastructure).

This package is test infrastructure only.  The CUDA library never calls it;
only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  It is a plain, slow, obviously-correct
restatement of the paper's definitions (NumPy / SciPy, float64), written to
be checked against the paper by eye:

* ``hierarchy`` - index tree, aggregation matrices pi and pibar, W
  (Sec. 4.1 Definition defindextree / Construction defmulires,
  Eq. (eq:eigdeiud3dd); Sec. 4.6 Lemma lemwk, Constructions const1/const2).
* ``exact``     - Algorithm 1 (exact gamblet transform / solve, Sec. 5.2)
  with the level-q initialisation psi^(q) = phi described there.
* ``local``     - Algorithm 2's localized setup (Sec. 5.3, Definition defb:
  patch solves on i^rho) and the one-pass localized solve.
* ``direct``    - direct sparse solve of A u = g (SuperLU) refined with
  extended-precision residuals.
* ``brute``     - Galerkin projections onto V^(k) = span{A^-1 pi_k^T}
  without the level recursion (Sec. 4.2 Theorem thmgugyug0), tiny grids.
* ``adjoint``   - gradient of J = 1/2 |u - u_obs|^2 with respect to the
  cell log-coefficients through a direct adjoint solve.
* ``local_adjoint`` - gradient of J through the one-pass localized map
  (reverse mode through Algorithm 2's solve and localized setup).
* ``massinit``  - the level-q initialisation by the mass matrix
  (Algorithm 1 lines 1-5, Algorithm 2 lines 2a-5 with Definition
  deflocinvm).
"""
