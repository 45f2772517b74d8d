"""Plain FP64 CPU oracle for the smoothed-circulant-embedding MLMC hot path.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import anything from this package.  The
product (the CUDA library and its Python binding) never imports, links or runs
it, and this package imports nothing from the product: the two share no code.

Every function is a slow, direct statement of what the paper (Istratuca &
Teckentrup, "Smoothed Circulant Embedding with Applications to Multilevel Monte
Carlo Methods for PDEs with Random Coefficients") defines, citing the section,
equation or algorithm it follows.  Library primitives (matrix products, a sort,
numpy's FFT, scipy's sparse direct solver and Bessel function) are used as
single steps; nothing is blocked, fused or reordered.

Modules
  rng         Philox4x32-10 counter generator and the Box-Muller normal spec
  covariance  Matern / separable-exponential covariances, smooth periodisation
  embedding   first column, eigenvalues (naive DFT), PSD check and padding,
              smoothing masks (Algorithm 2 step 4(b))
  field       Algorithm 1 step 4(a)-(f): xi -> w -> v = F w -> u -> Z -> k
  qmc         randomly shifted rank-1 lattice normals (the MLQMC sampler)
  darcy       P1 finite elements with nodal quadrature, direct solve, QoIs
  field3d     the d = 3 embedding (C_ext over Z^3, threefold DFT) and field
  darcy3d     the d = 3 Darcy problem on Kuhn tetrahedra, direct solve, QoIs
  mlmc        level differences, level sums, MLMC estimator and N_l rule

Parity status: every function is pinned by a test in tests/test_oracle_*.py.
The tau-selection rules of §3.6 (``mlmc.tau_exponential``, ``mlmc.tau_matern``)
take the ratio C_s / C_alpha as an input, because the paper does not give it;
for every value of it they are pinned against the error bounds they balance
and against each other (tests/test_oracle_tau.py).
"""
