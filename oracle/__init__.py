"""Plain FP64 CPU oracle for HMC on Bayesian multinomial (softmax) regression.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
this package.  The product path (the CUDA library and its Python binding)
never imports, links or calls anything here, and nothing here imports the
product.  The two sides share no code: the only common input is the seeded
data generator, which holds none of the method's arithmetic.

What it computes follows Beam, Ghosh & Doyle, "Fast Hamiltonian Monte Carlo
Using GPU Computing" (arXiv 1402.4089):

* ``model``  -- softmax (Eq. softmax, Sec. 2.1), log-likelihood (Eq. loglike),
  log-posterior kernel (Eq. logkernel / logkernelGPU) and its gradient
  (Eq. gradient / fullgrad, Appendix), with the identifiability constraint
  beta_K = 0 (Sec. 2.1) and two priors (standard-Cauchy of the paper,
  Gaussian of the benchmark workloads);
* ``hmc``    -- the leapfrog map (Eqs. hmc1-hmc3, Sec. 1.1), the Metropolis
  test with momentum (Eq. accept), L steps per proposal, and the annealed
  burn-in acceptance of Sec. 3.2;
* ``philox`` -- the counter-based generator (Philox4x64-10, Salmon et al.,
  SC'11) and Box-Muller normals used for momenta and accept uniforms;
* ``quant``  -- BF16 and per-column-scaled FP8 E4M3 storage formats of X;
* ``ess``    -- effective sample size (Geyer's initial monotone sequence) and
  Monte-Carlo standard errors.

Readings of the paper that this oracle takes (the paper is ambiguous, garbled
or inconsistent at these points):

* prior-gradient sign: the Appendix prints +2b/(1+b^2); the derivative of
  -log(1+b^2) is -2b/(1+b^2), which is what is used (the FD pin fixes it);
* kinetic energy: Eq. accept prints eta.eta; with unit-mass dynamics
  (theta += eps*eta) and eta ~ N(0, I) the Hamiltonian is -log K + eta.eta/2,
  which is used (the prior-only moment pin fixes it);
* "(p-1) x k" in the Appendix is read as the p x (K-1) free block.

Every function in this package has a pin in ``tests/test_oracle_*.py``
against something other than itself (finite differences, closed forms,
textbook special cases, invariants, a library routine, brute force).
"""
