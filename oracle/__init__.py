"""CPU FP64 oracle for the iterative Vecchia-Laplace hot path (test infrastructure).

This package is the reference that the CUDA path is checked against. It is plain,
slow and written to be read against the paper (Kuendig & Sigrist, "Iterative
Methods for Vecchia-Laplace Approximations for Latent Gaussian Process Models"):
numpy/scipy in float64, per-row loops where the paper defines a per-row
quantity, library primitives (dense solves, sparse LU, symmetric eigensolvers)
only as single steps.

It is test infrastructure only: the product library never imports, links or
runs anything here. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline legs of ``bench.py`` use it. It shares no code with the CUDA path;
both sides read their inputs from ``workloads`` and each implements the
Philox4x64-10 generator from its published definition.

Modules
-------
rng        Philox4x64-10, Rademacher probes, Box-Muller Gaussians
geometry   nearest-previous-neighbour sets (Section 2.1), test neighbours
           (Section 4.1), level schedules of the triangular factor
vecchia    covariance functions (Section 4.1) and the Vecchia factor B, D
           (Section 2.1)
krylov     preconditioned CG with the Lanczos tridiagonal (Appendix, "PCG
           algorithm"), explicit Lanczos with full reorthogonalisation,
           e1^T log(T) e1
laplace    likelihoods (Bernoulli-logit, Poisson-log; gamma-log with shape xi,
           Section 5), Newton mode (Eq. newton), L^VLA (Eq. VLA_loss) with the
           exact sparse-LU log-determinant, same-probe SLQ (Eqs. logdetsplit,
           def_SLQ) for the VADU and LVA preconditioners (Section 3.1.1),
           predictive means/variances (Eq. latentpostpredictive, Algorithm
           simAlgo)
lrac       pivoted Cholesky of Sigma and the LRAC preconditioner (Section
           3.1.2, Eqs. pcls2, logdetsplit2)
gradients  derivatives of L^VLA in (sigma2, rho), the offset F, the coefficients
           beta of F = X beta and the gamma shape xi: factor derivatives, the exact
           gradient with the implicit mode term, and the same-probe stochastic
           trace estimate with the control variate (Section 3, appendix)
lanczos_pred  predictive variances by preconditioned partial Lanczos with full
           reorthogonalisation (Section 4, preconditioners P_L1 and P_L2)
textbook   the dense GP Laplace approximation in the covariance
           parametrisation (Rasmussen & Williams 2006, Algorithms 3.1 and 3.2),
           used only to pin the Vecchia-Laplace oracle at m = n - 1
"""
