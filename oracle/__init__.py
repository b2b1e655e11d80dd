"""Plain, slow FP64 CPU oracle of the multilevel PUM solver (test infrastructure).

This package is test infrastructure only.  It is imported by the tests, by
``__graft_entry__.smoke()`` and by the CPU-baseline leg of ``bench.py``; the
CUDA library never imports, links or calls it, and it shares no code with the
library.  Every function follows one passage of the paper (section, equation,
algorithm or definition cited in its docstring) and uses NumPy/SciPy only for
library primitives (dense solves, Cholesky, sparse matrix products, Gauss
points), so that it can be checked against the paper by eye.

Modules:
    pum     Section 4 / Example 5.1 / Example 5.4: cover, partition of unity,
            local Legendre spaces, Nitsche forms, load vector, mass matrix,
            L2-projection prolongation and Galerkin coarse operators.
    pum3d   Example 5.3: the same construction on the unit cube for the biharmonic
            equation (Nitsche face terms, projection, prolongation, hierarchy).
    pum_raise  Example 5.1's space with the degree raised on boundary patches
            (variable local dimension; assembly, projection, prolongation).
    learned Candidate pools, features, labels and the scoring network of the
            learned adaptive pattern (not a method of the paper; Algorithm 1 is its
            teacher and judge).
    blocks  Definition 2.1: block-sparse matrices and their patterns.
    fsai    Definition 2.2, Lemma 2.7, Algorithm 1 and Section 2.2: block-FSAI
            (static, adaptive, nested) and the Kaporin-type measure.
    cheb    Algorithm 3 (fourth-kind Chebyshev smoothing), Eq. (3.6) closed form,
            and the Lanczos estimate of lambda_max (Section 5 set-up).
    solver  V(k,k)-cycle with Galerkin hierarchy, preconditioned CG and the
            convergence factors of Example 5.1.
    rng     SplitMix64 counter generator (Lanczos start vectors).
"""
