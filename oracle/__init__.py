"""FP64 CPU oracle for the adaptive non-standard-form apply.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
restatement of Beylkin, Cheruvu and Perez, "Fast Adaptive Algorithms in the
Non-Standard Form for Multidimensional Problems", written in numpy/scipy FP64.
Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import it.  The CUDA library in
``paper_0706_0747_gb300`` never imports, links or calls anything here, and this
package imports nothing from it: the two share no code, tables or constants.

Modules, each following the paper step by step:

* ``basis``    -- Legendre scaling functions, Gauss-Legendre quadrature,
                  two-scale filters, cross-correlations (Appendix).
* ``gauss_sum``-- Gaussian-sum approximation of K_{mu,alpha} (Sec. 3,
                  eqs. IntegralRepr / KernelApproxByGaussians).
* ``operator`` -- 1-D blocks F^{j;m,l} (eq. KernelFactor), block norms
                  (eq. BlockNorms), the 18-term estimate
                  (eq. NormEstimateUsing1DBlocks) and per-scale term ranges
                  (Sec. 4, Core/Boundary subsets).
* ``tree``     -- adaptive and redundant trees (Sec. 2.2, Algorithm 1),
                  two-scale decomposition / reconstruction.
* ``apply``    -- Algorithm 3 (modified ns-form apply in d=3), the adaptive
                  projection of eq. g_assemble and the final truncation.

Parity status of every function is listed in its module header.
"""
