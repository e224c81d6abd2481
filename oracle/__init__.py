"""CPU FP64 oracle for the random-sampling multiscale solver -- TEST INFRASTRUCTURE.

This package is a plain, slow, obviously correct restatement of what the
method of K. Chen, Q. Li, J. Lu and S. J. Wright ("Random sampling and
efficient algorithms for multiscale PDEs", arXiv:1807.08848) computes,
written to check the CUDA library against.  It is not part of the product: only the test-suite, the smoke check and the CPU-baseline leg of the
benchmark may import it.  It shares no code with the CUDA library (the two
meet only in `synth`, which draws inputs and holds none of the method's
arithmetic).

Where the CUDA library iterates (PCG, CGLS, source iteration) the oracle uses
a direct solver, so each step yields its exact result up to rounding:

* `philox`   -- counter-based Philox4x32-10 generator + Box-Muller normals
                (the i.i.d. Gaussian boundary data of Sec. 3.3, Eq.
                rte_random and Eq. elliptic_random).
* `elliptic` -- Sec. 5: medium, 5-point operator, buffered local solves
                (Algorithm alg:summary, RanLocalSolu / DetLocalSolu), snapshot
                matrices, SVD basis with truncation (Sec. 3.2, Eq. svd),
                edge operators, the reduced least-squares system Eq.
                elliptic_cond_reduced (and its constrained variant), the
                overlapping restricted additive Schwarz variant of the online
                step on the reduced bases, and the reconstruction.
* `kinetic`  -- Sec. 4: discrete-ordinates slab transport, buffered local
                solves with random inflow (Eq. rte_random), reduced basis and
                the least-squares glue Eq. rte_cond_reduced.

Sections are numbered as in the paper (1 introduction ... 5 elliptic
example); equations are named by their labels in the paper's source.  Every
function names the passage it follows.  Where the paper is silent the
docstrings state the reading taken.
"""
