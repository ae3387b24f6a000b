"""Plain, slow, FP64 CPU oracle for the k-th eigenvalue method of
Apriansyah & Yokota, "Computing the k-th Eigenvalue of Symmetric H^2-Matrices".

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it.  It shares no code with the CUDA path
(the two meet only at the seeded inputs of ``workloads``).

Modules
-------
dense : kernel matrices, Bunch-Kaufman LDL^T inertia, Sturm counts, Jacobi
        eigenvalues, Gershgorin bounds and the bisection of Algorithm 1.
h2    : the cluster tree, the block structure, the nested-basis H^2
        construction (Sec. 3.1) and the generalized H^2-LDL factorization with
        fill-in recompression (Sec. 3.2-3.4), counted by Sylvester's law (Sec. 4).
"""
