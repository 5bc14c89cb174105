"""CPU oracle for the localized model-order-reduction hot path (plain, slow, FP64).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package.  The CUDA library never calls
it and shares no code with it: it has its own subdomain construction, its own
assembly, sparse direct solves (SuperLU through SciPy) and dense LAPACK
factorisations (NumPy) in place of the GPU's iterative solves and batched kernels.

Modules
-------
rng        Philox-4x32-10 counter-based generator and FP32 Box-Muller normals
fem        P1 tetrahedral element matrices and sparse assembly (Sec. 2, Sec. 4)
subdomains overlapping subdomains, r-hop extensions, index sets I, B (Sec. 3, 7.1)
basis      per-subdomain optimal local basis, explicit and randomized (Sec. 4, Sec. 6)
reduced    stitching, projection Q^T A Q (explicit and interface-only), reduced solve
           (Eq. (11), Eq. (23), Sec. 6 step 3)
pipeline   the whole path on one mesh

Every function is pinned by ``tests/test_oracle_*.py`` against facts fixed by the
paper or by mathematics (closed forms, lemmas, brute force, published known-answer
vectors); none is marked "parity unpinned".
"""
